"""The host set-up of the scalar potential (Alg. 1, Sec. 2.1) in the library
(slp_debug_fem_assemble: the same code slp_potential_create runs before it
touches the device) against the FP64 oracle (oracle/fem.py): node classes,
outward boundary faces with normals, 1/h and the fourth node, the free-node
stiffness matrix and the load operator.  CPU only."""
import numpy as np
import pytest

from oracle import fem
from synthetic import meshes

R = 0.2


@pytest.fixture(scope="module")
def slp():
    import paper_1305_3162_gb300 as m
    from paper_1305_3162_gb300 import _build
    _build.build()
    m.load()
    return m


def _renumbered_ball():
    """The n = 4 ball with its nodes renumbered at random and every other
    tetrahedron given the opposite orientation."""
    X, K = meshes.ball_tets(4, R)
    rng = np.random.default_rng(11)
    perm = rng.permutation(X.shape[0])
    inv = np.empty_like(perm)
    inv[perm] = np.arange(perm.size)
    K = inv[K].astype(np.int32)
    K[::2, [2, 3]] = K[::2, [3, 2]]
    return X[perm], K


MESHES = {
    "ball_n4": lambda: meshes.ball_tets(4, R),
    "shell_n4": lambda: meshes.shell_tets(4, 0.1, R),
    "slab_3x3x2": lambda: meshes.cube_tets(3, 0.4, 2),
    "ball_renumbered_mixed_orientation": _renumbered_ball,
}


@pytest.mark.parametrize("name", list(MESHES))
def test_host_assembly_equals_the_oracle(slp, name):
    X, K = MESHES[name]()
    a = slp.slp_debug_fem_assemble(X, K)
    faces, owner, opp = fem.boundary_faces(X, K)
    bnd = np.zeros(X.shape[0], dtype=bool)
    bnd[faces.ravel()] = True
    free = np.nonzero(~bnd)[0]
    bnodes = np.nonzero(bnd)[0]

    # node classes, each numbered in ascending node order
    slot = a["node_slot"]
    assert a["n_free"] == free.size and a["n_boundary"] == bnodes.size
    assert np.array_equal(slot[free], np.arange(free.size))
    assert np.array_equal(slot[bnodes], -1 - np.arange(bnodes.size))

    # faces: the same triangles, wound the same way (outward), the same
    # unit normal, 1/h = |S| / (3 |T|) of the owning tetrahedron, and the
    # owner's fourth node as a free index (or -1)
    F = a["faces"]
    assert F.shape[0] == faces.shape[0]
    key = {tuple(sorted(f)): i for i, f in enumerate(faces.tolist())}
    vol, _ = fem.p1_gradients(X, K)
    for j in range(F.shape[0]):
        i = key[tuple(sorted(F[j, :3].tolist()))]
        p, q, r = X[F[j, 0]], X[F[j, 1]], X[F[j, 2]]
        n = np.cross(q - p, r - p)
        po, qo, ro = X[faces[i, 0]], X[faces[i, 1]], X[faces[i, 2]]
        no = np.cross(qo - po, ro - po)
        area2 = np.linalg.norm(no)
        assert n @ no > 0
        assert np.allclose(a["face_geom"][j, :3], no / area2, rtol=0, atol=1e-14)
        assert a["face_geom"][j, 3] == pytest.approx(0.5 * area2 / (3.0 * vol[owner[i]]), rel=1e-12)
        assert F[j, 3] == (-1 if bnd[opp[i]] else slot[opp[i]])

    # S(free, free), rows in CSR with ascending columns
    nf = free.size
    ptr, col, val = a["s_ptr"], a["s_col"], a["s_val"]
    assert ptr[0] == 0 and ptr[-1] == col.size and np.all(np.diff(ptr) >= 1)
    for r in range(nf):
        assert np.all(np.diff(col[ptr[r]:ptr[r + 1]]) > 0)
    Sg = np.zeros((nf, nf))
    rows = np.repeat(np.arange(nf), np.diff(ptr))
    Sg[rows, col] = val
    So = fem.stiffness(X, K).toarray()[np.ix_(free, free)]
    assert np.abs(Sg - So).max() <= 1e-13 * np.abs(So).max()

    # the load operator: b(free) for smooth and rough nodal fields
    bp, bc, bv = a["b_ptr"], a["b_col"], a["b_val"]
    brows = np.repeat(np.arange(nf), np.diff(bp))
    assert np.all(bc != free[brows])  # the row's own node is left out
    rng = np.random.default_rng(3)
    for m in (X / np.linalg.norm(X, axis=1).max(), rng.standard_normal(X.shape)):
        bg = np.zeros(nf)
        np.add.at(bg, brows, np.einsum("ed,ed->e", bv, m[bc] - m[free[brows]]))
        bo = fem.load(X, K, m)[free]
        assert np.abs(bg - bo).max() <= 1e-12 * max(np.abs(bo).max(), 1e-300)


def test_host_assembly_refuses_bad_meshes(slp):
    X, K = meshes.ball_tets(4, R)
    with pytest.raises(slp.SlpError) as e:
        slp.slp_debug_fem_assemble(X, np.vstack([K, K[:1]]))  # a face in three tetrahedra
    assert e.value.status == slp.SLP_ERR_MESH
    bad = K.copy()
    bad[0, 3] = X.shape[0]
    with pytest.raises(slp.SlpError) as e:
        slp.slp_debug_fem_assemble(X, bad)
    assert e.value.status == slp.SLP_ERR_MESH
    flat = K.copy()
    flat[0, 3] = flat[0, 2]
    with pytest.raises(slp.SlpError) as e:
        slp.slp_debug_fem_assemble(X, flat)  # degenerate tetrahedron
    assert e.value.status == slp.SLP_ERR_MESH
