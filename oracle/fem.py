"""FP64 CPU oracle for the scalar potential of Alg. 1 (phi = phi_1 + phi_2).

TEST INFRASTRUCTURE ONLY, like the rest of this package: the test suite,
``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may use it; the
library shares no code with it.

The split of Sec. 2.1, written out step by step on a P1 tetrahedral mesh:

* phi_1: the Dirichlet problem  -Lap phi_1 = -div m  in the body, phi_1 = 0 on
  its boundary, in the weak form of Sec. 2.1 (find phi_1 in H_0^1 with
  int grad phi_1 . grad v = int m . grad v for every v in H_0^1); P1
  elements, the stiffness matrix a_km = sum_T int_T grad eta_m . grad eta_k
  and the load b_k = sum_T int_T m . grad eta_k with m the P1 interpolant of
  the nodal values; only the free (non-boundary) rows and columns are solved
  (the subsystem of Sec. 2.1 with zero Dirichlet data), here by a sparse
  direct solve (scipy's SuperLU), where the paper uses ILU-preconditioned CG;
  for meshes too large for the direct solve, scipy's conjugate gradients
  with a Jacobi preconditioner to a relative residual of 1e-13
  (``phi1_iterative``, pinned to the direct solve).
* g: on every boundary triangle S_j the integral mean of m . n_j (the L2
  projection of Sec. 2.2) minus the normal derivative of phi_1 from the
  tetrahedron that owns the triangle (grad phi_1 is constant there).
* phi_2: the single layer potential of g, element-wise constant, integrated
  exactly over every boundary triangle (``oracle.slp_p0``), at every node.

Pinned by tests/test_oracle_fem_pins.py: the closed forms of Sec. 4 (uniform
magnetisation: phi_1 = 0 and phi = m . x / 3; the hedgehog m = x/|x|:
phi = |x| - R), converging under refinement, and the P1 mass and stiffness
forms on polynomials they integrate exactly.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import slp_p0


def boundary_faces(nodes, tets):
    """Faces that belong to one tetrahedron only, wound so that their normal
    points away from the tetrahedron's fourth vertex (outward).  Returns
    (faces [F][3], owner tet [F], opposite vertex [F])."""
    tets = np.asarray(tets, dtype=np.int64)
    local = [(1, 2, 3, 0), (0, 2, 3, 1), (0, 1, 3, 2), (0, 1, 2, 3)]
    faces, owner, opp = [], [], []
    for a, b, c, o in local:
        faces.append(tets[:, [a, b, c]])
        owner.append(np.arange(tets.shape[0]))
        opp.append(tets[:, o])
    faces = np.concatenate(faces)
    owner = np.concatenate(owner)
    opp = np.concatenate(opp)
    key = np.sort(faces, axis=1)
    _, inv, cnt = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    if cnt.max() > 2:
        raise ValueError("a face is shared by more than two tetrahedra")
    once = cnt[inv.ravel()] == 1
    faces, owner, opp = faces[once], owner[once], opp[once]
    x = nodes
    nrm = np.cross(x[faces[:, 1]] - x[faces[:, 0]], x[faces[:, 2]] - x[faces[:, 0]])
    inward = np.einsum("ij,ij->i", nrm, x[opp] - x[faces[:, 0]]) > 0
    faces[inward] = faces[inward][:, [0, 2, 1]]
    return faces, owner, opp


def p1_gradients(nodes, tets):
    """Volumes |T| and the constant gradients of the four barycentric
    (hat) functions on each tetrahedron: grad eta_a = rows of J^-T."""
    x = nodes[np.asarray(tets, dtype=np.int64)]
    J = np.stack([x[:, 1] - x[:, 0], x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]], axis=2)  # columns = edges
    vol = np.abs(np.linalg.det(J)) / 6.0
    Jinv = np.linalg.inv(J)  # rows of J^-1 are grad eta_1..3
    G = np.empty((x.shape[0], 4, 3))
    G[:, 1:, :] = Jinv
    G[:, 0, :] = -Jinv.sum(axis=1)
    return vol, G


def stiffness(nodes, tets):
    """a_km = sum_T |T| grad eta_m . grad eta_k (Sec. 2.1), N x N CSR."""
    vol, G = p1_gradients(nodes, tets)
    K = np.einsum("t,tad,tbd->tab", vol, G, G)
    t = np.asarray(tets, dtype=np.int64)
    rows = np.repeat(t, 4, axis=1).ravel()
    cols = np.tile(t, (1, 4)).ravel()
    n = nodes.shape[0]
    return sp.csr_matrix((K.ravel(), (rows, cols)), shape=(n, n))


def mass(nodes, tets):
    """P1 mass matrix, int_T eta_a eta_b = |T| (1 + delta_ab) / 20."""
    vol, _ = p1_gradients(nodes, tets)
    loc = (np.ones((4, 4)) + np.eye(4)) / 20.0
    K = vol[:, None, None] * loc[None]
    t = np.asarray(tets, dtype=np.int64)
    rows = np.repeat(t, 4, axis=1).ravel()
    cols = np.tile(t, (1, 4)).ravel()
    n = nodes.shape[0]
    return sp.csr_matrix((K.ravel(), (rows, cols)), shape=(n, n))


def load(nodes, tets, m):
    """b_k = sum_T int_T m . grad eta_k, m the P1 interpolant: its mean over
    T is the mean of the four nodal values."""
    vol, G = p1_gradients(nodes, tets)
    t = np.asarray(tets, dtype=np.int64)
    mbar = m[t].mean(axis=1)
    contrib = vol[:, None] * np.einsum("tad,td->ta", G, mbar)
    b = np.zeros(nodes.shape[0])
    np.add.at(b, t.ravel(), contrib.ravel())
    return b


def phi1(nodes, tets, m):
    """The Dirichlet solve of Sec. 2.1: phi_1 = 0 at boundary nodes, the
    free subsystem S(fn, fn) x = b(fn) solved directly."""
    faces, _, _ = boundary_faces(nodes, tets)
    bnd = np.zeros(nodes.shape[0], dtype=bool)
    bnd[faces.ravel()] = True
    free = np.nonzero(~bnd)[0]
    S = stiffness(nodes, tets)
    b = load(nodes, tets, np.asarray(m, dtype=np.float64))
    out = np.zeros(nodes.shape[0])
    if free.size:
        out[free] = spla.spsolve(S[free][:, free].tocsc(), b[free])
    return out


def phi1_iterative(nodes, tets, m, rtol: float = 1e-13):
    """phi_1 as in ``phi1``, the free subsystem solved by scipy's conjugate
    gradients (Jacobi preconditioner) to |r| <= rtol |b|."""
    faces, _, _ = boundary_faces(nodes, tets)
    bnd = np.zeros(nodes.shape[0], dtype=bool)
    bnd[faces.ravel()] = True
    free = np.nonzero(~bnd)[0]
    S = stiffness(nodes, tets)[free][:, free].tocsr()
    b = load(nodes, tets, np.asarray(m, dtype=np.float64))[free]
    out = np.zeros(nodes.shape[0])
    if free.size:
        dinv = 1.0 / S.diagonal()
        M = spla.LinearOperator(S.shape, matvec=lambda v: dinv * v)
        try:
            x, info = spla.cg(S, b, rtol=rtol, atol=0.0, maxiter=100000, M=M)
        except TypeError:  # scipy before 1.12 names it tol
            x, info = spla.cg(S, b, tol=rtol, atol=0.0, maxiter=100000, M=M)
        if info != 0:
            raise RuntimeError(f"conjugate gradients did not converge ({info})")
        out[free] = x
    return out


def potential_at(nodes, tets, m, sel, phi_1=None, nthreads: int = 0):
    """phi = phi_1 + phi_2 at the nodes sel only (phi_1 everywhere, by the
    iterative solve unless given): for meshes whose all-node sum is too long.
    Returns (phi[sel], phi_1)."""
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    m = np.ascontiguousarray(m, dtype=np.float64)
    p1 = phi1_iterative(nodes, tets, m) if phi_1 is None else phi_1
    faces, g = charges(nodes, tets, m, p1)
    used = np.unique(faces.ravel())
    ren = -np.ones(nodes.shape[0], dtype=np.int64)
    ren[used] = np.arange(used.size)
    p2 = slp_p0(nodes[used], ren[faces].astype(np.int32), g, nthreads=nthreads, x=nodes[sel])
    return p1[sel] + p2, p1


def charges(nodes, tets, m, phi_1):
    """g_j on every boundary triangle: mean of m . n_j minus d phi_1 / dn
    from the owning tetrahedron (Sec. 2.1, Sec. 2.2).  Returns (faces, g)."""
    faces, owner, _ = boundary_faces(nodes, tets)
    x = nodes
    nrm = np.cross(x[faces[:, 1]] - x[faces[:, 0]], x[faces[:, 2]] - x[faces[:, 0]])
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    mbar = np.asarray(m, dtype=np.float64)[faces].mean(axis=1)
    _, G = p1_gradients(nodes, tets[owner])
    grad = np.einsum("tad,ta->td", G, phi_1[np.asarray(tets, dtype=np.int64)[owner]])
    g = np.einsum("ij,ij->i", mbar, nrm) - np.einsum("ij,ij->i", grad, nrm)
    return faces, g


def potential(nodes, tets, m, nthreads: int = 0):
    """phi = phi_1 + phi_2 at every node (Alg. 1).  Returns (phi, phi_1, g)."""
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    m = np.ascontiguousarray(m, dtype=np.float64)
    p1 = phi1(nodes, tets, m)
    faces, g = charges(nodes, tets, m, p1)
    # the boundary surface as its own mesh: boundary nodes renumbered
    used = np.unique(faces.ravel())
    ren = -np.ones(nodes.shape[0], dtype=np.int64)
    ren[used] = np.arange(used.size)
    p2 = slp_p0(nodes[used], ren[faces].astype(np.int32), g, nthreads=nthreads, x=nodes)
    return p1 + p2, p1, g


def p1_errors(nodes, tets, e):
    """L2 norm and H1 seminorm of the P1 function with nodal values e (the
    error of nodal interpolations, as in Sec. 4): sqrt(e^T M e), sqrt(e^T S e)."""
    M = mass(nodes, tets)
    S = stiffness(nodes, tets)
    return float(np.sqrt(max(e @ (M @ e), 0.0))), float(np.sqrt(max(e @ (S @ e), 0.0)))
