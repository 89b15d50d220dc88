"""Seeded synthetic surface meshes shaped like the paper's test bodies.

These generators produce geometry only (vertex coordinates and outward-wound
triangles).  They contain none of the single-layer-potential arithmetic and
are shared, as plain inputs, by the FP64 oracle and by the CUDA path.

Shapes (Sec. 4 of the paper uses a cube, a sphere and a thin film):
  * ``box``       axis-aligned cuboid, each face a structured grid of squares,
                  every square split into two triangles;
  * ``cube``      the unit cube as a ``box``;
  * ``icosphere`` an icosahedron subdivided ``level`` times, vertices
                  projected onto the sphere;
  * ``torus``     a parametric torus with major radius R and minor radius r;
  * ``ball_tets`` a tetrahedral volume mesh of a ball (the finite element
                  mesh of the paper's sphere tests, Sec. 2.1 and Sec. 4);
  * ``cube_tets`` a tetrahedral volume mesh of a cube (six tetrahedra per
                  cell of a structured grid);
  * ``shell_tets`` a tetrahedral mesh of a spherical shell (two boundary
                  spheres: the outer one and the surface of the cavity).

All surface meshes are closed, 2-manifold and oriented with outward normals
(counter-clockwise winding seen from outside); volume meshes list each
tetrahedron with positive orientation.
"""
from __future__ import annotations

import numpy as np


def box(lx: float, ly: float, lz: float, nx: int, ny: int, nz: int,
        center=(0.0, 0.0, 0.0)):
    """Surface of the cuboid [-lx/2, lx/2] x [-ly/2, ly/2] x [-lz/2, lz/2].

    Face grids have nx x ny squares on the two z faces, nx x nz on the two y
    faces and ny x nz on the two x faces.  Returns (V[float64 n,3],
    T[int32 m,3]) with 2*2*(nx*ny + ny*nz + nx*nz) triangles and
    2*(nx*ny + ny*nz + nx*nz) + 2 vertices.
    """
    n = (nx, ny, nz)
    ext = (lx, ly, lz)
    idx = -np.ones((nx + 1, ny + 1, nz + 1), dtype=np.int64)
    # mark lattice points on the boundary
    I, J, K = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    onb = (I == 0) | (I == nx) | (J == 0) | (J == ny) | (K == 0) | (K == nz)
    idx[onb] = np.arange(int(onb.sum()))
    pts = np.stack([I[onb], J[onb], K[onb]], axis=1).astype(np.float64)
    V = np.empty_like(pts)
    for q in range(3):
        V[:, q] = pts[:, q] / n[q] * ext[q] - 0.5 * ext[q] + center[q]

    tris = []
    # For each face: the two in-face axes (a, b) ordered so that a x b points outward.
    for axis in range(3):
        for side in (0, 1):
            a, b = [(1, 2), (2, 0), (0, 1)][axis]
            if side == 0:
                a, b = b, a  # flip orientation on the low face
            na, nb = n[a], n[b]
            ia, ib = np.meshgrid(np.arange(na), np.arange(nb), indexing="ij")
            ia = ia.ravel()
            ib = ib.ravel()

            def lat(da, db):
                c = [None, None, None]
                c[axis] = np.full(ia.shape, side * n[axis])
                c[a] = ia + da
                c[b] = ib + db
                return idx[c[0], c[1], c[2]]

            p00, p10, p11, p01 = lat(0, 0), lat(1, 0), lat(1, 1), lat(0, 1)
            tris.append(np.stack([p00, p10, p11], axis=1))
            tris.append(np.stack([p00, p11, p01], axis=1))
    T = np.concatenate(tris, axis=0).astype(np.int32)
    return V, T


def cube(nper: int, side: float = 1.0):
    """Cube of edge ``side`` centred at the origin, nper x nper squares per face."""
    return box(side, side, side, nper, nper, nper)


_ICO_FACES = np.array([
    [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
    [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
    [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
    [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)


def icosphere(level: int, radius: float = 1.0):
    """Icosahedron refined ``level`` times by edge bisection, projected to the sphere.

    Level L has 20*4**L triangles and 10*4**L + 2 vertices.
    """
    t = (1.0 + 5.0 ** 0.5) / 2.0
    V = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
                  [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                  [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    F = _ICO_FACES.copy()
    for _ in range(level):
        nv = V.shape[0]
        e = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]], axis=0)
        e.sort(axis=1)
        key = e[:, 0] * (nv + 1) + e[:, 1]
        uniq, inv = np.unique(key, return_inverse=True)
        a = uniq // (nv + 1)
        b = uniq % (nv + 1)
        mid = V[a] + V[b]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        V = np.concatenate([V, mid], axis=0)
        m = F.shape[0]
        ab = nv + inv[:m]
        bc = nv + inv[m:2 * m]
        ca = nv + inv[2 * m:]
        F = np.concatenate([
            np.stack([F[:, 0], ab, ca], 1),
            np.stack([F[:, 1], bc, ab], 1),
            np.stack([F[:, 2], ca, bc], 1),
            np.stack([ab, bc, ca], 1)], axis=0)
    return V * radius, F.astype(np.int32)


def torus(R: float, r: float, nu: int, nv: int):
    """Torus around the z axis: nu segments along the tube, nv around it."""
    u = 2 * np.pi * np.arange(nu) / nu
    v = 2 * np.pi * np.arange(nv) / nv
    U, W = np.meshgrid(u, v, indexing="ij")
    x = (R + r * np.cos(W)) * np.cos(U)
    y = (R + r * np.cos(W)) * np.sin(U)
    z = r * np.sin(W)
    V = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    i, j = np.meshgrid(np.arange(nu), np.arange(nv), indexing="ij")
    i = i.ravel()
    j = j.ravel()
    p00 = i * nv + j
    p10 = ((i + 1) % nu) * nv + j
    p11 = ((i + 1) % nu) * nv + (j + 1) % nv
    p01 = i * nv + (j + 1) % nv
    T = np.concatenate([np.stack([p00, p10, p11], 1), np.stack([p00, p11, p01], 1)], axis=0)
    return V, T.astype(np.int32)


def mesh_stats(V, T):
    """Vertex/triangle counts and the outward signed volume (positive when outward)."""
    P = V[T]
    vol = np.einsum("ij,ij->i", P[:, 0], np.cross(P[:, 1], P[:, 2])).sum() / 6.0
    return {"n_vertices": int(V.shape[0]), "n_triangles": int(T.shape[0]), "signed_volume": float(vol)}


_KUHN = []
for _order in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
    _bits, _path = 0, [0]
    for _a in _order:
        _bits |= 4 >> _a
        _path.append(_bits)
    _KUHN.append(_path)  # corners (bit 2: first index, bit 0: third) on the path 000 -> 111


def ball_tets(n: int, radius: float = 1.0, layers: int | None = None, core: float = 0.5):
    """Tetrahedral mesh of the ball of the given radius about the origin.

    A cubed sphere: an inner cube [-c, c]^3 (c = core * radius) of n^3
    cells, and a shell of ``layers`` (default n/2) hexahedral layers
    between the cube's surface and the sphere, six patches of n x n columns;
    a shell node over the cube-surface point q at layer k sits at
    (1 - t) q + t radius q/|q| with t = k/layers.  Every hexahedron, in its
    index coordinates (each patch indexed along increasing global axes and
    outward), is cut into the six tetrahedra along its main diagonal, so
    that neighbouring cells cut their shared faces alike (a conforming
    mesh), and no tetrahedron has all four nodes on the sphere.  n even.
    Returns (nodes [N][3] float64, tets [K][4] int32), every tet positively
    oriented.
    """
    if n < 2 or n % 2:
        raise ValueError("n must be even and at least 2")
    nr = max(1, n // 2) if layers is None else int(layers)
    H = n // 2
    W = n + 1

    def key(q, k):
        return (((q[:, 0] + H) * W + (q[:, 1] + H)) * W + (q[:, 2] + H)) * (nr + 1) + k

    def corner_offsets(b):
        return b >> 2 & 1, b >> 1 & 1, b & 1

    g = np.arange(-H, H + 1)
    Q = np.stack([x.ravel() for x in np.meshgrid(g, g, g, indexing="ij")], 1)
    keys = [key(Q, 0)]
    pos = [Q * (core * radius / H)]
    tet_keys = []
    c = np.arange(-H, H)
    base = np.stack([x.ravel() for x in np.meshgrid(c, c, c, indexing="ij")], 1)
    for path in _KUHN:
        tet_keys.append(np.stack([key(base + np.array(corner_offsets(b)), 0) for b in path], 1))
    for ax in range(3):
        o = [d for d in range(3) if d != ax]
        for side in (-1, 1):
            u, v = (x.ravel() for x in np.meshgrid(g, g, indexing="ij"))
            q = np.zeros((u.size, 3), dtype=np.int64)
            q[:, ax] = side * H
            q[:, o[0]], q[:, o[1]] = u, v
            qp = q * (core * radius / H)
            for k in range(1, nr + 1):
                t = k / nr
                keys.append(key(q, k))
                pos.append((1 - t) * qp + t * radius * qp / np.linalg.norm(qp, axis=1, keepdims=True))
            uu, vv, kk = (x.ravel() for x in np.meshgrid(c, c, np.arange(nr), indexing="ij"))
            for path in _KUHN:
                cols = []
                for b in path:
                    du, dv, dk = corner_offsets(b)
                    qq = np.zeros((uu.size, 3), dtype=np.int64)
                    qq[:, ax] = side * H
                    qq[:, o[0]], qq[:, o[1]] = uu + du, vv + dv
                    cols.append(key(qq, kk + dk))
                tet_keys.append(np.stack(cols, 1))
    keys = np.concatenate(keys)
    pos = np.concatenate(pos)
    uk, first = np.unique(keys, return_index=True)
    nodes = pos[first]
    allk = np.concatenate(tet_keys)
    tets = np.searchsorted(uk, allk)
    a, b, cc, d = (nodes[tets[:, q]] for q in range(4))
    vol = np.einsum("ij,ij->i", b - a, np.cross(cc - a, d - a))
    flip = vol < 0
    tets[flip, 2], tets[flip, 3] = tets[flip, 3].copy(), tets[flip, 2].copy()
    return nodes, tets.astype(np.int32)


def cube_tets(n: int, side: float = 1.0, nz: int | None = None):
    """Tetrahedral mesh of the cube [-side/2, side/2]^3 (or, with nz cells
    along z, of the slab of cubic cells side/n on a side and nz thick): n x n
    x nz cells, each cut into the six tetrahedra along its main diagonal
    (the cut _KUHN lists, conforming between cells).  Tetrahedra at the
    edges have all four nodes on the surface; with nz = 1 every node is.
    Returns (nodes [N][3], tets [K][4] int32), positively oriented."""
    nz = n if nz is None else int(nz)
    if n < 1 or nz < 1:
        raise ValueError("n and nz must be at least 1")
    g = np.linspace(-0.5 * side, 0.5 * side, n + 1)
    gz = (np.arange(nz + 1) - 0.5 * nz) * (side / n)
    nodes = np.stack([x.ravel() for x in np.meshgrid(g, g, gz, indexing="ij")], 1)

    def idx(i, j, k):
        return (i * (n + 1) + j) * (nz + 1) + k

    i, j, k = (x.ravel() for x in np.meshgrid(np.arange(n), np.arange(n), np.arange(nz), indexing="ij"))
    tets = np.concatenate([np.stack([idx(i + (b >> 2 & 1), j + (b >> 1 & 1), k + (b & 1)) for b in path], 1)
                           for path in _KUHN])
    a, b, cc, d = (nodes[tets[:, q]] for q in range(4))
    vol = np.einsum("ij,ij->i", b - a, np.cross(cc - a, d - a))
    flip = vol < 0
    tets[flip, 2], tets[flip, 3] = tets[flip, 3].copy(), tets[flip, 2].copy()
    return nodes, tets.astype(np.int32)


def shell_tets(n: int, r_in: float, radius: float, layers: int | None = None):
    """Tetrahedral mesh of the spherical shell r_in <= |x| <= radius: the
    cubed-sphere patches of ``ball_tets`` (n x n columns over each face of
    the cube) with ``layers`` (default n/2) hexahedral layers from the inner
    sphere to the outer one, node k of a column at radius
    r_in + (radius - r_in) k / layers, every hexahedron cut into six
    tetrahedra along its diagonal as in ``ball_tets``.  n even.  Returns
    (nodes [N][3], tets [K][4] int32), positively oriented."""
    if n < 2 or n % 2 or not (0.0 < r_in < radius):
        raise ValueError("n must be even and 0 < r_in < radius")
    nr = max(1, n // 2) if layers is None else int(layers)
    H = n // 2
    W = n + 1

    def key(q, k):
        return (((q[:, 0] + H) * W + (q[:, 1] + H)) * W + (q[:, 2] + H)) * (nr + 1) + k

    g = np.arange(-H, H + 1)
    c = np.arange(-H, H)
    keys, pos, tet_keys = [], [], []
    for ax in range(3):
        o = [d for d in range(3) if d != ax]
        for side in (-1, 1):
            u, v = (x.ravel() for x in np.meshgrid(g, g, indexing="ij"))
            q = np.zeros((u.size, 3), dtype=np.int64)
            q[:, ax] = side * H
            q[:, o[0]], q[:, o[1]] = u, v
            dirs = q / np.linalg.norm(q, axis=1, keepdims=True)
            for k in range(nr + 1):
                keys.append(key(q, k))
                pos.append(dirs * (r_in + (radius - r_in) * k / nr))
            uu, vv, kk = (x.ravel() for x in np.meshgrid(c, c, np.arange(nr), indexing="ij"))
            for path in _KUHN:
                cols = []
                for b in path:
                    du, dv, dk = b >> 2 & 1, b >> 1 & 1, b & 1
                    qq = np.zeros((uu.size, 3), dtype=np.int64)
                    qq[:, ax] = side * H
                    qq[:, o[0]], qq[:, o[1]] = uu + du, vv + dv
                    cols.append(key(qq, kk + dk))
                tet_keys.append(np.stack(cols, 1))
    keys = np.concatenate(keys)
    pos = np.concatenate(pos)
    uk, first = np.unique(keys, return_index=True)
    nodes = pos[first]
    tets = np.searchsorted(uk, np.concatenate(tet_keys))
    a, b, cc, d = (nodes[tets[:, q]] for q in range(4))
    vol = np.einsum("ij,ij->i", b - a, np.cross(cc - a, d - a))
    flip = vol < 0
    tets[flip, 2], tets[flip, 3] = tets[flip, 3].copy(), tets[flip, 2].copy()
    return nodes, tets.astype(np.int32)


def tet_volumes(nodes, tets):
    """Signed volumes of the tetrahedra (positive when positively oriented)."""
    a, b, c, d = (nodes[tets[:, q]] for q in range(4))
    return np.einsum("ij,ij->i", b - a, np.cross(c - a, d - a)) / 6.0
