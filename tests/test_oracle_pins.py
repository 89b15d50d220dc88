"""Pins of the FP64 oracle against facts fixed by mathematics (no GPU).

Each check is chosen so a plausible mistake in the oracle fails it:
  * quadrature exactness (wrong point, weight or point order) -> monomial test;
  * 1/(4 pi), area, kernel power -> sphere eigenvalue tests (Sec. 4 sphere);
  * normal orientation / sign -> uniformly magnetised sphere, phi = z/3;
  * P1 interpolation of nodal m -> linear field, nodal vs point input;
  * the quadrature sum itself -> analytic integral of 1/|x-y| over a
    flat triangle (closed form, cross-checked by a Duffy-transformed
    Gauss-Legendre rule, the singular treatment of Sec. 3.4);
  * invariances: linearity, translation, scaling, axis permutation.
"""
import math

import numpy as np
import pytest

from synthetic import fields, meshes


# ---------------------------------------------------------------- helpers
def _monomial_integral(a, b, c):
    """Exact integral of l1^a l2^b l3^c over a triangle of area 1/2 (unit simplex):
    a! b! c! / (a+b+c+2)!  (the classical Dirichlet integral)."""
    return math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(a + b + c + 2)


def triangle_potential_closed_form(v0, v1, v2, x):
    """Integral of 1/|x - y| over the flat triangle (v0,v1,v2), dA(y).

    Edge-sum closed form for a uniformly charged planar polygon (Wilton et al.
    1984; Graglia 1993): with h the signed height of x over the plane, rho
    its projection, and for each edge (traversed counter-clockwise about the
    normal) the in-plane outward unit normal u, the edge direction l, the
    signed distances l-/l+ of the end points along l, P0 the distance of rho
    to the edge line along u, R+/R- the distances from x to the end points
    and R0^2 = P0^2 + h^2:

      I = sum_e P0 ln((R+ + l+)/(R- + l-))
          - |h| sum_e [atan(P0 l+ / (R0^2 + |h| R+)) - atan(P0 l- / (R0^2 + |h| R-))].
    """
    v = [np.asarray(p, float) for p in (v0, v1, v2)]
    x = np.asarray(x, float)
    nrm = np.cross(v[1] - v[0], v[2] - v[0])
    nrm /= np.linalg.norm(nrm)
    h = float(np.dot(x - v[0], nrm))
    rho = x - h * nrm
    ah = abs(h)
    total = 0.0
    for e in range(3):
        pm, pp = v[e], v[(e + 1) % 3]
        L = pp - pm
        lhat = L / np.linalg.norm(L)
        u = np.cross(lhat, nrm)
        lm = float(np.dot(pm - rho, lhat))
        lp = float(np.dot(pp - rho, lhat))
        P0 = float(np.dot(pm - rho, u))
        Rm = float(np.linalg.norm(x - pm))
        Rp = float(np.linalg.norm(x - pp))
        R02 = P0 * P0 + h * h
        if abs(P0) > 1e-14 * np.linalg.norm(L):  # P0 = 0: the log term vanishes
            total += P0 * math.log((Rp + lp) / (Rm + lm))
        if ah > 0:
            total -= ah * (math.atan(P0 * lp / (R02 + ah * Rp)) - math.atan(P0 * lm / (R02 + ah * Rm)))
    return total


def _duffy_about_v0(v0, v1, v2, x, n):
    """Duffy substitution about v0 (Sec. 3.4 of the paper):
    y = v0 + s (v1 - v0) + s t (v2 - v1), dA = 2|S| s ds dt, then a tensor
    Gauss-Legendre rule on [0,1]^2.  The factor s cancels the 1/r singularity
    when x sits at (or above) v0."""
    g, w = np.polynomial.legendre.leggauss(n)
    g = 0.5 * (g + 1)
    w = 0.5 * w
    S, Tt = np.meshgrid(g, g, indexing="ij")
    W = np.outer(w, w)
    Y = v0[None, None] + S[..., None] * (v1 - v0) + (S * Tt)[..., None] * (v2 - v1)
    area2 = np.linalg.norm(np.cross(v1 - v0, v2 - v0))
    r = np.linalg.norm(Y - x, axis=-1)
    return float(area2 * np.sum(W * S / r))


def triangle_potential_duffy(v0, v1, v2, x, n=80):
    """Same integral, numerically: split the triangle at the projection rho of
    x onto its plane into the three signed sub-triangles (rho, v_e, v_e+1) and
    integrate each with the Duffy rule about rho, where the integrand is
    nearly singular."""
    v = [np.asarray(p, float) for p in (v0, v1, v2)]
    x = np.asarray(x, float)
    nrm = np.cross(v[1] - v[0], v[2] - v[0])
    nrm /= np.linalg.norm(nrm)
    rho = x - np.dot(x - v[0], nrm) * nrm
    total = 0.0
    for e in range(3):
        a, b = v[e], v[(e + 1) % 3]
        sgn = np.sign(np.dot(np.cross(a - rho, b - rho), nrm))
        if sgn == 0:
            continue
        total += sgn * _duffy_about_v0(rho, a, b, x, n)
    return total


def _rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# ---------------------------------------------------------------- rules
@pytest.mark.parametrize("q,deg", [(1, 1), (3, 2), (7, 5)])
def test_rule_exact_to_degree(oracle_lib, q, deg):
    lam, w = oracle_lib.rule(q)
    assert np.all(w > 0)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(lam.sum(axis=1), 1.0, atol=1e-15)
    assert np.all(lam > 0)  # interior points only
    worst_exact = 0.0
    worst_next = 0.0
    for a in range(deg + 2):
        for b in range(deg + 2 - a):
            for c in range(deg + 2 - a - b):
                quad = 0.5 * np.sum(w * lam[:, 0] ** a * lam[:, 1] ** b * lam[:, 2] ** c)
                err = abs(quad - _monomial_integral(a, b, c))
                if a + b + c <= deg:
                    worst_exact = max(worst_exact, err)
                else:
                    worst_next = max(worst_next, err)
    assert worst_exact < 1e-15
    assert worst_next > 1e-6  # and no more: this is the rule of that degree


def test_rule_point_order_contract(oracle_lib):
    lam, w = oracle_lib.rule(3)
    assert np.allclose(lam, [[2 / 3, 1 / 6, 1 / 6], [1 / 6, 2 / 3, 1 / 6], [1 / 6, 1 / 6, 2 / 3]])
    lam, w = oracle_lib.rule(7)
    a1 = (6 - 15 ** 0.5) / 21
    assert np.allclose(lam[0], 1 / 3)
    assert np.allclose(lam[1], [a1, a1, 1 - 2 * a1])
    assert np.allclose(lam[3], [1 - 2 * a1, a1, a1])
    assert abs(w[0] - 9 / 40) < 1e-16


# ---------------------------------------------------------------- triangle integral
TRI = (np.array([0.1, -0.2, 0.05]), np.array([0.9, 0.1, -0.1]), np.array([0.2, 0.7, 0.3]))


@pytest.mark.parametrize("x", [
    (0.4, 0.2, 0.9), (2.0, -1.0, 0.5), (-0.3, 0.3, -0.4), (0.35, 0.25, 0.08), (5.0, 4.0, -3.0)])
def test_closed_form_matches_duffy(x):
    cf = triangle_potential_closed_form(*TRI, x)
    du = triangle_potential_duffy(*TRI, x, n=120)
    assert abs(cf - du) <= 1e-12 * abs(du)


def test_closed_form_at_vertex_singular():
    # x = v0: the Duffy rule about v0 is exact there (integrand becomes smooth).
    cf = triangle_potential_closed_form(*TRI, TRI[0])
    du = triangle_potential_duffy(*TRI, TRI[0], n=60)
    assert abs(cf - du) <= 1e-12 * abs(du)


@pytest.mark.parametrize("q,deg", [(3, 2), (7, 5)])
def test_oracle_quadrature_converges_to_triangle_integral(oracle_lib, q, deg):
    """Single-triangle mesh: the oracle's point sum at distance d converges to
    the exact integral like (h/d)^(deg+1)."""
    V = np.array(TRI)
    T = np.array([[0, 1, 2]], dtype=np.int32)
    y, wk, nrm = oracle_lib.sources(V, T, q)
    qk = oracle_lib.charges(V, T, q, 0, np.ones(q))
    c = V.mean(axis=0)
    dirn = np.array([0.3, -0.5, 0.81])
    dirn /= np.linalg.norm(dirn)
    errs = []
    for d in (4.0, 8.0, 16.0):
        x = (c + d * dirn)[None]
        phi, _ = oracle_lib.direct(x, y, qk)
        exact = triangle_potential_closed_form(*TRI, x[0]) / (4 * np.pi)
        errs.append(abs(phi[0] - exact) / abs(exact))
    # order of the quadrature error in the distance
    rate1 = math.log2(errs[0] / errs[1])
    rate2 = math.log2(errs[1] / errs[2])
    assert rate1 > deg + 0.5 and rate2 > deg + 0.5, (errs, rate1, rate2)
    assert errs[2] < 1e-5


# ---------------------------------------------------------------- sphere closed forms
def _sph(y):
    r = np.linalg.norm(y, axis=1)
    return y / r[:, None]


@pytest.mark.parametrize("q", [3, 7])
def test_sphere_unit_charge_potential_is_radius(oracle_lib, q):
    """sigma = 1 on the sphere of radius R gives phi = R on the surface."""
    errs = []
    for lev in (2, 3, 4):
        V, T = meshes.icosphere(lev, 1.0)
        phi = oracle_lib.slp(V, T, q, 0, np.ones(T.shape[0] * q))
        errs.append(np.abs(phi - 1.0).max())
    assert errs[0] > errs[1] > errs[2]
    assert errs[0] / errs[1] > 2.0 and errs[1] / errs[2] > 2.0
    assert errs[2] < 4e-3
    # scaling with the radius: phi = R
    V, T = meshes.icosphere(3, 2.5)
    phi = oracle_lib.slp(V, T, q, 0, np.ones(T.shape[0] * q))
    assert np.abs(phi / 2.5 - 1.0).max() < 1.2 * errs[1] + 1e-12


@pytest.mark.parametrize("ell", [1, 2, 3])
def test_sphere_harmonic_eigenvalues(oracle_lib, ell):
    """For sigma = P_l(cos theta) on the unit sphere, the single layer
    potential on the surface is P_l(cos theta) / (2l + 1)."""
    V, T = meshes.icosphere(4, 1.0)
    y, _, _ = oracle_lib.sources(V, T, 7)
    P = {1: lambda c: c, 2: lambda c: 0.5 * (3 * c * c - 1), 3: lambda c: 0.5 * (5 * c ** 3 - 3 * c)}[ell]
    # tilt the axis so no mesh symmetry helps
    ax = np.array([0.3, -0.4, 0.866])
    ax /= np.linalg.norm(ax)
    sigma = P(_sph(y) @ ax)
    phi = oracle_lib.slp(V, T, 7, 0, sigma)
    expect = P(_sph(V) @ ax) / (2 * ell + 1)
    assert np.abs(phi - expect).max() < 4e-3


def test_uniformly_magnetised_sphere(oracle_lib):
    """m = e3 in a sphere: sigma = m.n and phi = x3 / 3 (Sec. 4, phi_1 = 0)."""
    errs = []
    for lev in (2, 3, 4):
        V, T = meshes.icosphere(lev, 1.0)
        phi = oracle_lib.slp_nodal(V, T, 7, fields.uniform(V, (0, 0, 1)))
        errs.append(np.abs(phi - V[:, 2] / 3).max())
    assert errs[0] > errs[1] > errs[2]
    assert errs[0] / errs[1] > 2.0 and errs[1] / errs[2] > 2.0
    assert errs[2] < 3e-3
    # radius 0.2 as in the paper's test: phi scales with R for the same m
    V, T = meshes.icosphere(3, 0.2)
    phi = oracle_lib.slp_nodal(V, T, 7, fields.uniform(V, (0, 0, 1)))
    assert np.abs(phi - V[:, 2] / 3).max() < 0.2 * 1.2 * errs[1]


# ---------------------------------------------------------------- input kinds
@pytest.mark.parametrize("q", [3, 7])
def test_nodal_interpolation_matches_pointwise_for_linear_field(oracle_lib, q):
    """P1 interpolation reproduces a linear field exactly, so nodal m = A v
    must equal pointwise m = A y."""
    V, T = meshes.cube(3)
    A = np.array([[0.3, -1.2, 0.5], [0.7, 0.1, -0.4], [-0.2, 0.9, 1.1]])
    y, _, nrm = oracle_lib.sources(V, T, q)
    q_nodal = oracle_lib.charges(V, T, q, 2, V @ A.T)
    q_point = oracle_lib.charges(V, T, q, 1, y @ A.T)
    assert np.abs(q_nodal - q_point).max() < 1e-15
    # and sigma = m.n with outward normals: for m = e_x, only the x faces carry charge +-1
    qk = oracle_lib.charges(V, T, q, 2, fields.uniform(V, (1, 0, 0)))
    _, wk, _ = oracle_lib.sources(V, T, q)
    sig = qk / wk
    nx = np.repeat(nrm[:, 0], q)
    assert np.allclose(sig, nx)
    assert np.isclose(np.sum(qk), 0.0, atol=1e-14)  # total charge of a closed surface


# ---------------------------------------------------------------- invariances
def test_linearity_translation_scaling_permutation(oracle_lib):
    V, T = meshes.box(1.0, 0.6, 0.3, 5, 3, 2)
    Q = T.shape[0] * 3
    s1 = fields.random_sigma(Q, 11)
    s2 = fields.random_sigma(Q, 12)
    p1 = oracle_lib.slp(V, T, 3, 0, s1)
    p2 = oracle_lib.slp(V, T, 3, 0, s2)
    p12 = oracle_lib.slp(V, T, 3, 0, 2.0 * s1 - 0.5 * s2)
    assert _rel_l2(p12, 2.0 * p1 - 0.5 * p2) < 1e-14
    # translation of the whole geometry
    pt = oracle_lib.slp(V + np.array([3.0, -7.0, 1.5]), T, 3, 0, s1)
    assert _rel_l2(pt, p1) < 1e-12
    # scaling: areas ~ s^2, distances ~ s  ->  phi ~ s
    ps = oracle_lib.slp(2.5 * V, T, 3, 0, s1)
    assert _rel_l2(ps, 2.5 * p1) < 1e-14
    # axis permutation (a rotation composed with a reflection keeps |x - y|)
    perm = [2, 0, 1]
    pp = oracle_lib.slp(V[:, perm], T, 3, 0, s1)
    assert _rel_l2(pp, p1) < 1e-14


def test_direct_subset_matches_full(oracle_lib):
    V, T = meshes.icosphere(2)
    y, _, _ = oracle_lib.sources(V, T, 7)
    qk = oracle_lib.charges(V, T, 7, 0, fields.random_sigma(y.shape[0], 3))
    full, used = oracle_lib.direct(V, y, qk)
    sel = np.array([0, 5, 17, 100, 161])
    sub, _ = oracle_lib.direct_subset(V, sel, y, qk)
    assert used >= 1
    assert np.array_equal(sub, full[sel])


def test_mesh_generators_closed_and_outward():
    for V, T, nv, nt in [(*meshes.cube(8), 386, 768), (*meshes.icosphere(5), 10242, 20480),
                         (*meshes.box(2000, 500, 20, 400, 100, 4), 84002, 168000),
                         (*meshes.torus(2.0, 0.5, 40, 20), 800, 1600)]:
        st = meshes.mesh_stats(V, T)
        assert st["n_vertices"] == nv and st["n_triangles"] == nt
        assert st["signed_volume"] > 0
        # every directed edge appears once and its reverse once (closed, consistently oriented)
        e = np.concatenate([T[:, [0, 1]], T[:, [1, 2]], T[:, [2, 0]]]).astype(np.int64)
        key = e[:, 0] * (nv + 1) + e[:, 1]
        rkey = e[:, 1] * (nv + 1) + e[:, 0]
        assert np.unique(key).size == key.size
        assert np.array_equal(np.sort(key), np.sort(rkey))


# ---------------------------------------------------------------- triangle-integrated (P0) definition
@pytest.mark.parametrize("x", [(0.2, 0.3, 0.5), (0.2, 0.3, 0.0), (1.5, -0.4, 0.05), (0.0, 0.0, 0.0),
                               (0.5, 0.5, 0.0), (-3.0, 2.0, 1.0), (0.1, 0.1, -1e-6)])
def test_oracle_triangle_integral_matches_duffy_and_python_closed_form(oracle_lib, x):
    """The C closed form against the Duffy-transformed Gauss-Legendre rule
    about the projection of x (Sec. 3.4), including x on the plane, at a
    vertex and on an edge, and against the closed form written in Python."""
    rng = np.random.default_rng(5)
    for _ in range(4):
        v0 = rng.normal(size=3) * 0.1
        v1 = v0 + np.array([1.0, 0.1, 0.0]) + rng.normal(size=3) * 0.05
        v2 = v0 + np.array([0.2, 0.9, 0.0]) + rng.normal(size=3) * 0.05
        for xx in (np.asarray(x, float), v0, 0.5 * (v0 + v1)):
            c = oracle_lib.triangle_integral(v0, v1, v2, xx)
            assert abs(c - triangle_potential_closed_form(v0, v1, v2, xx)) <= 1e-13 * max(1.0, abs(c))
            assert abs(c - triangle_potential_duffy(v0, v1, v2, xx, 200)) <= 1e-12 * max(1.0, abs(c))


def test_oracle_triangle_integral_far_field_limit(oracle_lib):
    """Far from the triangle, the integral tends to |S| / |x - c| (c the
    centroid) with a relative correction of order (size / distance)^2."""
    v0, v1, v2 = np.array([0.0, 0, 0]), np.array([1.0, 0, 0]), np.array([0.0, 1, 0])
    area, c = 0.5, (v0 + v1 + v2) / 3
    prev = None
    for dist in (10.0, 20.0, 40.0, 80.0):
        x = c + dist * np.array([0.3, 0.5, 0.81]) / np.linalg.norm([0.3, 0.5, 0.81])
        err = abs(oracle_lib.triangle_integral(v0, v1, v2, x) * dist / area - 1.0)
        assert err < 1.0 / dist ** 2
        if prev is not None:
            assert err < prev / 3.0
        prev = err


def test_oracle_element_charges_are_integral_means(oracle_lib):
    """For a linear field m(x) = A x, the P1 interpolant is exact and the
    integral mean of m . n over a triangle is n . A c (c the centroid)."""
    V, T = meshes.icosphere(2)
    A = np.array([[0.3, -1.0, 0.2], [0.5, 0.1, 0.7], [-0.4, 0.2, 1.1]])
    g = oracle_lib.element_charges(V, T, V @ A.T)
    c = V[T].mean(axis=1)
    n = np.cross(V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]])
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    assert np.abs(g - np.einsum("ij,ij->i", c @ A.T, n)).max() < 1e-14


def test_oracle_p0_sphere_closed_forms_converge_at_second_order(oracle_lib):
    """Exact triangle integrals of element-wise constant charges on the
    icosphere: sigma = 1 gives phi = R and the uniformly magnetised sphere
    (g_j = n_j . e_z) gives phi = z/3 (Sec. 4), up to the flat-facet
    geometry error, which falls by about 4x per refinement (second order;
    the point rules above converge at first order)."""
    prev = None
    for level in (2, 3, 4):
        V, T = meshes.icosphere(level)
        sel = np.arange(0, V.shape[0], max(1, V.shape[0] // 300))
        e1 = np.abs(oracle_lib.slp_p0(V, T, np.ones(T.shape[0]), sel=sel) - 1.0).max()
        gz = oracle_lib.element_charges(V, T, np.tile([0.0, 0.0, 1.0], (V.shape[0], 1)))
        e2 = np.abs(oracle_lib.slp_p0(V, T, gz, sel=sel) - V[sel, 2] / 3).max()
        assert e1 < 0.3 / 4 ** level and e2 < 0.15 / 4 ** level, (level, e1, e2)
        if prev is not None:
            assert e1 < prev[0] / 3.5 and e2 < prev[1] / 3.5
        prev = (e1, e2)


def test_oracle_p0_invariances_and_subset(oracle_lib):
    """Linearity in g, translation invariance, phi(sX) = s phi(X) for the
    same g, and the subset form equal to the full one."""
    V, T = meshes.cube(4)
    rng = np.random.default_rng(3)
    g1, g2 = rng.uniform(-1, 1, T.shape[0]), rng.uniform(-1, 1, T.shape[0])
    p1, p2 = oracle_lib.slp_p0(V, T, g1), oracle_lib.slp_p0(V, T, g2)
    p12 = oracle_lib.slp_p0(V, T, 2.0 * g1 - 0.5 * g2)
    assert _rel_l2(p12, 2.0 * p1 - 0.5 * p2) < 1e-13
    assert _rel_l2(oracle_lib.slp_p0(V + np.array([3.0, -2.0, 7.0]), T, g1), p1) < 1e-12
    assert _rel_l2(oracle_lib.slp_p0(2.5 * V, T, g1), 2.5 * p1) < 1e-13
    sel = np.array([0, 5, 17, V.shape[0] - 1])
    assert np.array_equal(oracle_lib.slp_p0(V, T, g1, sel=sel), p1[sel])


def test_oracle_p0_off_surface_points_match_the_sphere_potentials(oracle_lib):
    """At points off the surface: sigma = 1 on the sphere of radius 1 gives
    phi = 1 inside and 1/|x| outside; the uniformly magnetised sphere gives
    z/3 inside and z/(3|x|^3) outside (Sec. 4).  The flat-facet error falls
    at second order, as on the surface."""
    rng = np.random.default_rng(8)
    d = rng.normal(size=(60, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    r = np.concatenate([rng.uniform(0.0, 0.7, 30), rng.uniform(1.3, 2.0, 30)])
    x = d * r[:, None]
    inside = r < 1
    ref1 = np.where(inside, 1.0, 1.0 / r)
    refz = np.where(inside, x[:, 2] / 3, x[:, 2] / (3 * r ** 3))
    prev = None
    for level in (2, 3, 4):
        V, T = meshes.icosphere(level)
        e1 = np.abs(oracle_lib.slp_p0(V, T, np.ones(T.shape[0]), x=x) - ref1).max()
        gz = oracle_lib.element_charges(V, T, np.tile([0.0, 0.0, 1.0], (V.shape[0], 1)))
        e2 = np.abs(oracle_lib.slp_p0(V, T, gz, x=x) - refz).max()
        assert e1 < 0.5 / 4 ** level and e2 < 0.2 / 4 ** level, (level, e1, e2)
        if prev is not None:
            assert e1 < prev[0] / 3.5 and e2 < prev[1] / 3.5, (level, e1, e2, prev)
        prev = (e1, e2)
