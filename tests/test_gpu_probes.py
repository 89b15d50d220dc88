"""Probe sets: the single layer potential at points off the boundary (the
interior nodes of the finite element mesh, Sec. 2 and Algorithm 1) from the
same evaluation as the boundary nodes.  The probes reuse the grid the
evaluation leaves behind (interpolation, Sec. 3.3) and get their own rows of
the near-field operator (Sec. 3.4)."""
import numpy as np
import pytest

import oracle
from synthetic import fields, meshes
from tests.gpu_util import lib, rel_l2, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


def _points(rng, n_in, n_shell):
    """Points inside the unit sphere and points just inside its surface."""
    d = rng.normal(size=(n_in + n_shell, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    r = np.concatenate([rng.uniform(0.0, 0.9, n_in), rng.uniform(0.93, 0.985, n_shell)])
    return d * r[:, None]


def _torus_points(rng, n_tube, n_hole, R=1.0, r=0.4):
    """Points inside the tube of the torus about the z axis and points in
    its hole (outside the magnet, inside its bounding box and enclosing
    ball)."""
    u = rng.uniform(0, 2 * np.pi, n_tube)
    v = rng.uniform(0, 2 * np.pi, n_tube)
    s = r * np.sqrt(rng.uniform(0, 0.9, n_tube))
    tube = np.stack([(R + s * np.cos(v)) * np.cos(u), (R + s * np.cos(v)) * np.sin(u), s * np.sin(v)], 1)
    a = rng.uniform(0, 2 * np.pi, n_hole)
    rho = (R - r) * np.sqrt(rng.uniform(0, 0.9, n_hole))
    hole = np.stack([rho * np.cos(a), rho * np.sin(a), rng.uniform(-0.8 * r, 0.8 * r, n_hole)], 1)
    return np.vstack([tube, hole])


def _plan(slp, V, T, tol, prec, grid, integration=0, kernel_mode=0, near_mode=None):
    o = slp.slp_default_opts()
    o.precision = prec
    o.integration = integration
    o.kernel_mode = kernel_mode
    if near_mode is not None:
        o.near_mode = near_mode
    for d in range(3):
        o.grid[d] = grid[d]
    return slp.slp_plan(V, T, 3, tol, o)


def _eval(slp, plan, probe, kind, data, n_pts, prec):
    torch = torch_cuda()
    dt = torch.float64 if prec == 64 else torch.float32
    info = slp.slp_query(plan)
    d_in = to_dev(data, prec)
    d_phi = torch.zeros(info["n_targets"], dtype=dt, device="cuda")
    d_pts = torch.zeros(n_pts, dtype=dt, device="cuda")
    slp.slp_eval_probe(plan, probe, kind, d_in, d_phi, d_pts, torch.cuda.current_stream())
    torch.cuda.synchronize()
    slp.slp_check(plan)
    return d_phi.double().cpu().numpy(), d_pts.double().cpu().numpy()


CASES = [
    # (name, mesh, tol, prec, grid, integration, kernel_mode)
    ("points_fp32", "sphere3", 1e-5, 32, (64, 64, 64), 0, 0),
    ("points_fp64", "sphere3", 1e-10, 64, (64, 64, 64), 0, 0),
    ("points_fp32_L4_128", "sphere4", 1e-5, 32, (128, 128, 128), 0, 0),
    ("points_fp32_torus", "torus", 1e-5, 32, (128, 128, 64), 0, 0),
    ("triangles_fp32", "sphere3", 1e-5, 32, (64, 64, 64), 1, 0),
    ("triangles_fp64", "sphere3", 1e-10, 64, (64, 64, 64), 1, 0),
    ("triangles_fp64_torus", "torus", 1e-10, 64, (64, 64, 32), 1, 0),
    ("triangles_fp64_expsum", "sphere3", 1e-4, 64, (64, 64, 64), 1, 3),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_probes_match_the_oracle_off_the_surface(case):
    """phi at interior, near-surface and exterior points equals the oracle's
    definition (the quadrature sum for point plans, exact triangle integrals
    for triangle-integrated plans) within the plan tolerance; phi at the
    vertices from the same call equals slp_eval's."""
    name, mesh, tol, prec, grid, integ, kmode = case
    slp = lib()
    rng = np.random.default_rng(11)
    if mesh == "torus":
        V, T = meshes.torus(1.0, 0.4, 48, 16)
        x = _torus_points(rng, 300, 120)
        near = np.abs(np.hypot(np.hypot(x[:, 0], x[:, 1]) - 1.0, x[:, 2]) - 0.4) < 0.05
    else:
        V, T = meshes.icosphere(int(mesh[-1]))
        x = _points(rng, 300, 120)
        near = np.linalg.norm(x, axis=1) > 0.92
    plan = _plan(slp, V, T, tol, prec, grid, integ, kmode, None if integ else slp.SLP_NEAR_PRECOMPUTED)
    probe = slp.slp_probe_create(plan, x)
    try:
        q = slp.slp_probe_query(probe)
        assert q["n_points"] == x.shape[0] and q["near_nnz"] > 0
        m = fields.smooth_random(V, 5)
        phi_v, phi_x = _eval(slp, plan, probe, slp.SLP_INPUT_NODAL_MAG, m, x.shape[0], prec)
        if integ:
            g = oracle.element_charges(V, T, m)
            ref_x = oracle.slp_p0(V, T, g, x=x)
            ref_v = oracle.slp_p0(V, T, g)
            _, phi_xg = _eval(slp, plan, probe, slp.SLP_INPUT_ELEMENT, g, x.shape[0], prec)
            assert rel_l2(phi_xg, ref_x) <= tol, rel_l2(phi_xg, ref_x)
        else:
            y, _, _ = oracle.sources(V, T, 3)
            qk = oracle.charges(V, T, 3, oracle.KIND_NODAL_MAG, m)
            ref_x, _ = oracle.direct(x, y, qk)
            ref_v, _ = oracle.direct(V, y, qk)
        err_x, err_v = rel_l2(phi_x, ref_x), rel_l2(phi_v, ref_v)
        err_near = rel_l2(phi_x[near], ref_x[near])
        print(f"{name}: probes rel-L2 {err_x:.3e} (near-surface {err_near:.3e}), vertices {err_v:.3e}, "
              f"{q['near_nnz']} probe near entries")
        assert err_x <= tol and err_near <= 2 * tol and err_v <= tol, (err_x, err_near, err_v)
    finally:
        slp.slp_probe_destroy(probe)
        slp.slp_destroy(plan)


def test_probes_of_a_uniformly_magnetised_sphere():
    """m = e_z on the unit sphere: phi = z/3 inside (Sec. 4), up to the
    flat-facet error of the icosphere (below 4e-4 at 5120 triangles, the
    oracle's pinned bound)."""
    slp = lib()
    V, T = meshes.icosphere(4)
    plan = _plan(slp, V, T, 1e-10, 64, (64, 64, 64), integration=1)
    x = _points(np.random.default_rng(2), 200, 40)
    probe = slp.slp_probe_create(plan, x)
    try:
        m = np.tile([0.0, 0.0, 1.0], (V.shape[0], 1))
        _, phi_x = _eval(slp, plan, probe, slp.SLP_INPUT_NODAL_MAG, m, x.shape[0], 64)
        ref = x[:, 2] / 3
        assert np.abs(phi_x - ref).max() < 4e-4, np.abs(phi_x - ref).max()
    finally:
        slp.slp_probe_destroy(probe)
        slp.slp_destroy(plan)


def test_probe_refusals():
    """Probes need the precomputed near field or triangle integrals, lie in
    the mesh's bounding box and enclosing ball (a corner of the sphere's box
    is outside the ball) and on grid rows the plan transforms (between two
    spheres on opposite corners of their box, the plane z = 0 holds no row
    that either reaches), and belong to the plan they are evaluated with."""
    slp = lib()
    V, T = meshes.icosphere(2)
    fly = _plan(slp, V, T, 1e-5, 32, (32, 32, 32), near_mode=slp.SLP_NEAR_ON_THE_FLY)
    pre = _plan(slp, V, T, 1e-5, 32, (32, 32, 32), near_mode=slp.SLP_NEAR_PRECOMPUTED)
    other = _plan(slp, V, T, 1e-5, 32, (32, 32, 32), near_mode=slp.SLP_NEAR_PRECOMPUTED)
    probe = None
    try:
        with pytest.raises(slp.SlpError) as e:
            slp.slp_probe_create(fly, np.zeros((2, 3)))
        assert e.value.status == slp.SLP_ERR_UNSUPPORTED
        for bad in ([0.0, 0.0, 1.5], [0.9, 0.9, 0.9]):
            with pytest.raises(slp.SlpError) as e:
                slp.slp_probe_create(pre, np.array([[0.0, 0.0, 0.0], bad]))
            assert e.value.status == slp.SLP_ERR_INVALID_ARG
        V2 = np.vstack([V - 2.0, V + 2.0])
        T2 = np.vstack([T, T + V.shape[0]]).astype(np.int32)
        pair = _plan(slp, V2, T2, 1e-5, 32, (256, 256, 256), near_mode=slp.SLP_NEAR_PRECOMPUTED)
        try:
            ok = slp.slp_probe_create(pair, np.array([[-2.0, -2.0, -2.0], [2.0, 2.3, 2.0]]))
            slp.slp_probe_destroy(ok)
            with pytest.raises(slp.SlpError) as e:
                slp.slp_probe_create(pair, np.array([[-2.0, -2.0, -2.0], [2.0, -2.0, 0.0]]))
            assert e.value.status == slp.SLP_ERR_UNSUPPORTED
        finally:
            slp.slp_destroy(pair)
        probe = slp.slp_probe_create(pre, np.zeros((2, 3)))
        torch = torch_cuda()
        buf = torch.zeros(3 * V.shape[0], dtype=torch.float32, device="cuda")
        with pytest.raises(slp.SlpError) as e:
            slp.slp_eval_probe(other, probe, slp.SLP_INPUT_NODAL_MAG, buf, buf, buf)
        assert e.value.status == slp.SLP_ERR_INVALID_ARG
        with pytest.raises(slp.SlpError) as e:
            slp.slp_eval_probe(pre, probe, slp.SLP_INPUT_SIGMA, buf, buf, buf)
        assert e.value.status == slp.SLP_ERR_UNSUPPORTED
    finally:
        slp.slp_probe_destroy(probe)
        for p in (fly, pre, other):
            slp.slp_destroy(p)


@pytest.mark.parametrize("integration", [0, 1], ids=["points", "triangles"])
def test_probes_at_the_vertices_equal_the_boundary_result(integration):
    """Probes placed on the mesh vertices themselves get the same near-field
    rows and window weights as the plan's targets, so phi at those probes
    equals phi at the vertices (FP64, to rounding of the summation order)."""
    slp = lib()
    V, T = meshes.icosphere(3)
    plan = _plan(slp, V, T, 1e-10, 64, (64, 64, 64), integration, 0,
                 None if integration else slp.SLP_NEAR_PRECOMPUTED)
    probe = slp.slp_probe_create(plan, V)
    try:
        m = fields.smooth_random(V, 9)
        phi_v, phi_x = _eval(slp, plan, probe, slp.SLP_INPUT_NODAL_MAG, m, V.shape[0], 64)
        assert np.abs(phi_x - phi_v).max() <= 1e-13 * np.abs(phi_v).max(), np.abs(phi_x - phi_v).max()
    finally:
        slp.slp_probe_destroy(probe)
        slp.slp_destroy(plan)
