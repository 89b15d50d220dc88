"""End-to-end parity of slp_eval against the FP64 direct-sum oracle.

Tolerances are the relative L2 errors the plans are built for: 1e-10 for
the FP64 path, 1e-5 for the FP32 path (the arithmetic budget of the FP32
kernels is far below 1e-5: ~1e-7 per spread/FFT/gather value and a few
1e-7 for the compensated-free near-field sums of a few thousand terms).
"""
import numpy as np
import pytest

import oracle
from synthetic import fields, meshes, workloads
from tests.gpu_util import lib, rel_l2, run, torch_cuda

pytestmark = pytest.mark.gpu


def _plan(slp, V, T, q, tol, prec, grid=(0, 0, 0), **kw):
    o = slp.slp_default_opts()
    o.precision = prec
    for d in range(3):
        o.grid[d] = grid[d]
    for k, v in kw.items():
        setattr(o, k, v)
    return slp.slp_plan(V, T, q, tol, o)


def test_cube_fp64_workload():
    """Cube 8x8 per face, 3-point rule, grid 32^3, FP64, tolerance 1e-10."""
    slp = lib()
    w = workloads.cube()
    plan = _plan(slp, w.V, w.T, w.quad, w.tolerance, w.precision, w.grid)
    try:
        info = slp.slp_query(plan)
        assert info["grid"] == [32, 32, 32]
        phi = run(slp, plan, slp.SLP_INPUT_NODAL_MAG, w.m_nodal, 64)
        ref = oracle.slp_nodal(w.V, w.T, w.quad, w.m_nodal)
        assert rel_l2(phi, ref) <= 1e-10
    finally:
        slp.slp_destroy(plan)


@pytest.mark.parametrize("kind", [0, 1, 2])
@pytest.mark.parametrize("prec,tol", [(32, 1e-5), (64, 1e-10)])
def test_input_kinds_sphere_L3(kind, prec, tol):
    slp = lib()
    V, T = meshes.icosphere(3)
    q = 7
    Q = T.shape[0] * q
    data = {0: fields.random_sigma(Q, 21), 1: fields.random_mag(Q, 22), 2: fields.vortex(V, 23)}[kind]
    plan = _plan(slp, V, T, q, tol, prec, (64, 64, 64))
    try:
        phi = run(slp, plan, kind, data, prec)
        ref = oracle.slp(V, T, q, kind, data)
        assert rel_l2(phi, ref) <= tol
    finally:
        slp.slp_destroy(plan)


@pytest.mark.parametrize("fuse,fcol,table", [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)],
                         ids=["separate", "fused-plane", "fused-column", "spread-table"])
def test_sphere_L5_workload(fuse, fcol, table):
    """Sphere level 5 (20480 triangles), 7-point rule, grid 128^3, FP32, 1e-5,
    with the FFT passes separate, x and y fused per plane, and y, z, inverse
    y fused per x frequency; and with the spread reading window tables."""
    slp = lib()
    w = workloads.sphere()
    plan = _plan(slp, w.V, w.T, w.quad, w.tolerance, w.precision, w.grid, fuse_plane_passes=fuse,
                 fuse_column_passes=fcol, spread_table=table)
    try:
        info = slp.slp_query(plan)
        assert info["grid"] == [128, 128, 128] and not info["grid_raised"]
        assert info["fused_plane_passes"] == fuse
        assert info["fused_column_passes"] == fcol
        assert info["spread_table"] == table
        phi = run(slp, plan, slp.SLP_INPUT_NODAL_MAG, w.m_nodal, 32)
        ref = oracle.slp_nodal(w.V, w.T, w.quad, w.m_nodal)
        err = rel_l2(phi, ref)
        assert err <= 1e-5, err
        # per-target error report
        rel_t = np.abs(phi - ref) / np.abs(ref).max()
        assert rel_t.max() < 1e-4
    finally:
        slp.slp_destroy(plan)


@pytest.mark.parametrize("case", ["cube-L32-fp64", "sphere3-L64-fp32", "sphere3-L64-fp64", "sphere4-L128-fp32",
                                  "sphere4-L256-fp32"])
def test_fused_column_passes_match_separate(case):
    """The fused column passes (FY, FZ * D * IZ, IY in one cluster launch)
    give the separate passes' result at every length they compile for, in
    both precisions; where they do not apply (256^3 here: too many modes per
    CTA) the plan keeps the separate passes."""
    slp = lib()
    if case.startswith("cube"):
        V, T = meshes.cube(8)
        q, L = 3, 32
    else:
        V, T = meshes.icosphere(3 if "sphere3" in case else 4)
        q, L = 7, int(case.split("-L")[1].split("-")[0])
    prec = 64 if case.endswith("fp64") else 32
    tol = 1e-10 if prec == 64 else 1e-5
    m = fields.smooth_random(V, 77)
    res = {}
    for fcol in (0, 1):
        plan = _plan(slp, V, T, q, tol, prec, (L, L, L), fuse_plane_passes=0, fuse_column_passes=fcol)
        try:
            info = slp.slp_query(plan)
            res[fcol] = (info["fused_column_passes"], run(slp, plan, slp.SLP_INPUT_NODAL_MAG, m, prec))
        finally:
            slp.slp_destroy(plan)
    assert res[0][0] == 0
    assert res[1][0] == (0 if L == 256 else 1)
    assert rel_l2(res[1][1], res[0][1]) < (1e-13 if prec == 64 else 2e-6)
    assert rel_l2(res[1][1], oracle.slp_nodal(V, T, q, m)) <= tol


def test_repeat_and_host_entry_point():
    """Two evaluations in a row agree (the spread grid is re-zeroed), and the
    host-buffer entry point gives the same numbers."""
    slp = lib()
    V, T = meshes.icosphere(3)
    m = fields.vortex(V, 5)
    plan = _plan(slp, V, T, 7, 1e-5, 32, (64, 64, 64))
    try:
        a = run(slp, plan, 2, m, 32)
        b = run(slp, plan, 2, m, 32)
        assert rel_l2(a, b) < 1e-6
        h_in = np.ascontiguousarray(m, dtype=np.float32)
        h_out = np.zeros(V.shape[0], dtype=np.float32)
        slp.slp_eval_host(plan, 2, h_in, h_out, None)
        assert rel_l2(h_out.astype(np.float64), a) < 1e-6
    finally:
        slp.slp_destroy(plan)


@pytest.mark.parametrize("prec,tol", [(32, 1e-5), (64, 1e-10)])
def test_deterministic_mode_bitwise(prec, tol):
    """deterministic = 1: the spread is the product with the point gridding
    matrix and the near field sums in item order, so the same input gives
    the same bits on every evaluation, with other evaluations (another state,
    sigma input) run in between, for nodal and sigma inputs."""
    slp = lib()
    V, T = meshes.icosphere(3)
    m = fields.vortex(V, 6)
    sigma = fields.random_sigma(T.shape[0] * 7, 8)
    plan = _plan(slp, V, T, 7, tol, prec, (64, 64, 64), deterministic=1)
    try:
        info = slp.slp_query(plan)
        assert info["deterministic_spread"] == 1 and info["grid_matrix_nnz"] == T.shape[0] * 7 * (2 * info["m"]) ** 3
        a = run(slp, plan, slp.SLP_INPUT_NODAL_MAG, m, prec)
        assert rel_l2(a, oracle.slp_nodal(V, T, 7, m)) <= tol
        s1 = run(slp, plan, slp.SLP_INPUT_SIGMA, sigma, prec)
        assert rel_l2(s1, oracle.slp(V, T, 7, oracle.KIND_SIGMA, sigma)) <= tol
        run(slp, plan, slp.SLP_INPUT_NODAL_MAG, fields.vortex(V, 7), prec)
        b = run(slp, plan, slp.SLP_INPUT_NODAL_MAG, m, prec)
        s2 = run(slp, plan, slp.SLP_INPUT_SIGMA, sigma, prec)
        assert np.array_equal(a, b) and np.array_equal(s1, s2)
    finally:
        slp.slp_destroy(plan)


def test_torus_fp32():
    slp = lib()
    w = workloads.torus(nu=96, nv=32)
    plan = _plan(slp, w.V, w.T, w.quad, 1e-5, 32, (128, 128, 64))
    try:
        phi = run(slp, plan, 2, w.m_nodal, 32)
        ref = oracle.slp_nodal(w.V, w.T, w.quad, w.m_nodal)
        assert rel_l2(phi, ref) <= 1e-5
    finally:
        slp.slp_destroy(plan)


def test_plate_workload_sampled():
    """Thin plate 2000x500x20 (168000 triangles), 3-point rule, FP32.  The
    requested 512x128x16 grid cannot resolve the smooth kernel along z at
    1e-5, so the plan raises it; checked at 2048 sampled nodes."""
    slp = lib()
    w = workloads.plate()
    plan = _plan(slp, w.V, w.T, w.quad, w.tolerance, w.precision, w.grid)
    try:
        info = slp.slp_query(plan)
        assert info["grid_raised"] == 1
        phi = run(slp, plan, 2, w.m_nodal, 32)
        rng = np.random.default_rng(w.seed)
        sel = np.sort(rng.choice(w.V.shape[0], 2048, replace=False))
        y, _, _ = oracle.sources(w.V, w.T, w.quad)
        qk = oracle.charges(w.V, w.T, w.quad, 2, w.m_nodal)
        ref, _ = oracle.direct_subset(w.V, sel, y, qk)
        assert rel_l2(phi[sel], ref) <= 1e-5
    finally:
        slp.slp_destroy(plan)


@pytest.mark.parametrize("prec,tol", [(32, 1e-5), (64, 1e-10)])
def test_near_field_modes_agree(prec, tol):
    """Nodal input: the precomputed vertex-based near-field operator and the
    per-evaluation near field give the same potential, both within the
    tolerance of the oracle."""
    slp = lib()
    V, T = meshes.icosphere(4)
    m = fields.vortex(V, 31)
    ref = oracle.slp_nodal(V, T, 7, m)
    out = {}
    for mode in (slp.SLP_NEAR_PRECOMPUTED, slp.SLP_NEAR_ON_THE_FLY):
        plan = _plan(slp, V, T, 7, tol, prec, (64, 64, 64), near_mode=mode)
        try:
            info = slp.slp_query(plan)
            assert info["near_mode"] == mode
            if mode == slp.SLP_NEAR_PRECOMPUTED:
                assert info["near_matrix_nnz"] > 0
                assert 0 < info["near_pairs_within"] <= info["near_pairs"]
            out[mode] = run(slp, plan, slp.SLP_INPUT_NODAL_MAG, m, prec)
            assert rel_l2(out[mode], ref) <= tol
        finally:
            slp.slp_destroy(plan)
    assert rel_l2(out[slp.SLP_NEAR_PRECOMPUTED], out[slp.SLP_NEAR_ON_THE_FLY]) <= tol


def test_separable_mode_precomputed_near_field():
    """All-pairs separable kernel with the precomputed operator (cube, FP64)."""
    slp = lib()
    w = workloads.cube()
    plan = _plan(slp, w.V, w.T, w.quad, w.tolerance, 64, w.grid, near_mode=slp.SLP_NEAR_PRECOMPUTED)
    try:
        info = slp.slp_query(plan)
        assert info["kernel_mode"] == slp.SLP_KERNEL_SEPARABLE and info["near_mode"] == slp.SLP_NEAR_PRECOMPUTED
        phi = run(slp, plan, slp.SLP_INPUT_NODAL_MAG, w.m_nodal, 64)
        assert rel_l2(phi, oracle.slp_nodal(w.V, w.T, w.quad, w.m_nodal)) <= 1e-10
    finally:
        slp.slp_destroy(plan)


@pytest.mark.parametrize("grid", [(1024, 1024, 64), (64, 64, 1024), (512, 512, 512)],
                         ids=["xy1024", "z1024", "512cube"])
def test_long_transforms(grid):
    """Transform lengths 512 and 1024 (the compile-time column engine at its
    largest lengths, the compile-time inverse x pass, the z pass with its
    register budget): a small slab elongated along the long axes, FP32, 1e-5."""
    slp = lib()
    dims = [4.0 if g >= 512 else 0.5 for g in grid]
    nseg = [16 if g >= 512 else 2 for g in grid]
    V, T = meshes.box(*dims, *nseg)
    m = fields.smooth_random(V, 31)
    plan = _plan(slp, V, T, 3, 1e-5, 32, grid, allow_grid_raise=0)
    try:
        info = slp.slp_query(plan)
        assert info["grid"] == list(grid)
        phi = run(slp, plan, slp.SLP_INPUT_NODAL_MAG, m, 32)
        ref = oracle.slp_nodal(V, T, 3, m)
        assert rel_l2(phi, ref) <= 1e-5
    finally:
        slp.slp_destroy(plan)


def test_timeline_milestones_are_ordered():
    """slp_debug_timeline runs the concurrent evaluation: the spread ends
    before the FFT passes, and the gather ends last (it waits for the near
    branch); the result is the same evaluation."""
    slp = lib()
    torch = pytest.importorskip("torch")
    V, T = meshes.icosphere(3)
    m = fields.vortex(V, 41)
    plan = _plan(slp, V, T, 7, 1e-5, 32, (64, 64, 64))
    try:
        d_in = torch.as_tensor(m, dtype=torch.float32, device="cuda")
        d_phi = torch.empty(V.shape[0], dtype=torch.float32, device="cuda")
        tl = slp.slp_debug_timeline(plan, slp.SLP_INPUT_NODAL_MAG, d_in, d_phi)
        assert 0 < tl["spread"] <= tl["fft"] <= tl["gather"]
        assert 0 < tl["near"] <= tl["gather"]
        ref = run(slp, plan, slp.SLP_INPUT_NODAL_MAG, m, 32)
        assert rel_l2(d_phi.double().cpu().numpy(), ref) < 1e-6
    finally:
        slp.slp_destroy(plan)


def _tetrahedron():
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    T = np.array([[0, 2, 1], [0, 1, 3], [0, 3, 2], [1, 2, 3]], np.int32)
    return V, T


@pytest.mark.parametrize("prec,tol", [(32, 1e-5), (64, 1e-10)])
def test_tetrahedron(prec, tol):
    """The smallest closed surface: 4 targets, 4 triangles, automatic grid."""
    slp = lib()
    V, T = _tetrahedron()
    m = np.array([[1.0, 0.2, -0.3], [0.0, 1.0, 0.5], [0.3, -0.4, 1.0], [-1.0, 0.5, 0.2]])
    plan = _plan(slp, V, T, 7, tol, prec)
    try:
        phi = run(slp, plan, slp.SLP_INPUT_NODAL_MAG, m, prec)
        ref = oracle.slp_nodal(V, T, 7, m)
        assert rel_l2(phi, ref) <= tol
    finally:
        slp.slp_destroy(plan)


def test_far_from_origin_and_zero_input():
    """A sphere centred at (1000, -2000, 500): FP32 keeps its accuracy because
    positions are stored as integer cells plus fractions relative to the
    torus; and a zero magnetisation gives exactly zero."""
    slp = lib()
    V, T = meshes.icosphere(3)
    V = V + np.array([1000.0, -2000.0, 500.0])
    m = fields.vortex(V - V.mean(0), 51)
    plan = _plan(slp, V, T, 7, 1e-5, 32, (64, 64, 64))
    try:
        phi = run(slp, plan, slp.SLP_INPUT_NODAL_MAG, m, 32)
        ref = oracle.slp_nodal(V, T, 7, m)
        assert rel_l2(phi, ref) <= 1e-5
        zero = run(slp, plan, slp.SLP_INPUT_NODAL_MAG, np.zeros_like(m), 32)
        assert np.all(zero == 0.0)
    finally:
        slp.slp_destroy(plan)


@pytest.mark.parametrize("body,level,grid,prec,near,bar",
                         [("sphere", 3, 64, 32, 0, 1e-4), ("sphere", 4, 128, 32, 0, 1e-4),
                          ("sphere", 3, 64, 64, 1, 1e-4), ("sphere", 4, 128, 64, 2, 1e-4),
                          ("cube", 12, 64, 64, 0, 2e-4)],
                         ids=["sphere-L3-64-fp32", "sphere-L4-128-fp32", "sphere-L3-64-fp64-onthefly",
                              "sphere-L4-128-fp64-precomputed", "cube12-64-fp64"])
def test_expsum_kernel_mode_at_the_papers_accuracy(body, level, grid, prec, near, bar):
    """The paper's kernel (EXPSUM: exponential sum of Gaussians, Sec. 3.3,
    separable one-period Fourier coefficients, near kernel 1/r - N_s) through
    the same spread / FFT / gather path, against the FP64 oracle, at plan
    tolerance 1e-4.  On the sphere every pair distance stays inside the
    sum's interval [eps, P/2] and the error stays within the tolerance
    (measured 4.1e-5 at 64^3, 5.9e-6 at 128^3); on the cube the
    corner-to-corner pairs (0.69 P) lie beyond P/2, where the Gaussians no
    longer follow 1/r exactly (measured 7.4e-5), so the cube's bar is twice
    the tolerance."""
    slp = lib()
    V, T = meshes.icosphere(level) if body == "sphere" else meshes.cube(level)
    q = 7 if body == "sphere" else 3
    plan = _plan(slp, V, T, q, 1e-4, prec, (grid, grid, grid), kernel_mode=slp.SLP_KERNEL_EXPSUM, near_mode=near)
    try:
        info = slp.slp_query(plan)
        assert info["kernel_mode"] == slp.SLP_KERNEL_EXPSUM and info["expsum_terms"] > 5
        m = fields.vortex(V, 21)
        phi = run(slp, plan, slp.SLP_INPUT_NODAL_MAG, m, prec)
        ref = oracle.slp_nodal(V, T, q, m)
        err = rel_l2(phi, ref)
        print(f"EXPSUM {body} {level} grid {grid} FP{prec}: rel-L2 {err:.3e}, S' = {info['expsum_terms']}, "
              f"eps/P = {info['eps_near'] / info['period'][0]:.4f}")
        assert err <= bar, err
        # sigma input (on-the-fly near field) gives the same potential
        sig = oracle.charges(V, T, q, oracle.KIND_NODAL_MAG, m)
        _, wk, _ = oracle.sources(V, T, q)
        phi_s = run(slp, plan, slp.SLP_INPUT_SIGMA, sig / wk, prec)
        assert rel_l2(phi_s, phi) <= (1e-5 if prec == 32 else 1e-10)
    finally:
        slp.slp_destroy(plan)


def test_pipelined_host_evaluation_matches_device_evaluation():
    """slp_eval_host_async: six states through the two staging slots (copy-in,
    evaluation and copy-out on separate streams, each call's output in its own
    page-locked buffer) give the results of slp_eval on the same states."""
    slp = lib()
    torch = torch_cuda()
    V, T = meshes.icosphere(3)
    plan = _plan(slp, V, T, 7, 1e-5, 32, (64, 64, 64))
    try:
        states = [fields.vortex(V, 40 + i) for i in range(6)]
        h_in = [torch.as_tensor(m.ravel(), dtype=torch.float32).pin_memory() for m in states]
        h_out = [torch.full((V.shape[0],), float("nan"), dtype=torch.float32).pin_memory() for _ in states]
        stream = torch.cuda.current_stream()
        for a, b in zip(h_in, h_out):
            slp.slp_eval_host_async(plan, slp.SLP_INPUT_NODAL_MAG, a, b, stream)
        slp.slp_eval_host_wait(plan)
        for m, b in zip(states, h_out):
            ref = run(slp, plan, slp.SLP_INPUT_NODAL_MAG, m, 32)
            assert rel_l2(b.numpy().astype(np.float64), ref) < 1e-6
    finally:
        slp.slp_destroy(plan)
