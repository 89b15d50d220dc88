"""Triangle-integrated plans (opts.integration = 1): element-wise constant
charges, the gridding matrix of window integrals over the triangles (Sec. 3.1)
and exact near-field integrals (Sec. 3.4), against the oracle's
triangle-integrated definition (closed-form integrals of every pair)."""
import numpy as np
import pytest

import oracle
from synthetic import fields, meshes
from tests.gpu_util import lib, rel_l2, run, torch_cuda

pytestmark = pytest.mark.gpu


def _plan(slp, V, T, tol, prec, grid, kernel_mode=0, q=3):
    o = slp.slp_default_opts()
    o.precision = prec
    o.integration = 1
    o.kernel_mode = kernel_mode
    for d in range(3):
        o.grid[d] = grid[d]
    return slp.slp_plan(V, T, q, tol, o)


CASES = [
    # (name, mesh, tol, prec, grid, kernel_mode)
    ("sphere_L3_fp32", lambda: meshes.icosphere(3), 1e-5, 32, (64, 64, 64), 0),
    ("sphere_L4_fp32_128", lambda: meshes.icosphere(4), 1e-5, 32, (128, 128, 128), 0),
    ("sphere_L3_fp64", lambda: meshes.icosphere(3), 1e-10, 64, (64, 64, 64), 0),
    ("cube8_fp64_separable", lambda: meshes.cube(8), 1e-10, 64, (32, 32, 32), 0),
    ("box_fp32_aniso", lambda: meshes.box(2.0, 1.0, 0.5, 12, 6, 3), 1e-5, 32, (128, 64, 64), 0),
    ("sphere_L3_fp64_expsum", lambda: meshes.icosphere(3), 1e-4, 64, (64, 64, 64), 3),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_triangle_integrals_match_the_p0_oracle(case):
    """Nodal m (projected to element charges on the device) and the same
    element charges given directly both reproduce phi_i = (1/4pi) sum_j g_j
    int_{S_j} 1/|x_i - y| dA within the plan tolerance (the exp-sum kernel
    at its own accuracy, the tolerance 1e-4)."""
    name, mk, tol, prec, grid, kmode = case
    slp = lib()
    V, T = mk()
    plan = _plan(slp, V, T, tol, prec, grid, kmode)
    try:
        info = slp.slp_query(plan)
        assert info["integration"] == 1 and info["grid_matrix_nnz"] > 0 and info["near_tri_nnz"] > 0
        m = fields.smooth_random(V, 31)
        g = oracle.element_charges(V, T, m)
        ref = oracle.slp_p0(V, T, g)
        phi_m = run(slp, plan, slp.SLP_INPUT_NODAL_MAG, m, prec)
        phi_g = run(slp, plan, slp.SLP_INPUT_ELEMENT, g, prec)
        err_m, err_g = rel_l2(phi_m, ref), rel_l2(phi_g, ref)
        print(f"{name}: rel-L2 nodal {err_m:.3e} element {err_g:.3e} (tol {tol:g}); grid matrix "
              f"{info['grid_matrix_nnz']}, near {info['near_tri_nnz']} entries")
        assert err_m <= tol and err_g <= tol, (err_m, err_g)
    finally:
        slp.slp_destroy(plan)


def test_triangle_integral_gridding_stage_against_numpy():
    """The gridding product alone (stage SPREAD with element charges) equals
    sum_j g_j int_{S_j} Psi(r - u(y)) dA(y) evaluated in numpy with a finer
    (12 x 12) Duffy-Gauss rule and the window of Sec. 3.2."""
    slp = lib()
    torch = torch_cuda()
    V, T = meshes.icosphere(2)
    plan = _plan(slp, V, T, 1e-8, 64, (32, 32, 32))
    try:
        info = slp.slp_query(plan)
        L, m = info["grid"], info["m"]
        P, ctr = np.array(info["period"]), np.array(info["center"])
        g = np.random.default_rng(4).uniform(-1, 1, T.shape[0])
        run(slp, plan, slp.SLP_INPUT_ELEMENT, g, 64, slp.SLP_STAGE_SPREAD)
        A = slp.slp_debug_copy(plan, slp.SLP_BUF_GRID_A, np.float64).reshape(L[2], L[1], L[0])
        x, w = np.polynomial.legendre.leggauss(12)
        x, w = 0.5 * (x + 1), 0.5 * w
        S, Tt = np.meshgrid(x, x, indexing="ij")
        a, b = S.ravel(), (S * Tt).ravel()
        wt = (np.outer(w, w) * S).ravel()
        ref = np.zeros_like(A)
        U = (V - ctr) / P * np.array(L) + 0.5 * np.array(L)
        for j, (i0, i1, i2) in enumerate(T):
            area2 = np.linalg.norm(np.cross(V[i1] - V[i0], V[i2] - V[i0]))
            Y = U[i0] + a[:, None] * (U[i1] - U[i0]) + b[:, None] * (U[i2] - U[i1])
            lo = np.floor(U[[i0, i1, i2]].min(axis=0)).astype(int) - m + 1
            hi = np.floor(U[[i0, i1, i2]].max(axis=0)).astype(int) + m
            ax = [np.arange(lo[d], hi[d] + 1) for d in range(3)]
            win = [np.array([[slp.slp_debug_window(m, r - y) for r in ax[d]] for y in Y[:, d]]) for d in range(3)]
            box = np.einsum("p,pi,pj,pk->kji", wt * area2 * g[j], win[0], win[1], win[2])
            ref[np.ix_(ax[2] % L[2], ax[1] % L[1], ax[0] % L[0])] += box
        assert rel_l2(A, ref) < 1e-9, rel_l2(A, ref)
    finally:
        slp.slp_destroy(plan)


def test_triangle_integral_plans_refuse_point_inputs_and_batch():
    """SIGMA/MAG inputs need quadrature points and are refused; ELEMENT input
    is refused by point plans; the batched entry point runs element charges."""
    slp = lib()
    torch = torch_cuda()
    V, T = meshes.icosphere(2)
    plan = _plan(slp, V, T, 1e-5, 32, (32, 32, 32))
    o = slp.slp_default_opts()
    for d in range(3):
        o.grid[d] = 32
    point_plan = slp.slp_plan(V, T, 3, 1e-5, o)
    try:
        d_phi = torch.empty(V.shape[0], dtype=torch.float32, device="cuda")
        d_s = torch.zeros(3 * T.shape[0], dtype=torch.float32, device="cuda")
        with pytest.raises(slp.SlpError) as e:
            slp.slp_eval(plan, slp.SLP_INPUT_SIGMA, d_s, d_phi, torch.cuda.current_stream())
        assert e.value.status == slp.SLP_ERR_UNSUPPORTED
        with pytest.raises(slp.SlpError) as e:
            slp.slp_eval(point_plan, slp.SLP_INPUT_ELEMENT, d_s, d_phi, torch.cuda.current_stream())
        assert e.value.status == slp.SLP_ERR_UNSUPPORTED
        gs = [oracle.element_charges(V, T, fields.smooth_random(V, s)) for s in (1, 2, 3)]
        d_in = torch.as_tensor(np.concatenate(gs), dtype=torch.float32, device="cuda")
        d_out = torch.empty(3 * V.shape[0], dtype=torch.float32, device="cuda")
        slp.slp_eval_batched([plan], slp.SLP_INPUT_ELEMENT, [d_in], [d_out], [3], torch.cuda.current_stream())
        torch.cuda.synchronize()
        got = d_out.double().cpu().numpy().reshape(3, -1)
        for k in range(3):
            assert rel_l2(got[k], oracle.slp_p0(V, T, gs[k])) <= 1e-5
    finally:
        slp.slp_destroy(plan)
        slp.slp_destroy(point_plan)
