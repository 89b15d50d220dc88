"""Kernel-by-kernel checks of one evaluation against plain numpy references
of the same stage (tests/stage_ref.py), on the plan's own sorted data."""
import numpy as np
import pytest

from synthetic import fields, meshes
from tests import stage_ref as ref
from tests.gpu_util import lib, rel_l2, run

pytestmark = pytest.mark.gpu


def _plan(slp, V, T, q, tol, prec, grid, kernel_mode=0, fuse=-1, table=-1):
    o = slp.slp_default_opts()
    o.precision = prec
    for d in range(3):
        o.grid[d] = grid[d]
    o.kernel_mode = kernel_mode
    o.fuse_plane_passes = fuse
    o.spread_table = table
    return slp.slp_plan(V, T, q, tol, o)


CASES = [
    # (name, mesh, q, tol, prec, grid, kernel_mode, rtol)
    ("sphere_L3_fp64_radial", lambda: meshes.icosphere(3), 7, 1e-8, 64, (64, 64, 64), 1, 1e-11),
    ("sphere_L3_fp32_radial", lambda: meshes.icosphere(3), 7, 1e-5, 32, (64, 64, 64), 1, 2e-5),
    ("box_fp32_aniso", lambda: meshes.box(2.0, 1.0, 0.5, 12, 6, 3), 3, 1e-5, 32, (128, 64, 64), 1, 2e-5),
    ("sphere_L3_fp32_table", lambda: meshes.icosphere(3), 7, 1e-5, 32, (64, 64, 64), 1, 2e-5),
    ("sphere_L3_fp64_expsum", lambda: meshes.icosphere(3), 7, 1e-4, 64, (64, 64, 64), 3, 1e-11),
    ("sphere_L3_fp32_expsum", lambda: meshes.icosphere(3), 7, 1e-4, 32, (64, 64, 64), 3, 2e-5),
    ("cube_fp64_separable", lambda: meshes.cube(8), 3, 1e-10, 64, (32, 32, 32), 2, 1e-11),
]


@pytest.mark.parametrize("fuse", [0, 1], ids=["separate", "fused"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_stages(case, fuse):
    """With fused plane passes, the FFT_Y stage runs FX + FY as one kernel
    (checked against the y transform of the separate FX output) and the
    IFFT_X stage runs IY + IX as one kernel (checked against the x transform
    of the separate IY output)."""
    name, mk, q, tol, prec, grid, kmode, rtol = case
    slp = lib()
    V, T = mk()
    table = 1 if name.endswith("_table") else 0
    plan = _plan(slp, V, T, q, tol, prec, grid, kmode, fuse, table)
    try:
        info = slp.slp_query(plan)
        assert info["fused_plane_passes"] == fuse
        assert info["spread_table"] == table
        L = info["grid"]
        n = info["modes"]
        m = info["m"]
        Kx = n[0] // 2
        fdt = np.float64 if prec == 64 else np.float32
        sigma = fields.random_sigma(T.shape[0] * q, 7)

        # charges
        run(slp, plan, slp.SLP_INPUT_SIGMA, sigma, prec, slp.SLP_STAGE_CHARGES)
        qb = slp.slp_debug_copy(plan, slp.SLP_BUF_QBUF, fdt).astype(np.float64)
        import oracle
        qk = oracle.charges(V, T, q, 0, sigma)
        perm = slp.slp_debug_host_array(plan, slp.SLP_HOST_SRC_PERM)
        assert np.abs(qb - qk[perm]).max() <= 4 * np.finfo(fdt).eps * np.abs(qk).max()

        # spread
        run(slp, plan, slp.SLP_INPUT_SIGMA, sigma, prec, slp.SLP_STAGE_SPREAD)
        A = slp.slp_debug_copy(plan, slp.SLP_BUF_GRID_A, fdt).astype(np.float64).reshape(L[2], L[1], L[0])
        sg = slp.slp_debug_host_array(plan, slp.SLP_HOST_SRC_GRID)
        A_ref = ref.spread(sg, qb, L, m)
        assert rel_l2(A, A_ref) < rtol, "spread"

        # active region: FY..IY work on planes z0 .. z0 + nz - 1, the x passes
        # and IY on the active rows of those planes; elsewhere the buffers are
        # zero (grid A rows there are zero, so the forward spectra are too)
        # and the inverse results are not computed (the gather never reads them)
        iv = slp.slp_debug_host_array(plan, slp.SLP_HOST_PLANE_ROWS).reshape(L[2], 2)
        z0, nz = slp.slp_debug_host_array(plan, slp.SLP_HOST_ACTIVE_Z)
        zact = ((np.arange(L[2]) - z0) % L[2]) < nz
        ract = ((np.arange(L[1])[None, :] - iv[:, :1]) % L[1]) < iv[:, 1:]
        assert np.all(A[~ract] == 0), "spread outside the active rows"

        # forward x
        run(slp, plan, slp.SLP_INPUT_SIGMA, sigma, prec, slp.SLP_STAGE_FFT_X)
        cdt = np.complex128 if prec == 64 else np.complex64
        S1 = slp.slp_debug_copy(plan, slp.SLP_BUF_S1, cdt).astype(np.complex128).reshape(L[2], L[1], Kx)
        S1_ref = ref.fft_x(A, Kx)
        assert rel_l2(S1, S1_ref) < rtol, "fft x"
        A_after = slp.slp_debug_copy(plan, slp.SLP_BUF_GRID_A, fdt)
        assert not np.any(A_after), "fft x must leave grid A zeroed"

        # forward y
        run(slp, plan, slp.SLP_INPUT_SIGMA, sigma, prec, slp.SLP_STAGE_FFT_Y)
        S2 = slp.slp_debug_copy(plan, slp.SLP_BUF_S2, cdt).astype(np.complex128).reshape(L[2], n[1], Kx)
        assert rel_l2(S2, ref.fft_y(S1, n[1])) < rtol, "fft y"

        # z, multiply, inverse z
        run(slp, plan, slp.SLP_INPUT_SIGMA, sigma, prec, slp.SLP_STAGE_FFT_Z)
        S2b = slp.slp_debug_copy(plan, slp.SLP_BUF_S2, cdt).astype(np.complex128).reshape(L[2], n[1], Kx)
        dtab = slp.slp_debug_copy(plan, slp.SLP_BUF_DTAB, fdt).astype(np.float64)
        S2b_ref = ref.fft_z_multiply(S2, dtab, n, L[2])
        assert rel_l2(S2b[zact], S2b_ref[zact]) < rtol, "fft z"
        assert not np.any(S2b[~zact])

        # inverse y
        run(slp, plan, slp.SLP_INPUT_SIGMA, sigma, prec, slp.SLP_STAGE_IFFT_Y)
        S1b = slp.slp_debug_copy(plan, slp.SLP_BUF_S1, cdt).astype(np.complex128).reshape(L[2], L[1], Kx)
        assert rel_l2(S1b[ract], ref.ifft_y(S2b, L[1])[ract]) < rtol, "ifft y"
        assert not np.any(S1b[~ract])

        # inverse x
        run(slp, plan, slp.SLP_INPUT_SIGMA, sigma, prec, slp.SLP_STAGE_IFFT_X)
        G = slp.slp_debug_copy(plan, slp.SLP_BUF_GRID_B, fdt).astype(np.float64).reshape(L[2], L[1], L[0])
        assert rel_l2(G[ract], ref.ifft_x(S1b, L[0])[ract]) < rtol, "ifft x"
        assert not np.any(G[~ract])

        # gather
        phi_far = run(slp, plan, slp.SLP_INPUT_SIGMA, sigma, prec, slp.SLP_STAGE_GATHER)
        tg = slp.slp_debug_host_array(plan, slp.SLP_HOST_TGT_GRID)
        tperm = slp.slp_debug_host_array(plan, slp.SLP_HOST_TGT_PERM)
        far_sorted = ref.gather(tg, G, L, m)
        far_ref = np.zeros_like(far_sorted)
        far_ref[tperm] = far_sorted
        assert rel_l2(phi_far, far_ref) < rtol, "gather"

        # near field (radial and exp-sum kernels; the separable kernel is checked end to end)
        phi = run(slp, plan, slp.SLP_INPUT_SIGMA, sigma, prec)
        if info["kernel_mode"] in (slp.SLP_KERNEL_RADIAL, slp.SLP_KERNEL_EXPSUM):
            sp = slp.slp_debug_host_array(plan, slp.SLP_HOST_SRC_POINTS).reshape(-1, 3)
            if info["kernel_mode"] == slp.SLP_KERNEL_RADIAL:
                near_sorted = ref.near_radial(V[tperm], sp, qb, info["eps_near"], info["sigma_g"])
            else:
                wg = slp.slp_debug_host_array(plan, slp.SLP_HOST_EXPSUM).reshape(-1, 2)
                near_sorted = ref.near_expsum(V[tperm], sp, qb, info["eps_near"], wg[:, 0], wg[:, 1],
                                              info["period"][0])
            near_ref = np.zeros_like(near_sorted)
            near_ref[tperm] = near_sorted
            scale = np.linalg.norm(phi)
            assert np.linalg.norm((phi - phi_far) - near_ref) / scale < rtol, "near field"
    finally:
        slp.slp_destroy(plan)
