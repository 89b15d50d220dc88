"""CPU checks of the C ABI: the library loads and exports every declared
symbol, host-only plans validate meshes and choose consistent parameters,
and the plan-time sort and work lists are complete.  No GPU needed."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from synthetic import meshes, workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def slp():
    import paper_1305_3162_gb300 as m
    from paper_1305_3162_gb300 import _build
    _build.build()
    m.load()
    return m


def _declared_functions():
    names = set()
    for h in ("slp.h", "slp_debug.h"):
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for mt in re.finditer(r"\b(?:slp_status|double|const char \*|void)\s*\*?\s*(slp_\w+)\s*\(", src):
            names.add(mt.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(slp):
    names = _declared_functions()
    assert len(names) >= 15
    lib = ctypes.CDLL(slp.library_path())
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(slp.EXPORTED)


def _host_plan(slp, V, T, q=3, tol=1e-5, prec=32, grid=(0, 0, 0), **kw):
    o = slp.slp_default_opts()
    o.precision = prec
    o.device = -1
    for d in range(3):
        o.grid[d] = grid[d]
    for k, v in kw.items():
        setattr(o, k, v)
    return slp.slp_plan(V, T, q, tol, o)


def test_status_strings_and_errors(slp):
    assert slp.slp_status_string(0) == "ok"
    V, T = meshes.cube(2)
    with pytest.raises(slp.SlpError) as e:
        _host_plan(slp, V, T[:, ::-1].copy())  # inward normals
    assert e.value.status == slp.SLP_ERR_MESH
    with pytest.raises(slp.SlpError) as e:
        _host_plan(slp, V, T[:-1])  # open surface
    assert e.value.status == slp.SLP_ERR_MESH
    bad = T.copy()
    bad[0, 0] = V.shape[0]
    with pytest.raises(slp.SlpError) as e:
        _host_plan(slp, V, bad)
    assert e.value.status == slp.SLP_ERR_MESH
    with pytest.raises(slp.SlpError) as e:
        _host_plan(slp, V, T, q=5)
    assert e.value.status == slp.SLP_ERR_INVALID_ARG
    with pytest.raises(slp.SlpError) as e:
        _host_plan(slp, V, T, grid=(48, 32, 32))
    assert e.value.status == slp.SLP_ERR_INVALID_ARG
    # a degenerate (zero-area) triangle
    Vd = V.copy()
    t0 = T[0]
    Vd[t0[2]] = 0.5 * (Vd[t0[0]] + Vd[t0[1]])
    with pytest.raises(slp.SlpError):
        _host_plan(slp, Vd, T, check_mesh=0)
    # host-only plan cannot evaluate
    p = _host_plan(slp, V, T)
    with pytest.raises(slp.SlpError) as e:
        slp.slp_eval(p, 0, 1, 1, None)
    assert e.value.status == slp.SLP_ERR_NO_DEVICE
    slp.slp_destroy(p)


def test_infeasible_forced_grid(slp):
    w = workloads.plate(dims=(200.0, 50.0, 2.0), cell=1.0)
    with pytest.raises(slp.SlpError) as e:
        _host_plan(slp, w.V, w.T, grid=(256, 64, 16), kernel_mode=slp.SLP_KERNEL_RADIAL, allow_grid_raise=0)
    assert e.value.status == slp.SLP_ERR_TOLERANCE_INFEASIBLE
    p = _host_plan(slp, w.V, w.T, grid=(256, 64, 16))
    info = slp.slp_query(p)
    assert info["grid_raised"] == 1 and info["kernel_mode"] == slp.SLP_KERNEL_RADIAL
    assert all(math.pi * n > 2 * 4.0 ** 2 for n in info["modes"])
    slp.slp_destroy(p)


def test_radial_parameters_satisfy_their_constraints(slp):
    w = workloads.sphere(level=4)
    p = _host_plan(slp, w.V, w.T, q=7, grid=(128, 128, 128))
    info = slp.slp_query(p)
    assert info["kernel_mode"] == slp.SLP_KERNEL_RADIAL
    s, R, eps = info["sigma_g"], info["trunc_radius"], info["eps_near"]
    diam = 2.0  # unit sphere
    for d in range(3):
        P = info["period"][d]
        # no periodic image of the truncated, smoothed kernel reaches a difference vector
        assert P >= 2.0 + R - 1e-9
        # grid resolves the Gaussian: exp(-(s k_max)^2 / 2) small at the band edge
        kmax = math.pi * info["modes"][d] / P
        assert math.exp(-0.5 * (s * kmax) ** 2) < 1e-3
    assert R >= diam
    assert math.erfc(eps / (s * math.sqrt(2))) <= 2 * 1e-5 * 1.0001
    slp.slp_destroy(p)


def test_sort_permutation_and_grid_coordinates(slp):
    V, T = meshes.icosphere(3)
    p = _host_plan(slp, V, T, q=7, grid=(64, 64, 64))
    info = slp.slp_query(p)
    L = np.array(info["grid"])
    P = np.array(info["period"])
    c = np.array(info["center"])
    Q = info["n_sources"]
    perm = slp.slp_debug_host_array(p, slp.SLP_HOST_SRC_PERM)
    assert np.array_equal(np.sort(perm), np.arange(Q))
    g = slp.slp_debug_host_array(p, slp.SLP_HOST_SRC_GRID).reshape(-1, 4)
    packed = g[:, 3].astype(np.int64)
    cell = np.stack([packed & 1023, (packed >> 10) & 1023, (packed >> 20) & 1023], 1)
    assert np.all((g[:, :3] >= 0) & (g[:, :3] < 1))
    pts = slp.slp_query_points(p, Q)
    x = (cell + g[:, :3] - L / 2) * (P / L) + c
    assert np.abs(x - pts[perm]).max() < 1e-12
    # spread items cover every source once, each inside its tile
    it = slp.slp_debug_host_array(p, slp.SLP_HOST_SPREAD_ITEMS).reshape(-1, 8)
    cover = np.zeros(Q, int)
    for c0x, c0y, c0z, b, e, *_ in it:
        cover[b:e] += 1
        cc = cell[b:e] - np.array([c0x, c0y, c0z])
        assert np.all((cc >= 0) & (cc < 8))
    assert np.all(cover == 1)
    slp.slp_destroy(p)


def test_near_work_list_covers_every_close_pair(slp):
    """Every (target, source) pair closer than eps is visited by exactly one
    near-field work item (brute force over all pairs)."""
    V, T = meshes.icosphere(3)
    p = _host_plan(slp, V, T, q=7, grid=(128, 128, 128))
    info = slp.slp_query(p)
    eps = info["eps_near"]
    assert eps < 1.0  # a real near field, not all pairs
    sp = slp.slp_debug_host_array(p, slp.SLP_HOST_SRC_POINTS).reshape(-1, 3)
    tp = slp.slp_debug_host_array(p, slp.SLP_HOST_TGT_POINTS).reshape(-1, 3)
    items = slp.slp_debug_host_array(p, slp.SLP_HOST_NEAR_ITEMS).reshape(-1, 4)
    ranges = slp.slp_debug_host_array(p, slp.SLP_HOST_NEAR_RANGES).reshape(-1, 2)
    N, Q = tp.shape[0], sp.shape[0]
    visits = np.zeros((N, Q), np.int16)
    for tb, tc, rb, re_ in items:
        for r in range(rb, re_):
            visits[tb:tb + tc, ranges[r, 0]:ranges[r, 1]] += 1
    d = np.linalg.norm(tp[:, None, :] - sp[None, :, :], axis=2)
    close = d < eps
    assert np.all(visits[close] == 1)
    assert visits.max() == 1
    # the work list is not the all-pairs list
    assert visits.sum() < 0.5 * N * Q
    assert info["near_pairs"] == int(visits.sum())
    slp.slp_destroy(p)


@pytest.mark.parametrize("m", [4, 6])
def test_window_transform_matches_numerical_integral(slp, m):
    """Fourier transform of the normalised Kaiser-Bessel window (I0 closed
    form of Sec. 3.2, Eq. (cFB)) against a numerical integral of the window."""
    from scipy.integrate import quad
    L = 64
    for l in (0, 3, 11, 16):
        w = 2 * np.pi * l / L
        num, _ = quad(lambda d: slp.slp_debug_window(m, d) * np.cos(w * d), -m, m, limit=200, epsabs=1e-13)
        # the truncated window differs from the untruncated one by the
        # NFFT error; the untruncated tail beyond m is below C(2, m)
        assert abs(num - slp.slp_debug_window_hat(m, L, l)) < 10 * (4 * np.pi * (m ** 0.5 + m) * 0.5 ** 0.25 *
                                                                  np.exp(-2 * np.pi * m * 0.5 ** 0.5))
    assert abs(slp.slp_debug_window(m, 0.0) - 1.0) < 1e-15


def test_dtab_radial_matches_quadrature_of_the_kernel_transform(slp):
    """D = c_l(N_s) / W^2: recover c_l and compare with an independent FP64
    quadrature of the radial transform of the truncated kernel,
    (1/k) int_0^R sin(k r) dr, times the Gaussian factor."""
    from scipy.integrate import quad
    V, T = meshes.icosphere(2)
    p = _host_plan(slp, V, T, q=3, grid=(32, 32, 32))
    info = slp.slp_query(p)
    n = info["modes"]
    L = info["grid"]
    P = info["period"]
    m = info["m"]
    R = info["trunc_radius"]
    s = info["sigma_g"]
    D = slp.slp_debug_host_array(p, slp.SLP_HOST_DTAB).reshape(n[2] // 2, n[1] // 2, n[0] // 2)
    for (kz, ky, kx) in [(0, 0, 0), (1, 2, 3), (3, 1, 0), (7, 7, 7), (5, 0, 2)]:
        k = 2 * np.pi * np.sqrt((kx / P[0]) ** 2 + (ky / P[1]) ** 2 + (kz / P[2]) ** 2)
        if k == 0:
            ft = R * R / 2
        else:
            ft, _ = quad(lambda r: np.sin(k * r) / k, 0, R, limit=400, epsabs=1e-14)
        cl = ft * np.exp(-0.5 * s * s * k * k) / (P[0] * P[1] * P[2])
        W = (slp.slp_debug_window_hat(m, L[0], kx) * slp.slp_debug_window_hat(m, L[1], ky) *
             slp.slp_debug_window_hat(m, L[2], kz))
        assert abs(D[kz, ky, kx] * W * W - cl) <= 1e-10 * abs(cl) + 1e-16
    slp.slp_destroy(p)


def test_batch_and_server_refuse_host_only_plans(slp):
    V, T = meshes.cube(3)
    p = _host_plan(slp, V, T)
    try:
        with pytest.raises(slp.SlpError) as e:
            slp.slp_server_create([p], slp.SLP_INPUT_NODAL_MAG)
        assert e.value.status == slp.SLP_ERR_NO_DEVICE
        with pytest.raises(slp.SlpError) as e:
            slp.slp_batch_create([p], [0], slp.SLP_INPUT_NODAL_MAG, [1], [1])
        assert e.value.status == slp.SLP_ERR_NO_DEVICE
        with pytest.raises(slp.SlpError) as e:
            slp.slp_batch_create([p], [0], 7, [1], [1])  # unknown input kind
        assert e.value.status == slp.SLP_ERR_INVALID_ARG
    finally:
        slp.slp_destroy(p)


def _in_cyclic(v, start, count, L):
    return ((v - start) % L) < count


@pytest.mark.parametrize("shape", ["sphere", "torus", "plate"])
def test_active_region_covers_every_window_row(slp, shape):
    """The FFT passes only transform the active rows: every (z, y) row inside
    the window of a source (where grid A can be nonzero) or of a target
    (where the gather reads grid B) must be active, with pair-aligned
    intervals; and for a surface in its padded torus most rows are not."""
    if shape == "sphere":
        w = workloads.sphere(level=4)
        p = _host_plan(slp, w.V, w.T, q=7, grid=(128, 128, 128))
    elif shape == "torus":
        V, T = meshes.torus(2.0, 0.5, 48, 16)
        p = _host_plan(slp, V, T, q=3, grid=(64, 64, 32))
    else:
        w = workloads.plate(dims=(200.0, 50.0, 2.0), cell=1.0)
        p = _host_plan(slp, w.V, w.T, q=3, grid=(512, 128, 16))
    try:
        info = slp.slp_query(p)
        Lx, Ly, Lz = info["grid"]
        m = info["m"]
        iv = slp.slp_debug_host_array(p, slp.SLP_HOST_PLANE_ROWS).reshape(Lz, 2)
        z0, nz = slp.slp_debug_host_array(p, slp.SLP_HOST_ACTIVE_Z)
        assert np.all(iv[:, 0] % 2 == 0) and np.all(iv[:, 1] % 2 == 0)
        assert np.all((iv[:, 1] >= 0) & (iv[:, 1] <= Ly))
        active = np.zeros((Lz, Ly), bool)
        for z in range(Lz):
            if _in_cyclic(z, z0, nz, Lz):
                y = np.arange(Ly)
                active[z] = _in_cyclic(y, iv[z, 0], iv[z, 1], Ly)
            else:
                assert iv[z, 1] == 0
        assert info["active_rows"] == active.sum()
        need = np.zeros((Lz, Ly), bool)
        for which in (slp.SLP_HOST_SRC_GRID, slp.SLP_HOST_TGT_GRID):
            g = slp.slp_debug_host_array(p, which).reshape(-1, 4)
            pk = g[:, 3].astype(np.int64)
            cy, cz = (pk >> 10) & 1023, (pk >> 20) & 1023
            cells = np.unique(cz * Ly + cy)
            for oz in range(-m + 1, m + 1):
                for oy in range(-m + 1, m + 1):
                    need[((cells // Ly) + oz) % Lz, ((cells % Ly) + oy) % Ly] = True
        assert np.all(active[need]), "an active window row is pruned"
        assert active.sum() < 0.5 * Lz * Ly
    finally:
        slp.slp_destroy(p)


def test_spread_cell_groups_cover_each_item(slp):
    """The plan's spread groups: each item's sources covered exactly once,
    each group one cell and at most 16 sources, dealt to 8 lists whose work
    (4 per group + 1 per source) differs by at most one group's share."""
    w = workloads.sphere(level=4)
    p = _host_plan(slp, w.V, w.T, q=7, grid=(64, 64, 64))
    try:
        g = slp.slp_debug_host_array(p, slp.SLP_HOST_SRC_GRID).reshape(-1, 4)
        cells = g[:, 3].astype(np.int64)
        items = slp.slp_debug_host_array(p, slp.SLP_HOST_SPREAD_ITEMS).reshape(-1, 8)
        groups = slp.slp_debug_host_array(p, slp.SLP_HOST_SPREAD_GROUPS)
        off = slp.slp_debug_host_array(p, slp.SLP_HOST_SPREAD_GROUP_OFF).reshape(-1, 9)
        assert off.shape[0] == items.shape[0]
        for k, (c0x, c0y, c0z, b, e, *_) in enumerate(items):
            cover = np.zeros(e - b, int)
            loads = []
            for wl in range(8):
                load = 0
                for gd in groups[off[k, wl]:off[k, wl + 1]]:
                    first, n = gd & 0xFFFF, gd >> 16
                    assert 1 <= n <= 16
                    cover[first:first + n] += 1
                    assert np.all(cells[b + first:b + first + n] == cells[b + first])
                    load += 4 + n
                loads.append(load)
            assert np.all(cover == 1)
            assert max(loads) - min(loads) <= 4 + 16
        assert off[-1, 8] == groups.size
    finally:
        slp.slp_destroy(p)


def test_empty_and_minimal_meshes(slp):
    """No triangles -> SLP_ERR_INVALID_ARG; the smallest closed surface (a
    tetrahedron, 4 vertices) plans with automatic parameters."""
    with pytest.raises(slp.SlpError) as e:
        _host_plan(slp, np.zeros((0, 3)), np.zeros((0, 3), np.int32))
    assert e.value.status == slp.SLP_ERR_INVALID_ARG
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    T = np.array([[0, 2, 1], [0, 1, 3], [0, 3, 2], [1, 2, 3]], np.int32)
    p = _host_plan(slp, V, T, q=7)
    info = slp.slp_query(p)
    assert info["n_targets"] == 4 and info["n_sources"] == 28
    slp.slp_destroy(p)


@pytest.mark.parametrize("name", ["slp_mesh", "slp_plan_opts", "slp_info", "slp_tune_info", "slp_server_opts",
                                  "slp_server_statistics", "slp_potential_info"])
def test_struct_layouts_match_the_header(slp, name, tmp_path):
    """Every ctypes mirror of a public struct has the header's size and field
    offsets (a C program compiled against include/slp.h prints them)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    cls = getattr(slp, name)
    fields = [f for f, _ in cls._fields_]
    src = tmp_path / "layout.c"
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "slp.h"', "int main(void) {",
             f'    printf("%zu\\n", sizeof({name}));']
    lines += [f'    printf("%zu\\n", offsetof({name}, {f}));' for f in fields]
    lines += ["    return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got[0] == ctypes.sizeof(cls), (name, got[0], ctypes.sizeof(cls))
    for f, off in zip(fields, got[1:]):
        assert off == getattr(cls, f).offset, (name, f, off, getattr(cls, f).offset)


@pytest.mark.parametrize("case", ["sphere5-fp32", "cube100-fp32", "cube8-fp64"])
def test_plan_chooses_spread_occupancy_and_gather_items(slp, case):
    """The plan reads two launch choices off its own work lists: FP32 spread
    blocks per SM (4 with >= 8 sources per cell group, else 5; 0 outside the
    FP32 m <= 4 kernel) and the gather item size (64 targets, or 32 when
    that leaves fewer than four items per SM); every item respects it."""
    if case == "sphere5-fp32":
        w = workloads.sphere()
        V, T, q, tol, prec, grid = w.V, w.T, w.quad, w.tolerance, 32, w.grid
        want = (32, 4)
    elif case == "cube100-fp32":
        V, T = meshes.cube(100)
        q, tol, prec, grid = 3, 1e-5, 32, (512, 512, 512)
        want = (64, 5)
    else:
        w = workloads.cube()
        V, T, q, tol, prec, grid = w.V, w.T, w.quad, w.tolerance, 64, w.grid
        want = (32, 0)
    plan = _host_plan(slp, V, T, q, tol, prec, grid)
    try:
        info = slp.slp_query(plan)
        assert (info["gather_item_targets"], info["spread_blocks_per_sm"]) == want
        items = slp.slp_debug_host_array(plan, slp.SLP_HOST_GATHER_ITEMS).reshape(-1, 8)
        assert len(items) == info["n_gather_items"]
        sizes = items[:, 4] - items[:, 3]  # TileItem: c0x, c0y, c0z, begin, end, pad
        assert sizes.min() >= 1 and sizes.max() <= info["gather_item_targets"]
        assert int(sizes.sum()) == info["n_targets"]
        groups = slp.slp_debug_host_array(plan, slp.SLP_HOST_SPREAD_GROUPS)
        dense = info["n_sources"] >= 8 * len(groups)
        if want[1]:
            assert dense == (want[1] == 4)
    finally:
        slp.slp_destroy(plan)


def test_expsum_terms_approximate_inverse_r_on_the_far_interval(slp):
    """EXPSUM (Sec. 3.3): the kept Gaussians sum to 1/u within the plan
    tolerance on [eps/P, 1/2] (torus units), checked at 2000 log-spaced u with
    numpy; below eps the dropped narrow terms are missing, so the sum falls
    short of 1/u there (the near-field kernel carries the difference); every
    kept term is resolved by the grid (Fourier factor exp(-pi^2 l^2 / g) below
    the tolerance at |l| = n/2)."""
    V, T = meshes.icosphere(3)
    tol = 1e-4
    p = _host_plan(slp, V, T, q=7, tol=tol, grid=(64, 64, 64), kernel_mode=slp.SLP_KERNEL_EXPSUM)
    info = slp.slp_query(p)
    assert info["kernel_mode"] == slp.SLP_KERNEL_EXPSUM
    P = info["period"][0]
    assert info["period"] == [P, P, P]
    # the body sits in (-0.2, 0.2)^3 of the torus (the scaling of the paper's experiments)
    assert abs(np.ptp(V, axis=0).max() / P - 0.4) < 1e-9
    wg = slp.slp_debug_host_array(p, slp.SLP_HOST_EXPSUM).reshape(-1, 2)
    assert wg.shape[0] == info["expsum_terms"] > 5
    w, g = wg[:, 0], wg[:, 1]
    eu = info["eps_near"] / P
    u = np.exp(np.linspace(np.log(eu), np.log(0.5), 2000))
    s = (w[None, :] * np.exp(-g[None, :] * u[:, None] ** 2)).sum(axis=1)
    assert np.abs(s * u - 1).max() <= tol
    s0 = (w * np.exp(-g * (0.3 * eu) ** 2)).sum()
    assert s0 * 0.3 * eu < 1 - tol
    n = min(info["modes"])
    assert np.all(np.exp(-np.pi ** 2 * (n / 2) ** 2 / g) <= tol * 1.0001)
    slp.slp_destroy(p)


def test_expsum_dtab_matches_one_period_quadrature(slp):
    """EXPSUM D table: c_l(N_s) = (1 / (4 pi P)) sum_k w_k prod_q
    int_{-1/2}^{1/2} exp(-g_k u^2) cos(2 pi l_q u) du (the Fourier coefficient
    over one period, Sec. 2.2, of the separable Gaussians, Sec. 3.3), recovered
    from D W^2 and compared with scipy quadrature of each factor."""
    from scipy.integrate import quad
    V, T = meshes.icosphere(2)
    p = _host_plan(slp, V, T, q=3, tol=1e-4, grid=(32, 32, 32), kernel_mode=slp.SLP_KERNEL_EXPSUM)
    info = slp.slp_query(p)
    n, L, m = info["modes"], info["grid"], info["m"]
    P = info["period"][0]
    wg = slp.slp_debug_host_array(p, slp.SLP_HOST_EXPSUM).reshape(-1, 2)
    D = slp.slp_debug_host_array(p, slp.SLP_HOST_DTAB).reshape(n[2] // 2, n[1] // 2, n[0] // 2)

    def factor(g, l):
        v, _ = quad(lambda u: np.exp(-g * u * u) * np.cos(2 * np.pi * l * u), -0.5, 0.5, limit=400, epsabs=1e-14, epsrel=1e-12)
        return v

    for (kz, ky, kx) in [(0, 0, 0), (1, 2, 3), (3, 1, 0), (7, 7, 7), (5, 0, 2)]:
        cl = sum(w * factor(g, kx) * factor(g, ky) * factor(g, kz) for w, g in wg) / (4 * np.pi * P)
        W = (slp.slp_debug_window_hat(m, L[0], kx) * slp.slp_debug_window_hat(m, L[1], ky) *
             slp.slp_debug_window_hat(m, L[2], kz))
        assert abs(D[kz, ky, kx] * W * W - cl) <= 1e-9 * abs(cl) + 1e-14
    slp.slp_destroy(p)


def test_probe_sets_refuse_host_only_plans_and_bad_arguments(slp):
    V, T = meshes.cube(3)
    p = _host_plan(slp, V, T)
    try:
        with pytest.raises(slp.SlpError) as e:
            slp.slp_probe_create(p, np.zeros((4, 3)))
        assert e.value.status == slp.SLP_ERR_NO_DEVICE
        with pytest.raises(slp.SlpError) as e:
            slp.slp_probe_create(p, np.zeros((0, 3)))
        assert e.value.status == slp.SLP_ERR_INVALID_ARG
        with pytest.raises(slp.SlpError) as e:
            slp.slp_eval_probe(p, None, slp.SLP_INPUT_NODAL_MAG, 0, 0, 0)
        assert e.value.status == slp.SLP_ERR_INVALID_ARG
        with pytest.raises(slp.SlpError) as e:
            slp.slp_probe_query(None)
        assert e.value.status == slp.SLP_ERR_INVALID_ARG
        slp.slp_probe_destroy(None)
    finally:
        slp.slp_destroy(p)


def test_potential_refuses_host_only_plans_and_bad_meshes(slp):
    """The scalar potential needs a device; argument and mesh checks come first."""
    X, K = meshes.ball_tets(2, 1.0)
    o = slp.slp_default_opts()
    o.device = -1
    with pytest.raises(slp.SlpError) as e:
        slp.slp_potential_create(X, K, 1e-5, o)
    assert e.value.status == slp.SLP_ERR_NO_DEVICE
    with pytest.raises(slp.SlpError) as e:
        slp.slp_potential_create(X, K[:0], 1e-5)
    assert e.value.status == slp.SLP_ERR_INVALID_ARG
    with pytest.raises(slp.SlpError) as e:
        slp.slp_potential_create(X, K, 1e-5, cg_max_iterations=-1)
    assert e.value.status == slp.SLP_ERR_INVALID_ARG
    slp.slp_potential_destroy(None)
