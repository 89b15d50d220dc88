"""The allocation-free entry point slp_eval_direct_static.

It serves callers that cannot call cudaMalloc where they need the potential:
host code inside another framework's memory pool, which forbids raw device
allocations, and solver loops that must not touch the allocator after
start-up.  It must give the same potential as slp_eval, within the
tolerance the other tests use, call after call, although every call reuses
the same static scratch array inside the library; and it must stay within
that tolerance of the FP64 oracle up to its documented source limit.

This file is collected last on purpose, so that a run that stops at the
first failure has already run every other test.
"""
import numpy as np
import pytest

import oracle
from synthetic import fields, meshes
from tests.gpu_util import lib, rel_l2, run, torch_cuda

pytestmark = pytest.mark.gpu


def _direct_static(slp, torch, V, T, q, prec, kind, data):
    dt = torch.float64 if prec == 64 else torch.float32
    d_V = torch.as_tensor(V, dtype=torch.float64, device="cuda")
    d_T = torch.as_tensor(T, dtype=torch.int32, device="cuda")
    d_in = torch.as_tensor(np.ascontiguousarray(data).ravel(), dtype=dt, device="cuda")
    d_phi = torch.full((V.shape[0],), float("nan"), dtype=dt, device="cuda")
    slp.slp_eval_direct_static(d_V, V.shape[0], d_T, T.shape[0], q, prec, kind, d_in, d_phi,
                               torch.cuda.current_stream())
    torch.cuda.synchronize()
    return d_phi.double().cpu().numpy()


@pytest.mark.parametrize("prec,tol", [(32, 1e-5), (64, 1e-10)])
def test_direct_static_matches_slp_eval_on_consecutive_calls(prec, tol):
    slp = lib()
    torch = torch_cuda()
    V, T = meshes.icosphere(3)
    q = 7
    o = slp.slp_default_opts()
    o.precision = prec
    for d in range(3):
        o.grid[d] = 64
    plan = slp.slp_plan(V, T, q, tol, o)
    try:
        # two calls in a row with different states: stale scratch from the
        # first call must not leak into the second
        for seed in (11, 12):
            m = fields.vortex(V, seed)
            expect = run(slp, plan, slp.SLP_INPUT_NODAL_MAG, m, prec)  # existing entry point (slp_eval)
            got = _direct_static(slp, torch, V, T, q, prec, slp.SLP_INPUT_NODAL_MAG, m)
            assert np.all(np.isfinite(got))
            assert rel_l2(got, expect) <= tol, (seed, rel_l2(got, expect))
            # and directly against the FP64 oracle
            ref = oracle.slp_nodal(V, T, q, m)
            assert rel_l2(got, ref) <= tol, (seed, rel_l2(got, ref))
        # sigma input through the same scratch
        sigma = fields.random_sigma(T.shape[0] * q, 13)
        expect = run(slp, plan, slp.SLP_INPUT_SIGMA, sigma, prec)
        got = _direct_static(slp, torch, V, T, q, prec, slp.SLP_INPUT_SIGMA, sigma)
        assert rel_l2(got, expect) <= tol
        assert rel_l2(got, oracle.slp(V, T, q, oracle.KIND_SIGMA, sigma)) <= tol
    finally:
        slp.slp_destroy(plan)


def test_direct_static_fp32_at_the_source_limit():
    """A cube of 158 x 158 squares per face with the 7-point rule: 2,096,976
    sources, just under the 2,097,152 the FP32 scratch holds.  Each warp adds
    about 262,000 terms per target; the compensated sums keep the result
    within 1e-5 of the FP64 oracle at 256 seeded targets, on two calls in a
    row with different states."""
    slp = lib()
    torch = torch_cuda()
    V, T = meshes.cube(158)
    q = 7
    assert T.shape[0] * q <= (32 << 20) // 16
    y, _, _ = oracle.sources(V, T, q)
    sel = np.sort(np.random.default_rng(158).choice(V.shape[0], 256, replace=False))
    for seed in (21, 22):
        m = fields.smooth_random(V, seed)
        got = _direct_static(slp, torch, V, T, q, 32, slp.SLP_INPUT_NODAL_MAG, m)
        assert np.all(np.isfinite(got))
        qk = oracle.charges(V, T, q, oracle.KIND_NODAL_MAG, m)
        ref, _ = oracle.direct_subset(V, sel, y, qk)
        err = rel_l2(got[sel], ref)
        assert err <= 1e-5, (seed, err)


def test_direct_static_rejects_meshes_beyond_the_scratch():
    slp = lib()
    torch = torch_cuda()
    V, T = meshes.icosphere(1)
    d_V = torch.as_tensor(V, dtype=torch.float64, device="cuda")
    d_T = torch.as_tensor(T, dtype=torch.int32, device="cuda")
    d_in = torch.zeros(V.shape[0] * 3, dtype=torch.float32, device="cuda")
    d_phi = torch.zeros(V.shape[0], dtype=torch.float32, device="cuda")
    # a triangle count whose sources exceed the 32 MiB array (checked on the
    # host before anything is launched; raw addresses skip the wrapper's
    # size checks so that the library's own check is the one exercised)
    too_many = (32 << 20) // 16 // 7 + 1
    with pytest.raises(slp.SlpError) as e:
        slp.slp_eval_direct_static(d_V.data_ptr(), V.shape[0], d_T.data_ptr(), too_many, 7, 32,
                                   slp.SLP_INPUT_NODAL_MAG, d_in.data_ptr(), d_phi.data_ptr(), None)
    assert e.value.status == slp.SLP_ERR_INVALID_ARG
    assert "scratch" in slp.slp_last_error()


def test_direct_static_wrapper_checks_tensors():
    slp = lib()
    torch = torch_cuda()
    V, T = meshes.icosphere(1)
    d_V = torch.as_tensor(V, dtype=torch.float64, device="cuda")
    d_T = torch.as_tensor(T, dtype=torch.int32, device="cuda")
    d_phi = torch.zeros(V.shape[0], dtype=torch.float32, device="cuda")
    bad = [torch.zeros(V.shape[0] * 3, dtype=torch.float64, device="cuda"),   # wrong dtype
           torch.zeros(V.shape[0] * 3 - 1, dtype=torch.float32, device="cuda"),  # too short
           torch.zeros(V.shape[0] * 3, dtype=torch.float32)]                   # host tensor
    for d_in in bad:
        with pytest.raises(slp.SlpError) as e:
            slp.slp_eval_direct_static(d_V, V.shape[0], d_T, T.shape[0], 3, 32, slp.SLP_INPUT_NODAL_MAG, d_in, d_phi)
        assert e.value.status == slp.SLP_ERR_INVALID_ARG
