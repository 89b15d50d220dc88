"""The allocation-free entry point slp_eval_direct_static.

It serves callers that cannot call cudaMalloc where they need the potential
(a stream being captured into a CUDA graph, a host inside another
framework's memory pool, a loop that must not touch the allocator after
start-up).  It must give the same potential as slp_eval, within the
tolerance the other tests use, call after call, although every call
reuses the same static scratch array inside the library.

This file is collected last on purpose, so that a run that stops at the
first failure has already run every other test.
"""
import numpy as np
import pytest

from synthetic import fields, meshes
from tests.gpu_util import lib, rel_l2, run, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol", [(32, 1e-5), (64, 1e-10)])
def test_direct_static_matches_slp_eval_on_consecutive_calls(prec, tol):
    slp = lib()
    torch = torch_cuda()
    dt = torch.float64 if prec == 64 else torch.float32
    V, T = meshes.icosphere(3)
    q = 7
    o = slp.slp_default_opts()
    o.precision = prec
    for d in range(3):
        o.grid[d] = 64
    plan = slp.slp_plan(V, T, q, tol, o)
    try:
        d_V = torch.as_tensor(V, dtype=torch.float64, device="cuda")
        d_T = torch.as_tensor(T, dtype=torch.int32, device="cuda")
        stream = torch.cuda.current_stream()
        # two calls in a row with different states: stale scratch from the
        # first call must not leak into the second
        for seed in (11, 12):
            m = fields.vortex(V, seed)
            expect = run(slp, plan, slp.SLP_INPUT_NODAL_MAG, m, prec)  # existing entry point (slp_eval)
            d_m = torch.as_tensor(m, dtype=dt, device="cuda")
            d_phi = torch.full((V.shape[0],), float("nan"), dtype=dt, device="cuda")
            slp.slp_eval_direct_static(d_V, V.shape[0], d_T, T.shape[0], q, prec, slp.SLP_INPUT_NODAL_MAG, d_m,
                                       d_phi, stream)
            torch.cuda.synchronize()
            got = d_phi.double().cpu().numpy()
            assert np.all(np.isfinite(got))
            assert rel_l2(got, expect) <= tol, (seed, rel_l2(got, expect))
        # sigma input through the same scratch
        sigma = fields.random_sigma(T.shape[0] * q, 13)
        expect = run(slp, plan, slp.SLP_INPUT_SIGMA, sigma, prec)
        d_s = torch.as_tensor(sigma, dtype=dt, device="cuda")
        d_phi = torch.empty(V.shape[0], dtype=dt, device="cuda")
        slp.slp_eval_direct_static(d_V, V.shape[0], d_T, T.shape[0], q, prec, slp.SLP_INPUT_SIGMA, d_s, d_phi, stream)
        torch.cuda.synchronize()
        assert rel_l2(d_phi.double().cpu().numpy(), expect) <= tol
    finally:
        slp.slp_destroy(plan)


def test_direct_static_rejects_meshes_beyond_the_scratch():
    slp = lib()
    torch = torch_cuda()
    V, T = meshes.icosphere(1)
    d_V = torch.as_tensor(V, dtype=torch.float64, device="cuda")
    d_T = torch.as_tensor(T, dtype=torch.int32, device="cuda")
    d_in = torch.zeros(V.shape[0] * 3, dtype=torch.float32, device="cuda")
    d_phi = torch.zeros(V.shape[0], dtype=torch.float32, device="cuda")
    # a triangle count whose sources exceed the 32 MiB array (checked on the
    # host before anything is launched)
    too_many = (32 << 20) // 16 // 7 + 1
    with pytest.raises(slp.SlpError) as e:
        slp.slp_eval_direct_static(d_V, V.shape[0], d_T, too_many, 7, 32, slp.SLP_INPUT_NODAL_MAG, d_in, d_phi, None)
    assert e.value.status == slp.SLP_ERR_INVALID_ARG
    assert "scratch" in slp.slp_last_error()
