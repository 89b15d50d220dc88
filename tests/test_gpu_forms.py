"""Batched form (many states and uneven meshes in one CUDA graph) and the
grid autotuner: results equal the one-at-a-time evaluation and the oracle."""
import numpy as np
import pytest

import oracle
from synthetic import fields, meshes
from tests.gpu_util import lib, rel_l2, run, torch_cuda

pytestmark = pytest.mark.gpu


def _plan(slp, V, T, q, tol, prec, grid):
    o = slp.slp_default_opts()
    o.precision = prec
    for d in range(3):
        o.grid[d] = grid[d]
    return slp.slp_plan(V, T, q, tol, o)


def test_batch_matches_individual_evaluations():
    slp = lib()
    torch = torch_cuda()
    meshes_ = [(*meshes.icosphere(3), 7, (64, 64, 64)), (*meshes.cube(6), 3, (64, 64, 64)),
               (*meshes.torus(2.0, 0.5, 48, 16), 3, (64, 64, 32))]
    plans = [_plan(slp, V, T, q, 1e-5, 32, g) for V, T, q, g in meshes_]
    try:
        plan_of, ins, outs, states = [], [], [], []
        for pi, (V, T, q, g) in enumerate(meshes_):
            for s in range(5):
                m = fields.smooth_random(V, 100 * pi + s)
                states.append((pi, m))
                plan_of.append(pi)
                ins.append(torch.as_tensor(m, dtype=torch.float32, device="cuda"))
                outs.append(torch.full((V.shape[0],), float("nan"), dtype=torch.float32, device="cuda"))
        batch = slp.slp_batch_create(plans, plan_of, slp.SLP_INPUT_NODAL_MAG, ins, outs, lanes_per_plan=2)
        try:
            q = slp.slp_batch_query(batch)
            assert q["n_items"] == 15 and q["n_lanes"] == 6 and q["kernel_launches"] > 0
            for rep in range(2):  # the graph can be relaunched
                for o in outs:
                    o.fill_(float("nan"))
                slp.slp_batch_run(batch, torch.cuda.current_stream())
                torch.cuda.synchronize()
                for (pi, m), o in zip(states, outs):
                    got = o.double().cpu().numpy()
                    assert np.all(np.isfinite(got))
                    ref = run(slp, plans[pi], slp.SLP_INPUT_NODAL_MAG, m, 32)
                    assert rel_l2(got, ref) < 1e-6
            # and against the oracle for one item per mesh
            for pi, (V, T, qq, g) in enumerate(meshes_):
                k = plan_of.index(pi)
                ref = oracle.slp_nodal(V, T, qq, states[k][1])
                assert rel_l2(outs[k].double().cpu().numpy(), ref) <= 1e-5
        finally:
            slp.slp_batch_destroy(batch)
    finally:
        for p in plans:
            slp.slp_destroy(p)


def test_autotuner_picks_a_feasible_fast_grid():
    slp = lib()
    V, T = meshes.icosphere(4)
    o = slp.slp_default_opts()
    o.precision = 32
    plan, rec = slp.slp_plan_autotune(V, T, 7, 1e-5, o, reps=3)
    try:
        cands = rec["candidates"]
        assert len(cands) >= 2
        ms = [c["ms"] for c in cands if c["ms"] > 0]
        assert cands[rec["chosen"]]["ms"] == min(ms)
        info = slp.slp_query(plan)
        assert info["grid"] == cands[rec["chosen"]]["grid"]
        m = fields.vortex(V, 3)
        phi = run(slp, plan, slp.SLP_INPUT_NODAL_MAG, m, 32)
        assert rel_l2(phi, oracle.slp_nodal(V, T, 7, m)) <= 1e-5
    finally:
        slp.slp_destroy(plan)


def test_eval_states_matches_single_evaluations():
    """slp_eval_states: 11 nodal states (a chunk of 8 sharing one pass over the
    near-field operator, then 3) give the results of 11 slp_eval calls; a
    sigma input (no shared pass) as well."""
    slp = lib()
    torch = torch_cuda()
    V, T = meshes.icosphere(3)
    plan = _plan(slp, V, T, 7, 1e-5, 32, (64, 64, 64))
    try:
        assert slp.slp_query(plan)["near_mode"] == slp.SLP_NEAR_PRECOMPUTED
        S = 11
        ms = np.stack([fields.smooth_random(V, 300 + k) for k in range(S)])
        d_in = torch.as_tensor(ms.reshape(-1), dtype=torch.float32, device="cuda")
        d_out = torch.full((S * V.shape[0],), float("nan"), dtype=torch.float32, device="cuda")
        slp.slp_eval_states(plan, slp.SLP_INPUT_NODAL_MAG, S, d_in, d_out)
        torch.cuda.synchronize()
        got = d_out.double().cpu().numpy().reshape(S, -1)
        for k in range(S):
            ref = run(slp, plan, slp.SLP_INPUT_NODAL_MAG, ms[k], 32)
            assert rel_l2(got[k], ref) < 1e-6, k
        assert rel_l2(got[9], oracle.slp_nodal(V, T, 7, ms[9])) <= 1e-5
        Q = T.shape[0] * 7
        sig = np.stack([fields.random_sigma(Q, 400 + k) for k in range(2)])
        d_sig = torch.as_tensor(sig.reshape(-1), dtype=torch.float32, device="cuda")
        d_out2 = torch.empty(2 * V.shape[0], dtype=torch.float32, device="cuda")
        slp.slp_eval_states(plan, slp.SLP_INPUT_SIGMA, 2, d_sig, d_out2)
        torch.cuda.synchronize()
        got2 = d_out2.double().cpu().numpy().reshape(2, -1)
        for k in range(2):
            assert rel_l2(got2[k], run(slp, plan, slp.SLP_INPUT_SIGMA, sig[k], 32)) < 1e-6
    finally:
        slp.slp_destroy(plan)


@pytest.mark.parametrize("prec,tol,fuse,fcol", [(32, 1e-5, 1, 0), (32, 1e-5, 0, 1), (64, 1e-10, 0, 1), (64, 1e-10, 0, 0)],
                         ids=["fp32-fused-plane", "fp32-fused-column", "fp64-fused-column", "fp64"])
def test_eval_states_fused_passes_and_fp64(prec, tol, fuse, fcol):
    """State-batched far field through the fused plane passes (FP32), the
    fused column passes (FP32, FP64) and the separate passes (FP64): 5
    states against single evaluations and the oracle."""
    slp = lib()
    torch = torch_cuda()
    V, T = meshes.icosphere(3)
    o = slp.slp_default_opts()
    o.precision = prec
    for d in range(3):
        o.grid[d] = 64
    o.fuse_plane_passes = fuse
    o.fuse_column_passes = fcol
    plan = slp.slp_plan(V, T, 7, tol, o)
    try:
        info = slp.slp_query(plan)
        assert info["fused_plane_passes"] == fuse
        assert info["fused_column_passes"] == fcol
        S = 5
        dt = torch.float64 if prec == 64 else torch.float32
        ms = np.stack([fields.smooth_random(V, 500 + k) for k in range(S)])
        d_in = torch.as_tensor(ms.reshape(-1), dtype=dt, device="cuda")
        d_out = torch.empty(S * V.shape[0], dtype=dt, device="cuda")
        slp.slp_eval_states(plan, slp.SLP_INPUT_NODAL_MAG, S, d_in, d_out)
        torch.cuda.synchronize()
        got = d_out.double().cpu().numpy().reshape(S, -1)
        for k in range(S):
            ref = run(slp, plan, slp.SLP_INPUT_NODAL_MAG, ms[k], prec)
            assert rel_l2(got[k], ref) < (1e-12 if prec == 64 else 1e-6), k
        assert rel_l2(got[2], oracle.slp_nodal(V, T, 7, ms[2])) <= tol
    finally:
        slp.slp_destroy(plan)
