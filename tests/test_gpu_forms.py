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
    """The tuner times two grids, then one knob at a time (window tables,
    spread occupancy, gather item size, FFT pass arrangement); the plan it
    returns is the fastest candidate it timed (within the 1 % a change must
    gain to be kept), carries that candidate's settings, and meets the
    tolerance against the oracle."""
    slp = lib()
    V, T = meshes.icosphere(4)
    o = slp.slp_default_opts()
    o.precision = 32
    plan, rec = slp.slp_plan_autotune(V, T, 7, 1e-5, o, reps=3)
    try:
        cands = rec["candidates"]
        assert len(cands) >= 5
        ms = [c["ms"] for c in cands if c["ms"] > 0]
        # an alternative replaces the incumbent only when faster by more than 1 %
        assert cands[rec["chosen"]]["ms"] <= 1.01 * min(ms)
        # every knob took more than one value among the candidates (a fused FFT
        # arrangement the grid cannot use is not timed)
        for knob in ("spread_table", "spread_blocks", "gather_item_targets"):
            assert len({c[knob] for c in cands}) >= 2, knob
        info = slp.slp_query(plan)
        c = cands[rec["chosen"]]
        assert info["grid"] == c["grid"]
        assert info["spread_table"] == c["spread_table"] and info["gather_item_targets"] == c["gather_item_targets"]
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


def test_eval_batched_one_call_matches_individual_evaluations():
    """slp_eval_batched: every state of every entry equals slp_eval on it; a
    second call with the same buffers (refilled in place) replays the cached
    graph with the new inputs; a plan may appear in two entries."""
    slp = lib()
    torch = torch_cuda()
    meshes_ = [(*meshes.icosphere(3), 7, (64, 64, 64)), (*meshes.cube(6), 3, (64, 64, 64))]
    plans = [_plan(slp, V, T, q, 1e-5, 32, g) for V, T, q, g in meshes_]
    try:
        entries = [(0, 3), (1, 5), (0, 2)]  # (plan, states)
        d_in, d_out = [], []
        for pi, ns in entries:
            V = meshes_[pi][0]
            d_in.append(torch.empty(ns * 3 * V.shape[0], dtype=torch.float32, device="cuda"))
            d_out.append(torch.empty(ns * V.shape[0], dtype=torch.float32, device="cuda"))
        for rep in range(2):
            states = []
            for e, (pi, ns) in enumerate(entries):
                V = meshes_[pi][0]
                ms = [fields.smooth_random(V, 1000 * rep + 10 * e + k) for k in range(ns)]
                states.append(ms)
                d_in[e].copy_(torch.as_tensor(np.concatenate([m.ravel() for m in ms]), dtype=torch.float32))
                d_out[e].fill_(float("nan"))
            slp.slp_eval_batched([plans[pi] for pi, _ in entries], slp.SLP_INPUT_NODAL_MAG, d_in, d_out,
                                 [ns for _, ns in entries], torch.cuda.current_stream())
            torch.cuda.synchronize()
            for e, (pi, ns) in enumerate(entries):
                N = meshes_[pi][0].shape[0]
                got = d_out[e].double().cpu().numpy().reshape(ns, N)
                assert np.all(np.isfinite(got))
                for k in range(ns):
                    ref = run(slp, plans[pi], slp.SLP_INPUT_NODAL_MAG, states[e][k], 32)
                    assert rel_l2(got[k], ref) < 1e-6, (rep, e, k)
        V, T, q, _ = meshes_[1]
        ref = oracle.slp_nodal(V, T, q, states[1][4])
        assert rel_l2(d_out[1].double().cpu().numpy().reshape(5, -1)[4], ref) <= 1e-5
    finally:
        for p in plans:
            slp.slp_destroy(p)


@pytest.mark.parametrize("kind", ["nodal", "sigma"])
def test_checked_evaluation_reports_nonfinite_input(kind):
    """opts.check_finite: a NaN placed in the host input (no GPU fault is
    involved) is reported by slp_check as SLP_ERR_NONFINITE; the status is
    cleared by the report; a clean input then passes; without the option the
    same input is not reported."""
    slp = lib()
    torch = torch_cuda()
    V, T = meshes.icosphere(2)
    q = 7
    if kind == "nodal":
        k_in = slp.SLP_INPUT_NODAL_MAG
        clean = fields.vortex(V, 5).ravel()
    else:
        k_in = slp.SLP_INPUT_SIGMA
        clean = fields.random_sigma(T.shape[0] * q, 5)
    bad = clean.copy()
    bad[7] = np.nan
    for check in (1, 0):
        o = slp.slp_default_opts()
        o.precision = 32
        o.check_finite = check
        for d in range(3):
            o.grid[d] = 32
        plan = slp.slp_plan(V, T, q, 1e-5, o)
        try:
            d_phi = torch.empty(V.shape[0], dtype=torch.float32, device="cuda")
            d_bad = torch.as_tensor(bad, dtype=torch.float32, device="cuda")
            slp.slp_eval(plan, k_in, d_bad, d_phi, torch.cuda.current_stream())
            if check:
                with pytest.raises(slp.SlpError) as e:
                    slp.slp_check(plan)
                assert e.value.status == slp.SLP_ERR_NONFINITE
            else:
                slp.slp_check(plan)
            d_ok = torch.as_tensor(clean, dtype=torch.float32, device="cuda")
            slp.slp_eval(plan, k_in, d_ok, d_phi, torch.cuda.current_stream())
            slp.slp_check(plan)
            assert np.all(np.isfinite(d_phi.cpu().numpy()))
        finally:
            slp.slp_destroy(plan)


def test_batched_workload_full_item_list():
    """The whole batched workload (64 sphere states plus 16 uneven meshes x 4
    states, grids autotuned where the workload leaves them open) in one CUDA
    graph: every item equals slp_eval on it, and one state per mesh is within
    1e-5 of the FP64 oracle at up to 256 seeded targets."""
    from synthetic import workloads
    slp = lib()
    torch = torch_cuda()
    work = workloads.batched_items()
    plans, plan_of, d_in, d_out, states = [], [], [], [], []
    try:
        for pi, (name, V, T, q, grid, sts) in enumerate(work):
            o = slp.slp_default_opts()
            o.precision = 32
            if grid is not None:
                for d in range(3):
                    o.grid[d] = grid[d]
                plans.append(slp.slp_plan(V, T, q, 1e-5, o))
            else:
                h, _ = slp.slp_plan_autotune(V, T, q, 1e-5, o, reps=2)
                plans.append(h)
            for m in sts:
                plan_of.append(pi)
                states.append((pi, m))
                d_in.append(torch.as_tensor(m, dtype=torch.float32, device="cuda"))
                d_out.append(torch.full((V.shape[0],), float("nan"), dtype=torch.float32, device="cuda"))
        assert len(states) == 128
        batch = slp.slp_batch_create(plans, plan_of, slp.SLP_INPUT_NODAL_MAG, d_in, d_out)
        try:
            slp.slp_batch_run(batch, torch.cuda.current_stream())
            torch.cuda.synchronize()
            seen = set()
            for (pi, m), o in zip(states, d_out):
                got = o.double().cpu().numpy()
                assert np.all(np.isfinite(got))
                ref = run(slp, plans[pi], slp.SLP_INPUT_NODAL_MAG, m, 32)
                assert rel_l2(got, ref) < 1e-6, work[pi][0]
                if pi not in seen:
                    seen.add(pi)
                    name, V, T, q, _, _ = work[pi]
                    sel = np.sort(np.random.default_rng(pi).choice(V.shape[0], min(256, V.shape[0]), replace=False))
                    y, _, _ = oracle.sources(V, T, q)
                    qk = oracle.charges(V, T, q, oracle.KIND_NODAL_MAG, m)
                    ref_o, _ = oracle.direct_subset(V, sel, y, qk)
                    assert rel_l2(got[sel], ref_o) <= 1e-5, name
        finally:
            slp.slp_batch_destroy(batch)
    finally:
        for p in plans:
            slp.slp_destroy(p)
