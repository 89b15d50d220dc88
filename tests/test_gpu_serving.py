"""Served form: requests on resident plans, continuous batching, admission by
an HBM budget.  Each result must be the same alone and in a mix of
concurrent requests (within the FP32 tolerance), and match the oracle."""
import numpy as np
import pytest

import oracle
from synthetic import fields, meshes
from tests.gpu_util import lib, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu


def _plans(slp, deterministic=0):
    specs = [(*meshes.icosphere(3), 7, (64, 64, 64)), (*meshes.cube(10), 3, (64, 64, 64)),
             (*meshes.torus(2.0, 0.5, 48, 16), 3, (64, 64, 32))]
    plans = []
    for V, T, q, g in specs:
        o = slp.slp_default_opts()
        o.precision = 32
        o.deterministic = deterministic
        for d in range(3):
            o.grid[d] = g[d]
        plans.append(slp.slp_plan(V, T, q, 1e-5, o))
    return specs, plans


def _pinned(a):
    torch = torch_cuda()
    t = torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).pin_memory()
    return t


@pytest.mark.parametrize("deterministic", [0, 1], ids=["default", "deterministic"])
def test_result_same_alone_and_in_the_mix(deterministic):
    """The probe request alone and inside a mix of 40 concurrent requests:
    within 1e-6 by default (the tiled spread adds with atomics), bitwise
    equal with deterministic plans."""
    slp = lib()
    torch = torch_cuda()
    specs, plans = _plans(slp, deterministic)
    o = slp.slp_server_default_opts()
    o.slots_per_plan = 2
    o.hbm_budget_bytes = 1 << 30
    server = slp.slp_server_create(plans, slp.SLP_INPUT_NODAL_MAG, o)
    try:
        V0 = specs[0][0]
        probe = np.stack([fields.vortex(V0, 77), fields.vortex(V0, 78)])  # 2 states
        h_in = _pinned(probe.reshape(-1))
        h_alone = torch.zeros(2 * V0.shape[0], dtype=torch.float32).pin_memory()
        rid = slp.slp_server_submit(server, 0, 2, h_in, h_alone)
        assert slp.slp_server_wait(server, rid, 60.0) == slp.SLP_REQ_DONE
        alone = h_alone.numpy().astype(np.float64).copy()

        # the same request inside a mix of 40 concurrent requests on all meshes
        rng = np.random.default_rng(5)
        keep = []
        ids = []
        h_mix = torch.zeros(2 * V0.shape[0], dtype=torch.float32).pin_memory()
        for k in range(40):
            if k == 20:
                ids.append(("probe", slp.slp_server_submit(server, 0, 2, h_in, h_mix)))
                continue
            pi = int(rng.integers(0, 3))
            V = specs[pi][0]
            ns = int(rng.integers(1, 5))
            m = np.concatenate([fields.smooth_random(V, 1000 * k + j).reshape(-1) for j in range(ns)])
            hi = _pinned(m)
            ho = torch.zeros(ns * V.shape[0], dtype=torch.float32).pin_memory()
            keep.append((pi, ns, m, hi, ho))
            ids.append((len(keep) - 1, slp.slp_server_submit(server, pi, ns, hi, ho)))
        for tag, rid2 in ids:
            assert slp.slp_server_wait(server, rid2, 120.0) == slp.SLP_REQ_DONE
        mix = h_mix.numpy().astype(np.float64)
        assert rel_l2(mix, alone) <= 1e-6
        if deterministic:
            assert np.array_equal(mix, alone)
        st = slp.slp_server_stats(server)
        assert st["completed"] == 41 and st["rejected"] == 0
        assert st["max_inflight"] >= 2  # requests overlapped on the device
        assert st["latency_p99_ms"] >= st["latency_p50_ms"] > 0
        assert st["arena_peak_bytes"] <= st["arena_bytes"]
    finally:
        slp.slp_server_destroy(server)
    # results against the oracle, for the probe and for a few mix requests
    V, T, q, _ = specs[0]
    for j in range(2):
        ref = oracle.slp_nodal(V, T, q, probe[j])
        assert rel_l2(alone[j * V.shape[0]:(j + 1) * V.shape[0]], ref) <= 1e-5
    for pi, ns, m, hi, ho in keep[:6]:
        V, T, q, _ = specs[pi]
        ref = oracle.slp_nodal(V, T, q, m[:3 * V.shape[0]].reshape(-1, 3))
        assert rel_l2(ho.numpy()[:V.shape[0]].astype(np.float64), ref) <= 1e-5
    for p in plans:
        slp.slp_destroy(p)


def test_admission_by_budget_rejection_cancel_and_timeout():
    slp = lib()
    torch = torch_cuda()
    specs, plans = _plans(slp)
    o = slp.slp_server_default_opts()
    o.slots_per_plan = 1
    o.hbm_budget_bytes = 4 << 20  # no extra slot scratch: the whole budget is the request arena
    server = slp.slp_server_create(plans, slp.SLP_INPUT_NODAL_MAG, o)
    try:
        V = specs[0][0]
        nb = V.shape[0]
        # a request that can never fit 4 MiB: rejected at once
        big = 400
        h_big = torch.zeros(big * 3 * nb, dtype=torch.float32).pin_memory()
        o_big = torch.zeros(big * nb, dtype=torch.float32).pin_memory()
        rid = slp.slp_server_submit(server, 0, big, h_big, o_big)
        st, res = slp.slp_server_status(server, rid)
        assert st == slp.SLP_REQ_REJECTED and res == slp.SLP_ERR_OOM
        # many requests for one plan with one slot: they queue; cancel the last
        m = fields.vortex(V, 9).reshape(-1)
        hin = _pinned(np.tile(m, 8))
        outs, ids = [], []
        for k in range(12):
            ho = torch.zeros(8 * nb, dtype=torch.float32).pin_memory()
            outs.append(ho)
            ids.append(slp.slp_server_submit(server, 0, 8, hin, ho))
        state, _ = slp.slp_server_status(server, ids[-1])
        if state == slp.SLP_REQ_QUEUED:
            slp.slp_server_cancel(server, ids[-1])
            assert slp.slp_server_status(server, ids[-1])[0] == slp.SLP_REQ_CANCELLED
            ids = ids[:-1]
        # a host-side wait with a tiny limit on queued work reports a timeout
        with pytest.raises(slp.SlpError) as e:
            slp.slp_server_wait(server, ids[-1], 1e-6)
        assert e.value.status == slp.SLP_ERR_TIMEOUT
        for rid2 in ids:
            assert slp.slp_server_wait(server, rid2, 120.0) == slp.SLP_REQ_DONE
        first = outs[0].numpy().astype(np.float64)
        for ho in outs[1:len(ids)]:
            assert rel_l2(ho.numpy().astype(np.float64), first) <= 1e-6
        stats = slp.slp_server_stats(server)
        assert stats["rejected"] == 1 and stats["arena_peak_bytes"] <= stats["arena_bytes"]
    finally:
        slp.slp_server_destroy(server)
    for p in plans:
        slp.slp_destroy(p)
