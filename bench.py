#!/usr/bin/env python
"""Benchmark of the single-layer-potential evaluation (slp_eval) on GB300.

Workload (default): sphere of radius 1, icosahedron refined 5 times (20480
triangles, 10242 boundary nodes), 7-point rule (143360 sources), seeded
vortex magnetisation at the nodes, oversampled grid 128^3, FP32, plan
tolerance 1e-5.  One step = one slp_eval of one magnetisation state (the
whole hot path: charges, spread, pruned FFT, kernel multiply, inverse FFT,
gather, near field).  Eight seeded states are resident in HBM and cycled.

Metric: boundary targets per second, counted only when the result of every
checked state is within rel-L2 1e-5 of the FP64 direct-sum oracle.

Timing: W warm-up steps, then K timed steps.  The working set (8 MB grid,
~10 MB of plan data) fits in the 129 MB L2, so L2 is flushed before every
step by writing a 512 MB buffer; each step is bracketed by CUDA events on
the launch stream and the K event intervals are summed.  A barrier and
torch.cuda.synchronize() bracket the timed loop; the max over ranks is
reported.  N > 1 GPUs run independent replicas (the evaluation does not
shard), so scaling is weak.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

`--impl reference` times the FP64 oracle (plain C direct sum, OpenMP) on the
host cores instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "SLP boundary targets/s at rel-L2 <=1e-5 vs FP64 oracle"
UNIT = "targets/s"
N_STATES = 8
FLUSH_BYTES = 512 << 20
PARITY_FULL_MAX = 60000   # larger meshes: parity at PARITY_SAMPLE seeded targets
PARITY_SAMPLE = 512
NEAR_FLOPS_PER_PAIR = 30  # FP32 operations per (target, source) pair inside eps, erfc included


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _max_over_ranks(dist, seconds, device="cuda"):
    """Largest of the ranks' timed regions (the whole-job time of N replicas)."""
    if not dist:
        return seconds
    import torch
    t = torch.tensor([seconds], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _throughput(n_targets, steps, world_size, seconds):
    """Whole-job targets/s: every rank evaluates `steps` states of n_targets."""
    return n_targets * steps * world_size / seconds


def _workload(name):
    from synthetic import workloads
    if name == "sphere":
        return workloads.sphere()
    if name == "cube":
        return workloads.cube()
    if name == "plate":
        return workloads.plate()
    if name == "cube400":
        return workloads.cube_large()
    if name == "cube100":  # a 512^3 grid: the large-grid kernels at a size ncu can capture
        return workloads.cube_large(nper=100, grid=(512, 512, 512))
    raise ValueError(name)


def _states(w, n):
    from synthetic import fields
    if w.name.startswith("sphere"):
        return [fields.vortex(w.V, w.seed + 1000 * i) for i in range(n)]
    return [fields.smooth_random(w.V, w.seed + 1000 * i) for i in range(n)]


def _algorithmic(info, stage, w, pairs_within):
    """Algorithmic bytes (or FLOPs) of one launch of `stage` (FP32 model)."""
    es = 4 if info["precision"] == 32 else 8
    L = info["grid"]
    n = info["modes"]
    G = L[0] * L[1] * L[2]
    Kx = n[0] // 2
    N = info["n_targets"]
    Q = info["n_sources"]
    M = info["n_triangles"]
    # the FFT passes touch only the active rows (R of them, in Za planes)
    R = info["active_rows"]
    Za = info["active_planes"]
    ga = es * R * L[0]                # active rows of a real grid
    s1 = 2 * es * R * Kx              # active rows of S1 (complex [Lz][Ly][Kx])
    s2 = 2 * es * Za * n[1] * Kx      # active planes of S2 (complex [Lz][ny][Kx])
    table = {
        "charges": ("hbm", 3 * es * N + 3 * es * Q + 4 * Q + 32 * M),
        # the spread's floor is arithmetic: one multiply-add per (source, window point)
        "spread": ("alu", 2 * Q * (2 * info["m"]) ** 3),
        "fft_x": ("hbm", 2 * ga + s1),           # read A, write zeros back, write S1
        "fft_y": ("hbm", s1 + s2),
        "fft_xy": ("hbm", 2 * ga + s2),          # fused: read A, zeros back, write S2
        "fft_z_mul": ("hbm", 2 * s2 + es * n[2] * n[1] * Kx // 4),
        "ifft_y": ("hbm", s2 + s1),
        "ifft_x": ("hbm", s1 + ga),
        "ifft_yx": ("hbm", s2 + ga),             # fused: read S2, write grid B
        "gather": ("hbm", ga + 4 * es * N + 4 * N + es * N),
        "near": (("hbm", info["near_matrix_nnz"] * 4 * es + 8 * (N + 1) + 3 * es * N + 2 * es * N + 4 * N)
                 if info["near_mode"] == 2 else ("alu", NEAR_FLOPS_PER_PAIR * pairs_within)),
        "near_reduce": ("hbm", 0),
    }
    return table[stage]


def run_ours(args):
    import torch

    import paper_1305_3162_gb300 as slp
    from paper_1305_3162_gb300 import _build

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    else:
        dist = None
    assert torch.cuda.is_available(), "bench.py needs a CUDA device"
    _build.build()
    dev = torch.cuda.current_device()
    w = _workload(args.workload)
    plan = slp.Plan(w.V, w.T, quadrature=w.quad, tolerance=w.tolerance, precision=w.precision, grid=w.grid,
                    device=dev)
    info = plan.info
    dt = torch.float32 if w.precision == 32 else torch.float64
    states = _states(w, N_STATES)
    d_states = [torch.as_tensor(s, dtype=dt, device="cuda") for s in states]
    d_phi = torch.empty(w.n_targets, dtype=dt, device="cuda")
    stream = torch.cuda.current_stream()
    kind = slp.SLP_INPUT_NODAL_MAG

    # ---- parity gate (FP64 oracle on the host) for two of the states; large
    # meshes at PARITY_SAMPLE seeded targets
    import oracle
    errs = []
    sel = None
    if w.n_targets > PARITY_FULL_MAX:
        rng = np.random.default_rng(w.seed)
        sel = np.sort(rng.choice(w.n_targets, PARITY_SAMPLE, replace=False))
        y_src, _, _ = oracle.sources(w.V, w.T, w.quad)
    for i in (0, N_STATES - 1):
        plan.eval(kind, d_states[i], d_phi, stream)
        torch.cuda.synchronize()
        slp.slp_check(plan.handle)
        phi = d_phi.double().cpu().numpy()
        if sel is None:
            ref = oracle.slp_nodal(w.V, w.T, w.quad, states[i])
        else:
            qk = oracle.charges(w.V, w.T, w.quad, 2, states[i])
            ref, _ = oracle.direct_subset(w.V, sel, y_src, qk)
            phi = phi[sel]
        errs.append(float(np.linalg.norm(phi - ref) / np.linalg.norm(ref)))
    rel_l2 = max(errs)
    parity_ok = rel_l2 <= w.tolerance

    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    # ---- warm-up
    for i in range(args.warmup):
        flush.fill_(float(i))
        plan.eval(kind, d_states[i % N_STATES], d_phi, stream)
    torch.cuda.synchronize()

    # ---- timed region
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    sampler = ClockSampler(dev)
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))
        ev0[i].record(stream)
        plan.eval(kind, d_states[i % N_STATES], d_phi, stream)
        ev1[i].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    total_s = _max_over_ranks(dist, sum(step_ms) / 1e3)
    value = _throughput(w.n_targets, args.steps, ws, total_s)

    # ---- per-kernel durations (CUDA events on the launch stream, after an L2 flush)
    prof = {}
    for r in range(max(5, min(args.steps, 20))):
        flush.fill_(float(r))
        d = slp.slp_debug_profile(plan.handle, kind, d_states[r % N_STATES], d_phi, stream)
        for k, v in d.items():
            prof.setdefault(k, []).append(v)
    prof_ms = {k: statistics.median(v) for k, v in prof.items()}
    if info.get("fused_plane_passes"):
        # the fused plane passes fill the x slots; the y slots stay empty
        prof_ms["fft_xy"] = prof_ms.pop("fft_x", 0.0) + prof_ms.pop("fft_y", 0.0)
        prof_ms["ifft_yx"] = prof_ms.pop("ifft_y", 0.0) + prof_ms.pop("ifft_x", 0.0)

    # pairs inside eps (host, plan geometry; for the near-field work model)
    from scipy.spatial import cKDTree
    y = slp.slp_query_points(plan.handle, w.n_sources)
    cnt = cKDTree(y).query_ball_point(w.V, info["eps_near"], return_length=True, workers=-1)
    pairs_within = int(np.sum(cnt))

    dom = max((k for k in prof_ms if prof_ms[k] > 0), key=lambda k: prof_ms[k])
    peaks, peak_src = _peaks()
    bound, work = _algorithmic(info, dom, w, pairs_within)
    dom_s = prof_ms[dom] / 1e3
    if bound == "hbm":
        achieved = work / dom_s / 1e9
        peak = float(peaks["hbm_gbs"])
        unit = "GB/s"
    else:
        achieved = work / dom_s / 1e12
        mhz = float(peaks.get("sm_max_mhz", 2070.0))
        peak = 152 * 128 * 2 * mhz * 1e6 / 1e12  # FP32 FMA lanes x 2 flops x clock
        unit = "TFLOP/s"
    traffic = None
    tr_path = os.path.join(ROOT, "profiles", f"dram_traffic_{w.name}_fp{w.precision}.txt")
    if os.path.exists(tr_path):
        with open(tr_path) as f:
            tr = json.load(f)
        ent = tr.get(args.workload, {}).get(dom)
        if ent and ent.get("source_hash") == _kernel_source_hash():
            traffic = ent.get("bytes_per_launch")
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
                "traffic": traffic, "kernel": dom, "kernel_ms": prof_ms[dom],
                "peak_source": ("sm_max_mhz of " if bound == "alu" else "") + peak_src}
    hbm_peak = float(peaks["hbm_gbs"])
    per_kernel = {}
    for k, v in prof_ms.items():
        if v <= 0:
            continue
        b, wk = _algorithmic(info, k, w, pairs_within)
        per_kernel[k] = {"ms": round(v, 5), "bound": b,
                         ("gbs" if b == "hbm" else "tflops"): round(wk / (v / 1e3) / (1e9 if b == "hbm" else 1e12), 2)}
        if b == "hbm":
            per_kernel[k]["hbm_frac"] = round(wk / (v / 1e3) / 1e9 / hbm_peak, 4)

    # ---- end to end through the host-buffer entry point (pinned memory)
    h_in = [torch.as_tensor(s, dtype=dt).pin_memory() for s in states]
    h_out = torch.empty(w.n_targets, dtype=dt).pin_memory()
    for i in range(3):
        slp.slp_eval_host(plan.handle, kind, h_in[i % N_STATES], h_out, stream)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    te0 = time.perf_counter()
    for i in range(args.steps):
        slp.slp_eval_host(plan.handle, kind, h_in[i % N_STATES], h_out, stream)
    torch.cuda.synchronize()
    te = _max_over_ranks(dist, time.perf_counter() - te0)
    es = 4 if w.precision == 32 else 8
    e2e = {"value": _throughput(w.n_targets, args.steps, ws, te), "unit": UNIT,
           "h2d_bytes_per_step": 3 * es * w.n_targets, "d2h_bytes_per_step": es * w.n_targets}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = _cpu_baseline(w, states[0], args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value if parity_ok else 0.0, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_s * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if w.precision == 32 else "f64", "data": "synthetic (seeded meshes and magnetisations)",
            "config": {"workload": f"{w.name}_q{w.quad}_grid{'x'.join(map(str, w.grid))}_fp{w.precision}",
                       "n_targets": w.n_targets, "n_sources": w.n_sources, "grid": info["grid"], "m": info["m"],
                       "input": "nodal magnetisation", "states": N_STATES, "tolerance": w.tolerance,
                       "l2_flush": f"{FLUSH_BYTES >> 20} MB write before every step",
                       "parallelism": "replicas" if ws > 1 else "single GPU",
                       "eps_near": info["eps_near"], "pairs_within_eps": pairs_within,
                       "near_pairs_visited": info["near_pairs"], "near_mode": ["auto", "on_the_fly", "precomputed"][info["near_mode"]],
                       "near_matrix_nnz": info["near_matrix_nnz"],
                       "gather_item_targets": info.get("gather_item_targets"),
                       "spread_blocks_per_sm": info.get("spread_blocks_per_sm"),
                       "fft_passes": ("fused plane" if info.get("fused_plane_passes") else
                                      "fused column" if info.get("fused_column_passes") else "separate")},
            "rel_l2": rel_l2, "parity_ok": parity_ok,
            "roofline": roofline, "per_kernel": per_kernel,
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": info["launches_per_eval"] * args.steps,
            "wall_s_timed_loop": wall,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if dist:
        dist.destroy_process_group()


def _kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1305_3162_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _cpu_baseline(w, m_nodal, seconds):
    """The FP64 oracle (plain C, all host cores) on the full workload, repeated
    until about `seconds` of CPU time have elapsed."""
    import oracle
    y, _, _ = oracle.sources(w.V, w.T, w.quad)
    qk = oracle.charges(w.V, w.T, w.quad, oracle.KIND_NODAL_MAG, m_nodal)
    reps = 0
    t0 = time.perf_counter()
    used = 0
    while True:
        _, used = oracle.direct(w.V, y, qk)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds or reps >= 1000:
            break
    return {"value": w.n_targets * reps / el, "unit": UNIT, "cores": int(used), "kind": "oracle",
            "sample": f"all {w.n_targets} targets x {w.n_sources} sources (direct sum), {reps} repetitions, "
                      f"{el:.1f} s"}


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return
    w = _workload(args.workload)
    from synthetic import fields  # noqa: F401
    states = _states(w, N_STATES)
    import oracle
    y, _, _ = oracle.sources(w.V, w.T, w.quad)
    qks = [oracle.charges(w.V, w.T, w.quad, oracle.KIND_NODAL_MAG, s) for s in states]
    # each step: the direct sum on a bounded sample of targets (all of them when
    # that fits the per-step budget), timed on the host cores
    n_sel = w.n_targets
    pairs = w.n_targets * w.n_sources
    if pairs > 3e9:
        n_sel = max(256, int(3e9 // w.n_sources))
    rng = np.random.default_rng(w.seed)
    sel = np.sort(rng.choice(w.n_targets, n_sel, replace=False)) if n_sel < w.n_targets else np.arange(w.n_targets)
    used = 1
    for i in range(args.warmup):
        _, used = oracle.direct_subset(w.V, sel, y, qks[i % N_STATES])
    t0 = time.perf_counter()
    for i in range(args.steps):
        _, used = oracle.direct_subset(w.V, sel, y, qks[i % N_STATES])
    el = time.perf_counter() - t0
    value = n_sel * args.steps / el
    sample = f"{n_sel} of {w.n_targets} targets x {w.n_sources} sources per step (direct sum)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded meshes and magnetisations)",
            "config": {"workload": f"{w.name}_q{w.quad}_grid{'x'.join(map(str, w.grid))}_fp{w.precision}",
                       "n_targets": w.n_targets, "n_sources": w.n_sources},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": int(used), "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _batched_workload():
    """64 seeded smooth states on the level-5 sphere, plus 16 meshes of uneven
    size (cubes, spheres, plates; ~1.2k to ~200k triangles) with 4 states each."""
    from synthetic import fields, meshes
    items = []
    V, T = meshes.icosphere(5)
    items.append(("sphere_L5", V, T, 7, (128, 128, 128), [fields.smooth_random(V, 7000 + i) for i in range(64)]))
    shapes = [("cube10", meshes.cube(10), 3), ("cube20", meshes.cube(20), 3), ("cube40", meshes.cube(40), 3),
              ("cube70", meshes.cube(70), 3), ("cube100", meshes.cube(100), 3), ("cube128", meshes.cube(128), 3),
              ("sphere_L3", meshes.icosphere(3), 7), ("sphere_L4", meshes.icosphere(4), 7),
              ("sphere_L5b", meshes.icosphere(5, 2.0), 3), ("sphere_L6", meshes.icosphere(6), 3),
              ("sphere_L4b", meshes.icosphere(4, 0.5), 3),
              ("plate_a", meshes.box(400.0, 100.0, 4.0, 40, 10, 2), 3),
              ("plate_b", meshes.box(1000.0, 250.0, 10.0, 100, 25, 2), 3),
              ("plate_c", meshes.box(2000.0, 500.0, 20.0, 200, 50, 2), 3),
              ("plate_d", meshes.box(1000.0, 1000.0, 20.0, 150, 150, 3), 3),
              ("plate_e", meshes.box(2000.0, 500.0, 20.0, 300, 75, 3), 3)]
    for k, (name, (V, T), q) in enumerate(shapes):
        items.append((name, V, T, q, None, [fields.smooth_random(V, 8000 + 10 * k + i) for i in range(4)]))
    return items


def run_batched(args):
    """Batched form: every (mesh, state) evaluation in one CUDA graph, against
    the same evaluations issued one at a time on one stream."""
    import torch

    import oracle
    import paper_1305_3162_gb300 as slp
    from paper_1305_3162_gb300 import _build
    _build.build()
    work = _batched_workload()
    plans, tune, plan_of, d_in, d_out, states, n_targets = [], [], [], [], [], [], 0
    t_plan = time.perf_counter()
    for pi, (name, V, T, q, grid, sts) in enumerate(work):
        o = slp.slp_default_opts()
        o.precision = 32
        if grid is not None:
            for d in range(3):
                o.grid[d] = grid[d]
            plans.append(slp.slp_plan(V, T, q, 1e-5, o))
            tune.append({"mesh": name, "grid": list(grid), "autotuned": False})
        else:
            h, rec = slp.slp_plan_autotune(V, T, q, 1e-5, o, reps=3)
            plans.append(h)
            c = rec["candidates"][rec["chosen"]]
            tune.append({"mesh": name, "grid": c["grid"], "ms": round(c["ms"], 4), "autotuned": True,
                         "kernel_mode": c["kernel_mode"], "candidates": len(rec["candidates"])})
        for m in sts:
            plan_of.append(pi)
            d_in.append(torch.as_tensor(m, dtype=torch.float32, device="cuda"))
            d_out.append(torch.empty(V.shape[0], dtype=torch.float32, device="cuda"))
            states.append((pi, m))
            n_targets += V.shape[0]
    t_plan = time.perf_counter() - t_plan
    stream = torch.cuda.current_stream()
    batch = slp.slp_batch_create(plans, plan_of, slp.SLP_INPUT_NODAL_MAG, d_in, d_out, lanes_per_plan=args.lanes)
    bq = slp.slp_batch_query(batch)
    # parity: one state per mesh at up to 512 sampled targets (FP64 oracle)
    slp.slp_batch_run(batch, stream)
    torch.cuda.synchronize()
    worst = 0.0
    per_mesh = {}
    seen = set()
    for k, (pi, m) in enumerate(states):
        if pi in seen:
            continue
        seen.add(pi)
        name, V, T, q, _, _ = work[pi]
        rng = np.random.default_rng(pi)
        sel = np.sort(rng.choice(V.shape[0], min(512, V.shape[0]), replace=False))
        y, _, _ = oracle.sources(V, T, q)
        qk = oracle.charges(V, T, q, oracle.KIND_NODAL_MAG, m)
        ref, _ = oracle.direct_subset(V, sel, y, qk)
        got = d_out[k].double().cpu().numpy()[sel]
        err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        per_mesh[name] = err
        worst = max(worst, err)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def timed(fn, reps):
        ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
        ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
        for i in range(reps):
            flush.fill_(float(i))
            ev0[i].record(stream)
            fn()
            ev1[i].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in zip(ev0, ev1)) / reps

    def one_at_a_time():
        for (pi, _), a, b in zip(states, d_in, d_out):
            slp.slp_eval(plans[pi], slp.SLP_INPUT_NODAL_MAG, a, b, stream)

    for _ in range(args.warmup):
        slp.slp_batch_run(batch, stream)
        one_at_a_time()
    torch.cuda.synchronize()
    ms_batch = timed(lambda: slp.slp_batch_run(batch, stream), args.steps)
    ms_plain = timed(one_at_a_time, args.steps)
    line = {"metric": METRIC + " (batched form)", "value": n_targets / (ms_batch / 1e3), "unit": UNIT,
            "mode": "batched", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_batch,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic (seeded meshes and magnetisations)",
            "config": {"workload": "64 states on sphere L5 + 16 meshes x 4 states", "items": len(states),
                       "targets_per_step": n_targets, "lanes_per_plan": args.lanes, "graph": bq,
                       "l2_flush": f"{FLUSH_BYTES >> 20} MB write before every step", "plans_s": round(t_plan, 2),
                       "tuning": tune},
            "rel_l2_worst_sampled": worst, "parity_ok": worst <= 1e-5,
            "rel_l2_sampled_per_mesh": per_mesh,
            "one_at_a_time": {"value": n_targets / (ms_plain / 1e3), "ms_per_step": ms_plain},
            "speedup_vs_one_at_a_time": ms_plain / ms_batch}
    print(json.dumps(line), flush=True)
    slp.slp_batch_destroy(batch)
    for p in plans:
        slp.slp_destroy(p)


def _served_pool():
    """Eight resident meshes (cube, sphere, plate, torus), ~2k to 1.92M triangles."""
    from synthetic import meshes
    return [("cube13", meshes.cube(13), 3, (64, 64, 64)),
            ("sphere_L5", meshes.icosphere(5), 7, (128, 128, 128)),
            ("plate_2000x500x20_c10", meshes.box(2000.0, 500.0, 20.0, 200, 50, 2), 3, (512, 128, 128)),
            ("torus_400x100", meshes.torus(2.0, 0.5, 400, 100), 3, (256, 256, 128)),
            ("sphere_L6", meshes.icosphere(6), 3, (256, 256, 256)),
            ("plate_2000x500x20_c5", meshes.box(2000.0, 500.0, 20.0, 400, 100, 4), 3, (512, 256, 256)),
            ("torus_800x200", meshes.torus(2.0, 0.5, 800, 200), 3, (512, 512, 256)),
            ("cube400", meshes.cube(400), 3, (1024, 1024, 1024))]


def run_served(args):
    """Served form: seeded Poisson arrivals (mean 2000 requests/s) over the eight
    resident meshes, 1..32 states per request, admission by an HBM budget."""
    import torch

    import oracle
    import paper_1305_3162_gb300 as slp
    from paper_1305_3162_gb300 import _build
    from synthetic import fields
    _build.build()
    pool = _served_pool()
    plans, info = [], []
    t0 = time.perf_counter()
    for name, (V, T), q, grid in pool:
        o = slp.slp_default_opts()
        o.precision = 32
        for d in range(3):
            o.grid[d] = grid[d]
        h = slp.slp_plan(V, T, q, 1e-5, o)
        plans.append(h)
        inf = slp.slp_query(h)
        info.append({"mesh": name, "triangles": int(T.shape[0]), "targets": int(V.shape[0]), "grid": inf["grid"],
                     "near": ["auto", "on_the_fly", "precomputed"][inf["near_mode"]],
                     "plan_gb": round(inf["bytes_device"] / 2 ** 30, 2)})
    t_plan = time.perf_counter() - t0
    # a pool of 32 seeded states per mesh, page-locked; a request takes a slice
    states = []
    for k, (name, (V, T), q, grid) in enumerate(pool):
        st = np.stack([fields.smooth_random(V, 9000 + 100 * k + j) for j in range(32)]).astype(np.float32)
        states.append(torch.from_numpy(st.reshape(32, -1)).pin_memory())
    rng = np.random.default_rng(fields.workload_seed(4))
    n_req = args.requests
    arrivals = np.cumsum(rng.exponential(1.0 / args.rate, size=n_req))
    which = rng.integers(0, len(pool), size=n_req)
    nst = rng.integers(1, 33, size=n_req)
    start = np.array([rng.integers(0, 33 - n) for n in nst])
    # outputs: a ring of 8 buffers of 32 states per mesh (the bench reads only the probes)
    rings = [[torch.empty(32 * V.shape[0], dtype=torch.float32).pin_memory() for _ in range(8)]
             for name, (V, T), q, grid in pool]
    so = slp.slp_server_default_opts()
    so.slots_per_plan = args.slots
    so.hbm_budget_bytes = int(args.budget_gb * 2 ** 30)
    server = slp.slp_server_create(plans, slp.SLP_INPUT_NODAL_MAG, so)
    # probes: one private request per mesh, before the stream, for parity
    probe_out = []
    for k, (name, (V, T), q, grid) in enumerate(pool):
        ho = torch.empty(V.shape[0], dtype=torch.float32).pin_memory()
        rid = slp.slp_server_submit(server, k, 1, states[k][0], ho)
        probe_out.append((rid, ho))
    for rid, _ in probe_out:
        slp.slp_server_wait(server, rid, 600.0)
    # the timed stream: submit each request at its arrival time (open loop)
    ids = []
    ring_pos = [0] * len(pool)
    tstart = time.perf_counter()
    for i in range(n_req):
        k = int(which[i])
        now = time.perf_counter() - tstart
        if arrivals[i] > now:
            time.sleep(arrivals[i] - now)
        ho = rings[k][ring_pos[k] % 8]
        ring_pos[k] += 1
        src = states[k][int(start[i])]
        ids.append(slp.slp_server_submit(server, k, int(nst[i]), src, ho))
    for rid in ids:
        slp.slp_server_wait(server, rid, 3600.0)
    wall = time.perf_counter() - tstart
    stats = slp.slp_server_stats(server)
    slp.slp_server_destroy(server)
    # the same requests one state at a time through the plain host-buffer entry
    # point (copy in, evaluate, copy out, synchronise), back to back
    stream = torch.cuda.current_stream()
    t1 = time.perf_counter()
    for i in range(n_req):
        k = int(which[i])
        nV = pool[k][1][0].shape[0]
        ho = rings[k][0]
        for j in range(int(nst[i])):
            src = states[k][int(start[i]) + j]
            slp.slp_eval_host(plans[k], slp.SLP_INPUT_NODAL_MAG, src, ho[j * nV:(j + 1) * nV], stream)
    torch.cuda.synchronize()
    wall_single = time.perf_counter() - t1
    # parity of the probes (oracle at up to 256 sampled nodes)
    errs = {}
    for k, (name, (V, T), q, grid) in enumerate(pool):
        sel = np.sort(np.random.default_rng(k).choice(V.shape[0], min(256, V.shape[0]), replace=False))
        y, _, _ = oracle.sources(V, T, q)
        m = states[k][0].numpy().reshape(-1, 3).astype(np.float64)
        qk = oracle.charges(V, T, q, oracle.KIND_NODAL_MAG, m)
        ref, _ = oracle.direct_subset(V, sel, y, qk)
        got = probe_out[k][1].numpy().astype(np.float64)[sel]
        errs[name] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    targets = int(sum(int(nst[i]) * pool[int(which[i])][1][0].shape[0] for i in range(n_req)))
    line = {"metric": METRIC + " (served form)", "value": targets / wall, "unit": UNIT, "mode": "served",
            "n_gpus": 1, "higher_is_better": True, "dtype": "f32", "data": "synthetic (seeded meshes and magnetisations)",
            "config": {"workload": "Poisson arrivals over 8 resident meshes", "rate_req_per_s": args.rate,
                       "requests": n_req, "states_per_request": "uniform 1..32", "slots_per_plan": args.slots,
                       "hbm_budget_gb": args.budget_gb, "plans_s": round(t_plan, 1), "meshes": info},
            "latency_p50_ms": stats["latency_p50_ms"], "latency_p99_ms": stats["latency_p99_ms"],
            "queue_wait_p50_ms": stats["queue_wait_p50_ms"], "queue_wait_p99_ms": stats["queue_wait_p99_ms"],
            "wall_s": wall, "server": stats, "probe_rel_l2_sampled": errs,
            "parity_ok": max(errs.values()) <= 1e-5,
            "one_at_a_time": {"value": targets / wall_single, "wall_s": wall_single,
                              "path": "slp_eval_host per state, same requests, back to back"},
            "speedup_vs_one_at_a_time": wall_single / wall}
    print(json.dumps(line), flush=True)
    for p in plans:
        slp.slp_destroy(p)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="sphere", choices=["sphere", "cube", "plate", "cube400", "cube100"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--mode", choices=["plain", "batched", "served"], default="plain",
                    help="plain: the headline single evaluation; batched/served: the other forms")
    ap.add_argument("--lanes", type=int, default=1,
                    help="batched form: concurrent scratch sets per plan (a lane batches its states itself)")
    ap.add_argument("--slots", type=int, default=1, help="served form: concurrent request slots per plan")
    ap.add_argument("--rate", type=float, default=2000.0, help="served form: mean arrivals per second")
    ap.add_argument("--requests", type=int, default=400, help="served form: requests in the arrival stream")
    ap.add_argument("--budget-gb", type=float, default=48.0, help="served form: HBM budget of the server")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "batched":
        run_batched(args)
    elif args.mode == "served":
        run_served(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
