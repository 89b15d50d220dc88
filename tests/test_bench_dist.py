"""The replica path of bench.py on CPU: two gloo ranks, each with its own
timed region; both must report the slower rank's time, and the whole-job
throughput counts the work of every rank."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench._dist() == (ws, rank, rank)
        local = 0.5 + rank  # rank 1 is slower
        t = bench._max_over_ranks(dist, local, device="cpu")
        v = bench._throughput(1000, 10, ws, t)
        out[rank] = (t, v)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_throughput():
    ws = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, ws, port, out)) for r in range(ws)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(ws):
        t, v = res[r]
        assert t == pytest.approx(1.5)
        assert v == pytest.approx(1000 * 10 * ws / 1.5)


def test_dominant_kernel_breaks_noise_ties_toward_hbm():
    """The roofline's kernel: the longest median, except that kernels within
    3 % of it count as a tie, which goes to an HBM-bound kernel; a clear
    winner is kept whatever its bound."""
    import bench
    bound = {"spread": "alu", "near": "hbm", "gather": "hbm", "fft_x": "hbm"}.get
    sphere = {"spread": 0.02458, "near": 0.02445, "gather": 0.0101, "fft_x": 0.0093}
    assert bench._dominant_kernel(sphere, bound) == "near"
    assert bench._dominant_kernel({**sphere, "near": 0.02470}, bound) == "near"
    cube_fp64 = {"spread": 0.0506, "near": 0.0120, "gather": 0.0101}
    assert bench._dominant_kernel(cube_fp64, bound) == "spread"
    assert bench._dominant_kernel({"gather": 0.010, "near": 0.0099, "spread": 0.0}, bound) == "gather"


def test_single_process_is_unchanged():
    import bench
    assert bench._max_over_ranks(None, 0.25) == 0.25
    assert bench._throughput(10, 4, 1, 2.0) == 20.0
