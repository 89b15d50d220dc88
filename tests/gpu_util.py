"""Shared helpers of the GPU tests: library loading and device round trips."""
from __future__ import annotations

import numpy as np


def lib():
    import paper_1305_3162_gb300 as slp
    from paper_1305_3162_gb300 import _build
    _build.build()
    slp.load()
    return slp


def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("CUDA device required")
    return torch


def to_dev(a, prec):
    torch = torch_cuda()
    dt = torch.float64 if prec == 64 else torch.float32
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def run(slp, plan, kind, data, prec, last_stage=None):
    """Evaluate (or run up to a stage) on the current stream; returns phi (numpy, user order)."""
    torch = torch_cuda()
    d_in = to_dev(data, prec)
    dt = torch.float64 if prec == 64 else torch.float32
    info = slp.slp_query(plan)
    d_phi = torch.zeros(info["n_targets"], dtype=dt, device="cuda")
    if last_stage is None:
        slp.slp_eval(plan, kind, d_in, d_phi, torch.cuda.current_stream())
    else:
        slp.slp_debug_run(plan, kind, d_in, d_phi, torch.cuda.current_stream(), last_stage)
    torch.cuda.synchronize()
    slp.slp_check(plan)
    return d_phi.double().cpu().numpy()


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
