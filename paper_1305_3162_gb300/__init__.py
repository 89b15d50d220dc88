"""GB300 single-layer-potential library (NUFFT method of Exl & Schrefl).

Thin Python binding of the C ABI in ``include/slp.h``: the functions below
carry the same names as the C entry points and only marshal arguments
(numpy arrays for host data, torch CUDA tensors or raw device pointers for
device data, a CUDA stream handle).  Every step of an evaluation runs in the
library's own CUDA kernels; there is no CPU or PyTorch fallback: if the
compiled library is missing, loading raises.

Build the library with ``paper_1305_3162_gb300._build.build()`` (or
``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from ._build import LIB as _LIB_PATH

# ------------------------------------------------------------------ constants
SLP_OK = 0
SLP_ERR_INVALID_ARG = 1
SLP_ERR_MESH = 2
SLP_ERR_TOLERANCE_INFEASIBLE = 3
SLP_ERR_OOM = 4
SLP_ERR_CUDA = 5
SLP_ERR_TIMEOUT = 6
SLP_ERR_NONFINITE = 7
SLP_ERR_NO_DEVICE = 8
SLP_ERR_UNSUPPORTED = 9

SLP_QUAD_1, SLP_QUAD_3, SLP_QUAD_7 = 1, 3, 7
SLP_INPUT_SIGMA, SLP_INPUT_MAG, SLP_INPUT_NODAL_MAG, SLP_INPUT_ELEMENT = 0, 1, 2, 3
SLP_KERNEL_AUTO, SLP_KERNEL_RADIAL, SLP_KERNEL_SEPARABLE, SLP_KERNEL_EXPSUM = 0, 1, 2, 3
SLP_NEAR_AUTO, SLP_NEAR_ON_THE_FLY, SLP_NEAR_PRECOMPUTED = 0, 1, 2

SLP_STAGE_CHARGES, SLP_STAGE_SPREAD, SLP_STAGE_FFT_X, SLP_STAGE_FFT_Y, SLP_STAGE_FFT_Z = 0, 1, 2, 3, 4
SLP_STAGE_IFFT_Y, SLP_STAGE_IFFT_X, SLP_STAGE_GATHER, SLP_STAGE_NEAR = 5, 6, 7, 8
SLP_BUF_QBUF, SLP_BUF_GRID_A, SLP_BUF_GRID_B, SLP_BUF_S1, SLP_BUF_S2, SLP_BUF_DTAB = 0, 1, 2, 3, 4, 5
(SLP_HOST_SRC_PERM, SLP_HOST_TGT_PERM, SLP_HOST_SRC_GRID, SLP_HOST_TGT_GRID, SLP_HOST_SPREAD_ITEMS,
 SLP_HOST_GATHER_ITEMS, SLP_HOST_NEAR_ITEMS, SLP_HOST_NEAR_RANGES, SLP_HOST_DTAB, SLP_HOST_SRC_POINTS,
 SLP_HOST_TGT_POINTS, SLP_HOST_PLANE_ROWS, SLP_HOST_ACTIVE_Z, SLP_HOST_SPREAD_GROUPS,
 SLP_HOST_SPREAD_GROUP_OFF, SLP_HOST_EXPSUM) = range(16)


class SlpError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: status {status}: {detail}")
        self.status = status


# ------------------------------------------------------------------ structs
class slp_mesh(ctypes.Structure):
    _fields_ = [("vertices", ctypes.POINTER(ctypes.c_double)), ("n_vertices", ctypes.c_int64),
                ("triangles", ctypes.POINTER(ctypes.c_int32)), ("n_triangles", ctypes.c_int64)]


class slp_plan_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("grid", ctypes.c_int * 3), ("m", ctypes.c_int),
                ("kernel_mode", ctypes.c_int), ("near_mode", ctypes.c_int), ("deterministic", ctypes.c_int),
                ("device", ctypes.c_int), ("allow_grid_raise", ctypes.c_int), ("check_mesh", ctypes.c_int),
                ("fuse_plane_passes", ctypes.c_int), ("fuse_column_passes", ctypes.c_int),
                ("check_finite", ctypes.c_int), ("integration", ctypes.c_int), ("spread_table", ctypes.c_int),
                ("gather_item_targets", ctypes.c_int), ("spread_blocks", ctypes.c_int)]


SLP_TUNE_MAX = 16


class slp_tune_info(ctypes.Structure):
    _fields_ = [("n_candidates", ctypes.c_int), ("chosen", ctypes.c_int),
                ("grid", (ctypes.c_int * 3) * SLP_TUNE_MAX), ("ms", ctypes.c_double * SLP_TUNE_MAX),
                ("kernel_mode", ctypes.c_int * SLP_TUNE_MAX), ("spread_table", ctypes.c_int * SLP_TUNE_MAX),
                ("spread_blocks", ctypes.c_int * SLP_TUNE_MAX), ("gather_item_targets", ctypes.c_int * SLP_TUNE_MAX),
                ("fft_passes", ctypes.c_int * SLP_TUNE_MAX)]

    def to_dict(self):
        n = self.n_candidates
        return {"chosen": self.chosen,
                "candidates": [{"grid": list(self.grid[i]), "ms": self.ms[i], "kernel_mode": self.kernel_mode[i],
                                "spread_table": self.spread_table[i], "spread_blocks": self.spread_blocks[i],
                                "gather_item_targets": self.gather_item_targets[i],
                                "fft_passes": ["separate", "fused plane", "fused column"][self.fft_passes[i]]}
                               for i in range(n)]}


SLP_REQ_QUEUED, SLP_REQ_RUNNING, SLP_REQ_DONE, SLP_REQ_REJECTED, SLP_REQ_CANCELLED, SLP_REQ_FAILED = 1, 2, 3, 4, 5, 6


class slp_server_opts(ctypes.Structure):
    _fields_ = [("slots_per_plan", ctypes.c_int), ("hbm_budget_bytes", ctypes.c_int64), ("reserved", ctypes.c_int * 6)]


class slp_server_statistics(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("rejected", ctypes.c_int64), ("cancelled", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("targets_done", ctypes.c_int64), ("latency_p50_ms", ctypes.c_double),
                ("latency_p99_ms", ctypes.c_double), ("latency_max_ms", ctypes.c_double),
                ("queue_wait_p50_ms", ctypes.c_double), ("queue_wait_p99_ms", ctypes.c_double),
                ("makespan_s", ctypes.c_double), ("arena_bytes", ctypes.c_int64), ("arena_peak_bytes", ctypes.c_int64),
                ("slot_scratch_bytes", ctypes.c_int64), ("n_slots", ctypes.c_int64), ("max_inflight", ctypes.c_int64)]

    def to_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class slp_potential_info(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("n_tets", ctypes.c_int64), ("n_free", ctypes.c_int64),
                ("n_boundary", ctypes.c_int64), ("n_faces", ctypes.c_int64), ("stiffness_nnz", ctypes.c_int64),
                ("load_nnz", ctypes.c_int64), ("cg_iterations", ctypes.c_int64), ("cg_corrections", ctypes.c_int64),
                ("cg_max_iterations", ctypes.c_int64), ("cg_residual", ctypes.c_double),
                ("cg_tolerance", ctypes.c_double), ("ms_phi1", ctypes.c_double), ("ms_phi2", ctypes.c_double),
                ("surface_plan", ctypes.c_void_p)]


class slp_info(ctypes.Structure):
    _fields_ = [("n_targets", ctypes.c_int64), ("n_sources", ctypes.c_int64), ("n_triangles", ctypes.c_int64),
                ("quadrature", ctypes.c_int), ("precision", ctypes.c_int), ("grid", ctypes.c_int * 3),
                ("modes", ctypes.c_int * 3), ("m", ctypes.c_int), ("kernel_mode", ctypes.c_int),
                ("near_mode", ctypes.c_int), ("grid_raised", ctypes.c_int), ("center", ctypes.c_double * 3),
                ("period", ctypes.c_double * 3), ("sigma_g", ctypes.c_double), ("trunc_radius", ctypes.c_double),
                ("eps_near", ctypes.c_double), ("tolerance", ctypes.c_double), ("near_pairs", ctypes.c_int64),
                ("near_pairs_within", ctypes.c_int64), ("near_matrix_nnz", ctypes.c_int64),
                ("bytes_device", ctypes.c_int64), ("n_spread_items", ctypes.c_int64),
                ("n_gather_items", ctypes.c_int64), ("n_near_items", ctypes.c_int64),
                ("launches_per_eval", ctypes.c_int), ("active_rows", ctypes.c_int64),
                ("active_planes", ctypes.c_int), ("fused_plane_passes", ctypes.c_int),
                ("fused_column_passes", ctypes.c_int), ("gather_item_targets", ctypes.c_int),
                ("spread_blocks_per_sm", ctypes.c_int), ("spread_table", ctypes.c_int),
                ("expsum_terms", ctypes.c_int), ("integration", ctypes.c_int), ("grid_matrix_nnz", ctypes.c_int64),
                ("grid_matrix_rows", ctypes.c_int64), ("near_tri_nnz", ctypes.c_int64),
                ("deterministic_spread", ctypes.c_int)]

    def to_dict(self):
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            if isinstance(v, ctypes.Array):
                v = list(v)
            out[name] = v
        return out


# ------------------------------------------------------------------ loading
_lib = None

#: C entry points the binding requires (the declarations of include/slp.h and include/slp_debug.h)
EXPORTED = ["slp_default_opts", "slp_plan", "slp_eval", "slp_eval_states", "slp_eval_host", "slp_eval_host_async",
            "slp_eval_host_wait", "slp_probe_create", "slp_eval_probe", "slp_probe_query", "slp_probe_destroy",
            "slp_potential_create", "slp_potential_eval", "slp_potential_query", "slp_potential_destroy",
            "slp_query", "slp_query_points",
            "slp_check", "slp_destroy", "slp_status_string", "slp_last_error",
            "slp_debug_run", "slp_debug_copy", "slp_debug_buffer_bytes", "slp_debug_host_count",
            "slp_debug_host_array", "slp_debug_window", "slp_debug_window_hat", "slp_debug_profile",
            "slp_debug_timeline", "slp_debug_fem_assemble",
            "slp_debug_stage_name", "slp_eval_direct_static", "slp_batch_create", "slp_batch_run",
            "slp_batch_query", "slp_batch_destroy", "slp_eval_batched", "slp_plan_autotune", "slp_server_default_opts",
            "slp_server_create", "slp_server_submit", "slp_server_status", "slp_server_wait", "slp_server_cancel",
            "slp_server_stats", "slp_server_destroy"]


def library_path() -> str:
    return _LIB_PATH


def load():
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"CUDA library not built: {_LIB_PATH} is missing "
                          "(run paper_1305_3162_gb300._build.build())")
    lib = ctypes.CDLL(_LIB_PATH)
    vp = ctypes.c_void_p
    St = ctypes.c_int
    I64 = ctypes.c_int64
    sig = {
        "slp_default_opts": ([ctypes.POINTER(slp_plan_opts)], St),
        "slp_plan": ([ctypes.POINTER(slp_mesh), ctypes.c_int, ctypes.c_double, ctypes.POINTER(slp_plan_opts),
                      ctypes.POINTER(vp)], St),
        "slp_eval": ([vp, ctypes.c_int, vp, vp, vp], St),
        "slp_eval_host": ([vp, ctypes.c_int, vp, vp, vp], St),
        "slp_eval_host_async": ([vp, ctypes.c_int, vp, vp, vp], St),
        "slp_eval_host_wait": ([vp], St),
        "slp_probe_create": ([vp, ctypes.POINTER(ctypes.c_double), I64, ctypes.POINTER(vp)], St),
        "slp_eval_probe": ([vp, vp, ctypes.c_int, vp, vp, vp, vp], St),
        "slp_probe_query": ([vp, ctypes.POINTER(I64), ctypes.POINTER(I64)], St),
        "slp_probe_destroy": ([vp], St),
        "slp_potential_create": ([ctypes.POINTER(ctypes.c_double), I64, ctypes.POINTER(ctypes.c_int32), I64,
                                  ctypes.c_double, ctypes.POINTER(slp_plan_opts), ctypes.c_double, ctypes.c_int,
                                  ctypes.POINTER(vp)], St),
        "slp_potential_eval": ([vp, vp, vp, vp, vp], St),
        "slp_potential_query": ([vp, ctypes.POINTER(slp_potential_info)], St),
        "slp_potential_destroy": ([vp], St),
        "slp_eval_states": ([vp, ctypes.c_int, ctypes.c_int, vp, vp, vp], St),
        "slp_query": ([vp, ctypes.POINTER(slp_info)], St),
        "slp_query_points": ([vp, ctypes.POINTER(ctypes.c_double)], St),
        "slp_check": ([vp], St),
        "slp_destroy": ([vp], St),
        "slp_status_string": ([ctypes.c_int], ctypes.c_char_p),
        "slp_last_error": ([], ctypes.c_char_p),
        "slp_debug_run": ([vp, ctypes.c_int, vp, vp, vp, ctypes.c_int], St),
        "slp_debug_copy": ([vp, ctypes.c_int, vp, I64], St),
        "slp_debug_buffer_bytes": ([vp, ctypes.c_int, ctypes.POINTER(I64)], St),
        "slp_debug_host_count": ([vp, ctypes.c_int, ctypes.POINTER(I64)], St),
        "slp_debug_host_array": ([vp, ctypes.c_int, vp, I64], St),
        "slp_debug_window": ([ctypes.c_int, ctypes.c_double], ctypes.c_double),
        "slp_debug_window_hat": ([ctypes.c_int, ctypes.c_int, ctypes.c_double], ctypes.c_double),
        "slp_debug_profile": ([vp, ctypes.c_int, vp, vp, vp, ctypes.POINTER(ctypes.c_float), ctypes.c_int], St),
        "slp_debug_timeline": ([vp, ctypes.c_int, vp, vp, vp, ctypes.POINTER(ctypes.c_float)], St),
        "slp_debug_stage_name": ([ctypes.c_int], ctypes.c_char_p),
        "slp_debug_fem_assemble": ([ctypes.POINTER(ctypes.c_double), I64, ctypes.POINTER(ctypes.c_int32), I64,
                                    ctypes.POINTER(I64), vp, vp, vp, vp, vp, vp, vp, vp, vp], St),
        "slp_eval_direct_static": ([vp, I64, vp, I64, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, vp], St),
        "slp_batch_create": ([ctypes.c_int, ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                              ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(vp)], St),
        "slp_batch_run": ([vp, vp], St),
        "slp_batch_query": ([vp, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64)], St),
        "slp_batch_destroy": ([vp], St),
        "slp_eval_batched": ([ctypes.c_int, ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(vp),
                              ctypes.POINTER(ctypes.c_int), vp], St),
        "slp_plan_autotune": ([ctypes.POINTER(slp_mesh), ctypes.c_int, ctypes.c_double, ctypes.POINTER(slp_plan_opts),
                               ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(slp_tune_info)], St),
        "slp_server_default_opts": ([ctypes.POINTER(slp_server_opts)], St),
        "slp_server_create": ([ctypes.c_int, ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(slp_server_opts),
                               ctypes.POINTER(vp)], St),
        "slp_server_submit": ([vp, ctypes.c_int, ctypes.c_int, vp, vp, ctypes.POINTER(I64)], St),
        "slp_server_status": ([vp, I64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)], St),
        "slp_server_wait": ([vp, I64, ctypes.c_double, ctypes.POINTER(ctypes.c_int)], St),
        "slp_server_cancel": ([vp, I64], St),
        "slp_server_stats": ([vp, ctypes.POINTER(slp_server_statistics)], St),
        "slp_server_destroy": ([vp], St),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _check(st: int, where: str):
    if st != SLP_OK:
        detail = load().slp_last_error().decode(errors="replace")
        raise SlpError(st, where, detail)


def _ptr(x):
    """Device or host address of a torch tensor, numpy array or integer."""
    if x is None:
        return None
    if isinstance(x, int):
        return ctypes.c_void_p(x)
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        return ctypes.c_void_p(x.ctypes.data)
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


# ------------------------------------------------------------------ C entry points
def slp_default_opts() -> slp_plan_opts:
    o = slp_plan_opts()
    _check(load().slp_default_opts(ctypes.byref(o)), "slp_default_opts")
    return o


def slp_plan(vertices, triangles, quadrature: int, tolerance: float, opts: slp_plan_opts | None = None):
    """Build a plan; returns an opaque handle (release with slp_destroy)."""
    lib = load()
    V = np.ascontiguousarray(vertices, dtype=np.float64)
    T = np.ascontiguousarray(triangles, dtype=np.int32)
    mesh = slp_mesh(V.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), V.shape[0],
                    T.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), T.shape[0])
    out = ctypes.c_void_p()
    o = opts if opts is not None else slp_default_opts()
    _check(lib.slp_plan(ctypes.byref(mesh), int(quadrature), float(tolerance), ctypes.byref(o), ctypes.byref(out)),
           "slp_plan")
    return out


def slp_eval(plan, input_kind: int, d_in, d_phi, stream=None):
    _check(load().slp_eval(plan, int(input_kind), _ptr(d_in), _ptr(d_phi), _stream(stream)), "slp_eval")


def slp_eval_states(plan, input_kind: int, n_states: int, d_in, d_phi, stream=None):
    """n_states evaluations of one plan (inputs back to back, outputs [n_states][N])."""
    _check(load().slp_eval_states(plan, int(input_kind), int(n_states), _ptr(d_in), _ptr(d_phi), _stream(stream)),
           "slp_eval_states")


def slp_eval_host(plan, input_kind: int, h_in, h_phi, stream=None):
    _check(load().slp_eval_host(plan, int(input_kind), _ptr(h_in), _ptr(h_phi), _stream(stream)), "slp_eval_host")


def _check_device_tensor(x, name, dtype_name, min_numel, where):
    """Raise SlpError unless torch tensor x is a contiguous CUDA tensor on the
    current device of the given dtype with at least min_numel elements (raw
    integer addresses are passed through unchecked)."""
    if isinstance(x, int) or not hasattr(x, "data_ptr"):
        if isinstance(x, np.ndarray):
            raise SlpError(SLP_ERR_INVALID_ARG, where, f"{name} is a host array; a device tensor is required")
        return
    import torch
    if not x.is_cuda:
        raise SlpError(SLP_ERR_INVALID_ARG, where, f"{name} is not a CUDA tensor")
    if x.device.index != torch.cuda.current_device():
        raise SlpError(SLP_ERR_INVALID_ARG, where, f"{name} is on {x.device}, not the current device")
    if str(x.dtype) != "torch." + dtype_name:
        raise SlpError(SLP_ERR_INVALID_ARG, where, f"{name} has dtype {x.dtype}, expected torch.{dtype_name}")
    if not x.is_contiguous():
        raise SlpError(SLP_ERR_INVALID_ARG, where, f"{name} is not contiguous")
    if x.numel() < min_numel:
        raise SlpError(SLP_ERR_INVALID_ARG, where, f"{name} holds {x.numel()} elements, needs {min_numel}")


def slp_eval_host_async(plan, input_kind: int, h_in, h_phi, stream=None):
    """Pipelined host-buffer evaluation (results valid after slp_eval_host_wait)."""
    _check(load().slp_eval_host_async(plan, int(input_kind), _ptr(h_in), _ptr(h_phi), _stream(stream)),
           "slp_eval_host_async")


def slp_probe_create(plan, points):
    """Attach evaluation points (host [n][3]) to a plan; returns the probe handle."""
    pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
    out = ctypes.c_void_p()
    _check(load().slp_probe_create(plan, pts.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), pts.shape[0],
                                   ctypes.byref(out)), "slp_probe_create")
    return out


def slp_eval_probe(plan, probe, input_kind, d_in, d_phi, d_phi_points, stream=None):
    """slp_eval at the mesh vertices plus the probe points from the same evaluation."""
    _check(load().slp_eval_probe(plan, probe, int(input_kind), _ptr(d_in), _ptr(d_phi), _ptr(d_phi_points),
                                 _stream(stream)), "slp_eval_probe")


def slp_probe_query(probe) -> dict:
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(load().slp_probe_query(probe, ctypes.byref(a), ctypes.byref(b)), "slp_probe_query")
    return {"n_points": a.value, "near_nnz": b.value}


def slp_probe_destroy(probe):
    if probe is not None:
        _check(load().slp_probe_destroy(probe), "slp_probe_destroy")


def slp_potential_create(nodes, tets, tolerance: float, opts: slp_plan_opts | None = None,
                         cg_tolerance: float = 0.0, cg_max_iterations: int = 0):
    """The scalar potential of a tetrahedral mesh (nodes [N][3], tets [K][4]);
    returns the handle (release with slp_potential_destroy)."""
    X = np.ascontiguousarray(nodes, dtype=np.float64)
    K = np.ascontiguousarray(tets, dtype=np.int32)
    out = ctypes.c_void_p()
    o = opts if opts is not None else slp_default_opts()
    _check(load().slp_potential_create(X.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), X.shape[0],
                                       K.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), K.shape[0],
                                       float(tolerance), ctypes.byref(o), float(cg_tolerance), int(cg_max_iterations),
                                       ctypes.byref(out)), "slp_potential_create")
    return out


def slp_debug_fem_assemble(nodes, tets) -> dict:
    """The host set-up of the scalar potential (include/slp_debug.h): node
    classes, outward boundary faces with normals and 1/h, S(free, free) and
    the load operator as numpy arrays."""
    X = np.ascontiguousarray(nodes, dtype=np.float64)
    K = np.ascontiguousarray(tets, dtype=np.int32)
    args = (X.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), X.shape[0],
            K.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), K.shape[0])
    counts = (ctypes.c_int64 * 5)()
    _check(load().slp_debug_fem_assemble(*args, counts, *([None] * 9)), "slp_debug_fem_assemble")
    nf, nb, nfc, snz, bnz = (int(c) for c in counts)
    out = {"n_free": nf, "n_boundary": nb,
           "node_slot": np.zeros(X.shape[0], np.int32), "faces": np.zeros((nfc, 4), np.int32),
           "face_geom": np.zeros((nfc, 4)), "s_ptr": np.zeros(nf + 1, np.int64), "s_col": np.zeros(snz, np.int32),
           "s_val": np.zeros(snz), "b_ptr": np.zeros(nf + 1, np.int64), "b_col": np.zeros(bnz, np.int32),
           "b_val": np.zeros((bnz, 3))}
    keys = ("node_slot", "faces", "face_geom", "s_ptr", "s_col", "s_val", "b_ptr", "b_col", "b_val")
    _check(load().slp_debug_fem_assemble(*args, counts, *[out[k].ctypes.data_as(ctypes.c_void_p) for k in keys]),
           "slp_debug_fem_assemble")
    return out


def slp_potential_eval(pot, d_m, d_phi, d_phi_1=None, stream=None):
    """phi = phi_1 + phi_2 at every node from the nodal m (and phi_1 when asked)."""
    _check(load().slp_potential_eval(pot, _ptr(d_m), _ptr(d_phi), _ptr(d_phi_1), _stream(stream)),
           "slp_potential_eval")


def slp_potential_query(pot) -> dict:
    info = slp_potential_info()
    _check(load().slp_potential_query(pot, ctypes.byref(info)), "slp_potential_query")
    return {name: getattr(info, name) for name, _ in info._fields_}


def slp_potential_destroy(pot):
    if pot is not None:
        _check(load().slp_potential_destroy(pot), "slp_potential_destroy")


def slp_eval_host_wait(plan):
    _check(load().slp_eval_host_wait(plan), "slp_eval_host_wait")


def slp_eval_direct_static(d_vertices, n_vertices, d_triangles, n_triangles, quadrature, precision, input_kind,
                           d_in, d_phi, stream=None):
    """Allocation-free direct evaluation (see include/slp.h): device mesh, input and output.

    Torch tensors are checked (CUDA, current device, dtype, contiguity,
    size) before their addresses reach the library."""
    where = "slp_eval_direct_static"
    nv, nt, q = int(n_vertices), int(n_triangles), int(quadrature)
    fdt = "float64" if int(precision) == 64 else "float32"
    need_in = {SLP_INPUT_SIGMA: q * nt, SLP_INPUT_MAG: 3 * q * nt, SLP_INPUT_NODAL_MAG: 3 * nv}.get(int(input_kind), 0)
    _check_device_tensor(d_vertices, "d_vertices", "float64", 3 * nv, where)
    _check_device_tensor(d_triangles, "d_triangles", "int32", 3 * nt, where)
    _check_device_tensor(d_in, "d_in", fdt, need_in, where)
    _check_device_tensor(d_phi, "d_phi", fdt, nv, where)
    _check(load().slp_eval_direct_static(_ptr(d_vertices), int(n_vertices), _ptr(d_triangles), int(n_triangles),
                                         int(quadrature), int(precision), int(input_kind), _ptr(d_in), _ptr(d_phi),
                                         _stream(stream)), "slp_eval_direct_static")


def slp_batch_create(plans, plan_of, input_kind, d_in, d_phi, lanes_per_plan=1):
    """Capture items (plans[plan_of[i]], d_in[i] -> d_phi[i]) into one CUDA graph; returns the batch handle."""
    n_plans = len(plans)
    n_items = len(plan_of)
    P = (ctypes.c_void_p * n_plans)(*[p.value if isinstance(p, ctypes.c_void_p) else p for p in plans])
    po = (ctypes.c_int * n_items)(*[int(i) for i in plan_of])
    ins = (ctypes.c_void_p * n_items)(*[_ptr(x).value for x in d_in])
    outs = (ctypes.c_void_p * n_items)(*[_ptr(x).value for x in d_phi])
    out = ctypes.c_void_p()
    _check(load().slp_batch_create(n_plans, P, n_items, po, int(input_kind), ins, outs, int(lanes_per_plan),
                                   ctypes.byref(out)), "slp_batch_create")
    return out


def slp_batch_run(batch, stream=None):
    _check(load().slp_batch_run(batch, _stream(stream)), "slp_batch_run")


def slp_batch_query(batch) -> dict:
    a, b, c, d = (ctypes.c_int64() for _ in range(4))
    _check(load().slp_batch_query(batch, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)),
           "slp_batch_query")
    return {"n_items": a.value, "n_lanes": b.value, "kernel_launches": c.value, "extra_scratch_bytes": d.value}


def slp_batch_destroy(batch):
    if batch is not None:
        _check(load().slp_batch_destroy(batch), "slp_batch_destroy")


def slp_eval_batched(plans, input_kind, d_in, d_phi, n_states_each, stream=None):
    """Evaluate n_states_each[i] states of plans[i] (inputs back to back in
    d_in[i], outputs [n][N_i] in d_phi[i]) in one cached CUDA graph."""
    n = len(plans)
    P = (ctypes.c_void_p * n)(*[p.value if isinstance(p, ctypes.c_void_p) else p for p in plans])
    ins = (ctypes.c_void_p * n)(*[_ptr(x).value for x in d_in])
    outs = (ctypes.c_void_p * n)(*[_ptr(x).value for x in d_phi])
    cnt = (ctypes.c_int * n)(*[int(c) for c in n_states_each])
    _check(load().slp_eval_batched(n, P, int(input_kind), ins, outs, cnt, _stream(stream)), "slp_eval_batched")


def slp_plan_autotune(vertices, triangles, quadrature, tolerance, opts=None, reps=5):
    """Plan on candidate grids, time each, keep the fastest; returns (plan handle, tuning record)."""
    lib = load()
    V = np.ascontiguousarray(vertices, dtype=np.float64)
    T = np.ascontiguousarray(triangles, dtype=np.int32)
    mesh = slp_mesh(V.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), V.shape[0],
                    T.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), T.shape[0])
    o = opts if opts is not None else slp_default_opts()
    out = ctypes.c_void_p()
    ti = slp_tune_info()
    _check(lib.slp_plan_autotune(ctypes.byref(mesh), int(quadrature), float(tolerance), ctypes.byref(o), int(reps),
                                 ctypes.byref(out), ctypes.byref(ti)), "slp_plan_autotune")
    return out, ti.to_dict()


def slp_server_default_opts() -> slp_server_opts:
    o = slp_server_opts()
    _check(load().slp_server_default_opts(ctypes.byref(o)), "slp_server_default_opts")
    return o


def slp_server_create(plans, input_kind, opts=None):
    n = len(plans)
    P = (ctypes.c_void_p * n)(*[p.value if isinstance(p, ctypes.c_void_p) else p for p in plans])
    o = opts if opts is not None else slp_server_default_opts()
    out = ctypes.c_void_p()
    _check(load().slp_server_create(n, P, int(input_kind), ctypes.byref(o), ctypes.byref(out)), "slp_server_create")
    return out


def slp_server_submit(server, plan_index, n_states, h_in, h_out) -> int:
    rid = ctypes.c_int64()
    _check(load().slp_server_submit(server, int(plan_index), int(n_states), _ptr(h_in), _ptr(h_out), ctypes.byref(rid)),
           "slp_server_submit")
    return rid.value


def slp_server_status(server, request_id):
    """(state, result status) of a request."""
    st = ctypes.c_int()
    res = ctypes.c_int()
    _check(load().slp_server_status(server, int(request_id), ctypes.byref(st), ctypes.byref(res)), "slp_server_status")
    return st.value, res.value


def slp_server_wait(server, request_id, timeout_s=60.0):
    """Wait for a request; raises SlpError on timeout or if the request failed or was rejected."""
    st = ctypes.c_int()
    _check(load().slp_server_wait(server, int(request_id), float(timeout_s), ctypes.byref(st)), "slp_server_wait")
    return st.value


def slp_server_cancel(server, request_id):
    _check(load().slp_server_cancel(server, int(request_id)), "slp_server_cancel")


def slp_server_stats(server) -> dict:
    st = slp_server_statistics()
    _check(load().slp_server_stats(server, ctypes.byref(st)), "slp_server_stats")
    return st.to_dict()


def slp_server_destroy(server):
    if server is not None:
        _check(load().slp_server_destroy(server), "slp_server_destroy")


def slp_query(plan) -> dict:
    info = slp_info()
    _check(load().slp_query(plan, ctypes.byref(info)), "slp_query")
    return info.to_dict()


def slp_query_points(plan, n_sources: int):
    pts = np.zeros((n_sources, 3))
    _check(load().slp_query_points(plan, pts.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "slp_query_points")
    return pts


def slp_check(plan):
    _check(load().slp_check(plan), "slp_check")


def slp_destroy(plan):
    if plan is not None:
        _check(load().slp_destroy(plan), "slp_destroy")


def slp_status_string(status: int) -> str:
    return load().slp_status_string(int(status)).decode()


def slp_last_error() -> str:
    return load().slp_last_error().decode(errors="replace")


def slp_debug_run(plan, input_kind, d_in, d_phi, stream=None, last_stage=SLP_STAGE_NEAR):
    _check(load().slp_debug_run(plan, int(input_kind), _ptr(d_in), _ptr(d_phi), _stream(stream), int(last_stage)),
           "slp_debug_run")


def slp_debug_copy(plan, buffer: int, dtype):
    n = ctypes.c_int64()
    _check(load().slp_debug_buffer_bytes(plan, int(buffer), ctypes.byref(n)), "slp_debug_buffer_bytes")
    out = np.zeros(n.value // np.dtype(dtype).itemsize, dtype=dtype)
    _check(load().slp_debug_copy(plan, int(buffer), _ptr(out), n.value), "slp_debug_copy")
    return out


_HOST_DTYPES = {SLP_HOST_SRC_PERM: np.int32, SLP_HOST_TGT_PERM: np.int32, SLP_HOST_SRC_GRID: np.float64,
                SLP_HOST_TGT_GRID: np.float64, SLP_HOST_SPREAD_ITEMS: np.int32, SLP_HOST_GATHER_ITEMS: np.int32,
                SLP_HOST_NEAR_ITEMS: np.int32, SLP_HOST_NEAR_RANGES: np.int32, SLP_HOST_DTAB: np.float64,
                SLP_HOST_SRC_POINTS: np.float64, SLP_HOST_TGT_POINTS: np.float64, SLP_HOST_PLANE_ROWS: np.int32,
                SLP_HOST_ACTIVE_Z: np.int32, SLP_HOST_SPREAD_GROUPS: np.int32, SLP_HOST_SPREAD_GROUP_OFF: np.int32,
                SLP_HOST_EXPSUM: np.float64}


def slp_debug_host_array(plan, which: int):
    n = ctypes.c_int64()
    _check(load().slp_debug_host_count(plan, int(which), ctypes.byref(n)), "slp_debug_host_count")
    out = np.zeros(n.value, dtype=_HOST_DTYPES[which])
    _check(load().slp_debug_host_array(plan, int(which), _ptr(out), n.value), "slp_debug_host_array")
    return out


def slp_debug_timeline(plan, input_kind, d_in, d_phi, stream=None):
    """Milestones (ms from the start) of one concurrent evaluation: spread,
    fft, near branch, gather."""
    ms = (ctypes.c_float * 4)()
    _check(load().slp_debug_timeline(plan, int(input_kind), _ptr(d_in), _ptr(d_phi), _stream(stream), ms),
           "slp_debug_timeline")
    return {"spread": ms[0], "fft": ms[1], "near": ms[2], "gather": ms[3]}


def slp_debug_profile(plan, input_kind, d_in, d_phi, stream=None) -> dict:
    """Per-kernel durations (ms) of one serial evaluation, CUDA events around
    each launch on the launch stream; only the kernels that launched appear."""
    n = 15
    ms = (ctypes.c_float * n)()
    _check(load().slp_debug_profile(plan, int(input_kind), _ptr(d_in), _ptr(d_phi), _stream(stream), ms, n),
           "slp_debug_profile")
    return {load().slp_debug_stage_name(i).decode(): float(ms[i]) for i in range(n) if ms[i] >= 0.0}


def slp_debug_window(m: int, d: float) -> float:
    return load().slp_debug_window(int(m), float(d))


def slp_debug_window_hat(m: int, L: int, l: float) -> float:
    return load().slp_debug_window_hat(int(m), int(L), float(l))


# ------------------------------------------------------------------ convenience
class Plan:
    """Owns an slp plan handle; ``eval`` enqueues on the given (or current) torch stream."""

    def __init__(self, vertices, triangles, quadrature=7, tolerance=1e-5, precision=32, grid=None, m=0,
                 kernel_mode=SLP_KERNEL_AUTO, near_mode=SLP_NEAR_AUTO, deterministic=False, device=0,
                 allow_grid_raise=True, check_mesh=True, fuse_plane_passes=-1, fuse_column_passes=-1,
                 spread_table=-1, integration=0):
        o = slp_default_opts()
        o.precision = int(precision)
        if grid is not None:
            for d in range(3):
                o.grid[d] = int(grid[d])
        o.m = int(m)
        o.kernel_mode = int(kernel_mode)
        o.near_mode = int(near_mode)
        o.deterministic = int(bool(deterministic))
        o.device = int(device)
        o.allow_grid_raise = int(bool(allow_grid_raise))
        o.check_mesh = int(bool(check_mesh))
        o.fuse_plane_passes = int(fuse_plane_passes)
        o.fuse_column_passes = int(fuse_column_passes)
        o.spread_table = int(spread_table)
        o.integration = int(integration)
        self.handle = slp_plan(vertices, triangles, quadrature, tolerance, o)
        self.info = slp_query(self.handle)
        self.n_targets = self.info["n_targets"]
        self.n_sources = self.info["n_sources"]
        self.precision = self.info["precision"]

    def eval(self, input_kind, d_in, d_phi, stream=None):
        if stream is None:
            import torch
            stream = torch.cuda.current_stream()
        slp_eval(self.handle, input_kind, d_in, d_phi, stream)

    def close(self):
        if self.handle is not None:
            slp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
