"""FP64 CPU oracle for the triangle-quadrature single layer potential.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use it.  The library in
``paper_1305_3162_gb300`` shares no code with it and never imports it.

The arithmetic lives in ``slp_oracle.c`` (plain C, compensated summation,
OpenMP over targets); this module only builds it with gcc and marshals numpy
arrays.  See that file's header for the definition and the citations.

Parity status: every function here is pinned by tests/test_oracle_pins.py
(quadrature exactness, closed-form sphere potentials, the analytic triangle
integral against a Duffy-transformed Gauss-Legendre rule, invariances; the
triangle-integrated definition by the same sphere closed forms, converging
faster than the point rules).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "slp_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libslp_oracle.so")
_lock = threading.Lock()
_lib = None

KIND_SIGMA = 0
KIND_MAG = 1
KIND_NODAL_MAG = 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, so compensated sums stay exact)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99", _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            d = ctypes.POINTER(ctypes.c_double)
            i32 = ctypes.POINTER(ctypes.c_int32)
            i64p = ctypes.POINTER(ctypes.c_int64)
            I64 = ctypes.c_int64
            lib.slpo_rule.argtypes = [ctypes.c_int, d, d]
            lib.slpo_sources.argtypes = [d, I64, i32, I64, ctypes.c_int, d, d, d]
            lib.slpo_charges.argtypes = [ctypes.c_int, d, I64, i32, I64, ctypes.c_int, d, d]
            lib.slpo_direct.argtypes = [d, I64, d, d, I64, d, ctypes.c_int]
            lib.slpo_direct_subset.argtypes = [d, i64p, I64, d, d, I64, d, ctypes.c_int]
            lib.slpo_triangle_integral.argtypes = [d, d, d, d]
            lib.slpo_triangle_integral.restype = ctypes.c_double
            lib.slpo_element_charges.argtypes = [d, I64, i32, I64, d, d]
            lib.slpo_direct_p0.argtypes = [d, i64p, I64, d, I64, i32, I64, d, d, ctypes.c_int]
            for f in (lib.slpo_rule, lib.slpo_sources, lib.slpo_charges, lib.slpo_direct, lib.slpo_direct_subset,
                      lib.slpo_element_charges, lib.slpo_direct_p0):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a, ct=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def rule(q: int):
    """Barycentric points (q,3) and weights (q,) of the q-point triangle rule."""
    lam = np.zeros((q, 3))
    w = np.zeros(q)
    if _load().slpo_rule(q, _p(lam), _p(w)) != 0:
        raise ValueError(f"no {q}-point rule")
    return lam, w


def sources(V, T, q: int):
    """Quadrature points y (M*q,3), weights w_s|S_j| (M*q,), outward normals (M,3)."""
    V = _f64(V)
    T = _i32(T)
    nt = T.shape[0]
    y = np.zeros((nt * q, 3))
    wk = np.zeros(nt * q)
    nrm = np.zeros((nt, 3))
    rc = _load().slpo_sources(_p(V), V.shape[0], _p(T, ctypes.c_int32), nt, q, _p(y), _p(wk), _p(nrm))
    if rc != 0:
        raise ValueError(f"slpo_sources failed ({rc})")
    return y, wk, nrm


def charges(V, T, q: int, kind: int, data):
    """Weighted charges w_s |S_j| sigma_{j,s} for the given input kind."""
    V = _f64(V)
    T = _i32(T)
    data = _f64(data)
    nt = T.shape[0]
    qk = np.zeros(nt * q)
    rc = _load().slpo_charges(kind, _p(V), V.shape[0], _p(T, ctypes.c_int32), nt, q, _p(data), _p(qk))
    if rc != 0:
        raise ValueError(f"slpo_charges failed ({rc})")
    return qk


def direct(x, y, qk, nthreads: int = 0):
    """phi_i = (1/4pi) sum_k qk / |x_i - y_k| (all pairs). Returns (phi, threads used)."""
    x = _f64(x)
    y = _f64(y)
    qk = _f64(qk)
    phi = np.zeros(x.shape[0])
    used = _load().slpo_direct(_p(x), x.shape[0], _p(y), _p(qk), y.shape[0], _p(phi), int(nthreads))
    return phi, used


def direct_subset(x, sel, y, qk, nthreads: int = 0):
    """The direct sum at the targets x[sel] only."""
    x = _f64(x)
    sel = np.ascontiguousarray(sel, dtype=np.int64)
    y = _f64(y)
    qk = _f64(qk)
    phi = np.zeros(sel.shape[0])
    used = _load().slpo_direct_subset(_p(x), _p(sel, ctypes.c_int64), sel.shape[0], _p(y), _p(qk),
                                      y.shape[0], _p(phi), int(nthreads))
    return phi, used


def slp(V, T, q: int, kind: int, data, nthreads: int = 0):
    """The single layer potential at every mesh vertex for the given input (FP64)."""
    y, _, _ = sources(V, T, q)
    qk = charges(V, T, q, kind, data)
    phi, _ = direct(V, y, qk, nthreads)
    return phi


def slp_nodal(V, T, q: int, m_nodal, nthreads: int = 0):
    """Convenience: nodal magnetisation input (P1 interpolation, sigma = m.n)."""
    return slp(V, T, q, KIND_NODAL_MAG, m_nodal, nthreads)


# ---------------------------------------------------------------- triangle-integrated (P0) definition
def triangle_integral(v0, v1, v2, x):
    """int over the flat triangle (v0, v1, v2) of 1/|x - y| dA(y) (closed form)."""
    a = [_f64(np.asarray(p, dtype=np.float64).reshape(3)) for p in (v0, v1, v2, x)]
    return float(_load().slpo_triangle_integral(*[_p(v) for v in a]))


def element_charges(V, T, m_nodal):
    """g_j: integral mean of m . n_j over triangle j for P1 nodal m."""
    V = _f64(V)
    T = _i32(T)
    m = _f64(m_nodal)
    g = np.zeros(T.shape[0])
    rc = _load().slpo_element_charges(_p(V), V.shape[0], _p(T, ctypes.c_int32), T.shape[0], _p(m), _p(g))
    if rc != 0:
        raise ValueError(f"slpo_element_charges failed ({rc})")
    return g


def slp_p0(V, T, g, sel=None, nthreads: int = 0, x=None):
    """phi_i = (1/4pi) sum_j g_j int_{S_j} 1/|x_i - y| dA(y) at the vertices
    (or at V[sel], or at the points x [n][3] when given), every triangle
    integrated exactly.  Returns phi."""
    V = _f64(V)
    T = _i32(T)
    g = _f64(g)
    X = V if x is None else _f64(np.asarray(x, dtype=np.float64).reshape(-1, 3))
    if sel is None:
        ns, sp = X.shape[0], None
    else:
        sel = np.ascontiguousarray(sel, dtype=np.int64)
        ns, sp = sel.shape[0], _p(sel, ctypes.c_int64)
    phi = np.zeros(ns)
    _load().slpo_direct_p0(_p(X), sp, ns, _p(V), V.shape[0], _p(T, ctypes.c_int32), T.shape[0], _p(g), _p(phi),
                           int(nthreads))
    return phi
