"""Plain FP64 CPU oracle for the 2D wave field of point sources (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this package.  It shares no code with the CUDA path.

The library (``wfp_oracle.c``) evaluates the exact retarded field of the paper's
model problem (Sec. 1, Eqs. wave2d, solnRep, Green, pointSources) by the
square-root substitution of Sec. 7, Eq. exactSol, with an independent
cosh-substitution quadrature as a cross-check, plus component oracles for the
local / near-history / far-history split of Sec. 3 (Eqs. ul, unh, ufh) and the
coincident-pair self term.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wfp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libwfp_oracle.so")

NPAR = 8
FAMILY = {"gauss3": 0, "erf": 1, "poly": 2}
KIND = {"full": 0, "local": 1, "near": 2, "far": 3}

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, OpenMP, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fno-fast-math", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        d, i, pd = ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_double)
        lib.wfo_field.argtypes = [i, i, pd, pd, i, pd, i, d, d, d, i, d, pd]
        lib.wfo_self.argtypes = [i, i, pd, pd, d, d, pd]
        lib.wfo_sigma.argtypes = [i, pd, d]
        lib.wfo_sigma.restype = d
        lib.wfo_phi.argtypes = [d, d, d]
        lib.wfo_phi.restype = d
        lib.wfo_dphi.argtypes = [d, d, d]
        lib.wfo_dphi.restype = d
        lib.wfo_i0.argtypes = [d]
        lib.wfo_i0.restype = d
        lib.wfo_set_resolution.argtypes = [i, d]
        lib.wfo_set_threads.argtypes = [i]
        lib.wfo_num_threads.restype = i
        lib.wfo_gl_rule.argtypes = [i, pd, pd]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def set_resolution(nodes: int = 20, hfac: float = 0.5) -> None:
    """Nodes per GL panel (20 or 40) and panel width as a fraction of the signal's feature scale."""
    if _load().wfo_set_resolution(int(nodes), float(hfac)) != 0:
        raise ValueError("nodes must be 20 or 40")


def set_threads(n: int) -> None:
    _load().wfo_set_threads(int(n))


def num_threads() -> int:
    return int(_load().wfo_num_threads())


def field(src_xy, params, eval_xyt, family="gauss3", kind="full", delta=0.0, Aplus=0.0, b=0.0,
          method=0, r_coinc=0.0) -> np.ndarray:
    """u at each (x, y, t) row of ``eval_xyt`` from sources ``src_xy`` (M x 2) with signal
    parameters ``params`` (M x 8).  ``kind`` selects the full field or one split component;
    ``method`` 0 is the square-root substitution (Eq. exactSol), 1 the cosh substitution."""
    src = _f64(src_xy).reshape(-1, 2)
    par = _f64(params).reshape(-1, NPAR)
    ev = _f64(eval_xyt).reshape(-1, 3)
    if par.shape[0] != src.shape[0]:
        raise ValueError("one parameter row per source")
    out = np.zeros(ev.shape[0])
    _load().wfo_field(FAMILY[family], src.shape[0], _ptr(src), _ptr(par), ev.shape[0], _ptr(ev), KIND[kind],
                      float(delta), float(Aplus), float(b), int(method), float(r_coinc), _ptr(out))
    return out


def self_term(params, times, delta, b, family="gauss3") -> np.ndarray:
    """(1/2pi) int_0^t phi(d) sigma(t - d) / d dd for each (signal row, time) pair."""
    par = _f64(params).reshape(-1, NPAR)
    t = _f64(times).reshape(-1)
    if par.shape[0] != t.shape[0]:
        raise ValueError("one parameter row per time")
    out = np.zeros(t.shape[0])
    _load().wfo_self(FAMILY[family], t.shape[0], _ptr(par), _ptr(t), float(delta), float(b), _ptr(out))
    return out


def sigma(params, t, family="gauss3") -> float:
    p = _f64(params).reshape(NPAR)
    return float(_load().wfo_sigma(FAMILY[family], _ptr(p), float(t)))


def phi(t, delta, b) -> float:
    return float(_load().wfo_phi(float(t), float(delta), float(b)))


def dphi(t, delta, b) -> float:
    return float(_load().wfo_dphi(float(t), float(delta), float(b)))


def i0(x) -> float:
    return float(_load().wfo_i0(float(x)))


def gl_rule(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    if _load().wfo_gl_rule(int(n), _ptr(x), _ptr(w)) != 0:
        raise ValueError("bad n")
    return x, w
