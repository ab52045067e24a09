"""Thin Python binding of the C ABI in include/wfp.h (argument marshalling only).

Every step of the evaluation runs in the CUDA library ``_build/libwfp.so``; there is no
Python or CPU fallback.  If the library is missing it is built in-tree with nvcc; if that is
impossible the import of the binding raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

WFP_OK, WFP_EINVAL, WFP_ENOMEM, WFP_ECUDA, WFP_ESTATE, WFP_ETIMEOUT, WFP_EUNSUPPORTED = range(7)
FP64, MIXED = 0, 1
LAG_AUTO, LAG_RECOMPUTE, LAG_STORE = 0, 1, 2
INTERP_HYBRID, INTERP_LAGRANGE = 0, 1
LOCAL_AUTO, LOCAL_STORED, LOCAL_FACTORED = 0, 1, 2
ORDER_AUTO, ORDER_CONCURRENT, ORDER_SERIAL = 0, 1, 2

_c_i64 = ctypes.c_int64
_c_dbl = ctypes.c_double
_pd = ctypes.POINTER(ctypes.c_double)


class wfp_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("eps", _c_dbl), ("W", ctypes.c_int), ("p", ctypes.c_int),
                ("Kf", _c_dbl), ("upsampfac", _c_dbl), ("kernel_width", ctypes.c_int),
                ("soe_nodes", ctypes.c_int), ("exclude_self", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("use_graph", ctypes.c_int), ("lag_mode", ctypes.c_int), ("spread_tile", ctypes.c_int),
                ("spread_chunk", ctypes.c_int), ("local_variant", ctypes.c_int), ("local_interp", ctypes.c_int),
                ("delta", _c_dbl), ("local_form", ctypes.c_int), ("step_order", ctypes.c_int)]


class wfp_info(ctypes.Structure):
    _fields_ = [("scale", _c_dbl), ("cx", _c_dbl), ("cy", _c_dbl), ("dt", _c_dbl), ("T", _c_dbl),
                ("K0", _c_dbl), ("eps", _c_dbl), ("b", _c_dbl), ("W", ctypes.c_int), ("p", ctypes.c_int),
                ("nmax", ctypes.c_int), ("delta", _c_dbl), ("K", _c_dbl), ("A", _c_dbl), ("Aplus", _c_dbl),
                ("dk", _c_dbl), ("L", ctypes.c_int), ("Kf", _c_dbl), ("Nh", ctypes.c_int),
                ("n_modes", _c_i64), ("n_far_modes", _c_i64), ("n_kappa", _c_i64), ("n_lambda", ctypes.c_int),
                ("soe_panels", ctypes.c_int), ("soe_nodes", ctypes.c_int), ("n_self_soe", ctypes.c_int),
                ("nf", ctypes.c_int), ("nb", ctypes.c_int), ("kernel_width", ctypes.c_int),
                ("upsampfac", _c_dbl), ("n_pairs", _c_i64), ("n_self", _c_i64), ("lag_active", ctypes.c_int),
                ("far_active", ctypes.c_int), ("precision", ctypes.c_int), ("device_bytes", _c_i64),
                ("lag_store", ctypes.c_int), ("s_levels", _c_i64), ("spread_tile", ctypes.c_int),
                ("spread_chunk", ctypes.c_int), ("local_variant", ctypes.c_int), ("local_form", ctypes.c_int),
                ("local_nc", ctypes.c_int), ("n_near_pairs", _c_i64), ("n_spread_tiles", _c_i64),
                ("bytes_local", _c_i64), ("bytes_grid", _c_i64), ("bytes_history", _c_i64),
                ("bytes_fft_work", _c_i64), ("step_order", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None

# every symbol declared in include/wfp.h and include/wfp_debug.h
EXPORTS = ["wfp_debug_eta_table", "wfp_debug_factored_table", "wfp_opts_default", "wfp_plan_create", "wfp_step", "wfp_destroy", "wfp_plan_get_info",
           "wfp_step_components", "wfp_select_params", "wfp_status_string", "wfp_last_error",
           "wfp_profile", "wfp_profile_read", "wfp_local_noalloc", "wfp_debug_eta", "wfp_debug_taps", "wfp_debug_phi",
           "wfp_debug_soe", "wfp_debug_self_soe", "wfp_debug_hankel", "wfp_debug_bounded_wait", "wfp_checkpoint_size",
           "wfp_checkpoint_save", "wfp_checkpoint_load", "wfp_server_create", "wfp_server_submit", "wfp_server_tick",
           "wfp_server_run", "wfp_server_query", "wfp_server_result", "wfp_server_destroy", "wfp_debug_alu_peak"]

SIGNAL_GAUSS3, SIGNAL_ERF = 0, 1
REQ_PENDING, REQ_ACTIVE, REQ_DONE, REQ_FAILED, REQ_BUILDING = range(5)


class wfp_request(ctypes.Structure):
    _fields_ = [("M", _c_i64), ("src_xy", _pd), ("Mt", _c_i64), ("tgt_xy", _pd), ("dt", _c_dbl), ("Nt", _c_i64),
                ("band_limit", _c_dbl), ("tol", _c_dbl), ("signal_family", ctypes.c_int),
                ("signal_params", _pd), ("n_out", ctypes.c_int), ("out_steps", ctypes.POINTER(_c_i64))]


class wfp_request_status(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int), ("steps_done", _c_i64), ("Nt", _c_i64), ("Mt", _c_i64),
                ("n_out", ctypes.c_int), ("t_submit", _c_dbl), ("t_admit", _c_dbl), ("t_done", _c_dbl),
                ("device_bytes", _c_i64), ("plan_bytes", _c_i64), ("t_active", _c_dbl)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


def lib():
    """Load (building if needed) the CUDA library and declare the ABI."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    L = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    L.wfp_opts_default.argtypes = [ctypes.POINTER(wfp_opts)]
    L.wfp_opts_default.restype = None
    L.wfp_plan_create.argtypes = [_c_i64, _pd, _c_i64, _pd, _c_dbl, _c_i64, _c_dbl, _c_dbl,
                                  ctypes.POINTER(wfp_opts), ctypes.POINTER(vp)]
    L.wfp_step.argtypes = [vp, vp, vp]
    L.wfp_destroy.argtypes = [vp]
    L.wfp_plan_get_info.argtypes = [vp, ctypes.POINTER(wfp_info)]
    L.wfp_step_components.argtypes = [vp, _pd, _pd, _pd]
    L.wfp_select_params.argtypes = [_c_dbl, _c_dbl, _c_i64, _c_dbl, _c_dbl, ctypes.POINTER(wfp_opts),
                                    ctypes.POINTER(wfp_info)]
    L.wfp_status_string.argtypes = [ctypes.c_int]
    L.wfp_status_string.restype = ctypes.c_char_p
    L.wfp_last_error.restype = ctypes.c_char_p
    L.wfp_local_noalloc.argtypes = [_c_i64, vp, _c_i64, vp, vp, ctypes.c_int, _c_dbl, _c_dbl, _c_dbl, vp, vp]
    L.wfp_local_noalloc.restype = ctypes.c_int
    L.wfp_profile.argtypes = [vp, ctypes.c_int]
    L.wfp_profile_read.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_char_p), _pd,
                                   ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int)]
    L.wfp_debug_eta.argtypes = [_c_dbl, _c_dbl, ctypes.c_int, ctypes.c_int, _c_dbl, _c_dbl, ctypes.c_int, _pd]
    L.wfp_debug_eta_table.argtypes = [_c_dbl, _c_dbl, ctypes.c_int, ctypes.c_int, _c_dbl, _c_dbl, ctypes.c_int, _pd]
    L.wfp_debug_eta_table.restype = ctypes.c_int
    L.wfp_debug_factored_table.argtypes = [_c_dbl, ctypes.c_int, ctypes.c_int, _c_dbl, _c_dbl, ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_int), _pd, _pd]
    L.wfp_debug_factored_table.restype = ctypes.c_int
    L.wfp_debug_taps.argtypes = [_c_dbl, _c_dbl, ctypes.c_int, _c_dbl, _c_dbl, _pd, _pd]
    L.wfp_debug_phi.argtypes = [_c_dbl, _c_dbl, _c_dbl, _pd, _pd, _pd]
    L.wfp_debug_soe.argtypes = [_c_dbl, ctypes.c_int, ctypes.c_int, _pd, _pd]
    L.wfp_debug_self_soe.argtypes = [_c_dbl, _c_dbl, _c_dbl, ctypes.c_int, _pd, _pd, ctypes.POINTER(ctypes.c_int)]
    L.wfp_debug_hankel.argtypes = [_c_dbl, _c_dbl, _c_dbl, _c_dbl, _c_dbl, ctypes.c_int, ctypes.c_int, _pd]
    L.wfp_debug_hankel.restype = ctypes.c_int
    L.wfp_checkpoint_size.argtypes = [vp, ctypes.POINTER(_c_i64)]
    L.wfp_checkpoint_save.argtypes = [vp, vp, _c_i64]
    L.wfp_checkpoint_load.argtypes = [vp, vp, _c_i64]
    for name in ("wfp_checkpoint_size", "wfp_checkpoint_save", "wfp_checkpoint_load"):
        getattr(L, name).restype = ctypes.c_int
    L.wfp_debug_bounded_wait.argtypes = [_c_dbl, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _pd]
    L.wfp_debug_bounded_wait.restype = ctypes.c_int
    L.wfp_debug_alu_peak.argtypes = [ctypes.c_int, _pd, _pd]
    L.wfp_debug_alu_peak.restype = ctypes.c_int
    L.wfp_server_create.argtypes = [_c_i64, ctypes.c_int, ctypes.POINTER(wfp_opts), ctypes.POINTER(vp)]
    L.wfp_server_submit.argtypes = [vp, ctypes.POINTER(wfp_request), ctypes.POINTER(_c_i64)]
    L.wfp_server_tick.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    L.wfp_server_run.argtypes = [vp]
    L.wfp_server_query.argtypes = [vp, _c_i64, ctypes.POINTER(wfp_request_status)]
    L.wfp_server_result.argtypes = [vp, _c_i64, _pd]
    L.wfp_server_destroy.argtypes = [vp]
    for name in ("wfp_server_create", "wfp_server_submit", "wfp_server_tick", "wfp_server_run",
                 "wfp_server_query", "wfp_server_result", "wfp_server_destroy"):
        getattr(L, name).restype = ctypes.c_int
    for name in ("wfp_plan_create", "wfp_step", "wfp_destroy", "wfp_plan_get_info", "wfp_step_components",
                 "wfp_profile", "wfp_profile_read",
                 "wfp_select_params", "wfp_debug_eta", "wfp_debug_taps", "wfp_debug_phi", "wfp_debug_soe", "wfp_debug_self_soe"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


class WFPError(RuntimeError):
    def __init__(self, code: int, where: str):
        L = lib()
        super().__init__(f"{where}: {L.wfp_status_string(code).decode()} ({L.wfp_last_error().decode()})")
        self.code = code


def _check(code: int, where: str):
    if code != WFP_OK:
        raise WFPError(code, where)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_pd)


def default_opts(**kw) -> wfp_opts:
    o = wfp_opts()
    lib().wfp_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if k == "stream":
            v = ctypes.c_void_p(v)
        setattr(o, k, v)
    return o


def select_params(halfside: float, dt: float, Nt: int, band_limit: float, tol: float, **opts) -> dict:
    info = wfp_info()
    _check(lib().wfp_select_params(halfside, dt, Nt, band_limit, tol, ctypes.byref(default_opts(**opts)),
                                   ctypes.byref(info)), "wfp_select_params")
    return info.as_dict()


class Plan:
    """One evaluation problem: M sources, Mt targets, Nt steps of size dt (Sec. 1)."""

    def __init__(self, src_xy, tgt_xy, dt: float, Nt: int, band_limit: float, tol: float = 1e-6, **opts):
        L = lib()
        self._src = np.ascontiguousarray(np.asarray(src_xy, dtype=np.float64).reshape(-1, 2))
        self._tgt = self._src if tgt_xy is None else np.ascontiguousarray(
            np.asarray(tgt_xy, dtype=np.float64).reshape(-1, 2))
        self.M, self.Mt = self._src.shape[0], self._tgt.shape[0]
        self._opts = default_opts(**opts)
        h = ctypes.c_void_p()
        _check(L.wfp_plan_create(self.M, _dptr(self._src), self.Mt, _dptr(self._tgt), dt, int(Nt), band_limit, tol,
                                 ctypes.byref(self._opts), ctypes.byref(h)), "wfp_plan_create")
        self._h = h

    def step(self, sigma_n, out=None):
        """sigma_n: M doubles (numpy array, or a torch CUDA float64 tensor); returns u_n (Mt)."""
        L = lib()
        if hasattr(sigma_n, "data_ptr"):  # torch tensor (host or device), marshalled by pointer
            if out is None:
                import torch
                out = torch.empty(self.Mt, dtype=torch.float64, device=sigma_n.device)
            _check(L.wfp_step(self._h, ctypes.c_void_p(sigma_n.data_ptr()), ctypes.c_void_p(out.data_ptr())),
                   "wfp_step")
            return out
        s = np.ascontiguousarray(np.asarray(sigma_n, dtype=np.float64))
        if s.size != self.M:
            raise ValueError("sigma_n must have M entries")
        if out is None:
            out = np.empty(self.Mt)
        _check(L.wfp_step(self._h, s.ctypes.data_as(ctypes.c_void_p), out.ctypes.data_as(ctypes.c_void_p)),
               "wfp_step")
        return out

    def components(self):
        u_l, u_h, u_s = np.empty(self.Mt), np.empty(self.Mt), np.empty(self.Mt)
        _check(lib().wfp_step_components(self._h, _dptr(u_l), _dptr(u_h), _dptr(u_s)), "wfp_step_components")
        return u_l, u_h, u_s

    def profile(self, enable: bool = True):
        _check(lib().wfp_profile(self._h, int(enable)), "wfp_profile")

    def profile_read(self) -> dict:
        n = 16
        names = (ctypes.c_char_p * n)()
        ms = np.zeros(n)
        cnt = np.zeros(n, dtype=np.int64)
        k = ctypes.c_int()
        _check(lib().wfp_profile_read(self._h, n, names, _dptr(ms), cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                      ctypes.byref(k)), "wfp_profile_read")
        return {names[i].decode(): (float(ms[i]), int(cnt[i])) for i in range(min(k.value, n))}

    def checkpoint(self) -> np.ndarray:
        """The plan's step-to-step state as a host byte array (wfp_checkpoint_save)."""
        n = _c_i64()
        _check(lib().wfp_checkpoint_size(self._h, ctypes.byref(n)), "wfp_checkpoint_size")
        buf = np.empty(n.value, dtype=np.uint8)
        _check(lib().wfp_checkpoint_save(self._h, buf.ctypes.data_as(ctypes.c_void_p), n.value), "wfp_checkpoint_save")
        return buf

    def restore(self, buf: np.ndarray):
        """Continue from a state saved by a plan of the same inputs and options (wfp_checkpoint_load)."""
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        _check(lib().wfp_checkpoint_load(self._h, buf.ctypes.data_as(ctypes.c_void_p), buf.size),
               "wfp_checkpoint_load")

    def info(self) -> dict:
        i = wfp_info()
        _check(lib().wfp_plan_get_info(self._h, ctypes.byref(i)), "wfp_plan_get_info")
        return i.as_dict()

    def close(self):
        if getattr(self, "_h", None):
            lib().wfp_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def local_noalloc(src_xy, tgt_xy, sigma_win, nmax: int, dt: float, band_limit: float, tol: float, out,
                  stream: int | None = None):
    """Local part of one step with no allocation (device tensors: src_xy (M,2), tgt_xy (Mt,2),
    sigma_win (nmax, M), out (Mt,), all float64)."""
    M = sigma_win.shape[1]
    Mt = out.shape[0]
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    _check(lib().wfp_local_noalloc(M, p(src_xy), Mt, p(tgt_xy), p(sigma_win), int(nmax), dt, band_limit, tol,
                                   p(out), ctypes.c_void_p(stream or 0)), "wfp_local_noalloc")
    return out


class Server:
    """Continuous-batching request server (wfp_server_* in include/wfp.h)."""

    def __init__(self, hbm_budget_bytes: int, max_active: int = 64, **opts):
        h = ctypes.c_void_p()
        _check(lib().wfp_server_create(int(hbm_budget_bytes), int(max_active), ctypes.byref(default_opts(**opts)),
                                       ctypes.byref(h)), "wfp_server_create")
        self._h = h

    def submit(self, src_xy, signal_params, dt: float, Nt: int, band_limit: float, tol: float = 1e-6,
               tgt_xy=None, out_steps=None, family: int = SIGNAL_GAUSS3) -> int:
        src = np.ascontiguousarray(src_xy, dtype=np.float64)
        par = np.ascontiguousarray(signal_params, dtype=np.float64)
        assert par.shape == (src.shape[0], 2 if family == SIGNAL_ERF else 8)
        tgt = None if tgt_xy is None else np.ascontiguousarray(tgt_xy, dtype=np.float64)
        steps = None if out_steps is None else np.ascontiguousarray(out_steps, dtype=np.int64)
        q = wfp_request(M=src.shape[0], src_xy=_dptr(src), Mt=(src if tgt is None else tgt).shape[0],
                        tgt_xy=None if tgt is None else _dptr(tgt), dt=dt, Nt=int(Nt), band_limit=band_limit,
                        tol=tol, signal_family=family, signal_params=_dptr(par),
                        n_out=0 if steps is None else steps.size,
                        out_steps=None if steps is None else steps.ctypes.data_as(ctypes.POINTER(_c_i64)))
        rid = _c_i64()
        _check(lib().wfp_server_submit(self._h, ctypes.byref(q), ctypes.byref(rid)), "wfp_server_submit")
        return rid.value

    def tick(self):
        a, p = ctypes.c_int(), ctypes.c_int()
        _check(lib().wfp_server_tick(self._h, ctypes.byref(a), ctypes.byref(p)), "wfp_server_tick")
        return a.value, p.value

    def run(self):
        _check(lib().wfp_server_run(self._h), "wfp_server_run")

    def query(self, rid: int) -> dict:
        st = wfp_request_status()
        _check(lib().wfp_server_query(self._h, rid, ctypes.byref(st)), "wfp_server_query")
        return st.as_dict()

    def result(self, rid: int) -> np.ndarray:
        st = self.query(rid)
        out = np.zeros((st["n_out"], st["Mt"]))
        _check(lib().wfp_server_result(self._h, rid, _dptr(out)), "wfp_server_result")
        return out

    def close(self):
        if getattr(self, "_h", None):
            lib().wfp_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ host-only diagnostics
def debug_factored_table(dt, W, p=20, eps=1e-8, band_limit=0.0, ng=20, precision=MIXED):
    """(coefficients kept, largest dropped relative tail, table [W-1][nmax][33]) of the factored local
    part's per-interval Chebyshev series."""
    nmax = W + 1 + p // 2
    tab = np.zeros((W - 1, nmax, 33))
    nc = ctypes.c_int(0)
    tail = np.zeros(1)
    _check(lib().wfp_debug_factored_table(dt, W, p, eps, band_limit, ng, precision, ctypes.byref(nc), _dptr(tail),
                                          _dptr(tab)), "wfp_debug_factored_table")
    return nc.value, float(tail[0]), tab


def alu_peak(fp64: bool = True) -> tuple[float, float]:
    """Measured FMA throughput of the current GPU: (TFLOP/s, ms of the timed launch)."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib().wfp_debug_alu_peak(int(fp64), ctypes.byref(tf), ctypes.byref(ms)), "wfp_debug_alu_peak")
    return tf.value, ms.value


def debug_eta(r, dt, W, p=20, eps=1e-8, band_limit=0.0, ng=20) -> np.ndarray:
    out = np.zeros(W + 1 + p // 2)
    _check(lib().wfp_debug_eta(r, dt, W, p, eps, band_limit, ng, _dptr(out)), "wfp_debug_eta")
    return out


def debug_eta_table(r, dt, W, p=20, eps=1e-8, band_limit=0.0, ng=20) -> np.ndarray:
    out = np.zeros(W + 1 + p // 2)
    _check(lib().wfp_debug_eta_table(r, dt, W, p, eps, band_limit, ng, _dptr(out)), "wfp_debug_eta_table")
    return out


def debug_taps(kappa, dt, W, eps, lagshift):
    taps, rot = np.zeros(4 * W), np.zeros(3)
    _check(lib().wfp_debug_taps(kappa, dt, W, eps, lagshift, _dptr(taps), _dptr(rot)), "wfp_debug_taps")
    return taps, rot


def debug_phi(t, delta, eps):
    a, b, c = _c_dbl(), _c_dbl(), _c_dbl()
    _check(lib().wfp_debug_phi(t, delta, eps, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "wfp_debug_phi")
    return a.value, b.value, c.value


def debug_hankel(kappa, A, Delta, eps, lam_max=36.0, panels=20, ng=32) -> np.ndarray:
    H = np.zeros(panels * ng)
    _check(lib().wfp_debug_hankel(kappa, A, Delta, eps, lam_max, panels, ng, _dptr(H)), "wfp_debug_hankel")
    return H


def debug_bounded_wait(limit_s: float, arrive: bool):
    """Run the device's bounded mbarrier wait once (GPU); returns (timed_out, waited_s)."""
    to, w = ctypes.c_int(), _c_dbl()
    _check(lib().wfp_debug_bounded_wait(limit_s, 1 if arrive else 0, ctypes.byref(to), ctypes.byref(w)),
           "wfp_debug_bounded_wait")
    return bool(to.value), w.value


def debug_self_soe(dlo, T, eps, cap=256):
    """The self term's sum of exponentials for 1/d on [dlo, T] (host); returns (lam, q)."""
    lam, q, n = np.zeros(cap), np.zeros(cap), ctypes.c_int()
    _check(lib().wfp_debug_self_soe(dlo, T, eps, cap, _dptr(lam), _dptr(q), ctypes.byref(n)), "wfp_debug_self_soe")
    return lam[:n.value].copy(), q[:n.value].copy()


def debug_soe(lam_max, panels, ng):
    lam, q = np.zeros(panels * ng), np.zeros(panels * ng)
    _check(lib().wfp_debug_soe(lam_max, panels, ng, _dptr(lam), _dptr(q)), "wfp_debug_soe")
    return lam, q
