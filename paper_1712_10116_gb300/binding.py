"""Thin ctypes binding of libtaichi_gb.so (C ABI in include/taichi_gb.h).

Argument marshalling only: every step of the solver runs in the library's CUDA kernels.
PyTorch supplies device memory and the CUDA stream.  Function names match the C entry points.
The library must have been built (``__graft_entry__.build()`` or ``python -m
paper_1712_10116_gb300.build``); loading fails loudly otherwise -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtaichi_gb.so")

TG_KERNEL_WENDLAND_C2 = 0
TG_KERNEL_PLUMMER = 1
TG_PREC_FP64 = 0
TG_PREC_FP32 = 1
TG_MAC_SIDE = 0
TG_MAC_SPHERE = 1

STATUS = {0: "TG_OK", -1: "TG_ERR_ARG", -2: "TG_ERR_OOM", -3: "TG_ERR_CUDA", -4: "TG_ERR_TIMEOUT",
          -5: "TG_ERR_NONFINITE", -6: "TG_ERR_CAPACITY", -7: "TG_ERR_STATE",
          -8: "TG_ERR_IO"}


class TGError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class tg_params(C.Structure):
    _fields_ = [("p", C.c_int), ("n_crit", C.c_int), ("kernel", C.c_int), ("precision", C.c_int),
                ("max_level", C.c_int), ("k_max", C.c_int), ("theta", C.c_double), ("kappa", C.c_double),
                ("eps", C.c_double), ("eta", C.c_double), ("dt_max", C.c_double), ("eta_tot", C.c_double),
                ("mac", C.c_int), ("batched", C.c_int)]


class tg_stats(C.Structure):
    _fields_ = [("evaluations", C.c_int64), ("sink_forces", C.c_int64), ("p2p_pairs", C.c_int64),
                ("m2l_pairs", C.c_int64), ("p2p_cell_pairs", C.c_int64), ("cells", C.c_int64),
                ("kdk_frames", C.c_int64), ("max_rung", C.c_int64), ("m2l_class_pairs", C.c_int64),
                ("list_regrowths", C.c_int64), ("host_syncs", C.c_int64)]


KERNEL_CLASSES = ["tree", "up", "walk", "m2l", "p2p", "down", "hhs", "other"]


class tg_tuning(C.Structure):
    _fields_ = [("n_crit", C.c_int), ("p2p_rows", C.c_int), ("m2l_blocks_per_sm", C.c_int), ("m2l_form", C.c_int),
                ("candidates", C.c_int),
                ("objective_ms", C.c_double), ("objective_ms_initial", C.c_double)]


class tg_profile(C.Structure):
    _fields_ = [("ms", C.c_double * 8), ("launches", C.c_int64 * 8)]


@dataclass
class Params:
    """Solver parameters (defaults: the paper's fiducial theta/p are 0.45/5, n_crit 64, eta 0.02)."""
    p: int = 5
    theta: float = 0.45
    eps: float = 0.01
    kernel: int = TG_KERNEL_WENDLAND_C2
    precision: int = TG_PREC_FP64
    n_crit: int = 64
    kappa: float = 1.0
    max_level: int = 21
    eta: float = 0.02
    dt_max: float = 1.0 / 64
    k_max: int = 10
    eta_tot: float = 0.0   # Eq. (9) minimum-timestep constraint, 0 = off
    mac: int = 0           # TG_MAC_SIDE (the paper's Eq. 1) or TG_MAC_SPHERE (enclosing radii)
    batched: int = 0       # 1: HOLD steps as one CUDA graph with a device-side work queue

    def to_c(self) -> tg_params:
        return tg_params(p=self.p, n_crit=self.n_crit, kernel=self.kernel, precision=self.precision,
                         max_level=self.max_level, k_max=self.k_max, theta=self.theta, kappa=self.kappa,
                         eps=self.eps, eta=self.eta, dt_max=self.dt_max, eta_tot=self.eta_tot, mac=self.mac,
                         batched=self.batched)


_lib = None
_lock = threading.Lock()
_vp = C.c_void_p
_i64 = C.c_int64


def load() -> C.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                                   "(python -c 'import __graft_entry__ as g; g.build()')")
            L = C.CDLL(LIB_PATH)
            L.tg_create.argtypes = [C.POINTER(tg_params), _vp, C.POINTER(_vp)]
            L.tg_destroy.argtypes = [_vp]
            L.tg_last_error.argtypes = [_vp]
            L.tg_last_error.restype = C.c_char_p
            L.tg_get_stats.argtypes = [_vp, C.POINTER(tg_stats)]
            L.tg_reset_stats.argtypes = [_vp]
            L.tg_build_tree.argtypes = [_vp, _i64, _vp]
            L.tg_fmm_forces.argtypes = [_vp, _i64, _vp, _vp, _vp, _vp, _vp]
            L.tg_direct_forces.argtypes = [_vp, _i64, _vp, _vp, _vp, _i64, _vp, _vp, _vp]
            L.tg_hhs_init.argtypes = [_vp, _i64, _vp, _vp, _vp]
            L.tg_hhs_step.argtypes = [_vp]
            L.tg_trad_init.argtypes = [_vp, _i64, _vp, _vp, _vp]
            L.tg_trad_step.argtypes = [_vp]
            L.tg_hhs_state.argtypes = [_vp, _vp, _vp, _vp, _vp]
            L.tg_hhs_set_accel.argtypes = [_vp, _vp, _vp, _vp]
            L.tg_diagnostics.argtypes = [_vp, C.POINTER(C.c_double)]
            L.tg_checkpoint.argtypes = [_vp, C.c_char_p]
            L.tg_restore.argtypes = [_vp, C.c_char_p]
            L.tg_tree_info.argtypes = [_vp, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(_i64),
                                       C.POINTER(_i64)]
            L.tg_get_tree.argtypes = [_vp] * 8
            L.tg_list_counts.argtypes = [_vp, C.POINTER(_i64), C.POINTER(_i64)]
            L.tg_get_lists.argtypes = [_vp] * 5
            L.tg_timesteps.argtypes = [_vp, _i64, _vp, _vp, _vp, _vp, _vp]
            L.tg_morton_sort_noalloc.argtypes = [_i64, _vp, _vp, _vp, _vp]
            L.tg_morton_sort_noalloc.restype = C.c_int
            L.tg_debug_control.argtypes = [_vp, C.c_int, _i64]
            L.tg_autotune.argtypes = [_vp, _i64, _vp, _vp, _vp, C.POINTER(tg_tuning)]
            L.tg_ensemble_step.argtypes = [C.POINTER(_vp), C.c_int]
            L.tg_ensemble_step.restype = C.c_int
            L.tg_get_tuning.argtypes = [_vp, C.POINTER(tg_tuning)]
            L.tg_set_tuning.argtypes = [_vp, C.POINTER(tg_tuning)]
            L.tg_set_profiling.argtypes = [_vp, C.c_int]
            L.tg_get_profile.argtypes = [_vp, C.POINTER(tg_profile)]
            for name in ("tg_create", "tg_destroy", "tg_get_stats", "tg_reset_stats", "tg_build_tree",
                         "tg_fmm_forces", "tg_direct_forces", "tg_hhs_init", "tg_hhs_step", "tg_hhs_state",
                         "tg_hhs_set_accel", "tg_diagnostics", "tg_tree_info", "tg_get_tree", "tg_list_counts",
                         "tg_get_lists", "tg_timesteps", "tg_set_profiling", "tg_get_profile", "tg_debug_control",
                         "tg_autotune", "tg_get_tuning", "tg_set_tuning"):
                getattr(L, name).restype = C.c_int
            _lib = L
    return _lib


def _check(ctx, rc: int):
    if rc != 0:
        msg = load().tg_last_error(ctx) if ctx else b""
        raise TGError(rc, (msg or b"").decode())


def _ptr(t) -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _stream_handle(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


# ---------------------------------------------------------------- entry points (same names)
def tg_create(params: Params, stream=None):
    ctx = _vp()
    cp = params.to_c()
    _check(None, load().tg_create(C.byref(cp), _vp(_stream_handle(stream)), C.byref(ctx)))
    return ctx


def tg_destroy(ctx):
    _check(None, load().tg_destroy(ctx))


def tg_get_stats(ctx) -> dict:
    s = tg_stats()
    _check(ctx, load().tg_get_stats(ctx, C.byref(s)))
    return {k: getattr(s, k) for k, _ in tg_stats._fields_}


def tg_reset_stats(ctx):
    _check(ctx, load().tg_reset_stats(ctx))


def tg_build_tree(ctx, pos: torch.Tensor):
    _check(ctx, load().tg_build_tree(ctx, pos.shape[1], _ptr(pos)))


def tg_fmm_forces(ctx, pos, mass, is_fast=None, acc=None, pot=None, want_pot=True):
    """pos (3, n) float64 CUDA, mass (n,), is_fast (n,) uint8 or None -> (acc (3, n), pot (n,) or None)."""
    n = mass.shape[0]
    if acc is None:
        acc = torch.empty((3, n), dtype=torch.float64, device=pos.device)
    if pot is None and want_pot:
        pot = torch.empty(n, dtype=torch.float64, device=pos.device)
    _check(ctx, load().tg_fmm_forces(ctx, n, _ptr(pos), _ptr(mass), _ptr(is_fast), _ptr(acc), _ptr(pot)))
    return acc, pot


def tg_direct_forces(ctx, pos, mass, is_fast=None, sinks=None):
    """Direct float64 summation for the sinks (int64 CUDA tensor of indices, None = all)."""
    n = mass.shape[0]
    ns = n if sinks is None else sinks.shape[0]
    acc = torch.empty((3, ns), dtype=torch.float64, device=pos.device)
    pot = torch.empty(ns, dtype=torch.float64, device=pos.device)
    _check(ctx, load().tg_direct_forces(ctx, n, _ptr(pos), _ptr(mass), _ptr(is_fast), ns, _ptr(sinks), _ptr(acc),
                                        _ptr(pot)))
    return acc, pot


def tg_hhs_init(ctx, pos, vel, mass):
    _check(ctx, load().tg_hhs_init(ctx, mass.shape[0], _ptr(pos), _ptr(vel), _ptr(mass)))


def tg_hhs_step(ctx):
    _check(ctx, load().tg_hhs_step(ctx))


def tg_hhs_state(ctx, n: int, device="cuda", with_total=False):
    rung = torch.empty(n, dtype=torch.int32, device=device)
    a_old = torch.empty(n, dtype=torch.float64, device=device)
    a_cur = torch.empty(n, dtype=torch.float64, device=device)
    a_tot = torch.empty(n, dtype=torch.float64, device=device) if with_total else None
    _check(ctx, load().tg_hhs_state(ctx, _ptr(rung), _ptr(a_old), _ptr(a_cur), _ptr(a_tot)))
    return (rung, a_old, a_cur, a_tot) if with_total else (rung, a_old, a_cur)


def tg_hhs_set_accel(ctx, a_old, a_cur, a_tot=None):
    _check(ctx, load().tg_hhs_set_accel(ctx, _ptr(a_old), _ptr(a_cur), _ptr(a_tot)))


def tg_diagnostics(ctx) -> np.ndarray:
    out = (C.c_double * 8)()
    _check(ctx, load().tg_diagnostics(ctx, out))
    return np.array(out[:])


def tg_trad_init(ctx, pos, vel, mass) -> None:
    _check(ctx, load().tg_trad_init(ctx, mass.shape[0], _ptr(pos), _ptr(vel), _ptr(mass)))


def tg_trad_step(ctx) -> None:
    _check(ctx, load().tg_trad_step(ctx))


def tg_checkpoint(ctx, path) -> None:
    _check(ctx, load().tg_checkpoint(ctx, os.fsencode(path)))


def tg_restore(ctx, path) -> None:
    _check(ctx, load().tg_restore(ctx, os.fsencode(path)))


def tg_tree_info(ctx):
    lo = (C.c_double * 3)()
    L = C.c_double()
    n = _i64()
    nc = _i64()
    _check(ctx, load().tg_tree_info(ctx, lo, C.byref(L), C.byref(n), C.byref(nc)))
    return np.array(lo[:]), L.value, n.value, nc.value


def tg_get_tree(ctx) -> dict:
    lo, L, n, nc = tg_tree_info(ctx)
    keys = np.zeros(n, np.uint64)
    perm = np.zeros(n, np.int64)
    level = np.zeros(nc, np.int32)
    coords = np.zeros((3, nc), np.int64)
    first = np.zeros(nc, np.int64)
    count = np.zeros(nc, np.int64)
    nchild = np.zeros(nc, np.int32)
    args = [a.ctypes.data_as(_vp) for a in (keys, perm, level, coords, first, count, nchild)]
    _check(ctx, load().tg_get_tree(ctx, *args))
    return dict(lo=lo, L=L, keys=keys, perm=perm, level=level, coords=coords, first=first, count=count,
                nchild=nchild)


def tg_get_lists(ctx):
    nm, npp = _i64(), _i64()
    _check(ctx, load().tg_list_counts(ctx, C.byref(nm), C.byref(npp)))
    m2l = np.zeros((2, nm.value), np.int64)
    p2p = np.zeros((2, npp.value), np.int64)
    _check(ctx, load().tg_get_lists(ctx, *[a.ctypes.data_as(_vp) for a in (m2l[0], m2l[1], p2p[0], p2p[1])]))
    return m2l, p2p


def tg_set_profiling(ctx, level: int):
    _check(ctx, load().tg_set_profiling(ctx, level))


def tg_get_profile(ctx) -> dict:
    pr = tg_profile()
    _check(ctx, load().tg_get_profile(ctx, C.byref(pr)))
    out = {name: {"ms": pr.ms[k], "launches": pr.launches[k]} for k, name in enumerate(KERNEL_CLASSES)}
    out["_all"] = {"ms": sum(pr.ms[k] for k in range(8)), "launches": sum(pr.launches[k] for k in range(8))}
    return out


TG_NOALLOC_MAX_N = 262144


def tg_morton_sort_noalloc(pos, keys_out=None, perm_out=None, stream=None):
    """Root cube, Morton keys and stable radix sort without any device allocation inside the
    library (scratch is a fixed static device array; n <= TG_NOALLOC_MAX_N).  Returns
    (keys (n,) uint64 as int64 storage, perm (n,) int64).  Calls overlapping on the GPU race."""
    n = pos.shape[1]
    if keys_out is None:
        keys_out = torch.empty(n, dtype=torch.int64, device=pos.device)
    if perm_out is None:
        perm_out = torch.empty(n, dtype=torch.int64, device=pos.device)
    # the library launches on the current device: make it pos's, and default to that device's stream
    with torch.cuda.device(pos.device):
        if stream is None:
            stream = torch.cuda.current_stream(pos.device)
        rc = load().tg_morton_sort_noalloc(n, _ptr(pos), _ptr(keys_out), _ptr(perm_out), _vp(_stream_handle(stream)))
    if rc != 0:
        raise TGError(rc, "tg_morton_sort_noalloc")
    return keys_out, perm_out


TG_DEBUG_FAIL_ALLOC = 1
TG_DEBUG_LIST_CAPACITY = 2
TG_DEBUG_QUEUE_LIMIT = 3
TG_DEBUG_QUEUE_HOLD = 4
TG_DEBUG_BATCH_CAPS = 5


def tg_debug_control(ctx, what: int, value: int):
    _check(ctx, load().tg_debug_control(ctx, what, value))


def _tuning_dict(t) -> dict:
    return {k: getattr(t, k) for k, _ in tg_tuning._fields_}


def tg_autotune(ctx, pos=None, mass=None, is_fast=None) -> dict:
    """Time evaluations of this system (pos, mass given) or rung-0 steps of the system bound by
    tg_hhs_init (pos = mass = None) over leaf size and launch shapes; the context keeps the fastest."""
    out = tg_tuning()
    n = 0 if mass is None else mass.shape[0]
    _check(ctx, load().tg_autotune(ctx, n, _ptr(pos), _ptr(mass), _ptr(is_fast), C.byref(out)))
    return _tuning_dict(out)


def tg_get_tuning(ctx) -> dict:
    out = tg_tuning()
    _check(ctx, load().tg_get_tuning(ctx, C.byref(out)))
    return _tuning_dict(out)


def tg_ensemble_step(ctxs) -> None:
    """One rung-0 HOLD step of every context (bound, batched, same stream) as one graph launch."""
    arr = (_vp * len(ctxs))(*[c.value if isinstance(c, _vp) else c for c in ctxs])
    _check(ctxs[0], load().tg_ensemble_step(arr, len(ctxs)))


def tg_set_tuning(ctx, tuning: dict):
    t = tg_tuning(**{k: tuning[k] for k, _ in tg_tuning._fields_ if k in tuning})
    _check(ctx, load().tg_set_tuning(ctx, C.byref(t)))


def tg_timesteps(ctx, a_old, a_cur, a_tot=None):
    n = a_old.shape[0]
    dt = torch.empty(n, dtype=torch.float64, device=a_old.device)
    rung = torch.empty(n, dtype=torch.int32, device=a_old.device)
    _check(ctx, load().tg_timesteps(ctx, n, _ptr(a_old), _ptr(a_cur), _ptr(a_tot), _ptr(dt), _ptr(rung)))
    return dt, rung


class Solver:
    """A context with its parameters; destroys the context when garbage-collected."""

    def __init__(self, params: Params, stream=None):
        self.params = params
        self.ctx = tg_create(params, stream)

    def fmm_forces(self, pos, mass, is_fast=None, want_pot=True):
        return tg_fmm_forces(self.ctx, pos, mass, is_fast, want_pot=want_pot)

    def autotune(self, pos=None, mass=None, is_fast=None):
        return tg_autotune(self.ctx, pos, mass, is_fast)

    def direct_forces(self, pos, mass, is_fast=None, sinks=None):
        return tg_direct_forces(self.ctx, pos, mass, is_fast, sinks)

    def hhs_init(self, pos, vel, mass):
        self._hhs = (pos, vel, mass)
        tg_hhs_init(self.ctx, pos, vel, mass)

    def hhs_step(self):
        tg_hhs_step(self.ctx)

    def trad_init(self, pos, vel, mass):
        self._hhs = (pos, vel, mass)
        tg_trad_init(self.ctx, pos, vel, mass)

    def trad_step(self):
        tg_trad_step(self.ctx)

    def checkpoint(self, path):
        tg_checkpoint(self.ctx, path)

    def restore(self, path):
        tg_restore(self.ctx, path)

    def diagnostics(self):
        return tg_diagnostics(self.ctx)

    def stats(self):
        return tg_get_stats(self.ctx)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            tg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
