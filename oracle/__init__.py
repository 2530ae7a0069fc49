"""Plain FP64 CPU oracle of the momentum-conserving FMM + HHS scheme (Zhu 2017).

TEST INFRASTRUCTURE ONLY.  The oracle is a slow, direct restatement of the method used to
check the CUDA path.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import it; the product package never does, and the two share no code.

The C source (``taichi_oracle.c``) cites the sections, equations and algorithms of the
paper it follows.  This module compiles it with gcc on first use and wraps it with ctypes.
All arrays are float64 numpy arrays; positions are passed as an (3, n) array.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "taichi_oracle.c")
_HDR = os.path.join(_HERE, "taichi_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

WENDLAND_C2 = 0
PLUMMER = 1


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, OpenMP, no FMA contraction)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("p", C.c_int), ("n_crit", C.c_int), ("kernel", C.c_int), ("max_level", C.c_int),
                ("theta", C.c_double), ("kappa", C.c_double), ("eps", C.c_double), ("mac", C.c_int)]


class HHSParams(C.Structure):
    _fields_ = [("eta", C.c_double), ("dt_max", C.c_double), ("k_max", C.c_int), ("eta_tot", C.c_double)]


class HHSStats(C.Structure):
    _fields_ = [("poisson_calls", C.c_int64), ("sink_forces", C.c_int64), ("kdk_frames", C.c_int64),
                ("max_rung", C.c_int32), ("trace_len", C.c_int32)]


MAC_SIDE, MAC_SPHERE = 0, 1


def params(p=4, theta=0.5, eps=0.01, kernel=WENDLAND_C2, n_crit=64, kappa=1.0, max_level=21, mac=MAC_SIDE) -> Params:
    return Params(p=p, n_crit=n_crit, kernel=kernel, max_level=max_level,
                  theta=theta, kappa=kappa, eps=eps, mac=mac)


_d = C.POINTER(C.c_double)
_i64 = C.POINTER(C.c_int64)
_i32 = C.POINTER(C.c_int32)
_u64 = C.POINTER(C.c_uint64)
_u8 = C.POINTER(C.c_uint8)
_vp = C.c_void_p


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_num_coeffs.restype = C.c_int
            L.orc_multi_index.argtypes = [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
            L.orc_softened.argtypes = [C.c_int, C.c_double, C.c_double, _d, _d]
            L.orc_dtensor.argtypes = [C.c_int, _d, C.c_int, C.c_double, _d]
            L.orc_direct.argtypes = [C.c_int64, _d, _d, _d, _d, _vp, C.c_int, C.c_double, C.c_int64, _vp,
                                     _d, _d, _d, _vp]
            L.orc_root_cube.argtypes = [C.c_int64, _d, _d, _d, _d, _d]
            L.orc_morton_keys.argtypes = [C.c_int64, _d, _d, _d, _d, C.c_double, _u64]
            L.orc_sort_keys.argtypes = [C.c_int64, _u64, _i64]
            L.orc_tree_build.argtypes = [C.c_int64, _d, _d, _d, C.POINTER(Params)]
            L.orc_tree_build.restype = _vp
            L.orc_tree_free.argtypes = [_vp]
            L.orc_tree_ncell.argtypes = [_vp]
            L.orc_tree_ncell.restype = C.c_int64
            L.orc_tree_cells.argtypes = [_vp, _i32, _i64, _i64, _i64, _i64, _i64, _i64, _i32]
            L.orc_tree_perm.argtypes = [_vp, _i64, _u64]
            L.orc_tree_geometry.argtypes = [_vp, _d, _d]
            L.orc_tree_walk.argtypes = [_vp, _i64, _i64]
            L.orc_tree_lists.argtypes = [_vp, _i64, _i64, _i64, _i64]
            L.orc_well_separated.argtypes = [_vp, C.c_int64, C.c_int64]
            L.orc_tree_radii.argtypes = [_vp, _d]
            L.orc_p2m.argtypes = [C.c_int, C.c_int64, _d, _d, _d, _d, _d, _d]
            L.orc_m2m.argtypes = [C.c_int, _d, _d, _d]
            L.orc_m2l.argtypes = [C.c_int, _d, _d, C.c_int, C.c_double, _d]
            L.orc_l2l.argtypes = [C.c_int, _d, _d, _d]
            L.orc_l2p.argtypes = [C.c_int, _d, _d, _d, _d]
            L.orc_fmm.argtypes = [C.c_int64, _d, _d, _d, _d, _vp, C.POINTER(Params), _d, _d, _d, _vp]
            L.orc_fmm_sample.argtypes = [C.c_int64, _d, _d, _d, _d, _vp, C.POINTER(Params), C.c_int64, _i64,
                                         _d, _d, _d, _vp]
            L.orc_timestep.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double]
            L.orc_timestep.restype = C.c_double
            L.orc_timestep_tot.argtypes = [C.c_double] * 6
            L.orc_trad_init.argtypes = [C.c_int64, _d, _d, _d, _d, C.POINTER(Params), C.POINTER(HHSParams), _d, _i32]
            L.orc_trad_step.argtypes = [C.c_int64, _d, _d, _d, _d, _d, _d, _d, C.POINTER(Params),
                                        C.POINTER(HHSParams), _d, _i32, C.POINTER(HHSStats)]
            L.orc_timestep_tot.restype = C.c_double
            L.orc_rung.argtypes = [C.c_double, C.c_double, C.c_int]
            L.orc_hhs_init.argtypes = [C.c_int64, _d, _d, _d, _d, C.POINTER(Params), _d, _d, _d]
            L.orc_hhs_step.argtypes = [C.c_int64, _d, _d, _d, _d, _d, _d, _d, C.POINTER(Params),
                                       C.POINTER(HHSParams), _d, _d, _d, _i32, C.POINTER(HHSStats), _vp, C.c_int32]
            L.orc_diagnostics.argtypes = [C.c_int64, _d, _d, _d, _d, _d, _d, _d, _vp, _d]
            _lib = L
    return _lib


def _p(a, t=_d):
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _opt_u8(a):
    if a is None:
        return None, None
    arr = np.ascontiguousarray(a, dtype=np.uint8)
    return arr, arr.ctypes.data_as(_vp)


def num_coeffs(p: int) -> int:
    return lib().orc_num_coeffs(p)


def multi_indices(p: int) -> np.ndarray:
    out = np.zeros((num_coeffs(p), 3), dtype=np.int64)
    a, b, c = C.c_int(), C.c_int(), C.c_int()
    for i in range(out.shape[0]):
        lib().orc_multi_index(i, C.byref(a), C.byref(b), C.byref(c))
        out[i] = (a.value, b.value, c.value)
    return out


def softened(kernel: int, eps: float, r: float):
    phi, g = C.c_double(), C.c_double()
    lib().orc_softened(kernel, eps, r, C.byref(phi), C.byref(g))
    return phi.value, g.value


def dtensor(p: int, d, kernel=WENDLAND_C2, eps=0.0) -> np.ndarray:
    d = _f64(d)
    D = np.zeros(num_coeffs(p))
    lib().orc_dtensor(p, _p(d), kernel, eps, _p(D))
    return D


def direct(pos, mass, eps, kernel=WENDLAND_C2, is_fast=None, sinks=None):
    """Direct summation; returns (acc (3, ns), pot (ns,))."""
    pos = _f64(pos)
    mass = _f64(mass)
    n = mass.shape[0]
    fast, fast_p = _opt_u8(is_fast)
    if sinks is None:
        ns, sp = n, None
    else:
        sinks = np.ascontiguousarray(sinks, dtype=np.int64)
        ns, sp = sinks.shape[0], sinks.ctypes.data_as(_vp)
    acc = np.zeros((3, ns))
    pot = np.zeros(ns)
    lib().orc_direct(n, _p(pos[0]), _p(pos[1]), _p(pos[2]), _p(mass), fast_p, kernel, eps, ns, sp,
                     _p(acc[0]), _p(acc[1]), _p(acc[2]), pot.ctypes.data_as(_vp))
    return acc, pot


def diagnostics(pos, vel, mass, pot=None):
    """Conservation diagnostics (Sec. 3.2): [P (3), L = sum m x cross v (3), E = sum m v^2/2 + sum m phi/2]."""
    pos = _f64(pos)
    vel = _f64(vel)
    mass = _f64(mass)
    out = np.zeros(7)
    pot = None if pot is None else _f64(pot)
    pp = None if pot is None else pot.ctypes.data_as(_vp)
    lib().orc_diagnostics(mass.shape[0], _p(pos[0]), _p(pos[1]), _p(pos[2]), _p(vel[0]), _p(vel[1]), _p(vel[2]),
                          _p(mass), pp, _p(out))
    return out


def root_cube(pos):
    pos = _f64(pos)
    lo = np.zeros(3)
    L = C.c_double()
    lib().orc_root_cube(pos.shape[1], _p(pos[0]), _p(pos[1]), _p(pos[2]), _p(lo), C.byref(L))
    return lo, L.value


def morton_keys(pos, lo, L):
    pos = _f64(pos)
    lo = _f64(lo)
    keys = np.zeros(pos.shape[1], dtype=np.uint64)
    lib().orc_morton_keys(pos.shape[1], _p(pos[0]), _p(pos[1]), _p(pos[2]), _p(lo), L, _p(keys, _u64))
    return keys


def sort_keys(keys):
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    perm = np.zeros(keys.shape[0], dtype=np.int64)
    lib().orc_sort_keys(keys.shape[0], _p(keys, _u64), _p(perm, _i64))
    return perm


class Tree:
    """Octree + Algorithm 4 lists of one evaluation (cells in BFS order)."""

    def __init__(self, pos, prm: Params):
        pos = _f64(pos)
        self._prm = prm
        self.n = pos.shape[1]
        self._h = lib().orc_tree_build(self.n, _p(pos[0]), _p(pos[1]), _p(pos[2]), C.byref(prm))
        nc = lib().orc_tree_ncell(self._h)
        self.ncell = nc
        self.level = np.zeros(nc, np.int32)
        self.coords = np.zeros((3, nc), np.int64)
        self.first = np.zeros(nc, np.int64)
        self.count = np.zeros(nc, np.int64)
        self.child_first = np.zeros(nc, np.int64)
        self.nchild = np.zeros(nc, np.int32)
        lib().orc_tree_cells(self._h, _p(self.level, _i32), _p(self.coords[0], _i64), _p(self.coords[1], _i64),
                             _p(self.coords[2], _i64), _p(self.first, _i64), _p(self.count, _i64),
                             _p(self.child_first, _i64), _p(self.nchild, _i32))
        self.perm = np.zeros(self.n, np.int64)
        self.keys = np.zeros(self.n, np.uint64)
        lib().orc_tree_perm(self._h, _p(self.perm, _i64), _p(self.keys, _u64))
        self.lo = np.zeros(3)
        L = C.c_double()
        lib().orc_tree_geometry(self._h, _p(self.lo), C.byref(L))
        self.L = L.value

    def lists(self):
        nm, npp = C.c_int64(), C.c_int64()
        lib().orc_tree_walk(self._h, C.byref(nm), C.byref(npp))
        m2l = np.zeros((2, nm.value), np.int64)
        p2p = np.zeros((2, npp.value), np.int64)
        lib().orc_tree_lists(self._h, _p(m2l[0], _i64), _p(m2l[1], _i64), _p(p2p[0], _i64), _p(p2p[1], _i64))
        return m2l, p2p

    def radii(self):
        r = np.zeros(self.ncell)
        lib().orc_tree_radii(self._h, _p(r))
        return r

    def well_separated(self, a, b) -> bool:
        return bool(lib().orc_well_separated(self._h, int(a), int(b)))

    def centre(self, c):
        side = self.L / 2.0 ** self.level[c]
        return self.lo + (self.coords[:, c] + 0.5) * side

    def side(self, c):
        return self.L / 2.0 ** self.level[c]

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_tree_free(h)
            self._h = None


def p2m(p, pos, mass, zc):
    pos = _f64(pos)
    mass = _f64(mass)
    zc = _f64(zc)
    M = np.zeros(num_coeffs(p))
    lib().orc_p2m(p, pos.shape[1], _p(pos[0]), _p(pos[1]), _p(pos[2]), _p(mass), _p(zc), _p(M))
    return M


def m2m(p, Mc, delta):
    Mc = _f64(Mc)
    delta = _f64(delta)
    Mp = np.zeros(num_coeffs(p))
    lib().orc_m2m(p, _p(Mc), _p(delta), _p(Mp))
    return Mp


def m2l(p, MB, d, kernel=WENDLAND_C2, eps=0.0):
    MB = _f64(MB)
    d = _f64(d)
    LA = np.zeros(num_coeffs(p))
    lib().orc_m2l(p, _p(MB), _p(d), kernel, eps, _p(LA))
    return LA


def l2l(p, Lp, delta):
    Lp = _f64(Lp)
    delta = _f64(delta)
    Lc = np.zeros(num_coeffs(p))
    lib().orc_l2l(p, _p(Lp), _p(delta), _p(Lc))
    return Lc


def l2p(p, Lc, rho):
    Lc = _f64(Lc)
    rho = _f64(rho)
    phi = C.c_double()
    a = np.zeros(3)
    lib().orc_l2p(p, _p(Lc), _p(rho), C.byref(phi), _p(a))
    return phi.value, a


def fmm(pos, mass, prm: Params, is_fast=None):
    """Full evaluation; returns (acc (3, n), pot (n,))."""
    pos = _f64(pos)
    mass = _f64(mass)
    n = mass.shape[0]
    fast, fast_p = _opt_u8(is_fast)
    acc = np.zeros((3, n))
    pot = np.zeros(n)
    rc = lib().orc_fmm(n, _p(pos[0]), _p(pos[1]), _p(pos[2]), _p(mass), fast_p, C.byref(prm),
                       _p(acc[0]), _p(acc[1]), _p(acc[2]), pot.ctypes.data_as(_vp))
    if rc != 0:
        raise ValueError(f"orc_fmm failed ({rc})")
    return acc, pot


def fmm_sample(pos, mass, prm: Params, sample, is_fast=None):
    """Evaluation for the listed sinks only; returns (acc (3, ns), pot (ns,))."""
    pos = _f64(pos)
    mass = _f64(mass)
    n = mass.shape[0]
    sample = np.ascontiguousarray(sample, dtype=np.int64)
    fast, fast_p = _opt_u8(is_fast)
    ns = sample.shape[0]
    acc = np.zeros((3, ns))
    pot = np.zeros(ns)
    rc = lib().orc_fmm_sample(n, _p(pos[0]), _p(pos[1]), _p(pos[2]), _p(mass), fast_p, C.byref(prm), ns,
                              _p(sample, _i64), _p(acc[0]), _p(acc[1]), _p(acc[2]), pot.ctypes.data_as(_vp))
    if rc != 0:
        raise ValueError(f"orc_fmm_sample failed ({rc})")
    return acc, pot


def timestep(eta, eps, a_old, a_cur) -> float:
    return lib().orc_timestep(eta, eps, a_old, a_cur)


def timestep_tot(eta, eps, a_old, a_cur, eta_tot, a_tot) -> float:
    return lib().orc_timestep_tot(eta, eps, a_old, a_cur, eta_tot, a_tot)


def rung(dt_i, dt_max, k_max) -> int:
    return lib().orc_rung(dt_i, dt_max, k_max)


class HHS:
    """State of one HOLD-integrated system (Algorithms 1-3) on the oracle."""

    def __init__(self, pos, vel, mass, prm: Params, eta=0.025, dt_max=1.0 / 64, k_max=10, eta_tot=0.0):
        self.pos = np.array(pos, dtype=np.float64, order="C")
        self.vel = np.array(vel, dtype=np.float64, order="C")
        self.mass = _f64(mass).copy()
        self.n = self.mass.shape[0]
        self.prm = prm
        self.hp = HHSParams(eta=eta, dt_max=dt_max, k_max=k_max, eta_tot=eta_tot)
        self.a_old = np.zeros(self.n)
        self.a_cur = np.zeros(self.n)
        self.a_tot = np.zeros(self.n)
        self.rung = np.zeros(self.n, np.int32)
        self.t = 0.0
        p = self.pos
        rc = lib().orc_hhs_init(self.n, _p(p[0]), _p(p[1]), _p(p[2]), _p(self.mass), C.byref(prm),
                                _p(self.a_old), _p(self.a_cur), _p(self.a_tot))
        if rc != 0:
            raise ValueError("orc_hhs_init failed")

    def step(self, trace_cap=0):
        stats = HHSStats()
        trace = np.zeros((max(trace_cap, 1), 4), np.int64)
        p, v = self.pos, self.vel
        rc = lib().orc_hhs_step(self.n, _p(p[0]), _p(p[1]), _p(p[2]), _p(v[0]), _p(v[1]), _p(v[2]),
                                _p(self.mass), C.byref(self.prm), C.byref(self.hp), _p(self.a_old),
                                _p(self.a_cur), _p(self.a_tot), _p(self.rung, _i32), C.byref(stats),
                                trace.ctypes.data_as(_vp) if trace_cap > 0 else None, trace_cap)
        if rc != 0:
            raise ValueError("orc_hhs_step failed")
        self.t += self.hp.dt_max
        return stats, trace[: stats.trace_len]

    def diagnostics(self, pot=None):
        if pot is None:
            _, pot = fmm(self.pos, self.mass, self.prm)
        out = np.zeros(7)
        p, v = self.pos, self.vel
        lib().orc_diagnostics(self.n, _p(p[0]), _p(p[1]), _p(p[2]), _p(v[0]), _p(v[1]), _p(v[2]),
                              _p(self.mass), pot.ctypes.data_as(_vp), _p(out))
        return out


class Traditional:
    """The traditional individual-timestep integrator of Sec. 2.3 on the oracle (block steps,
    kick-drift-kick per particle, forces on the active particles from all masses at unsynchronised
    positions)."""

    def __init__(self, pos, vel, mass, prm: Params, eta=0.025, dt_max=1.0 / 64, k_max=10):
        self.pos = np.array(pos, dtype=np.float64, order="C")
        self.vel = np.array(vel, dtype=np.float64, order="C")
        self.mass = _f64(mass).copy()
        self.n = self.mass.shape[0]
        self.prm = prm
        self.hp = HHSParams(eta=eta, dt_max=dt_max, k_max=k_max, eta_tot=0.0)
        self.acc = np.zeros((3, self.n))
        self.rung = np.zeros(self.n, np.int32)
        p = self.pos
        if lib().orc_trad_init(self.n, _p(p[0]), _p(p[1]), _p(p[2]), _p(self.mass), C.byref(prm), C.byref(self.hp),
                               _p(self.acc), _p(self.rung, _i32)) != 0:
            raise ValueError("orc_trad_init failed")

    def step(self):
        stats = HHSStats()
        p, v = self.pos, self.vel
        if lib().orc_trad_step(self.n, _p(p[0]), _p(p[1]), _p(p[2]), _p(v[0]), _p(v[1]), _p(v[2]), _p(self.mass),
                               C.byref(self.prm), C.byref(self.hp), _p(self.acc), _p(self.rung, _i32),
                               C.byref(stats)) != 0:
            raise ValueError("orc_trad_step failed")
        return stats


def num_threads() -> int:
    return lib().orc_num_threads()
