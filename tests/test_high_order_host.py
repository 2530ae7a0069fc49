"""Index arithmetic and harmonic fold / completion of the high-order expansion kernels (p up to 20),
checked on the host.

The header they live in is compiled with g++ (device qualifiers mapped to host ones).  The multi-index
order must match the total-degree order used everywhere else; the fold of the moments followed by the
reduced contraction and the completion of the locals must reproduce the full contraction
L^n = sum_j M^j D^{n+j} with the derivative tensor of 1/r taken from the oracle.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1712_10116_gb300", "csrc")

HARNESS = r"""
#define __host__
#define __device__
#define __forceinline__ inline
#include "high_order.cuh"
extern "C" int hi_index_c(int x, int y, int z) { return tg::hi_index(x, y, z); }
extern "C" void hi_decode_c(int k, int *x, int *y, int *z) { tg::hi_decode(k, *x, *y, *z); }
extern "C" void fold_c(const double *src, double *dst, int p, int ncp) { tg::hi_fold_row<double>(src, dst, p, ncp); }
extern "C" void complete_c(double *row, int p) { tg::hi_complete_row<double>(row, p); }
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("hi_host")
    (d / "h.cpp").write_text(HARNESS)
    so = d / "libhi.so"
    subprocess.run([gxx, "-O1", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", "-I", CSRC,
                    str(d / "h.cpp"), "-o", str(so)], check=True)
    lib = ctypes.CDLL(str(so))
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    lib.hi_index_c.argtypes = [ctypes.c_int] * 3
    lib.hi_decode_c.argtypes = [ctypes.c_int, ip, ip, ip]
    lib.fold_c.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int]
    lib.complete_c.argtypes = [dp, ctypes.c_int]
    return lib


def _order(p):
    # total degree, then x descending, then y descending
    return [(nx, o - nx - nz, nz) for o in range(p + 1) for nx in range(o, -1, -1) for nz in range(0, o - nx + 1)]


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def test_index_and_decode_follow_the_degree_order(lib):
    mi = _order(20)
    assert mi == [tuple(v) for v in oracle.multi_indices(20).tolist()]
    x, y, z = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    for k, (a, b, c) in enumerate(mi):
        assert lib.hi_index_c(a, b, c) == k
        lib.hi_decode_c(k, ctypes.byref(x), ctypes.byref(y), ctypes.byref(z))
        assert (x.value, y.value, z.value) == (a, b, c)


@pytest.mark.parametrize("p", [9, 14, 20])
def test_fold_and_completion_reproduce_the_full_contraction(lib, p):
    mi = _order(p)
    idx = {v: k for k, v in enumerate(mi)}
    nc = len(mi)
    D = oracle.dtensor(p, np.array([2.3, -1.1, 0.7]))          # derivatives of -1/r, harmonic
    omi = [tuple(v) for v in oracle.multi_indices(p).tolist()]
    Dt = {v: D[k] for k, v in enumerate(omi)}
    rng = np.random.default_rng(p)
    M = rng.uniform(-1.0, 1.0, nc)
    full = np.zeros(nc)
    for n, (nx, ny, nz) in enumerate(mi):
        for j, (jx, jy, jz) in enumerate(mi):
            if nx + ny + nz + jx + jy + jz <= p:
                full[n] += M[j] * Dt[(nx + jx, ny + jy, nz + jz)]
    Mf = np.zeros(nc)
    lib.fold_c(_dp(M), _dp(Mf), p, nc)
    assert all(Mf[k] == 0.0 for k, v in enumerate(mi) if v[2] >= 2)
    red = np.zeros(nc)
    for n, (nx, ny, nz) in enumerate(mi):
        if nz > 1:
            continue
        for j, (jx, jy, jz) in enumerate(mi):
            if jz <= 1 and nx + ny + nz + jx + jy + jz <= p:
                red[n] += Mf[j] * Dt[(nx + jx, ny + jy, nz + jz)]
    lib.complete_c(_dp(red), p)
    # an error in the algebra would be of order one; what is left is float64 rounding, which the
    # completion amplifies for large n_z (a coefficient becomes a long alternating sum of larger
    # ones): 3e-14 of the largest coefficient at p = 9, 9e-13 at p = 14, 4e-10 at p = 20 with these
    # unscaled random moments
    assert np.abs(red - full).max() < 1e-8 * np.abs(full).max()
