"""The harmonic M2L set of the generated float32 contractions, checked on the host.

For G = -1/|d| the derivative tensor is harmonic, so moments with j_z >= 2 can be folded onto lower
components and the locals with n_z >= 2 follow from those with n_z <= 1.  The generated header is
compiled with g++ (device qualifiers mapped to host ones) and the harmonic path (fold, reduced
contraction, completion) is compared with the full contraction on random offsets and moments, for
both sides, with and without the potential term, p = 1..6.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1712_10116_gb300", "csrc")

HARNESS = r"""
#include <cmath>
#define __device__
#define __forceinline__ inline
#define __restrict__
static inline float __ldg(const float *p) { return *p; }
static inline float rsqrtf(float x) { return 1.0f / std::sqrt(x); }
#include "m2l_gen.cuh"

template <int P>
static void run(const float *d, const float *Ms, float rho, int pot, float *La_full, float *Lb_full, float *La_h, float *Lb_h)
{
    constexpr int NC = M2LGen<P>::NC, NH = M2LGenH<P>::NC, ND = M2LGenH<P>::ND;
    float D[NC], La[NC], Lb[NC];
    M2LGen<P>::dtensor(d[0], d[1], d[2], 0.0f, D);
    if (pot) { M2LGen<P>::side_a(D, Ms, rho, La); M2LGen<P>::side_b(D, Ms, Lb); }
    else { M2LGen<P>::side_a_forces(D, Ms, rho, La); M2LGen<P>::side_b_forces(D, Ms, Lb); }
    for (int k = 0; k < NC; ++k) { La_full[k] = La[k]; Lb_full[k] = Lb[k]; }
    float Dh[ND], Mr[NH], Ra[NH], Rb[NH];
    M2LGenH<P>::reduce_moments(Ms, Mr);
    M2LGenH<P>::dtensor(d[0], d[1], d[2], Dh);
    if (pot) { M2LGenH<P>::side_a(Dh, Mr, rho, Ra); M2LGenH<P>::side_b(Dh, Mr, Rb); }
    else { M2LGenH<P>::side_a_forces(Dh, Mr, rho, Ra); M2LGenH<P>::side_b_forces(Dh, Mr, Rb); }
    M2LGenH<P>::complete_locals(Ra, La_h);
    M2LGenH<P>::complete_locals(Rb, Lb_h);
}

extern "C" int m2l_host(int p, const float *d, const float *Ms, float rho, int pot, float *a, float *b, float *ah, float *bh)
{
    switch (p) {
    case 1: run<1>(d, Ms, rho, pot, a, b, ah, bh); return 0;
    case 2: run<2>(d, Ms, rho, pot, a, b, ah, bh); return 0;
    case 3: run<3>(d, Ms, rho, pot, a, b, ah, bh); return 0;
    case 4: run<4>(d, Ms, rho, pot, a, b, ah, bh); return 0;
    case 5: run<5>(d, Ms, rho, pot, a, b, ah, bh); return 0;
    case 6: run<6>(d, Ms, rho, pot, a, b, ah, bh); return 0;
    }
    return 1;
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("m2l_host")
    src = d / "harness.cpp"
    src.write_text(HARNESS)
    so = d / "libm2lhost.so"
    subprocess.run([gxx, "-O1", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", "-I", CSRC, str(src), "-o", str(so)],
                   check=True)
    lib = ctypes.CDLL(str(so))
    f = ctypes.POINTER(ctypes.c_float)
    lib.m2l_host.argtypes = [ctypes.c_int, f, f, ctypes.c_float, ctypes.c_int, f, f, f, f]
    return lib


def _ncoef(p):
    return (p + 1) * (p + 2) * (p + 3) // 6


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("pot", [1, 0])
def test_harmonic_set_equals_full_contraction(lib, p, pot):
    rng = np.random.default_rng(1000 + 10 * p + pot)
    nc = _ncoef(p)
    worst = 0.0
    for trial in range(200):
        # a well-separated offset in units of the x cell (|d| between 2 and 6) and O(1) moments
        d = rng.normal(size=3)
        d *= rng.uniform(2.0, 6.0) / np.linalg.norm(d)
        d = d.astype(np.float32)
        Ms = rng.uniform(-1.0, 1.0, size=nc).astype(np.float32)
        rho = np.float32([0.5, 1.0, 2.0][trial % 3])
        out = [np.zeros(nc, np.float32) for _ in range(4)]
        assert lib.m2l_host(p, _ptr(d), _ptr(Ms), rho, pot, *map(_ptr, out)) == 0
        a, b, ah, bh = (o.astype(np.float64) for o in out)
        for full, harm in ((a, ah), (b, bh)):
            scale = np.abs(full).max()
            worst = max(worst, np.abs(full - harm).max() / scale)
            if not pot:
                assert harm[0] == 0.0
    # identical in exact arithmetic: only float32 rounding (two evaluation orders) separates them
    assert worst < 2e-5, worst


def test_harmonic_fold_leaves_harmonic_moments_alone(lib):
    # a moment set that is already supported on j_z <= 1 passes the fold unchanged, so the two
    # contractions see the same numbers and agree to rounding on every coefficient
    p = 4
    nc = _ncoef(p)
    mi = [(nx, ny, o - nx - ny) for o in range(p + 1) for nx in range(o, -1, -1) for ny in range(o - nx, -1, -1)]
    rng = np.random.default_rng(7)
    Ms = np.array([rng.uniform(-1, 1) if k[2] <= 1 else 0.0 for k in mi], np.float32)
    d = np.array([3.0, -1.0, 2.0], np.float32)
    out = [np.zeros(nc, np.float32) for _ in range(4)]
    lib.m2l_host(p, _ptr(d), _ptr(Ms), np.float32(1.0), 1, *map(_ptr, out))
    a, _, ah, _ = out
    assert np.allclose(ah, a, rtol=1e-5, atol=1e-6 * np.abs(a).max())
