"""The generated float32 M2L code (csrc/m2l_gen.cuh), compiled on the host with g++, against the M2L
definitions written out in float64 from symbolic derivatives (Sec. 2.1, Eq. 2).

Definitions (multi-indices of total degree <= p, Ms^j = M^j / j!):
  D^k(d)  = d^k/dd^k G(d),  G = -(|d|^2 + soft2)^(-1/2)        (derivatives by sympy, not a recurrence)
  side a:   L^n = sum_{|n|+|j| <= p} (-1)^|j| rho^|j| Ms^j D^{n+j}
  side b:   L^n = (-1)^|n| sum_{|n|+|j| <= p} Ms^j D^{n+j}
  forces:   the same with L^0 = 0 (the potential term)
  directed: L^n += side a (harmonic set, one source after another)
The harmonic set (soft2 = 0 only) folds the moments, contracts the (p+1)^2 components with j_z <= 1 and
completes the locals; its output must equal the definition too.  A wrong index, sign, power of rho or
dropped term in the generated code fails these comparisons.
"""
import ctypes
import functools
import os
import shutil
import subprocess
from math import factorial

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

// mode 0: full set (dtensor with soft2, side a, side b); mode 1: harmonic set (fold, contract, complete);
// mode 2: harmonic directed accumulation of two sources into one target
template <int P>
static void run(int mode, int forces, const float *d, float soft2, const float *Ms, const float *Ms2, float rho,
                float *La, float *Lb)
{
    constexpr int NC = M2LGen<P>::NC, NH = M2LGenH<P>::NC, ND = M2LGenH<P>::ND;
    if (mode == 0) {
        float D[NC], A[NC], B[NC];
        M2LGen<P>::dtensor(d[0], d[1], d[2], soft2, D);
        if (forces) { M2LGen<P>::side_a_forces(D, Ms, rho, A); M2LGen<P>::side_b_forces(D, Ms, B); }
        else { M2LGen<P>::side_a(D, Ms, rho, A); M2LGen<P>::side_b(D, Ms, B); }
        for (int k = 0; k < NC; ++k) { La[k] = A[k]; Lb[k] = B[k]; }
        return;
    }
    float Dh[ND], Mr[NH], Ra[NH], Rb[NH];
    M2LGenH<P>::reduce_moments(Ms, Mr);
    M2LGenH<P>::dtensor(d[0], d[1], d[2], Dh);
    if (mode == 1) {
        if (forces) { M2LGenH<P>::side_a_forces(Dh, Mr, rho, Ra); M2LGenH<P>::side_b_forces(Dh, Mr, Rb); }
        else { M2LGenH<P>::side_a(Dh, Mr, rho, Ra); M2LGenH<P>::side_b(Dh, Mr, Rb); }
        M2LGenH<P>::complete_locals(Ra, La);
        M2LGenH<P>::complete_locals(Rb, Lb);
        return;
    }
    // two sources at offsets d and -d (the second with moments Ms2) into one target's reduced locals
    float Mr2[NH], Dh2[ND];
    M2LGenH<P>::reduce_moments(Ms2, Mr2);
    M2LGenH<P>::dtensor(-d[0], -d[1], -d[2], Dh2);
    for (int k = 0; k < NH; ++k) Ra[k] = 0.0f;
    if (forces) { M2LGenH<P>::acc_forces(Dh, Mr, rho, Ra); M2LGenH<P>::acc_forces(Dh2, Mr2, rho, Ra); }
    else { M2LGenH<P>::acc(Dh, Mr, rho, Ra); M2LGenH<P>::acc(Dh2, Mr2, rho, Ra); }
    M2LGenH<P>::complete_locals(Ra, La);
}

extern "C" int m2l_gen_host(int p, int mode, int forces, const float *d, float soft2, const float *Ms, const float *Ms2,
                            float rho, float *La, float *Lb)
{
    switch (p) {
    case 1: run<1>(mode, forces, d, soft2, Ms, Ms2, rho, La, Lb); return 0;
    case 2: run<2>(mode, forces, d, soft2, Ms, Ms2, rho, La, Lb); return 0;
    case 3: run<3>(mode, forces, d, soft2, Ms, Ms2, rho, La, Lb); return 0;
    case 4: run<4>(mode, forces, d, soft2, Ms, Ms2, rho, La, Lb); return 0;
    case 5: run<5>(mode, forces, d, soft2, Ms, Ms2, rho, La, Lb); return 0;
    case 6: run<6>(mode, forces, d, soft2, Ms, Ms2, rho, La, Lb); return 0;
    }
    return 1;
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("m2l_gen_host")
    src = d / "harness.cpp"
    src.write_text(HARNESS)
    so = d / "libm2lgen.so"
    subprocess.run([gxx, "-O1", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", "-I", CSRC, str(src), "-o", str(so)],
                   check=True)
    lib = ctypes.CDLL(str(so))
    f = ctypes.POINTER(ctypes.c_float)
    lib.m2l_gen_host.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, f, ctypes.c_float, f, f, ctypes.c_float, f, f]
    return lib


def _mi(p):
    return [(nx, ny, o - nx - ny) for o in range(p + 1) for nx in range(o, -1, -1) for ny in range(o - nx, -1, -1)]


@functools.lru_cache(maxsize=None)
def _dfuncs(p):
    sp = pytest.importorskip("sympy")
    x, y, z, s2 = sp.symbols("x y z s2", real=True)
    G = -1 / sp.sqrt(x ** 2 + y ** 2 + z ** 2 + s2)
    out = {}
    for k in _mi(p):
        expr = G
        for var, cnt in zip((x, y, z), k):
            if cnt:
                expr = sp.diff(expr, var, cnt)
        out[k] = sp.lambdify((x, y, z, s2), expr, "math")
    return out


def _reference(p, d, soft2, Ms, rho, forces):
    mi = _mi(p)
    idx = {v: i for i, v in enumerate(mi)}
    fn = _dfuncs(p)
    D = {k: fn[k](float(d[0]), float(d[1]), float(d[2]), float(soft2)) for k in mi}
    La = np.zeros(len(mi))
    Lb = np.zeros(len(mi))
    for n in mi:
        for j in mi:
            if sum(n) + sum(j) > p:
                continue
            k = (n[0] + j[0], n[1] + j[1], n[2] + j[2])
            t = float(Ms[idx[j]]) * D[k]
            La[idx[n]] += (-1) ** sum(j) * float(rho) ** sum(j) * t
            Lb[idx[n]] += (-1) ** sum(n) * t
    if forces:
        La[0] = Lb[0] = 0.0
    return La, Lb


def _harmonic_moments(p, rng):
    # moments of point masses about the cell centre (Ms = M / j!): a real multipole, whose trace parts
    # the harmonic fold may move without changing any local
    mi = _mi(p)
    x = rng.uniform(-0.5, 0.5, (3, 6))
    m = rng.uniform(0.2, 1.0, 6)
    return np.array([(m * x[0] ** a * x[1] ** b * x[2] ** c).sum() / (factorial(a) * factorial(b) * factorial(c))
                     for a, b, c in mi], np.float32)


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _call(lib, p, mode, forces, d, soft2, Ms, Ms2, rho):
    nc = len(_mi(p))
    La = np.zeros(nc, np.float32)
    Lb = np.zeros(nc, np.float32)
    assert lib.m2l_gen_host(p, mode, forces, _ptr(d), np.float32(soft2), _ptr(Ms), _ptr(Ms2), np.float32(rho),
                            _ptr(La), _ptr(Lb)) == 0
    return La.astype(np.float64), Lb.astype(np.float64)


def _close(got, ref, tol=3e-5):
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= tol * scale, (np.abs(got - ref).max() / scale)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("forces", [0, 1])
@pytest.mark.parametrize("soft2", [0.0, 0.7])
def test_full_set_matches_the_definition(lib, p, forces, soft2):
    rng = np.random.default_rng(100 * p + 10 * forces + int(soft2 * 10))
    nc = len(_mi(p))
    for trial in range(4):
        d = rng.normal(size=3)
        d = (d * rng.uniform(2.0, 5.0) / np.linalg.norm(d)).astype(np.float32)
        Ms = rng.uniform(-1.0, 1.0, nc).astype(np.float32)
        rho = np.float32([0.5, 1.0, 2.0, 1.0][trial])
        La, Lb = _call(lib, p, 0, forces, d, soft2, Ms, Ms, rho)
        ra, rb = _reference(p, d, soft2, Ms, rho, forces)
        _close(La, ra)
        _close(Lb, rb)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("forces", [0, 1])
def test_harmonic_set_matches_the_definition(lib, p, forces):
    rng = np.random.default_rng(500 + 10 * p + forces)
    for trial in range(4):
        d = rng.normal(size=3)
        d = (d * rng.uniform(2.0, 5.0) / np.linalg.norm(d)).astype(np.float32)
        Ms = _harmonic_moments(p, rng)
        rho = np.float32([0.5, 1.0, 2.0, 1.0][trial])
        La, Lb = _call(lib, p, 1, forces, d, 0.0, Ms, Ms, rho)
        ra, rb = _reference(p, d, 0.0, Ms, rho, forces)
        _close(La, ra)
        _close(Lb, rb)


@pytest.mark.parametrize("p", [2, 4, 6])
@pytest.mark.parametrize("forces", [0, 1])
def test_harmonic_directed_accumulation_matches_the_definition(lib, p, forces):
    rng = np.random.default_rng(900 + p + forces)
    d = np.array([2.5, -1.5, 3.0], np.float32)
    Ms, Ms2 = _harmonic_moments(p, rng), _harmonic_moments(p, rng)
    rho = np.float32(0.5)
    La, _ = _call(lib, p, 2, forces, d, 0.0, Ms, Ms2, rho)
    r1, _ = _reference(p, d, 0.0, Ms, rho, forces)
    r2, _ = _reference(p, -d, 0.0, Ms2, rho, forces)
    _close(La, r1 + r2)
