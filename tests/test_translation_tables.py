"""The generated translation term lists that the M2M and L2L kernels read (csrc/tg_tables.cuh), checked
on the CPU against the definitions of the expansions (Sec. 2.1), not against the generator.

Expansions are stored normalised by the cell side s:  M~^j = sum_i m_i ((x_i - z)/s)^j  and
phi(x) = (1/s) sum_n L~^n ((x - z)/s)^n / n!.  A child's centre lies at z_P + sigma s_P/4 with
sigma in {-1, +1}^3.  M2M must reproduce the parent's moments of the child's particles exactly (a
moment of total degree n only needs child moments of degree <= n); L2L must re-expand a local
polynomial of degree p about the child's centre exactly.  Each list entry packs the coefficient
index (low 8 bits) and the parity of the offset power (bit a set: its a component is odd, and the
term changes sign when that component of sigma is negative).
"""
import itertools
import os
import re
from math import factorial

import numpy as np
import pytest

TABLES = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1712_10116_gb300", "csrc",
                      "tg_tables.cuh")
SIGMAS = list(itertools.product((-1, 1), repeat=3))


def _array(text, name):
    m = re.search(r"\b" + name + r"\[(\d+)\] = \{([^}]*)\}", text)
    assert m, name
    vals = [v.strip() for v in m.group(2).split(",")]
    assert len(vals) == int(m.group(1))
    if any("0x" in v and "p" in v for v in vals):
        return np.array([float.fromhex(v.rstrip("f")) for v in vals])
    return np.array([int(v) for v in vals])


@pytest.fixture(scope="module")
def tab():
    text = open(TABLES).read()
    t = {k: _array(text, k) for k in ("c_mi_x", "c_mi_y", "c_mi_z", "g_m2m_off", "g_m2m_kp", "g_m2m_cd", "g_m2m_cf",
                                      "g_l2l_off", "g_l2l_kp", "g_l2l_cd", "g_l2l_cf")}
    t["mi"] = np.stack([t["c_mi_x"], t["c_mi_y"], t["c_mi_z"]], axis=1)
    return t


def _sign(kp, sigma):
    neg = sum(1 << a for a in range(3) if sigma[a] < 0)
    return -1.0 if bin((int(kp) >> 8) & neg).count("1") & 1 else 1.0


def _moments(x, m, z, s, mi):
    u = (x - z[:, None]) / s
    return np.array([(m * u[0] ** a * u[1] ** b * u[2] ** c).sum() for a, b, c in mi])


def test_multi_index_order(tab):
    # total degree, then n_x descending, then n_y descending: the coefficients of degree <= p come first
    mi = [tuple(r) for r in tab["mi"]]
    assert len(mi) == len(set(mi)) == 165
    assert mi == sorted(mi, key=lambda v: (sum(v), -v[0], -v[1]))
    for p in range(9):
        assert sum(1 for v in mi if sum(v) <= p) == (p + 1) * (p + 2) * (p + 3) // 6


@pytest.mark.parametrize("prec", ["cd", "cf"])
def test_m2m_list_is_the_exact_translation(tab, prec):
    rng = np.random.default_rng(5)
    mi, off, kp, coef = tab["mi"], tab["g_m2m_off"], tab["g_m2m_kp"], tab["g_m2m_" + prec]
    sP = 2.0
    zP = np.array([0.3, -0.7, 1.1])
    for sigma in SIGMAS:
        zc = zP + np.array(sigma) * sP / 4
        x = zc[:, None] + rng.uniform(-sP / 4, sP / 4, (3, 40))
        m = rng.uniform(0.5, 1.5, 40)
        Mc = _moments(x, m, zc, sP / 2, mi)
        Mp = _moments(x, m, zP, sP, mi)
        out = np.array([sum(_sign(kp[i], sigma) * coef[i] * Mc[kp[i] & 0xff] for i in range(off[n], off[n + 1]))
                        for n in range(len(mi))])
        # float coefficients are exact (products of binomials and powers of two)
        assert np.allclose(out, Mp, rtol=1e-12, atol=1e-12 * np.abs(Mp).max()), sigma
    assert np.array_equal(tab["g_m2m_cf"], tab["g_m2m_cd"])


@pytest.mark.parametrize("p", [4, 6, 8])
@pytest.mark.parametrize("prec", ["cd", "cf"])
def test_l2l_list_reexpands_a_local_polynomial_exactly(tab, p, prec):
    rng = np.random.default_rng(11 + p)
    mi, off, kp, coef = tab["mi"], tab["g_l2l_off"], tab["g_l2l_kp"], tab["g_l2l_" + prec]
    nfact = np.array([factorial(a) * factorial(b) * factorial(c) for a, b, c in mi], dtype=float)
    nc = (p + 1) * (p + 2) * (p + 3) // 6
    sP = 4.0
    zP = np.array([-1.0, 0.5, 2.0])
    LP = np.zeros(len(mi))
    LP[:nc] = rng.standard_normal(nc)

    def phi(L, z, s, x, order):
        u = (x - z[:, None]) / s
        terms = [L[i] * u[0] ** a * u[1] ** b * u[2] ** c / nfact[i] for i, (a, b, c) in enumerate(mi)
                 if a + b + c <= order]
        return np.sum(terms, axis=0) / s

    for sigma in SIGMAS:
        zc = zP + np.array(sigma) * sP / 4
        Lc = np.zeros(len(mi))
        for n in range(nc):
            # order p takes the first (p - |n| + 1)(p - |n| + 2)(p - |n| + 3)/6 terms of the order-8 list of n
            q = p - int(mi[n].sum())
            cnt = (q + 1) * (q + 2) * (q + 3) // 6
            assert off[n] + cnt <= off[n + 1]
            Lc[n] = sum(_sign(kp[i], sigma) * coef[i] * LP[kp[i] & 0xff] for i in range(off[n], off[n] + cnt))
            for i in range(off[n], off[n] + cnt):
                assert int(mi[kp[i] & 0xff].sum()) <= p
        x = zc[:, None] + rng.uniform(-sP / 4, sP / 4, (3, 25))
        ref = phi(LP, zP, sP, x, p)
        got = phi(Lc, zc, sP / 2, x, p)
        # float: 1/d! is rounded to float as the float expansions use it
        tol = 1e-12 if prec == "cd" else 1e-6
        assert np.allclose(got, ref, rtol=tol, atol=tol * np.abs(ref).max()), (sigma, np.abs(got - ref).max())
