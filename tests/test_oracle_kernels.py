"""Pins of the oracle's pair kernels and derivative tensors against mathematics the paper fixes.

Wendland C2 softening, Eq. (8) Sec. 2.3; Plummer softening; Taylor derivative tensors of
G = -1/r used by the cell-cell interaction of Sec. 2.1.
"""
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _phi(kernel, eps, r):
    return oracle.softened(kernel, eps, r)[0]


def _g(kernel, eps, r):
    return oracle.softened(kernel, eps, r)[1]


def test_wendland_matches_printed_nested_form():
    # the coefficient table is read from the paper's nested form (Eq. 8), independent of the C code
    coef = {}
    for line in open(os.path.join(GOLDEN, "wendland_c2.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, c = line.split()
        coef[int(k)] = float(c)
    eps = 0.37
    for u in np.linspace(0.0, 0.999, 37):
        want = sum(c * u ** k for k, c in coef.items()) / eps
        assert _phi(oracle.WENDLAND_C2, eps, u * eps) == pytest.approx(want, rel=1e-13, abs=1e-13)


@pytest.mark.parametrize("eps", [0.005, 0.02, 1.0])
def test_wendland_c2_continuity_at_eps(eps):
    # C2 match to the Newtonian -1/r at r = eps: phi = -1/eps, phi' = 1/eps^2, phi'' = -2/eps^3
    k = oracle.WENDLAND_C2
    assert _phi(k, eps, eps * (1 - 1e-12)) == pytest.approx(-1.0 / eps, rel=1e-9)
    assert _phi(k, eps, eps) == pytest.approx(-1.0 / eps, rel=1e-15)
    # g = phi'/r is continuous: phi'(eps-) = 1/eps^2
    assert _g(k, eps, eps * (1 - 1e-12)) * eps == pytest.approx(1.0 / eps ** 2, rel=1e-9)
    # second derivative from below by a one-sided difference of phi' = r g
    h = 1e-5 * eps
    d1 = lambda r: r * _g(k, eps, r)
    phi2 = (d1(eps - h) - d1(eps - 2 * h)) / h
    assert phi2 == pytest.approx(-2.0 / eps ** 3, rel=1e-4)


def test_wendland_centre_value():
    eps = 0.01
    assert _phi(oracle.WENDLAND_C2, eps, 0.0) == pytest.approx(-3.0 / eps, rel=1e-15)
    assert _g(oracle.WENDLAND_C2, eps, 0.0) == pytest.approx(14.0 / eps ** 3, rel=1e-15)


def _density_from_potential(kernel, eps, r, h):
    # Poisson: 4 pi rho = (1/r^2) d/dr (r^2 phi'), with phi' = r g
    flux = lambda s: s * s * (s * _g(kernel, eps, s))
    return (flux(r + h) - flux(r - h)) / (2 * h) / (r * r) / (4 * math.pi)


def test_wendland_is_potential_of_wendland_c2_density():
    # Wendland (1995) C2 function (1-u)^4 (1+4u), normalised to unit mass: 21/(2 pi eps^3)
    eps = 0.3
    for u in [0.1, 0.25, 0.5, 0.7, 0.9]:
        r = u * eps
        rho = _density_from_potential(oracle.WENDLAND_C2, eps, r, 1e-5 * eps)
        want = 21.0 / (2.0 * math.pi * eps ** 3) * (1 - u) ** 4 * (1 + 4 * u)
        assert rho == pytest.approx(want, rel=1e-5)
    # vacuum outside eps, and unit enclosed mass r^2 phi'(r) = 1
    assert abs(_density_from_potential(oracle.WENDLAND_C2, eps, 1.5 * eps, 1e-5 * eps)) < 1e-4
    assert (1.2 * eps) ** 3 * _g(oracle.WENDLAND_C2, eps, 1.2 * eps) == pytest.approx(1.0, rel=1e-14)


def test_plummer_is_potential_of_plummer_density():
    eps = 0.2
    for u in [0.1, 0.5, 1.0, 2.0]:
        r = u * eps
        rho = _density_from_potential(oracle.PLUMMER, eps, r, 1e-5 * eps)
        want = 3.0 / (4.0 * math.pi * eps ** 3) * (1 + u * u) ** -2.5
        assert rho == pytest.approx(want, rel=1e-5)


def test_direct_is_antisymmetric_and_sums_to_zero():
    g = np.random.default_rng(3)
    pos = g.uniform(-1, 1, (3, 200))
    m = g.uniform(0.5, 2.0, 200)
    acc, _ = oracle.direct(pos, m, 0.05, oracle.WENDLAND_C2)
    assert np.abs((acc * m).sum(1)).max() <= 1e-14 * np.abs(acc * m).sum()
    # two particles: F_12 = -F_21 exactly (Eq. 2)
    p2 = np.array([[0.0, 0.3], [0.0, 0.1], [0.0, -0.2]])
    m2 = np.array([2.0, 0.5])
    a2, _ = oracle.direct(p2, m2, 0.05, oracle.PLUMMER)
    assert np.all(m2[0] * a2[:, 0] == -m2[1] * a2[:, 1])


def test_direct_plummer_sphere_mean_radial_acceleration():
    # mean radial acceleration in shells vs the Plummer model -r / (r^2 + 1)^(3/2) (G = M = a = 1)
    from paper_1712_10116_gb300 import ics
    pos, _, m = ics.plummer(4096, 1001)
    acc, pot = oracle.direct(pos, m, 1e-3, oracle.PLUMMER)
    r = np.linalg.norm(pos, axis=0)
    ar = (acc * pos).sum(0) / r
    for lo, hi in [(0.3, 0.5), (0.5, 0.8), (0.8, 1.2), (1.2, 2.0)]:
        sel = (r > lo) & (r < hi)
        want = -(r[sel] / (r[sel] ** 2 + 1) ** 1.5)
        assert np.mean(ar[sel]) == pytest.approx(np.mean(want), rel=0.05)
    # potential energy of the Plummer model: W = -3 pi / 32
    W = 0.5 * (m * pot).sum()
    assert W == pytest.approx(-3 * math.pi / 32, rel=0.03)


# ------------------------------------------------------------------ derivative tensors

def _mi(p):
    return oracle.multi_indices(p)


def _index(p):
    return {tuple(v): i for i, v in enumerate(_mi(p))}


def test_dtensor_low_order_closed_forms():
    d = np.array([0.3, -0.7, 1.1])
    x, y, z = d
    r = np.linalg.norm(d)
    D = oracle.dtensor(3, d)
    ix = _index(3)
    assert D[ix[(0, 0, 0)]] == pytest.approx(-1 / r, rel=1e-14)
    assert D[ix[(1, 0, 0)]] == pytest.approx(x / r ** 3, rel=1e-14)
    assert D[ix[(0, 0, 1)]] == pytest.approx(z / r ** 3, rel=1e-14)
    assert D[ix[(2, 0, 0)]] == pytest.approx(1 / r ** 3 - 3 * x * x / r ** 5, rel=1e-13)
    assert D[ix[(1, 1, 0)]] == pytest.approx(-3 * x * y / r ** 5, rel=1e-13)
    assert D[ix[(1, 1, 1)]] == pytest.approx(15 * x * y * z / r ** 7, rel=1e-13)
    assert D[ix[(3, 0, 0)]] == pytest.approx(-9 * x / r ** 5 + 15 * x ** 3 / r ** 7, rel=1e-12)


@pytest.mark.parametrize("kernel,eps", [(oracle.WENDLAND_C2, 0.0), (oracle.PLUMMER, 0.4)])
def test_dtensor_matches_finite_differences(kernel, eps):
    p = 8
    d = np.array([0.9, 0.4, -0.6])
    mi = _mi(p)
    ix = _index(p)
    D = oracle.dtensor(p, d, kernel, eps)
    h = 1e-5
    for k, (a, b, c) in enumerate(mi):
        if a + b + c >= p:
            continue
        for axis in range(3):
            e = np.zeros(3)
            e[axis] = h
            num = (oracle.dtensor(p, d + e, kernel, eps)[k] - oracle.dtensor(p, d - e, kernel, eps)[k]) / (2 * h)
            up = [a, b, c]
            up[axis] += 1
            exact = D[ix[tuple(up)]]
            assert num == pytest.approx(exact, rel=1e-6, abs=1e-8 * max(1.0, abs(exact)))


def test_dtensor_traceless_for_newton():
    p = 10
    d = np.array([-0.2, 1.3, 0.45])
    D = oracle.dtensor(p, d)
    ix = _index(p)
    scale = np.abs(D).max()
    for (a, b, c) in _mi(p - 2):
        lap = D[ix[(a + 2, b, c)]] + D[ix[(a, b + 2, c)]] + D[ix[(a, b, c + 2)]]
        assert abs(lap) <= 1e-12 * scale


def test_dtensor_parity():
    p = 7
    d = np.array([0.5, -0.25, 0.8])
    Dp = oracle.dtensor(p, d)
    Dm = oracle.dtensor(p, -d)
    order = _mi(p).sum(1)
    assert np.allclose(Dm, (-1.0) ** order * Dp, rtol=1e-14, atol=0)
