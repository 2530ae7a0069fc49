"""Pins of the oracle's expansion operators (P2M, M2M, M2L, L2L, L2P) against exact identities
and the convergence the multipole method guarantees (Sec. 2.1)."""
import numpy as np
import pytest

import oracle


def _cloud(seed, n, centre, half):
    g = np.random.default_rng(seed)
    pos = centre[:, None] + g.uniform(-half, half, (3, n))
    m = g.uniform(0.2, 1.0, n)
    return pos, m


@pytest.mark.parametrize("p", [2, 5, 8])
def test_m2m_is_exact_translation(p):
    # moments about z1 translated to z2 equal the moments computed about z2 directly
    pos, m = _cloud(1, 50, np.array([0.1, 0.2, 0.3]), 0.25)
    z1 = np.array([0.05, 0.25, 0.35])
    z2 = np.array([-0.2, 0.4, 0.1])
    M1 = oracle.p2m(p, pos, m, z1)
    M2 = oracle.p2m(p, pos, m, z2)
    Mt = oracle.m2m(p, M1, z1 - z2)
    assert np.allclose(Mt, M2, rtol=1e-12, atol=1e-13 * np.abs(M2).max())


def test_p2m_low_orders():
    pos, m = _cloud(2, 30, np.zeros(3), 0.5)
    zc = np.array([0.1, -0.1, 0.2])
    M = oracle.p2m(3, pos, m, zc)
    ix = {tuple(v): i for i, v in enumerate(oracle.multi_indices(3))}
    r = pos - zc[:, None]
    assert M[ix[(0, 0, 0)]] == pytest.approx(m.sum(), rel=1e-14)
    assert M[ix[(1, 0, 0)]] == pytest.approx((m * r[0]).sum(), rel=1e-12)
    assert M[ix[(1, 1, 0)]] == pytest.approx((m * r[0] * r[1]).sum(), rel=1e-12)
    assert M[ix[(0, 0, 3)]] == pytest.approx((m * r[2] ** 3).sum(), rel=1e-12)


@pytest.mark.parametrize("p", [1, 4, 7])
def test_l2l_is_exact_reexpansion(p):
    g = np.random.default_rng(4)
    nc = oracle.num_coeffs(p)
    Lp = g.standard_normal(nc)
    zp = np.array([0.0, 0.0, 0.0])
    zc = np.array([0.25, -0.25, 0.25])
    Lc = oracle.l2l(p, Lp, zc - zp)
    for _ in range(5):
        x = zc + g.uniform(-0.2, 0.2, 3)
        phi_p, a_p = oracle.l2p(p, Lp, x - zp)
        phi_c, a_c = oracle.l2p(p, Lc, x - zc)
        assert phi_c == pytest.approx(phi_p, rel=1e-12, abs=1e-12)
        assert np.allclose(a_c, a_p, rtol=1e-11, atol=1e-11)


def test_l2p_gradient_is_minus_grad_potential():
    g = np.random.default_rng(5)
    p = 6
    L = g.standard_normal(oracle.num_coeffs(p))
    rho = np.array([0.1, -0.05, 0.08])
    _, a = oracle.l2p(p, L, rho)
    h = 1e-6
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        num = -(oracle.l2p(p, L, rho + e)[0] - oracle.l2p(p, L, rho - e)[0]) / (2 * h)
        assert num == pytest.approx(a[k], rel=1e-7, abs=1e-8)


def _m2l_error(p, dist):
    zb = np.zeros(3)
    za = np.array([dist, 0.3 * dist, -0.2 * dist])
    src, ms = _cloud(6, 40, zb, 0.5)
    snk, _ = _cloud(7, 20, za, 0.5)
    M = oracle.p2m(p, src, ms, zb)
    L = oracle.m2l(p, M, za - zb)
    err = []
    for i in range(snk.shape[1]):
        phi, a = oracle.l2p(p, L, snk[:, i] - za)
        d = src - snk[:, i:i + 1]
        r = np.linalg.norm(d, axis=0)
        a_ex = (ms * d / r ** 3).sum(1)
        phi_ex = -(ms / r).sum()
        err.append(max(np.linalg.norm(a - a_ex) / np.linalg.norm(a_ex), abs(phi - phi_ex) / abs(phi_ex)))
    return max(err)


def test_m2l_converges_with_order():
    # cubes of side 1 at centre distance ~4.2: convergence ratio (r_A + r_B)/d ~ 0.41
    orders = (1, 2, 4, 6, 8, 10, 14, 20)   # up to the highest order of the sweeps (Sec. 3.2)
    errs = [_m2l_error(p, 4.0) for p in orders]
    assert all(b < a for a, b in zip(errs, errs[1:]))
    ratio = 2 * (np.sqrt(3) / 2) / np.linalg.norm([4.0, 1.2, 0.8])
    for p, e in zip(orders, errs):
        assert e < 3.0 * ratio ** (p + 1)
    assert errs[orders.index(10)] < 1e-5
    assert errs[-1] < 1e-10


def test_m2l_mutual_forces_cancel():
    # total force of B on A from M2L + L2P equals minus that of A on B (Sec. 2.1, F_AB = -F_BA)
    p = 5
    za = np.array([0.0, 0.0, 0.0])
    zb = np.array([3.0, 1.0, -2.0])
    pa, ma = _cloud(8, 30, za, 0.5)
    pb, mb = _cloud(9, 25, zb, 0.5)
    MA = oracle.p2m(p, pa, ma, za)
    MB = oracle.p2m(p, pb, mb, zb)
    LA = oracle.m2l(p, MB, za - zb)
    LB = oracle.m2l(p, MA, zb - za)
    FA = sum(ma[i] * oracle.l2p(p, LA, pa[:, i] - za)[1] for i in range(pa.shape[1]))
    FB = sum(mb[i] * oracle.l2p(p, LB, pb[:, i] - zb)[1] for i in range(pb.shape[1]))
    assert np.allclose(FA, -FB, rtol=1e-12, atol=1e-14 * np.abs(FA).max())
    # and this holds although each side is only approximate
    d = pb[:, None, :] - pa[:, :, None]
    r = np.linalg.norm(d, axis=0)
    F_exact = (ma[:, None] * mb[None, :] * d / r ** 3).sum((1, 2))
    assert not np.allclose(FA, F_exact, rtol=1e-10)
    assert np.allclose(FA, F_exact, rtol=1e-3)


def test_m2l_plummer_kernel_is_expansion_of_softened_potential():
    p = 8
    eps = 0.7
    zb = np.zeros(3)
    za = np.array([3.0, 0.5, 0.0])
    src, ms = _cloud(10, 10, zb, 0.3)
    M = oracle.p2m(p, src, ms, zb)
    L = oracle.m2l(p, M, za - zb, oracle.PLUMMER, eps)
    x = za + np.array([0.1, 0.05, -0.1])
    phi, a = oracle.l2p(p, L, x - za)
    d = src - x[:, None]
    s = np.sqrt((d ** 2).sum(0) + eps ** 2)
    assert phi == pytest.approx(-(ms / s).sum(), rel=1e-7)
    a_ex = (ms * d / s ** 3).sum(1)
    assert np.linalg.norm(a - a_ex) < 1e-6 * np.linalg.norm(a_ex)
