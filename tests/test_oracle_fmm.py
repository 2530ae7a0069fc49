"""Pins of the oracle's full FMM evaluation: reduction to direct summation, momentum
conservation (Sec. 2.1: F_AB = -F_BA), convergence in p and theta, masked kick pairs
(Algorithm 3 / Fig. 2), and the one-sink evaluation used for large inputs."""
import numpy as np
import pytest

import oracle
from paper_1712_10116_gb300 import ics


def _rel_err(a, b):
    return np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)


@pytest.mark.parametrize("kernel", [oracle.WENDLAND_C2, oracle.PLUMMER])
def test_tiny_theta_is_direct_summation(kernel):
    pos, _, m = ics.plummer(1500, 1001)
    prm = oracle.params(p=3, theta=1e-3, eps=0.02, kernel=kernel, n_crit=32)
    a, phi = oracle.fmm(pos, m, prm)
    ad, phid = oracle.direct(pos, m, 0.02, kernel)
    assert np.max(_rel_err(a, ad)) < 1e-12
    assert np.allclose(phi, phid, rtol=1e-12)


@pytest.mark.parametrize("p,theta,kappa", [(2, 0.8, 1.0), (4, 0.5, 1.0), (6, 0.3, 0.5), (5, 0.45, 1.0)])
@pytest.mark.parametrize("masked", [False, True])
@pytest.mark.parametrize("kernel", [oracle.WENDLAND_C2, oracle.PLUMMER])
def test_momentum_conserved_to_roundoff(p, theta, kappa, masked, kernel):
    pos, _, _ = ics.clustered(3000, 1007)
    m = ics.random_masses(3000, 5)
    fast = ics.random_fast_mask(3000, 6) if masked else None
    prm = oracle.params(p=p, theta=theta, eps=0.01, kernel=kernel, n_crit=24, kappa=kappa)
    a, _ = oracle.fmm(pos, m, prm, fast)
    total = np.abs(a * m).sum()
    assert np.abs((a * m).sum(axis=1)).max() < 1e-14 * total


def test_error_falls_with_order_and_angle():
    pos, _, m = ics.uniform_sphere(4000, 1002)
    ad, _ = oracle.direct(pos, m, 0.005)
    med = {}
    for p in (2, 4, 6):
        for theta in (0.7, 0.5):
            prm = oracle.params(p=p, theta=theta, eps=0.005)
            a, _ = oracle.fmm(pos, m, prm)
            med[p, theta] = np.median(_rel_err(a, ad))
    for theta in (0.7, 0.5):
        assert med[2, theta] > med[4, theta] > med[6, theta]
    for p in (2, 4, 6):
        assert med[p, 0.7] > med[p, 0.5]
    assert med[6, 0.5] < 1e-5  # well inside the 1e-4 median gate at the benchmark settings


def test_masked_pair_equals_two_masked_calls():
    # one evaluation with slow/fast classes = kickFS2S (all masses) for slow sinks and
    # kickS2F (fast masses set to zero) for fast sinks, Algorithm 3 and Fig. 2
    pos, _, _ = ics.plummer(2500, 1001)
    m = ics.random_masses(2500, 7)
    fast = ics.random_fast_mask(2500, 8, 0.4)
    prm = oracle.params(p=5, theta=0.5, eps=0.01)
    a, phi = oracle.fmm(pos, m, prm, fast)
    a_all, phi_all = oracle.fmm(pos, m, prm)
    m_masked = np.where(fast == 1, 0.0, m)
    a_s2f, phi_s2f = oracle.fmm(pos, m_masked, prm)
    want = np.where(fast[None, :] == 1, a_s2f, a_all)
    assert np.max(_rel_err(a, want)) < 1e-12
    assert np.allclose(phi, np.where(fast == 1, phi_s2f, phi_all), rtol=1e-12)
    # direct summation with the same classes agrees to the expansion error
    ad, _ = oracle.direct(pos, m, 0.01, is_fast=fast)
    assert np.median(_rel_err(a, ad)) < 1e-5


@pytest.mark.parametrize("masked", [False, True])
def test_one_sink_evaluation_matches_full(masked):
    pos, _, m = ics.clustered(3000, 1007)
    fast = ics.random_fast_mask(3000, 9) if masked else None
    prm = oracle.params(p=4, theta=0.5, eps=0.01, n_crit=16)
    a, phi = oracle.fmm(pos, m, prm, fast)
    sample = np.random.default_rng(1).choice(3000, 60, replace=False)
    a_s, phi_s = oracle.fmm_sample(pos, m, prm, sample, fast)
    assert np.max(_rel_err(a_s, a[:, sample])) < 1e-12
    assert np.allclose(phi_s, phi[sample], rtol=1e-12)


def test_edge_cases():
    prm = oracle.params(p=4, theta=0.5, eps=0.01, n_crit=4)
    # one particle: no force
    a, phi = oracle.fmm(np.zeros((3, 1)), np.ones(1), prm)
    assert np.all(a == 0) and np.all(phi == 0)
    # coincident particles: every cell at the deepest level stays a leaf; Wendland is finite at r = 0
    pos = np.zeros((3, 20))
    a, phi = oracle.fmm(pos, np.full(20, 0.05), prm)
    assert np.all(np.isfinite(a)) and np.all(a == 0)
    assert np.allclose(phi, -19 * 0.05 * 3 / 0.01)
    # two far groups: the root cube spans both
    g = np.random.default_rng(2)
    pos = np.concatenate([g.normal(0, 0.01, (3, 50)), g.normal(100, 0.01, (3, 50))], axis=1)
    m = np.full(100, 0.01)
    a, _ = oracle.fmm(pos, m, prm)
    ad, _ = oracle.direct(pos, m, 0.01)
    assert np.median(_rel_err(a, ad)) < 1e-6


def test_high_orders_converge_to_direct_summation():
    # orders up to 20 (the sweeps of Sec. 3.2): the error against direct summation keeps falling
    # geometrically and reaches the float64 roundoff level
    pos, _, _ = ics.clustered(500, 1007)
    m = ics.random_masses(500, 11)
    ad, _ = oracle.direct(pos, m, 0.01, oracle.WENDLAND_C2)
    med = []
    for p in (6, 12, 20):
        a, _ = oracle.fmm(pos, m, oracle.params(p=p, theta=0.5, eps=0.01, n_crit=8))
        med.append(np.median(_rel_err(a, ad)))
    assert med[0] > 30 * med[1] > 900 * med[2]
    assert med[2] < 1e-12

