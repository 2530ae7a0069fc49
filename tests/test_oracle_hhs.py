"""Pins of the oracle's HOLD integrator (Sec. 2.2, Algorithms 1-3): reduction to textbook
KDK leapfrog, the Poisson-call count the paper prints, the schedule of kicks and drifts, a
Kepler orbit, and momentum conservation to roundoff (Sec. 3.2.1)."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1712_10116_gb300 import ics

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_rung_brackets_the_timestep():
    dt_max = 1.0 / 64
    for dt_i in [1.0, dt_max, dt_max * 0.99, dt_max / 2, dt_max / 2 * 0.999, 1e-4, 1e-9]:
        k = oracle.rung(dt_i, dt_max, 30)
        assert dt_max / 2 ** k <= dt_i or k == 30
        if k > 0:
            assert dt_i < dt_max / 2 ** (k - 1)
    assert oracle.rung(1e-12, dt_max, 10) == 10
    # dt_i = sqrt(eta eps / (|a_old| + |a_cur|)): fixed by the two magnitudes' sum
    assert oracle.timestep(0.02, 0.01, 1.0, 3.0) == oracle.timestep(0.02, 0.01, 2.0, 2.0)
    assert oracle.timestep(0.02, 0.01, 0.0, 4.0) == pytest.approx(0.5 * math.sqrt(0.02 * 0.01), rel=1e-15)
    assert oracle.timestep(0.02, 0.01, 0.0, 0.0) == math.inf


def test_single_rung_is_textbook_kdk():
    # k_max = 0 keeps every particle on rung 0: Algorithms 1-3 reduce to kick-drift-kick
    pos, vel, m = ics.plummer(300, 1001)
    prm = oracle.params(p=4, theta=0.5, eps=0.01, kernel=oracle.PLUMMER, n_crit=16)
    dt = 1.0 / 64
    h = oracle.HHS(pos, vel, m, prm, eta=0.025, dt_max=dt, k_max=0)
    x, v = pos.copy(), vel.copy()
    for _ in range(4):
        a, _ = oracle.fmm(x, m, prm)
        v = v + a * (dt / 2)
        x = x + v * dt
        a, _ = oracle.fmm(x, m, prm)
        v = v + a * (dt / 2)
        stats, _ = h.step()
        assert stats.poisson_calls == 2 and stats.max_rung == 0
    assert np.array_equal(h.pos, x) and np.array_equal(h.vel, v)


def _two_rung_system(k, eta=0.02, eps=1e-3):
    """A circular binary that sits on rung k and 18 distant light particles on rung 0."""
    mb, s = 0.1, 0.05
    dt_bin = math.sqrt(eta * eps * s * s / mb)
    dt_max = dt_bin * 2.0 ** (k - 0.5)
    v = math.sqrt(mb / (2 * s))
    ang = np.linspace(0, 2 * np.pi, 18, endpoint=False)
    far = np.stack([10 * np.cos(ang), 10 * np.sin(ang), 0.3 * np.sin(3 * ang)])
    pos = np.concatenate([np.array([[-s / 2, s / 2], [0, 0], [0, 0]]), far], axis=1)
    vel = np.zeros_like(pos)
    vel[1, 0], vel[1, 1] = -v, v
    m = np.concatenate([[mb, mb], np.full(18, 0.8 / 18)])
    return pos, vel, m, dt_max


def _golden_calls():
    rows = {}
    for line in open(os.path.join(GOLDEN, "poisson_calls.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, hhs, shared = map(int, line.split())
        rows[k] = (hhs, shared)
    return rows


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_poisson_calls_per_step_match_paper(k):
    pos, vel, m, dt_max = _two_rung_system(k)
    prm = oracle.params(p=4, theta=0.5, eps=1e-3, n_crit=8)
    h = oracle.HHS(pos, vel, m, prm, eta=0.02, dt_max=dt_max, k_max=12)
    want = _golden_calls()[k][0]
    for _ in range(3):
        stats, _ = h.step()
        assert stats.max_rung == k
        assert set(np.unique(h.rung)) == {0, k}
        assert stats.poisson_calls == want


def test_schedule_follows_algorithms_1_and_2():
    pos, vel, m, dt_max = _two_rung_system(2)
    prm = oracle.params(p=4, theta=0.5, eps=1e-3, n_crit=8)
    h = oracle.HHS(pos, vel, m, prm, eta=0.02, dt_max=dt_max, k_max=12)
    _, trace = h.step(trace_cap=256)
    S2F, FS2S, DRIFT = 0, 1, 2
    rung2_kdk = [(FS2S, 2, 2, 2), (DRIFT, 2, 2, 0), (FS2S, 2, 2, 2)]
    empty_kdk = [(DRIFT, 1, 0, 0)]                      # rung 1 holds no slow particle
    half = rung2_kdk + empty_kdk + rung2_kdk            # EVOLVE_HOLD(1, fast, ...) on the binary
    kdk0 = [(S2F, 0, 2, 18), (FS2S, 0, 18, 20), (DRIFT, 0, 18, 0), (FS2S, 0, 18, 20), (S2F, 0, 2, 18)]
    want = half + kdk0 + half
    assert [tuple(r) for r in trace] == want


def test_kepler_circular_orbit():
    pos, vel, m, a = ics.two_body(1.0, 0.0)
    prm = oracle.params(p=4, theta=0.5, eps=1e-4, n_crit=8)
    dt_max = 1.0 / 64
    h = oracle.HHS(pos, vel, m, prm, eta=0.02, dt_max=dt_max, k_max=10)
    E0 = h.diagnostics()[6]
    period = 2 * math.pi * a ** 1.5
    nsteps = int(round(period / dt_max))
    for _ in range(nsteps):
        h.step()
    # back near the start after one period; energy and the circular radius conserved
    phase = 2 * math.pi * (nsteps * dt_max) / period
    want = 0.5 * np.array([-math.cos(phase), -math.sin(phase), 0.0])
    assert np.linalg.norm(h.pos[:, 0] - want) < 1e-4
    sep = np.linalg.norm(h.pos[:, 1] - h.pos[:, 0])
    assert sep == pytest.approx(1.0, abs=1e-5)
    E1 = h.diagnostics()[6]
    assert abs(E1 / E0 - 1) < 1e-6
    assert set(np.unique(h.rung)) == {3}


def test_momentum_conserved_over_multirung_run():
    # Sec. 3.2.1: FMM + HHS conserves the total momentum to roundoff
    pos, vel, m = ics.clustered(1200, 1007)
    m = ics.random_masses(1200, 3)
    vel = vel - (vel * m).sum(1, keepdims=True) / m.sum()
    prm = oracle.params(p=4, theta=0.5, eps=0.002, n_crit=16)
    h = oracle.HHS(pos, vel, m, prm, eta=0.02, dt_max=1.0 / 16, k_max=8)
    P0 = (h.vel * m).sum(1)
    scale = (np.abs(h.vel) * m).sum()
    rungs = set()
    for _ in range(3):
        stats, _ = h.step()
        rungs |= set(np.unique(h.rung).tolist())
        P = (h.vel * m).sum(1)
        assert np.abs(P - P0).max() < 1e-14 * max(scale, 1.0)
    assert len(rungs) >= 3  # the run really used several rungs


# ---------------------------------------------------------------- Eq. (9): minimum timestep from |a|_tot
def test_eq9_timestep_exact_values():
    # eta * eps = 1/4 and |a_old| + |a_cur| = 4: the default timestep is sqrt(1/16) = 1/4 exactly
    assert oracle.timestep_tot(0.5, 0.5, 1.0, 3.0, 0.0, 16.0) == 0.25          # constraint off
    assert oracle.timestep_tot(0.5, 0.5, 1.0, 3.0, 0.5, 16.0) == 0.125         # sqrt(1/64) binds
    assert oracle.timestep_tot(0.5, 0.5, 1.0, 3.0, 0.5, 1.0) == 0.25           # sqrt(1/4) = 1/2 does not
    assert oracle.timestep_tot(0.5, 0.5, 1.0, 3.0, 0.5, 0.0) == 0.25           # no total acceleration yet
    assert oracle.timestep_tot(0.5, 0.5, 0.0, 0.0, 0.5, 4.0) == 0.25           # only the constraint is finite


def _plummer_run(eta_tot, steps=2, k_max=6, n=400):
    pos, vel, m = ics.plummer(n, 1001)
    prm = oracle.params(p=4, theta=0.5, eps=0.01, kernel=oracle.PLUMMER, n_crit=16)
    h = oracle.HHS(pos, vel, m, prm, eta=0.025, dt_max=1.0 / 16, k_max=k_max, eta_tot=eta_tot)
    rungs = []
    for _ in range(steps):
        h.step()
        rungs.append(h.rung.copy())
    return h, rungs


def test_eq9_constraint_that_never_binds_changes_nothing():
    h0, r0 = _plummer_run(0.0)
    h1, r1 = _plummer_run(1e9)
    assert np.array_equal(h0.pos, h1.pos) and np.array_equal(h0.vel, h1.vel)
    assert all(np.array_equal(a, b) for a, b in zip(r0, r1))


def test_eq9_binding_constraint_deepens_rungs():
    _, r0 = _plummer_run(0.0)
    _, r1 = _plummer_run(0.0025)
    assert all(np.all(b >= a) for a, b in zip(r0, r1))
    assert any(np.any(b > a) for a, b in zip(r0, r1))


def test_eq9_records_the_total_acceleration_at_rung_0():
    # k_max = 0: the second kickFS2S of rung 0 sees the whole system at the end-of-step positions
    pos, vel, m = ics.plummer(300, 1004)
    prm = oracle.params(p=4, theta=0.5, eps=0.01, kernel=oracle.PLUMMER, n_crit=16)
    h = oracle.HHS(pos, vel, m, prm, eta=0.025, dt_max=1.0 / 64, k_max=0, eta_tot=0.01)
    a0, _ = oracle.fmm(pos, m, prm)
    assert np.array_equal(h.a_tot, np.sqrt((a0 ** 2).sum(0)))                # from the initial evaluation
    h.step()
    a1, _ = oracle.fmm(h.pos, m, prm)
    assert np.allclose(h.a_tot, np.sqrt((a1 ** 2).sum(0)), rtol=1e-14, atol=0)


# ---------------------------------------------------------------- traditional individual timesteps
def test_traditional_single_rung_is_textbook_kdk():
    pos, vel, m = ics.plummer(300, 1001)
    prm = oracle.params(p=4, theta=0.5, eps=0.01, kernel=oracle.PLUMMER, n_crit=16)
    dt = 1.0 / 64
    t = oracle.Traditional(pos, vel, m, prm, eta=0.025, dt_max=dt, k_max=0)
    x, v = pos.copy(), vel.copy()
    a, _ = oracle.fmm(x, m, prm)
    for _ in range(3):
        v = v + a * (0.5 * dt)
        x = x + v * dt
        a, _ = oracle.fmm(x, m, prm)
        v = v + a * (0.5 * dt)
        st = t.step()
        assert st.poisson_calls == 1 and st.sink_forces == 300
    assert np.array_equal(t.pos, x) and np.array_equal(t.vel, v)


def test_traditional_binary_sets_the_boundaries():
    # a tight binary among far particles: it alone sits on rung k, so one step of dt_max has 2^k
    # boundaries (force evaluations), the last one shared with everybody else
    for k in (2, 4):
        pos, vel, m, dt_max = _two_rung_binary(k)
        prm = oracle.params(p=4, theta=0.5, eps=1e-3, kernel=oracle.PLUMMER, n_crit=8)
        t = oracle.Traditional(pos, vel, m, prm, eta=0.02, dt_max=dt_max, k_max=12)
        st = t.step()
        assert st.max_rung == k
        assert st.poisson_calls == 2 ** k
        assert st.sink_forces == 2 * 2 ** k + (len(m) - 2)


def _two_rung_binary(k, eta=0.02, eps=1e-3):
    mb, sep = 0.1, 0.05
    dt_bin = np.sqrt(eta * eps / (mb / sep ** 2))
    dt_max = dt_bin * 2.0 ** (k - 0.5)
    v = np.sqrt(mb / (2 * sep))
    ang = np.linspace(0, 2 * np.pi, 18, endpoint=False)
    far = np.stack([10 * np.cos(ang), 10 * np.sin(ang), 0.3 * np.sin(3 * ang)])
    pos = np.concatenate([np.array([[-sep / 2, sep / 2], [0, 0], [0, 0]]), far], axis=1)
    vel = np.zeros_like(pos)
    vel[1, 0], vel[1, 1] = -v, v
    m = np.concatenate([[mb, mb], np.full(18, 0.8 / 18)])
    return pos, vel, m, dt_max


def test_traditional_scheme_breaks_momentum_conservation():
    # Sec. 3.2.1: forces on active particles from unsynchronised inactive ones, without reaction,
    # leave a momentum error far above roundoff; HHS keeps it at roundoff on the same system
    pos, vel, m = ics.plummer(800, 1005)
    m = ics.random_masses(800, 41)
    vel = vel - (vel * m).sum(1, keepdims=True) / m.sum()
    prm = oracle.params(p=5, theta=0.45, eps=0.01, kernel=oracle.PLUMMER, n_crit=16)
    t = oracle.Traditional(pos, vel, m, prm, eta=0.02, dt_max=1.0 / 8, k_max=8)
    h = oracle.HHS(pos, vel, m, prm, eta=0.02, dt_max=1.0 / 8, k_max=8)
    for _ in range(2):
        t.step()
        h.step()
    scale = (m * np.abs(vel).sum(0)).sum()
    p_trad = np.abs((t.vel * m).sum(1)).max() / scale
    p_hhs = np.abs((h.vel * m).sum(1)).max() / scale
    assert len(np.unique(t.rung)) >= 3
    assert p_hhs < 1e-14
    assert p_trad > 1e3 * max(p_hhs, 1e-16)


# ---------------------------------------------------------------- conservation diagnostics (Sec. 3.2)
def test_diagnostics_circular_kepler_pair():
    # two masses 1/2 on a circular orbit of separation a = 1 (G = M = 1): P = 0,
    # L = mu a v_rel = (1/4) a sqrt(1/a) along +z, E = -m1 m2 / (2 a)
    pos, vel, m, a = ics.two_body(1.0, 0.0)
    _, pot = oracle.direct(pos, m, 1e-4)
    d = oracle.diagnostics(pos, vel, m, pot)
    assert np.abs(d[:3]).max() < 1e-16
    assert d[3:6] == pytest.approx([0.0, 0.0, 0.25 * a * math.sqrt(1.0 / a)], abs=1e-16)
    assert d[6] == pytest.approx(-0.25 / (2.0 * a), rel=1e-15)


def test_diagnostics_rigid_rotation_and_translation():
    # v = u + omega x x: P = M u + omega x (sum m x), and L = sum m x cross u + I omega with the inertia tensor
    # I = sum m (|x|^2 1 - x x^T) (the x cross (omega cross x) expansion); K = (1/2) sum m |v|^2
    g = np.random.default_rng(11)
    n = 257
    pos = g.standard_normal((3, n))
    m = ics.random_masses(n, 5)
    u = np.array([0.3, -0.2, 0.7])
    om = np.array([-0.4, 1.1, 0.25])
    vel = u[:, None] + np.cross(om, pos.T).T
    d = oracle.diagnostics(pos, vel, m)
    assert d[:3] == pytest.approx(m.sum() * u + np.cross(om, (pos * m).sum(1)), rel=1e-13, abs=1e-15)
    inertia = np.einsum("i,ji,ki->jk", m, pos, pos)
    I = np.eye(3) * np.trace(inertia) - inertia
    L_want = np.cross((pos * m).sum(1), u) + I @ om
    assert d[3:6] == pytest.approx(L_want, rel=1e-12, abs=1e-14)
    K = 0.5 * float((m * (vel * vel).sum(0)).sum())
    assert d[6] == pytest.approx(K, rel=1e-13)


def test_diagnostics_plummer_virial_and_binding_energy():
    # a Plummer sphere drawn from its distribution function is in virial equilibrium, 2K + W = 0, and
    # its potential energy is W = -3 pi / 32 (G = M = a = 1; Plummer-softened with a small eps the
    # pairwise sum differs little).  Both hold within the sampling noise of 8192 particles.
    n = 8192
    pos, vel, m = ics.plummer(n, 1001)
    _, pot = oracle.direct(pos, m, 1e-3, kernel=oracle.PLUMMER)
    d_all = oracle.diagnostics(pos, vel, m, pot)
    K = oracle.diagnostics(pos, vel, m)[6]
    W = d_all[6] - K
    assert W == pytest.approx(-3.0 * math.pi / 32.0, rel=0.05)
    assert 2.0 * K / -W == pytest.approx(1.0, abs=0.06)
