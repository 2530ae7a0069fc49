"""Parity of the benchmarked paths against the oracle: the conservation diagnostics (Sec. 3.2), the
cold-collapse evaluation at the bench's own parameters (n_crit = 96, masked and unmasked kick pairs,
full size, sampled sinks including the innermost and outermost particles), float32 HOLD steps
(Algorithms 1-3), and the disk galaxy integrated with HHS in float64 and float32."""
import numpy as np
import pytest
import torch

import oracle
from paper_1712_10116_gb300 import ics

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1712_10116_gb300 import binding as tg
    DEV = torch.device("cuda:0")

FP32_TOL = 1e-5     # per-particle relative difference, against max(|a_i|, 0.1 x median |a|)
FP32_FLOOR = 0.1


def _t(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def _oprm(prm):
    return oracle.params(p=prm.p, theta=prm.theta, eps=prm.eps, kernel=prm.kernel, n_crit=prm.n_crit,
                         kappa=prm.kappa, max_level=prm.max_level, mac=prm.mac)


def _rel(a, b, floor=0.0):
    nb = np.linalg.norm(b, axis=0)
    return np.linalg.norm(a - b, axis=0) / np.maximum(nb, floor * np.median(nb))


def _check_fp32(a, a_o, tag):
    r = _rel(a, a_o, FP32_FLOOR)
    u = _rel(a, a_o)
    print(f"fp32 parity {tag}: floored max {r.max():.3e} (bound {FP32_TOL:.0e}); unfloored max {u.max():.3e}, "
          f"p99.9 {np.percentile(u, 99.9):.3e}, median {np.median(u):.3e}")
    assert r.max() < FP32_TOL, (tag, r.max())


# ---------------------------------------------------------------- P, L, E (Sec. 3.2)
@pytest.mark.parametrize("kernel", [0, 1])
def test_diagnostics_match_oracle(kernel):
    n = 3000
    pos, vel, mass = ics.plummer(n, 1001)
    mass = ics.random_masses(n, 41)
    prm = tg.Params(p=4, theta=0.5, eps=0.01, kernel=kernel, precision=tg.TG_PREC_FP64, n_crit=32, eta=0.025,
                    dt_max=1.0 / 32, k_max=6)
    s = tg.Solver(prm)
    P, V, M = _t(pos), _t(vel), _t(mass)
    s.hhs_init(P, V, M)
    h = oracle.HHS(pos, vel, mass, _oprm(prm), eta=0.025, dt_max=1.0 / 32, k_max=6)
    for step in range(3):
        d = s.diagnostics()
        o = h.diagnostics()
        p_scale = float((mass * np.abs(h.vel).sum(0)).sum())
        l_scale = float((mass * np.linalg.norm(h.pos, axis=0) * np.linalg.norm(h.vel, axis=0)).sum())
        assert np.abs(d[:3] - o[:3]).max() < 1e-12 * p_scale, step
        assert np.abs(d[3:6] - o[3:6]).max() < 1e-12 * l_scale, step
        assert abs(d[6] - o[6]) < 1e-12 * abs(o[6]), step
        assert d[7] == pytest.approx(step / 32.0, abs=1e-15)
        s.hhs_step()
        h.step()


# ---------------------------------------------------------------- the bench's evaluation, full size
@pytest.mark.parametrize("masked", [False, True])
def test_cold_collapse_bench_parameters_sampled(masked):
    # uniform sphere N = 2^20, eps = 0.005, p = 6, theta = 0.5, n_crit = 96 (the bench's leaf size),
    # float32; 512 random sinks plus the 64 innermost and 64 outermost particles
    n = 1 << 20
    pos, _, mass = ics.uniform_sphere(n, 1002)
    fast = ics.random_fast_mask(n, 17) if masked else None
    prm = tg.Params(p=6, theta=0.5, eps=0.005, kernel=0, precision=tg.TG_PREC_FP32, n_crit=96)
    s = tg.Solver(prm)
    acc, _ = s.fmm_forces(_t(pos), _t(mass), None if fast is None else _t(fast, torch.uint8), want_pot=False)
    r = np.linalg.norm(pos, axis=0)
    order = np.argsort(r)
    rng = np.random.default_rng(5)
    sample = np.unique(np.concatenate([rng.choice(n, 512, replace=False), order[:64], order[-64:]]))
    a_o, _ = oracle.fmm_sample(pos, mass, _oprm(prm), sample, fast)
    a = acc.cpu().numpy()[:, sample]
    # floor from the typical force of the whole sample (the innermost particles feel almost nothing)
    _check_fp32(a, a_o, f"cold collapse 2^20 n_crit=96 masked={masked}")
    if not masked:
        ad, _ = s.direct_forces(_t(pos), _t(mass), None, _t(sample, torch.int64))
        ad = ad.cpu().numpy()
        e = np.linalg.norm(a - ad, axis=0) / np.linalg.norm(ad, axis=0)
        assert np.median(e) < 1e-4


# ---------------------------------------------------------------- float32 HOLD steps
def _compare_hhs(s, P, V, h, n, tag, fp32):
    rung = tg.tg_hhs_state(s.ctx, n)[0].cpu().numpy()
    x, v = P.cpu().numpy(), V.cpu().numpy()
    if not fp32:
        assert np.array_equal(rung, h.rung), tag
        assert np.abs(x - h.pos).max() < 1e-11 * np.abs(h.pos).max(), tag
        assert np.abs(v - h.vel).max() < 1e-10 * np.abs(h.vel).max(), tag
        return 0
    # float32 forces differ from the oracle's by ~1e-7..1e-5 relative, so a particle whose timestep sits
    # that close to a rung threshold dt_max / 2^k may take the other rung: those are reported and left
    # out; the rest must sit on the same rung and follow the same trajectory to float32 accuracy
    flip = rung != h.rung
    dt = np.sqrt(s.params.eta * s.params.eps / np.maximum(h.a_old + h.a_cur, 1e-300))
    near = np.zeros(n, bool)
    for k in range(s.params.k_max + 1):
        near |= np.abs(dt / (s.params.dt_max / 2 ** k) - 1.0) < 1e-4
    print(f"{tag}: {flip.sum()} of {n} particles on another rung ({(flip & near).sum()} within 1e-4 of a threshold)")
    assert flip.sum() <= max(3, n // 1000), tag
    ok = ~flip
    # a force error of up to 1e-5 of |a| over the run's time T moves a velocity by ~1e-5 |a| T; with
    # |a| T below the system's velocity scale (true for both runs here) that stays under 1e-4 of
    # max |v|, and positions under 1e-5 of max |x|.  Timesteps are recomputed many times inside a
    # rung-0 step, so a particle can also take the other rung for part of the step and come back:
    # its velocity then differs by up to the size of one kick at its rung, |a_i| dt_max / 2^rung.
    # Such particles are reported; there may be a few, each within that one-kick bound.
    xs = np.abs(h.pos).max()
    vs = np.abs(h.vel).max()
    dx = np.abs(x - h.pos)[:, ok].max() / xs
    dvi = np.abs(v - h.vel).max(axis=0)
    out = ok & (dvi > 1e-4 * vs)
    kick = (h.a_old + h.a_cur) * (s.params.dt_max / 2.0 ** h.rung)
    print(f"{tag}: max |dx| / max|x| = {dx:.2e}, max |dv| / max|v| = {dvi[ok & ~out].max() / vs:.2e}; "
          f"{out.sum()} particles beyond 1e-4 max|v|, worst at {(dvi[out] / kick[out]).max() if out.any() else 0:.2e} "
          f"of one kick at their rung")
    assert dx < 1e-5, tag
    assert out.sum() <= max(3, n // 1000), tag
    assert np.all(dvi[out] <= kick[out]), tag
    return int(flip.sum() + out.sum())


def test_hhs_fp32_matches_oracle():
    n = 4096
    pos, vel, mass = ics.plummer(n, 1001)
    prm = tg.Params(p=4, theta=0.5, eps=0.01, kernel=0, precision=tg.TG_PREC_FP32, n_crit=32, eta=0.025,
                    dt_max=1.0 / 16, k_max=8)
    s = tg.Solver(prm)
    P, V, M = _t(pos), _t(vel), _t(mass)
    s.hhs_init(P, V, M)
    h = oracle.HHS(pos, vel, mass, _oprm(prm), eta=0.025, dt_max=1.0 / 16, k_max=8)
    for step in range(3):
        s.hhs_step()
        h.step()
        _compare_hhs(s, P, V, h, n, f"plummer 4096 fp32 step {step}", True)
    assert len(np.unique(h.rung)) >= 3


# ---------------------------------------------------------------- disk galaxy with HHS
DISK_N = 1 << 14
DISK_PRM = dict(p=6, theta=0.6, eps=0.02, kernel=0, n_crit=96, eta=0.025, dt_max=2.0, k_max=14)


@pytest.fixture(scope="module")
def disk_oracle_run():
    # one oracle trajectory (three rung-0 steps), shared by the float64 and float32 comparisons
    pos, vel, mass = ics.disk_galaxy(DISK_N, 1003, velocities=True)
    prm = tg.Params(precision=tg.TG_PREC_FP64, **DISK_PRM)
    h = oracle.HHS(pos, vel, mass, _oprm(prm), eta=DISK_PRM["eta"], dt_max=DISK_PRM["dt_max"], k_max=DISK_PRM["k_max"])
    states = []
    for _ in range(3):
        st, _ = h.step()
        states.append((h.pos.copy(), h.vel.copy(), h.rung.copy(), h.a_old.copy(), h.a_cur.copy()))
    return (pos, vel, mass), states


class _State:
    def __init__(self, st):
        self.pos, self.vel, self.rung, self.a_old, self.a_cur = st


def test_disk_galaxy_hhs_fp64_matches_oracle(disk_oracle_run):
    (pos, vel, mass), states = disk_oracle_run
    s = tg.Solver(tg.Params(precision=tg.TG_PREC_FP64, **DISK_PRM))
    P, V, M = _t(pos), _t(vel), _t(mass)
    s.hhs_init(P, V, M)
    for step in range(3):
        s.hhs_step()
        _compare_hhs(s, P, V, _State(states[step]), DISK_N, f"disk 2^14 fp64 step {step}", False)
    assert s.stats()["max_rung"] >= 6


def test_disk_galaxy_hhs_fp32_matches_oracle(disk_oracle_run):
    # The galaxy's dense centre is collisional on these time scales (t = 0..6 in units where its
    # crossing time is ~0.1), so two trajectories that start apart by float32 rounding separate
    # exponentially: after the first rung-0 step they still agree to float32 accuracy, later only
    # statistically.  The float32 forces are held to their bound on every state of the oracle's
    # trajectory, kick pairs included.
    (pos, vel, mass), states = disk_oracle_run
    prm = tg.Params(precision=tg.TG_PREC_FP32, **DISK_PRM)
    s = tg.Solver(prm)
    P, V, M = _t(pos), _t(vel), _t(mass)
    s.hhs_init(P, V, M)
    s.hhs_step()
    _compare_hhs(s, P, V, _State(states[0]), DISK_N, "disk 2^14 fp32 step 0", True)
    s.hhs_step()
    s.hhs_step()
    st = _State(states[2])
    rung = tg.tg_hhs_state(s.ctx, DISK_N)[0].cpu().numpy()
    dv = np.abs(V.cpu().numpy() - st.vel).max(axis=0) / np.abs(st.vel).max()
    print(f"disk 2^14 fp32 after 3 steps: {(rung != st.rung).sum()} particles on another rung, median |dv| / max|v| "
          f"{np.median(dv):.2e}, {(dv > 1e-4).sum()} beyond 1e-4")
    assert (rung != st.rung).mean() < 0.01 and np.median(dv) < 1e-6 and (dv > 1e-4).mean() < 0.03
    ev = tg.Solver(prm)
    for k, (x, _, r, _, _) in enumerate(states):
        fast = (r > np.median(r)).astype(np.uint8)
        floor = _rounding_floor(ev, x, mass, DISK_PRM["eps"])
        for mask in (None, fast):
            acc, _ = ev.fmm_forces(_t(x), M, None if mask is None else _t(mask, torch.uint8), want_pot=False)
            a_o, _ = oracle.fmm(x, mass, _oprm(prm), mask)
            a = acc.cpu().numpy()
            nb = np.linalg.norm(a_o, axis=0)
            bound = FP32_TOL * np.maximum(nb, FP32_FLOOR * np.median(nb)) + floor
            d = np.linalg.norm(a - a_o, axis=0)
            r = d / np.maximum(nb, FP32_FLOOR * np.median(nb))
            print(f"disk 2^14 state {k} masked={mask is not None}: floored max {r.max():.3e}, "
                  f"{int((r >= FP32_TOL).sum())} particles past 1e-5 (all within their rounding floor: "
                  f"{bool(np.all(d < bound))}), worst d / bound {(d / bound).max():.3f}")
            assert np.all(d < bound), (k, (d / bound).max())


def _rounding_floor(s, x, mass, eps):
    """Per-particle force error that float32 positions relative to a leaf centre allow: each coordinate
    of a particle and of its neighbours is rounded by up to u s_leaf (u = 2^-24 of the leaf side s_leaf;
    the leaf is the one the library's tree gives the particle), and the force on i moves by at most
    sum_j 3 m_j g(r_ij) per unit of relative displacement (the tidal tensor of each pair is bounded by
    3 m_j g).  Both ends of a pair can be rounded: floor_i = 2 sqrt(3) u s_leaf,i sum_j 3 m_j g(r_ij).
    In the sparse outer leaves of a small disk (s_leaf of several units) a neighbour at r ~ eps puts this
    near 1e-5 of the particle's force."""
    tg.tg_build_tree(s.ctx, _t(x))
    tr = tg.tg_get_tree(s.ctx)
    n = x.shape[1]
    leaf_level = np.zeros(n, np.int64)
    for c in np.nonzero(tr["nchild"] == 0)[0]:
        sorted_pos = np.arange(tr["first"][c], tr["first"][c] + tr["count"][c])
        leaf_level[tr["perm"][sorted_pos]] = tr["level"][c]
    s_leaf = tr["L"] / 2.0 ** leaf_level
    sens = np.zeros(n)
    for i0 in range(0, n, 1024):
        d = x[:, None, :] - x[:, i0:i0 + 1024, None]
        rr = np.sqrt((d * d).sum(0))
        u = rr / eps
        with np.errstate(divide="ignore", invalid="ignore"):
            g = np.where(u < 1, (21 * u ** 5 - 90 * u ** 4 + 140 * u ** 3 - 84 * u ** 2 + 14) / eps ** 3, rr ** -3.0)
        g[rr == 0] = 0.0
        sens[i0:i0 + 1024] = (3.0 * mass[None, :] * g).sum(1)
    return 2.0 * np.sqrt(3.0) * 2.0 ** -24 * s_leaf * sens
