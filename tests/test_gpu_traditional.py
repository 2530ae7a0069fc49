"""The traditional individual-timestep integrator (Sec. 2.3) on the GPU against the oracle's, and the
momentum contrast with HHS that the paper reports (Sec. 3.2.1)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1712_10116_gb300 import ics

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1712_10116_gb300 import binding as tg
    DEV = torch.device("cuda:0")


def _t(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def _oprm(prm):
    return oracle.params(p=prm.p, theta=prm.theta, eps=prm.eps, kernel=prm.kernel, n_crit=prm.n_crit,
                         kappa=prm.kappa, max_level=prm.max_level, mac=prm.mac)


@pytest.mark.parametrize("kernel", [0, 1])
def test_traditional_fp64_matches_oracle(kernel):
    n = 1500
    pos, vel, mass = ics.plummer(n, 1001)
    prm = tg.Params(p=4, theta=0.5, eps=0.01, kernel=kernel, precision=tg.TG_PREC_FP64, n_crit=32, eta=0.025,
                    dt_max=1.0 / 16, k_max=6)
    s = tg.Solver(prm)
    P, V, M = _t(pos), _t(vel), _t(mass)
    s.trad_init(P, V, M)
    o = oracle.Traditional(pos, vel, mass, _oprm(prm), eta=0.025, dt_max=1.0 / 16, k_max=6)
    rung, _, _ = tg.tg_hhs_state(s.ctx, n)
    assert np.array_equal(rung.cpu().numpy(), o.rung)
    for step in range(2):
        tg.tg_reset_stats(s.ctx)
        s.trad_step()
        ost = o.step()
        st = s.stats()
        assert st["evaluations"] == ost.poisson_calls, step
        assert st["sink_forces"] == ost.sink_forces, step
        assert st["max_rung"] == ost.max_rung, step
        rung, _, _ = tg.tg_hhs_state(s.ctx, n)
        assert np.array_equal(rung.cpu().numpy(), o.rung), step
        assert np.abs(P.cpu().numpy() - o.pos).max() < 1e-11 * np.abs(o.pos).max()
        assert np.abs(V.cpu().numpy() - o.vel).max() < 1e-10 * np.abs(o.vel).max()
    assert len(np.unique(o.rung)) >= 2
    assert s.diagnostics()[7] == pytest.approx(2.0 / 16)


def test_traditional_momentum_error_versus_hhs():
    # the same system and parameters on both integrators, float64: HHS keeps sum m v at roundoff
    # (mutual interactions), the traditional scheme does not (Sec. 3.2.1)
    n = 6000
    pos, vel, mass = ics.clustered(n, 1007)
    mass = ics.random_masses(n, 31)
    vel = vel - (vel * mass).sum(1, keepdims=True) / mass.sum()
    prm = tg.Params(p=5, theta=0.45, eps=0.002, precision=tg.TG_PREC_FP64, n_crit=64, eta=0.02, dt_max=1.0 / 16,
                    k_max=8)
    scale = float((mass * np.abs(vel).sum(0)).sum())
    drift = {}
    for name in ("hhs", "trad"):
        s = tg.Solver(prm)
        P, V, M = _t(pos), _t(vel), _t(mass)
        (s.hhs_init if name == "hhs" else s.trad_init)(P, V, M)
        d0 = s.diagnostics()
        for _ in range(2):
            (s.hhs_step if name == "hhs" else s.trad_step)()
        d1 = s.diagnostics()
        drift[name] = np.abs(d1[:3] - d0[:3]).max() / scale
    assert drift["hhs"] < 1e-12
    assert drift["trad"] > 1e3 * max(drift["hhs"], 1e-16)


def test_integrators_need_their_own_init():
    pos, vel, mass = ics.plummer(300, 1002)
    s = tg.Solver(tg.Params(p=4, eps=0.01, kernel=1, precision=tg.TG_PREC_FP64, n_crit=16))
    with pytest.raises(tg.TGError):
        s.trad_step()
    P, V, M = _t(pos), _t(vel), _t(mass)
    s.trad_init(P, V, M)
    with pytest.raises(tg.TGError):
        s.hhs_step()
    with pytest.raises(tg.TGError):
        s.checkpoint("/tmp/never_written.ckpt")
    s.trad_step()
    s.hhs_init(P, V, M)
    with pytest.raises(tg.TGError):
        s.trad_step()
    s.hhs_step()
