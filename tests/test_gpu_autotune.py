"""The autotuner (tg_autotune): it times evaluations of the caller's system (or rung-0 steps of the bound
system) over the leaf size and the float32 launch shapes, keeps the fastest in the context, changes no
counter of the caller's work and no state of the bound system, and leaves the evaluation correct: forces
after tuning match the oracle at the chosen leaf size."""
import numpy as np
import pytest
import torch

import oracle
from paper_1712_10116_gb300 import ics

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1712_10116_gb300 import binding as tg
    DEV = torch.device("cuda:0")


def _t(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def test_defaults_before_tuning():
    s = tg.Solver(tg.Params(p=6, n_crit=64, precision=tg.TG_PREC_FP32))
    t = tg.tg_get_tuning(s.ctx)
    assert t["n_crit"] == 64 and t["p2p_rows"] == 2 and t["m2l_blocks_per_sm"] == 16 and t["m2l_form"] == 0
    assert t["candidates"] == 0
    s.close()


@pytest.mark.parametrize("precision", [1, 0])
def test_autotune_picks_a_candidate_and_stays_correct(precision):
    n = 1 << 15 if precision == 1 else 6000
    pos, _, mass = ics.plummer(n, 1001)
    fast = ics.random_fast_mask(n, 17)
    prm = tg.Params(p=6 if precision == 1 else 4, theta=0.5, eps=0.01, kernel=0, precision=precision, n_crit=96)
    s = tg.Solver(prm)
    P, M, F = _t(pos), _t(mass), _t(fast, torch.uint8)
    t = s.autotune(P, M, F)
    assert t["n_crit"] in (48, 64, 80, 96, 112, 128, 160, 192)
    if precision == 1:
        assert t["p2p_rows"] in (1, 2, 3) and t["m2l_blocks_per_sm"] in (4, 8, 16, 32) and t["m2l_form"] in (0, 1)
        assert t["candidates"] == 1 + 7 + 1 + 2 + 3 + 1
    else:
        assert t["p2p_rows"] == 2 and t["m2l_blocks_per_sm"] == 16 and t["candidates"] == 8
    assert 0 < t["objective_ms"] <= 1.25 * t["objective_ms_initial"]
    assert tg.tg_get_tuning(s.ctx) == t
    st = s.stats()
    assert st["evaluations"] == 0 and st["sink_forces"] == 0   # tuning is not counted as work
    # the tuned context evaluates the system like the oracle at the chosen leaf size
    acc, _ = s.fmm_forces(P, M, F)
    a_o, _ = oracle.fmm(pos, mass, oracle.params(p=prm.p, theta=0.5, eps=0.01, n_crit=t["n_crit"]), fast)
    a = acc.cpu().numpy()
    nb = np.linalg.norm(a_o, axis=0)
    r = np.linalg.norm(a - a_o, axis=0) / np.maximum(nb, 0.1 * np.median(nb))
    assert r.max() < (1e-5 if precision == 1 else 1e-12), r.max()
    s.close()


@pytest.mark.parametrize("batched", [1, 0])
def test_step_autotune_leaves_the_bound_system_as_it_was(batched):
    """Step objective (no particles given): rung-0 HOLD steps of the bound system are timed; the bound
    positions, velocities, integrator state and time come back unchanged, and the next step of the tuned
    context equals a step of a fresh context created with the chosen settings."""
    n = 6000
    pos, vel, mass = ics.plummer(n, 1001)
    prm = dict(p=4, theta=0.5, eps=0.01, kernel=1, precision=tg.TG_PREC_FP32, n_crit=64, dt_max=1 / 16, k_max=6,
               batched=batched)
    s = tg.Solver(tg.Params(**prm))
    P, V, M = _t(pos), _t(vel), _t(mass)
    s.hhs_init(P, V, M)
    s.hhs_step()   # a state with rungs and |a| bookkeeping from a real step
    P0, V0 = P.clone(), V.clone()
    state0 = tg.tg_hhs_state(s.ctx, n, DEV, with_total=True)
    time0 = s.diagnostics()[7]
    t = s.autotune()
    torch.cuda.synchronize()
    assert t["candidates"] == 1 + 7 + 1 + 2 + 3 + 1 - (1 if prm["kernel"] == 1 else 0)
    assert t["n_crit"] in (48, 64, 80, 96, 112, 128, 160, 192) and t["objective_ms"] > 0
    assert torch.equal(P, P0) and torch.equal(V, V0)
    for a, b in zip(tg.tg_hhs_state(s.ctx, n, DEV, with_total=True), state0):
        assert torch.equal(a, b)
    assert s.diagnostics()[7] == time0
    # the tuned context steps like a fresh one with the chosen settings (same state, same parameters)
    ref = tg.Solver(tg.Params(**dict(prm, n_crit=t["n_crit"])))
    tg.tg_set_tuning(ref.ctx, t)
    Pr, Vr = P0.clone(), V0.clone()
    ref.hhs_init(Pr, Vr, M)
    tg.tg_hhs_set_accel(ref.ctx, *state0[1:])
    s.hhs_step()
    ref.hhs_step()
    torch.cuda.synchronize()
    # float32 forces summed in atomic order: the two steps agree to the rounding of the kicks, except for
    # the rare particle whose timestep sits on a rung threshold and takes the other branch
    dp = (P - Pr).abs().amax(0)
    assert float((dp > 1e-6).double().mean()) < 0.01 and float(dp.median()) < 1e-9, (dp.max(), dp.median())
    s.close()
    ref.close()
