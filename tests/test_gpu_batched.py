"""The batched HOLD step (tg_params.batched = 1): the recursion of Algorithms 1-2 as a device-side
work queue inside one CUDA graph per rung-0 step.  It must run the same operations as the host-driven
step -- the same Poisson-call count (Sec. 2.2), the same rungs and, in float64, the same trajectory to
1e-12 -- read the host once per step, give up with TG_ERR_TIMEOUT (state restored) when its bounded
loop runs out, and restore, regrow and redo a step whose lists or cells outgrow their buffers."""
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


def _run(prm, pos, vel, mass, steps):
    s = tg.Solver(prm)
    P, V, M = _t(pos), _t(vel), _t(mass)
    s.hhs_init(P, V, M)
    tg.tg_reset_stats(s.ctx)
    for _ in range(steps):
        s.hhs_step()
    torch.cuda.synchronize()
    rung = tg.tg_hhs_state(s.ctx, mass.shape[0])[0].cpu().numpy()
    out = P.cpu().numpy(), V.cpu().numpy(), rung, s.stats()
    s.close()
    return out


def _two_rung_system(k, eta=0.02, eps=1e-3):
    # a tight binary (rung k) among slow particles (rung 0): the paper's 2 + 2 + 2^(k+1) Poisson calls
    mb, sep = 0.1, 0.05
    dt_bin = np.sqrt(eta * eps * sep * sep / mb)
    dt_max = dt_bin * 2.0 ** (k - 0.5)
    v = np.sqrt(mb / (2 * sep))
    ang = np.linspace(0, 2 * np.pi, 18, endpoint=False)
    far = np.stack([10 * np.cos(ang), 10 * np.sin(ang), 0.3 * np.sin(3 * ang)])
    pos = np.concatenate([np.array([[-sep / 2, sep / 2], [0, 0], [0, 0]]), far], axis=1)
    vel = np.zeros_like(pos)
    vel[1, 0], vel[1, 1] = -v, v
    m = np.concatenate([[mb, mb], np.full(18, 0.8 / 18)])
    return pos, vel, m, dt_max


@pytest.mark.parametrize("k", [1, 3, 5])
def test_batched_poisson_calls_equal_plain_and_paper(k):
    pos, vel, m, dt_max = _two_rung_system(k)
    base = dict(p=4, theta=0.5, eps=1e-3, kernel=0, precision=tg.TG_PREC_FP64, n_crit=4, eta=0.02, dt_max=dt_max,
                k_max=8)
    xp, vp, rp, sp = _run(tg.Params(**base), pos, vel, m, 1)
    xb, vb, rb, sb = _run(tg.Params(batched=1, **base), pos, vel, m, 1)
    assert sb["evaluations"] == sp["evaluations"] == 2 + 2 + 2 ** (k + 1) - 2   # kick pairs: two calls each
    assert sb["kdk_frames"] == sp["kdk_frames"] and sb["max_rung"] == sp["max_rung"] == k
    assert sb["sink_forces"] == sp["sink_forces"]
    assert np.array_equal(rb, rp)
    assert np.abs(xb - xp).max() < 1e-12 * np.abs(xp).max()
    assert np.abs(vb - vp).max() < 1e-12 * np.abs(vp).max()


@pytest.mark.parametrize("kernel", [0, 1])
def test_batched_fp64_plummer_matches_plain_and_oracle(kernel):
    n = 1500
    pos, vel, mass = ics.plummer(n, 1001)
    base = dict(p=4, theta=0.5, eps=0.01, kernel=kernel, precision=tg.TG_PREC_FP64, n_crit=32, eta=0.025,
                dt_max=1.0 / 16, k_max=6)
    xp, vp, rp, sp = _run(tg.Params(**base), pos, vel, mass, 3)
    xb, vb, rb, sb = _run(tg.Params(batched=1, **base), pos, vel, mass, 3)
    assert sb["evaluations"] == sp["evaluations"] and sb["sink_forces"] == sp["sink_forces"]
    assert np.array_equal(rb, rp)
    assert np.abs(xb - xp).max() < 1e-12 * np.abs(xp).max()
    assert np.abs(vb - vp).max() < 1e-12 * np.abs(vp).max()
    # and the oracle's HOLD integrator (two masked Poisson calls per kick pair) agrees as for the plain path
    h = oracle.HHS(pos, vel, mass, oracle.params(p=4, theta=0.5, eps=0.01, kernel=kernel, n_crit=32), eta=0.025,
                   dt_max=1.0 / 16, k_max=6)
    for _ in range(3):
        h.step()
    assert np.array_equal(rb, h.rung)
    assert np.abs(xb - h.pos).max() < 1e-11 * np.abs(h.pos).max()

    # after its first step (which sizes the buffers with one plain evaluation and captures the graph) the
    # batched step waits on the host twice per step: the finiteness check of its inputs and its end
    s = tg.Solver(tg.Params(batched=1, **base))
    P, V, M = _t(pos), _t(vel), _t(mass)
    s.hhs_init(P, V, M)
    s.hhs_step()
    tg.tg_reset_stats(s.ctx)
    s.hhs_step()
    s.hhs_step()
    assert s.stats()["host_syncs"] == 4
    s.close()


def test_batched_fp32_disk_matches_plain():
    n = 1 << 16
    pos, vel, mass = ics.disk_galaxy(n, 1003, velocities=True)
    base = dict(p=6, theta=0.6, eps=0.02, kernel=0, precision=tg.TG_PREC_FP32, n_crit=96, eta=0.025, dt_max=2.0,
                k_max=14)
    xp, vp, rp, sp = _run(tg.Params(**base), pos, vel, mass, 1)
    xb, vb, rb, sb = _run(tg.Params(batched=1, **base), pos, vel, mass, 1)
    flips = int((rb != rp).sum())
    print(f"disk 2^16 fp32: {sb['evaluations']} evaluations (plain {sp['evaluations']}), max rung {sb['max_rung']}, "
          f"{flips} rung differences, host syncs {sb['host_syncs']} (plain {sp['host_syncs']})")
    assert sb["max_rung"] >= 5 and abs(sb["evaluations"] - sp["evaluations"]) <= 2
    assert flips <= n // 1000
    ok = rb == rp
    assert np.abs(xb - xp)[:, ok].max() < 1e-6 * np.abs(xp).max()
    assert np.median(np.abs(vb - vp)[:, ok]) < 1e-7 * np.abs(vp).max()


def test_batched_queue_limit_times_out_and_restores():
    pos, vel, mass = ics.plummer(2000, 1001)
    prm = tg.Params(p=4, theta=0.5, eps=0.01, precision=tg.TG_PREC_FP32, n_crit=32, dt_max=1 / 16, k_max=6, batched=1)
    s = tg.Solver(prm)
    P, V, M = _t(pos), _t(vel), _t(mass)
    s.hhs_init(P, V, M)
    s.hhs_step()   # sizes and captures the graph
    P0, V0 = P.clone(), V.clone()
    state0 = tg.tg_hhs_state(s.ctx, 2000, DEV, with_total=True)
    tg.tg_debug_control(s.ctx, tg.TG_DEBUG_QUEUE_LIMIT, 200)
    tg.tg_debug_control(s.ctx, tg.TG_DEBUG_QUEUE_HOLD, 1)   # the scheduler publishes nothing
    with pytest.raises(tg.TGError, match="TIMEOUT"):
        s.hhs_step()
    torch.cuda.synchronize()
    assert torch.equal(P, P0) and torch.equal(V, V0)
    for a, b in zip(tg.tg_hhs_state(s.ctx, 2000, DEV, with_total=True), state0):
        assert torch.equal(a, b)
    # a limit too small for the step's own operations also ends in a timeout, with nothing changed
    tg.tg_debug_control(s.ctx, tg.TG_DEBUG_QUEUE_HOLD, 0)
    tg.tg_debug_control(s.ctx, tg.TG_DEBUG_QUEUE_LIMIT, 3)
    with pytest.raises(tg.TGError, match="TIMEOUT"):
        s.hhs_step()
    assert torch.equal(P, P0) and torch.equal(V, V0)
    # released, the same context steps on
    tg.tg_debug_control(s.ctx, tg.TG_DEBUG_QUEUE_LIMIT, 0)
    s.hhs_step()
    torch.cuda.synchronize()
    assert not torch.equal(P, P0)
    s.close()


def test_batched_overflow_restores_regrows_and_redoes_the_step():
    # a Plummer sphere with a softening that keeps it far from close encounters: the float64 trajectories
    # of the plain and the regrown batched steps then differ only by the rounding of their float atomics
    n = 20000
    pos, vel, mass = ics.plummer(n, 1001)
    base = dict(p=5, theta=0.45, eps=0.01, precision=tg.TG_PREC_FP64, n_crit=32, eta=0.02, dt_max=1.0 / 16, k_max=8)
    xp, vp, rp, sp = _run(tg.Params(**base), pos, vel, mass, 2)
    s = tg.Solver(tg.Params(batched=1, **base))
    P, V, M = _t(pos), _t(vel), _t(mass)
    s.hhs_init(P, V, M)
    tg.tg_debug_control(s.ctx, tg.TG_DEBUG_BATCH_CAPS, 256)   # lists of 256 entries, 256 cells
    tg.tg_reset_stats(s.ctx)
    for _ in range(2):
        s.hhs_step()
    torch.cuda.synchronize()
    st = s.stats()
    assert st["list_regrowths"] >= 2   # both lists and cells ran out at least once
    assert st["evaluations"] == sp["evaluations"]
    x, v = P.cpu().numpy(), V.cpu().numpy()
    assert np.abs(x - xp).max() < 1e-12 * np.abs(xp).max()
    assert np.abs(v - vp).max() < 1e-12 * np.abs(vp).max()
    s.close()


# ---------------------------------------------------------------- ensemble: one graph launch for many systems
def _ensemble_members(precision, batched, systems, base):
    out = []
    for pos, vel, mass in systems:
        s = tg.Solver(tg.Params(precision=precision, batched=batched, **base))
        P, V, M = _t(pos), _t(vel), _t(mass)
        s.hhs_init(P, V, M)
        out.append((s, P, V, M))
    return out


def test_ensemble_step_equals_the_members_own_steps():
    # six Plummer / King systems of different sizes, each with its own rungs; float64, so that the one-launch
    # ensemble and the members' own batched steps agree to 1e-12
    sizes = [1500, 3001, 700, 5000, 2048, 4097]
    systems = [ics.plummer(n, 1001 + i) if i % 2 == 0 else ics.king(n, 6.0, 1005 + i, velocities=True)
               for i, n in enumerate(sizes)]
    base = dict(p=4, theta=0.5, eps=0.01, kernel=1, n_crit=32, eta=0.025, dt_max=1.0 / 32, k_max=8)
    ens = _ensemble_members(tg.TG_PREC_FP64, 1, systems, base)
    own = _ensemble_members(tg.TG_PREC_FP64, 1, systems, base)
    for s, *_ in ens + own:
        tg.tg_reset_stats(s.ctx)
    for _ in range(2):
        tg.tg_ensemble_step([s.ctx for s, *_ in ens])
        for s, *_ in own:
            s.hhs_step()
    torch.cuda.synchronize()
    for (se, Pe, Ve, _), (so, Po, Vo, _) in zip(ens, own):
        a, b = se.stats(), so.stats()
        assert a["evaluations"] == b["evaluations"] and a["sink_forces"] == b["sink_forces"]
        assert a["max_rung"] == b["max_rung"]
        re = tg.tg_hhs_state(se.ctx, Pe.shape[1])[0]
        ro = tg.tg_hhs_state(so.ctx, Po.shape[1])[0]
        assert torch.equal(re, ro)
        assert (Pe - Po).abs().max().item() < 1e-12 * Po.abs().max().item()
        assert (Ve - Vo).abs().max().item() < 1e-12 * Vo.abs().max().item()
        assert tg.tg_diagnostics(se.ctx)[7] == pytest.approx(2.0 / 32)
    # one wait per ensemble step on the first member's context (the sizing call aside)
    s0 = ens[0][0]
    tg.tg_reset_stats(s0.ctx)
    tg.tg_ensemble_step([s.ctx for s, *_ in ens])
    assert s0.stats()["host_syncs"] == 2
    for s, *_ in ens + own:
        s.close()


def test_ensemble_step_rejects_bad_member_lists():
    pos, vel, mass = ics.plummer(800, 1001)
    base = dict(p=4, theta=0.5, eps=0.01, kernel=1, n_crit=32, dt_max=1.0 / 32, k_max=6)
    a = _ensemble_members(tg.TG_PREC_FP32, 1, [(pos, vel, mass)], base)[0][0]
    b = _ensemble_members(tg.TG_PREC_FP32, 0, [(pos, vel, mass)], base)[0][0]
    with pytest.raises(tg.TGError):
        tg.tg_ensemble_step([a.ctx, a.ctx])      # twice
    with pytest.raises(tg.TGError):
        tg.tg_ensemble_step([a.ctx, b.ctx])      # a plain (not batched) member
    a.close()
    b.close()
