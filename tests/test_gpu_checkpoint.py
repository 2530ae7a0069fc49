"""Checkpoint and resume of an HHS run through the C ABI (tg_checkpoint / tg_restore).

A run that is checkpointed after two rung-0 steps and resumed in a fresh context must continue
exactly like the uninterrupted run; every malformed or mismatched resume must be refused without
touching the bound state.
"""
import os

import numpy as np
import pytest
import torch

import paper_1712_10116_gb300.binding as tg
from paper_1712_10116_gb300 import ics

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _params(**kw):
    base = dict(p=4, theta=0.5, eps=0.01, kernel=1, precision=tg.TG_PREC_FP64, n_crit=32, eta=0.025,
                dt_max=1.0 / 64, k_max=8, eta_tot=0.01)
    base.update(kw)
    return tg.Params(**base)


def _system(n=3000, seed=1001):
    pos, vel, mass = ics.plummer(n, seed)
    t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)
    return t(pos), t(vel), t(mass)


def _state(s, n):
    return tuple(a.cpu().numpy() for a in tg.tg_hhs_state(s.ctx, n, with_total=True))


def test_resume_continues_the_run(tmp_path):
    n = 3000
    P, V, M = _system(n)
    P0, V0 = P.clone(), V.clone()
    s1 = tg.Solver(_params())
    s1.hhs_init(P, V, M)
    for _ in range(2):
        s1.hhs_step()
    path = str(tmp_path / "run.ckpt")
    s1.checkpoint(path)
    t_ckpt = s1.diagnostics()[7]
    for _ in range(2):
        s1.hhs_step()
    d1 = s1.diagnostics()
    # a fresh context, bound to arrays that still hold the initial state
    P2, V2 = P0.clone(), V0.clone()
    s2 = tg.Solver(_params())
    s2.hhs_init(P2, V2, M)
    s2.restore(path)
    assert s2.diagnostics()[7] == t_ckpt
    for _ in range(2):
        s2.hhs_step()
    d2 = s2.diagnostics()
    assert d2[7] == d1[7]
    # float64 throughout; only the order of the float64 atomic sums can differ between the runs
    assert torch.allclose(P2, P, rtol=1e-11, atol=1e-13)
    assert torch.allclose(V2, V, rtol=1e-11, atol=1e-13)
    r1, o1, c1, t1 = _state(s1, n)
    r2, o2, c2, t2 = _state(s2, n)
    assert np.array_equal(r1, r2)
    assert np.allclose(o1, o2, rtol=1e-11, atol=0) and np.allclose(c1, c2, rtol=1e-11, atol=0)
    assert np.allclose(t1, t2, rtol=1e-11, atol=0)


def _expect(code, fn, *args):
    with pytest.raises(tg.TGError) as e:
        fn(*args)
    assert e.value.code == code, e.value


def test_refused_resumes_leave_the_state_alone(tmp_path):
    n = 2000
    P, V, M = _system(n, seed=1003)
    s = tg.Solver(_params())
    _expect(-7, s.checkpoint, str(tmp_path / "early.ckpt"))      # before tg_hhs_init
    _expect(-7, s.restore, str(tmp_path / "early.ckpt"))
    s.hhs_init(P, V, M)
    s.hhs_step()
    good = str(tmp_path / "good.ckpt")
    s.checkpoint(good)
    raw = open(good, "rb").read()

    # a second system to resume into
    Pb, Vb, _ = _system(n, seed=1003)
    target = tg.Solver(_params())
    target.hhs_init(Pb, Vb, M)
    keep_p, keep_v = Pb.clone(), Vb.clone()
    keep_state = _state(target, n)

    _expect(-8, target.restore, str(tmp_path / "missing.ckpt"))
    bad = str(tmp_path / "flipped.ckpt")
    b = bytearray(raw)
    b[len(b) // 2] ^= 0x01
    open(bad, "wb").write(bytes(b))
    _expect(-8, target.restore, bad)                                   # checksum
    short = str(tmp_path / "short.ckpt")
    open(short, "wb").write(raw[:-9])
    _expect(-8, target.restore, short)                                 # truncated
    junk = str(tmp_path / "junk.ckpt")
    open(junk, "wb").write(b"not a checkpoint at all" * 10)
    _expect(-8, target.restore, junk)                                  # no magic

    other = tg.Solver(_params(eps=0.02))                               # different parameters
    Po, Vo, _ = _system(n, seed=1003)
    other.hhs_init(Po, Vo, M)
    _expect(-7, other.restore, good)

    small = tg.Solver(_params())                                       # different n
    Ps, Vs, Ms = _system(n - 1, seed=1003)
    small.hhs_init(Ps, Vs, Ms)
    _expect(-7, small.restore, good)

    heavy = tg.Solver(_params())                                       # different masses
    Ph, Vh, _ = _system(n, seed=1003)
    Mh = M * 2
    heavy.hhs_init(Ph, Vh, Mh)
    _expect(-7, heavy.restore, good)

    # nothing reached the bound arrays or the integrator state of the refused target
    assert torch.equal(Pb, keep_p) and torch.equal(Vb, keep_v)
    after = _state(target, n)
    assert all(np.array_equal(a, b) for a, b in zip(keep_state, after))
    # and the good file still resumes
    target.restore(good)
    assert torch.equal(Pb, P) and torch.equal(Vb, V)
    assert not os.path.exists(good + ".tmp")
