"""The other workloads of the benchmark table, at full size, on the float32 GPU path: parity with the
oracle on sampled sinks (the oracle evaluates them one by one over the whole tree), the FMM error
against float64 direct summation on the same sinks, and momentum.

* isolated disk galaxy, N = 2^22: exponential disk + Hernquist bulge + NFW halo, eps = 0.02,
  p = 6, theta = 0.6 (Wendland C2);
* clustered box, N = 2^24: Zel'dovich-displaced lattice with 1000 NFW clumps, eps = 1e-3, p = 6,
  theta = 0.5 (Wendland C2);
* ensemble of 64 independent Plummer / King (W0 = 6) systems with N log-uniform in 2^10 .. 2^17,
  p = 4, theta = 0.5, Plummer softening eps = 0.01, one evaluation per system through one context.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1712_10116_gb300.binding as tg
from paper_1712_10116_gb300 import ics

pytestmark = pytest.mark.gpu
DEV = "cuda"
FP32_TOL = 1e-5     # per-sink relative difference, floored at 0.1 x the median force
FP32_FLOOR = 0.1


def _t(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def _rel(a, b, floor=0.0):
    nb = np.linalg.norm(b, axis=0)
    return np.linalg.norm(a - b, axis=0) / np.maximum(nb, floor * np.median(nb))


def _check_sampled(pos, mass, kw, seed, n_sample=40):
    s = tg.Solver(tg.Params(precision=tg.TG_PREC_FP32, **kw))
    acc, _ = s.fmm_forces(_t(pos), _t(mass))
    a_all = acc.cpu().numpy()
    s.close()
    sample = np.random.default_rng(seed).choice(pos.shape[1], n_sample, replace=False)
    a = a_all[:, sample]
    oprm = oracle.params(p=kw["p"], theta=kw["theta"], eps=kw["eps"], kernel=kw["kernel"], n_crit=kw["n_crit"])
    a_o, _ = oracle.fmm_sample(pos, mass, oprm, sample)
    assert _rel(a, a_o, FP32_FLOOR).max() < FP32_TOL
    ad, _ = oracle.direct(pos, mass, kw["eps"], kw["kernel"], sinks=sample)
    assert np.median(_rel(a, ad)) < 1e-4            # the accuracy gate of the metric
    res = np.abs((a_all * mass).sum(1)).max() / np.abs(a_all * mass).sum()
    assert res < 1e-6, res


def test_disk_galaxy_full_size_sampled():
    pos, mass = ics.disk_galaxy(1 << 22)
    _check_sampled(pos, mass, dict(p=6, theta=0.6, eps=0.02, kernel=0, n_crit=64), seed=6)


def test_clustered_box_full_size_sampled():
    pos, mass = ics.clustered_box(256)
    _check_sampled(pos, mass, dict(p=6, theta=0.5, eps=1e-3, kernel=0, n_crit=64), seed=5)


def test_ensemble_of_64_systems():
    systems = ics.ensemble()
    assert len(systems) == 64
    s = tg.Solver(tg.Params(p=4, theta=0.5, eps=0.01, kernel=1, precision=tg.TG_PREC_FP32, n_crit=64))
    worst = 0.0
    for k, (pos, mass) in enumerate(systems):
        acc, _ = s.fmm_forces(_t(pos), _t(mass))
        a = acc.cpu().numpy()
        res = np.abs((a * mass).sum(1)).max() / np.abs(a * mass).sum()
        assert res < 1e-6, (k, res)
        if k % 8 == 0 or k % 8 == 1:                  # Plummer and King members against the oracle
            n = pos.shape[1]
            sample = np.random.default_rng(k).choice(n, min(n, 48), replace=False)
            a_o, _ = oracle.fmm_sample(pos, mass, oracle.params(p=4, theta=0.5, eps=0.01, kernel=1, n_crit=64),
                                       sample)
            worst = max(worst, _rel(a[:, sample], a_o, FP32_FLOOR).max())
    s.close()
    assert worst < FP32_TOL, worst
