"""Pins of the oracle's alternative multipole acceptance criterion (the enclosing-sphere radius the
paper names as the better choice, Sec. 2.3 and Sec. 4): radii that enclose, acceptance that keeps
particle pairs apart, covering walk, accuracy that follows theta, and momentum to roundoff."""
import numpy as np
import pytest

import oracle
from paper_1712_10116_gb300 import ics


def _centre(t, c):
    side = t.L / 2.0 ** t.level[c]
    return t.lo + (t.coords[:, c] + 0.5) * side


@pytest.mark.parametrize("kind", ["plummer", "clustered"])
def test_radii_enclose_the_particles(kind):
    pos = (ics.plummer(1500, 1001) if kind == "plummer" else ics.clustered(1500, 1007))[0]
    t = oracle.Tree(pos, oracle.params(p=3, n_crit=16, mac=oracle.MAC_SPHERE))
    r = t.radii()
    sp = pos[:, t.perm]
    for c in range(t.ncell):
        z = _centre(t, c)
        d = np.sqrt(((sp[:, t.first[c]:t.first[c] + t.count[c]] - z[:, None]) ** 2).sum(0))
        if t.nchild[c] == 0:
            assert r[c] == pytest.approx(d.max(), rel=1e-15, abs=0)       # leaves: the farthest particle
        else:
            assert r[c] >= d.max() * (1 - 1e-15)                           # parents: a sphere that encloses
            kids = range(t.child_first[c], t.child_first[c] + t.nchild[c])
            assert r[c] == pytest.approx(max(np.sqrt(3) * t.L / 2.0 ** (t.level[c] + 2) + r[k] for k in kids),
                                         rel=1e-15)


@pytest.mark.parametrize("theta", [0.35, 0.6])
def test_accepted_pairs_keep_particles_apart(theta):
    pos, _, _ = ics.clustered(1200, 1007)
    t = oracle.Tree(pos, oracle.params(p=3, theta=theta, n_crit=12, kernel=oracle.PLUMMER, mac=oracle.MAC_SPHERE))
    m2l, p2p = t.lists()
    assert m2l.shape[1] > 0
    sp = pos[:, t.perm]
    for a, b in m2l.T[:: max(1, m2l.shape[1] // 300)]:
        d = np.linalg.norm(_centre(t, a) - _centre(t, b))
        pa = sp[:, t.first[a]:t.first[a] + t.count[a]]
        pb = sp[:, t.first[b]:t.first[b] + t.count[b]]
        closest = np.sqrt(((pa[:, :, None] - pb[:, None, :]) ** 2).sum(0)).min()
        assert closest > (1 - theta) * d            # R_a + R_b < theta d leaves at least (1 - theta) d


def test_walk_still_covers_every_pair_once():
    n = 700
    pos, _, _ = ics.plummer(n, 1003)
    t = oracle.Tree(pos, oracle.params(p=3, theta=0.5, n_crit=16, kernel=oracle.PLUMMER, mac=oracle.MAC_SPHERE))
    m2l, p2p = t.lists()
    cover = np.zeros((n, n), np.int64)
    for a, b in np.concatenate([m2l, p2p], axis=1).T:
        cover[t.first[a]:t.first[a] + t.count[a], t.first[b]:t.first[b] + t.count[b]] += 1
    assert np.all(cover == 1)


def test_accuracy_follows_theta_and_momentum_is_kept():
    n = 2000
    pos, _, mass = ics.plummer(n, 1004)
    mass = ics.random_masses(n, 5)
    a_d, _ = oracle.direct(pos, mass, 0.01, oracle.PLUMMER)
    errs = []
    for theta in (0.7, 0.5, 0.3):
        a, _ = oracle.fmm(pos, mass, oracle.params(p=4, theta=theta, eps=0.01, kernel=oracle.PLUMMER, n_crit=16,
                                                   mac=oracle.MAC_SPHERE))
        errs.append(np.median(np.linalg.norm(a - a_d, axis=0) / np.linalg.norm(a_d, axis=0)))
        res = np.abs((a * mass).sum(1)).max() / np.abs(a * mass).sum()
        assert res < 1e-14
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-4
