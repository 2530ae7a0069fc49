"""Pins of the oracle's root cube, Morton keys, sort, octree and Algorithm 4 walk
(Sec. 2.3): brute force on small inputs, structural invariants, and the coverage invariant
(every ordered particle pair handled exactly once, by P2P or by one cell-cell pair)."""
import numpy as np
import pytest

import oracle
from paper_1712_10116_gb300 import ics


def _keys_bruteforce(pos, lo, L):
    # independent bit-by-bit interleave of floor((x - lo) / (L / 2^21))
    h = L / 2.0 ** 21
    c = np.floor((pos - lo[:, None]) / h).astype(np.int64)
    c = np.clip(c, 0, 2 ** 21 - 1)
    keys = []
    for i in range(pos.shape[1]):
        k = 0
        for b in range(20, -1, -1):
            for a in range(3):
                k = (k << 1) | int((c[a, i] >> b) & 1)
        keys.append(k)
    return np.array(keys, dtype=np.uint64)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_root_cube_and_keys(seed):
    g = np.random.default_rng(seed)
    pos = g.standard_normal((3, 300)) * np.array([[3.0], [0.5], [1.0]]) + 7.0
    lo, L = oracle.root_cube(pos)
    assert 2.0 ** np.round(np.log2(L)) == L
    assert np.all(pos >= lo[:, None]) and np.all(pos < (lo + L)[:, None])
    ext = (pos.max(1) - pos.min(1)).max()
    assert ext <= L < 2.0 * ext * (1 + 2 ** -20)
    h = L / 2 ** 21
    assert np.all(np.floor(lo / h) * h == lo)
    keys = oracle.morton_keys(pos, lo, L)
    assert np.array_equal(keys, _keys_bruteforce(pos, lo, L))


def test_sort_is_stable_key_then_index():
    g = np.random.default_rng(9)
    keys = g.integers(0, 50, 500).astype(np.uint64)
    perm = oracle.sort_keys(keys)
    want = np.lexsort((np.arange(500), keys))
    assert np.array_equal(perm, want)


def _tree_case(kind, n):
    if kind == "plummer":
        pos, _, _ = ics.plummer(n, 1001)
    elif kind == "clustered":
        pos, _, _ = ics.clustered(n, 1007)
    else:
        pos, _, _ = ics.uniform_sphere(n, 1002)
    return pos


@pytest.mark.parametrize("kind", ["plummer", "clustered", "sphere"])
@pytest.mark.parametrize("n_crit", [8, 64])
def test_octree_structure(kind, n_crit):
    pos = _tree_case(kind, 3000)
    prm = oracle.params(p=3, theta=0.5, eps=0.01, n_crit=n_crit)
    t = oracle.Tree(pos, prm)
    assert t.level[0] == 0 and t.first[0] == 0 and t.count[0] == pos.shape[1]
    assert np.all(np.diff(t.level) >= 0)  # BFS order
    leaf = t.nchild == 0
    # leaves hold <= n_crit (unless at the deepest level), split cells hold > n_crit
    assert np.all(t.count[leaf & (t.level < 21)] <= n_crit)
    assert np.all(t.count[~leaf] > n_crit)
    # children partition the parent's range, in order
    for c in np.where(~leaf)[0]:
        kids = t.child_first[c] + np.arange(t.nchild[c])
        assert t.first[kids[0]] == t.first[c]
        assert np.all(t.first[kids[1:]] == t.first[kids[:-1]] + t.count[kids[:-1]])
        assert t.count[kids].sum() == t.count[c]
        assert np.all(t.level[kids] == t.level[c] + 1)
        assert np.all(t.coords[:, kids] // 2 == t.coords[:, c:c + 1])
    # leaves partition the particles, and each particle lies inside its leaf's cube
    assert t.count[leaf].sum() == pos.shape[1]
    sp = pos[:, t.perm]
    for c in np.where(leaf)[0]:
        lo = t.lo + t.coords[:, c] * t.side(c)
        q = sp[:, t.first[c]:t.first[c] + t.count[c]]
        assert np.all(q >= lo[:, None]) and np.all(q < (lo + t.side(c))[:, None])


def _ancestors(t):
    parent = np.full(t.ncell, -1, np.int64)
    for c in range(t.ncell):
        for k in range(t.nchild[c]):
            parent[t.child_first[c] + k] = c
    return parent


@pytest.mark.parametrize("kind,n,theta,p_crit", [("plummer", 700, 0.5, 16), ("clustered", 900, 0.7, 8),
                                                   ("sphere", 600, 0.35, 12)])
@pytest.mark.parametrize("kernel", [oracle.WENDLAND_C2, oracle.PLUMMER])
def test_walk_covers_every_pair_exactly_once(kind, n, theta, p_crit, kernel):
    pos = _tree_case(kind, n)
    prm = oracle.params(p=3, theta=theta, eps=0.02, n_crit=p_crit, kernel=kernel)
    t = oracle.Tree(pos, prm)
    m2l, p2p = t.lists()
    parent = _ancestors(t)
    leaf_of = np.zeros(n, np.int64)
    for c in np.where(t.nchild == 0)[0]:
        leaf_of[t.first[c]:t.first[c] + t.count[c]] = c
    # particle ranges of each cell in sorted order
    cover = np.zeros((n, n), np.int64)
    for a, b in p2p.T:
        assert t.nchild[a] == 0 and t.nchild[b] == 0
        cover[t.first[a]:t.first[a] + t.count[a], t.first[b]:t.first[b] + t.count[b]] += 1
    for a, b in m2l.T:
        cover[t.first[a]:t.first[a] + t.count[a], t.first[b]:t.first[b] + t.count[b]] += 1
    # the diagonal is covered once by the self pair P2P(A, A), whose evaluation skips i = j
    assert np.all(cover == 1)
    # lists are symmetric (directed closure of a symmetric walk)
    s_m2l = set(map(tuple, m2l.T))
    assert all((b, a) in s_m2l for a, b in s_m2l)
    s_p2p = set(map(tuple, p2p.T))
    assert all((b, a) in s_p2p for a, b in s_p2p)
    assert len(s_m2l) == m2l.shape[1] and len(s_p2p) == p2p.shape[1]
    del parent, leaf_of


def test_mac_decisions_match_float_geometry():
    # Eq. (1) with R = side (kappa = 1) evaluated from FP64 centres; ties are impossible here
    pos = _tree_case("plummer", 2000)
    prm = oracle.params(p=3, theta=0.6, eps=0.0, n_crit=16, kernel=oracle.PLUMMER)
    t = oracle.Tree(pos, prm)
    g = np.random.default_rng(11)
    cells = g.integers(0, t.ncell, (2, 3000))
    for a, b in cells.T:
        d = np.linalg.norm(t.centre(a) - t.centre(b))
        R = t.side(a) + t.side(b)
        want = d > R / prm.theta
        if abs(d - R / prm.theta) < 1e-9 * R:
            continue
        assert t.well_separated(a, b) == want


def test_softening_gap_rule():
    # Wendland: a cell pair with a gap below eps never uses M2L (Sec. 2.3)
    pos = _tree_case("sphere", 2000)
    eps = 0.3
    prm = oracle.params(p=3, theta=0.9, eps=eps, n_crit=8, kernel=oracle.WENDLAND_C2)
    t = oracle.Tree(pos, prm)
    m2l, p2p = t.lists()
    assert m2l.shape[1] > 0
    for a, b in m2l.T:
        gap = np.maximum(0.0, np.abs(t.centre(a) - t.centre(b)) - 0.5 * (t.side(a) + t.side(b)))
        assert np.linalg.norm(gap) > eps
    # Plummer: no gap rule, so some accepted pairs are closer than eps
    prm2 = oracle.params(p=3, theta=0.9, eps=eps, n_crit=8, kernel=oracle.PLUMMER)
    t2 = oracle.Tree(pos, prm2)
    m2l2, p2p2 = t2.lists()
    gaps = [np.linalg.norm(np.maximum(0.0, np.abs(t2.centre(a) - t2.centre(b)) - 0.5 * (t2.side(a) + t2.side(b))))
            for a, b in m2l2.T]
    assert min(gaps) < eps
    # the rule moves close pairs to direct summation
    assert p2p.shape[1] > p2p2.shape[1]


def test_walk_opens_both_cells():
    # every non-root pair's parent pair was not well separated, and children of equal-level
    # pairs come in full blocks (both cells opened, no one-sided split of equal cells)
    pos = _tree_case("clustered", 1500)
    prm = oracle.params(p=3, theta=0.5, eps=0.0, n_crit=16, kernel=oracle.PLUMMER)
    t = oracle.Tree(pos, prm)
    m2l, p2p = t.lists()
    parent = _ancestors(t)
    for a, b in np.concatenate([m2l, p2p], axis=1).T:
        if a == b or t.level[a] != t.level[b] or parent[a] < 0:
            continue
        pa, pb = parent[a], parent[b]
        assert not t.well_separated(pa, pb)
