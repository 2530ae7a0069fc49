"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on the same
seeded inputs.  Integer work (root cube, Morton keys, sort permutation, octree cells,
interaction lists, timestep rungs) must match bit for bit; forces to 1e-12 relative in the
float64 path and to the float32 bound below in the float32 path."""
import numpy as np
import pytest
import torch

import oracle
from paper_1712_10116_gb300 import ics

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1712_10116_gb300 import binding as tg
    DEV = torch.device("cuda:0")

# float32 path bound: |a_gpu - a_oracle| <= 1e-5 * max(|a_oracle|, 0.1 * median |a_oracle|) per
# particle.  Float32 positions relative to a leaf centre carry a rounding of ~6e-8 of the leaf size,
# so the absolute force error is ~1e-6 of the typical (median) force whatever a particle's own net
# force; particles whose contributions cancel to below 10% of the typical force are therefore held
# to 1e-5 of that floor, since their own float32 net force cannot be resolved to 1e-5 of itself.
FP32_TOL = 1e-5
FP32_FLOOR = 0.1


def _case(kind, n, seed=None):
    if kind == "plummer":
        return ics.plummer(n, seed or 1001)
    if kind == "sphere":
        return ics.uniform_sphere(n, seed or 1002)
    if kind == "clustered":
        return ics.clustered(n, seed or 1007)
    raise ValueError(kind)


def _t(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def _oprm(prm):
    return oracle.params(p=prm.p, theta=prm.theta, eps=prm.eps, kernel=prm.kernel, n_crit=prm.n_crit,
                         kappa=prm.kappa, max_level=prm.max_level, mac=prm.mac)


def _rel(a, b, floor=0.0):
    nb = np.linalg.norm(b, axis=0)
    den = np.maximum(nb, floor * np.median(nb))
    return np.linalg.norm(a - b, axis=0) / den


def _check_fp32(a, a_o, tag="", floor=FP32_FLOOR, tol=FP32_TOL):
    """Float32 parity: the floored per-particle bound is asserted; the unfloored distribution (each
    particle against its own force) is printed beside it."""
    r = _rel(a, a_o, floor)
    u = _rel(a, a_o)
    print(f"fp32 parity {tag}: floored max {r.max():.3e} (bound {tol:.0e}); unfloored max {u.max():.3e}, "
          f"p99.9 {np.percentile(u, 99.9):.3e}, median {np.median(u):.3e}")
    assert r.max() < tol, (tag, r.max(), np.median(r))
    return r


def _abs_pull(pos, mass, eps, kernel=0, chunk=512):
    """A_i = sum_j m_j |g(r_ij)| r_ij: the force particle i would feel if every pull were aligned.  The
    rounding error of any evaluation order of the force sum is bounded by a multiple of u A_i
    (u = unit roundoff), whatever the cancellation in the net force a_i."""
    n = pos.shape[1]
    out = np.zeros(n)
    for i0 in range(0, n, chunk):
        d = pos[:, None, :] - pos[:, i0:i0 + chunk, None]
        r = np.sqrt((d * d).sum(0))
        if kernel == 1:
            g = (r * r + eps * eps) ** -1.5
        else:
            u = r / eps
            with np.errstate(divide="ignore"):
                g = np.where(u < 1, (21 * u ** 5 - 90 * u ** 4 + 140 * u ** 3 - 84 * u ** 2 + 14) / eps ** 3, r ** -3.0)
        g[r == 0] = 0.0
        out[i0:i0 + chunk] = (mass[None, :] * g * r).sum(1)
    return out


@pytest.mark.parametrize("kind,n,n_crit", [("plummer", 5000, 64), ("clustered", 7777, 16), ("sphere", 3001, 8),
                                           ("plummer", 1, 64), ("sphere", 64, 64), ("sphere", 65, 64)])
def test_tree_bit_exact(kind, n, n_crit):
    pos, _, _ = _case(kind, n)
    prm = tg.Params(p=4, theta=0.5, eps=0.01, n_crit=n_crit)
    s = tg.Solver(prm)
    tg.tg_build_tree(s.ctx, _t(pos))
    g = tg.tg_get_tree(s.ctx)
    t = oracle.Tree(pos, _oprm(prm))
    assert np.array_equal(g["lo"], t.lo) and g["L"] == t.L
    assert np.array_equal(g["keys"], t.keys)
    assert np.array_equal(g["perm"], t.perm)
    assert np.array_equal(g["level"], t.level)
    assert np.array_equal(g["coords"], t.coords)
    assert np.array_equal(g["first"], t.first)
    assert np.array_equal(g["count"], t.count)
    assert np.array_equal(g["nchild"], t.nchild)


def test_tree_coincident_and_far_points():
    g_ = np.random.default_rng(5)
    pos = np.concatenate([np.zeros((3, 150)), g_.normal(1e3, 1e-3, (3, 40)), g_.normal(0, 1, (3, 97))], axis=1)
    prm = tg.Params(p=3, theta=0.5, eps=0.01, n_crit=8)
    s = tg.Solver(prm)
    tg.tg_build_tree(s.ctx, _t(pos))
    g = tg.tg_get_tree(s.ctx)
    t = oracle.Tree(pos, _oprm(prm))
    for k in ("keys", "perm", "level", "coords", "first", "count", "nchild"):
        assert np.array_equal(g[k], getattr(t, k)), k


def _directed(pairs):
    s = set()
    for a, b in pairs.T:
        s.add((int(a), int(b)))
        s.add((int(b), int(a)))
    return s


@pytest.mark.parametrize("kind,n,theta,n_crit,kernel", [
    ("plummer", 4000, 0.5, 32, 0), ("clustered", 6000, 0.7, 16, 1), ("sphere", 3000, 0.35, 24, 0)])
def test_interaction_lists_match_oracle(kind, n, theta, n_crit, kernel):
    pos, _, mass = _case(kind, n)
    prm = tg.Params(p=3, theta=theta, eps=0.02, n_crit=n_crit, kernel=kernel)
    s = tg.Solver(prm)
    s.fmm_forces(_t(pos), _t(mass))
    m2l, p2p = tg.tg_get_lists(s.ctx)
    t = oracle.Tree(pos, _oprm(prm))
    om2l, op2p = t.lists()
    # every unordered pair appears once on the GPU
    assert len({tuple(sorted(p)) for p in m2l.T}) == m2l.shape[1]
    assert len({tuple(sorted(p)) for p in p2p.T}) == p2p.shape[1]
    assert _directed(m2l) == set(map(tuple, om2l.T.tolist()))
    assert _directed(p2p) == set(map(tuple, op2p.T.tolist()))


@pytest.mark.parametrize("kind,n,theta,n_crit,kernel", [
    ("plummer", 4000, 0.5, 32, 0), ("clustered", 6000, 0.7, 16, 1), ("sphere", 3000, 0.35, 24, 0)])
def test_sphere_mac_lists_match_oracle(kind, n, theta, n_crit, kernel):
    # the enclosing-sphere criterion: radii and decisions in float64 with the oracle's rounding, so
    # the lists must be identical
    pos, _, mass = _case(kind, n)
    prm = tg.Params(p=3, theta=theta, eps=0.02, n_crit=n_crit, kernel=kernel, mac=tg.TG_MAC_SPHERE)
    s = tg.Solver(prm)
    s.fmm_forces(_t(pos), _t(mass))
    m2l, p2p = tg.tg_get_lists(s.ctx)
    t = oracle.Tree(pos, _oprm(prm))
    om2l, op2p = t.lists()
    assert _directed(m2l) == set(map(tuple, om2l.T.tolist()))
    assert _directed(p2p) == set(map(tuple, op2p.T.tolist()))
    # and it differs from the side criterion on the same input
    t_side = oracle.Tree(pos, oracle.params(p=3, theta=theta, eps=0.02, n_crit=n_crit, kernel=kernel))
    assert set(map(tuple, t_side.lists()[0].T.tolist())) != set(map(tuple, om2l.T.tolist()))


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("masked", [False, True])
def test_sphere_mac_forces_match_oracle(precision, masked):
    n = 6000
    pos, _, _ = _case("clustered", n)
    mass = ics.random_masses(n, 11)
    fast = ics.random_fast_mask(n, 12) if masked else None
    prm = tg.Params(p=5, theta=0.5, eps=0.01, kernel=0, precision=precision, n_crit=32, mac=tg.TG_MAC_SPHERE)
    s = tg.Solver(prm)
    acc, pot = s.fmm_forces(_t(pos), _t(mass), None if fast is None else _t(fast, torch.uint8))
    a_o, p_o = oracle.fmm(pos, mass, _oprm(prm), fast)
    if precision == tg.TG_PREC_FP64:
        assert _rel(acc.cpu().numpy(), a_o).max() < 1e-12
    else:
        _check_fp32(acc.cpu().numpy(), a_o)


@pytest.mark.parametrize("split", ["half", "shell"])
@pytest.mark.parametrize("p,kernel", [(6, 0), (5, 1)])
def test_fmm_fp32_spatial_classes_match_oracle(split, p, kernel):
    # fast particles in one region (a half-space, or an outer shell like the HHS rungs of a collapse):
    # most cells hold a single class, where M2L reuses or drops the class-1 contraction
    n = 12000
    pos, _, mass = _case("sphere", n)
    r = np.linalg.norm(pos, axis=0)
    fast = ((pos[0] > 0.1) if split == "half" else (r > 0.7)).astype(np.uint8)
    prm = tg.Params(p=p, theta=0.5, eps=0.005 if kernel == 0 else 0.01, kernel=kernel, precision=tg.TG_PREC_FP32,
                    n_crit=32)
    s = tg.Solver(prm)
    for want_pot in (True, False):
        acc, _ = s.fmm_forces(_t(pos), _t(mass), _t(fast, torch.uint8), want_pot=want_pot)
        a_o, _ = oracle.fmm(pos, mass, _oprm(prm), fast)
        _check_fp32(acc.cpu().numpy(), a_o)


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("p", [2, 4, 6])
@pytest.mark.parametrize("masked", [False, True])
def test_fmm_fp64_matches_oracle(kernel, p, masked):
    n = 6000
    pos, _, _ = _case("clustered", n)
    mass = ics.random_masses(n, 11)
    fast = ics.random_fast_mask(n, 12) if masked else None
    prm = tg.Params(p=p, theta=0.5, eps=0.01, kernel=kernel, precision=tg.TG_PREC_FP64, n_crit=32)
    s = tg.Solver(prm)
    acc, pot = s.fmm_forces(_t(pos), _t(mass), None if fast is None else _t(fast, torch.uint8))
    a_o, p_o = oracle.fmm(pos, mass, _oprm(prm), fast)
    a = acc.cpu().numpy()
    assert _rel(a, a_o).max() < 1e-12
    assert np.abs(pot.cpu().numpy() - p_o).max() < 1e-12 * np.abs(p_o).max()


@pytest.mark.parametrize("kind,kernel,p,theta", [("sphere", 0, 6, 0.5), ("plummer", 1, 4, 0.5),
                                                 ("clustered", 0, 5, 0.45)])
@pytest.mark.parametrize("masked", [False, True])
def test_fmm_fp32_matches_oracle(kind, kernel, p, theta, masked):
    n = 9000
    pos, _, mass = _case(kind, n)
    fast = ics.random_fast_mask(n, 13) if masked else None
    eps = 0.005 if kernel == 0 else 0.01
    prm = tg.Params(p=p, theta=theta, eps=eps, kernel=kernel, precision=tg.TG_PREC_FP32, n_crit=64)
    s = tg.Solver(prm)
    acc, pot = s.fmm_forces(_t(pos), _t(mass), None if fast is None else _t(fast, torch.uint8))
    a_o, p_o = oracle.fmm(pos, mass, _oprm(prm), fast)
    _check_fp32(acc.cpu().numpy(), a_o)
    assert np.abs(pot.cpu().numpy() - p_o).max() < FP32_TOL * np.abs(p_o).max()


@pytest.mark.parametrize("n_crit", [160, 256])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_leaves_wider_than_a_p2p_tile(n_crit, precision):
    # leaves of more than 128 particles: the P2P kernels take their columns in several tiles
    n = 20000
    pos, _, mass = _case("clustered", n)
    fast = ics.random_fast_mask(n, 19)
    prec = tg.TG_PREC_FP64 if precision == "fp64" else tg.TG_PREC_FP32
    prm = tg.Params(p=6, theta=0.5, eps=0.005, kernel=0, precision=prec, n_crit=n_crit)
    s = tg.Solver(prm)
    for mask in (None, fast):
        acc, _ = s.fmm_forces(_t(pos), _t(mass), None if mask is None else _t(mask, torch.uint8))
        a_o, _ = oracle.fmm(pos, mass, _oprm(prm), mask)
        if precision == "fp64":
            nb = np.linalg.norm(a_o, axis=0)
            assert (np.linalg.norm(acc.cpu().numpy() - a_o, axis=0) / nb).max() < 1e-12
        else:
            _check_fp32(acc.cpu().numpy(), a_o)
    s.close()


@pytest.mark.parametrize("kind", ["sphere", "clustered"])
@pytest.mark.parametrize("masked", [False, True])
def test_fmm_fp32_wide_softening(kind, masked):
    # eps well above the mean spacing: many particle pairs of neighbouring leaves lie inside the
    # Wendland kernel's support (Eq. 8), so the softened branch of P2P carries real weight
    n = 9000
    pos, _, mass = _case(kind, n)
    fast = ics.random_fast_mask(n, 17) if masked else None
    prm = tg.Params(p=5, theta=0.5, eps=0.1, kernel=0, precision=tg.TG_PREC_FP32, n_crit=64)
    s = tg.Solver(prm)
    acc, pot = s.fmm_forces(_t(pos), _t(mass), None if fast is None else _t(fast, torch.uint8))
    a_o, p_o = oracle.fmm(pos, mass, _oprm(prm), fast)
    _check_fp32(acc.cpu().numpy(), a_o)
    assert np.abs(pot.cpu().numpy() - p_o).max() < FP32_TOL * np.abs(p_o).max()


@pytest.mark.parametrize("rows", [1, 2, 3])
@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("masked", [False, True])
def test_p2p_rows_per_lane_match_oracle(rows, kernel, masked):
    # every rows-per-lane variant of the float32 P2P that the autotuner may choose, with and without the
    # potential: wide Wendland softening puts many pairs of neighbouring leaves inside eps (the clamped
    # pairs and their correction), and the mask adds the fast-row pass over the slow columns
    n = 9000
    pos, _, mass = _case("clustered", n)
    fast = ics.random_fast_mask(n, 23) if masked else None
    prm = tg.Params(p=5, theta=0.5, eps=0.1 if kernel == 0 else 0.01, kernel=kernel, precision=tg.TG_PREC_FP32,
                    n_crit=64)
    s = tg.Solver(prm)
    t = tg.tg_get_tuning(s.ctx)
    t["p2p_rows"] = rows
    tg.tg_set_tuning(s.ctx, t)
    assert tg.tg_get_tuning(s.ctx)["p2p_rows"] == rows
    a_o, p_o = oracle.fmm(pos, mass, _oprm(prm), fast)
    fs = None if fast is None else _t(fast, torch.uint8)
    for want_pot in (False, True):
        acc, pot = s.fmm_forces(_t(pos), _t(mass), fs, want_pot=want_pot)
        _check_fp32(acc.cpu().numpy(), a_o, f"rows {rows} kernel {kernel} masked {masked} pot {want_pot}")
        if want_pot:
            assert np.abs(pot.cpu().numpy() - p_o).max() < FP32_TOL * np.abs(p_o).max()
    s.close()


@pytest.mark.parametrize("kind,kernel,p", [("sphere", 0, 6), ("plummer", 1, 5), ("clustered", 0, 4)])
@pytest.mark.parametrize("masked", [False, True])
def test_fmm_fp32_forces_only(kind, kernel, p, masked):
    # accelerations without the potential (what the HHS kicks ask for): the float32 kernels then skip
    # the potential sums (P2P) and the L^0 term (M2L, L2P); the accelerations must not change
    n = 9000
    pos, _, mass = _case(kind, n)
    fast = ics.random_fast_mask(n, 19) if masked else None
    prm = tg.Params(p=p, theta=0.5, eps=0.005 if kernel == 0 else 0.01, kernel=kernel, precision=tg.TG_PREC_FP32,
                    n_crit=64)
    s = tg.Solver(prm)
    fs = None if fast is None else _t(fast, torch.uint8)
    acc_f, pot_f = s.fmm_forces(_t(pos), _t(mass), fs, want_pot=False)
    acc_p, _ = s.fmm_forces(_t(pos), _t(mass), fs, want_pot=True)
    assert pot_f is None
    a_o, _ = oracle.fmm(pos, mass, _oprm(prm), fast)
    _check_fp32(acc_f.cpu().numpy(), a_o, "forces only")
    # same arithmetic for the accelerations in both forms; the float32 atomics that sum the local
    # expansions (M2L) run in a different order on each launch, so the two agree to the float32 bound
    assert _rel(acc_f.cpu().numpy(), acc_p.cpu().numpy(), FP32_FLOOR).max() < FP32_TOL


@pytest.mark.parametrize("precision", [0, 1])
def test_momentum_conserved_on_gpu(precision):
    n = 20000
    pos, _, _ = _case("clustered", n)
    mass = ics.random_masses(n, 21)
    fast = ics.random_fast_mask(n, 22)
    prm = tg.Params(p=5, theta=0.45, eps=0.005, precision=precision, n_crit=64)
    s = tg.Solver(prm)
    acc, _ = s.fmm_forces(_t(pos), _t(mass), _t(fast, torch.uint8))
    a = acc.cpu().numpy()
    res = np.abs((a * mass).sum(1)).max() / np.abs(a * mass).sum()
    assert res < (1e-14 if precision == 0 else 1e-6), res


def test_direct_matches_oracle():
    n = 3000
    pos, _, mass = _case("plummer", n)
    fast = ics.random_fast_mask(n, 3)
    prm = tg.Params(p=3, eps=0.01, kernel=0)
    s = tg.Solver(prm)
    sinks = np.random.default_rng(1).choice(n, 500, replace=False)
    acc, pot = s.direct_forces(_t(pos), _t(mass), _t(fast, torch.uint8), _t(sinks, torch.int64))
    a_o, p_o = oracle.direct(pos, mass, 0.01, 0, fast, sinks)
    assert _rel(acc.cpu().numpy(), a_o).max() < 1e-13
    assert np.allclose(pot.cpu().numpy(), p_o, rtol=1e-13)


def test_timesteps_bit_exact():
    g_ = np.random.default_rng(7)
    n = 20000
    a_old = np.where(g_.uniform(size=n) < 0.3, 0.0, 10 ** g_.uniform(-3, 3, n))
    a_cur = 10 ** g_.uniform(-3, 3, n)
    a_cur[:5] = 0.0
    a_old[:3] = 0.0
    prm = tg.Params(eps=0.005, eta=0.025, dt_max=1.0 / 128, k_max=10)
    s = tg.Solver(prm)
    dt, rung = tg.tg_timesteps(s.ctx, _t(a_old), _t(a_cur))
    dt = dt.cpu().numpy()
    rung = rung.cpu().numpy()
    for i in range(n):
        want = oracle.timestep(0.025, 0.005, a_old[i], a_cur[i])
        assert dt[i] == want or (np.isinf(dt[i]) and np.isinf(want))
        assert rung[i] == oracle.rung(want, 1.0 / 128, 10)


def test_timesteps_eq9_bit_exact():
    # the Eq. (9) minimum timestep from |a|_tot, against the oracle's float64 function
    g_ = np.random.default_rng(9)
    n = 20000
    a_old = np.where(g_.uniform(size=n) < 0.3, 0.0, 10 ** g_.uniform(-3, 3, n))
    a_cur = 10 ** g_.uniform(-3, 3, n)
    a_tot = np.where(g_.uniform(size=n) < 0.1, 0.0, 10 ** g_.uniform(-3, 4, n))
    a_cur[:5] = 0.0
    a_old[:3] = 0.0
    prm = tg.Params(eps=0.005, eta=0.025, dt_max=1.0 / 128, k_max=10, eta_tot=0.004)
    s = tg.Solver(prm)
    dt, rung = tg.tg_timesteps(s.ctx, _t(a_old), _t(a_cur), _t(a_tot))
    dt = dt.cpu().numpy()
    rung = rung.cpu().numpy()
    bound = 0
    for i in range(n):
        want = oracle.timestep_tot(0.025, 0.005, a_old[i], a_cur[i], 0.004, a_tot[i])
        bound += want < oracle.timestep(0.025, 0.005, a_old[i], a_cur[i])
        assert dt[i] == want or (np.isinf(dt[i]) and np.isinf(want))
        assert rung[i] == oracle.rung(want, 1.0 / 128, 10)
    assert 0 < bound < n   # the constraint binds for some particles, not all


@pytest.mark.parametrize("n", [1, 2, 17])
def test_small_and_degenerate_inputs(n):
    pos, _, mass = _case("plummer", max(n, 1))
    prm = tg.Params(p=4, theta=0.5, eps=0.01, n_crit=8)
    s = tg.Solver(prm)
    acc, pot = s.fmm_forces(_t(pos), _t(mass))
    a_o, p_o = oracle.fmm(pos, mass, _oprm(prm))
    assert np.allclose(acc.cpu().numpy(), a_o, rtol=1e-12, atol=1e-300)
    assert np.allclose(pot.cpu().numpy(), p_o, rtol=1e-12, atol=1e-300)


def test_coincident_particles_and_all_fast():
    pos = np.zeros((3, 40))
    mass = np.full(40, 0.025)
    prm = tg.Params(p=4, theta=0.5, eps=0.01, n_crit=4)
    s = tg.Solver(prm)
    acc, pot = s.fmm_forces(_t(pos), _t(mass))
    assert torch.all(acc == 0)
    assert np.allclose(pot.cpu().numpy(), -39 * 0.025 * 3 / 0.01)
    # every particle fast: F-F pairs are skipped, so no force at all
    pos2, _, mass2 = _case("plummer", 500)
    acc2, pot2 = s.fmm_forces(_t(pos2), _t(mass2), torch.ones(500, dtype=torch.uint8, device=DEV))
    assert torch.all(acc2 == 0) and torch.all(pot2 == 0)


def test_empty_input():
    for precision in (tg.TG_PREC_FP64, tg.TG_PREC_FP32):
        s = tg.Solver(tg.Params(p=4, precision=precision))
        acc, pot = s.fmm_forces(torch.zeros((3, 0), dtype=torch.float64, device=DEV),
                                torch.zeros(0, dtype=torch.float64, device=DEV))
        assert acc.shape == (3, 0) and pot.shape == (0,)


@pytest.mark.parametrize("shape", ["planar", "collinear", "big_clump", "shallow"])
@pytest.mark.parametrize("precision", [0, 1])
def test_degenerate_geometry_matches_oracle(shape, precision):
    # flat and one-dimensional sets (zero extent along some axes), a clump of coincident particles
    # larger than one column stage (a deepest-level leaf with 300 > 128 particles), and a tree cut off
    # at level 1 (eight leaves of ~400 particles): the chunked P2P paths
    g = np.random.default_rng(31)
    n, max_level, n_crit = 3000, 21, 16
    if shape == "planar":
        pos = np.concatenate([g.uniform(-1, 1, (2, n)), np.zeros((1, n))])
    elif shape == "collinear":
        pos = np.concatenate([g.uniform(-1, 1, (1, n)), np.zeros((2, n))])
    elif shape == "big_clump":
        pos = np.concatenate([np.full((3, 300), 0.25), g.uniform(-1, 1, (3, n - 300))], axis=1)
    else:
        pos, max_level, n_crit = g.uniform(-1, 1, (3, n)), 1, 8
    mass = ics.random_masses(n, 32)
    fast = ics.random_fast_mask(n, 33)
    prm = tg.Params(p=4, theta=0.5, eps=0.02, kernel=0, precision=precision, n_crit=n_crit, max_level=max_level)
    s = tg.Solver(prm)
    for mask in (None, fast):
        acc, _ = s.fmm_forces(_t(pos), _t(mass), None if mask is None else _t(mask, torch.uint8))
        a_o, _ = oracle.fmm(pos, mass, _oprm(prm), mask)
        # on a line (and, less so, in a plane) the pulls from both sides cancel to a small net force
        # for the particles in the middle.  The rounding of a sum of terms is bounded by a multiple of
        # u * sum |terms| whatever the order, so each particle's bound is taken against
        # max(|a_i|, 0.1 A_i) with A_i its summed absolute pull: float32 rounding (u = 6e-8) over a few
        # thousand terms in blocked order stays near 1e-6 A_i, float64 near 1e-13 A_i
        a = acc.cpu().numpy()
        A = _abs_pull(pos, mass, 0.02)
        den = np.maximum(np.linalg.norm(a_o, axis=0), 0.1 * A)
        r = np.linalg.norm(a - a_o, axis=0) / den
        tol = 1e-12 if precision == tg.TG_PREC_FP64 else FP32_TOL
        print(f"{shape} {'fp64' if precision == 0 else 'fp32'} mask={mask is not None}: max {r.max():.3e} "
              f"against max(|a|, 0.1 A) (bound {tol:.0e}); unfloored max {_rel(a, a_o).max():.3e}")
        assert r.max() < tol, r.max()


def test_argument_errors_leave_outputs():
    prm = tg.Params()
    s = tg.Solver(prm)
    cpu = torch.zeros((3, 10), dtype=torch.float64)
    with pytest.raises((tg.TGError, ValueError)):
        tg.tg_fmm_forces(s.ctx, cpu, torch.zeros(10, dtype=torch.float64))
    with pytest.raises(tg.TGError):
        tg.tg_hhs_step(s.ctx)
    with pytest.raises(tg.TGError):
        tg.tg_create(tg.Params(p=0))
    with pytest.raises(tg.TGError):
        tg.tg_create(tg.Params(p=21))


# ---------------------------------------------------------------- HHS
def _two_rung_system(k, eta=0.02, eps=1e-3):
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
def test_poisson_calls_match_paper_count(k):
    # GPU evaluates each kick pair once: (2 + 2 + 2^(k+1)) masked calls = 2 + 2^(k+1) evaluations
    pos, vel, m, dt_max = _two_rung_system(k)
    prm = tg.Params(p=4, theta=0.5, eps=1e-3, n_crit=8, eta=0.02, dt_max=dt_max, k_max=12)
    s = tg.Solver(prm)
    P, V, M = _t(pos), _t(vel), _t(m)
    s.hhs_init(P, V, M)
    h = oracle.HHS(pos, vel, m, _oprm(prm), eta=0.02, dt_max=dt_max, k_max=12)
    for _ in range(2):
        tg.tg_reset_stats(s.ctx)
        s.hhs_step()
        st = s.stats()
        ost, _ = h.step()
        assert st["evaluations"] == ost.poisson_calls - 2
        assert st["sink_forces"] == ost.sink_forces
        assert st["max_rung"] == k


@pytest.mark.parametrize("kernel", [0, 1])
def test_hhs_fp64_matches_oracle(kernel):
    n = 1500
    pos, vel, mass = _case("plummer", n)
    eps = 0.01
    prm = tg.Params(p=4, theta=0.5, eps=eps, kernel=kernel, precision=tg.TG_PREC_FP64, n_crit=32, eta=0.025,
                    dt_max=1.0 / 16, k_max=6)
    s = tg.Solver(prm)
    P, V, M = _t(pos), _t(vel), _t(mass)
    s.hhs_init(P, V, M)
    h = oracle.HHS(pos, vel, mass, _oprm(prm), eta=0.025, dt_max=1.0 / 16, k_max=6)
    for step in range(3):
        s.hhs_step()
        h.step()
        rung, a_old, a_cur = tg.tg_hhs_state(s.ctx, n)
        assert np.array_equal(rung.cpu().numpy(), h.rung), step
        scale_x = np.abs(h.pos).max()
        assert np.abs(P.cpu().numpy() - h.pos).max() < 1e-11 * scale_x
        assert np.abs(V.cpu().numpy() - h.vel).max() < 1e-10 * np.abs(h.vel).max()
    assert len(np.unique(h.rung)) >= 2


@pytest.mark.parametrize("kernel", [0, 1])
def test_hhs_fp64_eq9_matches_oracle(kernel):
    # HHS with the Eq. (9) minimum timestep: |a|_tot from the whole system at rung 0 (one extra
    # all-masses evaluation on the GPU when a fast set exists) and the capped timesteps
    n = 1500
    pos, vel, mass = _case("plummer", n)
    eps = 0.01
    prm = tg.Params(p=4, theta=0.5, eps=eps, kernel=kernel, precision=tg.TG_PREC_FP64, n_crit=32, eta=0.025,
                    dt_max=1.0 / 16, k_max=6, eta_tot=0.006)
    s = tg.Solver(prm)
    P, V, M = _t(pos), _t(vel), _t(mass)
    s.hhs_init(P, V, M)
    h = oracle.HHS(pos, vel, mass, _oprm(prm), eta=0.025, dt_max=1.0 / 16, k_max=6, eta_tot=0.006)
    h0 = oracle.HHS(pos, vel, mass, _oprm(prm), eta=0.025, dt_max=1.0 / 16, k_max=6)
    for step in range(3):
        s.hhs_step()
        h.step()
        h0.step()
        rung, a_old, a_cur, a_tot = tg.tg_hhs_state(s.ctx, n, with_total=True)
        assert np.array_equal(rung.cpu().numpy(), h.rung), step
        assert np.allclose(a_tot.cpu().numpy(), h.a_tot, rtol=1e-11, atol=0), step
        scale_x = np.abs(h.pos).max()
        assert np.abs(P.cpu().numpy() - h.pos).max() < 1e-11 * scale_x
        assert np.abs(V.cpu().numpy() - h.vel).max() < 1e-10 * np.abs(h.vel).max()
    # the constraint is active in this run: some particles sit deeper than without it
    assert np.any(h.rung > h0.rung)


@pytest.mark.parametrize("precision", [0, 1])
def test_hhs_momentum_drift(precision):
    n = 20000
    pos, vel, mass = _case("clustered", n)
    mass = ics.random_masses(n, 31)
    vel = vel - (vel * mass).sum(1, keepdims=True) / mass.sum()
    prm = tg.Params(p=5, theta=0.45, eps=0.002, precision=precision, n_crit=64, eta=0.02, dt_max=1.0 / 16, k_max=8)
    s = tg.Solver(prm)
    P, V, M = _t(pos), _t(vel), _t(mass)
    s.hhs_init(P, V, M)
    d0 = s.diagnostics()
    for _ in range(2):
        s.hhs_step()
    d1 = s.diagnostics()
    scale = float((np.abs(vel) * mass).sum())
    drift = np.abs(d1[:3] - d0[:3]).max() / scale
    assert drift < (1e-14 if precision == 0 else 1e-6), drift
    assert s.stats()["max_rung"] >= 2


# ---------------------------------------------------------------- full-size workload, sampled
def test_cold_collapse_full_size_sampled():
    # the benchmark workload: uniform sphere N = 2^20, eps = 0.005, p = 6, theta = 0.5, float32
    n = 1 << 20
    pos, _, mass = _case("sphere", n)
    prm = tg.Params(p=6, theta=0.5, eps=0.005, kernel=0, precision=tg.TG_PREC_FP32, n_crit=64)
    s = tg.Solver(prm)
    acc, _ = s.fmm_forces(_t(pos), _t(mass))
    sample = np.random.default_rng(5).choice(n, 40, replace=False)
    a_o, _ = oracle.fmm_sample(pos, mass, _oprm(prm), sample)
    a = acc.cpu().numpy()[:, sample]
    r = np.linalg.norm(a - a_o, axis=0) / np.linalg.norm(a_o, axis=0)
    assert r.max() < FP32_TOL, r.max()
    # and the FMM error against FP64 direct summation is inside the 1e-4 median gate
    ad, _ = s.direct_forces(_t(pos), _t(mass), None, _t(sample, torch.int64))
    e = np.linalg.norm(a - ad.cpu().numpy(), axis=0) / np.linalg.norm(ad.cpu().numpy(), axis=0)
    assert np.median(e) < 1e-4


# ---------------------------------------------------------------- orders above the fixed tables
@pytest.mark.parametrize("p,kernel,masked,precision", [(10, 0, False, 0), (14, 0, True, 0), (20, 0, False, 0),
                                                       (20, 0, True, 0), (12, 1, False, 0), (12, 1, True, 0),
                                                       (10, 0, False, 1), (10, 0, True, 1)])
def test_high_order_matches_oracle(p, kernel, masked, precision):
    # table-free kernels for 8 < p <= 20 (harmonic M2L for Wendland, the full set for Plummer)
    n = 1200
    pos, _, _ = _case("clustered", n)
    mass = ics.random_masses(n, 11)
    fast = ics.random_fast_mask(n, 12) if masked else None
    prm = tg.Params(p=p, theta=0.5, eps=0.01, kernel=kernel, precision=precision, n_crit=32)
    s = tg.Solver(prm)
    acc, pot = s.fmm_forces(_t(pos), _t(mass), None if fast is None else _t(fast, torch.uint8))
    a_o, p_o = oracle.fmm(pos, mass, _oprm(prm), fast)
    a = acc.cpu().numpy()
    if precision == tg.TG_PREC_FP64:
        assert _rel(a, a_o).max() < 1e-12
        assert np.abs(pot.cpu().numpy() - p_o).max() < 1e-12 * np.abs(p_o).max()
    else:
        _check_fp32(a, a_o, f"p={p}")


def test_high_order_error_falls_to_roundoff():
    n = 1500
    pos, _, _ = _case("clustered", n)
    mass = ics.random_masses(n, 11)
    ad, _ = oracle.direct(pos, mass, 0.01, oracle.WENDLAND_C2)
    med = []
    for p in (8, 12, 16, 20):
        s = tg.Solver(tg.Params(p=p, theta=0.5, eps=0.01, kernel=0, precision=tg.TG_PREC_FP64, n_crit=32))
        acc, _ = s.fmm_forces(_t(pos), _t(mass))
        med.append(np.median(_rel(acc.cpu().numpy(), ad)))
    assert all(b < a / 20 for a, b in zip(med, med[1:]))
    assert med[-1] < 1e-12



# ---------------------------------------------------------------- both forms of the harmonic float32 M2L
@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("masked", [False, True])
def test_fp32_m2l_forms_match_oracle(form, masked):
    # 0: mutual, a lane per cell pair of a walk block, both sides combined across lanes (the default);
    # 1: directed, a warp per target cell over its source list
    n = 6000
    pos, _, _ = _case("clustered", n)
    mass = ics.random_masses(n, 11)
    fast = ics.random_fast_mask(n, 12) if masked else None
    prm = tg.Params(p=6, theta=0.5, eps=0.005, kernel=0, precision=tg.TG_PREC_FP32, n_crit=32)
    s = tg.Solver(prm)
    t = tg.tg_get_tuning(s.ctx)
    t["m2l_form"] = form
    tg.tg_set_tuning(s.ctx, t)
    acc, pot = s.fmm_forces(_t(pos), _t(mass), None if fast is None else _t(fast, torch.uint8))
    a_o, p_o = oracle.fmm(pos, mass, _oprm(prm), fast)
    _check_fp32(acc.cpu().numpy(), a_o, f"m2l form {form} masked={masked}")
    assert np.abs(pot.cpu().numpy() - p_o).max() < FP32_TOL * np.abs(p_o).max()
