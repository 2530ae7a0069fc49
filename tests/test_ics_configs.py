"""The seeded inputs of the benchmark table's other workloads, checked against the profiles they are
drawn from (CPU): component masses and shapes of the disk galaxy, the displacement scale and clump
mass of the clustered box, the King W0 = 6 concentration and the ensemble's size range."""
import numpy as np

from paper_1712_10116_gb300 import ics


def test_disk_galaxy_components():
    pos, mass = ics.disk_galaxy(200_000, seed=11)
    assert pos.shape == (3, 200_000) and abs(mass.sum() - 1.0) < 1e-12
    # particle numbers split like the masses (10 / 5 / 85 %), so every particle weighs 1/N
    assert np.allclose(mass, 1.0 / 200_000, rtol=1e-12)
    disk, bulge, halo = ics._disk_galaxy_parts(ics.rng(12), 200_000, 3.0, 0.3, 0.6, 10.0, 30.0)
    assert (disk.shape[1], bulge.shape[1], halo.shape[1]) == (20_000, 10_000, 170_000)
    R = np.hypot(disk[0], disk[1])
    assert abs(R.mean() / 6.0 - 1.0) < 0.02                    # <R> = 2 Rd for an exponential disk
    assert abs(np.median(np.abs(disk[2])) / (0.3 * np.arctanh(0.5)) - 1.0) < 0.03   # sech^2: median |z|
    rb = np.linalg.norm(bulge, axis=0)
    assert abs(np.median(rb) / (0.6 / (np.sqrt(2.0) - 1.0)) - 1.0) < 0.03   # Hernquist half-mass radius
    assert np.linalg.norm(halo, axis=0).max() <= 30.0 * (1 + 1e-9)   # NFW truncated at r200


def test_nfw_radii_follow_the_enclosed_mass():
    g = ics.rng(3)
    r = ics._nfw_radii(g, 100_000, 10.0, 30.0)
    x = np.array([0.5, 1.0, 3.0, 10.0])
    m = (np.log1p(x) - x / (1 + x)) / (np.log1p(10.0) - 10.0 / 11.0)
    emp = np.array([(r <= xi * 3.0).mean() for xi in x])
    assert np.abs(emp - m).max() < 0.01


def test_clustered_box_scale_and_clumps():
    pos, mass = ics.clustered_box(32, seed=4, n_clumps=50)
    assert pos.shape == (3, 32 ** 3) and np.allclose(mass, 1.0 / 32 ** 3)
    # most particles stay within a few cells of their lattice site; the clumps pull the rest in
    grid = (np.indices((32, 32, 32)).reshape(3, -1) + 0.5) / 32
    d = np.linalg.norm(pos - grid, axis=0) * 32
    assert 0.2 < np.median(d) < 2.0


def test_king_concentration():
    r, m = ics._king_profile(6.0)
    assert abs(np.log10(r[-1]) - 1.26) < 0.02                  # c = log10(r_t / r_c) for W0 = 6
    assert m[0] == 0.0 and m[-1] == 1.0 and np.all(np.diff(m) >= 0)
    pos, _ = ics.king(50_000, 6.0, seed=2)
    rr = np.linalg.norm(pos, axis=0)
    assert abs(np.median(rr) / 1.305 - 1.0) < 0.02


def test_ensemble_sizes():
    systems = ics.ensemble()
    sizes = np.array([p.shape[1] for p, _ in systems])
    assert len(systems) == 64 and sizes.min() >= 2 ** 10 and sizes.max() <= 2 ** 17
    assert all(abs(m.sum() - 1.0) < 1e-12 for _, m in systems)


# ---------------------------------------------------------------- disk galaxy velocities (Jeans moments)
def _disk_sample(n=1 << 15, seed=1003):
    pos, vel, mass = ics.disk_galaxy(n, seed, velocities=True)
    pos0, mass0 = ics.disk_galaxy(n, seed)
    assert np.array_equal(pos, pos0) and np.array_equal(mass, mass0)   # velocities do not move the particles
    return pos, vel, mass


def test_disk_galaxy_virial_ratio():
    # the sampled system is near equilibrium: 2K / |W| = 1 within a few per cent, W from float64 direct
    # summation of the sample (Wendland eps = 0.02, the workload's softening)
    import oracle
    pos, vel, m = _disk_sample()
    _, pot = oracle.direct(pos, m, 0.02)
    K = 0.5 * float((m * (vel * vel).sum(0)).sum())
    W = 0.5 * float((m * pot).sum())
    assert abs(2.0 * K / -W - 1.0) < 0.05
    assert np.abs((vel * m).sum(1)).max() < 1e-15   # centre-of-mass frame


def test_disk_galaxy_rotation_curve_matches_direct_forces():
    # the model's midplane circular speed (spherical parts + Freeman's thin exponential disk) against the
    # radial pull measured by direct summation on particles near the midplane, in three annuli
    import oracle
    pos, vel, m = _disk_sample()
    model = ics.DiskGalaxyModel()
    R = np.hypot(pos[0], pos[1])
    plane = np.nonzero(np.abs(pos[2]) < 0.15)[0]   # sinks near the midplane (any component)
    for r0 in (3.0, 6.0, 9.0):
        sel = plane[np.abs(R[plane] - r0) < 0.5][:400]
        assert sel.size >= 100
        acc, _ = oracle.direct(pos, m, 0.02, sinks=sel)
        aR = -(acc[0] * pos[0, sel] + acc[1] * pos[1, sel]) / R[sel]
        vc2_meas = float(np.mean(aR * R[sel]))
        assert abs(vc2_meas / float(model.vc2(np.array([r0]))[0]) - 1.0) < 0.08, r0


def test_disk_galaxy_toomre_q_measured_back():
    # Q = sigma_R kappa / (3.36 Sigma) at the reference radius 2.43 rd, with sigma_R and Sigma measured
    # from the disk particles of an annulus and kappa from the model's rotation curve
    n = 1 << 18
    g = ics.rng(1003)
    disk, bulge, halo = ics._disk_galaxy_parts(g, n, 3.0, 0.3, 0.6, 10.0, 30.0)
    model = ics.DiskGalaxyModel()
    v = ics.disk_galaxy_velocities(ics.rng(1003 + 7919), model, disk, bulge, halo)[:, :disk.shape[1]]
    R = np.hypot(disk[0], disk[1])
    r0, half = model.r_ref, 0.4
    sel = np.abs(R - r0) < half
    vR = (v[0, sel] * disk[0, sel] + v[1, sel] * disk[1, sel]) / R[sel]
    sigma_surf = sel.sum() * (0.1 / disk.shape[1]) / (np.pi * ((r0 + half) ** 2 - (r0 - half) ** 2))
    k2, _ = model.kappa2_omega2(np.array([r0]))
    q = vR.std() * np.sqrt(k2[0]) / (3.36 * sigma_surf)
    assert abs(q / 1.5 - 1.0) < 0.06
    # the disk rotates: mean v_phi there is positive and below the circular speed (asymmetric drift)
    vphi = (-v[0, sel] * disk[1, sel] + v[1, sel] * disk[0, sel]) / R[sel]
    assert 0.0 < vphi.mean() < np.sqrt(model.vc2(np.array([r0]))[0])


# ---------------------------------------------------------------- King velocities (lowered Maxwellian)
def _king_u2(w):
    # <u^2> of p(u) ~ u^2 (e^(W - u^2/2) - 1), 0 < u < sqrt(2W), by quadrature
    u = np.linspace(0.0, np.sqrt(2.0 * w), 4001)
    f = u * u * (np.exp(w - 0.5 * u * u) - 1.0)
    return np.trapezoid(u * u * f, u) / np.trapezoid(f, u)


def test_king_velocity_profile_follows_the_distribution_function():
    # the mean square speed at depth W(r), relative to the core's, is that of the lowered Maxwellian:
    # this checks the rejection sampler and the potential profile, whatever the velocity unit
    pos, vel, m = ics.king(60_000, 6.0, 1005, velocities=True)
    pos0, m0 = ics.king(60_000, 6.0, 1005)
    assert np.array_equal(pos, pos0)
    r_c, mfrac, wr = ics._king_solution(6.0)
    scale = 1.305 / np.interp(0.5, mfrac, r_c)
    r = np.linalg.norm(pos, axis=0) / scale          # in core radii
    v2 = (vel * vel).sum(0)
    core = r < 0.5
    ref = v2[core].mean() / np.mean([_king_u2(w) for w in np.interp(r[core], r_c, wr)])
    for lo, hi in [(1.0, 2.0), (3.0, 5.0), (6.0, 9.0)]:
        sel = (r >= lo) & (r < hi)
        want = np.mean([_king_u2(w) for w in np.interp(r[sel], r_c, wr)])
        assert abs(v2[sel].mean() / ref / want - 1.0) < 0.06, (lo, hi)


def test_king_virial_ratio_against_direct_summation():
    import oracle
    pos, vel, m = ics.king(12_000, 6.0, 1005, velocities=True)
    _, pot = oracle.direct(pos, m, 1e-3, kernel=oracle.PLUMMER)
    K = 0.5 * float((m * (vel * vel).sum(0)).sum())
    W = 0.5 * float((m * pot).sum())
    assert abs(2.0 * K / -W - 1.0) < 0.02
