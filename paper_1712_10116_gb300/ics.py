"""Seeded synthetic initial conditions (CPU, float64).

This module holds only input generators: it draws particle sets with the shapes, sizes and
density profiles of the paper's workloads and contains none of the solver's arithmetic.  Both
the CUDA path's tests/benchmark and the oracle tests take their inputs from here.

Random numbers come from numpy's Philox-4x32-10 counter-based generator (Salmon et al. 2011),
seeded per call.  Units: G = M = 1.  Positions and velocities are (3, n) float64 arrays,
masses (n,) float64 summing to 1.
"""
from __future__ import annotations

import functools

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


def _isotropic(g: np.random.Generator, n: int) -> np.ndarray:
    cos_t = g.uniform(-1.0, 1.0, n)
    phi = g.uniform(0.0, 2.0 * np.pi, n)
    sin_t = np.sqrt(1.0 - cos_t * cos_t)
    return np.stack([sin_t * np.cos(phi), sin_t * np.sin(phi), cos_t])


def _to_com_frame(pos, vel, mass):
    pos = pos - (pos * mass).sum(axis=1, keepdims=True) / mass.sum()
    vel = vel - (vel * mass).sum(axis=1, keepdims=True) / mass.sum()
    return pos, vel


def plummer(n: int, seed: int = 1001, a: float = 1.0, r_max: float = 50.0):
    """Plummer sphere (scale a, total mass 1), velocities from its distribution function.

    Radii invert the enclosed-mass profile M(<r) = r^3 / (r^2 + a^2)^(3/2); speeds use the
    rejection method of Aarseth, Henon & Wielen (1974) on q^2 (1 - q^2)^(7/2), q = v / v_esc.
    The rare far tail beyond r_max * a is redrawn.  Returned in the centre-of-mass frame.
    """
    g = rng(seed)
    r = np.empty(n)
    filled = 0
    while filled < n:
        x = g.uniform(0.0, 1.0, n - filled)
        x = x[x > 0]
        rr = a / np.sqrt(x ** (-2.0 / 3.0) - 1.0)
        rr = rr[rr < r_max * a]
        r[filled:filled + rr.size] = rr
        filled += rr.size
    pos = _isotropic(g, n) * r
    q = np.empty(n)
    filled = 0
    while filled < n:
        m = 2 * (n - filled) + 16
        x1 = g.uniform(0.0, 1.0, m)
        x2 = g.uniform(0.0, 0.1, m)
        ok = x2 < x1 * x1 * (1.0 - x1 * x1) ** 3.5
        acc = x1[ok][: n - filled]
        q[filled:filled + acc.size] = acc
        filled += acc.size
    v_esc = np.sqrt(2.0) * (1.0 + (r / a) ** 2) ** (-0.25) / np.sqrt(a)
    vel = _isotropic(g, n) * (q * v_esc)
    mass = np.full(n, 1.0 / n)
    pos, vel = _to_com_frame(pos, vel, mass)
    return pos, vel, mass


def uniform_sphere(n: int, seed: int = 1002, radius: float = 1.0):
    """Cold collapse input: uniform-density sphere at rest (virial ratio 0)."""
    g = rng(seed)
    r = radius * g.uniform(0.0, 1.0, n) ** (1.0 / 3.0)
    pos = _isotropic(g, n) * r
    vel = np.zeros((3, n))
    mass = np.full(n, 1.0 / n)
    return pos, vel, mass


def uniform_cube(n: int, seed: int = 1006, side: float = 1.0):
    """Cold collapse from a cube of unit side at rest (the paper's run-time test, Sec. 3.1)."""
    g = rng(seed)
    pos = g.uniform(-0.5 * side, 0.5 * side, (3, n))
    vel = np.zeros((3, n))
    mass = np.full(n, 1.0 / n)
    return pos, vel, mass


def cube_softening(n: int) -> float:
    """eps = 0.01 (N / 10^4)^(-1/3), the softening scaling of the cube collapse (Sec. 3.1)."""
    return 0.01 * (n / 1.0e4) ** (-1.0 / 3.0)


def two_body(separation: float = 1.0, eccentricity: float = 0.0):
    """Two equal masses (0.5 each) at apocentre of a Kepler orbit with semi-major axis
    `separation` / (1 + e); total mass 1, so the period is 2 pi a^(3/2)."""
    e = eccentricity
    a = separation / (1.0 + e)
    # relative speed at apocentre of an orbit with total mass 1
    v_rel = np.sqrt((1.0 - e) / (a * (1.0 + e)))
    pos = np.array([[-0.5 * separation, 0.5 * separation], [0.0, 0.0], [0.0, 0.0]])
    vel = np.array([[0.0, 0.0], [-0.5 * v_rel, 0.5 * v_rel], [0.0, 0.0]])
    mass = np.array([0.5, 0.5])
    return pos, vel, mass, a


def random_masses(n: int, seed: int, spread: float = 10.0) -> np.ndarray:
    """Unequal masses, log-uniform over a factor `spread`, normalised to total 1."""
    g = rng(seed)
    m = np.exp(g.uniform(0.0, np.log(spread), n))
    return m / m.sum()


def random_fast_mask(n: int, seed: int, fraction: float = 0.3) -> np.ndarray:
    """A random fast/slow partition (uint8, 1 = fast) for masked force evaluations."""
    g = rng(seed)
    return (g.uniform(0.0, 1.0, n) < fraction).astype(np.uint8)


def clustered(n: int, seed: int = 1007, n_clumps: int = 8, clump_scale: float = 0.05,
              background: float = 0.3):
    """A small clustered set: Plummer-like clumps on a uniform background in a unit cube.

    Used to exercise deep, uneven octrees in tests (not one of the benchmark workloads)."""
    g = rng(seed)
    n_bg = int(background * n)
    n_cl = n - n_bg
    centres = g.uniform(-0.4, 0.4, (3, n_clumps))
    which = g.integers(0, n_clumps, n_cl)
    x = g.uniform(0.0, 1.0, n_cl)
    x = np.clip(x, 1e-12, 1.0 - 1e-9)
    r = clump_scale / np.sqrt(x ** (-2.0 / 3.0) - 1.0)
    r = np.minimum(r, 0.5)
    cl = centres[:, which] + _isotropic(g, n_cl) * r
    bg = g.uniform(-0.5, 0.5, (3, n_bg))
    pos = np.concatenate([cl, bg], axis=1)
    perm = g.permutation(n)
    pos = pos[:, perm]
    vel = 0.1 * g.standard_normal((3, n))
    mass = np.full(n, 1.0 / n)
    return pos, vel, mass


def _nfw_radii(g: np.random.Generator, n: int, c: float, r200: float) -> np.ndarray:
    """Radii drawn from an NFW profile of concentration c truncated at r200: the enclosed mass
    m(x) = ln(1 + x) - x / (1 + x), x = r / r_s, r_s = r200 / c, inverted by bisection."""
    u = g.uniform(0.0, 1.0, n) * (np.log1p(c) - c / (1.0 + c))
    lo, hi = np.zeros(n), np.full(n, float(c))
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        below = np.log1p(mid) - mid / (1.0 + mid) < u
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    return 0.5 * (lo + hi) * (r200 / c)


def disk_galaxy(n: int = 1 << 22, seed: int = 1003, rd: float = 3.0, z0: float = 0.3, bulge_a: float = 0.6,
                halo_c: float = 10.0, r200: float = 30.0, velocities: bool = False, toomre_q: float = 1.5):
    """Isolated disk galaxy: an exponential disk (surface density ~ exp(-R/rd), vertical sech^2(z/z0))
    with 10 % of the mass and of the particles, a Hernquist bulge of scale bulge_a with 5 %, and an
    NFW halo (concentration halo_c, truncated at r200) with 85 %; equal masses within a component.

    Returns (pos, mass), or with velocities=True (pos, vel, mass): velocities from Jeans moments in the
    model's own potential (disk_galaxy_velocities), drawn from a separate stream so that the positions
    are the same either way."""
    g = rng(seed)
    disk, bulge, halo = _disk_galaxy_parts(g, n, rd, z0, bulge_a, halo_c, r200)
    nd, nb, nh = disk.shape[1], bulge.shape[1], halo.shape[1]
    pos = np.concatenate([disk, bulge, halo], axis=1)
    mass = np.concatenate([np.full(nd, 0.10 / nd), np.full(nb, 0.05 / nb), np.full(nh, 0.85 / nh)])
    perm = g.permutation(n)
    if not velocities:
        return np.ascontiguousarray(pos[:, perm]), mass[perm]
    model = DiskGalaxyModel(rd=rd, z0=z0, bulge_a=bulge_a, halo_c=halo_c, r200=r200, toomre_q=toomre_q)
    vel = disk_galaxy_velocities(rng(seed + 7919), model, disk, bulge, halo)
    vel = vel - (vel * mass).sum(axis=1, keepdims=True) / mass.sum()
    return np.ascontiguousarray(pos[:, perm]), np.ascontiguousarray(vel[:, perm]), mass[perm]


class DiskGalaxyModel:
    """Mass profiles and Jeans moments of the disk galaxy (G = 1, total mass 1).

    Spherical parts: Hernquist bulge (mass 0.05, scale a, truncated where its enclosed-mass fraction
    reaches 0.999, as the sampler does) and NFW halo (mass 0.85 within r200, concentration c).  The
    disk (mass 0.10, scale rd) enters the spheres' Jeans equation through its enclosed mass
    0.1 [1 - (1 + r/rd) e^(-r/rd)] (a spherical average), and the disk's own rotation curve through
    Freeman's (1970) exact midplane formula for a thin exponential disk."""

    M_DISK, M_BULGE, M_HALO = 0.10, 0.05, 0.85

    def __init__(self, rd=3.0, z0=0.3, bulge_a=0.6, halo_c=10.0, r200=30.0, toomre_q=1.5):
        self.rd, self.z0, self.a, self.c, self.r200, self.q = rd, z0, bulge_a, halo_c, r200, toomre_q
        s = np.sqrt(0.999)
        self.rt_bulge = bulge_a * s / (1.0 - s)
        self.rs = r200 / halo_c
        self._mu_c = np.log1p(halo_c) - halo_c / (1.0 + halo_c)
        self.r_ref = 2.43 * rd      # radius where Q is set (Hernquist 1993: the solar neighbourhood)

    # -- enclosed masses and densities of the spherical parts
    def m_bulge(self, r):
        r = np.minimum(r, self.rt_bulge)
        return self.M_BULGE / 0.999 * (r / (r + self.a)) ** 2

    def rho_bulge(self, r):
        return np.where(r < self.rt_bulge, self.M_BULGE / 0.999 * self.a / (2.0 * np.pi * r * (r + self.a) ** 3), 0.0)

    def m_halo(self, r):
        x = np.minimum(r, self.r200) / self.rs
        return self.M_HALO * (np.log1p(x) - x / (1.0 + x)) / self._mu_c

    def rho_halo(self, r):
        x = r / self.rs
        rho0 = self.M_HALO / (4.0 * np.pi * self.rs ** 3 * self._mu_c)
        return np.where(r < self.r200, rho0 / (x * (1.0 + x) ** 2), 0.0)

    def m_disk_sph(self, r):
        y = r / self.rd
        return self.M_DISK * (1.0 - (1.0 + y) * np.exp(-y))

    def m_total(self, r):
        return self.m_bulge(r) + self.m_halo(r) + self.m_disk_sph(r)

    def sigma_r2(self, comp, r):
        """Isotropic Jeans equation of a spherical component in the total enclosed mass:
        rho sigma^2 (r) = int_r^r_t rho(s) M(<s) / s^2 ds, integrated on a logarithmic grid."""
        rt = self.rt_bulge if comp == "bulge" else self.r200
        rho = self.rho_bulge if comp == "bulge" else self.rho_halo
        grid = np.geomspace(1e-5, rt, 6000)
        f = rho(grid) * self.m_total(grid) / grid ** 2
        seg = 0.5 * (f[1:] + f[:-1]) * np.diff(grid)
        tail = np.concatenate([np.cumsum(seg[::-1])[::-1], [0.0]])   # int_grid[i]^rt
        rs = np.clip(r, grid[0], rt)
        integral = np.interp(rs, grid, tail)
        with np.errstate(divide="ignore", invalid="ignore"):
            s2 = integral / rho(rs)
        return np.where(np.isfinite(s2), np.maximum(s2, 0.0), 0.0)

    # -- disk kinematics (epicyclic approximation)
    def sigma_disk(self, R):
        return self.M_DISK / (2.0 * np.pi * self.rd ** 2) * np.exp(-R / self.rd)

    def vc2(self, R):
        """Circular speed squared in the midplane: spheres plus Freeman's thin-disk term
        4 pi Sigma_0 rd y^2 [I0 K0 - I1 K1](y), y = R / (2 rd)."""
        from scipy.special import i0e, i1e, k0e, k1e
        y = np.maximum(R, 1e-12) / (2.0 * self.rd)
        sig0 = self.M_DISK / (2.0 * np.pi * self.rd ** 2)
        disk = 4.0 * np.pi * sig0 * self.rd * y * y * (i0e(y) * k0e(y) - i1e(y) * k1e(y))   # e^y e^-y cancel
        sph = (self.m_bulge(R) + self.m_halo(R)) / np.maximum(R, 1e-12)
        return sph + disk

    def kappa2_omega2(self, R):
        """kappa^2 = R dOmega^2/dR + 4 Omega^2 and Omega^2 = v_c^2 / R^2 (numerical derivative on a log grid)."""
        grid = np.geomspace(1e-3, 20.0 * self.rd + 1.0, 4000)
        om2 = self.vc2(grid) / grid ** 2
        k2 = grid * np.gradient(om2, grid) + 4.0 * om2
        Rc = np.clip(R, grid[0], grid[-1])
        return np.interp(Rc, grid, k2), np.interp(Rc, grid, om2)

    def sigma_R2_norm(self):
        """sigma_R^2 = A exp(-R/rd) (Hernquist 1993), with A set by Toomre's Q = sigma_R kappa / (3.36 Sigma)
        at r_ref."""
        k2, _ = self.kappa2_omega2(np.array([self.r_ref]))
        sR = 3.36 * self.q * self.sigma_disk(self.r_ref) / np.sqrt(k2[0])
        return sR * sR * np.exp(self.r_ref / self.rd)

    def disk_moments(self, R):
        """(sigma_R^2, sigma_phi^2, sigma_z^2, mean v_phi) of the disk at cylindrical radius R:
        sigma_z^2 = pi Sigma z0 (isothermal sheet), sigma_phi^2 = sigma_R^2 kappa^2 / (4 Omega^2), and the
        asymmetric drift v_phi^2 = v_c^2 + sigma_R^2 (1 - kappa^2 / (4 Omega^2) - 2 R / rd), clipped at 0."""
        sR2 = self.sigma_R2_norm() * np.exp(-R / self.rd)
        k2, om2 = self.kappa2_omega2(R)
        ratio = k2 / (4.0 * om2)
        sphi2 = sR2 * ratio
        sz2 = np.pi * self.sigma_disk(R) * self.z0
        vphi2 = self.vc2(R) + sR2 * (1.0 - ratio - 2.0 * R / self.rd)
        return sR2, sphi2, sz2, np.sqrt(np.maximum(vphi2, 0.0))


def disk_galaxy_velocities(g, model, disk, bulge, halo):
    """Velocities of the three components (positions as _disk_galaxy_parts returns them), concatenated:
    Gaussian draws with the Jeans moments of `model` (Hernquist 1993's approach); the bulge and the halo
    are isotropic, the disk streams with the asymmetric-drift-corrected rotation."""
    R = np.hypot(disk[0], disk[1])
    sR2, sphi2, sz2, vphi = model.disk_moments(R)
    vR = g.standard_normal(R.size) * np.sqrt(sR2)
    vp = vphi + g.standard_normal(R.size) * np.sqrt(sphi2)
    vz = g.standard_normal(R.size) * np.sqrt(sz2)
    cphi, sphi = disk[0] / np.maximum(R, 1e-300), disk[1] / np.maximum(R, 1e-300)
    vdisk = np.stack([vR * cphi - vp * sphi, vR * sphi + vp * cphi, vz])
    parts = [vdisk]
    for comp, p in (("bulge", bulge), ("halo", halo)):
        s = np.sqrt(model.sigma_r2(comp, np.sqrt((p * p).sum(0))))
        parts.append(g.standard_normal(p.shape) * s)
    return np.concatenate(parts, axis=1)


def _disk_galaxy_parts(g, n, rd, z0, bulge_a, halo_c, r200):
    """The three components of disk_galaxy, in that order, before they are mixed."""
    nd, nb = int(round(0.10 * n)), int(round(0.05 * n))
    nh = n - nd - nb
    R = g.gamma(2.0, rd, nd)                          # p(R) ~ R exp(-R / rd)
    phi = g.uniform(0.0, 2.0 * np.pi, nd)
    z = z0 * np.arctanh(g.uniform(-1.0, 1.0, nd) * (1.0 - 1e-12))
    disk = np.stack([R * np.cos(phi), R * np.sin(phi), z])
    s = np.sqrt(g.uniform(0.0, 0.999, nb))            # Hernquist: M(r) ~ r^2 / (r + a)^2
    bulge = _isotropic(g, nb) * (bulge_a * s / (1.0 - s))
    halo = _isotropic(g, nh) * _nfw_radii(g, nh, halo_c, r200)
    return disk, bulge, halo


def clustered_box(n_side: int = 256, seed: int = 1004, n_clumps: int = 1000, disp_rms: float = 0.5,
                  clump_cap: float = 0.5, c: float = 10.0):
    """Clustered cosmology-like set of n_side^3 equal-mass particles in the unit cube (isolated): a
    lattice displaced by the Zel'dovich approximation of a Gaussian random field with P(k) ~ k^-2,
    scaled to an rms displacement of disp_rms cells, then n_clumps NFW halos (concentration c) made
    by moving randomly chosen particles onto the halo profiles.  Halo masses are log-uniform in
    1e-5 .. 1e-2 of the total and rescaled to sum to clump_cap when they exceed it (their expected
    sum, 1.45, would exceed the total); r200 follows from M = 200 (4 pi / 3) r200^3 (mean density 1)."""
    g = rng(seed)
    ns = n_side
    n, h = ns ** 3, 1.0 / ns
    k1 = 2.0 * np.pi * np.fft.fftfreq(ns, d=h)
    kr = 2.0 * np.pi * np.fft.rfftfreq(ns, d=h)
    kx, ky, kz = np.meshgrid(k1, k1, kr, indexing="ij")
    k2 = kx * kx + ky * ky + kz * kz
    k2[0, 0, 0] = 1.0
    delta = (g.standard_normal(k2.shape) + 1j * g.standard_normal(k2.shape)) / np.sqrt(k2)   # sqrt(P(k)) = 1/k
    delta[0, 0, 0] = 0.0
    psi = np.empty((3, n))
    for a, ka in enumerate((kx, ky, kz)):
        psi[a] = np.fft.irfftn(1j * ka / k2 * delta, s=(ns, ns, ns), axes=(0, 1, 2)).reshape(-1)
    del kx, ky, kz, k2, delta
    psi *= disp_rms * h / np.sqrt((psi * psi).sum(axis=0).mean())
    pos = (np.indices((ns, ns, ns)).reshape(3, -1) + 0.5) * h + psi
    m = np.exp(g.uniform(np.log(1e-5), np.log(1e-2), n_clumps))
    if m.sum() > clump_cap:
        m *= clump_cap / m.sum()
    counts = np.maximum(1, np.round(m * n).astype(np.int64))
    order = g.permutation(n)
    centres = pos[:, g.integers(0, n, n_clumps)]
    start = 0
    for i in range(n_clumps):
        idx = order[start:start + counts[i]]
        start += counts[i]
        r200 = (3.0 * m[i] / (800.0 * np.pi)) ** (1.0 / 3.0)
        pos[:, idx] = centres[:, i:i + 1] + _isotropic(g, idx.size) * _nfw_radii(g, idx.size, c, r200)
    return np.ascontiguousarray(pos), np.full(n, 1.0 / n)


@functools.lru_cache(maxsize=4)
def _king_profile(w0: float, dr: float = 1e-3):
    """King (1966) model in core radii: the dimensionless potential W(r) from W(0) = w0 down to the
    tidal radius (W = 0), with density rho(W) ~ e^W erf(sqrt W) - sqrt(4W/pi) (1 + 2W/3) and
    W'' + 2W'/r = -9 rho(W) / rho(w0) (fourth-order Runge-Kutta).  Returns radii and the enclosed mass
    fraction, which is proportional to -r^2 W'(r)."""
    r, m, _ = _king_solution(w0, dr)
    return r, m


@functools.lru_cache(maxsize=4)
def _king_solution(w0: float, dr: float = 1e-3):
    """Radii, enclosed mass fractions and W(r) of the King model (see _king_profile)."""
    from math import erf, exp, pi, sqrt

    def rho(w):
        return exp(w) * erf(sqrt(w)) - sqrt(4.0 * w / pi) * (1.0 + 2.0 * w / 3.0) if w > 0 else 0.0

    r0 = rho(w0)

    def f(r, y):
        return (y[1], -9.0 * rho(y[0]) / r0 - 2.0 * y[1] / r)

    r = dr
    y = (w0 - 1.5 * dr * dr, -3.0 * dr)   # series start: W = w0 - 3/2 r^2
    rs, ms, ws = [0.0, r], [0.0, -r * r * y[1]], [w0, y[0]]
    while y[0] > 0.0:
        k1 = f(r, y)
        k2 = f(r + dr / 2, (y[0] + dr / 2 * k1[0], y[1] + dr / 2 * k1[1]))
        k3 = f(r + dr / 2, (y[0] + dr / 2 * k2[0], y[1] + dr / 2 * k2[1]))
        k4 = f(r + dr, (y[0] + dr * k3[0], y[1] + dr * k3[1]))
        y = (y[0] + dr / 6 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0]),
             y[1] + dr / 6 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1]))
        r += dr
        rs.append(r)
        ms.append(-r * r * y[1])
        ws.append(max(y[0], 0.0))
    ms = np.maximum.accumulate(np.array(ms))
    return np.array(rs), ms / ms[-1], np.array(ws)


def king(n: int, w0: float = 6.0, seed: int = 1005, r_half: float = 1.305, velocities: bool = False):
    """King (1966) sphere with central potential w0, positions and equal masses, scaled to the
    half-mass radius r_half (1.305 is that of the Plummer sphere with a = 1).

    With velocities=True also returns velocities from the King distribution function, a lowered
    Maxwellian f ~ exp(W - v^2 / (2 s^2)) - 1 for v^2 < 2 W s^2 (W the local dimensionless potential):
    speeds in units of s by rejection from p(u) ~ u^2 (e^(W - u^2/2) - 1), u < sqrt(2W), isotropic
    directions; s is then set by the virial theorem, 2K = -W_pot, with the potential energy of the
    spherical mass profile, -sum_i m_i M(< r_i) / r_i (G = 1).  Returns (pos, vel, mass), centre-of-mass
    frame for the velocities."""
    g = rng(seed)
    r, mfrac, wr = _king_solution(w0)
    u0 = g.uniform(0.0, 1.0, n)
    core = np.interp(u0, mfrac, r)                     # radii in core radii
    scale = r_half / np.interp(0.5, mfrac, r)
    pos = np.ascontiguousarray(_isotropic(g, n) * (core * scale))
    mass = np.full(n, 1.0 / n)
    if not velocities:
        return pos, mass
    w = np.interp(core, r, wr)                        # local depth W of every particle
    umax = np.sqrt(2.0 * np.maximum(w, 0.0))
    speed = np.zeros(n)
    todo = np.nonzero(umax > 0)[0]
    # envelope: p(u) <= u^2 e^(W - u^2/2) <= 2 e^(W - 1) / ... ; bound it by its maximum on a grid per W
    grid = np.linspace(0.0, 1.0, 257)[1:]
    while todo.size:
        uu = g.uniform(0.0, 1.0, todo.size) * umax[todo]
        wt = w[todo]
        f = uu * uu * (np.exp(wt - 0.5 * uu * uu) - 1.0)
        ug = grid[None, :] * umax[todo, None]
        fmax = (ug * ug * (np.exp(wt[:, None] - 0.5 * ug * ug) - 1.0)).max(axis=1) * 1.05
        ok = g.uniform(0.0, 1.0, todo.size) * fmax < f
        speed[todo[ok]] = uu[ok]
        todo = todo[~ok]
    vel = _isotropic(g, n) * speed
    # the velocity unit from the virial theorem of the sampled positions
    order = np.argsort(np.linalg.norm(pos, axis=0))
    rr = np.linalg.norm(pos, axis=0)[order]
    menc = np.cumsum(mass[order]) - mass[order]
    w_pot = -float(np.sum(mass[order] * menc / np.maximum(rr, 1e-12)))
    k_unit = 0.5 * float(np.sum(mass * (vel * vel).sum(0)))
    vel *= np.sqrt(-w_pot / (2.0 * k_unit))
    vel -= (vel * mass).sum(axis=1, keepdims=True) / mass.sum()
    return pos, np.ascontiguousarray(vel), mass


def ensemble(seed: int = 1005, n_systems: int = 64, log2n=(10.0, 17.0), velocities: bool = False):
    """Ensemble of independent systems: sizes round(2^U(10, 17)); even members Plummer spheres
    (a = 1), odd members King W0 = 6 spheres of the same half-mass radius; each of total mass 1.
    Returns a list of (pos, mass), or with velocities=True of (pos, vel, mass) (Plummer and King
    distribution functions)."""
    g = rng(seed)
    sizes = np.round(2.0 ** g.uniform(log2n[0], log2n[1], n_systems)).astype(np.int64)
    out = []
    for s, ns in enumerate(sizes):
        if s % 2 == 0:
            pos, vel, mass = plummer(int(ns), seed * 1000 + s)
            out.append((pos, vel, mass) if velocities else (pos, mass))
        else:
            out.append(king(int(ns), 6.0, seed * 1000 + s, velocities=velocities))
    return out
