"""Seeded synthetic initial conditions (CPU, float64).

This module holds only input generators: it draws particle sets with the shapes, sizes and
density profiles of the paper's workloads and contains none of the solver's arithmetic.  Both
the CUDA path's tests/benchmark and the oracle tests take their inputs from here.

Random numbers come from numpy's Philox-4x32-10 counter-based generator (Salmon et al. 2011),
seeded per call.  Units: G = M = 1.  Positions and velocities are (3, n) float64 arrays,
masses (n,) float64 summing to 1.
"""
from __future__ import annotations

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
