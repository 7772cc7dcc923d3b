"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests
and the benchmark.

This module holds no arithmetic of the lattice Boltzmann method itself: it
only draws deterministic pseudo-random numbers (SplitMix64, Steele, Lea &
Flood 2014) and builds initial density fields from caller-given phase
densities (rho_l, rho_v).  The paper is silent on initial conditions; the
fields below are the ones used throughout this repository:

    rho0 = rho_v + (rho_l - rho_v) * 0.5 * (1 - tanh(2 d / width)) + noise
    noise = amp * (2 xi - 1),  xi = (SplitMix64(seed ^ (y*nx + x)) >> 11) / 2^53

where d is the signed distance to the liquid region (slab: |y - ny/2| - h;
droplet: r - R about (nx/2, ny/2); droplet array: r - R about the centre of
the enclosing cell).  A bubble swaps the two phases.
"""
from __future__ import annotations

import numpy as np

MASK64 = (1 << 64) - 1
SLAB, DROPLET, BUBBLE, DROPLET_ARRAY = 0, 1, 2, 3
KINDS = {"slab": SLAB, "droplet": DROPLET, "bubble": BUBBLE, "droplet_array": DROPLET_ARRAY}


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied to each uint64 of x (vectorised)."""
    z = (np.asarray(x, dtype=np.uint64) + np.uint64(0x9E3779B97F4A7C15))
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def uniform01(seed: int, counters: np.ndarray) -> np.ndarray:
    """xi in [0, 1) with 53 random bits, one per counter."""
    with np.errstate(over="ignore"):
        z = splitmix64(np.uint64(seed & MASK64) ^ np.asarray(counters, dtype=np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def density_field(nx: int, ny: int, kind: str | int, rho_l: float, rho_v: float,
                  size: float, width: float = 4.0, seed: int = 0, noise_amp: float = 1e-6,
                  cell: int = 256) -> np.ndarray:
    """Initial density rho0[y, x] (float64) for a slab, droplet, bubble or droplet array.

    size: slab half-width h, or droplet / bubble radius R.
    cell: side of the square cells of a droplet array (one droplet per cell).
    """
    k = KINDS[kind] if isinstance(kind, str) else int(kind)
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64),
                       indexing="ij")
    if k == SLAB:
        d = np.abs(y - ny / 2.0) - size
    elif k in (DROPLET, BUBBLE):
        d = np.hypot(x - nx / 2.0, y - ny / 2.0) - size
    elif k == DROPLET_ARRAY:
        cx = np.floor(x / cell) * cell + cell / 2.0
        cy = np.floor(y / cell) * cell + cell / 2.0
        d = np.hypot(x - cx, y - cy) - size
    else:
        raise ValueError("unknown kind %r" % (kind,))
    inside = 0.5 * (1.0 - np.tanh(2.0 * d / width))
    if k == BUBBLE:
        rho = rho_l + (rho_v - rho_l) * inside
    else:
        rho = rho_v + (rho_l - rho_v) * inside
    if noise_amp:
        ctr = np.arange(nx * ny, dtype=np.uint64).reshape(ny, nx)
        rho = rho + noise_amp * (2.0 * uniform01(seed, ctr) - 1.0)
    return np.ascontiguousarray(rho)


def random_populations(nx: int, ny: int, seed: int, base: float = 0.2, amp: float = 0.02) -> np.ndarray:
    """A smooth-ish positive population field f[a, y, x] for step-level tests:
    w_a * (base + amp * (2 xi - 1)) per population, independent per (a, y, x)."""
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    ctr = np.arange(9 * nx * ny, dtype=np.uint64).reshape(9, ny, nx)
    xi = uniform01(seed, ctr)
    return np.ascontiguousarray(w[:, None, None] * (base + amp * (2.0 * xi - 1.0)))


def batch_instances(n: int, seed: int, sides=tuple(range(64, 513, 32)),
                    t_range=(0.5, 0.9), tau_range=(0.55, 1.2), k_range=(1.0 / 16, 1.0)):
    """Parameters of n independent instances (dicts): side, T/Tc, tau, K, radius
    or half-width, kind ('droplet' or 'slab'), seed.  Five uniform draws per
    instance from the SplitMix64 stream (seed, 8*i + j)."""
    out = []
    for i in range(n):
        xi = uniform01(seed, np.arange(8 * i, 8 * i + 6, dtype=np.uint64))
        side = int(sides[min(int(xi[0] * len(sides)), len(sides) - 1)])
        tr = t_range[0] + (t_range[1] - t_range[0]) * xi[1]
        tau = tau_range[0] + (tau_range[1] - tau_range[0]) * xi[2]
        K = k_range[0] + (k_range[1] - k_range[0]) * xi[3]
        radius = 10.0 + (side / 4.0 - 10.0) * xi[4]
        kind = "droplet" if xi[5] < 0.5 else "slab"
        out.append(dict(side=side, T_over_Tc=float(tr), tau=float(tau), K=float(K),
                        size=float(radius), kind=kind, seed=int(seed * 1000 + i)))
    return out
