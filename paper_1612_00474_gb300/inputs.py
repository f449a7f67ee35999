"""Seeded synthetic roller monolayers (host only; no mobility arithmetic here).

This is the one module that both the CUDA path's tests/benchmark and the oracle
take inputs from.  It draws configurations shaped like the paper's sedimented
roller suspensions (Sec. III: spheres of radius a above a wall, in a layer a few
radii thick) with a generator of its own:

  - N spheres in a square of side L = sqrt(N pi a^2 / phi) (in-plane area fraction phi);
  - x, y ~ U(0, L);  z = a + Exp(mean = zmean);
  - a candidate closer than 2a (3D centre distance) to an accepted sphere is rejected
    and redrawn (random sequential addition), so no pair overlaps initially.

Random numbers come from numpy's Philox bit generator keyed by the seed.  The
paper's own initial states are Monte-Carlo samples of the Gibbs-Boltzmann
distribution in a 60a x 4915a periodic strip; those are not available, and these
configurations stand in for them.
"""
import math

import numpy as np


def monolayer(N, seed=0, phi=0.4, a=1.0, zmean=0.5, max_tries=1000):
    """Particle-major positions, shape (N, 3), float64."""
    if N <= 0:
        return np.zeros((0, 3))
    L = math.sqrt(N * math.pi * a * a / phi)
    rng = np.random.Generator(np.random.Philox(key=seed))
    cell = 2.0 * a
    nc = max(1, int(L // cell))
    csz = L / nc
    grid = {}
    pos = np.zeros((N, 3))
    n = 0
    tries = 0
    d2 = (2.0 * a) ** 2
    while n < N:
        batch = rng.random((256, 3))
        for u in batch:
            x, y = u[0] * L, u[1] * L
            z = a - zmean * math.log1p(-u[2])
            cx, cy = min(int(x / csz), nc - 1), min(int(y / csz), nc - 1)
            ok = True
            for ix in (cx - 1, cx, cx + 1):
                for iy in (cy - 1, cy, cy + 1):
                    for j in grid.get((ix, iy), ()):
                        p = pos[j]
                        if (p[0] - x) ** 2 + (p[1] - y) ** 2 + (p[2] - z) ** 2 < d2:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if ok:
                pos[n] = (x, y, z)
                grid.setdefault((cx, cy), []).append(n)
                n += 1
                tries = 0
                if n == N:
                    break
            else:
                tries += 1
                if tries > max_tries:
                    raise RuntimeError(f"could not place sphere {n} of {N} at phi={phi}")
    return pos


def batch_sizes(B, lo=64, hi=2048, seed=0):
    """B instance sizes drawn log-uniformly in [lo, hi] (integers)."""
    rng = np.random.Generator(np.random.Philox(key=10_000 + seed))
    u = rng.random(B)
    return np.floor(np.exp(math.log(lo) + u * (math.log(hi + 1) - math.log(lo)))).astype(np.int64).clip(lo, hi)


def vectors(N, seed, scale=1.0):
    """Generic seeded (N, 3) test vectors (forces, torques, noise stand-ins) ~ N(0, scale^2)."""
    rng = np.random.Generator(np.random.Philox(key=20_000 + seed))
    return scale * rng.standard_normal((N, 3))


def to_soa(x):
    """(N, 3) particle-major -> flat SoA [x_0..x_{N-1} | y_0.. | z_0..] (the CUDA library's layout)."""
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64).T).ravel()


def from_soa(v, N):
    """Flat SoA of length 3N -> (N, 3) particle-major."""
    return np.asarray(v, dtype=np.float64).reshape(3, N).T.copy()
