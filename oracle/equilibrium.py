"""Equilibrium of a sedimented suspension (Appendix B): Metropolis sampling of the Gibbs-Boltzmann
distribution and the two statistics the paper compares Brownian dynamics against.

TEST INFRASTRUCTURE ONLY: see oracle/__init__.py.

  mc_sample          Metropolis Monte Carlo (mcmc.c) of exp(-U/kT), U = gravity + the soft wall and
                     pair potentials of Eq. (soft_potential), pseudo-periodic in x, y (minimum image);
                     the uniforms come from numpy's Philox keyed by the seed
  height_histogram   P(h), the density of sphere heights
  pair_correlation   g(r) with r the three-dimensional (minimum-image) centre distance, normalised as
                     for a two-dimensional suspension, so that g -> 1 for r >> a and g(r < 2a) = 0 for
                     hard spheres (Appendix B)
"""
import ctypes
import math

import numpy as np

from . import build as _build
from .core import lib

_mc = None


def _lib():
    global _mc
    if _mc is None:
        L = lib()
        dp = ctypes.POINTER(ctypes.c_double)
        i64, d = ctypes.c_int64, ctypes.c_double
        L.oracle_mc_energy.argtypes = [i64, dp, d, d, d, d, d, d]
        L.oracle_mc_energy.restype = d
        L.oracle_mc_sweeps.argtypes = [i64, dp, i64, dp, d, d, d, d, d, d, d, d]
        L.oracle_mc_sweeps.restype = i64
        _mc = L
    return _mc


def _p(x):
    return x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def mc_energy(pos, a=1.0, weight=1.0, U0=1.0, b=0.1, periodic=None):
    """Total energy U of a configuration (one-body terms plus each pair once)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    Lx, Ly = periodic if periodic is not None else (0.0, 0.0)
    return float(_lib().oracle_mc_energy(pos.shape[0], _p(pos), a, weight, U0, b, float(Lx), float(Ly)))


def mc_sample(pos0, nsamples, seed, thin=10, burn=200, step=0.15, kT=1.0, a=1.0, weight=1.0, U0=1.0, b=0.1,
              periodic=None):
    """nsamples configurations, one every `thin` sweeps after `burn` sweeps, from pos0 (N, 3).
    Returns (array (nsamples, N, 3), acceptance rate)."""
    pos = np.array(pos0, dtype=np.float64).reshape(-1, 3).copy()
    N = pos.shape[0]
    Lx, Ly = periodic if periodic is not None else (0.0, 0.0)
    rng = np.random.Generator(np.random.Philox(key=seed))
    L = _lib()
    acc = 0
    moves = 0

    def sweeps(n):
        nonlocal acc, moves
        u = rng.random(4 * N * n)
        acc += int(L.oracle_mc_sweeps(N, _p(pos), n, _p(u), step, kT, a, weight, U0, b, float(Lx), float(Ly)))
        moves += N * n

    if burn:
        sweeps(burn)
    out = np.empty((nsamples, N, 3))
    for k in range(nsamples):
        sweeps(thin)
        out[k] = pos
    return out, acc / max(1, moves)


def height_histogram(samples, edges):
    """Density of the heights of every sphere in every sample over the bins `edges`."""
    h = np.asarray(samples)[..., 2].ravel()
    cnt, _ = np.histogram(h, bins=edges)
    return cnt / (h.size * np.diff(edges))


def pair_correlation(samples, edges, periodic):
    """g(r) over the bins `edges` (Appendix B): the three-dimensional minimum-image distances of all
    pairs, counted per bin and divided by what a uniform two-dimensional suspension of the same
    number density would give, N (N - 1) / 2 / (Lx Ly) * pi (r_hi^2 - r_lo^2) per sample."""
    Lx, Ly = periodic
    S = np.asarray(samples)
    ns, N, _ = S.shape
    iu = np.triu_indices(N, 1)
    cnt = np.zeros(len(edges) - 1)
    for s in range(ns):
        p = S[s]
        dx = p[:, None, 0] - p[None, :, 0]
        dy = p[:, None, 1] - p[None, :, 1]
        dz = p[:, None, 2] - p[None, :, 2]
        dx -= Lx * np.rint(dx / Lx)
        dy -= Ly * np.rint(dy / Ly)
        r = np.sqrt(dx * dx + dy * dy + dz * dz)[iu]
        cnt += np.histogram(r, bins=edges)[0]
    shell = math.pi * (edges[1:] ** 2 - edges[:-1] ** 2)
    ideal = ns * (N * (N - 1) / 2.0) / (Lx * Ly) * shell
    return cnt / ideal


def one_sphere_height_density(h, a=1.0, weight=1.0, U0=1.0, b=0.1, kT=1.0):
    """Closed form P(h) of one sphere (no pairs), exp(-(weight h + U_wall(h))/kT), normalised by
    quadrature over [-2a, 40 kT/weight + 2a] (the density is negligible outside)."""
    def unnorm(x):
        x = np.asarray(x, dtype=np.float64)
        uw = np.where(x < a, U0 + U0 * (a - x) / b, U0 * np.exp(-(x - a) / b))
        return np.exp(-(weight * x + uw) / kT)
    xs = np.linspace(-2.0 * a, 40.0 * kT / weight + 2.0 * a, 400001)
    Z = np.trapezoid(unnorm(xs), xs)
    return unnorm(h) / Z
