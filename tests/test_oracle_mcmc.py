"""Pins of the Metropolis sampler and the equilibrium statistics of Appendix B (oracle/equilibrium.py).

  - One sphere: the sampled heights follow the closed-form Gibbs-Boltzmann density
    exp(-(m g h + U_wall(h))/kT) (Kolmogorov distance to its CDF).
  - The sampled energy is the one the forces come from: -grad U by central differences equals the
    oracle's forces (gravity, wall and pair steric terms, minimum image) on a configuration with
    overlaps, periodic and not.
  - g(r): uniform configurations of equal heights give g = 1 within the sampling noise (the
    two-dimensional normalisation of Appendix B), and no pair is counted below the smallest distance.
  - P(h) integrates to one over the bins that cover the sample.
"""
import math

import numpy as np

import oracle as O
from oracle import equilibrium as E


def test_one_sphere_heights_follow_closed_form():
    w, U0, b = 1.0 / 0.58, 4.0, 0.1
    S, acc = E.mc_sample(np.array([[0.0, 0.0, 1.5]]), 40000, seed=1, thin=25, burn=100, step=0.8, weight=w, U0=U0,
                         b=b)
    assert 0.2 < acc < 0.8
    h = np.sort(S[:, 0, 2])
    xs = np.linspace(0.5, 12.0, 200001)
    pdf = E.one_sphere_height_density(xs, weight=w, U0=U0, b=b)
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (pdf[1:] + pdf[:-1]) * np.diff(xs))])
    F = np.interp(h, xs, cdf)
    n = h.size
    ks = max(np.max(np.arange(1, n + 1) / n - F), np.max(F - np.arange(n) / n))
    assert ks <= 0.015, ks  # 40000 samples 25 single-sphere moves apart


def _grad_energy(pos, periodic, **kw):
    g = np.zeros_like(pos)
    eps = 1e-6
    for i in range(pos.shape[0]):
        for c in range(3):
            p1, p2 = pos.copy(), pos.copy()
            p1[i, c] += eps
            p2[i, c] -= eps
            g[i, c] = (E.mc_energy(p1, periodic=periodic, **kw) - E.mc_energy(p2, periodic=periodic, **kw)) / (2 * eps)
    return g


def test_energy_gradient_is_minus_the_oracle_forces():
    rng = np.random.default_rng(3)
    N = 12
    pos = np.zeros((N, 3))
    pos[:, :2] = rng.uniform(0, 6.0, (N, 2))
    pos[:, 2] = rng.uniform(0.8, 2.5, N)  # some spheres overlap the wall and each other
    kw = dict(a=1.0, weight=1.7, U0=4.0, b=0.1)
    for periodic in (None, (6.5, 7.0)):
        F = O.forces(pos, periodic=periodic, **kw)
        G = _grad_energy(pos, periodic, **kw)
        assert np.max(np.abs(-G - F)) <= 1e-6 * np.max(np.abs(F))


def test_pair_correlation_normalisation():
    rng = np.random.default_rng(5)
    L, N, ns = 40.0, 200, 40
    S = np.zeros((ns, N, 3))
    S[:, :, :2] = rng.uniform(0, L, (ns, N, 2))
    S[:, :, 2] = 1.5
    edges = np.linspace(0.5, 15.0, 30)
    g = E.pair_correlation(S, edges, (L, L))
    assert np.all(np.abs(g - 1.0) <= 0.1), g
    assert abs(float(np.mean(g)) - 1.0) <= 0.02
    S2 = S.copy()
    S2[:, :, 2] = 1.5
    g2 = E.pair_correlation(S2, np.array([0.0, 1e-9]), (L, L))
    assert g2[0] == 0.0


def test_height_histogram_is_a_density():
    rng = np.random.default_rng(7)
    S = rng.uniform(1.0, 3.0, (5, 100, 3))
    edges = np.linspace(0.9, 3.1, 23)
    P = E.height_histogram(S, edges)
    assert math.isclose(float(np.sum(P * np.diff(edges))), 1.0, rel_tol=1e-12)
