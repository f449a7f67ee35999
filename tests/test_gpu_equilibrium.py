"""Statistical check of the whole stochastic step (Appendix B): dilute spheres sedimented above the
wall, with gravity and the soft wall potential of Eq. (soft_potential) and no driving torque, must
sample the Gibbs-Boltzmann height distribution p(h) ~ exp(-(m g h + U_wall(h))/kT) under both
Euler-Maruyama and Adams-Bashforth.  The near-wall mobility drops to mu0/4 at contact, so without the
RFD drift kT d(mu_zz)/dz the distribution would be visibly wrong near the wall; the check compares
the mean height, the fraction of time below 1.3a and the whole CDF with the closed form.

Set-up: 1024 spheres on a square grid with spacing 60a (hydrodynamic coupling ~ (1/60)^3), heights
drawn from p(h) itself, U0 = 4 kT, b = 0.1a, weight m g = 1 kT/a, dt = 0.05 (about tau_U/10),
4000 steps, FP64 pairs with delta = 1e-6 a.
"""
import math

import numpy as np
import pytest

from paper_1612_00474_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

U0, B, WEIGHT, A = 4.0, 0.1, 1.0, 1.0


def potential(h):
    wall = np.where(h < A, U0 + U0 * (A - h) / B, U0 * np.exp(-(h - A) / B))
    return WEIGHT * h + wall


def gb_grid():
    h = np.linspace(0.0, 14.0, 280001)
    p = np.exp(-(potential(h) - potential(h).min()))
    cdf = np.cumsum(p)
    cdf /= cdf[-1]
    return h, p / np.trapezoid(p, h), cdf


@pytest.mark.parametrize("scheme", ["EM", "AB"])
def test_gibbs_boltzmann_heights(gpu_lib, scheme):
    h, p, cdf = gb_grid()
    mean_th = np.trapezoid(h * p, h)
    below_th = np.trapezoid(np.where(h < 1.3, p, 0.0), h)
    rng = np.random.default_rng(11)
    side = 32
    N = side * side
    xy = 60.0 * np.stack(np.meshgrid(np.arange(side), np.arange(side)), -1).reshape(-1, 2)
    z0 = np.interp(rng.random(N), cdf, h)
    pos = np.column_stack([xy, z0])
    ctx = gpu_lib.Context(max_N=N, precision="fp64", max_iter=32)
    q = torch.tensor(inputs.to_soa(pos), dtype=torch.float64, device="cuda")
    U = torch.zeros_like(q)
    samples = []
    try:
        for n in range(4000):
            ctx.step(q, U, n, 77, scheme=scheme, dt=0.05, delta=1e-6, tol=1e-3, weight=WEIGHT, U0=U0, b=B,
                     torque=(0.0, 0.0, 0.0))
            if n >= 200 and n % 5 == 0:
                samples.append(q[2 * N:].clone())
    finally:
        ctx.close()
    zs = torch.cat(samples).cpu().numpy()
    assert np.isfinite(zs).all() and zs.min() > 0.0
    mean = zs.mean()
    below = (zs < 1.3).mean()
    ks = np.max(np.abs(np.searchsorted(np.sort(zs), h) / zs.size - cdf))
    print(f"\n{scheme}: mean height {mean:.4f} (Gibbs-Boltzmann {mean_th:.4f}), P(h < 1.3a) {below:.4f} "
          f"({below_th:.4f}), KS distance {ks:.4f}, {zs.size} samples")
    assert abs(mean - mean_th) < 0.03 * mean_th, (mean, mean_th)
    assert abs(below - below_th) < 0.15 * below_th, (below, below_th)
    assert ks < 0.03, ks
