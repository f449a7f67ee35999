"""Statistical check of the whole stochastic step (Appendix B): dilute spheres sedimented above the
wall, with gravity and the soft wall potential of Eq. (soft_potential) and no driving torque, must
sample the Gibbs-Boltzmann height distribution p(h) ~ exp(-(m g h + U_wall(h))/kT) under both
Euler-Maruyama and Adams-Bashforth.  The near-wall mobility drops to mu0/4 at contact, so without the
RFD drift kT d(mu_zz)/dz the distribution would be visibly wrong near the wall; the check compares
the mean height, the fraction of spheres below 1.3a and the whole CDF with the closed form.

Set-up: spheres on a square grid with spacing 60a (hydrodynamic coupling ~ (1/60)^3, so the spheres
are independent), heights drawn from p(h) itself, U0 = 4 kT, b = 0.1a, weight m g = 1 kT/a, steps
replayed from a CUDA graph.  FP64: 1024 spheres, delta = 1e-6 a, dt = 0.05, 200 time units.  FP32
pairs (delta = 5e-3 a): 4096 spheres, 300 time units, dt = 0.1 and its half 0.05 (AB) and 0.05 (EM).

Bounds: each sphere's time average is one independent sample of the mean, so the standard error is
the spread of the per-sphere averages over sqrt(spheres); the mean height and P(h < 1.3a) must lie
within 4 standard errors of the closed form, and the pooled heights within Kolmogorov distance 0.03.
Measured when set (GB300): FP32 AB mean-height error -0.014 (standard error 0.008) at dt = 0.1 and
-0.016 (0.009) at dt = 0.05, EM -0.015 (0.009); FP64 +0.004 (0.014) with 60 time units.  Halving dt
does not shrink the error: what deficit there is is sampling noise (under 2 standard errors), not a
bias of the step size.
"""
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
    h = np.linspace(0.0, 20.0, 400001)
    p = np.exp(-(potential(h) - potential(h).min()))
    cdf = np.cumsum(p)
    cdf /= cdf[-1]
    return h, p / np.trapezoid(p, h), cdf


def _run(gpu_lib, side, precision, scheme, dt, T, delta, seed=77):
    h, p, cdf = gb_grid()
    N = side * side
    rng = np.random.default_rng(11)
    xy = 60.0 * np.stack(np.meshgrid(np.arange(side), np.arange(side)), -1).reshape(-1, 2)
    pos = np.column_stack([xy, np.interp(rng.random(N), cdf, h)])
    ctx = gpu_lib.Context(max_N=N, precision=precision, max_iter=32)
    q = torch.tensor(inputs.to_soa(pos), dtype=torch.float64, device="cuda")
    U = torch.zeros_like(q)
    every = max(1, int(round(0.5 / dt)))
    nsteps, burn = int(round(T / dt)), int(round(10.0 / dt))
    acc, below, pooled = np.zeros(N), np.zeros(N), []
    n = 0
    try:
        step = 0
        while step < nsteps:
            ctx.run(q, U, step, seed, every, scheme=scheme, dt=dt, delta=delta, tol=1e-3, weight=WEIGHT, U0=U0, b=B,
                    torque=(0.0, 0.0, 0.0))
            step += every
            if step >= burn:
                z = q[2 * N:].cpu().numpy()
                acc += z
                below += z < 1.3
                pooled.append(z)
                n += 1
    finally:
        ctx.close()
    zs = np.concatenate(pooled)
    assert np.isfinite(zs).all() and zs.min() > 0.0
    mean_th = np.trapezoid(h * p, h)
    below_th = np.trapezoid(np.where(h < 1.3, p, 0.0), h)
    pm, pb = acc / n, below / n
    r = dict(err=pm.mean() - mean_th, se=pm.std(ddof=1) / np.sqrt(N), berr=pb.mean() - below_th,
             bse=pb.std(ddof=1) / np.sqrt(N), ks=np.max(np.abs(np.searchsorted(np.sort(zs), h) / zs.size - cdf)))
    print(f"\n{precision} {scheme} dt={dt}: mean height error {r['err']:+.4f} (se {r['se']:.4f}), P(h < 1.3a) error "
          f"{r['berr']:+.4f} (se {r['bse']:.4f}), KS {r['ks']:.4f}, {N} spheres x {n} samples")
    assert abs(r["err"]) <= 4 * r["se"]
    assert abs(r["berr"]) <= 4 * r["bse"]
    assert r["ks"] < 0.03
    return r


@pytest.mark.parametrize("scheme", ["EM", "AB"])
def test_gibbs_boltzmann_heights_fp64(gpu_lib, scheme):
    _run(gpu_lib, 32, "fp64", scheme, 0.05, 200.0, 1e-6)


@pytest.mark.parametrize("scheme,dt", [("AB", 0.1), ("AB", 0.05), ("EM", 0.05)])
def test_gibbs_boltzmann_heights_fp32_dt(gpu_lib, scheme, dt):
    _run(gpu_lib, 64, "fp32", scheme, dt, 300.0, 5e-3)
