"""Equilibrium of an interacting sedimented suspension (Appendix B, Fig. 4, reduced in size): Brownian
dynamics with the Euler-Maruyama and Adams-Bashforth schemes must sample the Gibbs-Boltzmann
distribution that a Metropolis Monte Carlo run samples exactly -- the height density P(h) and the
quasi-two-dimensional pair correlation g(r) of Appendix B.  Only the pair terms (hydrodynamic and
steric) distinguish this from the dilute test: the RFD drift of the pair mobility and the Lanczos
noise of the coupled suspension are checked statistically here.

Set-up (Appendix B's parameters at a quarter of its size): 256 spheres, area fraction 0.25,
pseudo-periodic in x and y (square cell of side sqrt(256 pi / 0.25) a, the unit cell and its eight
neighbours for the hydrodynamics, minimum image for the forces), U0 = 4 kT, b = 0.1a, h_g = 1.58a
(weight kT / 0.58a), no torque, Lanczos tolerance 1e-4, float32 pairs with float64 Lanczos and
delta = 5e-3 a.  Both runs start from the last Monte Carlo configuration (equilibrium), as the
paper's runs start from Monte Carlo samples.  dt = 0.1 (about 0.2 of the steric time tau_U of the
paper's units); 12000 steps per scheme, sampled every 20.

Bounds: the statistical error of each histogram bin is estimated by batch means over 6 blocks of
each run (BD and Monte Carlo), and the comparison allows 4 combined standard errors plus a bias
allowance for the finite dt (1% of the mean height, 5% of the peak of P(h), 0.05 in g), and bounds
the L2 errors of P(h) and g(r) (the paper's measure, Fig. 4 inset) by 0.03 and 0.06.  Measured when
they were set (GB300): EM mean height -0.004 (standard error 0.006) off, L2 errors 0.011 and 0.032;
AB -0.014 (0.008), 0.011 and 0.026.
"""
import math

import numpy as np
import pytest

from oracle import equilibrium as E
from paper_1612_00474_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

N, PHI, U0, B, HG = 256, 0.25, 4.0, 0.1, 1.58
WEIGHT = 1.0 / (HG - 1.0)
L = math.sqrt(N * math.pi / PHI)
H_EDGES = np.linspace(0.8, 4.0, 33)
R_EDGES = np.linspace(1.6, 7.6, 25)
BLOCKS = 6


def _stats(samples):
    """P(h), g(r), mean height and their batch-means standard errors."""
    S = np.asarray(samples)
    blocks = np.array_split(S, BLOCKS)
    P = E.height_histogram(S, H_EDGES)
    g = E.pair_correlation(S, R_EDGES, (L, L))
    Pb = np.array([E.height_histogram(b, H_EDGES) for b in blocks])
    gb = np.array([E.pair_correlation(b, R_EDGES, (L, L)) for b in blocks])
    hb = np.array([b[..., 2].mean() for b in blocks])
    se = lambda x: x.std(axis=0, ddof=1) / math.sqrt(BLOCKS)  # noqa: E731
    return dict(P=P, g=g, h=S[..., 2].mean(), P_se=se(Pb), g_se=se(gb), h_se=float(se(hb)))


@pytest.fixture(scope="module")
def monte_carlo():
    p0 = inputs.monolayer(N, seed=21, phi=PHI)
    S, acc = E.mc_sample(p0, 480, seed=22, thin=8, burn=800, step=0.8, weight=WEIGHT, U0=U0, b=B, periodic=(L, L))
    return S, acc, _stats(S)


def _bd(gpu_lib, start, scheme, dt=0.1, nsteps=12000, every=20, seed=5):
    ctx = gpu_lib.Context(max_N=N, precision="fp32", max_iter=64)
    ctx.set_periodic(L, L)
    q = torch.tensor(inputs.to_soa(start), dtype=torch.float64, device="cuda")
    U = torch.zeros_like(q)
    samples = []
    try:
        for k in range(nsteps // every):
            ctx.run(q, U, k * every, seed, every, scheme=scheme, dt=dt, delta=5e-3, tol=1e-4, weight=WEIGHT, U0=U0,
                    b=B, torque=(0.0, 0.0, 0.0))
            samples.append(inputs.from_soa(q.cpu().numpy(), N))
    finally:
        ctx.close()
    return np.array(samples)


def _compare(bd, mc, label):
    dP = bd["P"] - mc["P"]
    dg = bd["g"] - mc["g"]
    sP = np.sqrt(bd["P_se"] ** 2 + mc["P_se"] ** 2)
    sg = np.sqrt(bd["g_se"] ** 2 + mc["g_se"] ** 2)
    dh = bd["h"] - mc["h"]
    sh = math.hypot(bd["h_se"], mc["h_se"])
    l2P = float(np.sqrt(np.sum(dP ** 2 * np.diff(H_EDGES))))
    l2g = float(np.sqrt(np.sum(dg ** 2 * np.diff(R_EDGES))))
    print(f"\n{label}: mean height {bd['h']:.4f} vs MC {mc['h']:.4f} (diff {dh:+.4f}, se {sh:.4f}); "
          f"P(h) L2 error {l2P:.4f}, max |dP|/se {np.max(np.abs(dP) / sP):.2f}; "
          f"g(r) L2 error {l2g:.4f}, max |dg|/se {np.max(np.abs(dg) / sg):.2f}, max |dg| {np.max(np.abs(dg)):.3f}")
    return dict(dh=dh, sh=sh, dP=dP, sP=sP, dg=dg, sg=sg, l2P=l2P, l2g=l2g)


@pytest.mark.parametrize("scheme", ["EM", "AB"])
def test_interacting_equilibrium(gpu_lib, monte_carlo, scheme):
    S_mc, acc, mc = monte_carlo
    assert 0.3 < acc < 0.7
    bd_samples = _bd(gpu_lib, S_mc[-1], scheme)
    assert np.isfinite(bd_samples).all() and bd_samples[..., 2].min() > 0.5
    r = _compare(_stats(bd_samples), mc, scheme)
    # 4 standard errors plus the finite-dt bias allowance (see the docstring for the measured values)
    assert abs(r["dh"]) <= 4 * r["sh"] + 0.01 * mc["h"]
    assert np.all(np.abs(r["dP"]) <= 4 * r["sP"] + 0.05 * mc["P"].max())
    assert np.all(np.abs(r["dg"]) <= 4 * r["sg"] + 0.05)
    assert r["l2P"] <= 0.03 and r["l2g"] <= 0.06
