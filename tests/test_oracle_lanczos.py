"""Pins of the oracle's Lanczos M^{1/2} W (Sec. II.C) against a dense eigendecomposition
(LAPACK through numpy) and its stated stopping rule."""
import numpy as np
import pytest

import oracle as O
from paper_1612_00474_gb300.inputs import monolayer, vectors


def _dense_sqrt_apply(M, w):
    lam, Q = np.linalg.eigh(M)
    return Q @ (np.sqrt(np.clip(lam, 0, None)) * (Q.T @ w))


@pytest.mark.parametrize("N", [1, 3, 16, 64])
def test_matches_dense_sqrt_tight(N):
    pos = monolayer(N, seed=N)
    W = vectors(N, 11 + N)
    tt, _ = O.dense(pos)
    ref = _dense_sqrt_apply(tt, W.ravel())
    g, m, eps, conv = O.lanczos_sqrt(pos, W, tol=1e-14, max_iter=3 * N + 5)
    assert conv
    assert O.rel_err(g, ref) <= 1e-12, (m, eps)


def test_matches_dense_sqrt_loose_tol():
    pos = monolayer(64, seed=9)
    W = vectors(64, 12)
    tt, _ = O.dense(pos)
    ref = _dense_sqrt_apply(tt, W.ravel())
    g, m, eps, conv = O.lanczos_sqrt(pos, W, tol=1e-3, max_iter=100)
    assert conv and eps <= 1e-3 and 2 <= m < 20
    assert O.rel_err(g, ref) <= 1e-2
    # the previous iterate did not meet the tolerance (stopping rule is "first k with eps_k <= tol")
    g2, m2, eps2, _ = O.lanczos_sqrt(pos, W, tol=1e-3, exact_iters=m - 1)
    assert m2 == m - 1 and (m - 1 < 2 or eps2 > 1e-3)


def test_single_iteration_and_exact_iters():
    pos = monolayer(8, seed=2)
    W = vectors(8, 3)
    g1, m1, eps1, _ = O.lanczos_sqrt(pos, W, exact_iters=1)
    tt, _ = O.dense(pos)
    w = W.ravel()
    v = w / np.linalg.norm(w)
    alpha = v @ tt @ v
    assert m1 == 1 and np.isnan(eps1)
    assert np.allclose(g1.ravel(), np.linalg.norm(w) * np.sqrt(alpha) * v, rtol=1e-14, atol=0)
    g5, m5, _, _ = O.lanczos_sqrt(pos, W, exact_iters=5)
    assert m5 == 5


def test_zero_and_invariant_subspace():
    pos = monolayer(4, seed=1)
    g, m, eps, conv = O.lanczos_sqrt(pos, np.zeros((4, 3)))
    assert m == 0 and conv and np.all(g == 0)
    # one isolated sphere: M is diagonal with two distinct values, so the Krylov space of a
    # generic W has dimension 2 and Lanczos breaks down (exactly) at k = 2
    pos1 = np.array([[0.0, 0.0, 1.3]])
    W = np.array([[0.3, -1.1, 0.7]])
    g, m, eps, conv = O.lanczos_sqrt(pos1, W, tol=1e-16, max_iter=10)
    tt, _ = O.dense(pos1)
    assert conv and m == 2
    assert O.rel_err(g, np.sqrt(np.diag(tt)) * W.ravel()) < 1e-13


def test_fluctuation_dissipation_statistics():
    """Sample covariance of g = M^{1/2} W over many W approaches M (N = 2)."""
    pos = np.array([[0.0, 0.0, 1.4], [2.3, 0.4, 1.8]])
    tt, _ = O.dense(pos)
    rng = np.random.default_rng(5)
    n = 4000
    G = np.array([O.lanczos_sqrt(pos, rng.standard_normal((2, 3)), tol=1e-12, max_iter=12)[0].ravel()
                  for _ in range(n)])
    C = G.T @ G / n
    # each entry's standard error is about sqrt((M_ii M_jj + M_ij^2)/n)
    se = np.sqrt((np.outer(np.diag(tt), np.diag(tt)) + tt**2) / n)
    assert np.all(np.abs(C - tt) < 5 * se)


# ---------------------------------------------------------------- block-diagonal preconditioner
def _published_self(z, a=1.0, eta=1.0):
    """Regularised diagonal of the translation self block from the published near-wall self
    mobilities mu0 (1 - 9x/16 + x^3/8 - x^5/16) parallel and mu0 (1 - 9x/8 + x^3/2 - x^5/8) normal,
    x = a / max(z, a), times s^2 with s = H0(z / a) (Appendix A regularisation)."""
    mu0 = 1.0 / (6.0 * np.pi * eta * a)
    s = np.clip(z / a, 0.0, 1.0)
    x = a / np.maximum(z, a)
    par = mu0 * (1 - 9 * x / 16 + x ** 3 / 8 - x ** 5 / 16)
    perp = mu0 * (1 - 9 * x / 8 + x ** 3 / 2 - x ** 5 / 8)
    return s[:, None] ** 2 * np.stack([par, par, perp], axis=1)


def test_self_diagonal_is_published_self_mobility():
    pos = monolayer(40, seed=5)
    pos[:5, 2] = [-0.2, 0.0, 0.4, 1.0, 7.5]  # below, on and near the wall, and far above it
    D = O.self_diagonal(pos)
    assert np.allclose(D, _published_self(pos[:, 2]), rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("N", [2, 7, 24])
def test_preconditioned_sqrt_covariance(N):
    """Full Krylov space: g = D^{1/2} (P M P)^{1/2} W with P = D^{-1/2}, and that map L has
    L L^T = M (the noise covariance), computed densely with LAPACK."""
    pos = monolayer(N, seed=30 + N)
    pos[0, 2] = 0.6  # one overlapping the wall
    W = vectors(N, 40 + N)
    tt, _ = O.dense(pos)
    D = O.self_diagonal(pos).ravel()
    P = 1.0 / np.sqrt(D)
    lam, Q = np.linalg.eigh(P[:, None] * tt * P[None, :])
    L = np.sqrt(D)[:, None] * (Q @ np.diag(np.sqrt(np.clip(lam, 0, None))) @ Q.T)
    assert np.allclose(L @ L.T, tt, rtol=0, atol=1e-12 * np.abs(tt).max())
    g, m, eps, conv = O.lanczos_sqrt(pos, W, tol=1e-14, max_iter=3 * N + 5, precondition=True)
    assert conv
    assert O.rel_err(g, L @ W.ravel()) <= 1e-11, (m, eps)


def test_preconditioned_sqrt_zero_mobility_rows():
    """Spheres on or below the wall have zero mobility rows: D = 0 there, and their noise is 0."""
    pos = monolayer(12, seed=3)
    pos[2, 2] = -0.5
    pos[5, 2] = 0.0
    W = vectors(12, 9)
    g, m, eps, conv = O.lanczos_sqrt(pos, W, tol=1e-12, max_iter=60, precondition=True)
    assert conv and np.all(g[2] == 0.0) and np.all(g[5] == 0.0)
    tt, _ = O.dense(pos)
    keep = np.ones(36, bool)
    keep[6:9] = keep[15:18] = False
    sub = tt[np.ix_(keep, keep)]
    D = O.self_diagonal(pos).ravel()[keep]
    P = 1.0 / np.sqrt(D)
    lam, Q = np.linalg.eigh(P[:, None] * sub * P[None, :])
    ref = np.sqrt(D) * (Q @ (np.sqrt(np.clip(lam, 0, None)) * (Q.T @ W.ravel()[keep])))
    assert O.rel_err(g.ravel()[keep], ref) <= 1e-9
