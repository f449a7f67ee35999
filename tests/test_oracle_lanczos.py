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
