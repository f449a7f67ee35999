"""Pins of the oracle's pseudo-periodic boundaries (Appendix B): minimum-image forces, hydrodynamics
with the unit cell and its eight neighbour cells."""
import numpy as np
import pytest

import oracle as O
from paper_1612_00474_gb300.inputs import vectors

L = (30.0, 24.0)


def _cluster(N, seed, extent=6.0):
    rng = np.random.default_rng(seed)
    p = np.zeros((N, 3))
    p[:, :2] = rng.uniform(0, extent, (N, 2)) + np.array([10.0, 8.0])
    p[:, 2] = rng.uniform(0.7, 3.0, N)
    return p


def test_equals_explicit_replicas():
    """A compact cluster (all pair offsets below L/2): the periodic product equals the unbounded product
    of the 3 x 3 replicated system evaluated at the central copies."""
    N = 9
    pos = _cluster(N, 1)
    F, T = vectors(N, 2), vectors(N, 3)
    rep = np.concatenate([pos + np.array([nx * L[0], ny * L[1], 0.0]) for nx in (0, -1, 1) for ny in (0, -1, 1)])
    ref = O.mobility_apply(rep, np.tile(F, (9, 1)), np.tile(T, (9, 1)), rows=(0, N))
    got = O.mobility_apply(pos, F, T, periodic=L)
    assert np.allclose(got, ref, rtol=0, atol=1e-14 * np.abs(ref).max())


def test_shift_invariance():
    N = 12
    rng = np.random.default_rng(4)
    pos = np.column_stack([rng.uniform(0, L[0], N), rng.uniform(0, L[1], N), rng.uniform(0.8, 2.5, N)])
    F, T = vectors(N, 5), vectors(N, 6)
    U = O.mobility_apply(pos, F, T, periodic=L)
    moved = pos.copy()
    moved[3, 0] += L[0]
    moved[7, 1] -= 2 * L[1]
    assert np.allclose(O.mobility_apply(moved, F, T, periodic=L), U, rtol=0, atol=1e-13 * np.abs(U).max())
    Fm = O.forces(moved, periodic=L)
    assert np.allclose(Fm, O.forces(pos, periodic=L), rtol=0, atol=1e-12)


def test_symmetric_and_reduces_to_unbounded_for_large_cells():
    N = 6
    pos = _cluster(N, 7)
    cols = [O.mobility_apply(pos, np.eye(3 * N)[k].reshape(N, 3), None, periodic=L).ravel() for k in range(3 * N)]
    M = np.array(cols).T
    assert np.max(np.abs(M - M.T)) < 1e-15 * np.abs(M).max()
    F = vectors(N, 8)
    big = (1e7, 1e7)
    assert np.allclose(O.mobility_apply(pos, F, None, periodic=big), O.mobility_apply(pos, F, None), rtol=0,
                       atol=1e-6 * np.abs(O.mobility_apply(pos, F, None)).max())


def test_minimum_image_forces():
    pos = np.array([[0.3, 5.0, 1.2], [L[0] - 0.6, 5.2, 1.3]])
    F = O.forces(pos, periodic=L)
    ref = O.forces(np.array([[0.3, 5.0, 1.2], [-0.6, 5.2, 1.3]]))
    assert np.allclose(F, ref, rtol=1e-14, atol=1e-14)
    assert F[0, 0] > 0  # pushed away across the boundary
