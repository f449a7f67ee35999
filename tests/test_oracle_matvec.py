"""Pins of the oracle's assembled mobility: matvec = dense product, symmetry, SPD with overlaps
(Appendix A), the regularisation limits, and the direct sum's structure."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1612_00474_gb300.inputs import monolayer, vectors

A = 1.0
MU0 = 1 / (6 * math.pi * A)


def _overlapping(N, seed):
    """Clusters with particle-particle overlaps and particles partly below or at the wall."""
    rng = np.random.default_rng(seed)
    p = np.zeros((N, 3))
    p[:, :2] = rng.uniform(0, 2.5 * math.sqrt(N), (N, 2))
    p[:, 2] = rng.uniform(-0.3, 3.0, N)
    p[: N // 4, :2] = p[0, :2] + rng.normal(0, 0.5, (N // 4, 2))  # a dense overlapping clump
    return p


@pytest.mark.parametrize("N", [1, 2, 7, 33])
def test_matvec_equals_dense(N):
    pos = _overlapping(N, N)
    F = vectors(N, 1)
    T = vectors(N, 2)
    tt, tr = O.dense(pos)
    U = O.mobility_apply(pos, F, T)
    ref = tt @ F.ravel() + tr @ T.ravel()
    assert np.allclose(U.ravel(), ref, rtol=0, atol=1e-14 * np.max(np.abs(ref)))


@pytest.mark.parametrize("seed", range(4))
def test_symmetric_positive_definite_with_overlaps(seed):
    pos = _overlapping(40, 10 + seed)
    tt, _ = O.dense(pos)
    assert np.max(np.abs(tt - tt.T)) <= 1e-15 * np.max(np.abs(tt))
    lam = np.linalg.eigvalsh(tt)
    assert lam.min() >= -1e-12 * lam.max(), lam[:5]


def test_monolayer_spd_and_pair_reciprocity():
    pos = monolayer(64, seed=3)
    tt, tr = O.dense(pos)
    assert np.linalg.eigvalsh(tt).min() > 0
    # pair block reciprocity M_ij = M_ji^T
    i, j = 5, 17
    assert np.allclose(tt[3 * i:3 * i + 3, 3 * j:3 * j + 3], tt[3 * j:3 * j + 3, 3 * i:3 * i + 3].T, rtol=0, atol=1e-17)


def test_regularisation_limits():
    """Blocks vanish smoothly (linearly) as a particle's centre reaches the wall; a particle
    below the wall does not move whatever the load (Appendix A)."""
    other = np.array([3.0, 0.5, 1.7])
    vals = []
    for z in (1.0, 0.5, 0.25, 1e-8, 0.0, -0.5):
        q = np.array([0.0, 0.0, z])
        tt_s, tr_s = O.pair_blocks(q, q, same=True)
        tt_p, tr_p = O.pair_blocks(q, other)
        vals.append((z, np.abs(tt_s).max(), np.abs(tt_p).max(), np.abs(tr_s).max(), np.abs(tr_p).max()))
    v = np.array(vals)
    # z <= a: blocks are the z=a blocks times H0(z)^2 (self) and H0(z) (pair)
    assert np.allclose(v[1, 1], 0.25 * v[0, 1]) and np.allclose(v[2, 1], 0.0625 * v[0, 1])
    assert np.allclose(v[1, 2], 0.5 * v[0, 2]) and np.allclose(v[1, 4], 0.5 * v[0, 4])
    assert np.all(v[4:, 1:] == 0.0)
    pos = np.array([[0.0, 0.0, -0.2], [2.5, 0.0, 1.5], [0.5, 2.2, 1.1]])
    U = O.mobility_apply(pos, vectors(3, 5), vectors(3, 6))
    assert np.all(U[0] == 0.0) and np.any(U[1] != 0.0)


def test_clamp_equivalence():
    """Mtilde uses z <- max(z, a): a particle at z in (0, a) sees the z=a geometry scaled by H0."""
    q = np.array([0.2, 0.1, 0.6])
    qa = np.array([0.2, 0.1, 1.0])
    other = np.array([2.6, -0.4, 1.3])
    tt, tr = O.pair_blocks(q, other)
    tta, tra = O.pair_blocks(qa, other)
    assert np.allclose(tt, 0.6 * tta, rtol=1e-15, atol=0) and np.allclose(tr, 0.6 * tra, rtol=1e-15, atol=0)


def test_rows_subset_and_linearity():
    pos = monolayer(50, seed=4)
    F, T = vectors(50, 7), vectors(50, 8)
    U = O.mobility_apply(pos, F, T)
    assert np.allclose(O.mobility_apply(pos, F, T, rows=(10, 20)), U[10:20], rtol=0, atol=0)
    tol = 1e-14 * np.max(np.abs(U))
    assert np.allclose(O.mobility_apply(pos, F, None) + O.mobility_apply(pos, None, T), U, rtol=0, atol=tol)
    assert np.allclose(O.mobility_apply(pos, 2.5 * F, None), 2.5 * O.mobility_apply(pos, F, None), rtol=0,
                       atol=2.5 * tol)


def test_single_roller_rolls():
    """One sphere near the wall under a +y torque and no force moves along +x only (Sec. III)."""
    U = O.mobility_apply(np.array([[0.0, 0.0, 1.5]]), None, np.array([[0.0, 1.0, 0.0]]))
    assert U[0, 0] > 0 and U[0, 1] == 0 and U[0, 2] == 0
    assert math.isclose(U[0, 0], MU0 * 3 / (32 * 1.5**4), rel_tol=1e-14)


def test_unbounded_mode():
    """wall=False is the free-space RPY mobility (Sec. II.C compares Lanczos with and without the
    wall): blocks equal the free-space ones, no clamp or H0, SPD."""
    pos = _overlapping(20, 77)
    tt, tr = O.dense(pos, wall=False)
    for i, j in [(0, 1), (3, 3), (5, 12)]:
        ref = O.freespace_tt(pos[i], pos[j], 1.0, 1.0, same=(i == j))
        assert np.allclose(tt[3 * i:3 * i + 3, 3 * j:3 * j + 3], ref, rtol=0, atol=1e-17)
        reft = O.freespace_tr(pos[i], pos[j], 1.0, 1.0, same=(i == j))
        assert np.allclose(tr[3 * i:3 * i + 3, 3 * j:3 * j + 3], reft, rtol=0, atol=1e-17)
    assert np.linalg.eigvalsh(tt).min() > 0
    F = vectors(20, 3)
    assert np.allclose(O.mobility_apply(pos, F, None, wall=False).ravel(), tt @ F.ravel(), rtol=0,
                       atol=1e-14 * np.abs(tt @ F.ravel()).max())
