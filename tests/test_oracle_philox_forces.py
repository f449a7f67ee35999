"""Pins of the oracle's Philox generator and noise, and of its force model (Eq. soft_potential)."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import philox


def test_philox4x64_round_structure_matches_numpy():
    """numpy's Philox bit generator is Philox4x64-10; it advances the counter before each block."""
    for key, ctr in [((0, 0), (0, 0, 0, 0)), ((7, 3), (5, 9, 2, 1)), ((2**64 - 1, 12345), (2**64 - 2, 0, 0, 0))]:
        g = np.random.Philox(counter=np.array(ctr, dtype=np.uint64), key=np.array(key, dtype=np.uint64))
        got = [int(v) for v in g.random_raw(8)]
        c = list(ctr)
        want = []
        for _ in range(2):
            # 256-bit little-endian counter increment
            carry = 1
            for w in range(4):
                s = c[w] + carry
                c[w] = s & (2**64 - 1)
                carry = s >> 64
            want += philox.philox4(c, key, width=64)
        assert got == want


def test_philox4x32_vectorised_equals_scalar():
    rng = np.random.default_rng(0)
    for _ in range(20):
        ctr = [int(v) for v in rng.integers(0, 2**32, 4)]
        key = [int(v) for v in rng.integers(0, 2**32, 2)]
        vec = philox.philox4x32_vec(*[np.array([v], dtype=np.uint64) for v in ctr], key[0], key[1])
        assert [int(v[0]) for v in vec] == philox.philox4(ctr, key, width=32)


def test_normals_statistics():
    from scipy import stats

    z = philox.normals(400_001, seed=123, step=7, stream=0)
    assert abs(z.mean()) < 5 / math.sqrt(z.size)
    assert abs(z.var() - 1) < 5 * math.sqrt(2 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    assert abs(np.corrcoef(z[:-1], z[1:])[0, 1]) < 5 / math.sqrt(z.size)
    w = philox.normals(400_001, seed=123, step=7, stream=1)
    assert abs(np.corrcoef(z, w)[0, 1]) < 5 / math.sqrt(z.size)
    v = philox.normals(400_001, seed=123, step=8, stream=0)
    assert abs(np.corrcoef(z, v)[0, 1]) < 5 / math.sqrt(z.size)


def test_noise_layout_and_prefix():
    a = O.noise(10, seed=5, step=2, stream=0)
    b = O.noise(11, seed=5, step=2, stream=0)
    assert a.shape == (10, 3) and np.array_equal(a, b[:10])   # index k = 3 i + c is canonical


def _energy(pos, U0=1.0, b=0.1, a=1.0, weight=1.0):
    """Total potential energy: Eq. (soft_potential) pairwise (d = 2a) and with the wall (d = a),
    plus gravity weight * z."""
    def U(r, d):
        return np.where(r < d, U0 + U0 * (d - r) / b, U0 * np.exp(-(r - d) / b))
    E = weight * pos[:, 2].sum() + U(pos[:, 2], a).sum()
    N = len(pos)
    for i in range(N):
        for j in range(i + 1, N):
            E += U(np.linalg.norm(pos[i] - pos[j]), 2 * a)
    return float(E)


@pytest.mark.parametrize("seed", range(3))
def test_forces_are_minus_energy_gradient(seed):
    rng = np.random.default_rng(seed)
    pos = np.zeros((6, 3))
    pos[:, :2] = rng.uniform(0, 4.0, (6, 2))
    pos[:, 2] = rng.uniform(0.7, 1.8, 6)
    F = O.forces(pos)
    h = 1e-6
    for i in range(6):
        for c in range(3):
            p1, p2 = pos.copy(), pos.copy()
            p1[i, c] += h
            p2[i, c] -= h
            fd = -(_energy(p1) - _energy(p2)) / (2 * h)
            assert abs(F[i, c] - fd) < 1e-6 * max(1.0, abs(fd)), (i, c, F[i, c], fd)


def test_force_details():
    # wall force continuous at z = a and equal to U0/b there; the paper's 44 kT barrier at U0=4, b=0.1a
    f_hi = O.forces(np.array([[0.0, 0.0, 1.0]]), U0=4.0, b=0.1)[0, 2]
    f_lo = O.forces(np.array([[0.0, 0.0, 1.0 - 1e-12]]), U0=4.0, b=0.1)[0, 2]
    assert math.isclose(f_hi, 40.0 - 1.0) and math.isclose(f_lo, 40.0 - 1.0)
    assert math.isclose(_energy(np.array([[0.0, 0.0, 0.0]]), U0=4.0, b=0.1, weight=0.0), 44.0)
    # coincident pair: no direction, no force between them
    F = O.forces(np.array([[1.0, 1.0, 5.0], [1.0, 1.0, 5.0]]), weight=0.0)
    assert np.allclose(F[:, :2], 0) and np.allclose(F[0], F[1])
