"""Pins of the oracle's free-space RPY blocks (tt and tr, both branches).

The integral form of Eq. (mobilityOverlap) is evaluated independently: the flow of a
sphere j loaded by a uniform surface force density (or by the surface density of a
point torque) is the textbook single-sphere Stokes solution -- rigid-body motion
inside the sphere, the Stokes-flow field outside -- and its average over the surface
of sphere i is taken by Gauss quadrature split where the two surfaces intersect.
That average must equal the oracle's block for both r >= 2a and the overlap branch.
"""
import math

import numpy as np
import pytest

import oracle as O

A = 1.0
ETA = 1.0
MU0 = 1.0 / (6 * math.pi * ETA * A)


def _sphere_nodes(r, n_t=64, n_p=64):
    """Quadrature nodes on the unit sphere around target i for a source at distance r along -z.

    cos(theta) of a node measured from +z (target minus source direction).  The surface of i
    enters sphere j where |r e_z + a n| = a, i.e. cos(theta) = -r/(2a); the theta integral is split
    there.  Returns unit normals n (k, 3) and weights summing to 1 (the surface average)."""
    cuts = [-1.0, 1.0]
    c = -r / (2 * A)
    if -1.0 < c < 1.0:
        cuts = [-1.0, c, 1.0]
    xg, wg = np.polynomial.legendre.leggauss(n_t)
    ct, wt = [], []
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        ct.append(0.5 * (hi - lo) * xg + 0.5 * (hi + lo))
        wt.append(0.5 * (hi - lo) * wg)
    ct = np.concatenate(ct)
    wt = np.concatenate(wt)
    ph = 2 * math.pi * np.arange(n_p) / n_p
    st = np.sqrt(1 - ct**2)
    n = np.stack([np.outer(st, np.cos(ph)), np.outer(st, np.sin(ph)), np.outer(ct, np.ones(n_p))], -1).reshape(-1, 3)
    w = np.outer(wt, np.full(n_p, 1.0 / n_p)).ravel() / 2.0
    return n, w


def _avg_translating(r):
    """Surface average over sphere i of the flow of sphere j (force F along each axis) -> 3x3."""
    n, w = _sphere_nodes(r)
    d = np.array([0, 0, r]) + A * n  # x - q_j for x on S_i
    dn = np.linalg.norm(d, axis=1)
    out = np.zeros((3, 3))
    for q in range(3):
        F = np.eye(3)[q]
        inside = dn <= A
        # outside: (1/8 pi eta)[(1/r + a^2/(3 r^3)) F + (1/r^3 - a^2/r^5) (r.F) r]   (Stokes' sphere)
        dF = d @ F
        u_out = (1 / (8 * math.pi * ETA)) * ((1 / dn + A**2 / (3 * dn**3))[:, None] * F
                                             + ((1 / dn**3 - A**2 / dn**5) * dF)[:, None] * d)
        u_in = MU0 * np.tile(F, (len(d), 1))  # rigid translation with U = F/(6 pi eta a)
        u = np.where(inside[:, None], u_in, u_out)
        out[:, q] = w @ u
    return out


def _avg_rotating(r):
    """Surface average over sphere i of the flow of sphere j carrying torque T -> 3x3 (u = M T)."""
    n, w = _sphere_nodes(r)
    d = np.array([0, 0, r]) + A * n
    dn = np.linalg.norm(d, axis=1)
    out = np.zeros((3, 3))
    for q in range(3):
        T = np.eye(3)[q]
        inside = dn <= A
        u_out = np.cross(T, d) / (8 * math.pi * ETA * dn[:, None] ** 3)   # rotlet outside
        u_in = np.cross(T, d) / (8 * math.pi * ETA * A**3)                 # rigid rotation, omega = T/(8 pi eta a^3)
        u = np.where(inside[:, None], u_in, u_out)
        out[:, q] = w @ u
    return out


@pytest.mark.parametrize("r", [0.3, 0.9, 1.5, 1.99, 2.0, 2.4, 3.0, 7.0])
def test_tt_equals_surface_average(r):
    M = O.freespace_tt([0, 0, r], [0, 0, 0], A, ETA)
    ref = _avg_translating(r)
    # quadrature of a piecewise-smooth integrand split at the kink: converges fast
    assert np.max(np.abs(M - ref)) <= 2e-9 * MU0, (M, ref)


@pytest.mark.parametrize("r", [0.3, 0.9, 1.5, 1.99, 2.0, 2.4, 3.0, 7.0])
def test_tr_equals_surface_average(r):
    M = O.freespace_tr([0, 0, r], [0, 0, 0], A, ETA)
    ref = _avg_rotating(r)
    assert np.max(np.abs(M - ref)) <= 2e-9 * MU0, (M, ref)


def test_continuity_at_contact():
    e = np.array([0.36, -0.48, 0.8])
    lo = O.freespace_tt(2 * A * (1 - 1e-13) * e, [0, 0, 0], A, ETA)
    hi = O.freespace_tt(2 * A * e, [0, 0, 0], A, ETA)
    ref = MU0 * (7 / 16 * np.eye(3) + 3 / 16 * np.outer(e, e))
    assert np.allclose(lo, ref, rtol=0, atol=1e-13) and np.allclose(hi, ref, rtol=0, atol=1e-15)
    lo = O.freespace_tr(2 * A * (1 - 1e-13) * e, [0, 0, 0], A, ETA)
    hi = O.freespace_tr(2 * A * e, [0, 0, 0], A, ETA)
    assert np.allclose(lo, hi, rtol=0, atol=1e-13)
    # magnitude 1/(32 pi eta a^2) at contact, direction T x e
    T = np.array([0.0, 1.0, 0.0])
    assert np.allclose(hi @ T, np.cross(T, e) / (32 * math.pi * ETA * A**2), atol=1e-16)


def test_self_and_coincident():
    q = np.array([1.0, 2.0, 3.0])
    assert np.allclose(O.freespace_tt(q, q, A, ETA, same=True), MU0 * np.eye(3), rtol=0, atol=1e-17)
    assert np.allclose(O.freespace_tr(q, q, A, ETA, same=True), 0.0, atol=0)
    # r -> 0 limit of the overlap branch is the self mobility
    M = O.freespace_tt(q + 1e-9, q, A, ETA)
    assert np.allclose(M, MU0 * np.eye(3), rtol=0, atol=1e-9)


def test_rotlet_sign_far():
    # torque +y at the origin, target at +z: T x r = y x z = +x
    M = O.freespace_tr([0, 0, 10.0], [0, 0, 0], A, ETA)
    u = M @ np.array([0, 1.0, 0])
    assert u[0] > 0 and abs(u[1]) < 1e-18 and abs(u[2]) < 1e-18
    assert math.isclose(u[0], 1 / (8 * math.pi * ETA * 100.0), rel_tol=1e-14)
