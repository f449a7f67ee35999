"""Pins of the oracle's wall (image) part of the Rotne-Prager-Blake tensors.

  1. Blake's image system: Oseen + G_img vanishes on the wall (no slip) and is divergence
     free in x (finite differences), and G_img -> 0 as the source recedes.
  2. Faxen step: for separated spheres the Faxen-operated image blocks equal the double
     surface average of Eq. (mobilityOverlap) (translation) and the surface average of the
     point-couple density (rotation), evaluated by Gauss quadrature on both spheres.
  3. Self mobility: mu_par/mu0 = 1 - 9/(16h) + 1/(8h^3) - 1/(16h^5) and
     mu_perp/mu0 = 1 - 9/(8h) + 1/(2h^3) - 1/(8h^5) (the published wall-corrected RPY
     self terms; their 1/h terms are the classical Faxen and Lorentz corrections); a +y torque
     rolls a sphere along +x (Sec. III) with coupling 3/(32 h^4) mu0/a.
  4. Screening: the in-plane pair mobility decays like r^-3 for r >> h (Sec. II.C); far from
     the wall the free-space RPY tensor is recovered.
"""
import math

import numpy as np
import pytest

import oracle as O

A = 1.0
ETA = 1.0
MU0 = 1.0 / (6 * math.pi * ETA * A)


def oseen8(r):
    rn = np.linalg.norm(r)
    return np.eye(3) / rn + np.outer(r, r) / rn**3


@pytest.mark.parametrize("seed", range(5))
def test_blake_no_slip(seed):
    rng = np.random.default_rng(seed)
    y = np.array([*rng.uniform(-3, 3, 2), rng.uniform(0.2, 4)])
    x = np.array([*rng.uniform(-3, 3, 2), 0.0])
    G = oseen8(x - y) + O.blake_image_raw(x, y)
    assert np.max(np.abs(G)) < 1e-14 * np.max(np.abs(oseen8(x - y)))


@pytest.mark.parametrize("seed", range(5))
def test_blake_divergence_free(seed):
    rng = np.random.default_rng(100 + seed)
    y = np.array([*rng.uniform(-2, 2, 2), rng.uniform(0.5, 3)])
    x = np.array([*rng.uniform(-2, 2, 2), rng.uniform(0.5, 3)])
    h = 1e-4
    div = np.zeros(3)
    for i in range(3):
        e = np.eye(3)[i] * h
        div += (O.blake_image_raw(x + e, y)[i] - O.blake_image_raw(x - e, y)[i]) / (2 * h)
    scale = np.max(np.abs(O.blake_image_raw(x, y))) / np.linalg.norm(x - np.array([y[0], y[1], -y[2]]))
    assert np.max(np.abs(div)) < 1e-7 * scale


def test_blake_vanishes_far_from_wall():
    x = np.array([0.3, -0.2, 1e6 + 1.0])
    y = np.array([0.0, 0.0, 1e6])
    assert np.max(np.abs(O.blake_image_raw(x, y))) < 2e-6


def _sphere(n_t, n_p):
    xg, wg = np.polynomial.legendre.leggauss(n_t)
    ph = 2 * math.pi * np.arange(n_p) / n_p
    st = np.sqrt(1 - xg**2)
    n = np.stack([np.outer(st, np.cos(ph)), np.outer(st, np.sin(ph)), np.outer(xg, np.ones(n_p))], -1).reshape(-1, 3)
    w = np.outer(wg / 2, np.full(n_p, 1.0 / n_p)).ravel()
    return n, w


CONFIGS = [
    ((0.0, 0.0, 1.5), (0.0, 0.0, 1.5)),      # self block at h = 1.5a
    ((0.0, 0.0, 2.7), (0.0, 0.0, 2.7)),      # self block at h = 2.7a
    ((3.1, 0.4, 1.6), (0.0, 0.0, 2.2)),      # separated pair
    ((-1.0, 2.5, 3.0), (0.5, -0.3, 1.4)),
]


@pytest.mark.parametrize("xi,xj", CONFIGS)
def test_faxen_tt_equals_surface_average(xi, xj):
    xi, xj = np.array(xi), np.array(xj)
    n, w = _sphere(20, 40)
    X = xi + A * n
    Y = xj + A * n
    ix, iy = np.meshgrid(np.arange(len(n)), np.arange(len(n)), indexing="ij")
    G = O.blake_image_raw_batch(X[ix, 0] - Y[iy, 0], X[ix, 1] - Y[iy, 1], X[ix, 2], Y[iy, 2])
    ww = (w[:, None] * w[None, :]).ravel()
    avg = np.einsum("k,kij->ij", ww, G)
    M = O.wall_image_tt(xi, xj, A)
    assert np.max(np.abs(avg - M)) < 1e-10 * np.max(np.abs(M)), (avg, M)


@pytest.mark.parametrize("xi,xj", CONFIGS)
def test_faxen_tr_equals_surface_average(xi, xj):
    """Torque T on sphere j as the surface force density f = 3/(8 pi a^3) T x n."""
    xi, xj = np.array(xi), np.array(xj)
    n, w = _sphere(20, 40)
    X = xi + A * n
    Y = xj + A * n
    ix, iy = np.meshgrid(np.arange(len(n)), np.arange(len(n)), indexing="ij")
    G = O.blake_image_raw_batch(X[ix, 0] - Y[iy, 0], X[ix, 1] - Y[iy, 1], X[ix, 2], Y[iy, 2])
    G = G.reshape(len(n), len(n), 3, 3)
    area = 4 * math.pi * A**2
    out = np.zeros((3, 3))
    for q in range(3):
        T = np.eye(3)[q]
        f = 3.0 / (8 * math.pi * A**3) * np.cross(T, n)      # (len(n), 3) density on S_j
        # u(x) = sum over S_j of G f dS ; then average over S_i
        u = np.einsum("abij,bj,b->ai", G, f, w * area)
        out[:, q] = w @ u
    M = O.wall_image_tr(xi, xj, A)
    assert np.max(np.abs(out - M)) < 1e-10 * np.max(np.abs(M)), (out, M)


@pytest.mark.parametrize("h", [1.0, 1.2, 1.5, 2.0, 3.0, 10.0])
def test_self_mobility_closed_form(h):
    q = np.array([0.4, -1.0, h])
    tt, tr = O.pair_blocks(q, q, same=True, a=A, eta=ETA)
    par = 1 - 9 / (16 * h) + 1 / (8 * h**3) - 1 / (16 * h**5)
    perp = 1 - 9 / (8 * h) + 1 / (2 * h**3) - 1 / (8 * h**5)
    ref = MU0 * np.diag([par, par, perp])
    assert np.allclose(tt, ref, rtol=0, atol=1e-15)
    c = MU0 / A * 3 / (32 * h**4)
    assert np.allclose(tr, np.array([[0, c, 0], [-c, 0, 0], [0, 0, 0]]), rtol=0, atol=1e-16)
    # +y torque rolls along +x
    assert (tr @ np.array([0, 1.0, 0]))[0] > 0


def test_pair_screening_r3():
    z = 1.3
    vals = []
    for r in (50.0, 100.0, 200.0, 400.0):
        tt, _ = O.pair_blocks(np.array([r, 0, z]), np.array([0, 0, z]), a=A, eta=ETA)
        vals.append(tt[0, 0] * r**3)
    vals = np.array(vals)
    assert np.all(np.abs(vals / vals[-1] - 1) < 0.02), vals
    # and the free-space 1/r part is gone: |M| r is small at r = 400
    tt, _ = O.pair_blocks(np.array([400.0, 0, z]), np.array([0, 0, z]), a=A, eta=ETA)
    free = O.freespace_tt(np.array([400.0, 0, z]), np.array([0, 0, z]), A, ETA)
    assert abs(tt[0, 0]) < 1e-3 * abs(free[0, 0])


def test_free_space_recovered_far_from_wall():
    """The wall part decays like a/h (tt) and faster (tr): free-space RPY is recovered."""
    dtt, dtr = [], []
    for H in (1e3, 1e5, 1e7):
        xi = np.array([2.5, 1.0, H + 0.7])
        xj = np.array([0.0, 0.0, H])
        tt, tr = O.pair_blocks(xi, xj, a=A, eta=ETA)
        dtt.append(np.max(np.abs(tt - O.freespace_tt(xi, xj, A, ETA))) * H / A)
        dtr.append(np.max(np.abs(tr - O.freespace_tr(xi, xj, A, ETA))) * H / A)
    assert abs(dtt[1] / dtt[2] - 1) < 1e-3 and abs(dtt[0] / dtt[2] - 1) < 1e-2
    assert dtt[2] < 2 * MU0
    assert dtr[0] < 1e-6 * MU0 and dtr[2] < 1e-20
