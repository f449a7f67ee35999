"""Pins of the oracle's RFD drift (Sec. II.A) and stochastic Adams-Bashforth step (Eq. AB)."""
import math

import numpy as np
import pytest

import oracle as O

A = 1.0
MU0 = 1 / (6 * math.pi * A)


def dmuzz_dz(h):
    """d/dh of mu_perp = mu0 (1 - 9/(8h) + 1/(2h^3) - 1/(8h^5)), differentiated by hand."""
    return MU0 / A * (9 / (8 * h**2) - 3 / (2 * h**4) + 5 / (8 * h**6))


@pytest.mark.parametrize("h", [1.1, 1.5, 2.5, 4.0])
def test_rfd_single_sphere_vertical(h):
    delta = 1e-4
    d = O.rfd_drift(np.array([[0.3, -0.2, h]]), np.array([[0.0, 0.0, 1.0]]), delta=delta)
    assert math.isclose(d[0, 2], dmuzz_dz(h), rel_tol=1e-7)
    assert d[0, 0] == 0.0 and d[0, 1] == 0.0


def test_rfd_mean_is_divergence():
    """E over W~ of the centred RFD is kT div M = (0, 0, d mu_zz/dz) for one sphere."""
    h = 1.3
    rng = np.random.default_rng(7)
    n = 20000
    acc = np.zeros((n, 3))
    q = np.array([[0.0, 0.0, h]])
    for s in range(n):
        acc[s] = O.rfd_drift(q, rng.standard_normal((1, 3)), delta=1e-5)[0]
    mean = acc.mean(0)
    se = acc.std(0) / math.sqrt(n)
    assert np.all(np.abs(mean - np.array([0, 0, dmuzz_dz(h)])) < 5 * se), (mean, se)


def test_rfd_in_plane_translation_invariance():
    """Displacing a whole layer in-plane changes nothing, so the in-plane drift of a pure in-plane W~
    averages to the in-plane divergence, which vanishes by translation invariance; here the exact
    statement: an in-plane rigid shift of both configurations leaves the drift unchanged."""
    pos = np.array([[0.0, 0.0, 1.2], [2.4, 0.3, 1.6], [1.0, 2.2, 1.1]])
    Wt = np.random.default_rng(3).standard_normal((3, 3))
    d1 = O.rfd_drift(pos, Wt, delta=1e-6)
    d2 = O.rfd_drift(pos + np.array([5.0, -3.0, 0.0]), Wt, delta=1e-6)
    assert np.allclose(d1, d2, rtol=0, atol=1e-8 * np.max(np.abs(d1)))


def _det_velocity(pos):
    F = O.forces(pos)
    T = np.tile([0.0, 1.0, 0.0], (len(pos), 1))
    return O.mobility_apply(pos, F, T)


def test_ab_deterministic_second_order():
    """kT = 0 removes noise and drift; AB (EM first step) is then second order for dq/dt = U(q)."""
    from scipy.integrate import solve_ivp

    q0 = np.array([[0.0, 0.0, 1.5], [4.0, 1.0, 1.2]])
    t_end = 0.4

    def rhs(t, y):
        return _det_velocity(y.reshape(-1, 3)).ravel()

    ref = solve_ivp(rhs, (0, t_end), q0.ravel(), method="DOP853", rtol=1e-13, atol=1e-14).y[:, -1]
    errs = []
    for nsteps in (10, 20, 40):
        dt = t_end / nsteps
        q, Up = q0.copy(), None
        for n in range(nsteps):
            q, Up, info = O.ab_step(q, Up, n, seed=0, dt=dt, kT=0.0, tol=1e-3)
        errs.append(np.linalg.norm(q.ravel() - ref))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.3 < r1 < 4.7 and 3.5 < r2 < 4.5, errs


def test_ab_step_composition():
    """The AB update equals its terms recombined: q + dt(3/2 U^n - 1/2 U^{n-1}) + sqrt(2 kT dt) g + dt d."""
    pos = np.array([[0.0, 0.0, 1.5], [2.5, 0.0, 1.3], [0.7, 2.4, 2.0]])
    Uprev = np.random.default_rng(1).standard_normal((3, 3)) * 0.01
    new, Un, info = O.ab_step(pos, Uprev, 3, seed=9, dt=0.01, detail=True)
    g, m, _, _ = O.lanczos_sqrt(pos, O.noise(3, 9, 3, 0), tol=1e-3)
    d = O.rfd_drift(pos, O.noise(3, 9, 3, 1), delta=1e-6)
    manual = pos + 0.01 * (1.5 * Un - 0.5 * Uprev) + math.sqrt(0.02) * g + 0.01 * d
    assert np.allclose(new, manual, rtol=0, atol=1e-15) and info["m"] == m
    # first step: EM (U^{-1} := U^0)
    new0, Un0, _ = O.ab_step(pos, None, 0, seed=9, dt=0.01)
    g0, _, _, _ = O.lanczos_sqrt(pos, O.noise(3, 9, 0, 0), tol=1e-3)
    d0 = O.rfd_drift(pos, O.noise(3, 9, 0, 1), delta=1e-6)
    assert np.allclose(new0, pos + 0.01 * Un0 + math.sqrt(0.02) * g0 + 0.01 * d0, rtol=0, atol=1e-15)


def test_em_deterministic_first_order():
    """kT = 0: Euler-Maruyama is first order in dt (AB is second order, test above)."""
    from scipy.integrate import solve_ivp

    q0 = np.array([[0.0, 0.0, 1.5], [4.0, 1.0, 1.2]])
    t_end = 0.4

    def rhs(t, y):
        return _det_velocity(y.reshape(-1, 3)).ravel()

    ref = solve_ivp(rhs, (0, t_end), q0.ravel(), method="DOP853", rtol=1e-13, atol=1e-14).y[:, -1]
    errs = []
    for nsteps in (20, 40, 80):
        dt = t_end / nsteps
        q, Up = q0.copy(), None
        for n in range(nsteps):
            q, Up, _ = O.ab_step(q, Up, n, seed=0, dt=dt, kT=0.0, scheme="EM")
        errs.append(np.linalg.norm(q.ravel() - ref))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 1.7 < r1 < 2.3 and 1.8 < r2 < 2.2, errs


@pytest.mark.parametrize("h", [1.2, 2.0])
def test_one_sided_rfd_first_order(h):
    """One-sided difference: derivative with an O(delta) error, halving with delta."""
    q = np.array([[0.1, 0.0, h]])
    e = np.array([[0.0, 0.0, 1.0]])
    errs = [abs(O.rfd_drift(q, e, delta=dl, one_sided=True)[0, 2] - dmuzz_dz(h)) for dl in (2e-3, 1e-3)]
    assert 1.8 < errs[0] / errs[1] < 2.2
    assert errs[1] < 1e-2 * abs(dmuzz_dz(h))


def test_em_step_composition():
    pos = np.array([[0.0, 0.0, 1.5], [2.5, 0.0, 1.3], [0.7, 2.4, 2.0]])
    Uprev = np.full((3, 3), 0.37)
    new, Un, info = O.ab_step(pos, Uprev, 4, seed=2, dt=0.02, scheme="EM", one_sided=True)
    g, _, _, _ = O.lanczos_sqrt(pos, O.noise(3, 2, 4, 0), tol=1e-3)
    d = O.rfd_drift(pos, O.noise(3, 2, 4, 1), delta=1e-6, one_sided=True)
    assert np.allclose(new, pos + 0.02 * Un + math.sqrt(0.04) * g + 0.02 * d, rtol=0, atol=1e-15)
