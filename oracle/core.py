"""Oracle for the Brownian-dynamics hot path: matvec, Lanczos sqrt, RFD drift, AB step.

TEST INFRASTRUCTURE ONLY: see oracle/__init__.py.

Arrays here are particle-major, shape (N, 3) (the paper orders q = {q_1 .. q_N},
Sec. II).  The pair arithmetic lives in rpb_oracle.c (plain FP64 loops); the
steps above it follow the paper in its own order with numpy FP64:

  matvec      U = M_tt F + M_tr T                      Sec. II.B, Sec. III (M_C T)
  lanczos     g_m ~ M^{1/2} W in K_m(M, W)             Sec. II.C (Krylov method of Ando et al.)
  rfd_drift   (kT/delta)[M(q + delta/2 W~) W~ - M(q - delta/2 W~) W~]     Sec. II.A, Eq. (EM)
  ab_step     q^{n+1} = q^n + dt[3/2 U^n - 1/2 U^{n-1}] + sqrt(2 kT dt) g + dt drift   Eq. (AB)
"""
import ctypes
import math

import numpy as np

from . import build as _build
from . import philox as _philox

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        i64 = ctypes.c_int64
        d = ctypes.c_double
        L.oracle_pair_blocks.argtypes = [dp, dp, ctypes.c_int, d, d, dp, dp]
        L.oracle_freespace_tt.argtypes = [dp, dp, d, d, ctypes.c_int, dp]
        L.oracle_freespace_tr.argtypes = [dp, dp, d, d, ctypes.c_int, dp]
        L.oracle_blake_image_raw.argtypes = [d, d, d, d, dp]
        L.oracle_blake_image_raw_batch.argtypes = [i64, dp, dp, dp, dp, dp]
        L.oracle_blake_image_raw_batch.restype = None
        L.oracle_wall_image_tt.argtypes = [d, d, d, d, d, dp]
        L.oracle_wall_image_tr.argtypes = [d, d, d, d, d, dp]
        L.oracle_matvec_rows.argtypes = [i64, i64, i64, dp, dp, dp, d, d, dp]
        L.oracle_matvec_rows_w.argtypes = [i64, i64, i64, dp, dp, dp, d, d, ctypes.c_int, dp]
        L.oracle_matvec_rows_w.restype = None
        L.oracle_dense_w.argtypes = [i64, dp, d, d, ctypes.c_int, dp, dp]
        L.oracle_dense_w.restype = None
        L.oracle_matvec_rows_p.argtypes = [i64, i64, i64, dp, dp, dp, d, d, ctypes.c_int, d, d, dp]
        L.oracle_matvec_rows_p.restype = None
        L.oracle_forces_p.argtypes = [i64, dp, d, d, d, d, d, d, dp]
        L.oracle_forces_p.restype = None
        L.oracle_matvec.argtypes = [i64, dp, dp, dp, d, d, dp]
        L.oracle_dense.argtypes = [i64, dp, d, d, dp, dp]
        L.oracle_forces.argtypes = [i64, dp, d, d, d, d, dp]
        for f in (L.oracle_pair_blocks, L.oracle_freespace_tt, L.oracle_freespace_tr, L.oracle_blake_image_raw,
                  L.oracle_wall_image_tt, L.oracle_wall_image_tr, L.oracle_matvec_rows, L.oracle_matvec,
                  L.oracle_dense, L.oracle_forces):
            f.restype = None
        _lib = L
    return _lib


def _p(x):
    if x is None:
        return None
    return x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c3(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1, 3))


# ---------------------------------------------------------------- pair blocks
def pair_blocks(qi, qj, same=False, a=1.0, eta=1.0):
    """Regularised 3x3 blocks (M_tt, M_tr) of target qi, source qj (Appendix A, Eq. effMob)."""
    qi = np.ascontiguousarray(qi, dtype=np.float64)
    qj = np.ascontiguousarray(qj, dtype=np.float64)
    tt = np.zeros(9)
    tr = np.zeros(9)
    lib().oracle_pair_blocks(_p(qi), _p(qj), int(same), a, eta, _p(tt), _p(tr))
    return tt.reshape(3, 3), tr.reshape(3, 3)


def freespace_tt(xi, xj, a=1.0, eta=1.0, same=False):
    out = np.zeros(9)
    lib().oracle_freespace_tt(_p(np.ascontiguousarray(xi, dtype=float)), _p(np.ascontiguousarray(xj, dtype=float)),
                              a, eta, int(same), _p(out))
    return out.reshape(3, 3)


def freespace_tr(xi, xj, a=1.0, eta=1.0, same=False):
    out = np.zeros(9)
    lib().oracle_freespace_tr(_p(np.ascontiguousarray(xi, dtype=float)), _p(np.ascontiguousarray(xj, dtype=float)),
                              a, eta, int(same), _p(out))
    return out.reshape(3, 3)


def blake_image_raw(x, y):
    """8 pi eta G_img(x, y) of Blake's image system (no Faxen operators)."""
    out = np.zeros(9)
    lib().oracle_blake_image_raw(x[0] - y[0], x[1] - y[1], x[2], y[2], _p(out))
    return out.reshape(3, 3)


def blake_image_raw_batch(rx, ry, zi, zj):
    """8 pi eta G_img at many points; arrays of equal length n -> (n, 3, 3)."""
    arrs = [np.ascontiguousarray(v, dtype=np.float64).ravel() for v in (rx, ry, zi, zj)]
    n = arrs[0].size
    out = np.zeros((n, 9))
    lib().oracle_blake_image_raw_batch(n, *[_p(v) for v in arrs], _p(out))
    return out.reshape(n, 3, 3)


def wall_image_tt(x, y, a=1.0):
    """(I + a^2/6 lap_x)(I + a^2/6 lap_y) 8 pi eta G_img at (x, y)."""
    out = np.zeros(9)
    lib().oracle_wall_image_tt(x[0] - y[0], x[1] - y[1], x[2], y[2], a, _p(out))
    return out.reshape(3, 3)


def wall_image_tr(x, y, a=1.0):
    """(I + a^2/6 lap_x)(1/2 curl_y) 8 pi eta G_img at (x, y)."""
    out = np.zeros(9)
    lib().oracle_wall_image_tr(x[0] - y[0], x[1] - y[1], x[2], y[2], a, _p(out))
    return out.reshape(3, 3)


# ---------------------------------------------------------------- matvec and dense
def mobility_apply(pos, F=None, T=None, a=1.0, eta=1.0, rows=None, wall=True, periodic=None):
    """U = M_tt F + M_tr T (Sec. II.B direct summation, Sec. III torque coupling); shape (N, 3).

    rows=(i0, i1) restricts the output to targets i0..i1-1 (all N sources are summed).
    wall=False: the unbounded-domain RPY mobility (no wall terms, no regularisation).
    periodic=(Lx, Ly): pseudo-periodic boundaries of Appendix B (minimum image plus the eight
    neighbour cells, see rpb_oracle.c)."""
    pos = _c3(pos)
    N = pos.shape[0]
    Fc = None if F is None else _c3(F)
    Tc = None if T is None else _c3(T)
    i0, i1 = (0, N) if rows is None else rows
    U = np.zeros((i1 - i0, 3))
    if periodic is not None:
        lib().oracle_matvec_rows_p(N, i0, i1, _p(pos), _p(Fc), _p(Tc), a, eta, int(bool(wall)), float(periodic[0]),
                                   float(periodic[1]), _p(U))
    else:
        lib().oracle_matvec_rows_w(N, i0, i1, _p(pos), _p(Fc), _p(Tc), a, eta, int(bool(wall)), _p(U))
    return U


def dense(pos, a=1.0, eta=1.0, wall=True):
    """Dense (M_tt, M_tr), each 3N x 3N, particle-major rows/columns (wall=False: unbounded domain)."""
    pos = _c3(pos)
    N = pos.shape[0]
    tt = np.zeros((3 * N, 3 * N))
    tr = np.zeros((3 * N, 3 * N))
    lib().oracle_dense_w(N, _p(pos), a, eta, int(bool(wall)), _p(tt), _p(tr))
    return tt, tr


def forces(pos, a=1.0, weight=1.0, U0=1.0, b=0.1, periodic=None):
    """Gravity -weight z plus the soft steric forces of Eq. (soft_potential); shape (N, 3).
    periodic=(Lx, Ly): minimum image convention (Appendix B)."""
    pos = _c3(pos)
    F = np.zeros_like(pos)
    if periodic is not None:
        lib().oracle_forces_p(pos.shape[0], _p(pos), a, weight, U0, b, float(periodic[0]), float(periodic[1]), _p(F))
    else:
        lib().oracle_forces(pos.shape[0], _p(pos), a, weight, U0, b, _p(F))
    return F


# ---------------------------------------------------------------- Lanczos (Sec. II.C)
def _tridiag_sqrt_e1(alpha, beta):
    """f(T) e_1 with f = sqrt for the symmetric tridiagonal T = tridiag(beta, alpha, beta).

    numpy's symmetric eigensolver is the library step; negative eigenvalues (round-off) are
    clamped to zero."""
    k = len(alpha)
    Tm = np.diag(alpha)
    if k > 1:
        Tm += np.diag(beta[: k - 1], 1) + np.diag(beta[: k - 1], -1)
    lam, Q = np.linalg.eigh(Tm)
    lam = np.clip(lam, 0.0, None)
    return Q @ (np.sqrt(lam) * Q[0, :])


def self_diagonal(pos, a=1.0, eta=1.0, wall=True, periodic=None):
    """Diagonal of the self blocks M_ii of M_tt, particle-major, shape (N, 3).

    The block-diagonal preconditioner Sec. II.C mentions keeps each particle's self mobility,
    including its interaction with the wall, and neglects its hydrodynamic interactions with other
    particles; in pseudo-periodic mode a particle's periodic images count as other particles, so
    the block is the same as without periods.  The translation self block of the wall-corrected
    (regularised) mobility is diagonal, so its diagonal is the block: taken from the oracle's own
    self block (pair_blocks with same=True), or mu0 I without the wall."""
    pos = _c3(pos)
    N = pos.shape[0]
    D = np.zeros((N, 3))
    for i in range(N):
        if wall:
            D[i] = np.diag(pair_blocks(pos[i], pos[i], same=True, a=a, eta=eta)[0])
        else:
            D[i] = np.diag(freespace_tt(pos[i], pos[i], a=a, eta=eta, same=True))
    return D


def lanczos_sqrt(pos, W, tol=1e-3, max_iter=100, exact_iters=None, a=1.0, eta=1.0, matvec=None, wall=True,
                 periodic=None, precondition=False):
    """g_m ~ M_tt^{1/2} W by m steps of Lanczos with full reorthogonalisation.

    Readings where the paper is silent (it cites the Krylov method of Ando et al.):
      - v_1 = W/|W|;  w = M v_k - beta_{k-1} v_{k-1};  alpha_k = v_k . w;  w -= alpha_k v_k;
        w is then orthogonalised against v_1..v_k by classical Gram-Schmidt applied twice;
        beta_k = |w|;  v_{k+1} = w / beta_k.
      - g_k = |W| V_k f(T_k) e_1 with f = sqrt.
      - error estimate eps_k = |g_k - g_{k-1}| / |g_{k-1}| (Sec. II.C), first available at k = 2;
        stop at the first k with eps_k <= tol; m = number of matvecs.
      - breakdown beta_k <= 1e-14 max|T_k| means the Krylov space is invariant: g_k is exact; stop.
      - W = 0 gives g = 0 with m = 0.
      - exact_iters=m runs exactly m iterations (unless breakdown) regardless of tol, so that
        two implementations can be compared at equal m.
      - precondition=True: the block-diagonal preconditioner that Sec. II.C reports trying (the
        paper's own runs do not use it).  With D the diagonal of the self blocks (self_diagonal)
        and P = D^{-1/2} (0 where D = 0), the iteration runs on P M P with the same W, and
        g = D^{1/2} y; then g = L W with L L^T = M, so the noise has the right covariance (it is a
        different square root than M^{1/2}).  eps_k and the stop are taken on the iterate y of
        the preconditioned operator (the paper states its criterion only without preconditioning).
    Returns (g (N,3), m, eps_m (nan if m < 2), converged)."""
    pos = _c3(pos)
    w0 = _c3(W).ravel()
    n = w0.size
    if matvec is None:
        def matvec(v):
            return mobility_apply(pos, v.reshape(-1, 3), None, a, eta, wall=wall, periodic=periodic).ravel()
    if precondition:
        D = self_diagonal(pos, a, eta, wall).ravel()
        Pd = np.where(D > 0.0, 1.0 / np.sqrt(np.where(D > 0.0, D, 1.0)), 0.0)
        y, m, eps, conv = lanczos_sqrt(pos, W, tol, max_iter, exact_iters, matvec=lambda v: Pd * matvec(Pd * v))
        return (np.sqrt(D) * y.ravel()).reshape(-1, 3), m, eps, conv
    nW = float(np.sqrt(w0 @ w0))
    if nW == 0.0:
        return np.zeros_like(w0).reshape(-1, 3), 0, float("nan"), True
    limit = exact_iters if exact_iters is not None else max_iter
    V = np.zeros((limit + 1, n))
    V[0] = w0 / nW
    alpha, beta = [], []
    g_prev = None
    eps = float("nan")
    converged = False
    m = 0
    for k in range(limit):
        w = matvec(V[k])
        if k > 0:
            w = w - beta[k - 1] * V[k - 1]
        ak = float(V[k] @ w)
        w = w - ak * V[k]
        for _ in range(2):
            c = V[: k + 1] @ w
            w = w - V[: k + 1].T @ c
        bk = float(np.sqrt(w @ w))
        alpha.append(ak)
        beta.append(bk)
        m = k + 1
        y = _tridiag_sqrt_e1(np.array(alpha), np.array(beta))
        g = nW * (V[: k + 1].T @ y)
        if g_prev is not None:
            eps = float(np.linalg.norm(g - g_prev) / np.linalg.norm(g_prev))
        tnorm = max(abs(v) for v in alpha + beta)
        breakdown = bk <= 1e-14 * tnorm
        if exact_iters is None and g_prev is not None and eps <= tol:
            converged = True
            break
        if breakdown:
            converged = True
            break
        V[k + 1] = w / bk
        g_prev = g
    return g.reshape(-1, 3), m, eps, converged


# ---------------------------------------------------------------- RFD (Sec. II.A)
def rfd_drift(pos, Wt, delta=1e-6, kT=1.0, a=1.0, eta=1.0, parts=False, one_sided=False, periodic=None):
    """(kT/delta)[M_tt(q + delta/2 W~) W~ - M_tt(q - delta/2 W~) W~]; the displaced configurations
    are regularised anew (clamp and H0 at the displaced heights).  parts=True also returns the two
    matvecs.  one_sided=True: (kT/delta)[M_tt(q + delta W~) W~ - M_tt(q) W~], the one-sided
    difference Sec. II.A mentions."""
    pos = _c3(pos)
    Wt = _c3(Wt)
    if one_sided:
        up = mobility_apply(pos + delta * Wt, Wt, None, a, eta, periodic=periodic)
        um = mobility_apply(pos, Wt, None, a, eta, periodic=periodic)
    else:
        up = mobility_apply(pos + 0.5 * delta * Wt, Wt, None, a, eta, periodic=periodic)
        um = mobility_apply(pos - 0.5 * delta * Wt, Wt, None, a, eta, periodic=periodic)
    d = (kT / delta) * (up - um)
    if parts:
        return d, up, um
    return d


# ---------------------------------------------------------------- noise
def noise(N, seed, step, stream, instance=0):
    """Standard normals for particle-major index k = 3 i + c, shape (N, 3).  Stream 0 is W (Lanczos),
    stream 1 is W~ (RFD)."""
    return _philox.normals(3 * N, seed, step, stream, instance).reshape(N, 3)


# ---------------------------------------------------------------- AB step (Eq. AB)
def ab_step(pos, U_prev, step, seed, dt=0.01, delta=1e-6, tol=1e-3, max_iter=100, kT=1.0, a=1.0, eta=1.0,
            weight=1.0, torque=(0.0, 1.0, 0.0), U0=1.0, b=0.1, exact_iters=None, detail=False, scheme="AB",
            one_sided=False, periodic=None, precondition=False):
    """One stochastic Adams-Bashforth step (scheme="AB", Eq. AB) or Euler-Maruyama step
    (scheme="EM", Eq. EM: q^{n+1} = q^n + dt U^n + sqrt(2 kT dt) g + dt drift).

    Readings: the deterministic velocity U^n = M_tt F^n + M_tr T (Sec. III: M_C T is treated like
    M F); the first AB step (step == 0, no U^{n-1}) is Euler-Maruyama, i.e. U^{-1} := U^0; the torque
    is the same constant vector on every particle.  one_sided selects the one-sided RFD;
    precondition the block-diagonal preconditioner of the Lanczos step (see lanczos_sqrt).
    Returns (q^{n+1}, U^n, info)."""
    pos = _c3(pos)
    N = pos.shape[0]
    F = forces(pos, a, weight, U0, b, periodic=periodic)
    T = np.tile(np.asarray(torque, dtype=np.float64), (N, 1))
    Un = mobility_apply(pos, F, T, a, eta, periodic=periodic)
    W = noise(N, seed, step, 0)
    Wt = noise(N, seed, step, 1)
    g, m, eps, conv = lanczos_sqrt(pos, W, tol, max_iter, exact_iters, a, eta, periodic=periodic,
                                   precondition=precondition)
    d, up, um = rfd_drift(pos, Wt, delta, kT, a, eta, parts=True, one_sided=one_sided, periodic=periodic)
    Up = Un if (scheme == "EM" or step == 0 or U_prev is None) else _c3(U_prev)
    new = pos + dt * (1.5 * Un - 0.5 * Up) + math.sqrt(2.0 * kT * dt) * g + dt * d
    info = dict(m=m, eps=eps, converged=conv)
    if detail:
        info.update(F=F, U=Un, W=W, Wt=Wt, g=g, drift=d, rfd_plus=up, rfd_minus=um)
    return new, Un, info


def rel_err(x, ref):
    """Relative 2-norm error |x - ref| / |ref| over the whole vector."""
    x = np.asarray(x, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(x - ref) / den) if den > 0 else float(np.linalg.norm(x - ref))
