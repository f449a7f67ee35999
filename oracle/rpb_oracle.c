/*
 * rpb_oracle.c -- plain FP64 CPU oracle for the Rotne-Prager-Blake mobility.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct reference that the
 * CUDA path is checked against.  Only tests/, the smoke check and the CPU-baseline leg of
 * the benchmark may load it.  It shares no code, header or constant table with the CUDA
 * library, and it never calls it.
 *
 * Layout here is particle-major (the paper's ordering of q = {q_1 .. q_N}, Sec. II):
 * pos[3*i + c], F[3*i + c], ... with c in {x, y, z}.
 *
 * Contents
 *   - free-space RPY translation-translation block, both branches (Sec. II.B: the
 *     unbounded-domain RPY tensor cited there, including the overlap branch r < 2a);
 *   - free-space translation-rotation block, both branches (Sec. III, Eq.
 *     mobilityDifferentialTR and the overlap generalisation cited beside it);
 *   - wall (image) part, generated mechanically by derive_wall.py from Blake's image
 *     solution and the Faxen operators (Eq. mobilityDifferential / mobilityDifferentialTR);
 *   - regularisation M = B Mtilde B, B_ii = H0(z_i/a), Mtilde at z <- max(z, a)
 *     (Appendix A, Eq. effMob); the same B and clamp are applied to M_tr (reading: the
 *     paper states B for M_tt; a particle touching the wall must stop whatever the load);
 *   - the matvec U = M_tt F + M_tr T as a plain double loop (Sec. II.B, direct summation);
 *   - dense assembly of M_tt and M_tr;
 *   - the soft steric potential forces, Eq. (soft_potential), plus gravity (Sec. III).
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "wall_image.c"

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* H0 of Appendix A: 0 below 0, x on [0,1], 1 above. */
static double H0(double x)
{
    if (x > 1.0) return 1.0;
    if (x >= 0.0) return x;
    return 0.0;
}

/* Free-space RPY translation-translation block for target xi, source xj (3x3, row-major).
 * same != 0 marks the self block (j == i): mu0 I. */
static void freespace_tt(const double *xi, const double *xj, double a, double eta, int same, double *M)
{
    const double mu0 = 1.0 / (6.0 * M_PI * eta * a);
    double r[3] = {xi[0] - xj[0], xi[1] - xj[1], xi[2] - xj[2]};
    double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    double rn = sqrt(r2);
    memset(M, 0, 9 * sizeof(double));
    if (same || rn == 0.0) {
        M[0] = M[4] = M[8] = mu0;
        return;
    }
    double e[3] = {r[0] / rn, r[1] / rn, r[2] / rn};
    double c1, c2;
    if (rn >= 2.0 * a) {
        /* 1/(8 pi eta r) [ (1 + 2a^2/(3r^2)) I + (1 - 2a^2/r^2) e e ] */
        double pre = 1.0 / (8.0 * M_PI * eta * rn);
        c1 = pre * (1.0 + 2.0 * a * a / (3.0 * r2));
        c2 = pre * (1.0 - 2.0 * a * a / r2);
    } else {
        /* mu0 [ (1 - 9r/(32a)) I + (3r/(32a)) e e ] */
        c1 = mu0 * (1.0 - 9.0 * rn / (32.0 * a));
        c2 = mu0 * (3.0 * rn / (32.0 * a));
    }
    for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q)
            M[3 * p + q] = (p == q ? c1 : 0.0) + c2 * e[p] * e[q];
}

/* Free-space translation-rotation block: velocity of target from torque on source.
 * u = c(r) T x e, written as the matrix u_p = sum_q M[p][q] T_q, (T x e)_p = eps_{pqk} T_q e_k. */
static void freespace_tr(const double *xi, const double *xj, double a, double eta, int same, double *M)
{
    double r[3] = {xi[0] - xj[0], xi[1] - xj[1], xi[2] - xj[2]};
    double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    memset(M, 0, 9 * sizeof(double));
    if (same || rn == 0.0) return; /* free-space self coupling is zero */
    double e[3] = {r[0] / rn, r[1] / rn, r[2] / rn};
    double c;
    if (rn >= 2.0 * a)
        c = 1.0 / (8.0 * M_PI * eta * rn * rn);
    else
        c = (1.0 / (16.0 * M_PI * eta * a * a)) * (rn / a) * (1.0 - 3.0 * rn / (8.0 * a));
    /* matrix of T -> T x e:  [[0, e_z, -e_y], [-e_z, 0, e_x], [e_y, -e_x, 0]] */
    M[0 * 3 + 1] = c * e[2];
    M[0 * 3 + 2] = -c * e[1];
    M[1 * 3 + 0] = -c * e[2];
    M[1 * 3 + 2] = c * e[0];
    M[2 * 3 + 0] = c * e[1];
    M[2 * 3 + 1] = -c * e[0];
}

/* Regularised pair blocks M_ij = s_i s_j Mtilde(q~_i, q~_j), tt and tr (Appendix A).
 * wall == 0 is the unbounded-domain mobility (no image terms, no clamp, s = 1), used to compare the
 * Lanczos convergence without the wall's screening (Sec. II.C, inset of Fig. 1). */
void oracle_pair_blocks_w(const double *qi, const double *qj, int same, double a, double eta, int wall, double *Mtt,
                          double *Mtr)
{
    double xi[3] = {qi[0], qi[1], wall ? fmax(qi[2], a) : qi[2]};
    double xj[3] = {qj[0], qj[1], wall ? fmax(qj[2], a) : qj[2]};
    double si = wall ? H0(qi[2] / a) : 1.0, sj = wall ? H0(qj[2] / a) : 1.0;
    double ftt[9], ftr[9], wtt[9], wtr[9];
    freespace_tt(xi, xj, a, eta, same, ftt);
    freespace_tr(xi, xj, a, eta, same, ftr);
    if (wall) {
        wall_image_tt(xi[0] - xj[0], xi[1] - xj[1], xi[2], xj[2], a, wtt);
        wall_image_tr(xi[0] - xj[0], xi[1] - xj[1], xi[2], xj[2], a, wtr);
    } else {
        memset(wtt, 0, sizeof(wtt));
        memset(wtr, 0, sizeof(wtr));
    }
    const double inv8pe = 1.0 / (8.0 * M_PI * eta);
    for (int k = 0; k < 9; ++k) {
        if (Mtt) Mtt[k] = si * sj * (ftt[k] + inv8pe * wtt[k]);
        if (Mtr) Mtr[k] = si * sj * (ftr[k] + inv8pe * wtr[k]);
    }
}

void oracle_pair_blocks(const double *qi, const double *qj, int same, double a, double eta, double *Mtt, double *Mtr)
{
    oracle_pair_blocks_w(qi, qj, same, a, eta, 1, Mtt, Mtr);
}

/* Unregularised pieces, exposed for the pins. */
void oracle_freespace_tt(const double *xi, const double *xj, double a, double eta, int same, double *M)
{
    freespace_tt(xi, xj, a, eta, same, M);
}
void oracle_freespace_tr(const double *xi, const double *xj, double a, double eta, int same, double *M)
{
    freespace_tr(xi, xj, a, eta, same, M);
}
void oracle_blake_image_raw(double rx, double ry, double zi, double zj, double *G)
{
    blake_image_raw(rx, ry, zi, zj, G);
}
void oracle_wall_image_tt(double rx, double ry, double zi, double zj, double a, double *M)
{
    wall_image_tt(rx, ry, zi, zj, a, M);
}
void oracle_wall_image_tr(double rx, double ry, double zi, double zj, double a, double *M)
{
    wall_image_tr(rx, ry, zi, zj, a, M);
}

/* U = M_tt F + M_tr T over targets [i0, i1) (all N sources).  F or T may be NULL. */
void oracle_matvec_rows_w(int64_t N, int64_t i0, int64_t i1, const double *pos, const double *F,
                          const double *T, double a, double eta, int wall, double *U)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = i0; i < i1; ++i) {
        double u[3] = {0.0, 0.0, 0.0};
        for (int64_t j = 0; j < N; ++j) {
            double Mtt[9], Mtr[9];
            oracle_pair_blocks_w(&pos[3 * i], &pos[3 * j], i == j, a, eta, wall, Mtt, Mtr);
            for (int p = 0; p < 3; ++p)
                for (int q = 0; q < 3; ++q) {
                    if (F) u[p] += Mtt[3 * p + q] * F[3 * j + q];
                    if (T) u[p] += Mtr[3 * p + q] * T[3 * j + q];
                }
        }
        for (int p = 0; p < 3; ++p) U[3 * (i - i0) + p] = u[p];
    }
}

void oracle_matvec_rows(int64_t N, int64_t i0, int64_t i1, const double *pos, const double *F,
                        const double *T, double a, double eta, double *U)
{
    oracle_matvec_rows_w(N, i0, i1, pos, F, T, a, eta, 1, U);
}

void oracle_matvec(int64_t N, const double *pos, const double *F, const double *T, double a, double eta,
                   double *U)
{
    oracle_matvec_rows_w(N, 0, N, pos, F, T, a, eta, 1, U);
}

/* Dense 3N x 3N matrices (row-major, particle-major indices 3i+c). Either output may be NULL. */
void oracle_dense_w(int64_t N, const double *pos, double a, double eta, int wall, double *Mtt, double *Mtr)
{
    const int64_t n3 = 3 * N;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = 0; j < N; ++j) {
            double btt[9], btr[9];
            oracle_pair_blocks_w(&pos[3 * i], &pos[3 * j], i == j, a, eta, wall, btt, btr);
            for (int p = 0; p < 3; ++p)
                for (int q = 0; q < 3; ++q) {
                    if (Mtt) Mtt[(3 * i + p) * n3 + 3 * j + q] = btt[3 * p + q];
                    if (Mtr) Mtr[(3 * i + p) * n3 + 3 * j + q] = btr[3 * p + q];
                }
        }
}

void oracle_dense(int64_t N, const double *pos, double a, double eta, double *Mtt, double *Mtr)
{
    oracle_dense_w(N, pos, a, eta, 1, Mtt, Mtr);
}

/* -dU/dr for the soft potential of Eq. (soft_potential): U0/b on r < d, (U0/b) exp(-(r-d)/b) above. */
static double soft_force(double r, double d, double U0, double b)
{
    if (r < d) return U0 / b;
    return (U0 / b) * exp(-(r - d) / b);
}

/* Deterministic forces: gravity (-weight z), pair steric (d = 2a, centre distance) and wall steric
 * (d = a, r = height), Sec. III.  A coincident pair (r == 0) has no direction and exerts nothing. */
void oracle_forces(int64_t N, const double *pos, double a, double weight, double U0, double b, double *F)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < N; ++i) {
        double f[3] = {0.0, 0.0, -weight};
        for (int64_t j = 0; j < N; ++j) {
            if (j == i) continue;
            double r[3] = {pos[3 * i] - pos[3 * j], pos[3 * i + 1] - pos[3 * j + 1], pos[3 * i + 2] - pos[3 * j + 2]};
            double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
            if (rn == 0.0) continue;
            double m = soft_force(rn, 2.0 * a, U0, b);
            for (int p = 0; p < 3; ++p) f[p] += m * r[p] / rn;
        }
        f[2] += soft_force(pos[3 * i + 2], a, U0, b);
        for (int p = 0; p < 3; ++p) F[3 * i + p] = f[p];
    }
}

/* ------------------------------------------------------------------ pseudo-periodic boundaries
 * Appendix B: periodic in x and y with periods Lx, Ly; forces by the minimum image convention;
 * hydrodynamic interactions with the particles of the unit cell and of its eight neighbour cells.
 * Reading: for each pair the in-plane minimum-image displacement d is taken and the mobility is summed
 * over the nine shifts d + (nx Lx, ny Ly), nx, ny in {-1, 0, 1}; the pair (i, i) with no shift is the
 * self block, its eight shifts are ordinary pairs. */
static double min_image(double d, double L)
{
    return d - L * nearbyint(d / L);
}

void oracle_matvec_rows_p(int64_t N, int64_t i0, int64_t i1, const double *pos, const double *F, const double *T,
                          double a, double eta, int wall, double Lx, double Ly, double *U)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = i0; i < i1; ++i) {
        double u[3] = {0.0, 0.0, 0.0};
        const double *qi = &pos[3 * i];
        for (int64_t j = 0; j < N; ++j) {
            const double dx = min_image(qi[0] - pos[3 * j], Lx), dy = min_image(qi[1] - pos[3 * j + 1], Ly);
            for (int nx = -1; nx <= 1; ++nx)
                for (int ny = -1; ny <= 1; ++ny) {
                    const double qj[3] = {qi[0] - (dx + nx * Lx), qi[1] - (dy + ny * Ly), pos[3 * j + 2]};
                    const int self = (i == j) && nx == 0 && ny == 0;
                    double Mtt[9], Mtr[9];
                    oracle_pair_blocks_w(qi, qj, self, a, eta, wall, Mtt, Mtr);
                    for (int p = 0; p < 3; ++p)
                        for (int q = 0; q < 3; ++q) {
                            if (F) u[p] += Mtt[3 * p + q] * F[3 * j + q];
                            if (T) u[p] += Mtr[3 * p + q] * T[3 * j + q];
                        }
                }
        }
        for (int p = 0; p < 3; ++p) U[3 * (i - i0) + p] = u[p];
    }
}

void oracle_forces_p(int64_t N, const double *pos, double a, double weight, double U0, double b, double Lx, double Ly,
                     double *F)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < N; ++i) {
        double f[3] = {0.0, 0.0, -weight};
        for (int64_t j = 0; j < N; ++j) {
            if (j == i) continue;
            double r[3] = {min_image(pos[3 * i] - pos[3 * j], Lx), min_image(pos[3 * i + 1] - pos[3 * j + 1], Ly),
                           pos[3 * i + 2] - pos[3 * j + 2]};
            double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
            if (rn == 0.0) continue;
            double m = soft_force(rn, 2.0 * a, U0, b);
            for (int p = 0; p < 3; ++p) f[p] += m * r[p] / rn;
        }
        f[2] += soft_force(pos[3 * i + 2], a, U0, b);
        for (int p = 0; p < 3; ++p) F[3 * i + p] = f[p];
    }
}

/* Raw image tensor at many points (for the surface-quadrature pins): out[9*k ..]. */
void oracle_blake_image_raw_batch(int64_t n, const double *rx, const double *ry, const double *zi,
                                  const double *zj, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) blake_image_raw(rx[k], ry[k], zi[k], zj[k], &out[9 * k]);
}
