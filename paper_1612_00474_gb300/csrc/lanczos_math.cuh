// lanczos_math.cuh -- per-warp step of the Lanczos square root shared by the single and batched
// kernels: the Ritz data of the tridiagonal T_{k+1}, the update y_k = |W| Q sqrt(Lambda) Q^T e_1,
// the error estimate eps_k and the stopping decision (Sec. II.C).
#pragma once

#include <cfloat>

#include "rpb_internal.cuh"

namespace rpb {

constexpr int kMaxIter = 64;      // largest supported Lanczos dimension

// Layout of the small state block (doubles).
struct LzLayout {
    int M;
    size_t alpha, beta, y, yprev, c1, c2, coef, status, total;
    explicit LzLayout(int max_iter) : M(max_iter)
    {
        size_t o = 0;
        alpha = o; o += M + 1;
        beta = o; o += M + 1;
        y = o; o += M + 1;
        yprev = o; o += M + 1;
        c1 = o; o += M + 1;
        c2 = o; o += M + 1;
        coef = o; o += M + 1;
        status = o; o += 8;
        total = o;
    }
};
// status words
enum { ST_EPS = 0, ST_INV_BETA = 1, ST_NW = 2, ST_INV_NW = 3, ST_STOP = 4, ST_BREAK = 5 };

// Symmetric tridiagonal eigen-decomposition by the implicit QL method with a Wilkinson-type shift
// (Bowdler, Martin, Reinsch & Wilkinson), then y = |W| Q sqrt(max(Lambda, 0)) Q^T e_1.
// Called by one full warp: every lane runs the (identical) scalar recurrence on private copies of d
// and e and applies the rotations to its own rows (lane, lane + 32) of Q, so no lane reads another's
// data until the end.  lz: this Krylov space's state block; alpha_k, beta_k: the new coefficients;
// q0, sl, red: warp-private shared scratch (kMaxIter, kMaxIter, 32 doubles).
__device__ __forceinline__ void lanczos_tail_warp(double *__restrict__ lz, const LzLayout &L, int k, double tol,
                                                  double alpha_k, double beta_k, double *q0, double *sl,
                                                  double *red)
{
    const int lane = threadIdx.x & 31;
    double *status = lz + L.status;
    const int n = k + 1;
    double d[kMaxIter], e[kMaxIter], z0[kMaxIter], z1[kMaxIter];
    for (int i = 0; i < n; ++i) {
        d[i] = (i == k) ? alpha_k : lz[L.alpha + i];
        e[i] = (i < k) ? lz[L.beta + i] : 0.0;
        z0[i] = (i == lane) ? 1.0 : 0.0;
        z1[i] = (i == lane + 32) ? 1.0 : 0.0;
    }
    double tnorm = 0.0;
    for (int i = 0; i < n; ++i) tnorm = fmax(tnorm, fmax(fabs(d[i]), fabs(e[i])));
    tnorm = fmax(tnorm, beta_k);
    for (int l = 0; l < n; ++l) {
        for (int iter = 0; iter < 100; ++iter) {
            int m = l;
            for (; m < n - 1; ++m) {
                const double dd = fabs(d[m]) + fabs(d[m + 1]);
                if (fabs(e[m]) <= DBL_EPSILON * dd) break;
            }
            if (m == l) break;
            double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
            // |g| <= |d| / (2 DBL_EPSILON |d|) here (e[l] passed the test above), so g^2 + 1 cannot
            // overflow and the square root needs no hypot
            double r = sqrt(fma(g, g, 1.0));
            g = d[m] - d[l] + e[l] / (g + copysign(r, g));
            double s = 1.0, c = 1.0, p = 0.0;
            bool restart = false;
            for (int i = m - 1; i >= l; --i) {
                const double f = s * e[i];
                const double bb = c * e[i];
                // Givens rotation from one reciprocal square root (the entries of T are of the order
                // of the mobility, far from the float64 overflow and underflow limits)
                const double r2 = fma(f, f, g * g);
                if (r2 == 0.0) {
                    e[i + 1] = 0.0;
                    d[i + 1] -= p;
                    e[m] = 0.0;
                    restart = true;
                    break;
                }
                const double ir = rsqrt(r2);
                e[i + 1] = r2 * ir;
                s = f * ir;
                c = g * ir;
                g = d[i + 1] - p;
                r = (d[i] - g) * s + 2.0 * c * bb;
                p = s * r;
                d[i + 1] = g + p;
                g = c * r - bb;
                const double a0 = z0[i + 1];
                z0[i + 1] = s * z0[i] + c * a0;
                z0[i] = c * z0[i] - s * a0;
                if (n > 32) {  // rows lane + 32 exist only beyond 32 dimensions (float64 costs per warp instruction)
                    const double a1 = z1[i + 1];
                    z1[i + 1] = s * z1[i] + c * a1;
                    z1[i] = c * z1[i] - s * a1;
                }
            }
            if (restart) continue;
            d[l] -= p;
            e[l] = g;
            e[m] = 0.0;
        }
    }
    if (lane == 0)
        for (int j = 0; j < n; ++j) q0[j] = z0[j];
    // the eigenvalues are the same in every lane: lane j takes the square root of the j-th
    if (lane < n) sl[lane] = sqrt(fmax(d[lane], 0.0));
    if (lane + 32 < n) sl[lane + 32] = sqrt(fmax(d[lane + 32], 0.0));
    __syncwarp();
    const double nW = status[ST_NW];
    double y0 = 0.0, y1 = 0.0;
    for (int j = 0; j < n; ++j) {
        const double cj = sl[j] * q0[j];
        y0 = fma(z0[j], cj, y0);
        if (n > 32) y1 = fma(z1[j], cj, y1);
    }
    y0 *= nW;
    y1 *= nW;
    // eps_k = |y - (yprev, 0)| / |yprev|
    double num = 0.0, den = 0.0;
    if (lane < n) {
        const double p0 = (lane < k) ? lz[L.yprev + lane] : 0.0;
        num += (y0 - p0) * (y0 - p0);
        den += p0 * p0;
    }
    if (lane + 32 < n) {
        const double p1 = (lane + 32 < k) ? lz[L.yprev + lane + 32] : 0.0;
        num += (y1 - p1) * (y1 - p1);
        den += p1 * p1;
    }
    // warp sums by a butterfly (a fixed order; every lane ends with the same totals)
    double snum = num, sden = den;
    for (int o = 16; o > 0; o >>= 1) {
        snum += __shfl_xor_sync(0xffffffffu, snum, o);
        sden += __shfl_xor_sync(0xffffffffu, sden, o);
    }
    (void)red;
    if (lane < n) {
        lz[L.y + lane] = y0;
        lz[L.yprev + lane] = y0;
    }
    if (lane + 32 < n) {
        lz[L.y + lane + 32] = y1;
        lz[L.yprev + lane + 32] = y1;
    }
    if (lane == 0) {
        lz[L.alpha + k] = alpha_k;
        lz[L.beta + k] = beta_k;
        const double eps = (k >= 1 && sden > 0.0) ? sqrt(snum / sden) : -1.0;
        const bool brk = beta_k <= 1e-14 * tnorm;
        const bool conv = (tol > 0.0 && k >= 1 && eps <= tol);
        status[ST_EPS] = eps;
        status[ST_BREAK] = brk ? 1.0 : 0.0;
        status[ST_STOP] = (brk || conv) ? 1.0 : 0.0;
        status[ST_INV_BETA] = brk ? 0.0 : 1.0 / beta_k;
    }
}

}  // namespace rpb
