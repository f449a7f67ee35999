// lanczos.cu -- g ~ M^{1/2} W by the Lanczos (Krylov) method of Sec. II.C, on the device.
//
// Iteration k (0-based), all float64:
//   w = M v_k                                   (pair kernels, context precision)
//   c = V_{0..k}^T w ;  w -= V c                (classical Gram-Schmidt, pass 1; c_k = alpha_k)
//   c' = V_{0..k}^T w ; w -= V c'               (pass 2: full reorthogonalisation)
//   alpha_k = c_k + c'_k ;  beta_k = |w| ;  v_{k+1} = w / beta_k
//   T_{k+1} = tridiag(beta, alpha, beta) -> eigenpairs (implicit QL, one warp) ->
//   y_k = |W| Q sqrt(Lambda) Q^T e_1 ;  g_k = V_{0..k} y_k
//   eps_k = |y_k - (y_{k-1}, 0)| / |y_{k-1}|  (equals |g_k - g_{k-1}| / |g_{k-1}| while V stays
//   orthonormal, which the reorthogonalisation maintains), first defined at k = 1.
// The first subtraction of pass 1 already removes alpha_k v_k and beta_{k-1} v_{k-1}, i.e. the
// three-term recurrence is a subset of the reorthogonalisation.
// Reductions are two-level (per-block partials, then a fixed-order sum): results do not depend on
// scheduling.  The stopping decision is read back once per iteration (one small device-to-host
// copy and a stream synchronisation).
#include <cfloat>
#include <cmath>

#include "rpb_internal.cuh"

namespace rpb {

constexpr int kMaxIter = 64;      // largest supported Lanczos dimension
constexpr int kBlasThreads = 256;

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

size_t lanczos_state_elems(int max_iter)
{
    return LzLayout(max_iter).total;
}

static int blas_grid(int64_t n, int num_sms)
{
    int64_t g = (n + kBlasThreads - 1) / kBlasThreads;
    const int64_t cap = 2 * (int64_t)num_sms;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

size_t lanczos_red_elems(int max_iter)
{
    // (max_iter + 1) dot products + one norm, each with up to 2 * SMs partials (SM count <= 1024)
    return (size_t)(max_iter + 3) * 2048;
}

__device__ __forceinline__ double block_sum(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0) {
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += sh[k];
    }
    __syncthreads();
    return r;  // valid in thread 0
}

// red[k * G + b] = sum over block b's rows of V[k][r] * w[r], k = 0 .. nvec-1 (grid = (G, nvec)).
__global__ void __launch_bounds__(kBlasThreads) dots_kernel(const double *__restrict__ V, size_t ld, int64_t n,
                                                             const double *__restrict__ w, double *__restrict__ red)
{
    __shared__ double sh[kBlasThreads / 32];
    const int G = gridDim.x;
    const double *v = V + (size_t)blockIdx.y * ld;
    double acc = 0.0;
    for (int64_t r = (int64_t)blockIdx.x * kBlasThreads + threadIdx.x; r < n; r += (int64_t)G * kBlasThreads)
        acc = fma(v[r], w[r], acc);
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) red[(size_t)blockIdx.y * G + blockIdx.x] = acc;
}

// Reduce the dots partials for k = 0 .. nvec-1 (fixed order), then w -= sum_k coef_k V[k].
// Block 0 stores the coefficients in coef_out.  With norm_out != null also writes per-block partial
// sums of the updated w^2 to norm_out[b].
__global__ void __launch_bounds__(kBlasThreads) project_out_kernel(const double *__restrict__ V, size_t ld, int64_t n,
                                                                    int nvec, const double *__restrict__ red, int Gred,
                                                                    double *__restrict__ w,
                                                                    double *__restrict__ coef_out,
                                                                    double *__restrict__ norm_out)
{
    __shared__ double coef[kMaxIter + 1];
    __shared__ double sh[kBlasThreads / 32];
    for (int k = threadIdx.x; k < nvec; k += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < Gred; ++b) s += red[(size_t)k * Gred + b];
        coef[k] = s;
        if (blockIdx.x == 0) coef_out[k] = s;
    }
    __syncthreads();
    double acc = 0.0;
    for (int64_t r = (int64_t)blockIdx.x * kBlasThreads + threadIdx.x; r < n; r += (int64_t)gridDim.x * kBlasThreads) {
        double x = w[r];
        for (int k = 0; k < nvec; ++k) x -= coef[k] * V[(size_t)k * ld + r];
        w[r] = x;
        acc = fma(x, x, acc);
    }
    if (norm_out) {
        acc = block_sum(acc, sh);
        if (threadIdx.x == 0) norm_out[blockIdx.x] = acc;
    }
}

// v[r] = w[r] * status[idx]
__global__ void scale_kernel(const double *__restrict__ w, int64_t n, const double *__restrict__ status, int idx,
                             double *__restrict__ v)
{
    const double s = status[idx];
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        v[r] = w[r] * s;
}

// |W| from its squared-norm partials.
__global__ void norm_init_kernel(const double *__restrict__ red, int G, double *__restrict__ status)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < G; ++b) s += red[b];
        const double nw = sqrt(s);
        status[ST_NW] = nw;
        status[ST_INV_NW] = nw > 0.0 ? 1.0 / nw : 0.0;
        status[ST_EPS] = -1.0;
        status[ST_STOP] = 0.0;
        status[ST_BREAK] = 0.0;
    }
}

// Symmetric tridiagonal eigen-decomposition by the implicit QL method with a Wilkinson-type shift
// (Bowdler, Martin, Reinsch & Wilkinson), then y = |W| Q sqrt(max(Lambda, 0)) Q^T e_1.
// One warp: every lane runs the (identical) scalar recurrence on private copies of d and e and
// applies the rotations to its own rows (lane, lane + 32) of Q, so no lane reads another's data
// until the end.
__global__ void __launch_bounds__(32) lanczos_tail_kernel(double *__restrict__ lz, LzLayout L, int k, double tol,
                                                          const double *__restrict__ red_norm, int Gred)
{
    __shared__ double q0[kMaxIter];   // row 0 of Q
    __shared__ double sl[kMaxIter];   // sqrt(lambda)
    __shared__ double red[32];
    const int lane = threadIdx.x;
    double *status = lz + L.status;
    const int n = k + 1;
    // alpha_k, beta_k
    double bn = 0.0;
    for (int b = 0; b < Gred; ++b) bn += red_norm[b];  // identical order in every lane
    const double alpha_k = lz[L.c1 + k] + lz[L.c2 + k];
    const double beta_k = sqrt(bn);
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
            double r = hypot(g, 1.0);
            g = d[m] - d[l] + e[l] / (g + copysign(r, g));
            double s = 1.0, c = 1.0, p = 0.0;
            bool restart = false;
            for (int i = m - 1; i >= l; --i) {
                const double f = s * e[i];
                const double bb = c * e[i];
                r = hypot(f, g);
                e[i + 1] = r;
                if (r == 0.0) {
                    d[i + 1] -= p;
                    e[m] = 0.0;
                    restart = true;
                    break;
                }
                s = f / r;
                c = g / r;
                g = d[i + 1] - p;
                r = (d[i] - g) * s + 2.0 * c * bb;
                p = s * r;
                d[i + 1] = g + p;
                g = c * r - bb;
                const double a0 = z0[i + 1], a1 = z1[i + 1];
                z0[i + 1] = s * z0[i] + c * a0;
                z0[i] = c * z0[i] - s * a0;
                z1[i + 1] = s * z1[i] + c * a1;
                z1[i] = c * z1[i] - s * a1;
            }
            if (restart) continue;
            d[l] -= p;
            e[l] = g;
            e[m] = 0.0;
        }
    }
    if (lane == 0)
        for (int j = 0; j < n; ++j) {
            q0[j] = z0[j];
            sl[j] = sqrt(fmax(d[j], 0.0));
        }
    __syncwarp();
    const double nW = status[ST_NW];
    double y0 = 0.0, y1 = 0.0;
    for (int j = 0; j < n; ++j) {
        const double cj = sl[j] * q0[j];
        y0 = fma(z0[j], cj, y0);
        y1 = fma(z1[j], cj, y1);
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
    red[lane] = num;
    __syncwarp();
    double snum = 0.0, sden = 0.0;
    for (int t = 0; t < 32; ++t) snum += red[t];
    __syncwarp();
    red[lane] = den;
    __syncwarp();
    for (int t = 0; t < 32; ++t) sden += red[t];
    __syncwarp();
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

// g[r] = sum_{k < m} y[k] V[k][r]   (y already carries |W|)
__global__ void combine_kernel(const double *__restrict__ V, size_t ld, int64_t n, int m, const double *__restrict__ y,
                               double *__restrict__ g)
{
    __shared__ double ys[kMaxIter];
    for (int k = threadIdx.x; k < m; k += blockDim.x) ys[k] = y[k];
    __syncthreads();
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int k = 0; k < m; ++k) acc = fma(ys[k], V[(size_t)k * ld + r], acc);
        g[r] = acc;
    }
}

int lanczos_impl(rpb_ctx *ctx, int64_t N, const double *pos, const double *W, double *g, double tol, int max_iter,
                 int *iters_out, double *err_out, int *converged_out)
{
    cudaStream_t st = ctx->stream;
    const int64_t n = 3 * N;
    const size_t ld = (size_t)3 * ctx->max_N;
    const LzLayout L(ctx->max_iter);
    double *lz = ctx->ws.lz;
    double *status = lz + L.status;
    double *red = ctx->ws.red;
    double *V = ctx->ws.V;
    double *w = ctx->ws.w;
    double *hs = ctx->ws.host_status;
    const int G = blas_grid(n, ctx->num_sms);
    double *red_norm = red + (size_t)(ctx->max_iter + 1) * G;
    int rc;

    // |W| and v_0 = W / |W|
    dots_kernel<<<dim3(G, 1), kBlasThreads, 0, st>>>(W, 0, n, W, red);
    norm_init_kernel<<<1, 32, 0, st>>>(red, G, status);
    scale_kernel<<<G, kBlasThreads, 0, st>>>(W, n, status, ST_INV_NW, V);
    count_launches(3);
    if ((rc = cuda_fail(cudaMemcpyAsync(hs, status, 8 * sizeof(double), cudaMemcpyDeviceToHost, st), "status copy")))
        return rc;
    if ((rc = cuda_fail(cudaStreamSynchronize(st), "lanczos init"))) return rc;
    if (hs[ST_NW] == 0.0) {
        if ((rc = cuda_fail(cudaMemsetAsync(g, 0, n * sizeof(double), st), "zero g"))) return rc;
        if (iters_out) *iters_out = 0;
        if (err_out) *err_out = -1.0;
        if (converged_out) *converged_out = 1;
        return RPB_OK;
    }
    int m = 0;
    bool stopped = false;
    double eps = -1.0;
    for (int k = 0; k < max_iter; ++k) {
        const double *vk = V + (size_t)k * ld;
        if ((rc = mobility_apply_impl(ctx, N, pos, vk, nullptr, w))) return rc;
        const int nv = k + 1;
        dots_kernel<<<dim3(G, nv), kBlasThreads, 0, st>>>(V, ld, n, w, red);
        project_out_kernel<<<G, kBlasThreads, 0, st>>>(V, ld, n, nv, red, G, w, lz + L.c1, nullptr);
        dots_kernel<<<dim3(G, nv), kBlasThreads, 0, st>>>(V, ld, n, w, red);
        project_out_kernel<<<G, kBlasThreads, 0, st>>>(V, ld, n, nv, red, G, w, lz + L.c2, red_norm);
        lanczos_tail_kernel<<<1, 32, 0, st>>>(lz, L, k, tol, red_norm, G);
        count_launches(5);
        if ((rc = cuda_fail(cudaMemcpyAsync(hs, status, 8 * sizeof(double), cudaMemcpyDeviceToHost, st),
                            "status copy")))
            return rc;
        if ((rc = cuda_fail(cudaStreamSynchronize(st), "lanczos iteration"))) return rc;
        m = k + 1;
        eps = hs[ST_EPS];
        if (hs[ST_STOP] != 0.0) {
            stopped = true;
            break;
        }
        if (k + 1 < max_iter) {
            scale_kernel<<<G, kBlasThreads, 0, st>>>(w, n, status, ST_INV_BETA, V + (size_t)(k + 1) * ld);
            count_launches(1);
        }
    }
    combine_kernel<<<G, kBlasThreads, 0, st>>>(V, ld, n, m, lz + L.y, g);
    count_launches(1);
    if ((rc = cuda_fail(cudaGetLastError(), "lanczos kernels"))) return rc;
    if (iters_out) *iters_out = m;
    if (err_out) *err_out = eps;
    const bool converged = stopped;
    if (converged_out) *converged_out = converged ? 1 : 0;
    if (tol > 0.0 && !converged) {
        set_error("lanczos: no convergence in %d iterations (eps=%g, tol=%g)", m, eps, tol);
        return RPB_ENOCONV;
    }
    return RPB_OK;
}

}  // namespace rpb
