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
// copy and a stream synchronisation), or, inside a graph-replayed run, taken on the device: each
// iteration after the first is a conditional node that the previous iteration enables.
#include <cfloat>
#include <cmath>

#include "lanczos_math.cuh"
#include "pair_math.cuh"

namespace rpb {

constexpr int kBlasThreads = 256;


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

// Sum of n partials by one warp in a fixed order (lane-strided sums, then a butterfly); every lane
// returns the total.
__device__ __forceinline__ double warp_sum_partials(const double *__restrict__ p, int n)
{
    const int lane = threadIdx.x & 31;
    double v = 0.0;
    for (int b = lane; b < n; b += 32) v += p[b];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
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
    const int warp = threadIdx.x >> 5;
    for (int k = warp; k < nvec; k += kBlasThreads / 32) {
        const double s = warp_sum_partials(red + (size_t)k * Gred, Gred);
        if ((threadIdx.x & 31) == 0) {
            coef[k] = s;
            if (blockIdx.x == 0) coef_out[k] = s;
        }
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

// v[r] = w[r] / |w|, |w|^2 summed from the norm partials by one warp in the fixed order the
// tridiagonal kernel uses for beta_k (so 1/|w| is bitwise its 1/beta_k).
__global__ void scale_norm_kernel(const double *__restrict__ w, int64_t n, const double *__restrict__ red_norm,
                                  int Gred, double *__restrict__ v)
{
    __shared__ double inv;
    if (threadIdx.x < 32) {
        const double bn = warp_sum_partials(red_norm, Gred);
        if (threadIdx.x == 0) inv = 1.0 / sqrt(bn);
    }
    __syncthreads();
    const double s = inv;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        v[r] = w[r] * s;
}

// |W| from its squared-norm partials.
__global__ void norm_init_kernel(const double *__restrict__ red, int G, double *__restrict__ status)
{
    const double s = warp_sum_partials(red, G);  // launched as one warp
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const double nw = sqrt(s);
        status[ST_NW] = nw;
        status[ST_INV_NW] = nw > 0.0 ? 1.0 / nw : 0.0;
        status[ST_EPS] = -1.0;
        status[ST_STOP] = 0.0;
        status[ST_BREAK] = 0.0;
    }
}

// One warp: the tridiagonal step for the single Krylov space (see lanczos_tail_warp).  Inside a
// replayed graph (runs != null) lane 0 then counts this run of iteration k, records m = k + 1 and lets
// the conditional node of iteration k + 1 run only if the iteration has not stopped.
__global__ void __launch_bounds__(32) lanczos_tail_kernel(double *__restrict__ lz, LzLayout L, int k, double tol,
                                                          const double *__restrict__ red_norm, int Gred,
                                                          cudaGraphConditionalHandle next = 0ull, int has_next = 0,
                                                          unsigned long long *__restrict__ runs = nullptr,
                                                          int *__restrict__ m_out = nullptr)
{
    __shared__ double q0[kMaxIter];
    __shared__ double sl[kMaxIter];
    __shared__ double red[32];
    const double bn = warp_sum_partials(red_norm, Gred);  // the same value in every lane
    lanczos_tail_warp(lz, L, k, tol, lz[L.c1 + k] + lz[L.c2 + k], sqrt(bn), q0, sl, red);
    if (runs && threadIdx.x == 0) {  // lane 0 wrote the status words
        *runs += 1ull;
        *m_out = k + 1;
        if (has_next) cudaGraphSetConditional(next, lz[L.status + ST_STOP] == 0.0 ? 1u : 0u);
    }
}

// g[r] = sum_{k < m} y[k] V[k][r]   (y already carries |W|); d_m (optional): read m from the device
__global__ void combine_kernel(const double *__restrict__ V, size_t ld, int64_t n, int m, const double *__restrict__ y,
                               double *__restrict__ g, const int *__restrict__ d_m)
{
    __shared__ double ys[kMaxIter];
    if (d_m) m = *d_m;
    for (int k = threadIdx.x; k < m; k += blockDim.x) ys[k] = y[k];
    __syncthreads();
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int k = 0; k < m; ++k) acc = fma(ys[k], V[(size_t)k * ld + r], acc);
        g[r] = acc;
    }
}

// Block-diagonal preconditioner (Sec. II.C reports trying it: each particle's self mobility, with
// its wall interaction, and no interactions between particles).  The translation self block of the
// wall-corrected, regularised mobility is diagonal, s_i^2 / (8 pi eta) (mu_par, mu_par, mu_perp) at
// the clamped height, so P = D^{-1/2} is a vector; P = 0 where D = 0 (spheres on or below the wall
// have no mobility).  Free space: D = mu0.
__global__ void precond_diag_kernel(const double *__restrict__ pos, int64_t N, PairConsts<double> c, double a,
                                    double scale, int wall, double *__restrict__ P)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const double z = pos[2 * N + i];
        double ux = 0.0, uy = 0.0, uz = 0.0;
        double k = scale;
        if (wall) {
            const double si = H0(z / a);
            k *= si * si;
            self_velocity<false, true>(fmax(z, a), 1.0, 1.0, 1.0, 0.0, 0.0, c, ux, uy, uz);
        } else {
            self_velocity<false, false>(z, 1.0, 1.0, 1.0, 0.0, 0.0, c, ux, uy, uz);
        }
        const double dx = k * ux, dz = k * uz;
        P[i] = dx > 0.0 ? 1.0 / sqrt(dx) : 0.0;
        P[N + i] = P[i];
        P[2 * N + i] = dz > 0.0 ? 1.0 / sqrt(dz) : 0.0;
    }
}

// out = x P (inverse: x / P, and 0 where P = 0), elementwise over 3N
// (x and out may be the same vector: no __restrict__ on them)
__global__ void precond_scale_kernel(const double *x, const double *__restrict__ P, int64_t n, int inverse,
                                     double *out)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const double p = P[r];
        out[r] = inverse ? (p > 0.0 ? x[r] / p : 0.0) : x[r] * p;
    }
}

int lanczos_precond_prepare(rpb_ctx *ctx, int64_t N, const double *pos)
{
    if (!ctx->precond) return RPB_OK;
    const double a = ctx->p.a;
    precond_diag_kernel<<<blas_grid(N, ctx->num_sms), kBlasThreads, 0, ctx->stream>>>(
        pos, N, make_consts<double>(a), a, 1.0 / (8.0 * kPi * ctx->p.eta), ctx->p.wall, ctx->ws.pc);
    count_launches(1);
    return cuda_fail(cudaGetLastError(), "preconditioner");
}

int precond_scale(rpb_ctx *ctx, int64_t N, const double *x, double *out, bool inverse)
{
    precond_scale_kernel<<<blas_grid(3 * N, ctx->num_sms), kBlasThreads, 0, ctx->stream>>>(x, ctx->ws.pc, 3 * N,
                                                                                         inverse ? 1 : 0, out);
    count_launches(1);
    return cuda_fail(cudaGetLastError(), "preconditioner scale");
}

int lanczos_init(rpb_ctx *ctx, int64_t N, const double *W, bool *nw_zero, bool graph)
{
    cudaStream_t st = ctx->stream;
    const int64_t n = 3 * N;
    const LzLayout L(ctx->max_iter);
    double *status = ctx->ws.lz + L.status;
    double *red = ctx->ws.red;
    double *hs = ctx->ws.host_status;
    const int G = blas_grid(n, ctx->num_sms);
    int rc;
    // |W| and v_0 = W / |W|
    dots_kernel<<<dim3(G, 1), kBlasThreads, 0, st>>>(W, 0, n, W, red);
    norm_init_kernel<<<1, 32, 0, st>>>(red, G, status);
    scale_kernel<<<G, kBlasThreads, 0, st>>>(W, n, status, ST_INV_NW, ctx->ws.V);
    count_launches(3);
    if (graph) {
        *nw_zero = false;
        return cuda_fail(cudaGetLastError(), "lanczos init");
    }
    if ((rc = cuda_fail(cudaMemcpyAsync(hs, status, 8 * sizeof(double), cudaMemcpyDeviceToHost, st), "status copy")))
        return rc;
    if ((rc = cuda_fail(cudaStreamSynchronize(st), "lanczos init"))) return rc;
    *nw_zero = hs[ST_NW] == 0.0;
    return RPB_OK;
}

int lanczos_impl(rpb_ctx *ctx, int64_t N, const double *pos, const double *W, double *g, double tol, int max_iter,
                 int *iters_out, double *err_out, int *converged_out, LzGraph *gr)
{
    bool zero = false;
    int rc;
    if ((rc = lanczos_precond_prepare(ctx, N, pos)) || (rc = lanczos_init(ctx, N, W, &zero, gr != nullptr))) return rc;
    if (zero) {
        if ((rc = cuda_fail(cudaMemsetAsync(g, 0, 3 * N * sizeof(double), ctx->stream), "zero g"))) return rc;
        if (iters_out) *iters_out = 0;
        if (err_out) *err_out = -1.0;
        if (converged_out) *converged_out = 1;
        return RPB_OK;
    }
    return lanczos_run(ctx, N, pos, g, tol, max_iter, false, iters_out, err_out, converged_out, gr);
}

// w = M v (with the preconditioner: P M P v), on the context's stream
static int lanczos_product(rpb_ctx *ctx, int64_t N, const double *pos, const double *v, double *w)
{
    int rc;
    if (!ctx->precond) return mobility_apply_impl(ctx, N, pos, v, nullptr, w);
    if ((rc = precond_scale(ctx, N, v, ctx->ws.pcx, false)) ||
        (rc = mobility_apply_impl(ctx, N, pos, ctx->ws.pcx, nullptr, w)))
        return rc;
    return precond_scale(ctx, N, w, w, false);
}

int lanczos_run(rpb_ctx *ctx, int64_t N, const double *pos, double *g, double tol, int max_iter, bool first_done,
                int *iters_out, double *err_out, int *converged_out, LzGraph *gr)
{
    const cudaStream_t main_st = ctx->stream;
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
    int m = 0;
    bool stopped = false;
    double eps = -1.0;
    if (gr) {  // one conditional handle per iteration after the first, on the graph being captured
        cudaStreamCaptureStatus cs;
        cudaGraph_t cg = nullptr;
        if ((rc = cuda_fail(cudaStreamGetCaptureInfo(main_st, &cs, nullptr, &cg, nullptr, nullptr, nullptr),
                            "capture info")))
            return rc;
        CondSet cs_all = {};
        for (int k = 1; k < max_iter; ++k) {
            gr->iter_launches[k] = 0;
            if ((rc = cuda_fail(cudaGraphConditionalHandleCreate(&gr->hnd[k], cg, 0u, cudaGraphCondAssignDefault),
                                "conditional handle")))
                return rc;
            cs_all.h[k - 1] = gr->hnd[k];
        }
        // the iterations' conditions start at 0 in every step (the graph may run the step in a loop)
        if (max_iter > 1) {
            graph_reset_conds_kernel<<<1, 64, 0, main_st>>>(cs_all, max_iter - 1);
            count_launches(1);
        }
    }
    // Host-driven: the tridiagonal step of iteration k runs on a side stream while the context's
    // stream goes on with v_{k+1} = w / |w| and, for short products, the product M v_{k+1} (discarded if
    // iteration k stopped); the norm partials alternate between two buffers so that the side stream's
    // reads never meet the next iteration's writes.
    if (!gr && !ctx->lz_side) {
        if ((rc = cuda_fail(cudaStreamCreateWithFlags(&ctx->lz_side, cudaStreamNonBlocking), "lanczos side stream")) ||
            (rc = cuda_fail(cudaEventCreateWithFlags(&ctx->lz_ev_a, cudaEventDisableTiming), "lanczos event")) ||
            (rc = cuda_fail(cudaEventCreateWithFlags(&ctx->lz_ev_t, cudaEventDisableTiming), "lanczos event")))
            return rc;
    }
    // Speculate only where a product is short: one product is wasted per solve (after the stopping
    // iteration) and about one tridiagonal step (~55 us) is saved per iteration; the estimate uses the
    // measured per-pair times of the one-way float64 and symmetric float32 kernels on this part.
    const double t_product = (ctx->Lx > 0.0 ? 9.0 : 1.0) * (double)N * (double)N *
                             (ctx->p.precision == RPB_FP64 ? 5e-10 : 1.3e-12);
    const bool speculate = t_product < 3e-4;
    bool have_product = false;  // w already holds M v_k (the speculative product of iteration k - 1)
    for (int k = 0; k < max_iter; ++k) {
        if (!gr) {
            const double *vk = V + (size_t)k * ld;
            double *rn = red + (size_t)(ctx->max_iter + 1 + (k & 1)) * G;
            rc = RPB_OK;
            if (!(k == 0 && first_done) && !have_product) rc = lanczos_product(ctx, N, pos, vk, w);
            have_product = false;
            if (rc) return rc;
            const int nv = k + 1;
            dots_kernel<<<dim3(G, nv), kBlasThreads, 0, main_st>>>(V, ld, n, w, red);
            project_out_kernel<<<G, kBlasThreads, 0, main_st>>>(V, ld, n, nv, red, G, w, lz + L.c1, nullptr);
            dots_kernel<<<dim3(G, nv), kBlasThreads, 0, main_st>>>(V, ld, n, w, red);
            project_out_kernel<<<G, kBlasThreads, 0, main_st>>>(V, ld, n, nv, red, G, w, lz + L.c2, rn);
            if ((rc = cuda_fail(cudaEventRecord(ctx->lz_ev_a, main_st), "event record")) ||
                (rc = cuda_fail(cudaStreamWaitEvent(ctx->lz_side, ctx->lz_ev_a, 0), "stream wait")))
                return rc;
            lanczos_tail_kernel<<<1, 32, 0, ctx->lz_side>>>(lz, L, k, tol, rn, G);
            count_launches(5);
            if ((rc = cuda_fail(cudaMemcpyAsync(hs, status, 8 * sizeof(double), cudaMemcpyDeviceToHost, ctx->lz_side),
                                "status copy")) ||
                (rc = cuda_fail(cudaEventRecord(ctx->lz_ev_t, ctx->lz_side), "event record")))
                return rc;
            if (k + 1 < max_iter) {  // v_{k+1} (unused if this iteration stops)
                scale_norm_kernel<<<G, kBlasThreads, 0, main_st>>>(w, n, rn, G, V + (size_t)(k + 1) * ld);
                count_launches(1);
                if (speculate) {
                    if ((rc = lanczos_product(ctx, N, pos, V + (size_t)(k + 1) * ld, w))) return rc;
                    have_product = true;
                }
            }
            if ((rc = cuda_fail(cudaEventSynchronize(ctx->lz_ev_t), "lanczos iteration"))) return rc;
            m = k + 1;
            eps = hs[ST_EPS];
            if (hs[ST_STOP] != 0.0) {
                stopped = true;
                break;
            }
            continue;
        }
        const bool cond = gr && k >= 1;
        if (cond) {
            if ((rc = graph_begin_if(main_st, gr->body, gr->hnd[k]))) return rc;
            ctx->stream = gr->body;
        }
        cudaStream_t st = ctx->stream;
        const uint64_t before = rpb_launch_count();
        const double *vk = V + (size_t)k * ld;
        // graph branch: iteration k's tridiagonal step beside v_{k+1} and its product M v_{k+1}, which
        // the body of iteration k + 1 then finds in w (discarded if iteration k stopped)
        cudaStream_t side = k == 0 ? gr->side0 : gr->side;
        const bool branch = speculate && gr->side0 != nullptr && gr->side != nullptr;
        rc = RPB_OK;
        if (!(k == 0 && first_done) && !(branch && k >= 1)) rc = lanczos_product(ctx, N, pos, vk, w);
        if (!rc) {
            const int nv = k + 1;
            dots_kernel<<<dim3(G, nv), kBlasThreads, 0, st>>>(V, ld, n, w, red);
            project_out_kernel<<<G, kBlasThreads, 0, st>>>(V, ld, n, nv, red, G, w, lz + L.c1, nullptr);
            dots_kernel<<<dim3(G, nv), kBlasThreads, 0, st>>>(V, ld, n, w, red);
            project_out_kernel<<<G, kBlasThreads, 0, st>>>(V, ld, n, nv, red, G, w, lz + L.c2, red_norm);
            count_launches(4);
            const bool has_next = k + 1 < max_iter;
            cudaStream_t tail_st = st;
            if (branch && has_next &&
                !(rc = cuda_fail(cudaEventRecord(gr->ev_fork, st), "event record")) &&
                !(rc = cuda_fail(cudaStreamWaitEvent(side, gr->ev_fork, 0), "stream wait")))
                tail_st = side;
            if (!rc) {
                lanczos_tail_kernel<<<1, 32, 0, tail_st>>>(lz, L, k, tol, red_norm, G,
                                                           has_next ? gr->hnd[k + 1] : 0ull, has_next ? 1 : 0,
                                                           gr->state->iter_runs + k, &gr->state->m);
                count_launches(1);
            }
            if (!rc && has_next) {  // v_{k+1} (unused when this iteration stopped)
                scale_norm_kernel<<<G, kBlasThreads, 0, st>>>(w, n, red_norm, G, V + (size_t)(k + 1) * ld);
                count_launches(1);
                if (tail_st != st) {
                    rc = lanczos_product(ctx, N, pos, V + (size_t)(k + 1) * ld, w);
                    const int jrc = cuda_fail(cudaEventRecord(gr->ev_join, side), "event record");
                    const int wrc = jrc ? jrc : cuda_fail(cudaStreamWaitEvent(st, gr->ev_join, 0), "stream wait");
                    if (!rc) rc = wrc;
                }
            }
            if (!rc) rc = cuda_fail(cudaGetLastError(), "lanczos kernels");
        }
        if (cond) {
            gr->iter_launches[k] = (int)(rpb_launch_count() - before);
            cudaGraph_t body_graph = nullptr;
            const int erc = cuda_fail(cudaStreamEndCapture(gr->body, &body_graph), "body capture end");
            ctx->stream = main_st;
            if (!rc) rc = erc;
        }
        if (rc) return rc;
        if (stopped) break;
    }
    // the combination reads y, which the side stream's tridiagonal step wrote
    if (!gr && (rc = cuda_fail(cudaStreamWaitEvent(main_st, ctx->lz_ev_t, 0), "stream wait"))) return rc;
    combine_kernel<<<G, kBlasThreads, 0, main_st>>>(V, ld, n, m, lz + L.y, g, gr ? &gr->state->m : nullptr);
    count_launches(1);
    if (ctx->precond && (rc = precond_scale(ctx, N, g, g, true))) return rc;  // g = D^{1/2} y
    if ((rc = cuda_fail(cudaGetLastError(), "lanczos kernels"))) return rc;
    if (gr) return RPB_OK;
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
