// api.cu -- the extern "C" entry points declared in include/rpb.h: argument checks, context and
// scratch management, and the sequence of the Adams-Bashforth step.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <new>

#include "rpb_internal.cuh"

namespace rpb {

static thread_local char g_err[512] = "";
static std::atomic<unsigned long long> g_launches{0};

void count_launches(int n)
{
    g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed);
}

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int cuda_fail(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return RPB_OK;
    set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    return RPB_ECUDA;
}

int fill_torque(rpb_ctx *ctx, int64_t N, const double *t, double *T);

static bool aligned8(const void *p)
{
    return ((uintptr_t)p & 7u) == 0;
}

static int check_ctx_N(rpb_ctx *ctx, int64_t N)
{
    if (!ctx) {
        set_error("null context");
        return RPB_EINVAL;
    }
    if (N <= 0 || N > ctx->max_N) {
        set_error("N=%lld outside [1, max_N=%lld]", (long long)N, (long long)ctx->max_N);
        return RPB_EINVAL;
    }
    return RPB_OK;
}

static int check_vec(const void *p, const char *name, bool nullable)
{
    if (!p) {
        if (nullable) return RPB_OK;
        set_error("%s is null", name);
        return RPB_EINVAL;
    }
    if (!aligned8(p)) {
        set_error("%s is not 8-byte aligned", name);
        return RPB_EINVAL;
    }
    return RPB_OK;
}

static void free_ws(Workspace &w)
{
    void *dev[] = {w.src, w.partial, w.V, w.w, w.red, w.lz, w.pos_a, w.pos_b, w.pos_w, w.cells,
                   w.vec_a, w.vec_b, w.vec_c, w.vec_d, w.vec_e, w.vec_f, w.vec_g,
                   w.sym_index, w.sym_tgt, w.sym_src, w.src2, w.pc, w.pcx};
    for (void *p : dev)
        if (p) cudaFree(p);
    if (w.host_status) cudaFreeHost(w.host_status);
    w = Workspace();
}

int check_step_args(rpb_ctx *ctx, int64_t N, const double *pos, const double *U_prev, int64_t step, double dt,
                    double delta, int max_iter, const rpb_force_params *fp, const rpb_step_options *opts)
{
    int rc;
    const int scheme = opts ? opts->scheme : RPB_SCHEME_AB;
    const int rfd = opts ? opts->rfd : RPB_RFD_CENTRED;
    if ((scheme != RPB_SCHEME_AB && scheme != RPB_SCHEME_EM) || (rfd != RPB_RFD_CENTRED && rfd != RPB_RFD_ONE_SIDED)) {
        set_error("bad step options (scheme=%d rfd=%d)", scheme, rfd);
        return RPB_EINVAL;
    }
    if ((rc = check_ctx_N(ctx, N)) || (rc = check_vec(pos, "pos", false)) || (rc = check_vec(U_prev, "U_prev", false)))
        return rc;
    if (!fp || !(fp->b > 0.0) || !(dt > 0.0) || !(delta > 0.0) || step < 0 || step > 0xffffffffLL) {
        set_error("bad step arguments (dt=%g delta=%g step=%lld)", dt, delta, (long long)step);
        return RPB_EINVAL;
    }
    if (max_iter < 1 || max_iter > ctx->max_iter) {
        set_error("max_iter=%d outside [1, %d]", max_iter, ctx->max_iter);
        return RPB_EINVAL;
    }
    if (U_prev == pos) {
        set_error("U_prev aliases pos");
        return RPB_EINVAL;
    }
    return RPB_OK;
}

// One time step (Eq. AB, or Eq. EM with scheme = RPB_SCHEME_EM), enqueued on ctx->stream.  gr == null:
// the Lanczos stop is read back per iteration and stats are written.  gr != null: the step is being
// captured into a graph (rpb_run): the step index and the first-step flag come from gr->state on the
// device, Lanczos iterations after the first are conditional nodes, and nothing is read back.
int step_impl(rpb_ctx *ctx, int64_t N, double *pos, double *U_prev, uint32_t step, uint64_t seed, double dt,
              double delta, double tol, int max_iter, const rpb_force_params *fp, int scheme, int rfd,
              rpb_step_stats *stats, LzGraph *gr)
{
    int rc;
    Workspace &w = ctx->ws;
    const unsigned int *d_step = gr ? &gr->state->step : nullptr;
    double *F = w.vec_a, *T = w.vec_b, *Un = w.vec_c, *W = w.vec_d, *Wt = w.vec_e, *g = w.vec_f, *drift = w.vec_g;
    if ((rc = forces_impl(ctx, N, pos, fp, F))) return rc;
    if ((rc = fill_torque(ctx, N, fp->torque, T))) return rc;
    int iters = 0, conv = 0;
    double err = -1.0;
    int lrc = RPB_OK;
    if (ctx->p.kT > 0.0) {
        if ((rc = philox_impl(ctx, N, seed, step, 0u, 0u, W, d_step))) return rc;
        if ((rc = philox_impl(ctx, N, seed, step, 1u, 0u, Wt, d_step))) return rc;
        if (mobility_apply2_ok(ctx, N)) {
            // the deterministic velocity and the first Lanczos product M v_0 share one pair pass
            // (with the preconditioner: M P v_0, scaled by P afterwards)
            bool zero = false;
            if ((rc = lanczos_precond_prepare(ctx, N, pos)) || (rc = lanczos_init(ctx, N, W, &zero, gr != nullptr)))
                return rc;
            if (zero) {
                if ((rc = mobility_apply_impl(ctx, N, pos, F, T, Un))) return rc;
                if ((rc = cuda_fail(cudaMemsetAsync(g, 0, 3 * N * sizeof(double), ctx->stream), "zero g")))
                    return rc;
                conv = 1;
            } else {
                if (ctx->precond) {
                    if ((rc = precond_scale(ctx, N, w.V, w.pcx, false)) ||
                        (rc = mobility_apply2_impl(ctx, N, pos, F, T, w.pcx, Un, w.w)) ||
                        (rc = precond_scale(ctx, N, w.w, w.w, false)))
                        return rc;
                } else if ((rc = mobility_apply2_impl(ctx, N, pos, F, T, w.V, Un, w.w))) {
                    return rc;
                }
                lrc = lanczos_run(ctx, N, pos, g, tol, max_iter, true, &iters, &err, &conv, gr);
            }
        } else {
            if ((rc = mobility_apply_impl(ctx, N, pos, F, T, Un))) return rc;
            lrc = lanczos_impl(ctx, N, pos, W, g, tol, max_iter, &iters, &err, &conv, gr);
        }
        if (lrc != RPB_OK && lrc != RPB_ENOCONV) return lrc;
        if ((rc = rfd_impl(ctx, N, pos, Wt, delta, drift, rfd == RPB_RFD_ONE_SIDED))) return rc;
    } else {
        if ((rc = mobility_apply_impl(ctx, N, pos, F, T, Un))) return rc;
        // kT = 0: no Brownian increment and no drift (both carry a factor kT); the deterministic
        // scheme needs neither the noise nor M^{1/2}
        if ((rc = cuda_fail(cudaMemsetAsync(g, 0, 3 * N * sizeof(double), ctx->stream), "clear g")) ||
            (rc = cuda_fail(cudaMemsetAsync(drift, 0, 3 * N * sizeof(double), ctx->stream), "clear drift")))
            return rc;
        err = 0.0;
        conv = 1;
    }
    const double noise = sqrt(2.0 * ctx->p.kT * dt);
    // Euler-Maruyama is the update with U^{n-1} := U^n (Eq. EM); AB uses that only on the first step
    const int em = scheme == RPB_SCHEME_EM || (!gr && step == 0);
    if ((rc = ab_update_impl(ctx, N, pos, U_prev, Un, g, drift, dt, noise, em, gr ? &gr->state->first : nullptr)))
        return rc;
    if (gr) return RPB_OK;
    if (stats) {
        stats->lanczos_iters = iters;
        stats->lanczos_err = err;
        stats->converged = conv;
    }
    if (lrc == RPB_ENOCONV) {
        set_error("lanczos: no convergence in %d iterations (eps=%g, tol=%g)", iters, err, tol);
        return RPB_ENOCONV;
    }
    return RPB_OK;
}

}  // namespace rpb

using namespace rpb;

extern "C" {

const char *rpb_last_error(void)
{
    return g_err;
}

uint64_t rpb_launch_count(void)
{
    return (uint64_t)g_launches.load(std::memory_order_relaxed);
}

int rpb_create(rpb_ctx **out, const rpb_params *p, int64_t max_N, int max_iter, void *stream)
{
    g_err[0] = 0;
    if (!out || !p) {
        set_error("null argument to rpb_create");
        return RPB_EINVAL;
    }
    *out = nullptr;
    if (!(p->a > 0.0) || !(p->eta > 0.0) || !(p->kT >= 0.0) || (p->precision != RPB_FP64 && p->precision != RPB_FP32) ||
        (p->wall != 0 && p->wall != 1)) {
        set_error("bad parameters (a=%g eta=%g kT=%g precision=%d wall=%d)", p->a, p->eta, p->kT, p->precision,
                  p->wall);
        return RPB_EINVAL;
    }
    if (max_N <= 0 || max_N > (int64_t)1 << 28) {
        set_error("max_N=%lld outside [1, 2^28]", (long long)max_N);
        return RPB_EINVAL;
    }
    if (max_iter < 1 || max_iter > 64) {
        set_error("max_iter=%d outside [1, 64]", max_iter);
        return RPB_EINVAL;
    }
    rpb_ctx *c = new (std::nothrow) rpb_ctx();
    if (!c) {
        set_error("host allocation failed");
        return RPB_ENOMEM;
    }
    c->p = *p;
    c->max_N = max_N;
    c->max_iter = max_iter;
    c->stream = (cudaStream_t)stream;
    {
        const char *v = getenv("RPB_FP32_PAIR");
        c->fp32_variant = (v && strcmp(v, "scalar") == 0) ? 0 : 1;
        const char *fu = getenv("RPB_FP32_SYM_FUSED");
        c->sym_fused = !(fu && strcmp(fu, "0") == 0);
    }
    int rc;
    if ((rc = cuda_fail(cudaGetDevice(&c->device), "cudaGetDevice")) ||
        (rc = cuda_fail(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device),
                        "cudaDeviceGetAttribute")) ||
        (rc = pair_occupancy(c))) {
        delete c;
        return rc;
    }
    Workspace &w = c->ws;
    const size_t n3 = (size_t)3 * max_N;
    const size_t vb = n3 * sizeof(double);
    w.partial_bytes = pair_partial_bytes(max_N, c->num_sms);
    w.red_elems = lanczos_red_elems(max_iter);
    struct {
        void **ptr;
        size_t bytes;
    } allocs[] = {
        {&w.src, (size_t)max_N * sizeof(SrcF64)},
        {&w.partial, w.partial_bytes},
        {(void **)&w.V, vb * (size_t)(max_iter + 1)},
        {(void **)&w.w, vb},
        {(void **)&w.red, w.red_elems * sizeof(double)},
        {(void **)&w.lz, lanczos_state_elems(max_iter) * sizeof(double)},
        {(void **)&w.pos_a, vb},
        {(void **)&w.pos_b, vb},
        {(void **)&w.pos_w, vb},
        {&w.cells, cell_lists_bytes(max_N)},
        {(void **)&w.vec_a, vb},
        {(void **)&w.vec_b, vb},
        {(void **)&w.vec_c, vb},
        {(void **)&w.vec_d, vb},
        {(void **)&w.vec_e, vb},
        {(void **)&w.vec_f, vb},
        {(void **)&w.vec_g, vb},
    };
    for (auto &a : allocs) {
        cudaError_t e = cudaMalloc(a.ptr, a.bytes);
        if (e != cudaSuccess) {
            set_error("cudaMalloc of %zu bytes failed: %s", a.bytes, cudaGetErrorString(e));
            cudaGetLastError();
            free_ws(w);
            delete c;
            return RPB_ENOMEM;
        }
    }
    {
        // the symmetric float32 translation-translation pass needs a triangle of column partials
        // (~N^2/128 * 12 bytes); used when that stays below 8 GB and RPB_FP32_SYM is not "0"
        const char *v = getenv("RPB_FP32_SYM");
        const size_t src_bytes = sym_src_part_bytes(max_N);
        c->sym_enabled = p->precision == RPB_FP32 && !(v && strcmp(v, "0") == 0) && max_N >= 2 * kTile &&
                         src_bytes <= ((size_t)8 << 30);
        // the two-right-hand-side pass (fused product and the first Lanczos product of a step) keeps
        // six components per partial: twice the scratch, used while that stays below 8 GB too;
        // RPB_FP32_SYM_RHS2=0 turns it off
        const char *v2 = getenv("RPB_FP32_SYM_RHS2");
        c->sym_rhs2 = c->sym_enabled && p->wall && !(v2 && strcmp(v2, "0") == 0) && 2 * src_bytes <= ((size_t)8 << 30);
        const size_t mult = c->sym_rhs2 ? 2 : 1;
        if (c->sym_enabled) {
            w.sym_index_ints = sym_index_ints(max_N, c->num_sms);
            w.sym_tgt_bytes = mult * sym_tgt_part_bytes(max_N, c->num_sms);
            w.sym_src_bytes = mult * src_bytes;
            if (cudaMalloc(&w.sym_index, 2 * w.sym_index_ints * sizeof(int)) != cudaSuccess ||
                cudaMalloc(&w.sym_tgt, w.sym_tgt_bytes) != cudaSuccess ||
                cudaMalloc(&w.sym_src, w.sym_src_bytes) != cudaSuccess ||
                (c->sym_rhs2 && cudaMalloc(&w.src2, (size_t)max_N * sizeof(float4)) != cudaSuccess)) {
                cudaGetLastError();
                set_error("cudaMalloc of the symmetric-pass scratch (%zu bytes) failed", src_bytes);
                free_ws(w);
                delete c;
                return RPB_ENOMEM;
            }
        }
    }
    if (cudaMallocHost((void **)&w.host_status, 8 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        set_error("pinned host allocation failed");
        free_ws(w);
        delete c;
        return RPB_ENOMEM;
    }
    if ((rc = cuda_fail(cudaMemsetAsync(w.lz, 0, lanczos_state_elems(max_iter) * sizeof(double), c->stream),
                        "memset"))) {
        free_ws(w);
        delete c;
        return rc;
    }
    *out = c;
    return RPB_OK;
}

int rpb_destroy(rpb_ctx *ctx)
{
    if (!ctx) return RPB_OK;
    g_err[0] = 0;
    int rc = cuda_fail(cudaStreamSynchronize(ctx->stream), "rpb_destroy sync");
    run_free(ctx);
    if (ctx->lz_side) cudaStreamSynchronize(ctx->lz_side);
    if (ctx->lz_ev_a) cudaEventDestroy(ctx->lz_ev_a);
    if (ctx->lz_ev_t) cudaEventDestroy(ctx->lz_ev_t);
    if (ctx->lz_side) cudaStreamDestroy(ctx->lz_side);
    free_ws(ctx->ws);
    delete ctx;
    return rc;
}

int rpb_set_stream(rpb_ctx *ctx, void *stream)
{
    if (!ctx) {
        set_error("null context");
        return RPB_EINVAL;
    }
    ctx->stream = (cudaStream_t)stream;
    return RPB_OK;
}

int rpb_set_periodic(rpb_ctx *ctx, double Lx, double Ly)
{
    g_err[0] = 0;
    if (!ctx) {
        set_error("null context");
        return RPB_EINVAL;
    }
    const bool off = Lx == 0.0 && Ly == 0.0;
    if (!off && !(Lx > 4.0 * ctx->p.a && Ly > 4.0 * ctx->p.a && std::isfinite(Lx) && std::isfinite(Ly))) {
        set_error("periods must both be 0 or both exceed 4a (Lx=%g Ly=%g)", Lx, Ly);
        return RPB_EINVAL;
    }
    ctx->Lx = off ? 0.0 : Lx;
    ctx->Ly = off ? 0.0 : Ly;
    return RPB_OK;
}

int rpb_set_preconditioner(rpb_ctx *ctx, int kind)
{
    g_err[0] = 0;
    if (!ctx) {
        set_error("null context");
        return RPB_EINVAL;
    }
    if (kind != RPB_PRECOND_NONE && kind != RPB_PRECOND_BLOCK_DIAGONAL) {
        set_error("unknown preconditioner %d", kind);
        return RPB_EINVAL;
    }
    Workspace &w = ctx->ws;
    if (kind != RPB_PRECOND_NONE && !w.pc) {
        const size_t vb = (size_t)3 * ctx->max_N * sizeof(double);
        if (cudaMalloc(&w.pc, vb) != cudaSuccess || cudaMalloc(&w.pcx, vb) != cudaSuccess) {
            cudaGetLastError();
            if (w.pc) cudaFree(w.pc);
            if (w.pcx) cudaFree(w.pcx);
            w.pc = w.pcx = nullptr;
            set_error("cudaMalloc of the preconditioner vectors (2 x %zu bytes) failed", vb);
            return RPB_ENOMEM;
        }
    }
    ctx->precond = kind;
    return RPB_OK;
}

int rpb_mobility_apply(rpb_ctx *ctx, int64_t N, const double *pos, const double *F, const double *T, double *U)
{
    g_err[0] = 0;
    int rc;
    if ((rc = check_ctx_N(ctx, N)) || (rc = check_vec(pos, "pos", false)) || (rc = check_vec(F, "F", true)) ||
        (rc = check_vec(T, "T", true)) || (rc = check_vec(U, "U", false)))
        return rc;
    if (U == pos || U == F || U == T) {
        set_error("U aliases an input");
        return RPB_EINVAL;
    }
    if (!F && !T) return cuda_fail(cudaMemsetAsync(U, 0, 3 * N * sizeof(double), ctx->stream), "memset U");
    return mobility_apply_impl(ctx, N, pos, F, T, U);
}

int rpb_mobility_apply_rows(rpb_ctx *ctx, int64_t N, const double *pos, const double *F, const double *T,
                            int64_t row0, int64_t row1, double *U_rows)
{
    g_err[0] = 0;
    int rc;
    if ((rc = check_ctx_N(ctx, N)) || (rc = check_vec(pos, "pos", false)) || (rc = check_vec(F, "F", true)) ||
        (rc = check_vec(T, "T", true)) || (rc = check_vec(U_rows, "U_rows", false)))
        return rc;
    if (row0 < 0 || row1 <= row0 || row1 > N || row0 % kTile != 0) {
        set_error("rows [%lld, %lld) not within [0, N=%lld) with the first a multiple of %d", (long long)row0,
                  (long long)row1, (long long)N, kTile);
        return RPB_EINVAL;
    }
    if (ctx->Lx > 0.0 || (ctx->p.precision == RPB_FP32 && !ctx->p.wall)) {
        set_error("row products are not offered with pseudo-periodic boundaries or float32 without the wall");
        return RPB_EINVAL;
    }
    if (U_rows == pos || U_rows == F || U_rows == T) {
        set_error("U_rows aliases an input");
        return RPB_EINVAL;
    }
    if (!F && !T)
        return cuda_fail(cudaMemsetAsync(U_rows, 0, 3 * (row1 - row0) * sizeof(double), ctx->stream), "memset U");
    return mobility_rows_impl(ctx, N, pos, F, T, row0, row1, U_rows);
}

int rpb_mobility_apply_part(rpb_ctx *ctx, int64_t N, const double *pos, const double *F, const double *T, int part,
                            int nparts, double *U)
{
    g_err[0] = 0;
    int rc;
    if ((rc = check_ctx_N(ctx, N)) || (rc = check_vec(pos, "pos", false)) || (rc = check_vec(F, "F", true)) ||
        (rc = check_vec(T, "T", true)) || (rc = check_vec(U, "U", false)))
        return rc;
    if (nparts < 1 || nparts > 4096 || part < 0 || part >= nparts) {
        set_error("share %d of %d: need 0 <= part < nparts <= 4096", part, nparts);
        return RPB_EINVAL;
    }
    if (U == pos || U == F || U == T) {
        set_error("U aliases an input");
        return RPB_EINVAL;
    }
    if (!F && !T) return cuda_fail(cudaMemsetAsync(U, 0, 3 * N * sizeof(double), ctx->stream), "memset U");
    return mobility_part_impl(ctx, N, pos, F, T, part, nparts, U);
}

int rpb_set_product_hook(rpb_ctx *ctx, rpb_product_hook hook, void *user)
{
    g_err[0] = 0;
    if (!ctx) {
        set_error("null context");
        return RPB_EINVAL;
    }
    ctx->hook = hook;
    ctx->hook_user = hook ? user : nullptr;
    return RPB_OK;
}

int rpb_mobility_apply2(rpb_ctx *ctx, int64_t N, const double *pos, const double *F, const double *T,
                        const double *P, double *U, double *U2)
{
    g_err[0] = 0;
    int rc;
    if ((rc = check_ctx_N(ctx, N)) || (rc = check_vec(pos, "pos", false)) || (rc = check_vec(F, "F", false)) ||
        (rc = check_vec(T, "T", true)) || (rc = check_vec(P, "P", false)) || (rc = check_vec(U, "U", false)) ||
        (rc = check_vec(U2, "U2", false)))
        return rc;
    const double *outs[] = {U, U2};
    for (const double *o : outs)
        if (o == pos || o == F || o == T || o == P) {
            set_error("an output aliases an input");
            return RPB_EINVAL;
        }
    if (U == U2) {
        set_error("U and U2 are the same buffer");
        return RPB_EINVAL;
    }
    if (T && mobility_apply2_ok(ctx, N)) return mobility_apply2_impl(ctx, N, pos, F, T, P, U, U2);
    if ((rc = mobility_apply_impl(ctx, N, pos, F, T, U))) return rc;
    return mobility_apply_impl(ctx, N, pos, P, nullptr, U2);
}

int rpb_lanczos_sqrt_apply(rpb_ctx *ctx, int64_t N, const double *pos, const double *W, double *g, double tol,
                           int max_iter, int *iters_out, double *err_out)
{
    g_err[0] = 0;
    int rc;
    if ((rc = check_ctx_N(ctx, N)) || (rc = check_vec(pos, "pos", false)) || (rc = check_vec(W, "W", false)) ||
        (rc = check_vec(g, "g", false)))
        return rc;
    if (max_iter < 1 || max_iter > ctx->max_iter) {
        set_error("max_iter=%d outside [1, %d]", max_iter, ctx->max_iter);
        return RPB_EINVAL;
    }
    if (g == W || g == pos) {
        set_error("g aliases an input");
        return RPB_EINVAL;
    }
    return lanczos_impl(ctx, N, pos, W, g, tol, max_iter, iters_out, err_out, nullptr);
}

int rpb_rfd_drift(rpb_ctx *ctx, int64_t N, const double *pos, const double *Wt, double delta, double *drift)
{
    g_err[0] = 0;
    int rc;
    if ((rc = check_ctx_N(ctx, N)) || (rc = check_vec(pos, "pos", false)) || (rc = check_vec(Wt, "Wt", false)) ||
        (rc = check_vec(drift, "drift", false)))
        return rc;
    if (!(delta > 0.0)) {
        set_error("delta must be > 0");
        return RPB_EINVAL;
    }
    if (drift == Wt || drift == pos) {
        set_error("drift aliases an input");
        return RPB_EINVAL;
    }
    return rfd_impl(ctx, N, pos, Wt, delta, drift);
}

int rpb_forces(rpb_ctx *ctx, int64_t N, const double *pos, const rpb_force_params *fp, double *F)
{
    g_err[0] = 0;
    int rc;
    if ((rc = check_ctx_N(ctx, N)) || (rc = check_vec(pos, "pos", false)) || (rc = check_vec(F, "F", false)))
        return rc;
    if (!fp || !(fp->b > 0.0)) {
        set_error("force parameters missing or b <= 0");
        return RPB_EINVAL;
    }
    if (F == pos) {
        set_error("F aliases pos");
        return RPB_EINVAL;
    }
    return forces_impl(ctx, N, pos, fp, F);
}

int rpb_philox_normal(rpb_ctx *ctx, int64_t N, uint64_t seed, uint32_t step, uint32_t stream_id, uint32_t instance,
                      double *out)
{
    g_err[0] = 0;
    int rc;
    if ((rc = check_ctx_N(ctx, N)) || (rc = check_vec(out, "out", false))) return rc;
    return philox_impl(ctx, N, seed, step, stream_id, instance, out);
}

int rpb_ab_step(rpb_ctx *ctx, int64_t N, double *pos, double *U_prev, int64_t step, uint64_t seed, double dt,
                double delta, double tol, int max_iter, const rpb_force_params *fp, rpb_step_stats *stats)
{
    return rpb_step(ctx, N, pos, U_prev, step, seed, dt, delta, tol, max_iter, fp, nullptr, stats);
}

int rpb_step(rpb_ctx *ctx, int64_t N, double *pos, double *U_prev, int64_t step, uint64_t seed, double dt,
             double delta, double tol, int max_iter, const rpb_force_params *fp, const rpb_step_options *opts,
             rpb_step_stats *stats)
{
    g_err[0] = 0;
    int rc;
    if ((rc = check_step_args(ctx, N, pos, U_prev, step, dt, delta, max_iter, fp, opts))) return rc;
    return step_impl(ctx, N, pos, U_prev, (uint32_t)step, seed, dt, delta, tol, max_iter, fp,
                     opts ? opts->scheme : RPB_SCHEME_AB, opts ? opts->rfd : RPB_RFD_CENTRED, stats, nullptr);
}

}  // extern "C"
