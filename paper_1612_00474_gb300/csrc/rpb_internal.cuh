// rpb_internal.cuh -- shared declarations of the CUDA translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/rpb.h"

namespace rpb {

constexpr int kTile = 128;        // sources staged per shared-memory tile = targets per block
constexpr int kPairThreads = 128; // threads per pair-kernel block (one target each)
constexpr double kPi = 3.14159265358979323846;

// Packed source records, built once per product from the float64 SoA inputs.
// s_j = H0(z_j / a) is folded into F and T; z is the clamped height max(z, a) (Appendix A).
struct alignas(16) SrcF32 {
    float4 p;  // x_hi, y_hi, x_lo, y_lo   (x = x_hi + x_lo exactly to ~2^-48 relative)
    float4 f;  // z~, s Fx, s Fy, s Fz
    float4 t;  // s Tx, s Ty, s Tz, 0
};
struct alignas(16) SrcF64 {
    double2 p;  // x, y
    double2 q;  // z~, s Fx
    double2 r;  // s Fy, s Fz
    double2 s;  // s Tx, s Ty
    double2 u;  // s Tz, 0
};

// Geometry constants of the pair formula, in units where velocities carry 1/(8 pi eta).
template <typename R>
struct PairConsts {
    R two_a;        // 2a
    R two_a2;       // 2a^2
    R two_3_a2;     // 2a^2/3
    R a2;           // a^2
    R near_c1;      // 4/(3a)          (mu0 in units of 1/(8 pi eta))
    R near_r;       // 9/(32a)
    R near_c2;      // 1/(8 a^2)
    R near_tr;      // 1/(2 a^3)
    R near_tr_r;    // 3/(8a)
    R four_a2;      // 4a^2 (overlap test on r^2)
};

template <typename R>
inline PairConsts<R> make_consts(double a)
{
    PairConsts<R> c;
    c.two_a = (R)(2.0 * a);
    c.two_a2 = (R)(2.0 * a * a);
    c.two_3_a2 = (R)(2.0 * a * a / 3.0);
    c.a2 = (R)(a * a);
    c.near_c1 = (R)(4.0 / (3.0 * a));
    c.near_r = (R)(9.0 / (32.0 * a));
    c.near_c2 = (R)(1.0 / (8.0 * a * a));
    c.near_tr = (R)(1.0 / (2.0 * a * a * a));
    c.near_tr_r = (R)(3.0 / (8.0 * a));
    c.four_a2 = (R)(4.0 * a * a);
    return c;
}

// Pair forces beyond 2a + kForceCutoffB b are left out: there the soft repulsion is below
// e^{-40} U0/b ~ 4e-18 U0/b, far under the float64 rounding of any force it would be added to.
constexpr double kForceCutoffB = 40.0;

// Cell lists of the force pass (pair.cu): header, then int arrays in one allocation.
constexpr int kCellGrid = 256;                  // at most kCellGrid x kCellGrid buckets (cells hashed modulo G)
constexpr int kCells = kCellGrid * kCellGrid;
constexpr int kCellMaxSorted = 512;             // a fuller cell hands the force pass to the all-pairs kernel
struct CellHeader {
    int overfull, pad[15];  // 64 bytes, followed by the bucket counts
};
__device__ __forceinline__ bool cell_overfull(const CellHeader *h)
{
    return *(volatile const int *)&h->overfull != 0;
}
struct CellLists {
    CellHeader *hdr;
    int *count, *start, *fill, *cellof, *idx;
    float4 *posf;  // float32 copies (x, y, z, index bits) in bucket order
};
// count, start and fill hold kCells + 1 entries each and are read and written as int4, so each array
// starts on a 16-byte boundary: stride kCellStride (a multiple of 4 ints) after a 64-byte header, in
// an allocation that cudaMalloc aligns to 256 bytes.
constexpr int kCellStride = kCells + 4;
static_assert(kCellStride % 4 == 0 && kCellStride >= kCells + 1, "bucket array stride");
inline size_t cell_lists_bytes(int64_t max_N)
{
    return 64 + sizeof(int) * (size_t)3 * kCellStride + sizeof(float4) * (size_t)max_N +
           sizeof(int) * (size_t)2 * max_N;
}
inline CellLists cell_lists(void *base, int64_t max_N)
{
    CellLists L;
    char *p = (char *)base;
    L.hdr = (CellHeader *)p;
    int *q = (int *)(p + 64);
    L.count = q;
    L.start = q + kCellStride;
    L.fill = q + 2 * kCellStride;
    L.posf = (float4 *)(q + 3 * kCellStride);  // 64 + 12 kCellStride bytes: 16-byte aligned
    L.cellof = (int *)(L.posf + max_N);
    L.idx = L.cellof + max_N;
    return L;
}

// One suspension of a batch in the symmetric pass: its first sphere in the packed layout, its size and
// its first tile in the batch's tile numbering.
struct SymInst {
    long long off;
    int N;
    int tile0;
};

// Symmetric pass over a batch of suspensions (float32): schedule and scratch, built by
// batch_sym_plan and owned by the batch context.
struct BatchSymPlan {
    int *index = nullptr;         // device: CTA table, segment table, row_seg, col_start, tile_inst
    size_t index_cap = 0;         // ints
    SymInst *sinst = nullptr;     // device, one per suspension
    int sinst_cap = 0;
    double *tgt = nullptr;        // segment partials, 3 x 128 doubles each
    size_t tgt_cap = 0;           // bytes
    float *srcp = nullptr;        // column partials, 3 x 128 floats each
    size_t src_cap = 0;           // bytes
    int ncta = 0, nseg = 0, ntiles = 0, seg_off = 0, row_off = 0, col_off = 0, inst_off = 0;
    bool valid = false;
    std::vector<int64_t> sizes;   // the suspension sizes the plan was built for
    int seg_tiles = 0;            // ... and the run length of its row cut
    int tt_minb = 5;              // resident CTAs per SM of the translation-translation kernel (4 or 5)
};

// A schedule of the symmetric pass on the device (sym_schedule_range): the CTA table and segment table
// (4 ints each), row_seg, col_start and col_rows at the given offsets of `index`, for share `part` of
// `nparts` equal shares of the triangle of N spheres.
struct SymSched {
    int *index = nullptr;
    int N = -1, part = 0, nparts = 1;
    int ncta = 0, nseg = 0, seg_off = 0, row_off = 0, col_off = 0, rows_off = 0;
};

// Scratch owned by a context.
struct Workspace {
    void *src = nullptr;          // packed sources, max_N records (SrcF64 size)
    void *partial = nullptr;      // pair-kernel partial sums
    size_t partial_bytes = 0;
    double *V = nullptr;          // Lanczos basis, (max_iter + 1) x 3 max_N
    double *w = nullptr;          // Lanczos work vector, 3 max_N
    double *red = nullptr;        // reduction partials
    size_t red_elems = 0;
    double *lz = nullptr;         // Lanczos small state (alpha, beta, y, y_prev, coefficients, status)
    double *pos_a = nullptr;      // displaced positions (RFD), 3 max_N
    double *pos_b = nullptr;
    double *pos_w = nullptr;      // positions folded into the unit cell (pseudo-periodic mode), 3 max_N
    void *cells = nullptr;        // cell lists of the force pass (cell_lists_bytes)
    double *vec_a = nullptr;      // 3 max_N scratch vectors for the AB step
    double *vec_b = nullptr;
    double *vec_c = nullptr;
    double *vec_d = nullptr;
    double *vec_e = nullptr;
    double *vec_f = nullptr;
    double *vec_g = nullptr;
    double *host_status = nullptr; // pinned host copy of the Lanczos status word
    double *pc = nullptr;          // block-diagonal preconditioner D^{-1/2} (3 max_N), rpb_set_preconditioner
    double *pcx = nullptr;         // a Krylov vector scaled by it
    // symmetric translation-translation pass (float32 contexts): schedules, row and column partials
    int *sym_index = nullptr;      // room for two schedules of sym_index_ints each (sym.index, sym_part.index)
    size_t sym_index_ints = 0;
    double *sym_tgt = nullptr;
    size_t sym_tgt_bytes = 0;
    float *sym_src = nullptr;
    size_t sym_src_bytes = 0;
    void *src2 = nullptr;          // second right-hand side of the two-RHS symmetric pass (float4 per sphere)
    SymSched sym;       // the whole triangle
    SymSched sym_part;  // one share of it (rpb_mobility_apply_part)
};

constexpr int kRunMaxIter = 64;  // = kMaxIter of the Lanczos state

// Device state of a graph-replayed run (rpb_run): the step index the noise is drawn with, whether the
// coming step is a first (Euler-Maruyama) step, the Lanczos dimension m of the latest step, and counters
// of the instance-steps that did not converge and of the runs of each Lanczos iteration.
struct RunState {
    unsigned int step;
    int first;
    int m;
    int left;  // steps left in the run
    unsigned long long unconv;
    unsigned long long iter_runs[kRunMaxIter];
};
struct RunCtx;  // run.cu

// Capture of the Lanczos iterations into a CUDA graph (rpb_run): iteration k >= 1 is the body of a
// conditional node hnd[k], captured on `body`; the last kernel of iteration k - 1 sets its condition on
// the device from the stopping test, and records m in state.
struct LzGraph {
    cudaStream_t body = nullptr;
    RunState *state = nullptr;
    // a second branch inside an iteration: the tridiagonal step beside the next iteration's product
    // (short products only; null: no branch).  A stream joined into a capture stays in it until the
    // capture ends, so the first iteration (captured with the step) and the conditional bodies (each
    // a capture of its own) fork onto different streams: side0 and side.
    cudaStream_t side0 = nullptr, side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaGraphConditionalHandle hnd[kRunMaxIter] = {};
    int iter_launches[kRunMaxIter] = {};  // kernels captured into iteration k's body
};

}  // namespace rpb

struct rpb_ctx {
    rpb_params p;
    int64_t max_N;
    int max_iter;
    cudaStream_t stream;
    int device;
    int num_sms;
    int fp32_variant;  // float32 pair kernel: 1 = packed float32x2 (default), 0 = scalar; env RPB_FP32_PAIR
    int sym_enabled;   // float32 translation-translation products use the symmetric pass; env RPB_FP32_SYM=0 off
    int sym_fused;     // products with torques also use the symmetric pass; env RPB_FP32_SYM_FUSED=0 off
    int sym_rhs2;      // a step's fused product and first Lanczos product share one pass; env RPB_FP32_SYM_RHS2=0 off
    double Lx = 0.0, Ly = 0.0;  // pseudo-periodic periods (0: unbounded in-plane), rpb_set_periodic
    int precond = 0;            // Lanczos preconditioner (RPB_PRECOND_*), rpb_set_preconditioner
    int f32_slots[2] = {0, 0};  // resident CTAs of the float32 one-way pair kernels (tt, with torques)
    rpb::Workspace ws;
    rpb::RunCtx *run = nullptr; // streams and device state of graph-replayed runs (rpb_run), made on first use
    rpb_product_hook hook = nullptr;  // products delegated to the caller (rpb_set_product_hook)
    void *hook_user = nullptr;
    int in_hook = 0;                  // inside the hook: products are computed here
    // host-driven Lanczos: the side stream its tridiagonal steps run on, and its two events
    cudaStream_t lz_side = nullptr;
    cudaEvent_t lz_ev_a = nullptr, lz_ev_t = nullptr;
};

namespace rpb {

// Error reporting (thread-local message).
void set_error(const char *fmt, ...);
// Count kernel launches enqueued by the library (reported by rpb_launch_count).
void count_launches(int n);
int cuda_fail(cudaError_t e, const char *what);

// Pair product: U = M_tt F + M_tr T with the context's precision.  F or T may be null.
// All pointers device, SoA float64.  Enqueued on ctx->stream.
int mobility_apply_impl(rpb_ctx *ctx, int64_t N, const double *pos, const double *F, const double *T,
                        double *U);
// Rows t0 .. t1 - 1 of the product (component stride ldu, ldu < 0: t1 - t0), one-way kernels over a
// target range.
int mobility_rows_impl(rpb_ctx *ctx, int64_t N, const double *pos, const double *F, const double *T, int64_t t0,
                       int64_t t1, double *U_rows, int64_t ldu = -1);
// Share `part` of `nparts` of the product (rpb_mobility_apply_part); never goes through the product hook.
int mobility_part_impl(rpb_ctx *ctx, int64_t N, const double *pos, const double *F, const double *T, int part,
                       int nparts, double *U);
// Whether mobility_apply2_impl can take this product (float32 symmetric pass with two right-hand sides).
bool mobility_apply2_ok(const rpb_ctx *ctx, int64_t N);
// U = M_tt F + M_tr T and U2 = M_tt P in one symmetric pass (F, T, P non-null).
int mobility_apply2_impl(rpb_ctx *ctx, int64_t N, const double *pos, const double *F, const double *T,
                         const double *P, double *U, double *U2);

// Packed source records from float64 SoA inputs (pair.cu); also used by the batched path.
__global__ void pack_f32_kernel(const double *__restrict__ pos, const double *__restrict__ F,
                                const double *__restrict__ T, int N, double a, int wall, SrcF32 *__restrict__ out);
__global__ void pack_f64_kernel(const double *__restrict__ pos, const double *__restrict__ F,
                                const double *__restrict__ T, int N, double a, int wall, SrcF64 *__restrict__ out);

// Number of column splits and chunk length the pair kernel uses for N targets.
// slots: resident CTAs of the float32 kernel over the GPU (0: unknown, fixed rule).
void pair_grid(int64_t N, int num_sms, int precision, int slots, int *splits, int64_t *chunk);
int pair_occupancy(rpb_ctx *ctx);
size_t pair_partial_bytes(int64_t max_N, int num_sms);
size_t sym_src_part_bytes(int64_t max_N);
size_t sym_tgt_part_bytes(int64_t max_N, int num_sms);
size_t sym_index_ints(int64_t max_N, int num_sms);

int forces_impl(rpb_ctx *ctx, int64_t N, const double *pos, const rpb_force_params *fp, double *F);

// Build (or keep, when the sizes are unchanged) the batched symmetric plan for B suspensions of sizes N
// packed one after another; grows the plan's scratch (not inside a stream capture).  Returns RPB_OK,
// or an error; *ok is false when the plan would need more than the scratch limit (the caller then uses
// the one-way kernels).
// seg_tiles: the run length of every suspension's row cut (the results depend on it, not on the
// companions).
int batch_sym_plan(BatchSymPlan &pl, int B, const int64_t *N, cudaStream_t st, bool *ok, int seg_tiles);
void batch_sym_free(BatchSymPlan &pl);
// U_b = M_tt F_b (+ M_tr T_b) for every suspension of the plan, from packed float32 sources; active
// masks suspensions (null: all).
int batch_sym_apply(const BatchSymPlan &pl, cudaStream_t st, const SrcF32 *src, int64_t total, const double *pos,
                    const double *F, const double *T, double *U, const int *active, double a, double eta);
// d_step (optional): a device word to read the step index from instead of `step` (graph replays).
int philox_impl(rpb_ctx *ctx, int64_t N, uint64_t seed, uint32_t step, uint32_t stream_id, uint32_t instance,
                double *out, const unsigned int *d_step = nullptr);
// Open a conditional (IF) node after the work captured so far on `st` and start capturing its body on
// `body`; the node runs its body when `h` was set non-zero during this launch of the graph.
int graph_begin_if(cudaStream_t st, cudaStream_t body, cudaGraphConditionalHandle h);
int graph_begin_cond(cudaStream_t st, cudaStream_t body, cudaGraphConditionalHandle h,
                     cudaGraphConditionalNodeType type);
// Adds a WHILE node (its handle created with the default value 1) after the capture dependencies of
// st and begins capturing its body on `body`; the body ends with graph_loop_tail_kernel.
int graph_begin_loop(cudaStream_t st, cudaStream_t body, cudaGraphConditionalHandle *h);
// The conditions of a set of conditional nodes, all set to 0 by graph_reset_conds_kernel: a condition
// keeps its value from one pass of a loop body to the next (the default is applied only when the
// graph is launched), so a body that decides its conditional nodes as it goes clears them first.
struct CondSet {
    cudaGraphConditionalHandle h[kRunMaxIter];
};
__global__ void graph_reset_conds_kernel(CondSet s, int n);
// *left = n (before the loop's graph is launched)
__global__ void graph_loop_init_kernel(int *left, int n);
// End of one pass of a loop body: --*left, and the loop runs again while *left > 0.
__global__ void graph_loop_tail_kernel(int *left, cudaGraphConditionalHandle h);
// Host-side preparation a product at this N needs (the symmetric pass's schedule), done before a
// stream capture so that the captured products find it in place.
int pair_prepare(rpb_ctx *ctx, int64_t N);
int lanczos_impl(rpb_ctx *ctx, int64_t N, const double *pos, const double *W, double *g, double tol, int max_iter,
                 int *iters_out, double *err_out, int *converged_out, LzGraph *gr = nullptr);
// The two halves of lanczos_impl: |W| and v_0 = W/|W| into ws.V (synchronises; *nw_zero when W = 0),
// then the iterations; with first_done the first product M v_0 is already in ws.w (with the
// preconditioner on: P M P v_0, see lanczos_precond_prepare).
// graph: inside a stream capture; nothing is read back (*nw_zero false: the noise W of a step is never 0).
int lanczos_init(rpb_ctx *ctx, int64_t N, const double *W, bool *nw_zero, bool graph = false);
// With ctx->precond set: P = D^{-1/2} at these positions into ws.pc (D: diagonal of the self blocks),
// so that the iteration runs on P M P and returns g = D^{1/2} y.  precond_scale: out = x * P
// elementwise (inverse: x / P, 0 where P = 0).
int lanczos_precond_prepare(rpb_ctx *ctx, int64_t N, const double *pos);
int precond_scale(rpb_ctx *ctx, int64_t N, const double *x, double *out, bool inverse);
// gr: inside a stream capture, the iterations after the first in conditional nodes (see LzGraph); the
// host outputs are then not written.
int lanczos_run(rpb_ctx *ctx, int64_t N, const double *pos, double *g, double tol, int max_iter, bool first_done,
                int *iters_out, double *err_out, int *converged_out, LzGraph *gr = nullptr);
int rfd_impl(rpb_ctx *ctx, int64_t N, const double *pos, const double *Wt, double delta, double *drift,
             int one_sided = 0);
// d_first (optional): a device word that, when non-zero, makes the update a first step (graph replays).
int ab_update_impl(rpb_ctx *ctx, int64_t N, double *pos, double *U_prev, const double *Un, const double *g,
                   const double *drift, double dt, double noise_scale, int first, const int *d_first = nullptr);

// Arguments of a time step (rpb_step, rpb_run), and the step itself (api.cu; see there).
int check_step_args(rpb_ctx *ctx, int64_t N, const double *pos, const double *U_prev, int64_t step, double dt,
                    double delta, int max_iter, const rpb_force_params *fp, const rpb_step_options *opts);
int step_impl(rpb_ctx *ctx, int64_t N, double *pos, double *U_prev, uint32_t step, uint64_t seed, double dt,
              double delta, double tol, int max_iter, const rpb_force_params *fp, int scheme, int rfd,
              rpb_step_stats *stats, LzGraph *gr);
// Streams and device state of graph-replayed runs (run.cu), released by rpb_destroy.
void run_free(rpb_ctx *ctx);

// Sizes of the Lanczos small-state block (doubles) for max_iter.
size_t lanczos_state_elems(int max_iter);
size_t lanczos_red_elems(int max_iter);

}  // namespace rpb
