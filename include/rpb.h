/*
 * rpb.h -- C ABI of the GB300 (sm_103a) Rotne-Prager-Blake Brownian-dynamics library.
 *
 * The library computes the hot path of Brownian dynamics of spheres (radius a) above a
 * no-slip wall at z = 0 (Balboa Usabiaga, Delmotte & Donev, "Brownian dynamics of confined
 * suspensions of active microrollers", 2017):
 *   - the matrix-free product U = M_tt F + M_tr T with the wall-corrected Rotne-Prager-
 *     Yamakawa (Rotne-Prager-Blake) mobility, regularised for wall overlaps (Sec. II.B,
 *     Sec. III, Appendix A);
 *   - the Lanczos approximation g_m ~ M^{1/2} W (Sec. II.C);
 *   - the random-finite-difference drift (Sec. II.A);
 *   - one stochastic Adams-Bashforth step (Eq. AB) with gravity, soft steric forces and a
 *     constant torque (Sec. III).
 *
 * Conventions for every entry point
 *   - All vector arguments are DEVICE pointers to float64 arrays in structure-of-arrays layout
 *     of length 3N: [x_0 .. x_{N-1} | y_0 .. y_{N-1} | z_0 .. z_{N-1}].  Base addresses must be
 *     8-byte aligned.  The caller owns every input and output buffer; the library never frees
 *     them.  Output buffers must not alias inputs unless stated.
 *   - A context owns its scratch memory (allocated once in rpb_create for up to max_N
 *     particles) and a CUDA stream (the caller's; the library never creates or destroys one).
 *     Calls are stream-ordered: they enqueue work on the context's stream and may return before
 *     the results exist, except where a result is returned through a host pointer (iteration
 *     counts, errors, statistics): those calls synchronise the stream before returning.
 *     A context must not be used from two host threads at once.
 *   - Return value: RPB_OK (0) or one of the error codes below; no exception crosses the ABI.
 *     rpb_last_error() gives a message for the calling thread's most recent failure.
 *   - Noise: the Philox counter index of a Gaussian is the particle-major index k = 3 i + c
 *     (the paper orders q = {q_1 .. q_N}, Sec. II), independent of the SoA layout above.
 */
#ifndef RPB_H
#define RPB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RPB_OK 0
#define RPB_EINVAL 1    /* null pointer, N <= 0 or N > max_N, bad parameter, misaligned pointer */
#define RPB_ENOMEM 2    /* device allocation failed in rpb_create */
#define RPB_ECUDA 3     /* a CUDA runtime call or kernel launch failed (message has the CUDA error) */
#define RPB_ENOCONV 4   /* Lanczos reached max_iter with eps > tol: results are still written */
#define RPB_ETIMEOUT 5  /* a bounded device-side wait expired.  Reserved: no kernel of this library waits
                           on another (the Lanczos stop and the step loop are graph conditions, the
                           stages plain stream order), so no call returns it */

#define RPB_FP64 0      /* pair arithmetic in float64 */
#define RPB_FP32 1      /* pair arithmetic in float32 (hi/lo split positions, compensated tile sums,
                           float64 self terms and cross-chunk sums); Lanczos always float64 */

typedef struct rpb_ctx rpb_ctx;

/* Physical and numerical parameters of a context. */
typedef struct {
    double a;        /* sphere radius (> 0) */
    double eta;      /* viscosity (> 0) */
    double kT;       /* thermal energy (>= 0) */
    int precision;   /* RPB_FP64 or RPB_FP32 */
    int wall;        /* 1: wall-corrected mobility with the regularisation of Appendix A (the method);
                        0: unbounded-domain RPY mobility (no image terms, no clamp, H0 = 1), for the
                        comparison of Sec. II.C without the wall's screening.  Batch contexts and
                        rpb_mobility_apply_noalloc accept only 1. */
} rpb_params;

/* Deterministic forcing of Sec. III: gravity -weight z_hat on every sphere, the soft steric
 * potential of Eq. (soft_potential) between spheres (d = 2a, centre distance) and with the wall
 * (d = a, height), and the same torque on every sphere. */
typedef struct {
    double weight;     /* buoyant weight m g (force along -z) */
    double U0;         /* steric energy scale */
    double b;          /* steric range (> 0) */
    double torque[3];  /* constant torque on every sphere */
} rpb_force_params;

/* Statistics of one Adams-Bashforth step (valid when rpb_ab_step returns). */
typedef struct {
    int lanczos_iters;    /* m: matvecs used for M^{1/2} W */
    double lanczos_err;   /* eps_m, the paper's relative-difference estimate (-1 if m < 2) */
    int converged;        /* 1 if eps_m <= tol or the Krylov space became invariant */
} rpb_step_stats;

/* Create a context for up to max_N spheres and Lanczos runs of up to max_iter iterations.
 * stream: a cudaStream_t (NULL = legacy default stream).  The device is the current one.
 * Allocates all scratch now (about (max_iter + 12) * 24 * max_N bytes plus partial-sum
 * buffers); returns RPB_ENOMEM if that fails.  *ctx is NULL on failure. */
int rpb_create(rpb_ctx **ctx, const rpb_params *p, int64_t max_N, int max_iter, void *stream);

/* Free the context's scratch (after synchronising its stream).  NULL is accepted. */
int rpb_destroy(rpb_ctx *ctx);

/* Change the stream later calls enqueue on. */
int rpb_set_stream(rpb_ctx *ctx, void *stream);

/* Pseudo-periodic boundaries parallel to the wall (Appendix B): periods Lx, Ly (> 4a), or both 0 to
 * switch them off (the default).  When on, forces use the minimum image convention and the products
 * sum every source's minimum image and its eight shifts by one period (the unit cell and its eight
 * neighbour cells), i.e. nine times the pair work: float32 products with forces at N >= 256 in the
 * symmetric kernel (each pair's nine images evaluated once for both directions), the others (float64,
 * smaller N, torque-only products) in one-way kernels; positions may lie outside the cell (they are
 * folded in for the computation, and returned unfolded). */
int rpb_set_periodic(rpb_ctx *ctx, double Lx, double Ly);

/* Preconditioner of the Lanczos square root (Sec. II.C reports trying a block-diagonal one; the
 * paper's own runs use none, which is the default).  RPB_PRECOND_BLOCK_DIAGONAL: with D the diagonal
 * of the particles' translation self blocks (each particle's mobility including its interaction
 * with the wall, none between particles; the block is diagonal, and 0 for a sphere on or below the
 * wall), rpb_lanczos_sqrt_apply and the Brownian part of rpb_ab_step / rpb_step run the iteration on
 * P M P with P = D^{-1/2} (0 where D = 0) and return g = D^{1/2} y: a sample with covariance M, but
 * not M^{1/2} W itself.  iters_out / lanczos_iters count the products with P M P, and the error
 * estimate and the stopping test are taken on y.  Allocates 2 vectors of 3 max_N doubles on the first
 * switch-on (RPB_ENOMEM if that fails; the setting is then unchanged); RPB_EINVAL for an unknown
 * kind.  Batch contexts do not use it. */
#define RPB_PRECOND_NONE 0
#define RPB_PRECOND_BLOCK_DIAGONAL 1
int rpb_set_preconditioner(rpb_ctx *ctx, int kind);

/* U = M_tt F + M_tr T  (Sec. II.B Eq. mobilityDifferential and mobilityOverlap; Sec. III Eq.
 * mobilityDifferentialTR; regularisation M = B Mtilde B of Appendix A Eq. effMob, applied to
 * both blocks).  pos: 3N positions.  F, T: 3N forces and torques; either may be NULL (treated
 * as zero; both NULL gives U = 0).  U: 3N output, must not alias pos, F or T.  Direct O(N^2)
 * summation over all ordered pairs including the self terms. */
int rpb_mobility_apply(rpb_ctx *ctx, int64_t N, const double *pos, const double *F, const double *T,
                       double *U);

/* Rows row0 .. row1 - 1 of U = M_tt F + M_tr T (the blocks as for rpb_mobility_apply; all N spheres
 * are sources): the direct summation of Sec. II.B restricted to a range of targets, so that
 * processes (one per GPU) can each compute a share of the rows of one suspension's product and
 * exchange them (rpb_set_product_hook).  row0 must be a multiple of 128, 0 <= row0 < row1 <= N.
 * U_rows: 3 (row1 - row0) doubles, SoA over the rows ([x_row0 .. x_row1-1 | y .. | z ..]); must not
 * alias an input.  F or T may be NULL (both NULL gives 0).  Not offered with pseudo-periodic
 * boundaries (RPB_EINVAL), nor for float32 contexts without the wall. */
int rpb_mobility_apply_rows(rpb_ctx *ctx, int64_t N, const double *pos, const double *F, const double *T,
                            int64_t row0, int64_t row1, double *U_rows);

/* Share `part` of `nparts` of U = M_tt F + M_tr T (Sec. II.B's direct summation split among
 * processes): the shares of parts 0 .. nparts-1 add up to the product (up to the rounding of that
 * sum), so a group of processes, one per GPU, each computing its share and summing them with an
 * all-reduce, obtains the product.  Where the context uses the symmetric pass (float32 pairs, wall
 * on, N >= 256, F given), share p evaluates the p-th of nparts equal contiguous runs of the unordered
 * (target tile, source tile) units of the upper triangle -- each pair once, both of its directions
 * (reciprocity, M_ji = M_ij^T), so nparts processes share the work of one symmetric pass -- and
 * share 0 adds the self terms; pseudo-periodic images included.  Otherwise share p is the rows of the
 * p-th of nparts tile-aligned row ranges (one-way kernels) and zeros elsewhere, or, for
 * pseudo-periodic one-way products and float32 contexts without the wall, the whole product for
 * share 0 and zeros for the others.  nparts = 1 is rpb_mobility_apply without the product hook.
 * pos, F, T as for rpb_mobility_apply; U: 3N doubles (every entry written), aliasing no input.
 * 0 <= part < nparts <= 4096, else RPB_EINVAL.  Never goes through the product hook (it is meant to
 * be called from one).  The symmetric share's schedule is built on the host and copied to the device
 * the first time a given (N, part, nparts) is used (the stream is synchronised then). */
int rpb_mobility_apply_part(rpb_ctx *ctx, int64_t N, const double *pos, const double *F, const double *T,
                            int part, int nparts, double *U);

/* A product computed by the caller: must write all 3N entries of U = M_tt F + M_tr T (F or T may be
 * NULL) on the context's stream and return RPB_OK, or an error code that the library passes on. */
typedef int (*rpb_product_hook)(void *user, int64_t N, const double *pos, const double *F, const double *T,
                                double *U);

/* Delegate every product of this context to hook (NULL restores the library's own): rpb_mobility_apply,
 * the products inside rpb_lanczos_sqrt_apply, rpb_rfd_drift, rpb_ab_step and rpb_step.  It lets a
 * suspension be shared among processes (each computes its share with rpb_mobility_apply_part and the
 * shares are summed, or its rows with rpb_mobility_apply_rows and the rows are gathered, Sec. II.B),
 * while everything else of the step --
 * forces, noise, the Lanczos recurrence and its float64 Gram-Schmidt and tridiagonal square root, the
 * drift and the update -- runs unchanged in every process on the gathered vectors.  Inside the hook,
 * products on this context are the library's own (no recursion).  With a hook, the two-right-hand-side
 * pass is not used, and rpb_run refuses to run (RPB_EINVAL). */
int rpb_set_product_hook(rpb_ctx *ctx, rpb_product_hook hook, void *user);

/* Two products at the same positions: U = M_tt F + M_tr T and U2 = M_tt P (the blocks as for
 * rpb_mobility_apply).  A time step needs both at once: the deterministic velocity and the first
 * Lanczos product M v_0 of Sec. II.C.  Where the context can (float32 pairs, wall on, no periodic
 * images, N >= 256, T given), one symmetric pass evaluates each pair's block once and applies it to
 * both right-hand sides -- the pass rpb_ab_step uses; otherwise two products.  F, P: 3N, non-null; T
 * may be NULL.  U, U2: 3N outputs, distinct, aliasing no input. */
int rpb_mobility_apply2(rpb_ctx *ctx, int64_t N, const double *pos, const double *F, const double *T,
                        const double *P, double *U, double *U2);

/* g ~ M_tt^{1/2} W by the Lanczos method (Sec. II.C; error estimate eps_m = |g_m - g_{m-1}| /
 * |g_{m-1}|).  Full reorthogonalisation (classical Gram-Schmidt twice) and the tridiagonal
 * square root are float64 in both precisions.  Stops at the first m >= 2 with eps_m <= tol; if
 * tol <= 0, runs exactly max_iter iterations (for comparisons at equal m).  Stops early (exact
 * result) if the Krylov space becomes invariant.  max_iter must be in [1, context max_iter].
 * W = 0 gives g = 0, m = 0.  W, g: 3N; g must not alias W or pos.  iters_out, err_out: host
 * pointers (may be NULL).  Waits on the host once per iteration for the stopping test (the
 * tridiagonal step and its status copy run on a side stream of the context, ordered after the
 * iteration's work by events; short products of the next iteration may already be enqueued then and
 * are discarded at the stop), and orders the stream after that side stream before returning.  Returns RPB_ENOCONV
 * if tol > 0 and max_iter was reached without convergence (g is still written). */
int rpb_lanczos_sqrt_apply(rpb_ctx *ctx, int64_t N, const double *pos, const double *W, double *g,
                           double tol, int max_iter, int *iters_out, double *err_out);

/* Random finite difference (Sec. II.A, last term of Eq. EM/AB without the dt factor):
 * drift = (kT/delta) [ M_tt(q + delta/2 Wt) Wt - M_tt(q - delta/2 Wt) Wt ], both displaced
 * configurations regularised anew.  Wt, drift: 3N; delta > 0.  The two matvecs run in the
 * context's pair precision (use RPB_FP64 when the drift must be accurate: its error is the
 * matvec error times a/delta). */
int rpb_rfd_drift(rpb_ctx *ctx, int64_t N, const double *pos, const double *Wt, double delta,
                  double *drift);

/* F = -weight z_hat + steric forces (Sec. III, Eq. soft_potential).  Pairs farther apart than
 * 2a + 40 b are skipped (their force is below e^-40 U0/b ~ 4e-18 U0/b).  A coincident pair exerts
 * nothing. */
int rpb_forces(rpb_ctx *ctx, int64_t N, const double *pos, const rpb_force_params *fp, double *F);

/* Standard normals from Philox4x32-10 (Salmon et al., SC'11): key = (seed low, seed high 32
 * bits), counter = (k / 2, step, stream_id, instance); two 53-bit uniforms in (0, 1] per counter
 * and the Box-Muller transform give normals k and k + 1.  out: 3N in SoA layout, out[c N + i]
 * holding index k = 3 i + c.  stream_id 0 is the Lanczos noise W, 1 the RFD noise W~. */
int rpb_philox_normal(rpb_ctx *ctx, int64_t N, uint64_t seed, uint32_t step, uint32_t stream_id,
                      uint32_t instance, double *out);

/* One stochastic Adams-Bashforth step (Eq. AB), in place:
 *   q <- q + dt (3/2 U^n - 1/2 U^{n-1}) + sqrt(2 kT dt) g + dt drift,   U^{n-1} <- U^n,
 * with U^n = M_tt F(q) + M_tr T, g = lanczos(W), drift = rfd(W~, delta), W and W~ from
 * rpb_philox_normal(seed, step, 0 / 1).  step == 0 is the first step: U^{n-1} is ignored and
 * taken equal to U^n (Euler-Maruyama).  pos, U_prev: 3N, in/out.  stats: host pointer (may be
 * NULL).  Synchronises the stream (Lanczos).  RPB_ENOCONV as for rpb_lanczos_sqrt_apply (the
 * step is still taken).  A context with kT = 0 takes the deterministic step: no noise is drawn and
 * neither the Lanczos square root nor the drift is computed (both carry a factor kT); stats then
 * report 0 iterations, converged. */
int rpb_ab_step(rpb_ctx *ctx, int64_t N, double *pos, double *U_prev, int64_t step, uint64_t seed,
                double dt, double delta, double tol, int max_iter, const rpb_force_params *fp,
                rpb_step_stats *stats);

/* Integrator and drift variants of rpb_step. */
#define RPB_SCHEME_AB 0       /* stochastic Adams-Bashforth, Eq. (AB) */
#define RPB_SCHEME_EM 1       /* Euler-Maruyama, Eq. (EM) */
#define RPB_RFD_CENTRED 0     /* (kT/delta)[M(q + delta/2 W~) W~ - M(q - delta/2 W~) W~], Sec. II.A */
#define RPB_RFD_ONE_SIDED 1   /* (kT/delta)[M(q + delta W~) W~ - M(q) W~], the one-sided difference Sec. II.A
                                 mentions (truncation error O(delta) instead of O(delta^2)) */
typedef struct {
    int scheme;   /* RPB_SCHEME_AB or RPB_SCHEME_EM */
    int rfd;      /* RPB_RFD_CENTRED or RPB_RFD_ONE_SIDED */
} rpb_step_options;

/* One time step as rpb_ab_step, with the integrator and the drift's difference chosen by opts
 * (NULL = Adams-Bashforth with the centred difference, i.e. rpb_ab_step).  Euler-Maruyama
 * (Eq. EM): q <- q + dt U^n + sqrt(2 kT dt) g + dt drift; U_prev is still set to U^n. */
int rpb_step(rpb_ctx *ctx, int64_t N, double *pos, double *U_prev, int64_t step, uint64_t seed, double dt,
             double delta, double tol, int max_iter, const rpb_force_params *fp, const rpb_step_options *opts,
             rpb_step_stats *stats);

/* nsteps time steps of one suspension, as nsteps calls of rpb_step with step indices step, step + 1,
 * ... (Eq. AB or Eq. EM; Sec. II.A-C for the drift and the Lanczos square root), with the same results
 * bit for bit: the step is captured once as the body of a loop (WHILE) node of a CUDA graph and the
 * graph is launched once, running nsteps steps with no host synchronisation in between.  Each
 * Lanczos iteration after the first is a conditional node that runs only while the stopping test of
 * Sec. II.C (eps_m <= tol, or an invariant Krylov space) has not been met, decided on the device by
 * the previous iteration, so a replay runs the iterations a host-driven step would, up to max_iter;
 * for short products the tridiagonal step of an iteration runs beside the next iteration's product
 * (a graph branch; the product is unused after the last iteration).  The step index keying the noise and the first-step flag
 * (step == 0 starts with an Euler-Maruyama step) advance on the device.
 *   - The work runs on a stream the context creates on first use (with a few hundred bytes of
 *     device state), ordered after the context's stream; the context's stream is ordered after the
 *     run, and the call returns when the run is complete.  Must not be called while the context's
 *     stream is being captured.
 *   - stats (may be NULL): the last step's Lanczos dimension m, eps_m and convergence.
 *     *unconverged (may be NULL): steps whose Lanczos stopped at max_iter without meeting tol.
 *   - Errors: as rpb_step; RPB_EINVAL also for nsteps < 0 or step + nsteps >= 2^32; RPB_ENOCONV if
 *     some step did not converge with tol > 0 (all steps are still taken).  nsteps = 0 does nothing. */
int rpb_run(rpb_ctx *ctx, int64_t N, double *pos, double *U_prev, int64_t step, uint64_t seed, int nsteps, double dt,
            double delta, double tol, int max_iter, const rpb_force_params *fp, const rpb_step_options *opts,
            rpb_step_stats *stats, int64_t *unconverged);

/* Message for the calling thread's most recent failed call ("" if none). */
const char *rpb_last_error(void);

/* Total number of CUDA kernel launches this library has enqueued since it was loaded (all contexts,
 * all threads); for accounting of device work, e.g. launches per step. */
uint64_t rpb_launch_count(void);

/* ---------------------------------------------------------------- ragged batches
 * Many independent suspensions of different sizes advanced by one call (the same method per
 * suspension: Sec. II-III and Appendix A as above).  Every instance keeps its state in its own
 * device buffers (SoA, 3 N_b doubles each); a call gathers them into the batch context's packed
 * scratch, runs each stage for all instances together, and scatters the results back.  Instance b
 * is computed the same way whatever the other instances are (its tiles, reductions and noise do
 * not depend on them), so its result alone and inside a batch agree to rounding. */
typedef struct rpb_batch rpb_batch;

/* Create a batch context for at most max_B instances totalling at most max_total_N spheres.
 * Allocates all scratch now (about (max_iter + 14) * 24 * max_total_N bytes). */
int rpb_batch_create(rpb_batch **bt, const rpb_params *p, int64_t max_total_N, int max_B, int max_iter,
                     void *stream);
int rpb_batch_destroy(rpb_batch *bt);
int rpb_batch_set_stream(rpb_batch *bt, void *stream);

/* U_b = M_tt F_b + M_tr T_b for b = 0 .. B-1.  N: host array of B sizes; pos, F, T, U: host arrays
 * of B device pointers (F or T may be NULL as a whole, i.e. zero for every instance). */
int rpb_batch_mobility_apply(rpb_batch *bt, int B, const int64_t *N, const double *const *pos,
                             const double *const *F, const double *const *T, double *const *U);

/* One stochastic Adams-Bashforth step (Eq. AB, as rpb_ab_step) for each instance, in place.
 * steps, seeds: host arrays of B per-instance step counters and Philox seeds (steps[b] == 0 is that
 * instance's first, Euler-Maruyama, step); instance b draws exactly the noise rpb_ab_step would
 * draw with seeds[b] and steps[b].  stats: host array of B entries (or NULL).  Synchronises the
 * stream.  RPB_ENOCONV if some instance's Lanczos did not converge (all steps are still taken). */
int rpb_batch_ab_step(rpb_batch *bt, int B, const int64_t *N, double *const *pos, double *const *U_prev,
                      const int64_t *steps, const uint64_t *seeds, double dt, double delta, double tol,
                      int max_iter, const rpb_force_params *fp, rpb_step_stats *stats);

/* nsteps AB steps of every instance (as repeated rpb_batch_ab_step) with one gather and one scatter
 * of the state, the step captured once as the body of a loop (WHILE) node of a CUDA graph that is
 * launched once, running nsteps steps with no host synchronisation in between.  Inside the graph each Lanczos iteration after the first is a
 * conditional node that runs while some instance is still active (decided on the device), up to
 * lanczos_iters iterations per step, with converged instances masked out (so lanczos_iters caps the
 * iteration count the tolerance needs; *unconverged, if not NULL, receives the number of
 * instance-steps that did not reach tol, and RPB_ENOCONV is returned if it is nonzero with tol > 0).  steps: each instance's
 * first step index (advanced on the device).  stats: the last step's statistics (B entries, or
 * NULL).  The work runs on a stream the batch context owns, ordered after the context's stream;
 * the call returns when it is complete. */
int rpb_batch_run(rpb_batch *bt, int B, const int64_t *N, double *const *pos, double *const *U_prev,
                  const int64_t *steps, const uint64_t *seeds, int nsteps, double dt, double delta, double tol,
                  int lanczos_iters, const rpb_force_params *fp, rpb_step_stats *stats, int64_t *unconverged);

/* Measured arithmetic peak of the current device (a measurement aid: the paper has none).  Runs
 * independent chains of fused multiply-adds on every SM -- packed float32x2 (RPB_PEAK_FFMA2, the
 * instruction the float32 pair kernels use), scalar float32 (RPB_PEAK_FFMA) or float64
 * (RPB_PEAK_DFMA) -- for about 40 ms per launch, one warm-up launch and three timed ones with CUDA
 * events on stream (a cudaStream_t, NULL = legacy default stream), and returns the best rate in
 * *tflops (an FMA counts 2 flops) and that launch's duration in *ms (may be NULL).  It runs at
 * whatever clocks the GPU is at (it changes no setting).  Synchronises the stream.  RPB_EINVAL for
 * an unknown kind or a null tflops, RPB_ECUDA for CUDA failures. */
#define RPB_PEAK_FFMA2 0
#define RPB_PEAK_FFMA 1
#define RPB_PEAK_DFMA 2
int rpb_fma_peak(int kind, void *stream, double *tflops, double *ms);

/* Tile schedule of a batch context's float32 products -- what its autotuner chooses (the batched
 * products are the direct summation of Sec. II.B over each suspension, the same method whatever the
 * schedule):
 *   seg_tiles   length, in 128-sphere tiles, of the runs into which the symmetric pass cuts every
 *               suspension's rows of tiles (one CTA per run), 1 .. 64.  The cut depends only on each
 *               suspension's own size, so for a given seg_tiles a suspension's result is the same bit
 *               for bit alone and in any mix; between values it differs in rounding only.
 *   ctas_per_sm resident CTAs per SM of the symmetric translation-translation kernel, 4 or 5 (no
 *               effect on the results).
 *   symmetric   1: the symmetric pass (both directions of a pair from one evaluation); 0: the
 *               one-way kernel (float64 contexts always use it).
 * The default is {8, 5, 1} (the environment variable RPB_FP32_BATCH_SYM=0 at creation makes it
 * one-way). */
typedef struct {
    int seg_tiles;
    int ctas_per_sm;
    int symmetric;
} rpb_batch_tiles;

/* Set (t; NULL = the default) or read the tile schedule.  RPB_EINVAL for values outside the ranges
 * above.  Takes effect from the next call. */
int rpb_batch_set_tiles(rpb_batch *bt, const rpb_batch_tiles *t);
int rpb_batch_get_tiles(rpb_batch *bt, rpb_batch_tiles *t);

/* Autotuner: for the batch of B suspensions of sizes N at positions pos (host array of B device
 * pointers), time every candidate schedule -- the symmetric pass with seg_tiles in {4, 8, 16, 32} at
 * 4 and 5 CTAs per SM, and the one-way kernel -- by reps products of each kind (unit loads; one
 * warm-up round first) with CUDA events on the context's stream, weighing ten translation-translation
 * products per fused one (a step's mix); make the fastest the context's schedule (kept until set
 * again) and return it in *best (may be NULL).  cand, cand_ms (may be NULL): the first max_cand
 * candidates and their weighted times in ms; *ncand (may be NULL): the number of candidates.  Float64
 * contexts have one candidate.  Synchronises the stream; allocates the symmetric plan's scratch. */
int rpb_batch_tune(rpb_batch *bt, int B, const int64_t *N, const double *const *pos, int reps, rpb_batch_tiles *best,
                   int max_cand, rpb_batch_tiles *cand, double *cand_ms, int *ncand);

/* Largest N accepted by rpb_mobility_apply_noalloc. */
#define RPB_NOALLOC_MAX_N 16384

/* U = M_tt F + M_tr T like rpb_mobility_apply, but without a context and without allocating.
 * The paper has no counterpart to this entry point; it exists for callers that cannot call
 * cudaMalloc -- for example a host application that hands out all device memory from its own
 * pool and allows no other allocation, or code running where the device-wide synchronisation an
 * allocation may cause is not acceptable.  rpb_create allocates a context's scratch, so such
 * callers cannot use rpb_mobility_apply.
 *   - Scratch: a fixed array of about 7.6 MB in the library's device image (packed sources for
 *     RPB_NOALLOC_MAX_N spheres plus the partial sums), present on every GPU that loads the
 *     library until the process exits.  The caller still passes pos, F, T and U (device pointers,
 *     SoA, as for rpb_mobility_apply); F or T may be NULL.
 *   - p: a, eta and precision are used (kT is ignored).  stream: a cudaStream_t (NULL = legacy
 *     default stream), on the current device.
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 *     with that device current, and the call looks it up again whenever the device's CUDA
 *     context has changed since (after cudaDeviceReset, or a primary context released and created
 *     anew, the array may have moved).  Make that first call, and the first call after such a
 *     change, outside any stream capture: made while the stream is being captured, it returns
 *     RPB_EINVAL with a message saying so.
 *   - Every call on a device shares the one array and leaves its contents behind; each call
 *     overwrites all of the scratch it reads, so nothing has to be cleared in between.  Calls
 *     whose kernels may overlap on the GPU (different streams, or different host threads) race on
 *     the array: order them on one stream or synchronise between them.
 *   - Errors: RPB_EINVAL for N <= 0 or N > RPB_NOALLOC_MAX_N (message states the limit), bad
 *     parameters, null pos or U, misaligned or aliasing pointers; RPB_ECUDA for CUDA failures. */
int rpb_mobility_apply_noalloc(int64_t N, const double *pos, const double *F, const double *T, double *U,
                               const rpb_params *p, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* RPB_H */
