// run.cu -- many time steps of one suspension replayed from a CUDA graph (rpb_run).
//
// A step (forces, noise, the fused product, Lanczos M^{1/2} W of Sec. II.C, the RFD drift of
// Sec. II.A and the update of Eq. AB) is captured once into a graph on a stream the context owns and
// replayed nsteps times with no host synchronisation in between.  Each Lanczos iteration after the
// first is a conditional (IF) node whose condition the previous iteration sets on the device from the
// stopping test, so a replay runs exactly the iterations a host-driven step runs; the step index that
// keys the noise and the first-step flag live on the device and advance at the end of each replay.
// The kernels, their arguments and their order are those of rpb_step, so the results are the same
// bit for bit.
#include <new>

#include "lanczos_math.cuh"
#include "rpb_internal.cuh"

namespace rpb {

static_assert(kRunMaxIter == kMaxIter, "run state sized for the Lanczos dimension");

struct RunCtx {
    cudaStream_t st = nullptr;    // capture and replay
    cudaStream_t body = nullptr;  // conditional bodies are captured here
    cudaEvent_t ev = nullptr;     // orders the run after the context's stream and back
    RunState *state = nullptr;    // device
    RunState *h_state = nullptr;  // pinned host copy
    double *h_status = nullptr;   // pinned host copy of the Lanczos status words
};

int graph_begin_if(cudaStream_t st, cudaStream_t body, cudaGraphConditionalHandle h)
{
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *edges = nullptr;
    size_t nd = 0;
    int rc;
    if ((rc = cuda_fail(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, &edges, &nd), "capture info")))
        return rc;
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeIf;
    p.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    if ((rc = cuda_fail(cudaGraphAddNode(&node, g, deps, edges, nd, &p), "conditional node")) ||
        (rc = cuda_fail(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies),
                        "capture dependencies")) ||
        (rc = cuda_fail(cudaStreamBeginCaptureToGraph(body, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                      cudaStreamCaptureModeThreadLocal),
                        "body capture")))
        return rc;
    return RPB_OK;
}

void run_free(rpb_ctx *ctx)
{
    RunCtx *r = ctx->run;
    if (!r) return;
    if (r->st) cudaStreamDestroy(r->st);
    if (r->body) cudaStreamDestroy(r->body);
    if (r->ev) cudaEventDestroy(r->ev);
    if (r->state) cudaFree(r->state);
    if (r->h_state) cudaFreeHost(r->h_state);
    if (r->h_status) cudaFreeHost(r->h_status);
    delete r;
    ctx->run = nullptr;
}

// First use: the streams, the event and the run state (a few hundred bytes of device memory).
static int run_setup(rpb_ctx *ctx)
{
    if (ctx->run) return RPB_OK;
    RunCtx *r = new (std::nothrow) RunCtx();
    if (!r) {
        set_error("host allocation failed");
        return RPB_ENOMEM;
    }
    ctx->run = r;
    int rc;
    if ((rc = cuda_fail(cudaStreamCreateWithFlags(&r->st, cudaStreamNonBlocking), "run stream")) ||
        (rc = cuda_fail(cudaStreamCreateWithFlags(&r->body, cudaStreamNonBlocking), "run body stream")) ||
        (rc = cuda_fail(cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming), "run event"))) {
        run_free(ctx);
        return rc;
    }
    if (cudaMalloc((void **)&r->state, sizeof(RunState)) != cudaSuccess ||
        cudaMallocHost((void **)&r->h_state, sizeof(RunState)) != cudaSuccess ||
        cudaMallocHost((void **)&r->h_status, 8 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        set_error("allocation of the run state failed");
        run_free(ctx);
        return RPB_ENOMEM;
    }
    return RPB_OK;
}

__global__ void run_init_kernel(RunState *s, unsigned int step)
{
    s->step = step;
    s->first = step == 0u ? 1 : 0;
    s->m = 0;
    s->unconv = 0ull;
    for (int k = 0; k < kRunMaxIter; ++k) s->iter_runs[k] = 0ull;
}

// End of a replayed step: the next step's index, no longer a first step, and whether this step's
// Lanczos stopped short of the tolerance (lanczos: the step ran the iteration; tol > 0).
__global__ void run_advance_kernel(RunState *s, const double *__restrict__ status, int lanczos, double tol)
{
    s->step += 1u;
    s->first = 0;
    if (lanczos && tol > 0.0 && status[ST_STOP] == 0.0) s->unconv += 1ull;
}

}  // namespace rpb

using namespace rpb;

extern "C" int rpb_run(rpb_ctx *ctx, int64_t N, double *pos, double *U_prev, int64_t step, uint64_t seed, int nsteps,
                       double dt, double delta, double tol, int max_iter, const rpb_force_params *fp,
                       const rpb_step_options *opts, rpb_step_stats *stats, int64_t *unconverged)
{
    int rc;
    if ((rc = check_step_args(ctx, N, pos, U_prev, step, dt, delta, max_iter, fp, opts))) return rc;
    if (nsteps < 0 || step + (int64_t)nsteps > 0xffffffffLL) {
        set_error("nsteps=%d outside [0, 2^32 - 1 - step]", nsteps);
        return RPB_EINVAL;
    }
    if (ctx->hook) {
        set_error("rpb_run: a context with a product hook cannot replay its steps from a graph");
        return RPB_EINVAL;
    }
    if (unconverged) *unconverged = 0;
    if (nsteps == 0) return RPB_OK;
    const int scheme = opts ? opts->scheme : RPB_SCHEME_AB;
    const int rfd = opts ? opts->rfd : RPB_RFD_CENTRED;
    if ((rc = run_setup(ctx))) return rc;
    RunCtx *r = ctx->run;
    const cudaStream_t user = ctx->stream;
    // host-side preparation before the capture, then the run ordered after the caller's stream
    if ((rc = pair_prepare(ctx, N)) || (rc = cuda_fail(cudaEventRecord(r->ev, user), "event record")) ||
        (rc = cuda_fail(cudaStreamWaitEvent(r->st, r->ev, 0), "stream wait")))
        return rc;
    run_init_kernel<<<1, 1, 0, r->st>>>(r->state, (unsigned int)step);
    count_launches(1);
    LzGraph gr;
    gr.body = r->body;
    gr.state = r->state;
    const LzLayout L(ctx->max_iter);
    const double *status = ctx->ws.lz + L.status;
    const bool lanczos = ctx->p.kT > 0.0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const uint64_t before = rpb_launch_count();
    ctx->stream = r->st;
    if ((rc = cuda_fail(cudaStreamBeginCapture(r->st, cudaStreamCaptureModeThreadLocal), "begin capture"))) {
        ctx->stream = user;
        return rc;
    }
    int brc = step_impl(ctx, N, pos, U_prev, (uint32_t)step, seed, dt, delta, tol, max_iter, fp, scheme, rfd, nullptr,
                        &gr);
    if (!brc) {
        run_advance_kernel<<<1, 1, 0, r->st>>>(r->state, status, lanczos ? 1 : 0, tol);
        count_launches(1);
        brc = cuda_fail(cudaGetLastError(), "run kernels");
    }
    const cudaError_t ec = cudaStreamEndCapture(r->st, &graph);
    ctx->stream = user;
    const int per_step = (int)(rpb_launch_count() - before);
    count_launches(-per_step);  // captured, not executed (counted below from the runs)
    if (brc || ec != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return brc ? brc : cuda_fail(ec, "end capture");
    }
    if ((rc = cuda_fail(cudaGraphInstantiate(&exec, graph, 0), "graph instantiate"))) {
        cudaGraphDestroy(graph);
        return rc;
    }
    for (int s = 0; s < nsteps && !rc; ++s) rc = cuda_fail(cudaGraphLaunch(exec, r->st), "graph launch");
    if (!rc &&
        !(rc = cuda_fail(cudaMemcpyAsync(r->h_state, r->state, sizeof(RunState), cudaMemcpyDeviceToHost, r->st),
                         "run state copy")) &&
        !(rc = cuda_fail(cudaMemcpyAsync(r->h_status, status, 8 * sizeof(double), cudaMemcpyDeviceToHost, r->st),
                         "status copy")) &&
        !(rc = cuda_fail(cudaEventRecord(r->ev, r->st), "event record")) &&
        !(rc = cuda_fail(cudaStreamWaitEvent(user, r->ev, 0), "stream wait")))
        rc = cuda_fail(cudaStreamSynchronize(r->st), "run");
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    if (rc) return rc;
    // kernels executed: the unconditional part every step, each iteration body once per run of it
    int64_t cond_part = 0, executed = 0;
    for (int k = 1; k < kRunMaxIter; ++k) {
        cond_part += gr.iter_launches[k];
        executed += (int64_t)gr.iter_launches[k] * (int64_t)r->h_state->iter_runs[k];
    }
    count_launches((int)((per_step - cond_part) * (int64_t)nsteps + executed));
    const int64_t unconv = (int64_t)r->h_state->unconv;
    if (unconverged) *unconverged = unconv;
    if (stats) {
        stats->lanczos_iters = lanczos ? r->h_state->m : 0;
        stats->lanczos_err = lanczos ? r->h_status[ST_EPS] : 0.0;
        stats->converged = lanczos ? (r->h_status[ST_STOP] != 0.0 ? 1 : 0) : 1;
    }
    if (unconv && tol > 0.0) {
        set_error("lanczos: %lld step(s) did not converge in %d iterations", (long long)unconv, max_iter);
        return RPB_ENOCONV;
    }
    return RPB_OK;
}
