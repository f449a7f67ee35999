// run.cu -- many time steps of one suspension replayed from a CUDA graph (rpb_run).
//
// A step (forces, noise, the fused product, Lanczos M^{1/2} W of Sec. II.C, the RFD drift of
// Sec. II.A and the update of Eq. AB) is captured once as the body of a WHILE node of a graph on a
// stream the context owns, and the graph is launched once: the body runs nsteps times with no host
// synchronisation in between, the last kernel of a step counting the steps down.  Each Lanczos
// iteration after the first is a conditional (IF) node inside that body whose condition the previous
// iteration sets on the device from the stopping test, so a replay runs exactly the iterations a
// host-driven step runs; the step index that keys the noise and the first-step flag live on the device
// and advance at the end of each step.
// The kernels, their arguments and their order are those of rpb_step, so the results are the same
// bit for bit.
#include <new>

#include "lanczos_math.cuh"
#include "rpb_internal.cuh"

namespace rpb {

static_assert(kRunMaxIter == kMaxIter, "run state sized for the Lanczos dimension");

struct RunCtx {
    cudaStream_t st = nullptr;    // capture and replay
    cudaStream_t loop = nullptr;  // the body of the loop over the steps is captured here
    cudaStream_t body = nullptr;  // the Lanczos iterations' conditional bodies are captured here
    cudaStream_t side0 = nullptr, side = nullptr;  // a second branch inside a Lanczos iteration (the tridiagonal
                                                   // step): in the first iteration, in the conditional ones
    cudaEvent_t ev = nullptr;     // orders the run after the context's stream and back
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;  // fork and join of that branch in the capture
    RunState *state = nullptr;    // device
    RunState *h_state = nullptr;  // pinned host copy
    double *h_status = nullptr;   // pinned host copy of the Lanczos status words
};

int graph_begin_if(cudaStream_t st, cudaStream_t body, cudaGraphConditionalHandle h)
{
    return graph_begin_cond(st, body, h, cudaGraphCondTypeIf);
}

__global__ void graph_reset_conds_kernel(CondSet s, int n)
{
    for (int k = threadIdx.x; k < n; k += blockDim.x) cudaGraphSetConditional(s.h[k], 0u);
}

__global__ void graph_loop_init_kernel(int *left, int n)
{
    *left = n;
}

__global__ void graph_loop_tail_kernel(int *left, cudaGraphConditionalHandle h)
{
    const int l = *left - 1;
    *left = l;
    cudaGraphSetConditional(h, l > 0 ? 1u : 0u);
}

int graph_begin_loop(cudaStream_t st, cudaStream_t body, cudaGraphConditionalHandle *h)
{
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    int rc;
    if ((rc = cuda_fail(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, nullptr, nullptr, nullptr), "capture info")) ||
        (rc = cuda_fail(cudaGraphConditionalHandleCreate(h, g, 1u, cudaGraphCondAssignDefault), "loop handle")))
        return rc;
    return graph_begin_cond(st, body, *h, cudaGraphCondTypeWhile);
}

int graph_begin_cond(cudaStream_t st, cudaStream_t body, cudaGraphConditionalHandle h,
                     cudaGraphConditionalNodeType type)
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
    p.conditional.type = type;
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
    for (cudaStream_t q : {r->st, r->loop, r->body, r->side0, r->side})
        if (q) cudaStreamDestroy(q);
    for (cudaEvent_t e : {r->ev, r->ev_fork, r->ev_join})
        if (e) cudaEventDestroy(e);
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
        (rc = cuda_fail(cudaStreamCreateWithFlags(&r->loop, cudaStreamNonBlocking), "run loop stream")) ||
        (rc = cuda_fail(cudaStreamCreateWithFlags(&r->body, cudaStreamNonBlocking), "run body stream")) ||
        (rc = cuda_fail(cudaStreamCreateWithFlags(&r->side0, cudaStreamNonBlocking), "run side stream")) ||
        (rc = cuda_fail(cudaStreamCreateWithFlags(&r->side, cudaStreamNonBlocking), "run side stream")) ||
        (rc = cuda_fail(cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming), "run event")) ||
        (rc = cuda_fail(cudaEventCreateWithFlags(&r->ev_fork, cudaEventDisableTiming), "run event")) ||
        (rc = cuda_fail(cudaEventCreateWithFlags(&r->ev_join, cudaEventDisableTiming), "run event"))) {
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

__global__ void run_init_kernel(RunState *s, unsigned int step, int nsteps)
{
    s->step = step;
    s->first = step == 0u ? 1 : 0;
    s->m = 0;
    s->left = nsteps;
    s->unconv = 0ull;
    for (int k = 0; k < kRunMaxIter; ++k) s->iter_runs[k] = 0ull;
}

// End of a replayed step: the next step's index, no longer a first step, whether this step's Lanczos
// stopped short of the tolerance (lanczos: the step ran the iteration; tol > 0), and the loop over the
// steps runs again while steps are left.
__global__ void run_advance_kernel(RunState *s, const double *__restrict__ status, int lanczos, double tol,
                                   cudaGraphConditionalHandle loop)
{
    s->step += 1u;
    s->first = 0;
    if (lanczos && tol > 0.0 && status[ST_STOP] == 0.0) s->unconv += 1ull;
    const int l = s->left - 1;
    s->left = l;
    cudaGraphSetConditional(loop, l > 0 ? 1u : 0u);
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
    run_init_kernel<<<1, 1, 0, r->st>>>(r->state, (unsigned int)step, nsteps);
    count_launches(1);
    LzGraph gr;
    gr.body = r->body;
    gr.state = r->state;
    gr.side0 = r->side0;
    gr.side = r->side;
    gr.ev_fork = r->ev_fork;
    gr.ev_join = r->ev_join;
    const LzLayout L(ctx->max_iter);
    const double *status = ctx->ws.lz + L.status;
    const bool lanczos = ctx->p.kT > 0.0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const uint64_t before = rpb_launch_count();
    // the graph: one WHILE node whose body is a step (run_advance_kernel counts the steps down), so
    // all nsteps run from one graph launch
    if ((rc = cuda_fail(cudaStreamBeginCapture(r->st, cudaStreamCaptureModeThreadLocal), "begin capture"))) return rc;
    cudaGraphConditionalHandle loop_h = 0;
    int brc = graph_begin_loop(r->st, r->loop, &loop_h);
    if (!brc) {
        ctx->stream = r->loop;
        brc = step_impl(ctx, N, pos, U_prev, (uint32_t)step, seed, dt, delta, tol, max_iter, fp, scheme, rfd, nullptr,
                        &gr);
        if (!brc) {
            run_advance_kernel<<<1, 1, 0, r->loop>>>(r->state, status, lanczos ? 1 : 0, tol, loop_h);
            count_launches(1);
            brc = cuda_fail(cudaGetLastError(), "run kernels");
        }
        cudaGraph_t loop_graph = nullptr;  // owned by the WHILE node
        const cudaError_t el = cudaStreamEndCapture(r->loop, &loop_graph);
        if (!brc && el != cudaSuccess) brc = cuda_fail(el, "loop body capture end");
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
    rc = cuda_fail(cudaGraphLaunch(exec, r->st), "graph launch");
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
