// sim.cu -- the coupled per-step loop (flow chart of Fig. 1) as CUDA graphs.
//
// One step = membrane forces (+ wall term) -> bond forces -> spreading ->
// lattice Boltzmann -> interpolation and advection -> adhesion update.  The
// kernel sequence of a step is captured once per lattice-buffer parity (the
// two graphs differ only in which population buffer they read) on a private
// capture stream and then replayed on the caller's stream, so a step costs
// one graph launch on the host.  The Philox step index lives in device memory
// (advanced by the last kernel of a step), so replays need no host updates.
#include <vector>

#include "pfsi_internal.cuh"

namespace pfsi {

struct SimCtx {
    LbCtx* lb;
    MemCtx* mem;
    BondCtx* bonds;
    double* X;
    float* F;
    float* U;
    int M;
    uint64_t step;
    cudaStream_t cap;
    cudaGraphExec_t exec[2];
    cudaEvent_t lb_ev[2];  // optional events around the lattice step (timing)
    SgCtx* sg;             // learned membrane surrogate, or null (plain solver)
    const void* sg_params;
};

namespace {

int enqueue_step(SimCtx* c, cudaStream_t s)
{
    int rc;
    if (c->sg) {
        rc = launch_membrane_global(c->mem, c->X, c->F, s);
        if (!rc) rc = launch_surrogate_forces(c->sg, c->sg_params, c->mem->xh, c->mem->xl, c->F, s);
    } else {
        rc = launch_membrane_forces(c->mem, c->X, c->F, s);
    }
    if (!rc && c->bonds) rc = launch_bonds_forces(c->bonds, c->X, c->F, c->M, s);
    if (!rc) rc = launch_ib_spread(c->lb, c->X, c->F, c->M, c->mem->chunks, c->mem->n_chunks, s);
    if (!rc && c->lb_ev[0])
        rc = check_cuda(cudaEventRecordWithFlags(c->lb_ev[0], s, cudaEventRecordExternal), "sim: lb timing event");
    if (!rc) rc = launch_lb_step(c->lb, s);
    if (!rc && c->lb_ev[1])
        rc = check_cuda(cudaEventRecordWithFlags(c->lb_ev[1], s, cudaEventRecordExternal), "sim: lb timing event");
    if (!rc) rc = launch_ib_interp(c->lb, c->X, c->U, c->M, 1, c->mem->chunks, c->mem->n_chunks, s);
    if (!rc && c->bonds) rc = launch_bonds_step(c->bonds, c->X, c->M, 0, c->bonds->counters + 3, s);
    return rc;
}

int capture(SimCtx* c, int parity)
{
    const int saved = c->lb->cur;
    c->lb->cur = parity;
    int rc = check_cuda(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal), "sim: begin capture");
    if (rc) {
        c->lb->cur = saved;
        return rc;
    }
    const int rc_enq = enqueue_step(c, c->cap);
    cudaGraph_t graph = nullptr;
    rc = check_cuda(cudaStreamEndCapture(c->cap, &graph), "sim: end capture");
    c->lb->cur = saved;
    if (rc_enq) {
        if (graph) cudaGraphDestroy(graph);
        return rc_enq;
    }
    if (rc) return rc;
    rc = check_cuda(cudaGraphInstantiate(&c->exec[parity], graph, 0), "sim: instantiate");
    cudaGraphDestroy(graph);
    return rc;
}

}  // namespace

}  // namespace pfsi

using namespace pfsi;

struct sim_ctx : pfsi::SimCtx {};

extern "C" int sim_create(lb_ctx* lb, mem_ctx* mem, bond_ctx* bonds, double* X, float* F, float* U, int M,
                          uint64_t first_step, sim_ctx** out)
{
    if (!lb || !mem || !X || !F || !U || !out || M < 1) return set_error(PFSI_ERR_ARG, "sim_create: bad argument");
    if (mem->n != M) return set_error(PFSI_ERR_ARG, "sim_create: node count differs from the membrane mesh");
    sim_ctx* c = new sim_ctx();
    c->lb = lb;
    c->mem = mem;
    c->bonds = bonds;
    c->X = X;
    c->F = F;
    c->U = U;
    c->M = M;
    c->step = first_step;
    c->exec[0] = c->exec[1] = nullptr;
    c->lb_ev[0] = c->lb_ev[1] = nullptr;
    int rc = check_cuda(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking), "sim_create: stream");
    if (!rc && bonds) {
        const unsigned long long s = first_step;
        rc = check_cuda(cudaMemcpy(bonds->counters + 3, &s, sizeof(s), cudaMemcpyHostToDevice), "sim_create: step");
    }
    if (rc) {
        delete c;
        return rc;
    }
    *out = c;
    return PFSI_OK;
}

extern "C" int sim_destroy(sim_ctx* c)
{
    if (!c) return PFSI_OK;
    for (int k = 0; k < 2; ++k)
        if (c->exec[k]) cudaGraphExecDestroy(c->exec[k]);
    if (c->cap) cudaStreamDestroy(c->cap);
    for (int k = 0; k < 2; ++k)
        if (c->lb_ev[k]) cudaEventDestroy(c->lb_ev[k]);
    delete c;
    return PFSI_OK;
}

extern "C" int sim_step(sim_ctx* c, int nsteps, void* stream)
{
    if (!c || nsteps < 0) return set_error(PFSI_ERR_ARG, "sim_step: bad argument");
    cudaStream_t s = as_stream(stream);
    for (int k = 0; k < nsteps; ++k) {
        const int parity = c->lb->cur;
        if (!c->exec[parity]) {
            const int rc = capture(c, parity);
            if (rc) return rc;
        }
        const int rc = check_cuda(cudaGraphLaunch(c->exec[parity], s), "sim_step: graph launch");
        if (rc) return rc;
        c->lb->cur ^= 1;
        c->step += 1;
    }
    return PFSI_OK;
}

extern "C" int sim_set_surrogate(sim_ctx* c, sg_ctx* sg, const void* params)
{
    if (!c || (sg && !params)) return set_error(PFSI_ERR_ARG, "sim_set_surrogate: bad argument");
    SgCtx* g = sg ? sg_internal(sg) : nullptr;
    if (g && sg_node_count(g) != c->M) return set_error(PFSI_ERR_ARG, "sim_set_surrogate: node count differs");
    for (int k = 0; k < 2; ++k) {
        if (c->exec[k]) cudaGraphExecDestroy(c->exec[k]);
        c->exec[k] = nullptr;
    }
    c->sg = g;
    c->sg_params = params;
    return PFSI_OK;
}

extern "C" int sim_time_lb(sim_ctx* c, int on)
{
    if (!c) return set_error(PFSI_ERR_ARG, "sim_time_lb: null context");
    const bool want = on != 0;
    if (want == (c->lb_ev[0] != nullptr)) return PFSI_OK;
    for (int k = 0; k < 2; ++k) {
        if (c->exec[k]) cudaGraphExecDestroy(c->exec[k]);
        c->exec[k] = nullptr;
        if (c->lb_ev[k]) cudaEventDestroy(c->lb_ev[k]);
        c->lb_ev[k] = nullptr;
    }
    if (!want) return PFSI_OK;
    for (int k = 0; k < 2; ++k) {
        const int rc = check_cuda(cudaEventCreate(&c->lb_ev[k]), "sim_time_lb: event");
        if (rc) return rc;
    }
    return PFSI_OK;
}

extern "C" int sim_lb_ms(sim_ctx* c, float* ms)
{
    if (!c || !ms) return set_error(PFSI_ERR_ARG, "sim_lb_ms: null argument");
    if (!c->lb_ev[0]) return set_error(PFSI_ERR_ARG, "sim_lb_ms: timing is off (sim_time_lb)");
    int rc = check_cuda(cudaEventSynchronize(c->lb_ev[1]), "sim_lb_ms: synchronise");
    if (!rc) rc = check_cuda(cudaEventElapsedTime(ms, c->lb_ev[0], c->lb_ev[1]), "sim_lb_ms: elapsed");
    return rc;
}

extern "C" int sim_step_index(const sim_ctx* c, uint64_t* out)
{
    if (!c || !out) return set_error(PFSI_ERR_ARG, "sim_step_index: null argument");
    *out = c->step;
    return PFSI_OK;
}

// ---------------------------------------------------------------------------
// Batches of independent chambers: one CUDA graph holds `k` steps of every
// chamber, each chamber's kernel chain captured on its own stream (a parallel
// branch of the graph), so a single graph launch runs all chambers
// concurrently and the GPU overlaps their kernels.
namespace pfsi {

struct BatchCtx {
    std::vector<SimCtx*> sims;
    int k;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> join;
    cudaStream_t cap;
    cudaEvent_t fork;
    cudaGraphExec_t exec[2];
};

namespace {

void batch_free(BatchCtx* b)
{
    for (int k = 0; k < 2; ++k)
        if (b->exec[k]) cudaGraphExecDestroy(b->exec[k]);
    for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->join) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->cap) cudaStreamDestroy(b->cap);
}

int batch_capture(BatchCtx* b, int parity)
{
    std::vector<int> saved;
    for (SimCtx* c : b->sims) {
        saved.push_back(c->lb->cur);
        c->lb->cur = parity;
    }
    int rc = check_cuda(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "batch: begin capture");
    int rc_enq = PFSI_OK;
    if (!rc) {
        rc_enq = check_cuda(cudaEventRecord(b->fork, b->cap), "batch: fork");
        for (size_t i = 0; i < b->sims.size() && !rc_enq; ++i) {
            rc_enq = check_cuda(cudaStreamWaitEvent(b->streams[i], b->fork, 0), "batch: branch");
            for (int s = 0; s < b->k && !rc_enq; ++s) rc_enq = enqueue_step(b->sims[i], b->streams[i]);
            if (!rc_enq) rc_enq = check_cuda(cudaEventRecord(b->join[i], b->streams[i]), "batch: join");
            if (!rc_enq) rc_enq = check_cuda(cudaStreamWaitEvent(b->cap, b->join[i], 0), "batch: join");
        }
        cudaGraph_t graph = nullptr;
        rc = check_cuda(cudaStreamEndCapture(b->cap, &graph), "batch: end capture");
        if (!rc && !rc_enq) rc = check_cuda(cudaGraphInstantiate(&b->exec[parity], graph, 0), "batch: instantiate");
        if (graph) cudaGraphDestroy(graph);
    }
    for (size_t i = 0; i < b->sims.size(); ++i) b->sims[i]->lb->cur = saved[i];
    return rc_enq ? rc_enq : rc;
}

}  // namespace

}  // namespace pfsi

struct batch_ctx : pfsi::BatchCtx {};

extern "C" int batch_create(sim_ctx** sims, int n, int steps_per_graph, batch_ctx** out)
{
    if (!sims || n < 1 || steps_per_graph < 1 || !out) return set_error(PFSI_ERR_ARG, "batch_create: bad argument");
    for (int i = 0; i < n; ++i) {
        if (!sims[i]) return set_error(PFSI_ERR_ARG, "batch_create: null chamber");
        if (sims[i]->lb->cur != sims[0]->lb->cur)
            return set_error(PFSI_ERR_ARG, "batch_create: chambers must be at the same lattice-buffer parity");
        for (int j = 0; j < i; ++j)
            if (sims[j] == sims[i]) return set_error(PFSI_ERR_ARG, "batch_create: a chamber appears twice");
    }
    batch_ctx* b = new batch_ctx();
    b->k = steps_per_graph;
    b->cap = nullptr;
    b->fork = nullptr;
    b->exec[0] = b->exec[1] = nullptr;
    int rc = check_cuda(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking), "batch_create: stream");
    if (!rc) rc = check_cuda(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), "batch_create: event");
    for (int i = 0; i < n && !rc; ++i) {
        b->sims.push_back(sims[i]);
        cudaStream_t s = nullptr;
        cudaEvent_t e = nullptr;
        rc = check_cuda(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "batch_create: stream");
        if (!rc) b->streams.push_back(s);
        if (!rc) rc = check_cuda(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "batch_create: event");
        if (!rc) b->join.push_back(e);
    }
    if (rc) {
        batch_free(b);
        delete b;
        return rc;
    }
    *out = b;
    return PFSI_OK;
}

extern "C" int batch_destroy(batch_ctx* b)
{
    if (!b) return PFSI_OK;
    batch_free(b);
    delete b;
    return PFSI_OK;
}

extern "C" int batch_step(batch_ctx* b, int nsteps, void* stream)
{
    if (!b || nsteps < 0 || nsteps % b->k) return set_error(PFSI_ERR_ARG, "batch_step: nsteps must be a multiple of steps_per_graph");
    cudaStream_t s = as_stream(stream);
    for (int done = 0; done < nsteps; done += b->k) {
        const int parity = b->sims[0]->lb->cur;
        if (!b->exec[parity]) {
            const int rc = batch_capture(b, parity);
            if (rc) return rc;
        }
        const int rc = check_cuda(cudaGraphLaunch(b->exec[parity], s), "batch_step: graph launch");
        if (rc) return rc;
        for (SimCtx* c : b->sims) {
            c->lb->cur ^= (b->k & 1);
            c->step += b->k;
        }
    }
    return PFSI_OK;
}
