// sim.cu -- the coupled per-step loop (flow chart of Fig. 1) as CUDA graphs.
//
// One step = membrane forces (+ wall term) -> bond forces -> spreading ->
// lattice Boltzmann -> interpolation and advection -> adhesion update.  The
// kernel sequence of a step is captured once per lattice-buffer parity (the
// two graphs differ only in which population buffer they read) on a private
// capture stream and then replayed on the caller's stream, so a step costs
// one graph launch on the host.  The Philox step index lives in device memory
// (advanced by the last kernel of a step), so replays need no host updates.
#include <algorithm>
#include <string>
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
    // multi-step graphs per length (kLongMulti, kMulti steps) and starting
    // parity: each step's adhesion update runs on a side branch beside the
    // next step's membrane pass
    cudaGraphExec_t multi[2][2];
    cudaStream_t side;
    cudaEvent_t fork, join;
    cudaEvent_t lb_ev[2];  // optional events around the lattice step (timing)
    SgCtx* sg;             // learned membrane surrogate, or null (plain solver)
    const void* sg_params;
    FemCtx* fem;           // finite-element bending, or null
    float fem_k0;
    BridgeCtx* br;         // platelet-platelet bridges, or null
    const TetherCtx* tether;  // pause-time tracking, or null
    // platelets out of the ligands' reach (FarSites): per-site platelet and
    // per-platelet flag, or null without bonds
    int* site_plt;
    int* plt_far;
    int* block_plt;
    int2* plt_nodes;
    // sim_step_record / sim_step_track: copy stream and per-slot events
    // (created on first use)
    cudaStream_t rec;
    std::vector<cudaEvent_t> rec_ready, rec_freed;
    // sim_step_track: step + centroids graphs per lattice parity, writing
    // slot `parity` of trk_scratch
    double* trk_scratch;
    cudaGraphExec_t trk_exec[2];
    // sim_step_track: kLongMulti overlapped steps with their centroids, per
    // lattice parity and slot group (the groups alternate between launches)
    cudaGraphExec_t trk_multi[2][2];
};

namespace {

// Steps per multi-step graph (even: the lattice parity returns).  sim_step
// runs kLongMulti-step graphs while that many steps remain, then kMulti-step
// ones (the last step's adhesion update of a graph has no next membrane pass
// beside it, so longer graphs leave fewer of them on the critical path:
// continuous channel stepping 51.0 -> 49.4 us per step); the tracked graphs
// run kLongMulti steps.
constexpr int kMulti = 4;
constexpr int kLongMulti = 8;

// Membrane forces of the current positions (F overwritten, then the
// optional finite-element bending added).  presplit: the previous step's
// interpolation left the hi/lo split of X and cleared the per-platelet sums.
int enqueue_front(SimCtx* c, cudaStream_t s, bool presplit = false)
{
    int rc;
    if (c->sg) {
        rc = launch_membrane_remainder(c->mem, c->X, c->F, s, presplit);
        if (!rc) rc = launch_surrogate_forces(c->sg, c->sg_params, c->mem, c->F, s);
    } else {
        rc = launch_membrane_forces(c->mem, c->X, c->F, s, presplit);
    }
    // the membrane pass (plain or global-only) left the hi/lo split of X in mem->xh, xl
    if (!rc && c->fem) rc = launch_fem_forces(c->fem, c->fem_k0, c->X, c->mem->xh, c->mem->xl, c->F, 1, nullptr, s);
    return rc;
}

// Bond and bridge forces and spreading: the part of a step before the
// lattice Boltzmann update.
int enqueue_pre_lb(SimCtx* c, cudaStream_t s)
{
    int rc = PFSI_OK;
    if (c->bonds) rc = launch_bonds_forces(c->bonds, c->X, c->F, c->M, s);
    if (!rc && c->br) rc = launch_bridge_forces(c->br, c->X, c->F, c->M, s);
    if (!rc) rc = launch_ib_spread(c->lb, c->X, c->F, c->M, c->mem->chunks, c->mem->perm, c->mem->n_chunks, s);
    return rc;
}

// Interpolation and advection after the lattice step.  split_next: the
// interpolation also prepares the next membrane pass's input (see
// NextSplit), which then runs with presplit.
int enqueue_post_lb(SimCtx* c, cudaStream_t s, bool split_next = false, bool track = false)
{
    NextSplit next;
    if (split_next) {
        next.h = c->mem->xh;
        next.l = c->mem->xl;
        next.acc = c->mem->acc;
        next.nacc = 2 * c->mem->nplt;
    }
    if (track) next.part = c->mem->cpart;   // chunk sums for the platelet centroids
    return launch_ib_interp(c->lb, c->X, c->U, c->M, 1, c->mem->chunks, c->mem->perm, c->mem->n_chunks, s, next);
}

// Bond and bridge forces, spreading, the lattice step, interpolation and
// advection.
int enqueue_middle(SimCtx* c, cudaStream_t s, bool split_next = false, bool track = false)
{
    int rc = enqueue_pre_lb(c, s);
    if (!rc && c->lb_ev[0])
        rc = check_cuda(cudaEventRecordWithFlags(c->lb_ev[0], s, cudaEventRecordExternal), "sim: lb timing event");
    if (!rc) rc = launch_lb_step(c->lb, s);
    if (!rc && c->lb_ev[1])
        rc = check_cuda(cudaEventRecordWithFlags(c->lb_ev[1], s, cudaEventRecordExternal), "sim: lb timing event");
    if (!rc) rc = enqueue_post_lb(c, s, split_next, track);
    return rc;
}

// The Monte-Carlo adhesion update of the step (reads X and the bond state).
int enqueue_adhesion(SimCtx* c, cudaStream_t s)
{
    int rc = PFSI_OK;
    if (c->bonds) {
        FarSites far;
        if (c->site_plt) {
            far.site_plt = c->site_plt;
            far.plt_far = c->plt_far;
            far.block_plt = c->block_plt;
            far.plt_nodes = c->plt_nodes;
            far.nplt = c->mem->nplt;
        }
        rc = launch_bonds_step(c->bonds, c->X, c->M, 0, c->bonds->counters + 3, s, c->site_plt ? &far : nullptr);
    }
    if (!rc && c->br) rc = launch_bridges_step(c->br, c->X, c->M, 0, bridge_step_counter(c->br), s);
    // tethers after the wall update; the bond step counter now counts this step
    if (!rc && c->tether) rc = launch_tether_update(c->tether, c->bonds->counters + 3, 0, s);
    return rc;
}

int enqueue_step(SimCtx* c, cudaStream_t s, bool track = false)
{
    int rc = enqueue_front(c, s);
    if (!rc) rc = enqueue_middle(c, s, false, track);
    if (!rc) rc = enqueue_adhesion(c, s);
    return rc;
}

// n steps in which step k's adhesion update (reads X after step k, writes
// only the bond and bridge state) runs on the side stream while step k + 1's
// membrane pass (reads X, writes only F and the membrane scratch) runs on
// `s`; step k + 1's bond forces wait for it.  Step k's interpolation also
// forms the hi/lo split of its advected X (the same FP64 operations as the
// split pass) for step k + 1's membrane pass, which skips its split.  Same
// results as n single steps.
int enqueue_overlapped(SimCtx* c, cudaStream_t s, int n, double* slots = nullptr)
{
    // slots (tracked graphs): after step k the platelet centroids go to
    // slots + 4 n_plt k, formed from the chunk sums of step k's
    // interpolation; they run on the side branch with the adhesion update
    // (the last step's on the main stream)
    const size_t slot = 4 * (size_t)c->mem->nplt;
    const bool track = slots != nullptr;
    int rc = enqueue_front(c, s);
    if (!rc) rc = enqueue_middle(c, s, n > 1, track);
    for (int k = 1; k < n && !rc; ++k) {
        rc = check_cuda(cudaEventRecord(c->fork, s), "sim: fork");
        if (!rc) rc = check_cuda(cudaStreamWaitEvent(c->side, c->fork, 0), "sim: fork");
        // step k's centroids from the chunk sums its interpolation wrote (read
        // before step k + 1's interpolation rewrites them: the join comes first)
        if (!rc && track) rc = launch_centroids_from_chunks(c->mem, slots + (k - 1) * slot, c->side);
        if (!rc) rc = enqueue_adhesion(c, c->side);
        if (!rc) rc = check_cuda(cudaEventRecord(c->join, c->side), "sim: join");
        if (!rc) rc = enqueue_front(c, s, true);
        if (!rc) rc = check_cuda(cudaStreamWaitEvent(s, c->join, 0), "sim: join");
        if (!rc) rc = enqueue_middle(c, s, k + 1 < n, track);
    }
    if (!rc && track) rc = launch_centroids_from_chunks(c->mem, slots + (n - 1) * slot, s);
    if (!rc) rc = enqueue_adhesion(c, s);
    return rc;
}

int enqueue_track(SimCtx* c, cudaStream_t s, int parity)
{
    int rc = enqueue_step(c, s, true);
    if (!rc) rc = launch_centroids_from_chunks(c->mem, c->trk_scratch + (size_t)parity * 4 * c->mem->nplt, s);
    return rc;
}

// What a captured graph holds.
enum GraphKind { kOneStep, kOneStepTracked, kLongSteps, kSteps, kStepsTracked };

// Captures one step, one step plus the platelet centroids, kLongMulti or
// kMulti overlapped steps, or kLongMulti overlapped steps with their centroids
// (into slot group `group` of the tracking scratch), starting at lattice
// parity `parity`.
int capture(SimCtx* c, int parity, GraphKind kind, int group = 0)
{
    const int saved = c->lb->cur;
    c->lb->cur = parity;
    int rc = check_cuda(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal), "sim: begin capture");
    if (rc) {
        c->lb->cur = saved;
        return rc;
    }
    const int rc_enq =
        kind == kOneStepTracked ? enqueue_track(c, c->cap, parity)
        : kind == kLongSteps    ? enqueue_overlapped(c, c->cap, kLongMulti)
        : kind == kSteps        ? enqueue_overlapped(c, c->cap, kMulti)
        : kind == kStepsTracked ? enqueue_overlapped(c, c->cap, kLongMulti,
                                                     c->trk_scratch + (size_t)(2 + group * kLongMulti) * 4 * c->mem->nplt)
                                : enqueue_step(c, c->cap);
    cudaGraph_t graph = nullptr;
    rc = check_cuda(cudaStreamEndCapture(c->cap, &graph), "sim: end capture");
    c->lb->cur = saved;
    if (rc_enq) {
        if (graph) cudaGraphDestroy(graph);
        return rc_enq;
    }
    if (rc) return rc;
    cudaGraphExec_t* dst = kind == kOneStepTracked ? &c->trk_exec[parity]
                           : kind == kLongSteps    ? &c->multi[0][parity]
                           : kind == kSteps        ? &c->multi[1][parity]
                           : kind == kStepsTracked ? &c->trk_multi[parity][group]
                                                   : &c->exec[parity];
    rc = check_cuda(cudaGraphInstantiate(dst, graph, 0), "sim: instantiate");
    cudaGraphDestroy(graph);
    return rc;
}

void drop_graphs(SimCtx* c)
{
    for (int k = 0; k < 2; ++k) {
        if (c->exec[k]) cudaGraphExecDestroy(c->exec[k]);
        c->exec[k] = nullptr;
        if (c->trk_exec[k]) cudaGraphExecDestroy(c->trk_exec[k]);
        c->trk_exec[k] = nullptr;
        for (int l = 0; l < 2; ++l) {
            if (c->multi[l][k]) cudaGraphExecDestroy(c->multi[l][k]);
            c->multi[l][k] = nullptr;
        }
        for (int g = 0; g < 2; ++g) {
            if (c->trk_multi[k][g]) cudaGraphExecDestroy(c->trk_multi[k][g]);
            c->trk_multi[k][g] = nullptr;
        }
    }
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
    c->multi[0][0] = c->multi[0][1] = c->multi[1][0] = c->multi[1][1] = nullptr;
    c->trk_multi[0][0] = c->trk_multi[0][1] = c->trk_multi[1][0] = c->trk_multi[1][1] = nullptr;
    c->side = nullptr;
    c->fork = c->join = nullptr;
    c->trk_exec[0] = c->trk_exec[1] = nullptr;
    c->trk_scratch = nullptr;
    c->fem = nullptr;
    c->fem_k0 = 0.0f;
    c->br = nullptr;
    c->tether = nullptr;
    c->lb_ev[0] = c->lb_ev[1] = nullptr;
    c->site_plt = c->plt_far = c->block_plt = nullptr;
    c->plt_nodes = nullptr;
    int rc = check_cuda(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking), "sim_create: stream");
    if (!rc) rc = check_cuda(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking), "sim_create: stream");
    if (!rc) rc = check_cuda(cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming), "sim_create: event");
    if (!rc) rc = check_cuda(cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming), "sim_create: event");
    if (!rc && bonds) {
        const unsigned long long s = first_step;
        rc = check_cuda(cudaMemcpy(bonds->counters + 3, &s, sizeof(s), cudaMemcpyHostToDevice), "sim_create: step");
    }
    if (!rc && bonds && bonds->R > 0 && mem->nplt > 0) {
        rc = check_cuda(cudaMalloc(&c->site_plt, sizeof(int) * (size_t)bonds->R), "sim_create: site platelets");
        if (!rc) rc = check_cuda(cudaMalloc(&c->plt_far, sizeof(int) * (size_t)mem->nplt), "sim_create: site platelets");
        if (!rc)
            rc = check_cuda(cudaMalloc(&c->block_plt, sizeof(int) * (size_t)((bonds->R + 255) / 256)),
                            "sim_create: site platelets");
        if (!rc) rc = check_cuda(cudaMalloc(&c->plt_nodes, sizeof(int2) * (size_t)mem->nplt), "sim_create: site platelets");
        if (!rc)
            rc = launch_site_platelets(bonds, mem->node_plt, mem->n, mem->nplt, c->site_plt, c->block_plt, c->plt_nodes,
                                       c->cap);
        if (!rc) rc = check_cuda(cudaStreamSynchronize(c->cap), "sim_create: site platelets");
    }
    if (rc) {
        if (c->site_plt) cudaFree(c->site_plt);
        if (c->plt_far) cudaFree(c->plt_far);
        if (c->block_plt) cudaFree(c->block_plt);
        if (c->plt_nodes) cudaFree(c->plt_nodes);
        delete c;
        return rc;
    }
    *out = c;
    return PFSI_OK;
}

extern "C" int sim_destroy(sim_ctx* c)
{
    if (!c) return PFSI_OK;
    drop_graphs(c);
    if (c->cap) cudaStreamDestroy(c->cap);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->fork) cudaEventDestroy(c->fork);
    if (c->join) cudaEventDestroy(c->join);
    for (int k = 0; k < 2; ++k)
        if (c->lb_ev[k]) cudaEventDestroy(c->lb_ev[k]);
    for (cudaEvent_t e : c->rec_ready) cudaEventDestroy(e);
    for (cudaEvent_t e : c->rec_freed) cudaEventDestroy(e);
    if (c->rec) cudaStreamDestroy(c->rec);
    if (c->site_plt) cudaFree(c->site_plt);
    if (c->plt_far) cudaFree(c->plt_far);
    if (c->block_plt) cudaFree(c->block_plt);
    if (c->plt_nodes) cudaFree(c->plt_nodes);
    delete c;
    return PFSI_OK;
}

extern "C" int sim_step(sim_ctx* c, int nsteps, void* stream)
{
    NvtxRange nvtx_range("sim_step");
    if (!c || nsteps < 0) return set_error(PFSI_ERR_ARG, "sim_step: bad argument");
    cudaStream_t s = as_stream(stream);
    int k = 0;
    // kMulti steps per graph launch (not while the lattice step is being
    // timed: those events belong to single steps)
    while (!c->lb_ev[0] && nsteps - k >= kMulti) {
        const int parity = c->lb->cur;
        const int l = nsteps - k >= kLongMulti ? 0 : 1;
        const int len = l == 0 ? kLongMulti : kMulti;
        if (!c->multi[l][parity]) {
            const int rc = capture(c, parity, l == 0 ? kLongSteps : kSteps);
            if (rc) return rc;
        }
        const int rc = check_cuda(cudaGraphLaunch(c->multi[l][parity], s), "sim_step: graph launch");
        if (rc) return rc;
        c->step += len;   // even: the lattice parity is unchanged
        k += len;
    }
    for (; k < nsteps; ++k) {
        const int parity = c->lb->cur;
        if (!c->exec[parity]) {
            const int rc = capture(c, parity, kOneStep);
            if (rc) return rc;
        }
        const int rc = check_cuda(cudaGraphLaunch(c->exec[parity], s), "sim_step: graph launch");
        if (rc) return rc;
        c->lb->cur ^= 1;
        c->step += 1;
    }
    return PFSI_OK;
}

extern "C" int sim_step_record(sim_ctx* c, int nsteps, double* dev_ring, double* host_ring, int ring, void* stream)
{
    NvtxRange nvtx_range("sim_step_record");
    if (!c || nsteps < 0 || !dev_ring || !host_ring || ring < 2 || ring > 64)
        return set_error(PFSI_ERR_ARG, "sim_step_record: bad argument");
    if (!aligned(dev_ring, 8) || !aligned(host_ring, 8)) return set_error(PFSI_ERR_ARG, "sim_step_record: misaligned ring");
    cudaStream_t s = as_stream(stream);
    int rc = PFSI_OK;
    if (!c->rec) rc = check_cuda(cudaStreamCreateWithFlags(&c->rec, cudaStreamNonBlocking), "sim_step_record: stream");
    while (!rc && (int)c->rec_ready.size() < ring) {
        cudaEvent_t a = nullptr, b = nullptr;
        rc = check_cuda(cudaEventCreateWithFlags(&a, cudaEventDisableTiming), "sim_step_record: event");
        if (!rc) rc = check_cuda(cudaEventCreateWithFlags(&b, cudaEventDisableTiming), "sim_step_record: event");
        if (!rc) {
            c->rec_ready.push_back(a);
            c->rec_freed.push_back(b);
        }
    }
    if (rc) return rc;
    const size_t bytes = (size_t)3 * c->M * sizeof(double);
    for (int k = 0; k < nsteps && !rc; ++k) {
        const int b = k % ring;
        rc = sim_step(c, 1, stream);
        if (!rc && k >= ring) rc = check_cuda(cudaStreamWaitEvent(s, c->rec_freed[b], 0), "sim_step_record: wait");
        double* snap = dev_ring + (size_t)b * 3 * c->M;
        if (!rc) rc = check_cuda(cudaMemcpyAsync(snap, c->X, bytes, cudaMemcpyDeviceToDevice, s), "sim_step_record: snapshot");
        if (!rc) rc = check_cuda(cudaEventRecord(c->rec_ready[b], s), "sim_step_record: record");
        if (!rc) rc = check_cuda(cudaStreamWaitEvent(c->rec, c->rec_ready[b], 0), "sim_step_record: wait");
        if (!rc)
            rc = check_cuda(cudaMemcpyAsync(host_ring + (size_t)b * 3 * c->M, snap, bytes, cudaMemcpyDeviceToHost, c->rec),
                            "sim_step_record: copy");
        if (!rc) rc = check_cuda(cudaEventRecord(c->rec_freed[b], c->rec), "sim_step_record: record");
    }
    // the caller's stream covers the last copies
    for (int b = 0; b < ring && b < nsteps && !rc; ++b)
        rc = check_cuda(cudaStreamWaitEvent(s, c->rec_freed[b], 0), "sim_step_record: join");
    return rc;
}

extern "C" int sim_step_track(sim_ctx* c, int nsteps, double* dev_scratch, double* host_out, void* stream)
{
    NvtxRange nvtx_range("sim_step_track");
    if (!c || nsteps < 0 || !dev_scratch || !host_out) return set_error(PFSI_ERR_ARG, "sim_step_track: bad argument");
    if (!aligned(dev_scratch, 8) || !aligned(host_out, 8)) return set_error(PFSI_ERR_ARG, "sim_step_track: misaligned buffer");
    cudaStream_t s = as_stream(stream);
    int rc = PFSI_OK;
    if (c->trk_scratch != dev_scratch) {
        for (int k = 0; k < 2; ++k) {
            if (c->trk_exec[k]) cudaGraphExecDestroy(c->trk_exec[k]);
            c->trk_exec[k] = nullptr;
            for (int g = 0; g < 2; ++g) {
                if (c->trk_multi[k][g]) cudaGraphExecDestroy(c->trk_multi[k][g]);
                c->trk_multi[k][g] = nullptr;
            }
        }
        c->trk_scratch = dev_scratch;
    }
    if (!c->rec) rc = check_cuda(cudaStreamCreateWithFlags(&c->rec, cudaStreamNonBlocking), "sim_step_track: stream");
    while (!rc && c->rec_ready.size() < 4) {
        cudaEvent_t a = nullptr, b = nullptr;
        rc = check_cuda(cudaEventCreateWithFlags(&a, cudaEventDisableTiming), "sim_step_track: event");
        if (!rc) rc = check_cuda(cudaEventCreateWithFlags(&b, cudaEventDisableTiming), "sim_step_track: event");
        if (!rc) {
            c->rec_ready.push_back(a);
            c->rec_freed.push_back(b);
        }
    }
    const int nplt = c->mem->nplt;
    const size_t bytes = (size_t)3 * nplt * sizeof(double);
    const size_t slot = (size_t)4 * nplt;
    // events 0, 1: single-step slots 0, 1; events 2, 3: slot groups 0, 1
    bool used[4] = {false, false, false, false};
    int k = 0, group = 0;
    while (!rc && !c->lb_ev[0] && nsteps - k >= kLongMulti) {
        const int p = c->lb->cur;   // unchanged by kLongMulti (even) steps
        if (!c->trk_multi[p][group]) rc = capture(c, p, kStepsTracked, group);
        cudaEvent_t ready = c->rec_ready[2 + group], freed = c->rec_freed[2 + group];
        if (!rc && used[2 + group]) rc = check_cuda(cudaStreamWaitEvent(s, freed, 0), "sim_step_track: wait");
        if (!rc) rc = check_cuda(cudaGraphLaunch(c->trk_multi[p][group], s), "sim_step_track: graph launch");
        if (!rc) rc = check_cuda(cudaEventRecord(ready, s), "sim_step_track: record");
        if (!rc) rc = check_cuda(cudaStreamWaitEvent(c->rec, ready, 0), "sim_step_track: wait");
        // the kLongMulti steps' centroids: strided slots -> consecutive host rows
        if (!rc)
            rc = check_cuda(cudaMemcpy2DAsync(host_out + (size_t)k * 3 * nplt, bytes,
                                              dev_scratch + (2 + (size_t)group * kLongMulti) * slot, slot * sizeof(double),
                                              bytes, kLongMulti, cudaMemcpyDeviceToHost, c->rec),
                            "sim_step_track: copy");
        if (!rc) rc = check_cuda(cudaEventRecord(freed, c->rec), "sim_step_track: record");
        used[2 + group] = true;
        c->step += kLongMulti;
        k += kLongMulti;
        group ^= 1;
    }
    for (; k < nsteps && !rc; ++k) {
        const int p = c->lb->cur;   // the step's graph writes slot p of the scratch
        if (!c->trk_exec[p]) rc = capture(c, p, kOneStepTracked);
        if (!rc && used[p]) rc = check_cuda(cudaStreamWaitEvent(s, c->rec_freed[p], 0), "sim_step_track: wait");
        if (!rc) rc = check_cuda(cudaGraphLaunch(c->trk_exec[p], s), "sim_step_track: graph launch");
        if (!rc) rc = check_cuda(cudaEventRecord(c->rec_ready[p], s), "sim_step_track: record");
        if (!rc) rc = check_cuda(cudaStreamWaitEvent(c->rec, c->rec_ready[p], 0), "sim_step_track: wait");
        if (!rc)
            rc = check_cuda(cudaMemcpyAsync(host_out + (size_t)k * 3 * nplt, dev_scratch + (size_t)p * slot, bytes,
                                            cudaMemcpyDeviceToHost, c->rec),
                            "sim_step_track: copy");
        if (!rc) rc = check_cuda(cudaEventRecord(c->rec_freed[p], c->rec), "sim_step_track: record");
        used[p] = true;
        if (!rc) {
            c->lb->cur ^= 1;
            c->step += 1;
        }
    }
    for (int b = 0; b < 4 && !rc; ++b)
        if (used[b]) rc = check_cuda(cudaStreamWaitEvent(s, c->rec_freed[b], 0), "sim_step_track: join");
    return rc;
}


namespace pfsi {
namespace {
__global__ void k_sim_check_x(const double* __restrict__ X, int n3, unsigned long long* __restrict__ cnt)
{
    unsigned long long c = 0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n3; t += gridDim.x * blockDim.x) c += !coord_in_range(X[t]);
    if (c) atomicAdd(cnt, c);
}
}  // namespace
}  // namespace pfsi

extern "C" int sim_check(sim_ctx* c, float u_max, unsigned long long* dev_scratch4, long long* out_host, void* stream)
{
    NvtxRange nvtx_range("sim_check");
    if (!c || !dev_scratch4 || !out_host) return set_error(PFSI_ERR_ARG, "sim_check: bad argument");
    const int rc_lb = lb_check(static_cast<lb_ctx*>(c->lb), u_max, dev_scratch4, out_host, stream);
    if (rc_lb != PFSI_OK && rc_lb != PFSI_ERR_UNSTABLE) return rc_lb;
    cudaStream_t s = as_stream(stream);
    int rc = check_cuda(cudaMemsetAsync(dev_scratch4 + 3, 0, sizeof(unsigned long long), s), "sim_check: clear");
    const int n3 = 3 * c->M;
    const int blocks = (n3 + 255) / 256 < 148 * 8 ? (n3 + 255) / 256 : 148 * 8;
    if (!rc && n3 > 0) {
        k_sim_check_x<<<blocks, 256, 0, s>>>(c->X, n3, dev_scratch4 + 3);
        rc = check_launch("sim_check");
    }
    unsigned long long h = 0;
    if (!rc) rc = check_cuda(cudaMemcpyAsync(&h, dev_scratch4 + 3, sizeof(h), cudaMemcpyDeviceToHost, s), "sim_check: copy");
    if (!rc) rc = check_cuda(cudaStreamSynchronize(s), "sim_check: synchronise");
    if (rc) return rc;
    out_host[3] = (long long)h;
    if (h)
        return set_error(PFSI_ERR_UNSTABLE,
                         "sim_check: " + std::to_string(h) + " node coordinates non-finite or beyond 1e8 lattice units");
    return rc_lb;
}

extern "C" int sim_set_fem_bending(sim_ctx* c, fem_ctx* fem, float k0)
{
    if (!c) return set_error(PFSI_ERR_ARG, "sim_set_fem_bending: bad argument");
    FemCtx* f = fem_internal(fem);
    if (f && fem_node_count(f) != c->M) return set_error(PFSI_ERR_ARG, "sim_set_fem_bending: node count differs");
    drop_graphs(c);
    c->fem = f;
    c->fem_k0 = k0;
    return PFSI_OK;
}

extern "C" int sim_set_bridges(sim_ctx* c, bridge_ctx* br)
{
    if (!c) return set_error(PFSI_ERR_ARG, "sim_set_bridges: bad argument");
    BridgeCtx* b = bridge_internal(br);
    if (b && bridge_bonds(b) != c->bonds)
        return set_error(PFSI_ERR_ARG, "sim_set_bridges: bridges not built on the simulation's bonds");
    drop_graphs(c);
    c->br = b;
    if (b) {
        const unsigned long long step = c->step;
        return check_cuda(cudaMemcpy(bridge_step_counter(b), &step, sizeof(step), cudaMemcpyHostToDevice),
                          "sim_set_bridges: step counter");
    }
    return PFSI_OK;
}

extern "C" int sim_set_tether(sim_ctx* c, tether_ctx* tr)
{
    if (!c) return set_error(PFSI_ERR_ARG, "sim_set_tether: null context");
    const TetherCtx* t = tether_internal(tr);
    if (t && (!c->bonds || t->bonds != c->bonds))
        return set_error(PFSI_ERR_ARG, "sim_set_tether: tracker not built on the simulation's bonds");
    drop_graphs(c);
    c->tether = t;
    return PFSI_OK;
}

extern "C" int sim_set_surrogate(sim_ctx* c, sg_ctx* sg, const void* params)
{
    if (!c || (sg && !params)) return set_error(PFSI_ERR_ARG, "sim_set_surrogate: bad argument");
    SgCtx* g = sg ? sg_internal(sg) : nullptr;
    if (g && sg_node_count(g) != c->M) return set_error(PFSI_ERR_ARG, "sim_set_surrogate: node count differs");
    drop_graphs(c);
    c->sg = g;
    c->sg_params = params;
    return PFSI_OK;
}

extern "C" int sim_time_lb(sim_ctx* c, int on)
{
    if (!c) return set_error(PFSI_ERR_ARG, "sim_time_lb: null context");
    const bool want = on != 0;
    if (want == (c->lb_ev[0] != nullptr)) return PFSI_OK;
    drop_graphs(c);
    for (int k = 0; k < 2; ++k) {
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
// chamber.  The chambers are dealt into groups of about equal cell counts;
// each group is an independent chain of the graph.  In a plain group (no
// chamber with a learned surrogate, finite-element bending, bridges or
// tethers) every kernel of a step is ONE launch for all the group's
// chambers (Multi lists; the lattice update as one batched launch per
// storage mode, LbBatch), so a step of any number of chambers is about a
// dozen kernel nodes.  Otherwise each chamber's kernels before the lattice
// update run on a branch of their own, the branches join, the batched
// lattice launch runs, and each chamber's interpolation and adhesion update
// run on branches again; the branch streams have the greatest priority and
// the lattice launches the least (the graph keeps both), so the block
// scheduler gives a freed SM slot to a waiting small kernel first.  Per
// chamber chains (no groups) keep each chamber's whole step, its own
// lattice launch included, on its branch.
namespace pfsi {

struct BatchCtx {
    std::vector<SimCtx*> sims;
    int k;
    std::vector<cudaStream_t> streams;   // per chamber
    std::vector<cudaEvent_t> join;       // per chamber
    cudaStream_t cap;
    cudaEvent_t fork;
    cudaGraphExec_t exec[2];
    int blocks_per_sm;                   // lattice launches' grid (0: every resident block)
    std::vector<std::vector<int>> group; // chambers of each group, in batch order
    std::vector<LbBatch*> lb;            // per group
    std::vector<cudaStream_t> gs;        // per group's chain (group 0: cap)
    std::vector<cudaEvent_t> gjoin;      // per group
};

namespace {

// Chamber groups of a new batch (batch_set_layout changes them).
constexpr int kBatchGroups = 1;

void batch_drop_graphs(BatchCtx* b)
{
    for (int k = 0; k < 2; ++k)
        if (b->exec[k]) {
            cudaGraphExecDestroy(b->exec[k]);
            b->exec[k] = nullptr;
        }
}

void batch_drop_groups(BatchCtx* b)
{
    for (LbBatch* l : b->lb) lb_batch_free(l);
    for (size_t g = 1; g < b->gs.size(); ++g) cudaStreamDestroy(b->gs[g]);
    for (cudaEvent_t e : b->gjoin) cudaEventDestroy(e);
    b->lb.clear();
    b->gs.clear();
    b->gjoin.clear();
    b->group.clear();
}

void batch_free(BatchCtx* b)
{
    batch_drop_graphs(b);
    batch_drop_groups(b);
    for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->join) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->cap) cudaStreamDestroy(b->cap);
}

// Deals the chambers into `groups` groups (largest lattice first, each to
// the group with the fewest cells so far) and builds each group's lattice
// batch, chain stream and join event.
int batch_make_groups(BatchCtx* b, int groups, int blocks_per_sm)
{
    batch_drop_graphs(b);
    batch_drop_groups(b);
    const int n = (int)b->sims.size();
    b->blocks_per_sm = blocks_per_sm;
    if (groups == 0) return PFSI_OK;   // per-chamber chains (see batch_capture)
    groups = std::min(groups, n);
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->sims[x]->lb->N > b->sims[y]->lb->N; });
    std::vector<long long> load(groups, 0);
    std::vector<int> owner(n);
    for (int i : order) {
        const int g = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        owner[i] = g;
        load[g] += b->sims[i]->lb->N;
    }
    b->group.assign(groups, {});
    for (int i = 0; i < n; ++i) b->group[owner[i]].push_back(i);
    int least = 0, greatest = 0;
    int rc = check_cuda(cudaDeviceGetStreamPriorityRange(&least, &greatest), "batch: priorities");
    for (int g = 0; g < groups && !rc; ++g) {
        std::vector<LbCtx*> lat;
        for (int i : b->group[g]) lat.push_back(b->sims[i]->lb);
        LbBatch* l = nullptr;
        rc = lb_batch_build(lat.data(), (int)lat.size(), &l);
        if (rc) break;
        b->lb.push_back(l);
        rc = lb_batch_configure_grid(l, blocks_per_sm, least);
        cudaStream_t st = b->cap;
        if (!rc && g > 0) rc = check_cuda(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "batch: stream");
        if (rc) break;
        b->gs.push_back(st);
        cudaEvent_t e = nullptr;
        rc = check_cuda(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "batch: event");
        if (!rc) b->gjoin.push_back(e);
    }
    return rc;
}

// The branches of one phase of group g: fork from the group's chain stream,
// `phase` on each of its chambers' streams, join back.
template <typename Phase>
int batch_branches(BatchCtx* b, int g, Phase phase)
{
    cudaStream_t chain = b->gs[g];
    int rc = check_cuda(cudaEventRecord(b->fork, chain), "batch: fork");
    for (int i : b->group[g]) {
        if (rc) break;
        rc = check_cuda(cudaStreamWaitEvent(b->streams[i], b->fork, 0), "batch: branch");
        if (!rc) rc = phase(b->sims[i], b->streams[i]);
        if (!rc) rc = check_cuda(cudaEventRecord(b->join[i], b->streams[i]), "batch: join");
        if (!rc) rc = check_cuda(cudaStreamWaitEvent(chain, b->join[i], 0), "batch: join");
    }
    return rc;
}

int batch_capture(BatchCtx* b, int parity)
{
    std::vector<int> saved;
    for (SimCtx* c : b->sims) {
        saved.push_back(c->lb->cur);
        c->lb->cur = parity;
    }
    const int groups = (int)b->group.size();
    int rc = check_cuda(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "batch: begin capture");
    int rc_enq = PFSI_OK;
    if (!rc) {
        rc_enq = check_cuda(cudaEventRecord(b->fork, b->cap), "batch: fork");
        // no groups: each chamber's whole step chain (its own lattice
        // launch included) on its branch
        for (size_t i = 0; i < b->sims.size() && groups == 0 && !rc_enq; ++i) {
            rc_enq = check_cuda(cudaStreamWaitEvent(b->streams[i], b->fork, 0), "batch: branch");
            for (int s = 0; s < b->k && !rc_enq; ++s) rc_enq = enqueue_step(b->sims[i], b->streams[i]);
            if (!rc_enq) rc_enq = check_cuda(cudaEventRecord(b->join[i], b->streams[i]), "batch: join");
            if (!rc_enq) rc_enq = check_cuda(cudaStreamWaitEvent(b->cap, b->join[i], 0), "batch: join");
        }
        for (int g = 1; g < groups && !rc_enq; ++g)
            rc_enq = check_cuda(cudaStreamWaitEvent(b->gs[g], b->fork, 0), "batch: group");
        // plain groups (no surrogate, finite-element bending, bridges or
        // tethers in any chamber) launch every kernel once for all chambers
        std::vector<std::vector<Chamber>> plain(groups);
        for (int g = 0; g < groups; ++g) {
            for (int i : b->group[g]) {
                const SimCtx* c = b->sims[i];
                if (c->sg || c->fem || c->br || c->tether) {
                    plain[g].clear();
                    break;
                }
                plain[g].push_back(Chamber{c->lb, c->mem, c->bonds, c->X, c->F, c->U, c->M});
            }
        }
        for (int s = 0; s < b->k && !rc_enq; ++s)
            for (int g = 0; g < groups && !rc_enq; ++g) {
                if (!plain[g].empty()) {
                    const Chamber* ch = plain[g].data();
                    const int n = (int)plain[g].size();
                    cudaStream_t st = b->gs[g];
                    rc_enq = launch_membrane_forces_multi(ch, n, st);
                    if (!rc_enq) rc_enq = launch_bonds_forces_multi(ch, n, st);
                    if (!rc_enq) rc_enq = launch_ib_spread_multi(ch, n, st);
                    if (!rc_enq) rc_enq = launch_lb_batch(b->lb[g], st);
                    if (!rc_enq) rc_enq = launch_ib_interp_multi(ch, n, st);
                    if (!rc_enq) rc_enq = launch_bonds_step_multi(ch, n, st);
                    continue;
                }
                rc_enq = batch_branches(b, g, [](SimCtx* c, cudaStream_t st) {
                    int r = enqueue_front(c, st);
                    if (!r) r = enqueue_pre_lb(c, st);
                    return r;
                });
                if (!rc_enq) rc_enq = launch_lb_batch(b->lb[g], b->gs[g]);   // advances the group's parities
                if (!rc_enq)
                    rc_enq = batch_branches(b, g, [](SimCtx* c, cudaStream_t st) {
                        int r = enqueue_post_lb(c, st);
                        if (!r) r = enqueue_adhesion(c, st);
                        return r;
                    });
            }
        for (int g = 1; g < groups && !rc_enq; ++g) {
            rc_enq = check_cuda(cudaEventRecord(b->gjoin[g], b->gs[g]), "batch: group join");
            if (!rc_enq) rc_enq = check_cuda(cudaStreamWaitEvent(b->cap, b->gjoin[g], 0), "batch: group join");
        }
        cudaGraph_t graph = nullptr;
        rc = check_cuda(cudaStreamEndCapture(b->cap, &graph), "batch: end capture");
        if (!rc && !rc_enq)
            rc = check_cuda(cudaGraphInstantiateWithFlags(&b->exec[parity], graph, cudaGraphInstantiateFlagUseNodePriority),
                            "batch: instantiate");
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
    int least = 0, greatest = 0;
    int rc = check_cuda(cudaDeviceGetStreamPriorityRange(&least, &greatest), "batch_create: priorities");
    if (!rc) rc = check_cuda(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking), "batch_create: stream");
    if (!rc) rc = check_cuda(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), "batch_create: event");
    for (int i = 0; i < n && !rc; ++i) {
        b->sims.push_back(sims[i]);
        cudaStream_t s = nullptr;
        cudaEvent_t e = nullptr;
        rc = check_cuda(cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, greatest), "batch_create: stream");
        if (!rc) b->streams.push_back(s);
        if (!rc) rc = check_cuda(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "batch_create: event");
        if (!rc) b->join.push_back(e);
    }
    if (!rc) rc = batch_make_groups(b, kBatchGroups, 0);
    if (rc) {
        batch_free(b);
        delete b;
        return rc;
    }
    *out = b;
    return PFSI_OK;
}

extern "C" int batch_set_layout(batch_ctx* b, int groups, int blocks_per_sm)
{
    if (!b || groups < 0 || blocks_per_sm < 0) return set_error(PFSI_ERR_ARG, "batch_set_layout: bad argument");
    return batch_make_groups(b, groups, blocks_per_sm);
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
    NvtxRange nvtx_range("batch_step");
    if (!b || nsteps < 0 || nsteps % b->k) return set_error(PFSI_ERR_ARG, "batch_step: nsteps must be a multiple of steps_per_graph");
    cudaStream_t s = as_stream(stream);
    for (int done = 0; done < nsteps; done += b->k) {
        const int parity = b->sims[0]->lb->cur;
        for (SimCtx* c : b->sims)
            if (c->lb->cur != parity)
                return set_error(PFSI_ERR_ARG, "batch_step: a chamber was stepped on its own (parities differ)");
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

extern "C" int batch_autotune(batch_ctx* b, int reps, void* stream, float* lb_ms_per_step)
{
    NvtxRange nvtx_range("batch_autotune");
    if (!b) return set_error(PFSI_ERR_ARG, "batch_autotune: null batch");
    float total = 0.f;
    int rc = PFSI_OK;
    for (LbBatch* l : b->lb) {
        float ms = 0.f;
        if (!rc) rc = lb_batch_tune(l, reps, as_stream(stream), &ms);
        total += ms;
    }
    batch_drop_graphs(b);   // the kernel nodes hold the old tile counts
    if (!rc && lb_ms_per_step) *lb_ms_per_step = total;
    return rc;
}
