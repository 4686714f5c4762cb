// pfsi_internal.cuh -- internal declarations shared by the CUDA translation
// units of the platelet fluid-structure library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/platelet_fsi.h"

namespace pfsi {

// ---------------------------------------------------------------- errors
int set_error(int code, const std::string& msg);
int check_cuda(cudaError_t e, const char* what);
int check_launch(const char* what);

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// NVTX range over a C-ABI call (visible to nsys and ncu's NVTX filters; a
// pointer check when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
inline bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// ---------------------------------------------------------------- dependent launch
// The kernels of the coupled step are launched with programmatic stream
// serialisation: a kernel's grid is dispatched as soon as the blocks of its
// predecessor in the stream (or graph) have exited, without waiting for the
// predecessor's completion to be processed, and the kernel itself calls
// pdl_wait() before its first global memory access.  pdl_wait() returns once
// all prerequisite grids have completed and their writes are visible, so the
// data dependencies are those of a plain launch; only dispatch overlaps the
// boundary (continuous channel stepping 59.2 -> 56.3 us per step).  No kernel
// triggers its successor early: blocks dispatched ahead and held in the wait
// made the 500-platelet step 12 % slower.  A no-op for a kernel launched
// without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... P, typename... A>
inline cudaError_t launch_pdl(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A&&... args)
{
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

// ---------------------------------------------------------------- multi-chamber launches
// A batch of chambers runs each of its kernels as ONE launch over all of
// them: entry e of the launch's list owns the blocks first[e] <= b <
// first[e + 1] of the grid and holds that chamber's arguments, and the
// kernel body sees b - first[e] as its block index.  The list travels as a
// kernel parameter (__grid_constant__, read through the constant bank), at
// most kMax entries per launch (a longer batch takes several launches).
template <class A, int kMax = 64>
struct Multi {
    static constexpr int Max = kMax;
    int n = 0;
    int first[kMax + 1] = {0};
    A a[kMax];
    bool full() const { return n == kMax; }
    void add(const A& args, int blocks)
    {
        a[n] = args;
        first[n + 1] = first[n] + blocks;
        ++n;
    }
    int blocks() const { return first[n]; }
};

// Entry of block b (binary search; entries own at least one block).
template <class A, int kMax>
__device__ __forceinline__ int multi_entry(const Multi<A, kMax>& t, int b)
{
    int lo = 0, hi = t.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (t.first[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Adds (args, blocks) to the last list of `lists` (a new one when it is full
// or there is none); entries of zero blocks are left out.
template <class A, int kMax>
inline void multi_push(std::vector<Multi<A, kMax>>& lists, const A& args, int blocks)
{
    if (blocks <= 0) return;
    if (lists.empty() || lists.back().full()) lists.emplace_back();
    lists.back().add(args, blocks);
}

// ---------------------------------------------------------------- D3Q19
// Directions in the paper's numbering (0-based), fixed by Eq. 23-30:
// 0..5 = +x,-x,+y,-y,+z,-z; 6..17 face diagonals; 18 rest.  constexpr
// functions so that unrolled loops fold them to immediates.
__host__ __device__ __forceinline__ constexpr int cxq(int q)
{
    return (q == 0 || q == 6 || q == 7 || q == 8 || q == 9)        ? 1
           : (q == 1 || q == 10 || q == 11 || q == 12 || q == 13) ? -1
                                                                   : 0;
}
__host__ __device__ __forceinline__ constexpr int cyq(int q)
{
    return (q == 2 || q == 6 || q == 10 || q == 14 || q == 15)     ? 1
           : (q == 3 || q == 7 || q == 11 || q == 16 || q == 17) ? -1
                                                                  : 0;
}
__host__ __device__ __forceinline__ constexpr int czq(int q)
{
    return (q == 4 || q == 8 || q == 12 || q == 14 || q == 16)     ? 1
           : (q == 5 || q == 9 || q == 13 || q == 15 || q == 17) ? -1
                                                                  : 0;
}
__host__ __device__ __forceinline__ constexpr int oppq(int q)
{
    return q == 18 ? 18
           : q < 6 ? (q ^ 1)
           : q == 6 ? 11 : q == 11 ? 6 : q == 7 ? 10 : q == 10 ? 7
           : q == 8 ? 13 : q == 13 ? 8 : q == 9 ? 12 : q == 12 ? 9
           : q == 14 ? 17 : q == 17 ? 14 : q == 15 ? 16 : 15;
}
// Eq. 21 weights
__host__ __device__ __forceinline__ constexpr float wq(int q)
{
    return q < 6 ? (1.0f / 18.0f) : q < 18 ? (1.0f / 36.0f) : (1.0f / 3.0f);
}

// On-site velocity wall (Eq. 23-30, Hecht and Harting) on shifted
// populations f~ = f - w: s = +1 at the bottom (k = 0), -1 at the top
// (k = nz - 1, the mirror image); the populations with c_z = s entering the
// fluid are set from the known ones so that the node carries the wall
// velocity vw.  With the shift, rho = (1 + S~)/(1 - s vz), S~ = sum over
// c_z = 0 of f~ + 2 sum over c_z = -s of f~ (the weights of those sets add up
// to 1), and N_x = 1/2 sum over c_z = 0 of c_x f~ - rho vx / 3 (Eq. 29).
template <int s>
__device__ __forceinline__ void onsite_wall(float* f, float3 vw)
{
    float S = 0.f, jx = 0.f, jy = 0.f;
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        if (czq(q) == 0) {
            S += f[q];
            if (cxq(q)) jx += cxq(q) * f[q];
            if (cyq(q)) jy += cyq(q) * f[q];
        } else if (czq(q) == -s) {
            S += 2.0f * f[q];
        }
    }
    const float rho = (1.0f + S) / (1.0f - s * vw.z);
    const float Nx = fmaf(rho * vw.x, -1.0f / 3.0f, 0.5f * jx);
    const float Ny = fmaf(rho * vw.y, -1.0f / 3.0f, 0.5f * jy);
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        if (czq(q) != s) continue;
        const float cv = cxq(q) * vw.x + cyq(q) * vw.y + czq(q) * vw.z;
        if (cxq(q) == 0 && cyq(q) == 0)
            f[q] = f[oppq(q)] + rho * cv * (1.0f / 3.0f);
        else
            f[q] = f[oppq(q)] + rho * cv * (1.0f / 6.0f) - cxq(q) * Nx - cyq(q) * Ny;
    }
}

// Mixed storage keeps a cell's 19 stored values in slot order, grouped by
// c_z so that each group of a plane is one contiguous block of the [slot][cell]
// array: slots 0..8 the directions with c_z = 0, 9..13 those with c_z = +1,
// 14..18 their opposites in the same order (slot 14 + i holds the opposite
// of slot 9 + i).
__host__ __device__ __forceinline__ constexpr int nslot(int q)
{
    return q <= 3 ? q
           : q == 6 ? 4 : q == 7 ? 5 : q == 10 ? 6 : q == 11 ? 7 : q == 18 ? 8
           : q == 4 ? 9 : q == 8 ? 10 : q == 12 ? 11 : q == 14 ? 12 : q == 16 ? 13
           : q == 5 ? 14 : q == 13 ? 15 : q == 9 ? 16 : q == 17 ? 17 : 18;
}

// Mixed storage (16-bit f*neq): a population is split as f*_q = E_q(m) +
// stored_q, with the moment record m = (v, rho - 1) of its cell and
// E_q = w_q (P + c.J + (c.J)^2 / 2), J = 3 rho v, P = rho - 1 - 1.5 rho v.v.
// E_q differs from the equilibrium of Eq. 20 only by w_q rho (1 - rho)
// (3 c.v)^2 / 2; the collision (which uses the equilibrium of Eq. 20) writes
// f*_q - E_q.  Every kernel that rebuilds populations uses these two
// functions, so the split is the same everywhere.
// record (v, rho - 1) -> (P, J): P = rho - 1 - 1.5 rho v.v, J = 3 rho v.
__device__ __forceinline__ float4 split_record(float4 m)
{
    const float r3 = fmaf(3.0f, m.w, 3.0f);
    const float vv = fmaf(m.x, m.x, fmaf(m.y, m.y, m.z * m.z));
    return make_float4(fmaf(-0.5f * r3, vv, m.w), r3 * m.x, r3 * m.y, r3 * m.z);
}

// c_q . (x, y, z) with the nonzero terms only (a sum started from 0.f would
// keep an addition for the sign of zero)
template <int q>
__device__ __forceinline__ float cdot(float x, float y, float z)
{
    constexpr int cx = cxq(q), cy = cyq(q), cz = czq(q);
    const float a = cx > 0 ? x : -x, b = cy > 0 ? y : -y, c = cz > 0 ? z : -z;
    if (cx != 0 && cy != 0) return a + b;
    if (cx != 0 && cz != 0) return a + c;
    if (cy != 0 && cz != 0) return b + c;
    if (cx != 0) return a;
    if (cy != 0) return b;
    if (cz != 0) return c;
    return 0.f;
}

// E_q / w_q of a record: P + c.J + (c.J)^2 / 2
template <int q>
__device__ __forceinline__ float split_eq(float4 r)
{
    const float cj = cdot<q>(r.y, r.z, r.w);
    return fmaf(cj, fmaf(cj, 0.5f, 1.0f), r.x);
}

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds, multipliers 0xD2511F53,
// 0xCD9E8D57, key schedule by the Weyl constants 0x9E3779B9, 0xBB67AE85.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}
// 53-bit uniform in [0,1) for (site, step, purpose) under key `seed`.
__device__ __forceinline__ double uniform53(uint64_t seed, uint32_t site, uint64_t step,
                                            uint32_t purpose)
{
    const uint4 r = philox4x32_10(make_uint4(site, (uint32_t)step, (uint32_t)(step >> 32), purpose),
                                  make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    const uint64_t bits = ((uint64_t)r.x << 21) | (uint64_t)(r.y >> 11);
    return (double)bits * 0x1.0p-53;
}

// ---------------------------------------------------------------- contexts
struct LbCtx {
    lb_params p;
    long long N;
    void* f[2];          // populations: FP32 shifted f - w, or 16-bit f^neq (mixed storage)
    int cur;             // index of the buffer holding the current state
    float4* g;
    float4* v;           // FP32 storage: (v, rho) written in forced rows
    float4* m[2];        // mixed storage: (v, rho - 1) of every cell, with f[]
    uint32_t* flags;
    int shape;           // launch shape of lb_step (0: default), see lb_set_shape
    struct LbTma* tma;   // mixed storage: tensor maps of the TMA-staged kernel (lb_tma.cu), or null
};

// TMA-staged step of the mixed storage (lb_tma.cu): usable when the row
// pitch of the 16-bit tensor is a multiple of 16 bytes (nx % 8 == 0).
bool lb_tma_supported(const LbCtx* c);
struct LbTma* lb_tma_create(const LbCtx* c);   // null if unsupported or the driver lacks TMA encoding
void lb_tma_destroy(struct LbTma* t);
// tile: 0 = 32 x 8 columns, 1 = 32 x 4
cudaError_t lb_tma_launch(const LbCtx* c, const struct LbTma* t, int tile, cudaStream_t s, float omega, float guo,
                          float3 body, float3 utop, float inv_scale);
// bit 0: a bounded wait of the TMA-staged kernel gave up (since the last clear)
int lb_tma_status(unsigned int* out, bool clear);

// Batched lattice step (lb.cu): one persistent launch per storage kind walks
// the tile list of every chamber of the batch.
struct LbBatch;
int lb_batch_build(LbCtx* const* lat, int n, LbBatch** out);
void lb_batch_free(LbBatch* b);
int launch_lb_batch(LbBatch* b, cudaStream_t s);      // one step of every chamber (parities advance)
int lb_batch_tune(LbBatch* b, int reps, cudaStream_t s, float* ms_out);   // state unchanged
int lb_batch_shapes(const LbBatch* b, int* shapes);   // per chamber; -1 for FP32 chambers
int lb_batch_assign_shapes(LbBatch* b, const int* shapes);
// grid of blocks_per_sm blocks per SM (0: every resident block); launch priority
int lb_batch_configure_grid(LbBatch* b, int blocks_per_sm, int priority);

// Velocity field the interpolation reads after a lattice step.
inline float4* velocity_field(const LbCtx* c) { return c->p.storage ? c->m[c->cur] : c->v; }

struct MemCtx {
    mem_params p;
    int n, nt, ne, np, nplt;
    // device views into the workspace; (h, l) pairs are double-float values
    const int* tri;            // [3*nt]
    const int* tri_plt;        // [nt]
    const float4* tri_rest;    // [2*nt] (|e1|^2 h,l, |e2|^2 h,l), (e1.e2 h,l, S0, 1/S0)
    const int4* edge;          // [ne] (i, j, k, l), chain k-i-j-l, l < 0 for a boundary edge
    const float4* edge_rest;   // [ne] (L0^2 h, L0^2 l, L0, -)
    const float4* edge_phi0;   // [ne] (cos phi0 h,l, sin phi0 h,l)
    const int* pair;           // [2*np]
    const float4* pair_rest;   // [np] (r0^2 h, r0^2 l, r0, -)
    const int* esl_off;    // [n+1] node -> 4*edge + slot (chain vertex k, i, j, l)
    const int* esl;
    const int* tcl_off;    // [n+1] node -> 4*triangle + corner
    const int* tcl;
    const int* psl_off;    // [n+1] node -> 2*pair + side
    const int* psl;
    const int* node_plt;   // [n]
    const uint8_t* is_mem; // [n]
    const double* plt_rest;// [4*nplt] S0, V0, 1/S0, 1/V0
    const int2* chunks;    // [n_chunks] (first entry of perm, count <= kIbChunk), runs of one platelet
    const int* perm;       // [n] nodes by platelet, in Morton order of the rest shape within each
    const int2* plt_range; // [nplt] (first entry of perm, count) of each platelet's nodes
    const int2* plt_chunks;// [nplt] (first chunk, count) of each platelet's chunks
    double* cpart;         // [3 * n_chunks] per-chunk sums of the advected positions (tracking)
    int n_chunks;
    int skip_edges;        // nonzero: edge elements (springs, bending) are neither computed nor gathered
    int skip_tris;         // nonzero: the nodes gather no triangle slots (global area and volume elsewhere)
    int tri_sums_only;     // nonzero: triangles add to the per-platelet sums but write no slots
    const int* plt_anchor; // [nplt]
    // per platelet (first node, nodes, first edge, edges), (first triangle,
    // triangles, first Morse pair, pairs) for the fused pass, or null when
    // the mesh does not group its elements by platelet
    const int4* plt_span;  // [2*nplt]
    int span_max_nodes;    // nodes of the largest platelet
    int path;              // 0: the three passes, 1: the fused pass where it applies
    // scratch, rewritten by every call
    double* acc;           // [2*nplt] sum of (S_t - S0_t), sum of tetrahedron volumes
    float2* coef;          // [nplt] k_s (S - S0)/S0, k_v (V - V0)/V0
    float* xh;             // [3n] positions, high floats
    float* xl;             // [3n] positions, low floats
    float4* eout;          // [4*ne] force on chain vertex k, i, j, l of each edge
    float4* tout;          // [4*nt] dS_t/dX per corner (w: k_t (S_t - S0_t)/S0_t), n/6
    float4* pout;          // [np] Morse force on the first node of each pair
};

struct BondCtx {
    bond_params p;
    int R;                 // sites
    int L;                 // ligands
    int window;            // r = ceil(d_capture) >= 1: ligands in reach lie in the 2r x 2r nodes around a site
    const int* site_tri;
    const double* site_w;
    const int* tri;
    int* bound;
    int* lig_count;
    // workspace
    int* nprop;            // [L] proposals this step
    int* cand;             // [L * kMaxCand]
    unsigned long long* counters;  // [4]: ruptures, formations, overflow, step (sim)
    const int* partner;    // bridge partner of each site (bridges.cu) or null
};
constexpr int kMaxCand = 64;

// Tether (pause-time) tracker over a bond context (bonds.cu).
struct TetherCtx {
    const BondCtx* bonds;
    int nplt;
    const int* off;               // [nplt + 1] per-platelet runs of `sites` (workspace)
    const int* sites;             // [R] site ids grouped by platelet, ascending within a platelet
    long long* state;             // caller [nplt]: step count at the tether's start, or -1
    long long* pauses;            // caller [cap]
    int cap;
    unsigned long long* count;    // caller [1]
};
const TetherCtx* tether_internal(const tether_ctx* t);
// After the adhesion update: the step count is *now_dev if now_dev, else now_host.
int launch_tether_update(const TetherCtx* c, const unsigned long long* now_dev, uint64_t now_host, cudaStream_t s);

// A node coordinate takes part in spreading and interpolation only if it lies
// within +-kFarCoord lattice units (false for NaN): the integer cell indices
// of its support then cannot overflow.  sim_check counts the coordinates
// outside that range (a run that blew up).
constexpr double kFarCoord = 1e8;
// The test on the bits (|x| as an unsigned integer orders like |x|, and NaN
// lies above every finite value): on the integer pipes, where fabs(x) <
// kFarCoord takes the FP64 pipe, which runs at a small fraction of the FP32
// rate on this part.
constexpr unsigned long long kFarCoordBits = 0x4197d78400000000ull;   // the bits of 1e8
__device__ __forceinline__ bool coord_in_range(double x)
{
    return ((unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull) < kFarCoordBits;
}
// (double)u exactly, on the integer pipes for normal u and zero (every other
// value, denormal, infinite or NaN, takes the conversion instruction).
__device__ __forceinline__ double widen(float u)
{
    const unsigned int b = __float_as_uint(u);
    const unsigned int e = (b >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) {
        if ((b & 0x7fffffffu) == 0u) return __longlong_as_double((long long)(b & 0x80000000u) << 32);
        return (double)u;
    }
    const unsigned long long r = ((unsigned long long)(b & 0x80000000u) << 32) |
                                 ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(b & 0x7fffffu) << 29);
    return __longlong_as_double((long long)r);
}

// Nodes per block of the IB kernels (also the largest chunk of the membrane's
// chunk table).
constexpr int kIbChunk = 64;

// One-time kernel attributes (large dynamic shared memory) of the IB kernels.
int ib_prepare();

// Launchers used by sim.cu (defined next to their kernels).
int launch_lb_step(LbCtx* c, cudaStream_t s);
// chunks: optional device table of (first entry, count <= kIbChunk) per block,
// used by the coupled step so that no block straddles two platelets; entries
// index perm (the nodes of each platelet in a spatially local order) when perm
// is non-null, else the nodes themselves; null chunks = fixed chunks of
// kIbChunk consecutive nodes.
int launch_ib_spread(LbCtx* c, const double* X, const float* F, int M, const int2* chunks, const int* perm,
                     int n_chunks, cudaStream_t s);
// next (optional, with advect): the next membrane pass's input -- the hi/lo
// float split of the advected X into h/l [3][M] and the per-platelet sums
// acc[0..nacc) cleared -- so that pass can skip its own; and, with part, the
// FP64 sum of the advected X over each block's nodes (part[3 block + d],
// fixed order), from which launch_centroids_from_chunks forms the platelet
// centroids.
struct NextSplit {
    float* h = nullptr;
    float* l = nullptr;
    double* acc = nullptr;
    int nacc = 0;
    double* part = nullptr;
};
// One chamber of a batch, as the multi-chamber launches take it (Multi):
// each of these runs its kernels for all n chambers as one launch per kernel
// (per kMax chambers), with the per-chamber results of the single-chamber
// launch functions above.
struct Chamber {
    LbCtx* lb;
    MemCtx* mem;
    BondCtx* bonds;   // or null
    double* X;
    float* F;
    float* U;
    int M;
};
int launch_membrane_forces_multi(const Chamber* ch, int n, cudaStream_t s);   // F overwritten
int launch_bonds_forces_multi(const Chamber* ch, int n, cudaStream_t s);
int launch_bonds_step_multi(const Chamber* ch, int n, cudaStream_t s);        // step index: counters[3]
int launch_ib_spread_multi(const Chamber* ch, int n, cudaStream_t s);
int launch_ib_interp_multi(const Chamber* ch, int n, cudaStream_t s);         // advects X

// Platelet centroids (out[3 p + d]) from the chunk sums of the last
// interpolation pass run with NextSplit::part = mem->cpart.
int launch_centroids_from_chunks(MemCtx* c, double* out, cudaStream_t s);
int launch_ib_interp(LbCtx* c, double* X, float* U, int M, int advect, const int2* chunks, const int* perm,
                     int n_chunks, cudaStream_t s, NextSplit split = NextSplit());
// presplit: mem->xh, xl hold the split of X and the per-platelet sums are
// clear (written by the previous step's interpolation): no split pass.
int launch_membrane_forces(MemCtx* c, const double* X, float* F, cudaStream_t s, bool presplit = false);
// Morse pairs and wall repulsion into F (overwritten; a mesh without Morse
// pairs gets F = 0 and leaves the wall term to the caller too), and the
// per-platelet coefficients k_s (S - S0)/S0, k_v (V - V0)/V0 into c->coef:
// the global area and volume forces themselves are left to the caller (the
// surrogate applies them per node from its one-ring).  Also splits X into
// c->xh, c->xl.
int launch_membrane_remainder(MemCtx* c, const double* X, float* F, cudaStream_t s, bool presplit = false);
int launch_bonds_forces(BondCtx* c, const double* X, float* F, int M, cudaStream_t s);
// Platelets out of the ligands' reach.  Every ligand lies on the wall plane,
// so a site whose platelet has all its nodes more than d_capture above the
// plane has no ligand in reach: the proposal pass skips such sites before it
// gathers their positions (the decision is the one the per-site height test
// takes, see k_plt_far).
struct FarSites {
    const int* site_plt = nullptr;   // [R] platelet of each site, -1: never skipped
    int* plt_far = nullptr;          // [nplt] workspace: 1 if the platelet is out of reach this step
    const int* block_plt = nullptr;  // [ceil(R / 256)] platelet of all sites of a proposal block, or -1
    const int2* plt_nodes = nullptr; // [nplt] (first node, nodes) of each platelet
    int nplt = 0;
};
// site_plt[s] = the platelet of site s's triangle, or -1 where the three
// corners are not of one platelet or the weights (w0, w1, 1 - w0 - w1) are
// not all nonnegative (the height bound of k_plt_far needs both);
// block_plt[b] = the platelet of all sites 256 b ... 256 b + 255, or -1;
// plt_nodes[p] = (first node, nodes) of platelet p, from node_plt [n].
int launch_site_platelets(const BondCtx* c, const int* node_plt, int n, int nplt, int* site_plt, int* block_plt,
                          int2* plt_nodes, cudaStream_t s);
// step_dev: device step counter (advanced by one after the update) or null
// to use step_host.  far (or null): skip the proposals of platelets out of
// reach, evaluated on X at the start of the update.
int launch_bonds_step(BondCtx* c, const double* X, int M, uint64_t step_host,
                      unsigned long long* step_dev, cudaStream_t s, const FarSites* far = nullptr);

struct SgCtx;
// Adds the surrogate's local membrane forces and the exact global area and
// volume forces to F, after launch_membrane_remainder(mem) (which leaves the
// split positions mem->xh, xl and the platelet coefficients mem->coef).
int launch_surrogate_forces(SgCtx* c, const void* params, const MemCtx* mem, float* F, cudaStream_t s);
SgCtx* sg_internal(sg_ctx* c);
int sg_node_count(const SgCtx* c);

struct BridgeCtx;
int launch_bridge_forces(BridgeCtx* c, const double* X, float* F, int M, cudaStream_t s);
int launch_bridges_step(BridgeCtx* c, const double* X, int M, uint64_t step_host, unsigned long long* step_dev,
                        cudaStream_t s);
BridgeCtx* bridge_internal(bridge_ctx* c);
unsigned long long* bridge_step_counter(BridgeCtx* c);
BondCtx* bridge_bonds(BridgeCtx* c);

struct FemCtx;
// Finite-element bending force (Eq. 6-10): F (+)= the nodal force; fields
// (nullable) receives the nodal normals, areas and curvatures.  xh, xl: the
// positions split into hi/lo floats ([3][n]), or null to split X first.
int launch_fem_forces(FemCtx* c, float k0, const double* X, const float* xh, const float* xl, float* F,
                      int accumulate, float* fields, cudaStream_t s);
FemCtx* fem_internal(fem_ctx* c);
int fem_node_count(const FemCtx* c);

}  // namespace pfsi

struct lb_ctx : pfsi::LbCtx {};
struct mem_ctx : pfsi::MemCtx {};
struct bond_ctx : pfsi::BondCtx {};
