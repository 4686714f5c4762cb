// bridges.cu -- platelet-platelet bridges GPIb-alpha - vWF - GPIb-alpha
// (Section 3.2, modelled like the wall bonds) for sm_103a.
//
// A bridge is one linear spring between receptor sites on two different
// platelets; partner[s] holds the other site or -1.  Per step, after the wall
// update:
//   k_br_rupture   (site i < partner j)  breaks with P_r = 1 - exp(-k_off dt),
//                                        Bell k_off of Eq. 12, F_b = sigma |x_b - l_b|
//   k_br_aabb      (one block per platelet) FP64 bounding box of its nodes
//   k_br_neighbors (platelet)            platelets whose boxes come within
//                                        d_capture (minimum image in x, y)
//   k_br_active    (site)                free sites (no wall bond, no bridge,
//                                        none ruptured this step) within
//                                        d_capture of a neighbour's box enter a
//                                        spatial hash (cells >= d_capture,
//                                        chained buckets)
//   k_br_choose    (active site)         scans the 27 cells around it: every pair
//                                        on different platelets closer than
//                                        d_capture succeeds with P_f = 1 - exp(-k_on dt),
//                                        k_on of Eq. 13; keeps the lowest-index
//                                        successful partner
//   k_br_match     (active site)         a bridge forms where two sites chose
//                                        each other
// Pair draws are Philox4x32-10 with counter (i, j, step lo, purpose), key
// (seed lo, seed hi ^ step hi), i < j, so both sites of a pair draw the same
// number; the pair vector is x_i - x_j for i < j in FP64, explicitly rounded.
// The hash and the box filter only prune candidates (every candidate is
// tested by distance), and the lowest-index choice does not depend on the
// order of the chains, so the outcome is independent of thread scheduling.
#include <vector>

#include "adhesion.cuh"

namespace pfsi {

namespace {
constexpr int kMaxNb = 16;          // neighbour platelets kept per platelet
constexpr int kBrThreads = 256;
}

struct BridgeCtx {
    bridge_params p;
    int R, nplt, B;                 // sites, platelets, hash buckets (power of two)
    int gx, gy;                     // hash cells along the periodic x, y
    double cell_x, cell_y, cell_z;  // cell sizes (>= d_capture)
    const int* site_tri;
    const double* site_w;
    const int* tri;
    const int* bound;
    int* partner;
    BondCtx* bonds;
    // workspace
    int* site_plt;                  // [R]
    int2* plt_nodes;                // [nplt] (first node, count)
    double4_32a* pos;                   // [R] site positions of the active sites
    int* act;                       // [R]
    int* choice;                    // [R]
    int* next;                      // [R] hash chains
    int* head;                      // [B]
    double4_32a* box;                   // [2 nplt] lo, hi
    int* nb;                        // [nplt][1 + kMaxNb] count (-1: overflow) and ids
    unsigned long long* counters;   // [4]: ruptures, formations, neighbour overflow, step (sim)
};

namespace {

__device__ __forceinline__ double pair_uniform53(uint64_t seed, uint32_t i, uint32_t j, uint64_t step,
                                                 uint32_t purpose)
{
    const uint4 r = philox4x32_10(make_uint4(i, j, (uint32_t)step, purpose),
                                  make_uint2((uint32_t)seed, (uint32_t)(seed >> 32) ^ (uint32_t)(step >> 32)));
    const uint64_t bits = ((uint64_t)r.x << 21) | (uint64_t)(r.y >> 11);
    return (double)bits * 0x1.0p-53;
}

// x_a - x_b, minimum image in x, y
__device__ __forceinline__ void pair_vector(const bridge_params& p, const SitePos& a, const SitePos& b, double* d)
{
    d[0] = min_image(__dsub_rn(a.x, b.x), p.box_nx);
    d[1] = min_image(__dsub_rn(a.y, b.y), p.box_ny);
    d[2] = __dsub_rn(a.z, b.z);
}

__device__ __forceinline__ SitePos site_of(const BridgeCtx& c, const double* __restrict__ X, int M, int s)
{
    return site_pos(c.site_tri, c.site_w, c.tri, X, M, s);
}

__global__ void k_br_forces(BridgeCtx c, const double* __restrict__ X, float* __restrict__ F, int M)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.R) return;
    const int j = c.partner[i];
    if (j <= i) return;
    const SitePos a = site_of(c, X, M, i), b = site_of(c, X, M, j);
    double d[3];
    pair_vector(c.p, a, b, d);
    const double xb = norm3_rn(d[0], d[1], d[2]);
    const double coef = -c.p.sigma * (xb - c.p.l_b) / xb;   // force on site i: coef d; on site j: -coef d
    const double fi[3] = {coef * d[0], coef * d[1], coef * d[2]};
    const double fj[3] = {-fi[0], -fi[1], -fi[2]};
    site_add_force(c.site_tri, c.site_w, c.tri, F, M, i, fi);
    site_add_force(c.site_tri, c.site_w, c.tri, F, M, j, fj);
}

__global__ void k_br_rupture(BridgeCtx c, const double* __restrict__ X, int M, uint64_t step_host,
                             const unsigned long long* __restrict__ step_dev)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.R) return;
    const int j = c.partner[i];
    if (j <= i) return;
    const uint64_t step = current_step(step_dev, step_host);
    const SitePos a = site_of(c, X, M, i), b = site_of(c, X, M, j);
    double d[3];
    pair_vector(c.p, a, b, d);
    const double Fb = __dmul_rn(c.p.sigma, fabs(__dsub_rn(norm3_rn(d[0], d[1], d[2]), c.p.l_b)));
    const double koff_dt = __dmul_rn(c.p.koff0_dt, exp(__ddiv_rn(__dmul_rn(c.p.gamma, Fb), c.p.kT)));
    const double Pr = -expm1(-koff_dt);
    if (pair_uniform53(c.p.seed, (uint32_t)i, (uint32_t)j, step, 16u) < Pr) {
        c.partner[i] = -2;   // free, but not before the next step
        c.partner[j] = -2;
        atomicAdd(&c.counters[0], 1ull);
    }
}

// Bounding box of each platelet's nodes (FP64, one block per platelet).
__global__ void __launch_bounds__(kBrThreads) k_br_aabb(BridgeCtx c, const double* __restrict__ X, int M)
{
    const int p = blockIdx.x;
    const int2 r = c.plt_nodes[p];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int k = threadIdx.x; k < r.y; k += blockDim.x) {
        const int n = r.x + k;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double v = X[d * M + n];
            lo[d] = fmin(lo[d], v);
            hi[d] = fmax(hi[d], v);
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            lo[d] = fmin(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], off));
            hi[d] = fmax(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], off));
        }
    __shared__ double s[kBrThreads / 32][6];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int d = 0; d < 3; ++d) {
            s[warp][d] = lo[d];
            s[warp][3 + d] = hi[d];
        }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            for (int d = 0; d < 3; ++d) {
                lo[d] = fmin(lo[d], s[w][d]);
                hi[d] = fmax(hi[d], s[w][3 + d]);
            }
        c.box[2 * p] = make_double4_32a(lo[0], lo[1], lo[2], 0.0);
        c.box[2 * p + 1] = make_double4_32a(hi[0], hi[1], hi[2], 0.0);
    }
}

// Gap between two boxes along one axis, minimum image over the period L
// (L = 0: not periodic); the margin makes the test conservative.
__device__ __forceinline__ double axis_gap(double lo_a, double hi_a, double lo_b, double hi_b, int L)
{
    double dc = 0.5 * (lo_a + hi_a) - 0.5 * (lo_b + hi_b);
    if (L > 0) dc -= (double)L * floor(dc / (double)L + 0.5);
    return fabs(dc) - 0.5 * (hi_a - lo_a) - 0.5 * (hi_b - lo_b);
}

__global__ void k_br_neighbors(BridgeCtx c)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= c.nplt) return;
    const double reach = c.p.d_capture * (1.0 + 1e-6) + 1e-9;
    const double4_32a la = c.box[2 * p], ha = c.box[2 * p + 1];
    int* out = c.nb + p * (1 + kMaxNb);
    int n = 0;
    for (int q = 0; q < c.nplt; ++q) {
        if (q == p) continue;
        const double4_32a lb = c.box[2 * q], hb = c.box[2 * q + 1];
        if (axis_gap(la.x, ha.x, lb.x, hb.x, c.p.box_nx) > reach) continue;
        if (axis_gap(la.y, ha.y, lb.y, hb.y, c.p.box_ny) > reach) continue;
        if (axis_gap(la.z, ha.z, lb.z, hb.z, 0) > reach) continue;
        if (n < kMaxNb) out[1 + n] = q;
        ++n;
    }
    if (n > kMaxNb) {
        atomicAdd(&c.counters[2], 1ull);
        n = -1;   // every free site of p is a candidate
    }
    out[0] = n;
}

__device__ __forceinline__ uint32_t bucket_of(const BridgeCtx& c, int cx, int cy, int cz)
{
    return ((uint32_t)cx * 73856093u ^ (uint32_t)cy * 19349663u ^ (uint32_t)cz * 83492791u) & (uint32_t)(c.B - 1);
}

// Hash cell of a position.  The periodic indices wrap modulo the cell
// count: a coordinate within rounding of a cell face may land in the
// neighbouring cell (also across the periodic seam), which the 27-cell scan
// still covers because the cells are wider than d_capture.
__device__ __forceinline__ void cell_of(const BridgeCtx& c, const SitePos& r, int& cx, int& cy, int& cz)
{
    const double nx = (double)c.p.box_nx, ny = (double)c.p.box_ny;
    const double xw = r.x - nx * floor(r.x / nx), yw = r.y - ny * floor(r.y / ny);
    cx = (int)floor(xw / c.cell_x) % c.gx;
    cy = (int)floor(yw / c.cell_y) % c.gy;
    cx += cx < 0 ? c.gx : 0;
    cy += cy < 0 ? c.gy : 0;
    cz = (int)floor(r.z / c.cell_z);
}

__global__ void k_br_active(BridgeCtx c, const double* __restrict__ X, int M)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= c.R) return;
    const int ps = c.partner[s];
    if (ps == -2) c.partner[s] = -1;   // ruptured this step: free from the next one
    int active = (ps == -1) && (c.bound[s] == -1);
    SitePos r{0.0, 0.0, 0.0};
    if (active) {
        r = site_of(c, X, M, s);
        const int p = c.site_plt[s];
        const int* nbl = c.nb + p * (1 + kMaxNb);
        const int n = nbl[0];
        if (n >= 0) {
            const double reach = c.p.d_capture * (1.0 + 1e-6) + 1e-9;
            bool near = false;
            for (int k = 0; k < n && !near; ++k) {
                const int q = nbl[1 + k];
                const double4_32a lb = c.box[2 * q], hb = c.box[2 * q + 1];
                near = axis_gap(r.x, r.x, lb.x, hb.x, c.p.box_nx) <= reach &&
                       axis_gap(r.y, r.y, lb.y, hb.y, c.p.box_ny) <= reach && axis_gap(r.z, r.z, lb.z, hb.z, 0) <= reach;
            }
            active = near;
        }
    }
    c.act[s] = active;
    if (!active) return;
    c.pos[s] = make_double4_32a(r.x, r.y, r.z, 0.0);
    int cx, cy, cz;
    cell_of(c, r, cx, cy, cz);
    c.next[s] = atomicExch(&c.head[bucket_of(c, cx, cy, cz)], s);
}

__global__ void k_br_choose(BridgeCtx c, uint64_t step_host, const unsigned long long* __restrict__ step_dev)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.R || !c.act[i]) return;
    const uint64_t step = current_step(step_dev, step_host);
    const double4_32a pi4 = c.pos[i];
    const SitePos ri{pi4.x, pi4.y, pi4.z};
    const int pi = c.site_plt[i];
    int cx, cy, cz;
    cell_of(c, ri, cx, cy, cz);
    const bridge_params& p = c.p;
    int best = -1;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int x = (cx + dx + c.gx) % c.gx, y = (cy + dy + c.gy) % c.gy;
                for (int j = c.head[bucket_of(c, x, y, cz + dz)]; j >= 0; j = c.next[j]) {
                    if (c.site_plt[j] == pi || (best >= 0 && j >= best)) continue;
                    const double4_32a pj4 = c.pos[j];
                    const SitePos rj{pj4.x, pj4.y, pj4.z};
                    const int a = i < j ? i : j, b = i < j ? j : i;
                    double d[3];
                    if (i < j)
                        pair_vector(p, ri, rj, d);
                    else
                        pair_vector(p, rj, ri, d);
                    const double xb = norm3_rn(d[0], d[1], d[2]);
                    if (!(xb < p.d_capture)) continue;
                    const double dev = fabs(__dsub_rn(xb, p.l_b));
                    const double ex =
                        __ddiv_rn(__dmul_rn(__dmul_rn(p.sigma, dev), __dsub_rn(p.gamma, __dmul_rn(0.5, dev))), p.kT);
                    const double kon_dt = __dmul_rn(p.kon0_dt, exp(ex));
                    const double Pf = -expm1(-kon_dt);
                    if (pair_uniform53(p.seed, (uint32_t)a, (uint32_t)b, step, 17u) < Pf) best = j;
                }
            }
    c.choice[i] = best;
}

__global__ void k_br_match(BridgeCtx c, unsigned long long* __restrict__ step_dev)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (step_dev && i == 0) *step_dev += 1ull;
    if (i >= c.R || !c.act[i]) return;
    const int j = c.choice[i];
    if (j > i && c.choice[j] == i) {
        c.partner[i] = j;
        c.partner[j] = i;
        atomicAdd(&c.counters[1], 1ull);
    }
}

int blocks(int n) { return (n + kBrThreads - 1) / kBrThreads; }

}  // namespace

int launch_bridge_forces(BridgeCtx* c, const double* X, float* F, int M, cudaStream_t s)
{
    if (c->R == 0) return PFSI_OK;
    k_br_forces<<<blocks(c->R), kBrThreads, 0, s>>>(*c, X, F, M);
    return check_launch("bridges_forces");
}

int launch_bridges_step(BridgeCtx* c, const double* X, int M, uint64_t step_host, unsigned long long* step_dev,
                        cudaStream_t s)
{
    if (c->R == 0) {
        if (step_dev) {
            // keep the step counter moving
            k_br_match<<<1, 32, 0, s>>>(*c, step_dev);
            return check_launch("bridges_step");
        }
        return PFSI_OK;
    }
    const BridgeCtx v = *c;
    k_br_rupture<<<blocks(c->R), kBrThreads, 0, s>>>(v, X, M, step_host, step_dev);
    k_br_aabb<<<c->nplt, kBrThreads, 0, s>>>(v, X, M);
    k_br_neighbors<<<blocks(c->nplt), kBrThreads, 0, s>>>(v);
    int rc = check_cuda(cudaMemsetAsync(c->head, 0xff, sizeof(int) * (size_t)c->B, s), "bridges_step: clear hash");
    if (rc) return rc;
    k_br_active<<<blocks(c->R), kBrThreads, 0, s>>>(v, X, M);
    k_br_choose<<<blocks(c->R), kBrThreads, 0, s>>>(v, step_host, step_dev);
    k_br_match<<<blocks(c->R), kBrThreads, 0, s>>>(v, step_dev);
    return check_launch("bridges_step");
}

namespace {

struct BrLayout {
    size_t site_plt, plt_nodes, pos, act, choice, next, head, box, nb, counters, node_plt, total;
    int B;
};

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

BrLayout br_layout(int R, int nplt, int M)
{
    BrLayout L;
    int B = 1024;
    while (B < R && B < (1 << 20)) B <<= 1;
    L.B = B;
    size_t o = 0;
    const size_t r = (size_t)(R > 0 ? R : 1);
    L.site_plt = o;
    o += al256(4 * r);
    L.plt_nodes = o;
    o += al256(8 * (size_t)nplt);
    L.pos = o;
    o += al256(32 * r);
    L.act = o;
    o += al256(4 * r);
    L.choice = o;
    o += al256(4 * r);
    L.next = o;
    o += al256(4 * r);
    L.head = o;
    o += al256(4 * (size_t)B);
    L.box = o;
    o += al256(64 * (size_t)nplt);
    L.nb = o;
    o += al256(4 * (size_t)nplt * (1 + kMaxNb));
    L.counters = o;
    o += al256(4 * sizeof(unsigned long long));
    L.node_plt = o;   // platelet of each node, used at create only
    o += al256(4 * (size_t)M);
    L.total = o;
    return L;
}

int check_bridge_params(const bridge_params* p, const char* who)
{
    if (!p) return set_error(PFSI_ERR_ARG, std::string(who) + ": bad argument");
    if (!(p->d_capture > 0.0) || !(p->sigma >= 0.0) || !(p->kT > 0.0) || !(p->kon0_dt >= 0.0) ||
        !(p->koff0_dt >= 0.0) || p->box_nx < 1 || p->box_ny < 1)
        return set_error(PFSI_ERR_ARG, std::string(who) + ": invalid parameters (d_capture > 0, kT > 0, rates >= 0, box >= 1)");
    return PFSI_OK;
}

__global__ void k_br_site_plt(int R, const int* __restrict__ site_tri, const int* __restrict__ tri,
                              const int* __restrict__ node_plt, int* __restrict__ out)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < R) out[s] = node_plt[tri[3 * site_tri[s]]];
}

}  // namespace

}  // namespace pfsi

using namespace pfsi;

struct bridge_ctx : pfsi::BridgeCtx {};

namespace pfsi {
BridgeCtx* bridge_internal(bridge_ctx* c) { return c; }
unsigned long long* bridge_step_counter(BridgeCtx* c) { return c->counters + 3; }
BondCtx* bridge_bonds(BridgeCtx* c) { return c->bonds; }
}

extern "C" int bridges_query_workspace(const bridge_params* p, int n_sites, int n_plt, int M, size_t* bytes)
{
    int rc = check_bridge_params(p, "bridges_query_workspace");
    if (rc) return rc;
    if (!bytes || n_sites < 0 || n_plt < 1 || M < 1) return set_error(PFSI_ERR_ARG, "bridges_query_workspace: bad argument");
    *bytes = br_layout(n_sites, n_plt, M).total;
    return PFSI_OK;
}

extern "C" int bridges_create(const bridge_params* p, bond_ctx* bonds, int n_plt, const int* node_plt, int M,
                              int* partner, void* ws, size_t ws_bytes, bridge_ctx** out)
{
    int rc = check_bridge_params(p, "bridges_create");
    if (rc) return rc;
    if (!bonds || !out || !ws || n_plt < 1 || M < 1 || !node_plt || (bonds->R > 0 && !partner))
        return set_error(PFSI_ERR_ARG, "bridges_create: bad argument");
    if (!aligned(ws, 256)) return set_error(PFSI_ERR_ARG, "bridges_create: workspace must be 256-byte aligned");
    const int R = bonds->R;
    const BrLayout L = br_layout(R, n_plt, M);
    if (ws_bytes < L.total) return set_error(PFSI_ERR_ARG, "bridges_create: workspace too small");
    // contiguous node range of every platelet
    std::vector<int2> range(n_plt, make_int2(0, 0));
    std::vector<int> seen(n_plt, 0);
    for (int n = 0; n < M; ++n) {
        const int q = node_plt[n];
        if (q < 0 || q >= n_plt) return set_error(PFSI_ERR_ARG, "bridges_create: platelet index out of range");
        if (!seen[q]) {
            seen[q] = 1;
            range[q] = make_int2(n, 0);
        } else if (range[q].x + range[q].y != n) {
            return set_error(PFSI_ERR_ARG, "bridges_create: the nodes of a platelet must be contiguous");
        }
        range[q].y += 1;
    }
    for (int q = 0; q < n_plt; ++q)
        if (!seen[q]) return set_error(PFSI_ERR_ARG, "bridges_create: a platelet has no nodes");
    const double d = p->d_capture * (1.0 + 1e-6);
    int gx = (int)floor(p->box_nx / d), gy = (int)floor(p->box_ny / d);
    gx = gx < 1 ? 1 : gx;
    gy = gy < 1 ? 1 : gy;
    char* b = (char*)ws;
    rc = check_cuda(cudaMemset(ws, 0, L.total), "bridges_create: clear");
    if (!rc)
        rc = check_cuda(cudaMemcpy(b + L.plt_nodes, range.data(), 8 * (size_t)n_plt, cudaMemcpyHostToDevice),
                        "bridges_create");
    if (!rc && R > 0) {
        int* node_plt_dev = (int*)(b + L.node_plt);
        rc = check_cuda(cudaMemcpy(node_plt_dev, node_plt, 4 * (size_t)M, cudaMemcpyHostToDevice), "bridges_create");
        if (!rc) {
            k_br_site_plt<<<(R + 255) / 256, 256>>>(R, bonds->site_tri, bonds->tri, node_plt_dev, (int*)(b + L.site_plt));
            rc = check_launch("bridges_create: site platelets");
        }
        if (!rc) rc = check_cuda(cudaDeviceSynchronize(), "bridges_create: synchronise");
    }
    if (rc) return rc;
    bridge_ctx* c = new bridge_ctx();
    c->p = *p;
    c->R = R;
    c->nplt = n_plt;
    c->B = L.B;
    c->gx = gx;
    c->gy = gy;
    c->cell_x = (double)p->box_nx / gx;
    c->cell_y = (double)p->box_ny / gy;
    c->cell_z = d;
    c->site_tri = bonds->site_tri;
    c->site_w = bonds->site_w;
    c->tri = bonds->tri;
    c->bound = bonds->bound;
    c->partner = partner;
    c->bonds = bonds;
    c->site_plt = (int*)(b + L.site_plt);
    c->plt_nodes = (int2*)(b + L.plt_nodes);
    c->pos = (double4_32a*)(b + L.pos);
    c->act = (int*)(b + L.act);
    c->choice = (int*)(b + L.choice);
    c->next = (int*)(b + L.next);
    c->head = (int*)(b + L.head);
    c->box = (double4_32a*)(b + L.box);
    c->nb = (int*)(b + L.nb);
    c->counters = (unsigned long long*)(b + L.counters);
    bonds->partner = partner;   // wall bonds skip bridged sites
    *out = c;
    return PFSI_OK;
}

extern "C" int bridges_destroy(bridge_ctx* c)
{
    if (c && c->bonds && c->bonds->partner == c->partner) c->bonds->partner = nullptr;
    delete c;
    return PFSI_OK;
}

extern "C" int bridges_forces(bridge_ctx* c, const double* X, float* F, int M, void* stream)
{
    if (!c || !X || !F || M < 1) return set_error(PFSI_ERR_ARG, "bridges_forces: bad argument");
    return launch_bridge_forces(c, X, F, M, as_stream(stream));
}

extern "C" int bridges_step(bridge_ctx* c, const double* X, int M, uint64_t step, void* stream)
{
    if (!c || !X || M < 1) return set_error(PFSI_ERR_ARG, "bridges_step: bad argument");
    return launch_bridges_step(c, X, M, step, nullptr, as_stream(stream));
}

extern "C" int bridges_status(bridge_ctx* c, long long* out_host)
{
    if (!c || !out_host) return set_error(PFSI_ERR_ARG, "bridges_status: bad argument");
    unsigned long long h[4];
    int rc = check_cuda(cudaMemcpy(h, c->counters, sizeof(h), cudaMemcpyDeviceToHost), "bridges_status");
    if (rc) return rc;
    out_host[0] = (long long)h[0];
    out_host[1] = (long long)h[1];
    out_host[2] = (long long)h[2];
    return PFSI_OK;
}

extern "C" int bridges_partner(bridge_ctx* c, int** partner_dev)
{
    if (!c || !partner_dev) return set_error(PFSI_ERR_ARG, "bridges_partner: bad argument");
    *partner_dev = c->partner;
    return PFSI_OK;
}
