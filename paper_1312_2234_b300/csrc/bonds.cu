// bonds.cu -- stochastic GPIb-alpha / vWF-A1 adhesion (Section 3.2) for sm_103a.
//
// Per step, three kernels:
//   rupture  (one thread per site)    bound sites break with P_r = 1 - exp(-k_off dt),
//                                     k_off = k_off0 exp(gamma F_b / kT), F_b = sigma |x_b - l_b| (Eq. 12)
//   propose  (one thread per site)    sites free at the start of the step test every
//                                     ligand within d_capture and below capacity (all
//                                     lie in the 2r x 2r lattice nodes around the site,
//                                     r = ceil(d_capture); 2x2 for d_capture <= 1) with
//                                     P_f = 1 - exp(-k_on dt), k_on of Eq. 13, and
//                                     propose to the lowest ligand id that succeeded
//   resolve  (one thread per ligand)  accepts its proposals in ascending site id up
//                                     to max_per_ligand bonds (at most 4 receptor
//                                     sites per vWF)
// so the outcome does not depend on thread scheduling.  Draws are Philox4x32-10
// keyed by the seed with counter (site, step, purpose).  The decision path
// (receptor position, bond length, rates) is FP64 with explicitly rounded
// operations in the order of the plain restatement, so that an event differs
// only when a uniform lands within an ulp of its probability.
#include <algorithm>
#include <cmath>
#include <vector>

#include "adhesion.cuh"

namespace pfsi {

namespace {

__device__ __forceinline__ SitePos site_position(const BondCtx& c, const double* __restrict__ X, int M, int s)
{
    return site_pos(c.site_tri, c.site_w, c.tri, X, M, s);
}

// vector from ligand `lig` to the receptor (minimum image in x, y)
__device__ __forceinline__ void bond_vector(const bond_params& p, const SitePos& r, int lig, double* d)
{
    const int li = lig % p.lig_ni, lj = lig / p.lig_ni;
    d[0] = min_image(__dsub_rn(r.x, (double)(p.lig_i0 + li)), p.box_nx);
    d[1] = min_image(__dsub_rn(r.y, (double)(p.lig_j0 + lj)), p.box_ny);
    d[2] = __dsub_rn(r.z, p.z_wall);
}

__device__ __forceinline__ void bond_forces(const BondCtx& c, const double* __restrict__ X, float* __restrict__ F,
                                            int M, int bx)
{
    const int s = bx * blockDim.x + threadIdx.x;
    if (s >= c.R) return;
    const int lig = c.bound[s];
    if (lig < 0) return;
    const SitePos r = site_position(c, X, M, s);
    double d[3];
    bond_vector(c.p, r, lig, d);
    const double xb = norm3_rn(d[0], d[1], d[2]);
    const double coef = -c.p.sigma * (xb - c.p.l_b) / xb;
    const double f[3] = {coef * d[0], coef * d[1], coef * d[2]};
    site_add_force(c.site_tri, c.site_w, c.tri, F, M, s, f);
}

__global__ void k_bond_forces(const __grid_constant__ BondCtx c, const double* __restrict__ X, float* __restrict__ F,
                              int M)
{
    pdl_wait();
    bond_forces(c, X, F, M, blockIdx.x);
}

// site_plt, plt_far (or null): a site of a platelet out of reach this step
// (k_plt_far) that breaks goes straight to free (-1): the proposal pass,
// which turns the ruptured state -2 into -1 without a proposal, skips that
// platelet's blocks.
__device__ __forceinline__ void bond_rupture(const BondCtx& c, const double* __restrict__ X, int M, uint64_t step_host,
                                             const unsigned long long* __restrict__ step_dev, int bx,
                                             const int* __restrict__ site_plt, const int* __restrict__ plt_far)
{
    const int s = bx * blockDim.x + threadIdx.x;
    if (s >= c.R) return;
    const int lig = c.bound[s];
    if (lig < 0) return;
    const uint64_t step = current_step(step_dev, step_host);
    const SitePos r = site_position(c, X, M, s);
    double d[3];
    bond_vector(c.p, r, lig, d);
    const double Fb = __dmul_rn(c.p.sigma, fabs(__dsub_rn(norm3_rn(d[0], d[1], d[2]), c.p.l_b)));
    const double koff_dt = __dmul_rn(c.p.koff0_dt, exp(__ddiv_rn(__dmul_rn(c.p.gamma, Fb), c.p.kT)));
    const double Pr = -expm1(-koff_dt);
    if (uniform53(c.p.seed, (uint32_t)s, step, 0u) < Pr) {
        const int q = site_plt ? site_plt[s] : -1;
        c.bound[s] = q >= 0 && plt_far[q] ? -1 : -2;  // -2: free, but not before the next step
        atomicSub(&c.lig_count[lig], 1);
        atomicAdd(&c.counters[0], 1ull);
    }
}

__global__ void k_bond_rupture(const __grid_constant__ BondCtx c, const double* __restrict__ X, int M, uint64_t step_host,
                               const unsigned long long* __restrict__ step_dev, const int* __restrict__ site_plt,
                               const int* __restrict__ plt_far)
{
    pdl_wait();
    bond_rupture(c, X, M, step_host, step_dev, blockIdx.x, site_plt, plt_far);
}

// Candidate (di, dj) of the window around node (i0, j0): the ligand there,
// if it is in the patch, below capacity and in reach, gets its own draw
// (purpose 1 + (dj + r - 1) 2r + (di + r - 1)); the lowest successful
// ligand id is kept in best.
__device__ __forceinline__ void propose_candidate(const BondCtx& c, const SitePos& r, int s, uint64_t step, int i0,
                                                  int j0, int di, int dj, int rw, int& best)
{
    const bond_params& p = c.p;
    int gi = (i0 + di) % p.box_nx, gj = (j0 + dj) % p.box_ny;
    if (gi < 0) gi += p.box_nx;
    if (gj < 0) gj += p.box_ny;
    if (gi < p.lig_i0 || gi >= p.lig_i0 + p.lig_ni) return;
    if (gj < p.lig_j0 || gj >= p.lig_j0 + p.lig_nj) return;
    const int lig = (gj - p.lig_j0) * p.lig_ni + (gi - p.lig_i0);
    if (c.lig_count[lig] >= p.max_per_ligand) return;
    double d[3];
    bond_vector(p, r, lig, d);
    const double xb = norm3_rn(d[0], d[1], d[2]);
    if (!(xb < p.d_capture)) return;
    const double dev = fabs(__dsub_rn(xb, p.l_b));
    const double ex = __ddiv_rn(__dmul_rn(__dmul_rn(p.sigma, dev), __dsub_rn(p.gamma, __dmul_rn(0.5, dev))), p.kT);
    const double kon_dt = __dmul_rn(p.kon0_dt, exp(ex));
    const double Pf = -expm1(-kon_dt);
    const double u = uniform53(p.seed, (uint32_t)s, step, (uint32_t)(1 + (dj + rw - 1) * 2 * rw + (di + rw - 1)));
    if (u < Pf && (best < 0 || lig < best)) best = lig;
}

// kR: the window half-width r at compile time (1: d_capture <= 1, the
// configurations' 0.64), or 0 to take it from the context at run time.
// site_plt, plt_far, block_plt (or null): the sites of a platelet out of
// reach this step (k_plt_far) return before their triangle and weights are
// loaded, and a block of 256 sites all of one such platelet returns at once
// (its ruptures of this step went straight to -1; between steps no site
// holds -2).
template <int kR>
__device__ __forceinline__ void bond_propose(const BondCtx& c, const double* __restrict__ X, int M, uint64_t step_host,
                                             const unsigned long long* __restrict__ step_dev, int blk,
                                             const int* __restrict__ site_plt, const int* __restrict__ plt_far,
                                             const int* __restrict__ block_plt)
{
    if (block_plt) {
        const int pb = __ldg(block_plt + blk);
        if (pb >= 0 && plt_far[pb]) return;
    }
    const int s = blk * blockDim.x + threadIdx.x;
    if (s >= c.R) return;
    const int b = c.bound[s];
    const int bridged = c.partner ? c.partner[s] : -1;
    const int q = site_plt ? __ldg(site_plt + s) : -1;
    if (b == -2) {
        c.bound[s] = -1;
        return;
    }
    if (b >= 0) return;
    if (bridged >= 0) return;
    if (q >= 0 && plt_far[q]) return;
    const int t = __ldg(c.site_tri + s);
    const double w0 = __ldg(c.site_w + 2 * s), w1 = __ldg(c.site_w + 2 * s + 1);
    const bond_params& p = c.p;
    // Out of reach of every ligand: the bond length is at least the height
    // above the wall plane (the margin covers the last-ulp rounding of the
    // norm), so skipping here cannot change a decision.
    {
        const double z = site_coord(X, M, 2, __ldg(c.tri + 3 * t), __ldg(c.tri + 3 * t + 1), __ldg(c.tri + 3 * t + 2),
                                    w0, w1);
        if (fabs(__dsub_rn(z, p.z_wall)) > p.d_capture * (1.0 + 1e-12)) return;
    }
    const uint64_t step = current_step(step_dev, step_host);
    const SitePos r = site_position(c, X, M, s);
    const double bx = (double)p.box_nx, by = (double)p.box_ny;
    const double xw = __dsub_rn(r.x, __dmul_rn(bx, floor(__ddiv_rn(r.x, bx))));
    const double yw = __dsub_rn(r.y, __dmul_rn(by, floor(__ddiv_rn(r.y, by))));
    const int i0 = (int)floor(xw), j0 = (int)floor(yw);
    const int rw = kR > 0 ? kR : c.window;
    int best = -1;
    if (kR > 0) {
#pragma unroll
        for (int dj = 1 - kR; dj <= kR; ++dj)
#pragma unroll
            for (int di = 1 - kR; di <= kR; ++di) propose_candidate(c, r, s, step, i0, j0, di, dj, rw, best);
    } else {
        for (int dj = 1 - rw; dj <= rw; ++dj)
            for (int di = 1 - rw; di <= rw; ++di) propose_candidate(c, r, s, step, i0, j0, di, dj, rw, best);
    }
    if (best >= 0) {
        const int slot = atomicAdd(&c.nprop[best], 1);
        if (slot < kMaxCand)
            c.cand[best * kMaxCand + slot] = s;
        else
            atomicAdd(&c.counters[2], 1ull);
    }
}

template <int kR>
__global__ void k_bond_propose(const __grid_constant__ BondCtx c, const double* __restrict__ X, int M, uint64_t step_host,
                               const unsigned long long* __restrict__ step_dev, const int* __restrict__ site_plt,
                               const int* __restrict__ plt_far, const int* __restrict__ block_plt)
{
    pdl_wait();
    bond_propose<kR>(c, X, M, step_host, step_dev, blockIdx.x, site_plt, plt_far, block_plt);
}

// One block per platelet: plt_far[p] = 1 if every node of platelet p lies more
// than d_capture (plus a margin) above the wall plane.  The sites kept by
// launch_site_platelets are combinations of one platelet's triangle corners
// with nonnegative weights summing to one, so a site's FP64 height is at
// least its platelet's lowest node height less the rounding of the
// combination (below 1e-9 while every |z| < 1e6, hence the 1e-6 margin and
// the 1e6 limit): the proposal's per-site height test rejects every such site,
// and skipping them changes no decision.  A NaN or far coordinate keeps its
// platelet in.
constexpr int kFarThreads = 512;
__global__ void __launch_bounds__(kFarThreads)
    k_plt_far(const FarSites f, const double* __restrict__ X, int M, double z_wall, double d_capture)
{
    pdl_wait();
    const int p = blockIdx.x;
    const int2 r = f.plt_nodes[p];
    const double* Z = X + 2 * (size_t)M + r.x;
    double m = INFINITY;
    int bad = 0;
#pragma unroll 4
    for (int k = threadIdx.x; k < r.y; k += kFarThreads) {
        const double z = Z[k];
        if (fabs(z) < 1e6)
            m = fmin(m, z);
        else
            bad = 1;
    }
    for (int o = 16; o > 0; o >>= 1) {
        m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    __shared__ double wm[kFarThreads / 32];
    __shared__ int wb[kFarThreads / 32];
    if ((threadIdx.x & 31) == 0) {
        wm[threadIdx.x >> 5] = m;
        wb[threadIdx.x >> 5] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kFarThreads / 32; ++w) {
            m = fmin(m, wm[w]);
            bad |= wb[w];
        }
        f.plt_far[p] = !bad && (m - z_wall > d_capture * (1.0 + 1e-12) + 1e-6);
    }
}

__global__ void k_site_platelets(const __grid_constant__ BondCtx c, const int* __restrict__ node_plt,
                                 int* __restrict__ site_plt)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= c.R) return;
    const int t = c.site_tri[s];
    const int a = c.tri[3 * t], b = c.tri[3 * t + 1], cc = c.tri[3 * t + 2];
    const double w0 = c.site_w[2 * s], w1 = c.site_w[2 * s + 1];
    const double w2 = __dsub_rn(__dsub_rn(1.0, w0), w1);   // as site_coord forms it
    const int p = node_plt[a];
    const bool one = p >= 0 && node_plt[b] == p && node_plt[cc] == p;
    site_plt[s] = one && w0 >= 0.0 && w1 >= 0.0 && w2 >= 0.0 ? p : -1;
}

// plt_nodes[p] = (first node, nodes) of platelet p (each platelet's nodes
// are one run of X, as the membrane mesh requires).
__global__ void k_plt_nodes(int n, const int* __restrict__ node_plt, int2* __restrict__ plt_nodes)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int p = node_plt[v];
    if (v == 0 || node_plt[v - 1] != p) {
        int e = v + 1;
        while (e < n && node_plt[e] == p) ++e;
        plt_nodes[p] = make_int2(v, e - v);
    }
}

// block_plt[b]: the platelet of all sites 256 b ... 256 b + 255 (the
// proposal's block b), or -1 if they are not all of one.
__global__ void k_block_platelets(int R, const int* __restrict__ site_plt, int* __restrict__ block_plt, int nb)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const int s0 = 256 * b, s1 = min(R, s0 + 256);
    int p = site_plt[s0];
    for (int s = s0 + 1; s < s1 && p >= 0; ++s)
        if (site_plt[s] != p) p = -1;
    block_plt[b] = p;
}

__device__ __forceinline__ void bond_resolve(const BondCtx& c, unsigned long long* __restrict__ step_dev, int bx)
{
    const int l = bx * blockDim.x + threadIdx.x;
    if (step_dev && l == 0) *step_dev += 1ull;
    if (l >= c.L) return;
    const int n = c.nprop[l];
    if (n == 0) return;
    const int m = n < kMaxCand ? n : kMaxCand;
    int* cand = c.cand + l * kMaxCand;
    // insertion sort by site id (short lists)
    for (int a = 1; a < m; ++a) {
        const int key = cand[a];
        int b = a - 1;
        while (b >= 0 && cand[b] > key) {
            cand[b + 1] = cand[b];
            --b;
        }
        cand[b + 1] = key;
    }
    int cnt = c.lig_count[l];
    int acc = 0;
    for (int a = 0; a < m && cnt < c.p.max_per_ligand; ++a) {
        c.bound[cand[a]] = l;
        ++cnt;
        ++acc;
    }
    c.lig_count[l] = cnt;
    c.nprop[l] = 0;
    if (acc) atomicAdd(&c.counters[1], (unsigned long long)acc);
}

__global__ void k_bond_resolve(const __grid_constant__ BondCtx c, unsigned long long* __restrict__ step_dev)
{
    pdl_wait();
    bond_resolve(c, step_dev, blockIdx.x);
}

// The bond kernels over several chambers, one launch each (see Multi).
struct BondArgs {
    BondCtx c;
    const double* X;
    float* F;
    int M;
    unsigned long long* step_dev;
};

__global__ void k_bond_forces_multi(const __grid_constant__ Multi<BondArgs> t)
{
    pdl_wait();
    const int e = multi_entry(t, blockIdx.x);
    const BondArgs& a = t.a[e];
    bond_forces(a.c, a.X, a.F, a.M, blockIdx.x - t.first[e]);
}

__global__ void k_bond_rupture_multi(const __grid_constant__ Multi<BondArgs> t)
{
    pdl_wait();
    const int e = multi_entry(t, blockIdx.x);
    const BondArgs& a = t.a[e];
    bond_rupture(a.c, a.X, a.M, 0, a.step_dev, blockIdx.x - t.first[e], nullptr, nullptr);
}

template <int kR>
__global__ void k_bond_propose_multi(const __grid_constant__ Multi<BondArgs> t)
{
    pdl_wait();
    const int e = multi_entry(t, blockIdx.x);
    const BondArgs& a = t.a[e];
    bond_propose<kR>(a.c, a.X, a.M, 0, a.step_dev, blockIdx.x - t.first[e], nullptr, nullptr, nullptr);
}

__global__ void k_bond_resolve_multi(const __grid_constant__ Multi<BondArgs> t)
{
    pdl_wait();
    const int e = multi_entry(t, blockIdx.x);
    bond_resolve(t.a[e].c, t.a[e].step_dev, blockIdx.x - t.first[e]);
}

// Tether tracking (Section 4.2): one block per platelet counts its bound
// sites (integer sum: exact in any order), then thread 0 opens or closes the
// platelet's tether event.
constexpr int kTetherThreads = 128;

__global__ void __launch_bounds__(kTetherThreads) k_tether(TetherCtx t, const int* __restrict__ bound,
                                                           const unsigned long long* __restrict__ now_dev,
                                                           uint64_t now_host)
{
    pdl_wait();
    const int p = blockIdx.x;
    const int b = t.off[p], e = t.off[p + 1];
    int n = 0;
    for (int k = b + (int)threadIdx.x; k < e; k += kTetherThreads) n += bound[t.sites[k]] >= 0;
    const bool tethered = __syncthreads_count(n > 0) > 0;
    if (threadIdx.x != 0) return;
    const long long now = (long long)(now_dev ? *now_dev : now_host);
    const long long start = t.state[p];
    if (tethered && start < 0) {
        t.state[p] = now;
    } else if (!tethered && start >= 0) {
        const unsigned long long slot = atomicAdd(t.count, 1ull);
        if (slot < (unsigned long long)t.cap) t.pauses[slot] = now - start;
        t.state[p] = -1;
    }
}

inline int blocks_for(int n, int t) { return (n + t - 1) / t; }

// workspace: nprop[L], cand[L * kMaxCand], counters[4]
size_t ws_bytes_for(int L)
{
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    return al(sizeof(int) * (size_t)L) + al(sizeof(int) * (size_t)L * kMaxCand) + al(4 * sizeof(unsigned long long));
}

}  // namespace

int launch_bonds_forces(BondCtx* c, const double* X, float* F, int M, cudaStream_t s)
{
    if (c->R == 0) return PFSI_OK;
    return check_cuda(launch_pdl(k_bond_forces, dim3(blocks_for(c->R, 256)), dim3(256), 0, s, *c, X, F, M),
                      "bonds_forces");
}

int launch_site_platelets(const BondCtx* c, const int* node_plt, int n, int nplt, int* site_plt, int* block_plt,
                          int2* plt_nodes, cudaStream_t s)
{
    if (c->R == 0) return PFSI_OK;
    int rc = check_cuda(cudaMemsetAsync(plt_nodes, 0, sizeof(int2) * (size_t)nplt, s), "site platelets");
    if (rc) return rc;
    k_plt_nodes<<<blocks_for(n, 256), 256, 0, s>>>(n, node_plt, plt_nodes);
    k_site_platelets<<<blocks_for(c->R, 256), 256, 0, s>>>(*c, node_plt, site_plt);
    const int nb = blocks_for(c->R, 256);
    k_block_platelets<<<blocks_for(nb, 128), 128, 0, s>>>(c->R, site_plt, block_plt, nb);
    return check_cuda(cudaGetLastError(), "site platelets");
}

int launch_bonds_step(BondCtx* c, const double* X, int M, uint64_t step_host,
                      unsigned long long* step_dev, cudaStream_t s, const FarSites* far)
{
    if (c->R > 0) {
        const int* site_plt = nullptr;
        const int* plt_far = nullptr;
        const int* block_plt = nullptr;
        int rc = PFSI_OK;
        if (far && far->nplt > 0) {
            rc = check_cuda(launch_pdl(k_plt_far, dim3(far->nplt), dim3(kFarThreads), 0, s, *far, X, M, c->p.z_wall,
                                       c->p.d_capture),
                            "bonds_step: platelets out of reach");
            if (rc) return rc;
            site_plt = far->site_plt;
            plt_far = far->plt_far;
            block_plt = far->block_plt;
        }
        rc = check_cuda(launch_pdl(k_bond_rupture, dim3(blocks_for(c->R, 256)), dim3(256), 0, s, *c, X, M, step_host,
                                   step_dev, site_plt, plt_far),
                        "bonds_step: rupture");
        if (rc) return rc;
        rc = check_cuda(launch_pdl(c->window == 1 ? k_bond_propose<1> : k_bond_propose<0>, dim3(blocks_for(c->R, 256)),
                                   dim3(256), 0, s, *c, X, M, step_host, step_dev, site_plt, plt_far, block_plt),
                        "bonds_step: propose");
        if (rc) return rc;
    }

    return check_cuda(launch_pdl(k_bond_resolve, dim3(blocks_for(c->L > 0 ? c->L : 1, 256)), dim3(256), 0, s, *c, step_dev),
                      "bonds_step: resolve");
}

int launch_bonds_forces_multi(const Chamber* ch, int n, cudaStream_t s)
{
    std::vector<Multi<BondArgs>> lists;
    for (int i = 0; i < n; ++i)
        if (ch[i].bonds)
            multi_push(lists, BondArgs{*ch[i].bonds, ch[i].X, ch[i].F, ch[i].M, nullptr}, blocks_for(ch[i].bonds->R, 256));
    int rc = PFSI_OK;
    for (const auto& t : lists)
        if (!rc) rc = check_cuda(launch_pdl(k_bond_forces_multi, dim3(t.blocks()), dim3(256), 0, s, t), "bonds_forces");
    return rc;
}

// Rupture, proposal and resolution of every chamber's bonds; each chamber's
// Philox step index is its device counter (counters[3]), advanced by its
// resolution pass.
int launch_bonds_step_multi(const Chamber* ch, int n, cudaStream_t s)
{
    std::vector<Multi<BondArgs>> sites, prop1, prop0, ligs;
    for (int i = 0; i < n; ++i) {
        BondCtx* c = ch[i].bonds;
        if (!c) continue;
        const BondArgs a{*c, ch[i].X, nullptr, ch[i].M, c->counters + 3};
        multi_push(sites, a, blocks_for(c->R, 256));
        multi_push(c->window == 1 ? prop1 : prop0, a, blocks_for(c->R, 256));
        multi_push(ligs, a, blocks_for(c->L > 0 ? c->L : 1, 256));
    }
    int rc = PFSI_OK;
    for (const auto& t : sites)
        if (!rc) rc = check_cuda(launch_pdl(k_bond_rupture_multi, dim3(t.blocks()), dim3(256), 0, s, t), "bonds_step: rupture");
    for (const auto& t : prop1)
        if (!rc)
            rc = check_cuda(launch_pdl(k_bond_propose_multi<1>, dim3(t.blocks()), dim3(256), 0, s, t), "bonds_step: propose");
    for (const auto& t : prop0)
        if (!rc)
            rc = check_cuda(launch_pdl(k_bond_propose_multi<0>, dim3(t.blocks()), dim3(256), 0, s, t), "bonds_step: propose");
    for (const auto& t : ligs)
        if (!rc) rc = check_cuda(launch_pdl(k_bond_resolve_multi, dim3(t.blocks()), dim3(256), 0, s, t), "bonds_step: resolve");
    return rc;
}

int launch_tether_update(const TetherCtx* c, const unsigned long long* now_dev, uint64_t now_host, cudaStream_t s)
{
    if (c->nplt == 0) return PFSI_OK;
    return check_cuda(launch_pdl(k_tether, dim3(c->nplt), dim3(kTetherThreads), 0, s, *c, (const int*)c->bonds->bound,
                                 now_dev, now_host),
                      "tether_update");
}

}  // namespace pfsi

using namespace pfsi;

struct tether_ctx : pfsi::TetherCtx {};

const pfsi::TetherCtx* pfsi::tether_internal(const tether_ctx* t) { return t; }

static size_t tether_ws_bytes(int n_sites, int n_plt)
{
    return (sizeof(int) * ((size_t)n_plt + 1) + 255) / 256 * 256 + sizeof(int) * (size_t)n_sites;
}

extern "C" int tether_query_workspace(int n_sites, int n_plt, size_t* bytes)
{
    if (!bytes || n_sites < 0 || n_plt < 0) return set_error(PFSI_ERR_ARG, "tether_query_workspace: bad argument");
    *bytes = tether_ws_bytes(n_sites, n_plt);
    return PFSI_OK;
}

extern "C" int tether_create(const bond_ctx* bonds, int n_plt, const int* site_plt, void* ws, size_t ws_bytes,
                             long long* state, long long* pauses, int capacity, unsigned long long* count,
                             tether_ctx** out)
{
    if (!bonds || !out || n_plt < 0 || capacity < 0 || !ws || !count || (n_plt > 0 && !state) ||
        (capacity > 0 && !pauses) || (bonds->R > 0 && !site_plt))
        return set_error(PFSI_ERR_ARG, "tether_create: bad argument");
    if (!aligned(ws, 256) || !aligned(state, 8) || !aligned(pauses, 8) || !aligned(count, 8))
        return set_error(PFSI_ERR_ARG, "tether_create: misaligned buffer");
    const int R = bonds->R;
    if (ws_bytes < tether_ws_bytes(R, n_plt)) return set_error(PFSI_ERR_ARG, "tether_create: workspace too small");
    // sites grouped by platelet (counting sort, ascending site ids within a platelet)
    std::vector<int> off((size_t)n_plt + 1, 0), sites((size_t)R);
    for (int s = 0; s < R; ++s) {
        if (site_plt[s] < 0 || site_plt[s] >= n_plt)
            return set_error(PFSI_ERR_ARG, "tether_create: site platelet out of range");
        ++off[site_plt[s] + 1];
    }
    for (int p = 0; p < n_plt; ++p) off[p + 1] += off[p];
    {
        std::vector<int> fill(off.begin(), off.end() - 1);
        for (int s = 0; s < R; ++s) sites[fill[site_plt[s]]++] = s;
    }
    char* base = static_cast<char*>(ws);
    int* d_off = reinterpret_cast<int*>(base);
    int* d_sites = reinterpret_cast<int*>(base + (sizeof(int) * ((size_t)n_plt + 1) + 255) / 256 * 256);
    int rc = check_cuda(cudaMemcpy(d_off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice),
                        "tether_create: copy");
    if (!rc && R > 0)
        rc = check_cuda(cudaMemcpy(d_sites, sites.data(), sizeof(int) * (size_t)R, cudaMemcpyHostToDevice),
                        "tether_create: copy");
    if (rc) return rc;
    tether_ctx* c = new tether_ctx();
    c->bonds = bonds;
    c->nplt = n_plt;
    c->off = d_off;
    c->sites = d_sites;
    c->state = state;
    c->pauses = pauses;
    c->cap = capacity;
    c->count = count;
    *out = c;
    return PFSI_OK;
}

extern "C" int tether_destroy(tether_ctx* c)
{
    delete c;
    return PFSI_OK;
}

extern "C" int tether_update(tether_ctx* c, uint64_t step, void* stream)
{
    NvtxRange nvtx_range("tether_update");
    if (!c) return set_error(PFSI_ERR_ARG, "tether_update: null context");
    return launch_tether_update(c, nullptr, step + 1, as_stream(stream));
}

static int check_bond_params(const bond_params* p, const char* who)
{
    if (!p) return set_error(PFSI_ERR_ARG, std::string(who) + ": null parameters");
    if (p->lig_ni < 1 || p->lig_nj < 1 || p->box_nx < 1 || p->box_ny < 1 || p->lig_i0 < 0 || p->lig_j0 < 0 ||
        p->lig_i0 + p->lig_ni > p->box_nx || p->lig_j0 + p->lig_nj > p->box_ny)
        return set_error(PFSI_ERR_ARG, std::string(who) + ": ligand patch outside the box");
    if (p->max_per_ligand < 1 || p->max_per_ligand > 32)
        return set_error(PFSI_ERR_ARG, std::string(who) + ": max_per_ligand must be 1..32");
    // every ligand in reach lies in the 2r x 2r nodes around a site; each
    // must appear there once
    if (!(p->d_capture > 0.0) || !(p->d_capture <= 8.0) || 2 * (int)std::ceil(p->d_capture) > p->box_nx ||
        2 * (int)std::ceil(p->d_capture) > p->box_ny)
        return set_error(PFSI_ERR_ARG, std::string(who) + ": d_capture must be in (0, 8] and 2 ceil(d_capture) "
                                                          "at most the box lengths");
    if (!(p->kT > 0.0)) return set_error(PFSI_ERR_ARG, std::string(who) + ": kT must be positive");
    return PFSI_OK;
}

extern "C" int bonds_query_workspace(const bond_params* p, int n_sites, size_t* bytes)
{
    int rc = check_bond_params(p, "bonds_query_workspace");
    if (rc) return rc;
    if (!bytes || n_sites < 0) return set_error(PFSI_ERR_ARG, "bonds_query_workspace: bad argument");
    *bytes = ws_bytes_for(p->lig_ni * p->lig_nj);
    return PFSI_OK;
}

extern "C" int bonds_create(const bond_params* p, int n_sites, const int* site_tri, const double* site_w,
                            const int* tri, int* bound, int* lig_count, void* ws, size_t ws_bytes,
                            bond_ctx** out)
{
    int rc = check_bond_params(p, "bonds_create");
    if (rc) return rc;
    if (!out || !ws || n_sites < 0 || (n_sites > 0 && (!site_tri || !site_w || !tri || !bound)) || !lig_count)
        return set_error(PFSI_ERR_ARG, "bonds_create: bad argument");
    if (!aligned(ws, 256)) return set_error(PFSI_ERR_ARG, "bonds_create: workspace must be 256-byte aligned");
    const int L = p->lig_ni * p->lig_nj;
    if (ws_bytes < ws_bytes_for(L)) return set_error(PFSI_ERR_ARG, "bonds_create: workspace too small");
    bond_ctx* c = new bond_ctx();
    c->p = *p;
    c->window = std::max(1, (int)std::ceil(p->d_capture));
    c->R = n_sites;
    c->L = L;
    c->site_tri = site_tri;
    c->site_w = site_w;
    c->tri = tri;
    c->bound = bound;
    c->lig_count = lig_count;
    c->partner = nullptr;
    char* base = static_cast<char*>(ws);
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    c->nprop = reinterpret_cast<int*>(base);
    c->cand = reinterpret_cast<int*>(base + al(sizeof(int) * L));
    c->counters = reinterpret_cast<unsigned long long*>(base + al(sizeof(int) * L) + al(sizeof(int) * (size_t)L * kMaxCand));
    rc = check_cuda(cudaMemsetAsync(c->nprop, 0, sizeof(int) * L, 0), "bonds_create: clear");
    if (!rc) rc = check_cuda(cudaMemsetAsync(c->counters, 0, 4 * sizeof(unsigned long long), 0), "bonds_create: clear");
    if (!rc) rc = check_cuda(cudaStreamSynchronize(0), "bonds_create: synchronise");
    if (rc) {
        delete c;
        return rc;
    }
    *out = c;
    return PFSI_OK;
}

extern "C" int bonds_destroy(bond_ctx* c)
{
    delete c;
    return PFSI_OK;
}

extern "C" int bonds_forces(bond_ctx* c, const double* X, float* F, int M, void* stream)
{
    NvtxRange nvtx_range("bonds_forces");
    if (!c || !X || !F || M < 0) return set_error(PFSI_ERR_ARG, "bonds_forces: bad argument");
    return launch_bonds_forces(c, X, F, M, as_stream(stream));
}

extern "C" int bonds_step(bond_ctx* c, const double* X, int M, uint64_t step, void* stream)
{
    NvtxRange nvtx_range("bonds_step");
    if (!c || !X || M < 0) return set_error(PFSI_ERR_ARG, "bonds_step: bad argument");
    return launch_bonds_step(c, X, M, step, nullptr, as_stream(stream));
}

extern "C" int bonds_status(bond_ctx* c, long long* out_host)
{
    if (!c || !out_host) return set_error(PFSI_ERR_ARG, "bonds_status: null argument");
    unsigned long long h[3];
    int rc = check_cuda(cudaMemcpy(h, c->counters, sizeof(h), cudaMemcpyDeviceToHost), "bonds_status: copy");
    if (rc) return rc;
    for (int k = 0; k < 3; ++k) out_host[k] = (long long)h[k];
    if (h[2]) return set_error(PFSI_ERR_CAPACITY, "bonds_status: a ligand received more than 64 proposals in one step");
    return PFSI_OK;
}
