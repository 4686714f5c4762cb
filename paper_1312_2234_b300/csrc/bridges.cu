// bridges.cu -- platelet-platelet bridges GPIb-alpha - vWF - GPIb-alpha
// (Section 3.2, modelled like the wall bonds) for sm_103a.
//
// A bridge is one linear spring between receptor sites on two different
// platelets; partner[s] holds the other site or -1.  Per step, after the wall
// update:
//   k_br_boxes     (one block per platelet) bounding box of its nodes
//                                        (FP32 bounds rounded outward)
//   k_br_neighbors (platelet pair)       platelets whose boxes come within
//                                        d_capture (minimum image in x, y)
//   k_br_active    (site)                a bridge (i, j) breaks with
//                                        P_r = 1 - exp(-k_off dt), Bell k_off of
//                                        Eq. 12, F_b = sigma |x_b - l_b| (both
//                                        ends take the same decision); free
//                                        sites (no wall bond, no bridge at the
//                                        start of the step) within
//                                        d_capture of a neighbour's box are
//                                        counted into spatial-hash buckets
//                                        (cells >= d_capture)
//   k_br_scan, k_br_scatter              counting sort of the active sites by
//                                        bucket (contiguous FP32 positions)
//   k_br_choose    (active site)         scans the 27 cells around it (an FP32
//                                        distance with a safe margin selects
//                                        the candidates that take the FP64
//                                        decision path): every pair
//                                        on different platelets closer than
//                                        d_capture succeeds with P_f = 1 - exp(-k_on dt),
//                                        k_on of Eq. 13; keeps the lowest-index
//                                        successful partner
//   k_br_match     (active site)         a bridge forms where two sites chose
//                                        each other
// Pair draws are Philox4x32-10 with counter (i, j, step lo, purpose), key
// (seed lo, seed hi ^ step hi), i < j, so both sites of a pair draw the same
// number; the pair vector is x_i - x_j for i < j in FP64, explicitly rounded.
// The hash, the box filter and the FP32 prefilter only prune candidates
// (every candidate in reach takes the FP64 test), and the lowest-index choice
// does not depend on the order within a bucket, so the outcome is
// independent of thread scheduling.
#include <cmath>
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
    int* key;                       // [R] bucket of each active site
    int* slot;                      // [R] its rank within the bucket
    int* count;                     // [B] active sites per bucket
    int* start;                     // [B] exclusive prefix of count
    float4* fpos;                   // [R] bucket-sorted: FP32 position wrapped into the box, platelet id bits
    int* sid;                       // [R] bucket-sorted site ids
    int4* cell;                     // [R] hash cell of each active site
    int4* scell;                    // [R] bucket-sorted hash cells
    // FP32 copies of the parameters for the candidate filter (host-computed:
    // FP64 arithmetic is a scarce pipe on this part)
    float f_sk, f_gamma, f_lb, f_kon0, f_dcap;
    int f_shortcut;
    float4* box;                    // [2 nplt] lo, hi (FP32, rounded outward)
    int* nb;                        // [nplt][kMaxNb] neighbour platelets
    int* nbc;                       // [nplt] neighbour count (> kMaxNb: overflow), after count[B]
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
    pdl_wait();
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

// Order-preserving unsigned key of a double (min/max without the FP64 pipe).
__device__ __forceinline__ unsigned long long order_key(double x)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double from_order_key(unsigned long long k)
{
    return __longlong_as_double((long long)((k >> 63) ? (k & 0x7fffffffffffffffull) : ~k));
}

// Bounding box of each platelet's nodes (one block per platelet), stored as
// FP32 bounds rounded outward.
__global__ void __launch_bounds__(kBrThreads) k_br_boxes(BridgeCtx c, const double* __restrict__ X, int M)
{
    pdl_wait();
    const int p = blockIdx.x;
    const int2 r = c.plt_nodes[p];
    unsigned long long lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0ull, 0ull, 0ull};
    for (int k = threadIdx.x; k < r.y; k += blockDim.x) {
        const int n = r.x + k;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const unsigned long long v = order_key(X[d * M + n]);
            lo[d] = v < lo[d] ? v : lo[d];
            hi[d] = v > hi[d] ? v : hi[d];
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const unsigned long long a = __shfl_xor_sync(0xffffffffu, lo[d], off);
            const unsigned long long b = __shfl_xor_sync(0xffffffffu, hi[d], off);
            lo[d] = a < lo[d] ? a : lo[d];
            hi[d] = b > hi[d] ? b : hi[d];
        }
    __shared__ unsigned long long s[kBrThreads / 32][6];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int d = 0; d < 3; ++d) {
            s[warp][d] = lo[d];
            s[warp][3 + d] = hi[d];
        }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int d = threadIdx.x;
        unsigned long long v = s[0][d];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            const unsigned long long x = s[w][d];
            v = d < 3 ? (x < v ? x : v) : (x > v ? x : v);
        }
        const double x = from_order_key(v);
        reinterpret_cast<float*>(c.box)[8 * p + (d < 3 ? d : d + 1)] = d < 3 ? __double2float_rd(x) : __double2float_ru(x);
    }
}

// Gap between two intervals along one axis (FP32), minimum image over the
// period L (L = 0: not periodic), and a bound of its rounding error.
__device__ __forceinline__ float axis_gap(float lo_a, float hi_a, float lo_b, float hi_b, int L, float& err)
{
    float dc = 0.5f * (lo_a + hi_a) - 0.5f * (lo_b + hi_b);
    if (L > 0) dc -= (float)L * rintf(dc / (float)L);
    err = 8.0f * (fabsf(lo_a) + fabsf(hi_a) + fabsf(lo_b) + fabsf(hi_b) + (float)L) * 0x1.0p-23f + 1e-6f;
    return fabsf(dc) - 0.5f * (hi_a - lo_a) - 0.5f * (hi_b - lo_b);
}

// Conservative test: the intervals (or a point and an interval) may come
// within `reach` of each other along every axis.
__device__ __forceinline__ bool boxes_near(const BridgeCtx& c, float4 la, float4 ha, float4 lb, float4 hb, float reach)
{
    float e, g;
    g = axis_gap(la.x, ha.x, lb.x, hb.x, c.p.box_nx, e);
    if (g > reach + e) return false;
    g = axis_gap(la.y, ha.y, lb.y, hb.y, c.p.box_ny, e);
    if (g > reach + e) return false;
    g = axis_gap(la.z, ha.z, lb.z, hb.z, 0, e);
    return g <= reach + e;
}

// One thread per ordered platelet pair (p, q): q joins p's neighbour list if
// their boxes come within d_capture.
__global__ void k_br_neighbors(BridgeCtx c)
{
    pdl_wait();
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)c.nplt * c.nplt) return;
    const int p = (int)(t / c.nplt), q = (int)(t - (long long)p * c.nplt);
    if (p == q) return;
    if (!boxes_near(c, c.box[2 * p], c.box[2 * p + 1], c.box[2 * q], c.box[2 * q + 1], (float)c.p.d_capture)) return;
    const int slot = atomicAdd(&c.nbc[p], 1);
    if (slot < kMaxNb) c.nb[p * kMaxNb + slot] = q;
    if (slot == kMaxNb) atomicAdd(&c.counters[2], 1ull);   // overflow: every free site of p is a candidate
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

// Per site: the rupture test of a standing bridge (evaluated identically by
// both ends: ordered pair, one draw, so each end writes only its own entry),
// then the candidate filter of the free sites and their bucket counts.
__global__ void k_br_active(BridgeCtx c, const double* __restrict__ X, int M, uint64_t step_host,
                            const unsigned long long* __restrict__ step_dev)
{
    pdl_wait();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= c.R) return;
    const int ps = c.partner[s];
    if (ps >= 0) {
        const int a = s < ps ? s : ps, b = s < ps ? ps : s;
        const SitePos ra = site_of(c, X, M, a), rb = site_of(c, X, M, b);
        double d[3];
        pair_vector(c.p, ra, rb, d);
        const double Fb = __dmul_rn(c.p.sigma, fabs(__dsub_rn(norm3_rn(d[0], d[1], d[2]), c.p.l_b)));
        const double koff_dt = __dmul_rn(c.p.koff0_dt, exp(__ddiv_rn(__dmul_rn(c.p.gamma, Fb), c.p.kT)));
        const double Pr = -expm1(-koff_dt);
        const uint64_t step = current_step(step_dev, step_host);
        if (pair_uniform53(c.p.seed, (uint32_t)a, (uint32_t)b, step, 16u) < Pr) {
            c.partner[s] = -1;   // free from the next step on
            if (s == a) atomicAdd(&c.counters[0], 1ull);
        }
        c.act[s] = 0;
        return;
    }
    int active = c.bound[s] == -1;
    SitePos r{0.0, 0.0, 0.0};
    if (active) {
        r = site_of(c, X, M, s);
        const int p = c.site_plt[s];
        const int n = c.nbc[p];
        if (n <= kMaxNb) {
            const float4 pt = make_float4((float)r.x, (float)r.y, (float)r.z, 0.0f);
            const float reach = (float)c.p.d_capture;
            bool near = false;
            for (int k = 0; k < n && !near; ++k) {
                const int q = c.nb[p * kMaxNb + k];
                near = boxes_near(c, pt, pt, c.box[2 * q], c.box[2 * q + 1], reach);
            }
            active = near;
        }
    }
    c.act[s] = active;
    if (!active) return;
    c.pos[s] = make_double4_32a(r.x, r.y, r.z, 0.0);
    int cx, cy, cz;
    cell_of(c, r, cx, cy, cz);
    const int b = (int)bucket_of(c, cx, cy, cz);
    c.key[s] = b;
    c.cell[s] = make_int4(cx, cy, cz, 0);
    c.slot[s] = atomicAdd(&c.count[b], 1);
}

// Exclusive prefix of the bucket counts (one block of kScanThreads threads;
// B is a power of two >= kScanThreads).
constexpr int kScanThreads = 1024;
__global__ void __launch_bounds__(kScanThreads) k_br_scan(BridgeCtx c)
{
    pdl_wait();
    __shared__ int part[kScanThreads];
    const int per = c.B / kScanThreads;   // power of two
    const int t = threadIdx.x;
    const int* cnt = c.count + (size_t)t * per;
    int sum = 0;
    if (per % 4 == 0) {
        for (int k = 0; k < per; k += 4) {
            const int4 v = *reinterpret_cast<const int4*>(cnt + k);
            sum += v.x + v.y + v.z + v.w;
        }
    } else {
        for (int k = 0; k < per; ++k) sum += cnt[k];
    }
    part[t] = sum;
    __syncthreads();
    for (int off = 1; off < kScanThreads; off <<= 1) {
        const int v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = part[t] - sum;
    int* st = c.start + (size_t)t * per;
    if (per % 4 == 0) {
        for (int k = 0; k < per; k += 4) {
            const int4 v = *reinterpret_cast<const int4*>(cnt + k);
            int4 o;
            o.x = run;
            o.y = run + v.x;
            o.z = o.y + v.y;
            o.w = o.z + v.z;
            run = o.w + v.w;
            *reinterpret_cast<int4*>(st + k) = o;
        }
    } else {
        for (int k = 0; k < per; ++k) {
            st[k] = run;
            run += cnt[k];
        }
    }
}

// FP32 copy of a position for the candidate prefilter: x, y wrapped into the
// box (FP64 wrap), so every coordinate is below max(nx, ny, |z|) in size.
__device__ __forceinline__ float4 prefilter_pos(const BridgeCtx& c, double x, double y, double z, int plt)
{
    const double nx = (double)c.p.box_nx, ny = (double)c.p.box_ny;
    return make_float4((float)(x - nx * floor(x / nx)), (float)(y - ny * floor(y / ny)), (float)z, __int_as_float(plt));
}

__global__ void k_br_scatter(BridgeCtx c)
{
    pdl_wait();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= c.R || !c.act[s]) return;
    const int k = c.start[c.key[s]] + c.slot[s];
    const double4_32a r = c.pos[s];
    c.fpos[k] = prefilter_pos(c, r.x, r.y, r.z, c.site_plt[s]);
    c.sid[k] = s;
    c.scell[k] = c.cell[s];
}

// One warp per active site, taken in bucket order from the sorted list (so
// neighbouring warps read the same cells); the lanes split every bucket's
// candidates and the warp keeps the lowest successful partner.
constexpr int kChooseThreads = 256;
__global__ void __launch_bounds__(kChooseThreads, 4)
    k_br_choose(BridgeCtx c, uint64_t step_host, const unsigned long long* __restrict__ step_dev)
{
    pdl_wait();
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    const int n_active = c.start[c.B - 1] + c.count[c.B - 1];
    const uint64_t step = current_step(step_dev, step_host);
    const bridge_params& p = c.p;
    const float nxf = (float)p.box_nx, nyf = (float)p.box_ny;
    const float inx = 1.0f / nxf, iny = 1.0f / nyf;
    // upper bound of P_f from the FP32 distance: P_f <= k_on dt, and the
    // exponent of Eq. 13 is a concave parabola in dev = |x_b - l_b|, largest
    // at dev = gamma, so its maximum over the distance interval is at gamma
    // clamped to the interval
    const float sk = c.f_sk, gam = c.f_gamma, lb = c.f_lb, kon0 = c.f_kon0;
    const bool shortcut = c.f_shortcut != 0;
    __shared__ int s_end[kChooseThreads / 32][32];
    __shared__ int s_base[kChooseThreads / 32][32];
    for (int w = warp; w < n_active; w += nwarps) {
        const int i = c.sid[w];
        const float4 fi = c.fpos[w];
        const int pi = __float_as_int(fi.w);
        const int4 ci = c.scell[w];
        const int cx = ci.x, cy = ci.y, cz = ci.z;
        SitePos ri{0.0, 0.0, 0.0};   // FP64 position, loaded only for the exact test
        bool have_ri = false;
        // FP32 distance error (coordinates rounded once, one subtraction, one
        // wrap, the norm) <= 4 ulp of the largest coordinate L plus ~1e-6
        // relative: eps bounds it with room to spare.  A candidate whose FP32
        // distance exceeds d_capture + eps is out of reach in FP64 too.
        const float L = fmaxf(fmaxf(nxf, nyf), fabsf(fi.z) + 4.0f * c.f_dcap);
        const float eps = 16.0f * L * 0x1.0p-23f + 1e-6f;
        const float reach = c.f_dcap + eps;
        const float reach2 = reach * reach;
        // the 27 neighbour buckets, one per lane, flattened into one index
        // range: candidate t lies in the bucket whose prefix interval holds it
        int k0 = 0, n = 0;
        if (lane < 27) {
            const int dx = lane % 3 - 1, dy = (lane / 3) % 3 - 1, dz = lane / 9 - 1;
            const int x = (cx + dx + c.gx) % c.gx, y = (cy + dy + c.gy) % c.gy;
            const int b = (int)bucket_of(c, x, y, cz + dz);
            k0 = c.start[b];
            n = c.count[b];
        }
        int incl = n;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += t;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        int* sh_end = s_end[threadIdx.x >> 5];
        int* sh_base = s_base[threadIdx.x >> 5];
        sh_end[lane] = incl;
        sh_base[lane] = k0 - (incl - n);   // candidate t of this bucket is fpos[t + base]
        __syncwarp();
        int best = -1;
        auto index_of = [&](int t) {
            int lo = 0;   // first bucket whose end exceeds t
#pragma unroll
            for (int step2 = 16; step2 > 0; step2 >>= 1)
                if (lo + step2 <= 26 && sh_end[lo + step2 - 1] <= t) lo += step2;
            return t + sh_base[lo];
        };
        auto visit = [&](int k, float4 f) {
            if (__float_as_int(f.w) == pi) return;
            float ex = f.x - fi.x, ey = f.y - fi.y;
            const float ez = f.z - fi.z;
            ex -= nxf * rintf(ex * inx);
            ey -= nyf * rintf(ey * iny);
            const float d2 = ex * ex + ey * ey + ez * ez;
            if (d2 > reach2) return;
            const int j = c.sid[k];
            if (best >= 0 && j >= best) return;
            const int a = i < j ? i : j, bb = i < j ? j : i;
            double u = -1.0;
            if (shortcut) {
                const float xb32 = sqrtf(d2);
                const float lo2 = xb32 - eps - lb, hi2 = xb32 + eps - lb;
                const float dlo = (lo2 <= 0.0f && hi2 >= 0.0f) ? 0.0f : fminf(fabsf(lo2), fabsf(hi2));
                const float dhi = fmaxf(fabsf(lo2), fabsf(hi2));
                const float dst = fminf(fmaxf(gam, dlo), dhi);
                float exu = sk * dst * (gam - 0.5f * dst);
                exu += 1e-5f * fabsf(exu) + 1e-5f;
                if (exu < -746.0f) return;   // exp of the FP64 exponent underflows: P_f = 0
                u = pair_uniform53(p.seed, (uint32_t)a, (uint32_t)bb, step, 17u);
                const double pf_up = fmax((double)(kon0 * expf(fminf(exu, 80.0f))) * 1.0001, 0x1.0p-54);
                if (u >= pf_up) return;
            }
            if (!have_ri) {
                const double4_32a pi4 = c.pos[i];
                ri = SitePos{pi4.x, pi4.y, pi4.z};
                have_ri = true;
            }
            const double4_32a pj4 = c.pos[j];
            const SitePos rj{pj4.x, pj4.y, pj4.z};
            double d[3];
            if (i < j)
                pair_vector(p, ri, rj, d);
            else
                pair_vector(p, rj, ri, d);
            const double xb = norm3_rn(d[0], d[1], d[2]);
            if (!(xb < p.d_capture)) return;
            const double dev = fabs(__dsub_rn(xb, p.l_b));
            const double exq =
                __ddiv_rn(__dmul_rn(__dmul_rn(p.sigma, dev), __dsub_rn(p.gamma, __dmul_rn(0.5, dev))), p.kT);
            const double kon_dt = __dmul_rn(p.kon0_dt, exp(exq));
            const double Pf = -expm1(-kon_dt);
            if (u < 0.0) u = pair_uniform53(p.seed, (uint32_t)a, (uint32_t)bb, step, 17u);
            if (u < Pf) best = j;
        };
        // two candidates per iteration, both loads issued before either is used
        for (int t = lane; t < total; t += 64) {
            const int ka = index_of(t);
            const bool two = t + 32 < total;
            const int kb = two ? index_of(t + 32) : ka;
            const float4 fa = c.fpos[ka];
            const float4 fb = c.fpos[kb];
            visit(ka, fa);
            if (two) visit(kb, fb);
        }
        __syncwarp();
        unsigned v = best < 0 ? 0xffffffffu : (unsigned)best;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, off));
        if (lane == 0) c.choice[i] = v == 0xffffffffu ? -1 : (int)v;
    }
}

__global__ void k_br_match(BridgeCtx c, unsigned long long* __restrict__ step_dev)
{
    pdl_wait();
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
    return check_cuda(launch_pdl(k_br_forces, dim3(blocks(c->R)), dim3(kBrThreads), 0, s, *c, X, F, M), "bridges_forces");
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
    int rc = check_cuda(cudaMemsetAsync(c->count, 0, sizeof(int) * ((size_t)c->B + c->nplt), s),
                        "bridges_step: clear counts");
    if (rc) return rc;
    rc = check_cuda(launch_pdl(k_br_boxes, dim3(c->nplt), dim3(kBrThreads), 0, s, v, X, M), "bridges_step: boxes");
    if (!rc) {
        const long long pairs = (long long)c->nplt * c->nplt;
        rc = check_cuda(launch_pdl(k_br_neighbors, dim3((unsigned)((pairs + kBrThreads - 1) / kBrThreads)), dim3(kBrThreads),
                                   0, s, v),
                        "bridges_step: neighbours");
    }
    if (!rc)
        rc = check_cuda(launch_pdl(k_br_active, dim3(blocks(c->R)), dim3(kBrThreads), 0, s, v, X, M, step_host, step_dev),
                        "bridges_step: active sites");
    if (!rc) rc = check_cuda(launch_pdl(k_br_scan, dim3(1), dim3(kScanThreads), 0, s, v), "bridges_step: scan");
    if (!rc)
        rc = check_cuda(launch_pdl(k_br_scatter, dim3(blocks(c->R)), dim3(kBrThreads), 0, s, v), "bridges_step: scatter");
    if (!rc) {
        // one warp per active site, grid-stride over the sorted active list
        const int warps_per_block = kChooseThreads / 32;
        int g = (c->R + warps_per_block - 1) / warps_per_block;
        g = g < 1 ? 1 : (g > 148 * 16 ? 148 * 16 : g);
        rc = check_cuda(launch_pdl(k_br_choose, dim3(g), dim3(kChooseThreads), 0, s, v, step_host, step_dev),
                        "bridges_step: choose");
    }
    if (!rc)
        rc = check_cuda(launch_pdl(k_br_match, dim3(blocks(c->R)), dim3(kBrThreads), 0, s, v, step_dev),
                        "bridges_step: match");
    if (rc) return rc;
    return check_launch("bridges_step");
}

namespace {

struct BrLayout {
    size_t site_plt, plt_nodes, pos, act, choice, key, slot, fpos, sid, cell, scell, count, start, box, nb, counters,
        node_plt, total;
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
    L.key = o;
    o += al256(4 * r);
    L.slot = o;
    o += al256(4 * r);
    L.fpos = o;
    o += al256(16 * r);
    L.sid = o;
    o += al256(4 * r);
    L.cell = o;
    o += al256(16 * r);
    L.scell = o;
    o += al256(16 * r);
    L.count = o;   // bucket counts, then the neighbour counts (cleared together)
    o += al256(4 * ((size_t)B + nplt));
    L.start = o;
    o += al256(4 * (size_t)B);
    L.box = o;
    o += al256(32 * (size_t)nplt);
    L.nb = o;
    o += al256(4 * (size_t)nplt * kMaxNb);
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
    c->key = (int*)(b + L.key);
    c->slot = (int*)(b + L.slot);
    c->fpos = (float4*)(b + L.fpos);
    c->sid = (int*)(b + L.sid);
    c->cell = (int4*)(b + L.cell);
    c->scell = (int4*)(b + L.scell);
    c->f_sk = (float)(p->sigma / p->kT);
    c->f_gamma = (float)p->gamma;
    c->f_lb = (float)p->l_b;
    c->f_kon0 = (float)p->kon0_dt;
    c->f_dcap = (float)p->d_capture;
    c->f_shortcut = std::isfinite(c->f_sk) && c->f_sk >= 0.0f && std::isfinite(c->f_kon0);
    c->count = (int*)(b + L.count);
    c->start = (int*)(b + L.start);
    c->box = (float4*)(b + L.box);
    c->nb = (int*)(b + L.nb);
    c->nbc = c->count + c->B;
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
    NvtxRange nvtx_range("bridges_forces");
    if (!c || !X || !F || M < 1) return set_error(PFSI_ERR_ARG, "bridges_forces: bad argument");
    return launch_bridge_forces(c, X, F, M, as_stream(stream));
}

extern "C" int bridges_step(bridge_ctx* c, const double* X, int M, uint64_t step, void* stream)
{
    NvtxRange nvtx_range("bridges_step");
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
