// membrane.cu -- hybrid membrane forces (Section 3.1, Eq. 2-11) for sm_103a.
//
// F = -grad(H_SCE + H_area + H_volume + H_bend + H_Morse) + F_wall per node:
//   H_SCE    sum over mesh edges k/2 (|R| - L0)^2                (Eq. 2-3)
//   H_area   k_s (S - S0)^2 / 2S0 + sum over triangles k_t (S_t - S0_t)^2 / 2S0_t  (Eq. 4)
//   H_volume k_v (V - V0)^2 / 2V0                                (Eq. 5)
//   H_bend   sum over edges k_b (1 - cos(phi - phi0)), phi the dihedral
//            (torsion) angle of the two triangles of the edge    (Eq. 6, reading)
//   H_Morse  sum over SCE pairs D[(1 - e^{-a(r - r0)})^2 - 1]
//   F_wall   F0 tau / (e^{tau eps} - 1) along +z on membrane nodes (Section 3.4.1)
//
// Design, three passes per call:
//   split     FP64 positions -> hi/lo float pairs (the only FP64 work besides
//             the per-platelet sums; B300's FP64 rate is a small fraction of
//             its FP32 rate);
//   elements  one thread per edge / triangle / Morse pair computes the
//             quantities that cancel at small strain (|R| - L0, S_t - S0_t,
//             phi - phi0, r - r0, the platelet's area change and volume) in
//             double-float arithmetic (ff.cuh), so forces keep ~7 digits at
//             any strain, and adds the per-platelet sums in FP64;
//             The same threads turn the scalars into FP32 force vectors, one
//             per (element, vertex): spring + bending for the four vertices
//             of an edge's dihedral chain, area gradients per triangle corner,
//             the Morse force per pair;
//   nodes     four lanes per node sum its element contributions from its own
//             lists (strided, independent loads, no atomics; a fixed shuffle
//             reduction) and apply the per-platelet global area and volume
//             terms and the wall repulsion.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "ff.cuh"
#include "pfsi_internal.cuh"

namespace pfsi {

namespace {

// ------------------------------------------------------------------ host topology
struct Topology {
    std::vector<int4> edge;   // (i, j, k, l)
    // per-node lists of element slots:
    //   esl: 4*edge + slot, slot 0..3 = vertex k, i, j, l of the edge's chain
    //   tcl: 4*triangle + corner, corner 0..2
    //   psl: 2*pair + side, side 0/1 = first/second node of the pair
    std::vector<int> esl_off, tcl_off, psl_off;
    std::vector<int> esl, tcl, psl;
};

int build_topology(int n, int nt, const int* tri, int np, const int* pairs, Topology& T,
                   std::string& err)
{
    for (int t = 0; t < 3 * nt; ++t)
        if (tri[t] < 0 || tri[t] >= n) {
            err = "triangle vertex index out of range";
            return PFSI_ERR_ARG;
        }
    for (int s = 0; s < 2 * np; ++s)
        if (pairs[s] < 0 || pairs[s] >= n) {
            err = "Morse pair index out of range";
            return PFSI_ERR_ARG;
        }
    struct D {
        int lo, hi, from, wing;
    };
    std::vector<D> d;
    d.reserve(3 * (size_t)nt);
    for (int t = 0; t < nt; ++t)
        for (int e = 0; e < 3; ++e) {
            const int a = tri[3 * t + e], b = tri[3 * t + (e + 1) % 3], c = tri[3 * t + (e + 2) % 3];
            if (a == b) {
                err = "degenerate triangle";
                return PFSI_ERR_ARG;
            }
            d.push_back({std::min(a, b), std::max(a, b), a, c});
        }
    std::sort(d.begin(), d.end(), [](const D& x, const D& y) {
        if (x.lo != y.lo) return x.lo < y.lo;
        if (x.hi != y.hi) return x.hi < y.hi;
        return x.from < y.from;
    });
    T.edge.clear();
    for (size_t s = 0; s < d.size();) {
        size_t e = s + 1;
        while (e < d.size() && d[e].lo == d[s].lo && d[e].hi == d[s].hi) ++e;
        if (e - s > 2) {
            err = "non-manifold edge (shared by more than two triangles)";
            return PFSI_ERR_ARG;
        }
        if (e - s == 2 && d[s].from == d[s + 1].from) {
            err = "inconsistently oriented triangles";
            return PFSI_ERR_ARG;
        }
        const int i = d[s].from, j = (i == d[s].lo) ? d[s].hi : d[s].lo;
        const int l = (e - s == 2) ? d[s + 1].wing : -1;
        T.edge.push_back(make_int4(i, j, d[s].wing, l));
        s = e;
    }
    const int ne = (int)T.edge.size();
    // per-node lists by counting sort
    auto csr = [n](std::vector<int>& off, std::vector<int>& list, const std::vector<int2>& owner_code) {
        off.assign(n + 1, 0);
        for (const int2& oc : owner_code) off[oc.x + 1]++;
        for (int v = 0; v < n; ++v) off[v + 1] += off[v];
        list.assign(owner_code.size(), 0);
        std::vector<int> fill(off.begin(), off.end() - 1);
        for (const int2& oc : owner_code) list[fill[oc.x]++] = oc.y;
    };
    std::vector<int2> oc;
    for (int e = 0; e < ne; ++e) {
        const int4 q = T.edge[e];
        oc.push_back(make_int2(q.x, 4 * e + 1));
        oc.push_back(make_int2(q.y, 4 * e + 2));
        if (q.w >= 0) {
            oc.push_back(make_int2(q.z, 4 * e + 0));
            oc.push_back(make_int2(q.w, 4 * e + 3));
        }
    }
    csr(T.esl_off, T.esl, oc);
    oc.clear();
    for (int t = 0; t < nt; ++t)
        for (int r = 0; r < 3; ++r) oc.push_back(make_int2(tri[3 * t + r], 4 * t + r));
    csr(T.tcl_off, T.tcl, oc);
    oc.clear();
    for (int q = 0; q < np; ++q) {
        oc.push_back(make_int2(pairs[2 * q], 2 * q));
        oc.push_back(make_int2(pairs[2 * q + 1], 2 * q + 1));
    }
    csr(T.psl_off, T.psl, oc);
    return PFSI_OK;
}

// Workspace layout: consecutive 256-byte aligned slices.
enum Slice {
    S_TRI, S_TRI_PLT, S_TRI_REST, S_EDGE, S_EDGE_REST, S_EDGE_PHI0, S_PAIR, S_PAIR_REST, S_ESL_OFF,
    S_ESL, S_TCL_OFF, S_TCL, S_PSL_OFF, S_PSL, S_NODE_PLT, S_IS_MEM, S_PLT_REST, S_PLT_ANCHOR, S_ACC,
    S_XH, S_XL, S_EOUT, S_TOUT, S_POUT, S_CHUNKS, S_PERM, S_PLT_RANGE, S_PLT_CHUNKS, S_CPART, S_PLT_SPAN, S_COUNT
};
struct Layout {
    size_t off[S_COUNT];
    size_t total;
};

Layout make_layout(int n, int nt, int ne, int np, int nplt, size_t n_esl, size_t n_tcl, size_t n_psl)
{
    const size_t N = n, T = nt, E = ne, P = np, Q = nplt;
    const size_t bytes[S_COUNT] = {
        12 * T, 4 * T, 32 * T, 16 * E, 16 * E, 16 * E, 8 * P, 16 * P, 4 * (N + 1), 4 * n_esl,
        4 * (N + 1), 4 * n_tcl, 4 * (N + 1), 4 * n_psl, 4 * N, N, 32 * Q, 4 * Q, 24 * Q, 12 * N, 12 * N,
        64 * E, 64 * T, 16 * P, 8 * ((N + kIbChunk - 1) / kIbChunk + Q), 4 * N, 8 * Q, 8 * Q,
        24 * ((N + kIbChunk - 1) / kIbChunk + Q), 32 * Q};
    Layout L;
    size_t o = 0;
    for (int s = 0; s < S_COUNT; ++s) {
        L.off[s] = o;
        o += (bytes[s] + 255) / 256 * 256;
    }
    L.total = o;
    return L;
}

// ------------------------------------------------------------------ host rest state
inline void dsub(const double* a, const double* b, double* r)
{
    r[0] = a[0] - b[0];
    r[1] = a[1] - b[1];
    r[2] = a[2] - b[2];
}
inline void dcross(const double* a, const double* b, double* r)
{
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}
inline double ddot(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
inline float2 split(double x)
{
    const float h = (float)x;
    return make_float2(h, (float)(x - (double)h));
}

// ------------------------------------------------------------------ device helpers
__device__ __forceinline__ float3 f3sub(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 f3cross(float3 a, float3 b)
{
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float f3dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// split positions: hi/lo floats of each coordinate, [3][n] each
struct Split {
    const float* h;
    const float* l;
    int n;
    __device__ __forceinline__ ff3 diff(int a, int b) const  // X_a - X_b, double-float
    {
        return {ff_diff(h[a], l[a], h[b], l[b]), ff_diff(h[n + a], l[n + a], h[n + b], l[n + b]),
                ff_diff(h[2 * n + a], l[2 * n + a], h[2 * n + b], l[2 * n + b])};
    }
};

// Pass 1: split FP64 positions into hi/lo floats; clear the per-platelet sums.
__device__ __forceinline__ void mem_split(const double* __restrict__ X, int n, float* __restrict__ xh,
                                          float* __restrict__ xl, double* __restrict__ acc, int nacc, int bx)
{
    const int t = bx * blockDim.x + threadIdx.x;
    if (t < 3 * n) {
        const double x = X[t];
        const float h = __double2float_rn(x);
        xh[t] = h;
        xl[t] = __double2float_rn(x - (double)h);
    }
    if (t < nacc) acc[t] = 0.0;
}

__global__ void __launch_bounds__(256) k_mem_split(const double* __restrict__ X, int n, float* __restrict__ xh,
                                                   float* __restrict__ xl, double* __restrict__ acc, int nacc)
{
    pdl_wait();
    mem_split(X, n, xh, xl, acc, nacc, blockIdx.x);
}

// Torsion gradient of the chain r1-r2-r3-r4 (Blondel and Karplus 1996), FP32,
// positions relative to r2.  g[0..3] = d phi / d r_a.
__device__ __forceinline__ void torsion_grad(float3 r1, float3 r3, float3 r4, float3 g[4])
{
    const float3 Fv = r1, G = make_float3(-r3.x, -r3.y, -r3.z), H = f3sub(r4, r3);
    const float3 A = f3cross(Fv, G), B = f3cross(H, G);
    const float A2 = f3dot(A, A), B2 = f3dot(B, B), gn = sqrtf(f3dot(G, G));
    const float FG = f3dot(Fv, G) / (A2 * gn), HG = f3dot(H, G) / (B2 * gn);
    const float ka = gn / A2, kb = gn / B2;
    g[0] = make_float3(-ka * A.x, -ka * A.y, -ka * A.z);
    g[3] = make_float3(kb * B.x, kb * B.y, kb * B.z);
    g[1] = make_float3((ka + FG) * A.x - HG * B.x, (ka + FG) * A.y - HG * B.y, (ka + FG) * A.z - HG * B.z);
    g[2] = make_float3(-FG * A.x + (HG - kb) * B.x, -FG * A.y + (HG - kb) * B.y, -FG * A.z + (HG - kb) * B.z);
}

__device__ __forceinline__ float3 ff3_float(ff3 a) { return make_float3(ff_float(a.x), ff_float(a.y), ff_float(a.z)); }

// Pass 2: one thread per edge, triangle or Morse pair.
//   edge:     spring magnitude k (|R| - L0)/|R| with |R|^2 - L0^2 in
//             double-float; bending dE/dphi = k_b sin(phi - phi0) with
//             sin(phi - phi0) = (y cos phi0 - x sin phi0)/(|A||B|), where for the
//             chain k-i-j-l  A = F x G, B = H x G, x = A.B, y = |G| (H.A);
//             writes the force on each of k, i, j, l (spring on i, j; bending
//             -dE/dphi grad phi on all four).
//   triangle: S_t - S0_t from 4(S^2 - S0^2) = da b + a0 db - dc (c + c0),
//             a = |e1|^2, b = |e2|^2, c = e1.e2 (da, db, dc in double-float);
//             writes per corner dS_t/dX (w = local coefficient k_t (S_t - S0_t)/S0_t)
//             and n/6 = (e1 x e2)/6 (dV/dX of every corner); adds S_t - S0_t and
//             the tetrahedron volume (1/6)(X_a - X_o).(e1 x e2) to its platelet's
//             FP64 sums.
//   pair:     Morse force on the first node, 2 D a (1 - e^{-a d}) e^{-a d} R/r,
//             d = r - r0 likewise.
// At most 48 registers (five blocks of 256 per SM; 8 bytes spilled): the
// channel's 178,000 elements then fit one wave, and the 500-platelet step is
// 24 us faster than at the 58 registers the compiler picks unbounded.  The
// single-chamber kernel takes six blocks (40 registers, 24 bytes spilled):
// full-scale step 1.596 -> 1.590 ms (seven or eight blocks spill ~160 bytes:
// 1.614 ms).
// One edge's contributions: out[0..3] = the force on chain vertex k, i, j, l
// (spring on i, j; bending -dE/dphi grad phi on all four); a boundary edge
// (q.w < 0) has the spring only, out[0] = out[3] = 0.  q: indices into X.
__device__ __forceinline__ void edge_forces(const Split& X, int4 q, float4 er, const float4* __restrict__ phi0, int e,
                                            const mem_params& P, float3 out[4])
{
    const ff3 dij = X.diff(q.y, q.x);
    const float qs = ff3_sqnorm_minus(dij, {er.x, er.y});
    const float r = sqrtf(er.x + qs);
    const float spring = P.k_spring * (qs / (r + er.z)) / r;
    const float3 r3 = ff3_float(dij);
    const float3 fs = make_float3(spring * r3.x, spring * r3.y, spring * r3.z);
    if (q.w >= 0) {
        float dE = 0.f;
        const ff3 Fv = X.diff(q.z, q.x), H = X.diff(q.w, q.y);
        if (P.k_b != 0.f) {
            const ff3 G = ff3_neg(dij);
            const ff3 A = ff3_cross(Fv, G), B = ff3_cross(H, G);
            const ff x = ff3_dot(A, B);
            const ff y = ff_mul(ff_sqrt(ff_add({er.x, er.y}, {qs, 0.f})), ff3_dot(H, A));
            const float4 ph = phi0[e];
            const ff num = ff_sub(ff_mul(y, {ph.x, ph.y}), ff_mul(x, {ph.z, ph.w}));
            dE = P.k_b * ff_float(num) / sqrtf(x.h * x.h + y.h * y.h);
        }
        float3 g[4];
        const float3 r1 = ff3_float(Fv), r4 = f3sub(ff3_float(H), make_float3(-r3.x, -r3.y, -r3.z));
        torsion_grad(r1, r3, r4, g);
        out[0] = make_float3(-dE * g[0].x, -dE * g[0].y, -dE * g[0].z);
        out[1] = make_float3(fs.x - dE * g[1].x, fs.y - dE * g[1].y, fs.z - dE * g[1].z);
        out[2] = make_float3(-fs.x - dE * g[2].x, -fs.y - dE * g[2].y, -fs.z - dE * g[2].z);
        out[3] = make_float3(-dE * g[3].x, -dE * g[3].y, -dE * g[3].z);
    } else {
        out[0] = out[3] = make_float3(0.f, 0.f, 0.f);
        out[1] = fs;
        out[2] = make_float3(-fs.x, -fs.y, -fs.z);
    }
}

// One triangle's area change S_t - S0_t (ds), its local coefficient
// k_t (S_t - S0_t)/S0_t (tsc), the corner gradients dS_t/dX (g[0..2]), the
// unnormalised normal e1 x e2 (nn) and 6 times the tetrahedron volume over
// the anchor o (V6).  a, b, cc, o: indices into X.
struct TriTerms {
    float ds, tsc;
    float3 g[3], nn;
    ff V6;
};
__device__ __forceinline__ TriTerms tri_terms(const Split& X, int a, int b, int cc, int o, float4 r0, float4 r1,
                                              const mem_params& P)
{
    TriTerms T;
    const ff3 e1 = X.diff(b, a), e2 = X.diff(cc, a);
    const float da = ff3_sqnorm_minus(e1, {r0.x, r0.y});
    const float db = ff3_sqnorm_minus(e2, {r0.z, r0.w});
    const float dc = ff3_dot_minus(e1, e2, {r1.x, r1.y});
    const float four = da * (r0.z + db) + r0.x * db - dc * ((r1.x + dc) + r1.x);
    const float S0 = r1.z, dS2 = 0.25f * four;
    T.ds = dS2 / (sqrtf(S0 * S0 + dS2) + S0);
    T.tsc = P.k_t * T.ds * r1.w;
    const float3 f1 = ff3_float(e1), f2 = ff3_float(e2);
    T.nn = f3cross(f1, f2);
    const float inv = 0.5f * rsqrtf(f3dot(T.nn, T.nn));
    const float3 nh = make_float3(T.nn.x * inv, T.nn.y * inv, T.nn.z * inv);  // nhat / 2
    T.g[0] = f3cross(nh, f3sub(f2, f1));
    T.g[1] = f3cross(nh, make_float3(-f2.x, -f2.y, -f2.z));
    T.g[2] = f3cross(nh, f1);
    T.V6 = ff3_dot(X.diff(a, o), ff3_cross(e1, e2));
    return T;
}

// Morse force on the first node of a pair (the second takes its opposite).
// A pair whose distance overflows FP32 (a node of a run that blew up, far
// away) gets the force the oracle's FP64 gives it there, zero, instead of the
// NaN of inf / inf.
__device__ __forceinline__ float3 pair_force(const Split& X, int i, int j, float4 pr, const mem_params& P)
{
    const ff3 d = X.diff(j, i);
    const float qs = ff3_sqnorm_minus(d, {pr.x, pr.y});
    const float r = sqrtf(pr.x + qs);
    if (!(r <= 3.0e38f)) return make_float3(0.f, 0.f, 0.f);
    const float ad = P.morse_a * (qs / (r + pr.z));
    const float sc = 2.0f * P.morse_D * P.morse_a * (-expm1f(-ad)) * expf(-ad) / r;
    const float3 R = ff3_float(d);
    return make_float3(sc * R.x, sc * R.y, sc * R.z);
}

__device__ __forceinline__ void mem_elements(const MemCtx& c, int bx)
{
    const int t = bx * blockDim.x + threadIdx.x;
    const Split X{c.xh, c.xl, c.n};
    const mem_params P = c.p;
    int plt = -1;
    ff dS{0.f, 0.f}, V6{0.f, 0.f};   // per-platelet sums, double-float (no FP64 arithmetic here)
    if (t < c.ne) {
        const int4 q = c.edge[t];
        float3 f[4];
        edge_forces(X, q, c.edge_rest[t], c.edge_phi0, t, P, f);
        float4* out = c.eout + 4 * (size_t)t;
        if (q.w >= 0) {
            out[0] = make_float4(f[0].x, f[0].y, f[0].z, 0.f);
            out[3] = make_float4(f[3].x, f[3].y, f[3].z, 0.f);
        }
        out[1] = make_float4(f[1].x, f[1].y, f[1].z, 0.f);
        out[2] = make_float4(f[2].x, f[2].y, f[2].z, 0.f);
    } else if (t < c.ne + c.nt) {
        const int k = t - c.ne;
        plt = c.tri_plt[k];
        const TriTerms T = tri_terms(X, c.tri[3 * k], c.tri[3 * k + 1], c.tri[3 * k + 2], c.plt_anchor[plt],
                                     c.tri_rest[2 * k], c.tri_rest[2 * k + 1], P);
        if (!c.tri_sums_only) {
            float4* out = c.tout + 4 * (size_t)k;
#pragma unroll
            for (int r = 0; r < 3; ++r) out[r] = make_float4(T.g[r].x, T.g[r].y, T.g[r].z, T.tsc);
            out[3] = make_float4(T.nn.x * (1.0f / 6.0f), T.nn.y * (1.0f / 6.0f), T.nn.z * (1.0f / 6.0f), 0.f);
        }
        V6 = T.V6;
        dS = ff{T.ds, 0.f};
    } else if (t < c.ne + c.nt + c.np) {
        const int s = t - c.ne - c.nt;
        const float3 f = pair_force(X, c.pair[2 * s], c.pair[2 * s + 1], c.pair_rest[s], P);
        c.pout[s] = make_float4(f.x, f.y, f.z, 0.f);
    }
    // per-platelet sums; triangles of a platelet are contiguous
    const int p0 = __shfl_sync(0xffffffffu, plt, 0);
    if (__all_sync(0xffffffffu, plt == p0)) {
        if (p0 >= 0) {
            for (int o = 16; o > 0; o >>= 1) {
                dS = ff_add(dS, ff{__shfl_down_sync(0xffffffffu, dS.h, o), __shfl_down_sync(0xffffffffu, dS.l, o)});
                V6 = ff_add(V6, ff{__shfl_down_sync(0xffffffffu, V6.h, o), __shfl_down_sync(0xffffffffu, V6.l, o)});
            }
            if ((threadIdx.x & 31) == 0) {
                atomicAdd(&c.acc[2 * p0], (double)dS.h + (double)dS.l);
                atomicAdd(&c.acc[2 * p0 + 1], ((double)V6.h + (double)V6.l) * (1.0 / 6.0));
            }
        }
    } else if (plt >= 0) {
        atomicAdd(&c.acc[2 * plt], (double)dS.h + (double)dS.l);
        atomicAdd(&c.acc[2 * plt + 1], ((double)V6.h + (double)V6.l) * (1.0 / 6.0));
    }
}

__global__ void __launch_bounds__(256, 6) k_mem_elements(const __grid_constant__ MemCtx c)
{
    pdl_wait();
    mem_elements(c, blockIdx.x);
}

// Pass 2b: per-platelet coefficients of the global area and volume terms
// (Eq. 4-5), k_s (S - S0)/S0 and k_v (V - V0)/V0, once per platelet.
__device__ __forceinline__ void mem_coef(const MemCtx& c, int bx)
{
    const int p = bx * blockDim.x + threadIdx.x;
    if (p >= c.nplt) return;
    const double* pr = c.plt_rest + 4 * p;  // S0, V0, 1/S0, 1/V0
    c.coef[p] = make_float2((float)((double)c.p.k_s * c.acc[2 * p] * pr[2]),
                            (float)((double)c.p.k_v * (c.acc[2 * p + 1] - pr[1]) * pr[3]));
}

__global__ void k_mem_coef(const __grid_constant__ MemCtx c)
{
    pdl_wait();
    mem_coef(c, blockIdx.x);
}

// Pass 3: the lanes of a node sum its element contributions and apply the
// per-platelet global area and volume coefficients and the wall repulsion.
// kNodeLanes lanes per node share its element slots (strided), then reduce by
// shuffles in a fixed order; the first lane adds the wall term and writes.
// Each lane first loads its first list entries of all three lists, then all
// their slots, so that its gathers are in flight together (a plain loop
// waits for each list entry, then its slot: channel step 61.8 -> 59.8 us).
// Two lanes per node, six edge, three triangle and two pair entries each in
// flight: full-scale membrane call 474 -> 435 us against four lanes with
// three, two and two (each lane also loads the node's list offsets and
// coefficients; one lane with twelve, six and three: 443 us).
constexpr int kNodeLanes = 2;
constexpr int kNodeThreads = 64;   // 32 nodes a block: full-scale step 1.573 -> 1.568 ms against 128

__device__ __forceinline__ void mem_nodes(float* __restrict__ F, const MemCtx& c, int bx)
{
    const int t = bx * blockDim.x + threadIdx.x;
    const int v = t / kNodeLanes, q = t % kNodeLanes;
    const bool on = v < c.n;
    const int n = c.n;
    const mem_params P = c.p;
    float fx = 0.f, fy = 0.f, fz = 0.f;
    if (on) {
        // the lane's first entries of each list, then their slots, all in
        // flight together; sums in list order, longer lists finish in loops
        constexpr int kE = 6, kT = 3, kP = 2;
        const int eb = c.esl_off[v] + q, ee = c.skip_edges ? eb : c.esl_off[v + 1];
        const int tb = c.tcl_off[v] + q, te = c.skip_tris ? tb : c.tcl_off[v + 1];
        const int pb = c.psl_off[v] + q, pe = c.psl_off[v + 1];
        int ei[kE], ti[kT], pi[kP];
#pragma unroll
        for (int u = 0; u < kE; ++u) ei[u] = eb + u * kNodeLanes < ee ? c.esl[eb + u * kNodeLanes] : -1;
#pragma unroll
        for (int u = 0; u < kT; ++u) ti[u] = tb + u * kNodeLanes < te ? c.tcl[tb + u * kNodeLanes] : -1;
#pragma unroll
        for (int u = 0; u < kP; ++u) pi[u] = pb + u * kNodeLanes < pe ? c.psl[pb + u * kNodeLanes] : -1;
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 ef[kE], tg[kT], tn[kT], pf[kP];
#pragma unroll
        for (int u = 0; u < kE; ++u) ef[u] = ei[u] >= 0 ? c.eout[ei[u]] : z4;
#pragma unroll
        for (int u = 0; u < kT; ++u) {
            tg[u] = ti[u] >= 0 ? c.tout[ti[u]] : z4;
            tn[u] = ti[u] >= 0 ? c.tout[ti[u] | 3] : z4;
        }
#pragma unroll
        for (int u = 0; u < kP; ++u) pf[u] = pi[u] >= 0 ? c.pout[pi[u] >> 1] : z4;
        const float2 cf = c.coef[c.node_plt[v]];
        const float cSg = cf.x, cV = cf.y;
#pragma unroll
        for (int u = 0; u < kE; ++u)
            if (ei[u] >= 0) {
                fx += ef[u].x;
                fy += ef[u].y;
                fz += ef[u].z;
            }
        for (int s = eb + kE * kNodeLanes; s < ee; s += kNodeLanes) {
            const float4 f = c.eout[c.esl[s]];
            fx += f.x;
            fy += f.y;
            fz += f.z;
        }
        // Eq. 4-5: F -= (k_t (S_t - S0_t)/S0_t + k_s (S - S0)/S0) dS_t/dX + k_v (V - V0)/V0 dV/dX
#pragma unroll
        for (int u = 0; u < kT; ++u)
            if (ti[u] >= 0) {
                const float cS = tg[u].w + cSg;
                fx -= cS * tg[u].x + cV * tn[u].x;
                fy -= cS * tg[u].y + cV * tn[u].y;
                fz -= cS * tg[u].z + cV * tn[u].z;
            }
        for (int s = tb + kT * kNodeLanes; s < te; s += kNodeLanes) {
            const int code = c.tcl[s];
            const float4 g = c.tout[code];
            const float4 n6 = c.tout[code | 3];
            const float cS = g.w + cSg;
            fx -= cS * g.x + cV * n6.x;
            fy -= cS * g.y + cV * n6.y;
            fz -= cS * g.z + cV * n6.z;
        }
#pragma unroll
        for (int u = 0; u < kP; ++u)
            if (pi[u] >= 0) {
                const float sg = (pi[u] & 1) ? -1.f : 1.f;
                fx += sg * pf[u].x;
                fy += sg * pf[u].y;
                fz += sg * pf[u].z;
            }
        for (int s = pb + kP * kNodeLanes; s < pe; s += kNodeLanes) {
            const int code = c.psl[s];
            const float4 f = c.pout[code >> 1];
            const float sg = (code & 1) ? -1.f : 1.f;
            fx += sg * f.x;
            fy += sg * f.y;
            fz += sg * f.z;
        }
    }
#pragma unroll
    for (int o = 1; o < kNodeLanes; o <<= 1) {
        fx += __shfl_xor_sync(0xffffffffu, fx, o);
        fy += __shfl_xor_sync(0xffffffffu, fy, o);
        fz += __shfl_xor_sync(0xffffffffu, fz, o);
    }
    if (!on || q != 0) return;
    // wall repulsion on surface nodes (Section 3.4.1)
    if (c.is_mem[v] && P.rep_F0 != 0.f) {
        const float eps = fmaxf((c.xh[2 * n + v] - P.z_wall) + c.xl[2 * n + v], P.rep_eps_min);
        fz += P.rep_F0 * P.rep_tau / expm1f(P.rep_tau * eps);
    }
    F[v] = fx;
    F[n + v] = fy;
    F[2 * n + v] = fz;
}

__global__ void __launch_bounds__(kNodeThreads) k_mem_nodes(float* __restrict__ F, const __grid_constant__ MemCtx c)
{
    pdl_wait();
    mem_nodes(F, c, blockIdx.x);
}

// The four passes over several chambers' membranes, one launch each (see
// Multi): the same per-thread code, each chamber's share of the grid
// indexing its own elements and nodes.
struct SplitArgs {
    const double* X;
    int n;
    float* xh;
    float* xl;
    double* acc;
    int nacc;
};
struct NodesArgs {
    float* F;
    MemCtx c;
};

__global__ void __launch_bounds__(256) k_mem_split_multi(const __grid_constant__ Multi<SplitArgs> t)
{
    pdl_wait();
    const int e = multi_entry(t, blockIdx.x);
    const SplitArgs& a = t.a[e];
    mem_split(a.X, a.n, a.xh, a.xl, a.acc, a.nacc, blockIdx.x - t.first[e]);
}

__global__ void __launch_bounds__(256, 5) k_mem_elements_multi(const __grid_constant__ Multi<MemCtx> t)
{
    pdl_wait();
    const int e = multi_entry(t, blockIdx.x);
    mem_elements(t.a[e], blockIdx.x - t.first[e]);
}

__global__ void k_mem_coef_multi(const __grid_constant__ Multi<MemCtx> t)
{
    pdl_wait();
    const int e = multi_entry(t, blockIdx.x);
    mem_coef(t.a[e], blockIdx.x - t.first[e]);
}

__global__ void __launch_bounds__(kNodeThreads) k_mem_nodes_multi(const __grid_constant__ Multi<NodesArgs> t)
{
    pdl_wait();
    const int e = multi_entry(t, blockIdx.x);
    mem_nodes(t.a[e].F, t.a[e].c, blockIdx.x - t.first[e]);
}

int node_blocks(const MemCtx* c) { return (int)(((long long)c->n * kNodeLanes + kNodeThreads - 1) / kNodeThreads); }

// ------------------------------------------------------------------ fused pass
// One block per platelet does all three passes for its nodes: the hi/lo
// split of its positions (or the presplit one) goes to shared memory; a
// first sweep over its triangles sums the area change and the volume
// (double-float per thread, then a fixed-order block reduction), which gives
// the platelet's global coefficients; then its edges, triangles (again, now
// with the coefficients) and Morse pairs add their vertex forces into
// per-node shared accumulators, and each node adds the wall term and writes
// F once.  The accumulators are 64-bit fixed point (2^-48 force units, each
// contribution clamped to +-256 units, far beyond any force of the model:
// ~1e-3 at 3 % strain): integer addition is exact, so the sums do not depend
// on the order the atomics land in, and 64-bit integer shared atomics are
// native where FP32 shared atomics loop on compare-and-swap.  The
// per-element arithmetic is that of the element pass (edge_forces,
// tri_terms, pair_force).  No per-element force slots go through global
// memory: at full scale those were ~820 MB written and read back per step.
constexpr int kFusedThreads = 1024;
constexpr size_t kFusedBytesPerNode = 3 * sizeof(long long) + 6 * sizeof(float);   // accumulators, hi, lo
constexpr size_t kFusedScratch = 2 * (kFusedThreads / 32) * sizeof(ff) + 64;
constexpr size_t kFusedMaxSmem = 227 * 1024;
constexpr float kFixedScale = 0x1p48f, kFixedUnit = 0x1p-48f, kFixedClamp = 256.0f;

__device__ __forceinline__ unsigned long long to_fixed(float f)
{
    return (unsigned long long)__float2ll_rn(fminf(fmaxf(f, -kFixedClamp), kFixedClamp) * kFixedScale);
}
__device__ __forceinline__ void fadd3(unsigned long long* acc, int nn, int u, float3 f)
{
    atomicAdd(acc + u, to_fixed(f.x));
    atomicAdd(acc + nn + u, to_fixed(f.y));
    atomicAdd(acc + 2 * nn + u, to_fixed(f.z));
}
__device__ __forceinline__ void fsub3(unsigned long long* acc, int nn, int u, float3 f)
{
    fadd3(acc, nn, u, make_float3(-f.x, -f.y, -f.z));
}

__device__ __forceinline__ void mem_fused(const MemCtx& c, const double* __restrict__ X, float* __restrict__ F,
                                          int presplit, int p)
{
    extern __shared__ __align__(16) unsigned long long fsm[];
    const int4 s0 = c.plt_span[2 * p], s1 = c.plt_span[2 * p + 1];
    const int v0 = s0.x, nn = s0.y, e0 = s0.z, ne = s0.w, t0 = s1.x, nt = s1.y, q0 = s1.z, nq = s1.w;
    const int n = c.n;
    unsigned long long* acc = fsm;                       // [3][nn] fixed-point force accumulators
    float* hx = reinterpret_cast<float*>(fsm + 3 * nn);  // [3][nn] high floats
    float* lx = hx + 3 * nn;                             // [3][nn] low floats
    ff* red = reinterpret_cast<ff*>(lx + 3 * nn);        // [2][warps]
    float* cf = reinterpret_cast<float*>(red + 2 * (kFusedThreads / 32));   // the two coefficients
    const mem_params P = c.p;

    for (int u = threadIdx.x; u < nn; u += kFusedThreads) {
        const int v = v0 + u;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            float h, l;
            if (presplit) {
                h = c.xh[d * n + v];
                l = c.xl[d * n + v];
            } else {   // the split pass's arithmetic; the split also stays in xh, xl
                const double x = X[d * n + v];
                h = __double2float_rn(x);
                l = __double2float_rn(x - (double)h);
                c.xh[d * n + v] = h;
                c.xl[d * n + v] = l;
            }
            hx[d * nn + u] = h;
            lx[d * nn + u] = l;
            acc[d * nn + u] = 0ull;
        }
    }
    __syncthreads();
    const Split Xs{hx, lx, nn};   // local node indices v - v0
    const int o = c.plt_anchor[p] - v0;

    // sweep 1: the platelet's area change and volume
    ff dS{0.f, 0.f}, V6{0.f, 0.f};
    for (int k = threadIdx.x; k < nt; k += kFusedThreads) {
        const int t = t0 + k;
        const TriTerms T = tri_terms(Xs, c.tri[3 * t] - v0, c.tri[3 * t + 1] - v0, c.tri[3 * t + 2] - v0, o,
                                     c.tri_rest[2 * t], c.tri_rest[2 * t + 1], P);
        dS = ff_add(dS, ff{T.ds, 0.f});
        V6 = ff_add(V6, T.V6);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        dS = ff_add(dS, ff{__shfl_down_sync(0xffffffffu, dS.h, off), __shfl_down_sync(0xffffffffu, dS.l, off)});
        V6 = ff_add(V6, ff{__shfl_down_sync(0xffffffffu, V6.h, off), __shfl_down_sync(0xffffffffu, V6.l, off)});
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        red[warp] = dS;
        red[kFusedThreads / 32 + warp] = V6;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double S = 0.0, V = 0.0;
        for (int w = 0; w < kFusedThreads / 32; ++w) {
            S += (double)red[w].h + (double)red[w].l;
            V += (double)red[kFusedThreads / 32 + w].h + (double)red[kFusedThreads / 32 + w].l;
        }
        V *= 1.0 / 6.0;
        const double* pr = c.plt_rest + 4 * p;  // S0, V0, 1/S0, 1/V0
        const float2 k2 = make_float2((float)((double)P.k_s * S * pr[2]), (float)((double)P.k_v * (V - pr[1]) * pr[3]));
        c.acc[2 * p] = S;
        c.acc[2 * p + 1] = V;
        c.coef[p] = k2;
        cf[0] = k2.x;
        cf[1] = k2.y;
    }
    __syncthreads();
    const float cSg = cf[0], cV = cf[1];

    // sweep 2: vertex forces into the accumulators
    for (int k = threadIdx.x; k < ne; k += kFusedThreads) {
        const int e = e0 + k;
        int4 q = c.edge[e];
        q.x -= v0;
        q.y -= v0;
        float3 f[4];
        if (q.w >= 0) {
            q.z -= v0;
            q.w -= v0;
        }
        edge_forces(Xs, q, c.edge_rest[e], c.edge_phi0, e, P, f);
        fadd3(acc, nn, q.x, f[1]);
        fadd3(acc, nn, q.y, f[2]);
        if (q.w >= 0) {
            fadd3(acc, nn, q.z, f[0]);
            fadd3(acc, nn, q.w, f[3]);
        }
    }
    // Eq. 4-5: F -= (k_t (S_t - S0_t)/S0_t + k_s (S - S0)/S0) dS_t/dX + k_v (V - V0)/V0 dV/dX
    for (int k = threadIdx.x; k < nt; k += kFusedThreads) {
        const int t = t0 + k;
        const int a = c.tri[3 * t] - v0, b = c.tri[3 * t + 1] - v0, cc = c.tri[3 * t + 2] - v0;
        const TriTerms T = tri_terms(Xs, a, b, cc, o, c.tri_rest[2 * t], c.tri_rest[2 * t + 1], P);
        const float cS = T.tsc + cSg;
        const float3 n6 = make_float3(T.nn.x * (1.0f / 6.0f), T.nn.y * (1.0f / 6.0f), T.nn.z * (1.0f / 6.0f));
        const int corner[3] = {a, b, cc};
#pragma unroll
        for (int r = 0; r < 3; ++r)
            fsub3(acc, nn, corner[r],
                  make_float3(cS * T.g[r].x + cV * n6.x, cS * T.g[r].y + cV * n6.y, cS * T.g[r].z + cV * n6.z));
    }
    for (int k = threadIdx.x; k < nq; k += kFusedThreads) {
        const int s = q0 + k;
        const int i = c.pair[2 * s] - v0, j = c.pair[2 * s + 1] - v0;
        const float3 f = pair_force(Xs, i, j, c.pair_rest[s], P);
        fadd3(acc, nn, i, f);
        fsub3(acc, nn, j, f);
    }
    __syncthreads();
    for (int u = threadIdx.x; u < nn; u += kFusedThreads) {
        const int v = v0 + u;
        float fz = __ll2float_rn((long long)acc[2 * nn + u]) * kFixedUnit;
        if (c.is_mem[v] && P.rep_F0 != 0.f) {   // wall repulsion on surface nodes (Section 3.4.1)
            const float eps = fmaxf((hx[2 * nn + u] - P.z_wall) + lx[2 * nn + u], P.rep_eps_min);
            fz += P.rep_F0 * P.rep_tau / expm1f(P.rep_tau * eps);
        }
        F[v] = __ll2float_rn((long long)acc[u]) * kFixedUnit;
        F[n + v] = __ll2float_rn((long long)acc[nn + u]) * kFixedUnit;
        F[2 * n + v] = fz;
    }
}

__global__ void __launch_bounds__(kFusedThreads, 1) k_mem_fused(const __grid_constant__ MemCtx c,
                                                               const double* __restrict__ X, float* __restrict__ F,
                                                               int presplit)
{
    pdl_wait();
    mem_fused(c, X, F, presplit, blockIdx.x);
}

// The fused pass over several chambers' platelets, one launch (see Multi):
// entry e owns one block per platelet of its chamber.
struct FusedArgs {
    MemCtx c;
    const double* X;
    float* F;
};
static_assert(sizeof(Multi<FusedArgs>) <= 32000, "the list must fit the kernel parameter space");

__global__ void __launch_bounds__(kFusedThreads, 1) k_mem_fused_multi(const __grid_constant__ Multi<FusedArgs> t)
{
    pdl_wait();
    const int e = multi_entry(t, blockIdx.x);
    mem_fused(t.a[e].c, t.a[e].X, t.a[e].F, 0, blockIdx.x - t.first[e]);
}

size_t fused_smem(const MemCtx* c) { return (size_t)c->span_max_nodes * kFusedBytesPerNode + kFusedScratch; }

// The fused pass runs when path 1 asks for it, for the plain membrane
// (springs and bending included) of a mesh that groups its elements by
// platelet.  It is not the default: at full scale it takes as long as the
// three passes (533 against 461 us; 463 with FP32 shared atomics, whose
// order is not fixed), because the double-float element arithmetic, not
// the slot traffic, bounds both; a block per platelet also leaves a
// 10-platelet channel on ten SMs (131 against 18 us).  Its sums are exact,
// so its forces do not depend on scheduling.
bool uses_fused(const MemCtx* c) { return c->plt_span && !c->skip_edges && c->path == 1; }

int fused_prepare()
{
    int rc = check_cuda(cudaFuncSetAttribute(k_mem_fused, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kFusedMaxSmem),
                        "membrane: fused pass shared memory");
    if (!rc)
        rc = check_cuda(cudaFuncSetAttribute(k_mem_fused_multi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kFusedMaxSmem),
                        "membrane: fused pass shared memory");
    return rc;
}

int launch_scalars(MemCtx* c, const double* X, cudaStream_t s, bool presplit = false)
{
    int rc = PFSI_OK;
    if (!presplit) {
        const int nsplit = 3 * c->n > 2 * c->nplt ? 3 * c->n : 2 * c->nplt;
        rc = check_cuda(launch_pdl(k_mem_split, dim3((nsplit + 255) / 256), dim3(256), 0, s, X, c->n, c->xh, c->xl,
                                   c->acc, 2 * c->nplt),
                        "membrane: split positions");
        if (rc) return rc;
    }
    const int nel = c->ne + c->nt + c->np;
    if (nel > 0) {
        rc = check_cuda(launch_pdl(k_mem_elements, dim3((nel + 255) / 256), dim3(256), 0, s, *c),
                        "membrane: element scalars");
    }
    if (!rc) {
        rc = check_cuda(launch_pdl(k_mem_coef, dim3((c->nplt + 127) / 128), dim3(128), 0, s, *c),
                        "membrane: platelet coefficients");
    }
    return rc;
}

}  // namespace

int launch_membrane_forces(MemCtx* c, const double* X, float* F, cudaStream_t s, bool presplit)
{
    if (uses_fused(c))
        return check_cuda(launch_pdl(k_mem_fused, dim3(c->nplt), dim3(kFusedThreads), fused_smem(c), s, *c, X, F,
                                     presplit ? 1 : 0),
                          "membrane_forces: fused pass");
    int rc = launch_scalars(c, X, s, presplit);
    if (rc) return rc;
    return check_cuda(launch_pdl(k_mem_nodes, dim3(node_blocks(c)), dim3(kNodeThreads), 0, s, F, *c),
                      "membrane_forces");
}

// The remainder's node pass (Morse pairs and wall repulsion only): one thread
// per node, its pair slots summed in list order (the first four loaded
// together).
__global__ void __launch_bounds__(256) k_mem_nodes_pairs(float* __restrict__ F, const __grid_constant__ MemCtx c)
{
    pdl_wait();
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= c.n) return;
    const int n = c.n;
    const int pb = c.psl_off[v], pe = c.psl_off[v + 1];
    constexpr int kP = 4;
    int pi[kP];
    float4 pf[kP];
#pragma unroll
    for (int u = 0; u < kP; ++u) pi[u] = pb + u < pe ? c.psl[pb + u] : -1;
#pragma unroll
    for (int u = 0; u < kP; ++u) pf[u] = pi[u] >= 0 ? c.pout[pi[u] >> 1] : make_float4(0.f, 0.f, 0.f, 0.f);
    float fx = 0.f, fy = 0.f, fz = 0.f;
#pragma unroll
    for (int u = 0; u < kP; ++u)
        if (pi[u] >= 0) {
            const float sg = (pi[u] & 1) ? -1.f : 1.f;
            fx += sg * pf[u].x;
            fy += sg * pf[u].y;
            fz += sg * pf[u].z;
        }
    for (int q = pb + kP; q < pe; ++q) {
        const int code = c.psl[q];
        const float4 f = c.pout[code >> 1];
        const float sg = (code & 1) ? -1.f : 1.f;
        fx += sg * f.x;
        fy += sg * f.y;
        fz += sg * f.z;
    }
    const mem_params P = c.p;
    if (c.is_mem[v] && P.rep_F0 != 0.f) {   // wall repulsion (Section 3.4.1), as the full node pass
        const float eps = fmaxf((c.xh[2 * n + v] - P.z_wall) + c.xl[2 * n + v], P.rep_eps_min);
        fz += P.rep_F0 * P.rep_tau / expm1f(P.rep_tau * eps);
    }
    F[v] = fx;
    F[n + v] = fy;
    F[2 * n + v] = fz;
}

int launch_membrane_remainder(MemCtx* c, const double* X, float* F, cudaStream_t s, bool presplit)
{
    MemCtx g = *c;
    g.p.k_spring = 0.f;
    g.p.k_t = 0.f;
    g.p.k_b = 0.f;
    g.ne = 0;            // element ids start at the triangles
    g.skip_edges = 1;
    g.skip_tris = 1;     // the nodes take no triangle slots ...
    g.tri_sums_only = 1; // ... and the triangles write none, only the per-platelet sums
    int rc = launch_scalars(&g, X, s, presplit);
    if (rc) return rc;
    if (g.np > 0)
        return check_cuda(launch_pdl(k_mem_nodes_pairs, dim3((g.n + 255) / 256), dim3(256), 0, s, F, g),
                          "membrane: pairs and wall");
    // no Morse pairs: F starts at zero and the caller adds the wall term
    return check_cuda(cudaMemsetAsync(F, 0, sizeof(float) * 3 * (size_t)g.n, s), "membrane: clear forces");
}

int launch_membrane_forces_multi(const Chamber* ch, int n, cudaStream_t s)
{
    std::vector<Multi<SplitArgs>> split;
    std::vector<Multi<MemCtx>> elems, coef;
    std::vector<Multi<NodesArgs>> nodes;
    std::vector<Multi<FusedArgs>> fused;
    std::vector<size_t> fused_bytes;
    for (int i = 0; i < n; ++i) {
        MemCtx* c = ch[i].mem;
        if (uses_fused(c)) {
            const bool fresh = fused.empty() || fused.back().full();
            multi_push(fused, FusedArgs{*c, ch[i].X, ch[i].F}, c->nplt);
            if (fresh) fused_bytes.push_back(0);
            fused_bytes.back() = std::max(fused_bytes.back(), fused_smem(c));
            continue;
        }
        const int nsplit = 3 * c->n > 2 * c->nplt ? 3 * c->n : 2 * c->nplt;
        multi_push(split, SplitArgs{ch[i].X, c->n, c->xh, c->xl, c->acc, 2 * c->nplt}, (nsplit + 255) / 256);
        multi_push(elems, *c, (c->ne + c->nt + c->np + 255) / 256);
        multi_push(coef, *c, (c->nplt + 127) / 128);
        multi_push(nodes, NodesArgs{ch[i].F, *c}, node_blocks(c));
    }
    int rc = PFSI_OK;
    for (const auto& t : split)
        if (!rc) rc = check_cuda(launch_pdl(k_mem_split_multi, dim3(t.blocks()), dim3(256), 0, s, t), "membrane: split");
    for (const auto& t : elems)
        if (!rc)
            rc = check_cuda(launch_pdl(k_mem_elements_multi, dim3(t.blocks()), dim3(256), 0, s, t), "membrane: elements");
    for (const auto& t : coef)
        if (!rc) rc = check_cuda(launch_pdl(k_mem_coef_multi, dim3(t.blocks()), dim3(128), 0, s, t), "membrane: coef");
    for (const auto& t : nodes)
        if (!rc) rc = check_cuda(launch_pdl(k_mem_nodes_multi, dim3(t.blocks()), dim3(kNodeThreads), 0, s, t), "membrane: nodes");
    for (size_t u = 0; u < fused.size() && !rc; ++u)
        rc = check_cuda(launch_pdl(k_mem_fused_multi, dim3(fused[u].blocks()), dim3(kFusedThreads), fused_bytes[u], s,
                                   fused[u]),
                        "membrane: fused pass");
    return rc;
}

}  // namespace pfsi

using namespace pfsi;

extern "C" int membrane_query_workspace(int n_nodes, int n_tri, const int* tri, int n_pairs, int n_plt,
                                        size_t* bytes)
{
    if (!bytes || n_nodes < 1 || n_tri < 0 || n_pairs < 0 || n_plt < 1 || (n_tri > 0 && !tri))
        return set_error(PFSI_ERR_ARG, "membrane_query_workspace: bad argument");
    Topology T;
    std::string err;
    int rc = build_topology(n_nodes, n_tri, tri, 0, nullptr, T, err);
    if (rc) return set_error(rc, "membrane_query_workspace: " + err);
    const Layout L = make_layout(n_nodes, n_tri, (int)T.edge.size(), n_pairs, n_plt, T.esl.size(), T.tcl.size(),
                                 2 * (size_t)n_pairs);
    *bytes = L.total;
    return PFSI_OK;
}

extern "C" int membrane_create(const mem_params* p, int n, int nt, const int* tri, int np,
                               const int* pairs, int nplt, const int* node_plt,
                               const unsigned char* is_membrane, const double* X0, void* ws,
                               size_t ws_bytes, mem_ctx** out)
{
    if (!p || !out || !ws || !node_plt || !is_membrane || !X0 || n < 1 || nt < 0 || np < 0 || nplt < 1 ||
        (nt > 0 && !tri) || (np > 0 && !pairs))
        return set_error(PFSI_ERR_ARG, "membrane_create: bad argument");
    if (!aligned(ws, 256)) return set_error(PFSI_ERR_ARG, "membrane_create: workspace must be 256-byte aligned");
    if ((long long)3 * n > INT_MAX) return set_error(PFSI_ERR_ARG, "membrane_create: too many nodes");
    for (int v = 0; v < n; ++v)
        if (node_plt[v] < 0 || node_plt[v] >= nplt)
            return set_error(PFSI_ERR_ARG, "membrane_create: node platelet index out of range");
    Topology T;
    std::string err;
    int rc = build_topology(n, nt, tri, np, pairs, T, err);
    if (rc) return set_error(rc, "membrane_create: " + err);
    const int ne = (int)T.edge.size();
    const Layout L = make_layout(n, nt, ne, np, nplt, T.esl.size(), T.tcl.size(), T.psl.size());
    if (ws_bytes < L.total) return set_error(PFSI_ERR_ARG, "membrane_create: workspace too small");
    for (int t = 0; t < nt; ++t)
        for (int r = 1; r < 3; ++r)
            if (node_plt[tri[3 * t + r]] != node_plt[tri[3 * t]])
                return set_error(PFSI_ERR_ARG, "membrane_create: triangle spans two platelets");
    for (int t = 1; t < nt; ++t)
        if (node_plt[tri[3 * t]] < node_plt[tri[3 * (t - 1)]])
            return set_error(PFSI_ERR_ARG, "membrane_create: triangles must be grouped by platelet");

    auto pos = [&](int v, double* r) {
        r[0] = X0[v];
        r[1] = X0[n + v];
        r[2] = X0[2 * n + v];
    };
    // rest state, FP64 on the host, stored as double-float where it enters a
    // cancelling difference
    std::vector<int> tri_plt(nt);
    std::vector<float4> tri_rest(2 * (size_t)nt);
    std::vector<double> S0(nplt, 0.0), V0(nplt, 0.0);
    std::vector<int> anchor(nplt, -1);
    for (int v = 0; v < n; ++v)
        if (is_membrane[v] && anchor[node_plt[v]] < 0) anchor[node_plt[v]] = v;
    for (int q = 0; q < nplt; ++q)
        if (anchor[q] < 0) anchor[q] = 0;
    for (int t = 0; t < nt; ++t) {
        double a[3], b[3], cc[3], e1[3], e2[3], nn[3], o[3], ra[3];
        pos(tri[3 * t], a);
        pos(tri[3 * t + 1], b);
        pos(tri[3 * t + 2], cc);
        dsub(b, a, e1);
        dsub(cc, a, e2);
        dcross(e1, e2, nn);
        const double St = 0.5 * std::sqrt(ddot(nn, nn));
        if (!(St > 0.0)) return set_error(PFSI_ERR_ARG, "membrane_create: zero-area rest triangle");
        const float2 A0 = split(ddot(e1, e1)), B0 = split(ddot(e2, e2)), C0 = split(ddot(e1, e2));
        tri_rest[2 * t] = make_float4(A0.x, A0.y, B0.x, B0.y);
        tri_rest[2 * t + 1] = make_float4(C0.x, C0.y, (float)St, (float)(1.0 / St));
        const int q = node_plt[tri[3 * t]];
        tri_plt[t] = q;
        pos(anchor[q], o);
        dsub(a, o, ra);
        S0[q] += St;
        V0[q] += ddot(ra, nn) / 6.0;
    }
    std::vector<float4> edge_rest(ne), edge_phi0(ne);
    for (int e = 0; e < ne; ++e) {
        const int4 q = T.edge[e];
        double ri[3], rj[3], R[3];
        pos(q.x, ri);
        pos(q.y, rj);
        dsub(rj, ri, R);
        const double L2 = ddot(R, R);
        const float2 l2 = split(L2);
        edge_rest[e] = make_float4(l2.x, l2.y, (float)std::sqrt(L2), 0.f);
        edge_phi0[e] = make_float4(1.f, 0.f, 0.f, 0.f);
        if (q.w >= 0) {
            double r1[3], r4[3], Fv[3], G[3], H[3], A[3], B[3], BxA[3];
            pos(q.z, r1);
            pos(q.w, r4);
            dsub(r1, ri, Fv);
            dsub(ri, rj, G);
            dsub(r4, rj, H);
            dcross(Fv, G, A);
            dcross(H, G, B);
            dcross(B, A, BxA);
            const double phi = std::atan2(ddot(BxA, G) / std::sqrt(ddot(G, G)), ddot(A, B));
            const float2 cs = split(std::cos(phi)), sn = split(std::sin(phi));
            edge_phi0[e] = make_float4(cs.x, cs.y, sn.x, sn.y);
        }
    }
    std::vector<float4> pair_rest(np);
    for (int s = 0; s < np; ++s) {
        double a[3], b[3], R[3];
        pos(pairs[2 * s], a);
        pos(pairs[2 * s + 1], b);
        dsub(b, a, R);
        const double r2 = ddot(R, R);
        const float2 q2 = split(r2);
        pair_rest[s] = make_float4(q2.x, q2.y, (float)std::sqrt(r2), 0.f);
    }
    std::vector<double> plt_rest(4 * (size_t)nplt);
    for (int q = 0; q < nplt; ++q) {
        if ((p->k_s != 0.f && !(S0[q] > 0.0)) || (p->k_v != 0.f && !(V0[q] > 0.0)))
            return set_error(PFSI_ERR_ARG, "membrane_create: platelet without area or volume");
        plt_rest[4 * q] = S0[q];
        plt_rest[4 * q + 1] = V0[q];
        plt_rest[4 * q + 2] = S0[q] > 0.0 ? 1.0 / S0[q] : 0.0;
        plt_rest[4 * q + 3] = V0[q] > 0.0 ? 1.0 / V0[q] : 0.0;
    }
    std::vector<uint8_t> mem_v(is_membrane, is_membrane + n);
    // IB chunk table: the nodes of each platelet in Morton order of the rest
    // shape (10 bits per axis over the platelet's own box), cut into runs of at
    // most kIbChunk; a chunk then covers a compact patch, and the spreading and
    // interpolation tiles of its bounding box stay small.
    std::vector<int> perm(n);
    {
        std::vector<double> lo(3 * (size_t)nplt, 1e300), hi(3 * (size_t)nplt, -1e300);
        for (int v = 0; v < n; ++v)
            for (int d = 0; d < 3; ++d) {
                const double x = X0[(size_t)d * n + v];
                lo[3 * node_plt[v] + d] = std::min(lo[3 * node_plt[v] + d], x);
                hi[3 * node_plt[v] + d] = std::max(hi[3 * node_plt[v] + d], x);
            }
        std::vector<unsigned long long> key(n);
        for (int v = 0; v < n; ++v) {
            const int q = node_plt[v];
            double ext = 0.0;
            for (int d = 0; d < 3; ++d) ext = std::max(ext, hi[3 * q + d] - lo[3 * q + d]);
            unsigned long long k = 0;
            for (int d = 0; d < 3; ++d) {
                const double t = ext > 0.0 ? (X0[(size_t)d * n + v] - lo[3 * q + d]) / ext : 0.0;
                const unsigned c = (unsigned)std::min(1023.0, std::max(0.0, t * 1023.0));
                for (int b = 0; b < 10; ++b) k |= (unsigned long long)((c >> b) & 1u) << (3 * b + d);
            }
            key[v] = ((unsigned long long)q << 32) | k;
        }
        for (int v = 0; v < n; ++v) perm[v] = v;
        std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return key[a] < key[b]; });
    }
    std::vector<int2> chunks;
    for (int v = 0; v < n;) {
        int e = v + 1;
        while (e < n && node_plt[perm[e]] == node_plt[perm[v]] && e - v < kIbChunk) ++e;
        chunks.push_back(make_int2(v, e - v));
        v = e;
    }
    // each platelet's nodes are one run of perm
    std::vector<int2> plt_range(nplt, make_int2(0, 0));
    for (int v = 0; v < n; ++v) {
        int2& r = plt_range[node_plt[perm[v]]];
        if (r.y == 0) r.x = v;
        r.y += 1;
    }
    // and one run of chunks
    std::vector<int2> plt_chunks(nplt, make_int2(0, 0));
    for (int ci = 0; ci < (int)chunks.size(); ++ci) {
        int2& r = plt_chunks[node_plt[perm[chunks[ci].x]]];
        if (r.y == 0) r.x = ci;
        r.y += 1;
    }
    {
        int runs = 1;
        for (int v = 1; v < n; ++v) runs += node_plt[v] != node_plt[v - 1];
        if (runs != nplt)
            return set_error(PFSI_ERR_ARG, "membrane_create: the nodes of each platelet must be contiguous");
    }
    // per-platelet spans of nodes, edges, triangles and Morse pairs for the
    // fused pass: usable when each platelet's elements are one run and its
    // positions and force accumulators fit in shared memory
    std::vector<int4> span(2 * (size_t)nplt, make_int4(0, 0, 0, 0));
    bool spans_ok = true;
    int span_max = 0;
    {
        // (first, count) of each platelet's run of elements into dst[2 q + at].z, .w
        auto runs_of = [&](int count, auto owner, int4* dst, int at) {
            std::vector<int> seen(nplt, 0);
            for (int e = 0; e < count;) {
                const int q = owner(e);
                int f = e + 1;
                while (f < count && owner(f) == q) ++f;
                if (seen[q]) spans_ok = false;   // a platelet's elements in two runs
                seen[q] = 1;
                dst[2 * q + at].z = e;
                dst[2 * q + at].w = f - e;
                e = f;
            }
        };
        for (int v = 0; v < n;) {
            int f = v + 1;
            while (f < n && node_plt[f] == node_plt[v]) ++f;
            span[2 * node_plt[v]].x = v;
            span[2 * node_plt[v]].y = f - v;
            span_max = std::max(span_max, f - v);
            v = f;
        }
        runs_of(ne, [&](int e) { return node_plt[T.edge[e].x]; }, span.data(), 0);
        std::vector<int4> tp(2 * (size_t)nplt, make_int4(0, 0, 0, 0));
        runs_of(nt, [&](int t) { return node_plt[tri[3 * t]]; }, tp.data(), 0);
        runs_of(np, [&](int s) { return node_plt[pairs[2 * s]]; }, tp.data(), 1);
        for (int q = 0; q < nplt; ++q) {
            span[2 * q + 1] = make_int4(tp[2 * q].z, tp[2 * q].w, tp[2 * q + 1].z, tp[2 * q + 1].w);
        }
        for (int s = 0; s < np && spans_ok; ++s)
            if (node_plt[pairs[2 * s]] != node_plt[pairs[2 * s + 1]]) spans_ok = false;
        if ((size_t)span_max * kFusedBytesPerNode + kFusedScratch > kFusedMaxSmem) spans_ok = false;
    }

    char* base = static_cast<char*>(ws);
    auto up = [&](int slice, const void* src, size_t bytes) -> int {
        if (bytes == 0) return PFSI_OK;
        return check_cuda(cudaMemcpy(base + L.off[slice], src, bytes, cudaMemcpyHostToDevice),
                          "membrane_create: upload");
    };
    rc = up(S_TRI, tri, sizeof(int) * 3 * (size_t)nt);
    if (!rc) rc = up(S_TRI_PLT, tri_plt.data(), sizeof(int) * nt);
    if (!rc) rc = up(S_TRI_REST, tri_rest.data(), sizeof(float4) * tri_rest.size());
    if (!rc) rc = up(S_EDGE, T.edge.data(), sizeof(int4) * ne);
    if (!rc) rc = up(S_EDGE_REST, edge_rest.data(), sizeof(float4) * ne);
    if (!rc) rc = up(S_EDGE_PHI0, edge_phi0.data(), sizeof(float4) * ne);
    if (!rc) rc = up(S_PAIR, pairs, sizeof(int) * 2 * (size_t)np);
    if (!rc) rc = up(S_PAIR_REST, pair_rest.data(), sizeof(float4) * np);
    if (!rc) rc = up(S_ESL_OFF, T.esl_off.data(), sizeof(int) * (n + 1));
    if (!rc) rc = up(S_ESL, T.esl.data(), sizeof(int) * T.esl.size());
    if (!rc) rc = up(S_TCL_OFF, T.tcl_off.data(), sizeof(int) * (n + 1));
    if (!rc) rc = up(S_TCL, T.tcl.data(), sizeof(int) * T.tcl.size());
    if (!rc) rc = up(S_PSL_OFF, T.psl_off.data(), sizeof(int) * (n + 1));
    if (!rc) rc = up(S_PSL, T.psl.data(), sizeof(int) * T.psl.size());
    if (!rc) rc = up(S_NODE_PLT, node_plt, sizeof(int) * n);
    if (!rc) rc = up(S_IS_MEM, mem_v.data(), n);
    if (!rc) rc = up(S_PLT_REST, plt_rest.data(), sizeof(double) * plt_rest.size());
    if (!rc) rc = up(S_PLT_ANCHOR, anchor.data(), sizeof(int) * nplt);
    if (!rc) rc = up(S_CHUNKS, chunks.data(), sizeof(int2) * chunks.size());
    if (!rc) rc = up(S_PERM, perm.data(), sizeof(int) * perm.size());
    if (!rc) rc = up(S_PLT_RANGE, plt_range.data(), sizeof(int2) * plt_range.size());
    if (!rc) rc = up(S_PLT_CHUNKS, plt_chunks.data(), sizeof(int2) * plt_chunks.size());
    if (!rc) rc = up(S_PLT_SPAN, span.data(), sizeof(int4) * span.size());
    if (!rc && spans_ok) rc = fused_prepare();
    if (rc) return rc;

    mem_ctx* c = new mem_ctx();
    c->p = *p;
    c->n = n;
    c->nt = nt;
    c->ne = ne;
    c->np = np;
    c->nplt = nplt;
    auto at = [&](int slice) { return base + L.off[slice]; };
    c->tri = reinterpret_cast<const int*>(at(S_TRI));
    c->tri_plt = reinterpret_cast<const int*>(at(S_TRI_PLT));
    c->tri_rest = reinterpret_cast<const float4*>(at(S_TRI_REST));
    c->edge = reinterpret_cast<const int4*>(at(S_EDGE));
    c->edge_rest = reinterpret_cast<const float4*>(at(S_EDGE_REST));
    c->edge_phi0 = reinterpret_cast<const float4*>(at(S_EDGE_PHI0));
    c->pair = reinterpret_cast<const int*>(at(S_PAIR));
    c->pair_rest = reinterpret_cast<const float4*>(at(S_PAIR_REST));
    c->esl_off = reinterpret_cast<const int*>(at(S_ESL_OFF));
    c->esl = reinterpret_cast<const int*>(at(S_ESL));
    c->tcl_off = reinterpret_cast<const int*>(at(S_TCL_OFF));
    c->tcl = reinterpret_cast<const int*>(at(S_TCL));
    c->psl_off = reinterpret_cast<const int*>(at(S_PSL_OFF));
    c->psl = reinterpret_cast<const int*>(at(S_PSL));
    c->node_plt = reinterpret_cast<const int*>(at(S_NODE_PLT));
    c->is_mem = reinterpret_cast<const uint8_t*>(at(S_IS_MEM));
    c->plt_rest = reinterpret_cast<const double*>(at(S_PLT_REST));
    c->plt_anchor = reinterpret_cast<const int*>(at(S_PLT_ANCHOR));
    c->chunks = reinterpret_cast<const int2*>(at(S_CHUNKS));
    c->perm = reinterpret_cast<const int*>(at(S_PERM));
    c->plt_range = reinterpret_cast<const int2*>(at(S_PLT_RANGE));
    c->plt_chunks = reinterpret_cast<const int2*>(at(S_PLT_CHUNKS));
    c->cpart = reinterpret_cast<double*>(at(S_CPART));
    c->n_chunks = (int)chunks.size();
    c->acc = reinterpret_cast<double*>(at(S_ACC));
    c->coef = reinterpret_cast<float2*>(c->acc + 2 * (size_t)nplt);
    c->xh = reinterpret_cast<float*>(at(S_XH));
    c->xl = reinterpret_cast<float*>(at(S_XL));
    c->eout = reinterpret_cast<float4*>(at(S_EOUT));
    c->tout = reinterpret_cast<float4*>(at(S_TOUT));
    c->pout = reinterpret_cast<float4*>(at(S_POUT));
    c->plt_span = spans_ok ? reinterpret_cast<const int4*>(at(S_PLT_SPAN)) : nullptr;
    c->span_max_nodes = span_max;
    c->path = 0;
    *out = c;
    return PFSI_OK;
}

extern "C" int membrane_set_path(mem_ctx* c, int path)
{
    if (!c || path < 0 || path > 1) return set_error(PFSI_ERR_ARG, "membrane_set_path: bad argument");
    c->path = path;
    return PFSI_OK;
}

extern "C" int membrane_get_path(const mem_ctx* c, int* fused)
{
    if (!c || !fused) return set_error(PFSI_ERR_ARG, "membrane_get_path: null argument");
    *fused = uses_fused(c) ? 1 : 0;
    return PFSI_OK;
}

extern "C" int membrane_destroy(mem_ctx* c)
{
    delete c;
    return PFSI_OK;
}

extern "C" int membrane_set_params(mem_ctx* c, const mem_params* p)
{
    if (!c || !p) return set_error(PFSI_ERR_ARG, "membrane_set_params: null argument");
    c->p = *p;
    return PFSI_OK;
}

extern "C" int membrane_forces(mem_ctx* c, const double* X, float* F, void* stream)
{
    NvtxRange nvtx_range("membrane_forces");
    if (!c || !X || !F) return set_error(PFSI_ERR_ARG, "membrane_forces: null argument");
    if (!aligned(X, 8) || !aligned(F, 4)) return set_error(PFSI_ERR_ARG, "membrane_forces: misaligned arrays");
    return launch_membrane_forces(c, X, F, as_stream(stream));
}

namespace pfsi {
namespace {

// Per-platelet sums of the node positions and node counts into acc[4 * nplt]
// (x, y, z sums then counts); lanes of a warp that share a platelet reduce
// first.
// One block per platelet: the FP64 sum of its nodes in a fixed order
// (strided partial sums, then a fixed-order block reduction), divided by
// the count.
constexpr int kCentroidThreads = 512;
__global__ void __launch_bounds__(kCentroidThreads)
    k_centroids(const double* __restrict__ X, int n, const int* __restrict__ perm, const int2* __restrict__ range,
                double* __restrict__ out)
{
    pdl_wait();
    const int p = blockIdx.x;
    const int2 r = range[p];
    double s[3] = {0.0, 0.0, 0.0};
#pragma unroll 4
    for (int k = threadIdx.x; k < r.y; k += kCentroidThreads) {
        const int v = perm[r.x + k];
        s[0] += X[v];
        s[1] += X[n + v];
        s[2] += X[2 * n + v];
    }
    __shared__ double red[3][kCentroidThreads];
    for (int d = 0; d < 3; ++d) red[d][threadIdx.x] = s[d];
    __syncthreads();
    for (int h = kCentroidThreads / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h)
            for (int d = 0; d < 3; ++d) red[d][threadIdx.x] += red[d][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x < 3) out[3 * p + threadIdx.x] = r.y > 0 ? red[threadIdx.x][0] / (double)r.y : 0.0;
}

// Platelet centroids from the chunk sums of the advected positions that the
// interpolation pass wrote (part[3 chunk + d], FP64 sums over the chunk's
// nodes): one warp per platelet, lane l adding chunks l, l + 32, ... of it,
// then a fixed shuffle tree (deterministic).
__global__ void __launch_bounds__(128) k_centroids_from_chunks(const double* __restrict__ part,
                                                               const int2* __restrict__ plt_chunks,
                                                               const int2* __restrict__ range, int nplt,
                                                               double* __restrict__ out)
{
    pdl_wait();
    const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (p >= nplt) return;   // whole warps
    const int2 r = plt_chunks[p];
    double s[3] = {0.0, 0.0, 0.0};
    for (int k = lane; k < r.y; k += 32)
        for (int d = 0; d < 3; ++d) s[d] += part[3 * (r.x + k) + d];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s[d] += __shfl_down_sync(0xffffffffu, s[d], o);
    if (lane == 0) {
        const int cnt = range[p].y;
        for (int d = 0; d < 3; ++d) out[3 * p + d] = cnt > 0 ? s[d] / (double)cnt : 0.0;
    }
}

}  // namespace

int launch_centroids_from_chunks(MemCtx* c, double* out, cudaStream_t s)
{
    if (c->nplt == 0) return PFSI_OK;
    return check_cuda(launch_pdl(k_centroids_from_chunks, dim3((c->nplt + 3) / 4), dim3(128), 0, s,
                                 (const double*)c->cpart, c->plt_chunks, (const int2*)c->plt_range, c->nplt, out),
                      "platelet centroids");
}
}  // namespace pfsi

extern "C" int membrane_centroids(mem_ctx* c, const double* X, double* out_dev, void* stream)
{
    NvtxRange nvtx_range("membrane_centroids");
    if (!c || !X || !out_dev) return set_error(PFSI_ERR_ARG, "membrane_centroids: null argument");
    if (!aligned(out_dev, 8)) return set_error(PFSI_ERR_ARG, "membrane_centroids: misaligned output");
    cudaStream_t s = as_stream(stream);
    if (c->nplt == 0) return PFSI_OK;
    return check_cuda(launch_pdl(k_centroids, dim3(c->nplt), dim3(kCentroidThreads), 0, s, X, c->n, c->perm,
                                 (const int2*)c->plt_range, out_dev),
                      "membrane_centroids");
}

extern "C" int membrane_measure(mem_ctx* c, const double* X, double* out_host, void* stream)
{
    NvtxRange nvtx_range("membrane_measure");
    if (!c || !X || !out_host) return set_error(PFSI_ERR_ARG, "membrane_measure: null argument");
    cudaStream_t s = as_stream(stream);
    int rc = launch_scalars(c, X, s);
    if (rc) return rc;
    std::vector<double> acc(2 * (size_t)c->nplt), rest(4 * (size_t)c->nplt);
    rc = check_cuda(cudaMemcpyAsync(acc.data(), c->acc, sizeof(double) * acc.size(), cudaMemcpyDeviceToHost, s),
                    "membrane_measure: copy");
    if (!rc)
        rc = check_cuda(cudaMemcpyAsync(rest.data(), c->plt_rest, sizeof(double) * rest.size(),
                                        cudaMemcpyDeviceToHost, s), "membrane_measure: copy");
    if (!rc) rc = check_cuda(cudaStreamSynchronize(s), "membrane_measure: synchronise");
    if (rc) return rc;
    for (int q = 0; q < c->nplt; ++q) {
        out_host[2 * q] = rest[4 * q] + acc[2 * q];
        out_host[2 * q + 1] = acc[2 * q + 1];
    }
    return PFSI_OK;
}
