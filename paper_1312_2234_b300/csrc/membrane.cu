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
//   nodes     one thread per node gathers those scalars times FP32
//             directions over its own lists of springs, triangles, dihedral
//             roles and Morse partners: each force is written once, without
//             atomics, in a fixed order.
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
    std::vector<int> spr_off, tri_off, dih_off, mor_off;
    std::vector<int2> spr, mor;
    std::vector<int4> trl;
    std::vector<int> dih;
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
    // counting sort into per-node lists
    auto csr = [n](std::vector<int>& off, const std::vector<int>& owner) {
        off.assign(n + 1, 0);
        for (int o : owner) off[o + 1]++;
        for (int v = 0; v < n; ++v) off[v + 1] += off[v];
    };
    std::vector<int> owner;
    // springs
    owner.clear();
    for (int e = 0; e < ne; ++e) {
        owner.push_back(T.edge[e].x);
        owner.push_back(T.edge[e].y);
    }
    csr(T.spr_off, owner);
    T.spr.assign(owner.size(), make_int2(0, 0));
    {
        std::vector<int> fill(T.spr_off.begin(), T.spr_off.end() - 1);
        for (int e = 0; e < ne; ++e) {
            T.spr[fill[T.edge[e].x]++] = make_int2(T.edge[e].y, e);
            T.spr[fill[T.edge[e].y]++] = make_int2(T.edge[e].x, e);
        }
    }
    // triangles, rotated so that the node comes first (orientation kept)
    owner.clear();
    for (int t = 0; t < 3 * nt; ++t) owner.push_back(tri[t]);
    csr(T.tri_off, owner);
    T.trl.assign(owner.size(), make_int4(0, 0, 0, 0));
    {
        std::vector<int> fill(T.tri_off.begin(), T.tri_off.end() - 1);
        for (int t = 0; t < nt; ++t)
            for (int r = 0; r < 3; ++r) {
                const int a = tri[3 * t + r], b = tri[3 * t + (r + 1) % 3], c = tri[3 * t + (r + 2) % 3];
                T.trl[fill[a]++] = make_int4(b, c, t, 0);
            }
    }
    // dihedral roles: chain k-i-j-l, role 0..3
    owner.clear();
    for (int e = 0; e < ne; ++e)
        if (T.edge[e].w >= 0) {
            owner.push_back(T.edge[e].z);
            owner.push_back(T.edge[e].x);
            owner.push_back(T.edge[e].y);
            owner.push_back(T.edge[e].w);
        }
    csr(T.dih_off, owner);
    T.dih.assign(owner.size(), 0);
    {
        std::vector<int> fill(T.dih_off.begin(), T.dih_off.end() - 1);
        for (int e = 0; e < ne; ++e)
            if (T.edge[e].w >= 0) {
                const int v[4] = {T.edge[e].z, T.edge[e].x, T.edge[e].y, T.edge[e].w};
                for (int r = 0; r < 4; ++r) T.dih[fill[v[r]]++] = 4 * e + r;
            }
    }
    // Morse partners
    owner.clear();
    for (int s = 0; s < 2 * np; ++s) owner.push_back(pairs[s]);
    csr(T.mor_off, owner);
    T.mor.assign(owner.size(), make_int2(0, 0));
    {
        std::vector<int> fill(T.mor_off.begin(), T.mor_off.end() - 1);
        for (int s = 0; s < np; ++s) {
            T.mor[fill[pairs[2 * s]]++] = make_int2(pairs[2 * s + 1], s);
            T.mor[fill[pairs[2 * s + 1]]++] = make_int2(pairs[2 * s], s);
        }
    }
    return PFSI_OK;
}

// Workspace layout: consecutive 256-byte aligned slices.
enum Slice {
    S_TRI, S_TRI_PLT, S_TRI_REST, S_EDGE, S_EDGE_REST, S_EDGE_PHI0, S_PAIR, S_PAIR_REST, S_SPR_OFF,
    S_SPR, S_TRI_OFF, S_TRL, S_DIH_OFF, S_DIH, S_MOR_OFF, S_MOR, S_NODE_PLT, S_IS_MEM, S_PLT_REST,
    S_PLT_ANCHOR, S_ACC, S_XH, S_XL, S_ESC, S_TSC, S_MSC, S_COUNT
};
struct Layout {
    size_t off[S_COUNT];
    size_t total;
};

Layout make_layout(int n, int nt, int ne, int np, int nplt, size_t n_spr, size_t n_trl, size_t n_dih,
                   size_t n_mor)
{
    const size_t N = n, T = nt, E = ne, P = np, Q = nplt;
    const size_t bytes[S_COUNT] = {
        12 * T, 4 * T, 32 * T, 16 * E, 16 * E, 16 * E, 8 * P, 16 * P, 4 * (N + 1), 8 * n_spr,
        4 * (N + 1), 16 * n_trl, 4 * (N + 1), 4 * n_dih, 4 * (N + 1), 8 * n_mor, 4 * N, N, 32 * Q,
        4 * Q, 16 * Q, 12 * N, 12 * N, 8 * E, 4 * T, 4 * P};
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
    __device__ __forceinline__ float3 rel(int a, int b) const  // X_a - X_b rounded to FP32
    {
        return make_float3((h[a] - h[b]) + (l[a] - l[b]), (h[n + a] - h[n + b]) + (l[n + a] - l[n + b]),
                           (h[2 * n + a] - h[2 * n + b]) + (l[2 * n + a] - l[2 * n + b]));
    }
};

// Pass 1: split FP64 positions into hi/lo floats; clear the per-platelet sums.
__global__ void __launch_bounds__(256) k_mem_split(const double* __restrict__ X, int n, float* __restrict__ xh,
                                                   float* __restrict__ xl, double* __restrict__ acc, int nacc)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < 3 * n) {
        const double x = X[t];
        const float h = __double2float_rn(x);
        xh[t] = h;
        xl[t] = __double2float_rn(x - (double)h);
    }
    if (t < nacc) acc[t] = 0.0;
}

// Pass 2: the cancelling scalars, one thread per edge, triangle or Morse pair.
//   edge:     spring magnitude k (|R| - L0)/|R| with |R|^2 - L0^2 in
//             double-float; bending dE/dphi = k_b sin(phi - phi0) with
//             sin(phi - phi0) = (y cos phi0 - x sin phi0)/(|A||B|), where for the
//             chain k-i-j-l  A = F x G, B = H x G, x = A.B, y = |G| (H.A).
//   triangle: S_t - S0_t from 4(S^2 - S0^2) = da b + a0 db - dc (c + c0),
//             a = |e1|^2, b = |e2|^2, c = e1.e2 (da, db, dc in double-float);
//             adds S_t - S0_t and the tetrahedron volume (1/6)(X_a - X_o).(e1 x e2)
//             to its platelet's FP64 sums.
//   pair:     Morse magnitude 2 D a (1 - e^{-a d}) e^{-a d}/r, d = r - r0 likewise.
__global__ void __launch_bounds__(256) k_mem_elements(MemCtx c)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const Split X{c.xh, c.xl, c.n};
    const mem_params P = c.p;
    int plt = -1;
    double dS = 0.0, V = 0.0;
    if (t < c.ne) {
        const int4 q = c.edge[t];
        const float4 er = c.edge_rest[t];
        const ff3 dij = X.diff(q.y, q.x);
        const float qs = ff3_sqnorm_minus(dij, {er.x, er.y});
        const float r = sqrtf(er.x + qs);
        const float spring = P.k_spring * (qs / (r + er.z)) / r;
        float bend = 0.f;
        if (q.w >= 0 && P.k_b != 0.f) {
            const ff3 Fv = X.diff(q.z, q.x), G = ff3_neg(dij), H = X.diff(q.w, q.y);
            const ff3 A = ff3_cross(Fv, G), B = ff3_cross(H, G);
            const ff x = ff3_dot(A, B);
            const ff y = ff_mul(ff_sqrt(ff_add({er.x, er.y}, {qs, 0.f})), ff3_dot(H, A));
            const float4 ph = c.edge_phi0[t];
            const ff num = ff_sub(ff_mul(y, {ph.x, ph.y}), ff_mul(x, {ph.z, ph.w}));
            bend = P.k_b * ff_float(num) / sqrtf(x.h * x.h + y.h * y.h);
        }
        c.esc[t] = make_float2(spring, bend);
    } else if (t < c.ne + c.nt) {
        const int k = t - c.ne;
        const int a = c.tri[3 * k], b = c.tri[3 * k + 1], cc = c.tri[3 * k + 2];
        plt = c.tri_plt[k];
        const float4 r0 = c.tri_rest[2 * k], r1 = c.tri_rest[2 * k + 1];
        const ff3 e1 = X.diff(b, a), e2 = X.diff(cc, a);
        const float da = ff3_sqnorm_minus(e1, {r0.x, r0.y});
        const float db = ff3_sqnorm_minus(e2, {r0.z, r0.w});
        const float dc = ff3_dot_minus(e1, e2, {r1.x, r1.y});
        const float four = da * (r0.z + db) + r0.x * db - dc * ((r1.x + dc) + r1.x);
        const float S0 = r1.z, dS2 = 0.25f * four;
        const float ds = dS2 / (sqrtf(S0 * S0 + dS2) + S0);
        c.tsc[k] = P.k_t * ds * r1.w;
        const ff v6 = ff3_dot(X.diff(a, c.plt_anchor[plt]), ff3_cross(e1, e2));
        dS = (double)ds;
        V = ((double)v6.h + (double)v6.l) * (1.0 / 6.0);
    } else if (t < c.ne + c.nt + c.np) {
        const int s = t - c.ne - c.nt;
        const int i = c.pair[2 * s], j = c.pair[2 * s + 1];
        const float4 pr = c.pair_rest[s];
        const float qs = ff3_sqnorm_minus(X.diff(j, i), {pr.x, pr.y});
        const float r = sqrtf(pr.x + qs);
        const float ad = P.morse_a * (qs / (r + pr.z));
        c.msc[s] = 2.0f * P.morse_D * P.morse_a * (-expm1f(-ad)) * expf(-ad) / r;
    }
    // per-platelet sums; triangles of a platelet are contiguous
    const int p0 = __shfl_sync(0xffffffffu, plt, 0);
    if (__all_sync(0xffffffffu, plt == p0)) {
        if (p0 >= 0) {
            for (int o = 16; o > 0; o >>= 1) {
                dS += __shfl_down_sync(0xffffffffu, dS, o);
                V += __shfl_down_sync(0xffffffffu, V, o);
            }
            if ((threadIdx.x & 31) == 0) {
                atomicAdd(&c.acc[2 * p0], dS);
                atomicAdd(&c.acc[2 * p0 + 1], V);
            }
        }
    } else if (plt >= 0) {
        atomicAdd(&c.acc[2 * plt], dS);
        atomicAdd(&c.acc[2 * plt + 1], V);
    }
}

// Pass 3: one thread per node gathers its terms: the precise scalars of pass
// 2 times FP32 directions.  No atomics, fixed order.
__global__ void __launch_bounds__(128) k_mem_nodes(float* __restrict__ F, MemCtx c)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= c.n) return;
    const int n = c.n;
    const Split X{c.xh, c.xl, n};
    const mem_params P = c.p;
    float fx = 0.f, fy = 0.f, fz = 0.f;

    // Eq. 3 springs: F_i = k (|R| - L0) R/|R|, R = X_j - X_i
    for (int s = c.spr_off[v]; s < c.spr_off[v + 1]; ++s) {
        const int2 e = c.spr[s];
        const float sc = c.esc[e.y].x;
        const float3 R = X.rel(e.x, v);
        fx += sc * R.x;
        fy += sc * R.y;
        fz += sc * R.z;
    }

    // Eq. 4-5: dS_t/dX_i = (1/2) nhat x (X_b - X_a) for the outward triangle
    // (i, a, b); dV/dX_i = (1/6) sum (X_a - X_i) x (X_b - X_i) over the fan.
    const int plt = c.node_plt[v];
    const double* pr = c.plt_rest + 4 * plt;  // S0, V0, 1/S0, 1/V0
    const float cSg = (float)((double)P.k_s * c.acc[2 * plt] * pr[2]);
    const float cV = (float)((double)P.k_v * (c.acc[2 * plt + 1] - pr[1]) * pr[3]);
    for (int s = c.tri_off[v]; s < c.tri_off[v + 1]; ++s) {
        const int4 t = c.trl[s];
        const float3 e1 = X.rel(t.x, v), e2 = X.rel(t.y, v);
        const float3 nn = f3cross(e1, e2);
        const float inv = rsqrtf(f3dot(nn, nn));
        const float3 gS = f3cross(make_float3(nn.x * inv, nn.y * inv, nn.z * inv), f3sub(e2, e1));
        const float cS = c.tsc[t.z] + cSg;
        fx -= 0.5f * cS * gS.x + cV * nn.x * (1.0f / 6.0f);
        fy -= 0.5f * cS * gS.y + cV * nn.y * (1.0f / 6.0f);
        fz -= 0.5f * cS * gS.z + cV * nn.z * (1.0f / 6.0f);
    }

    // bending: F -= dE/dphi grad(phi) for this node's role in the chain
    // k-i-j-l (Blondel and Karplus 1996 gradient of the torsion angle)
    if (P.k_b != 0.f) {
        for (int s = c.dih_off[v]; s < c.dih_off[v + 1]; ++s) {
            const int code = c.dih[s];
            const int e = code >> 2, role = code & 3;
            const int4 q = c.edge[e];
            const float3 r1 = X.rel(q.z, v), r2 = X.rel(q.x, v), r3 = X.rel(q.y, v), r4 = X.rel(q.w, v);
            const float3 Fv = f3sub(r1, r2), G = f3sub(r2, r3), H = f3sub(r4, r3);
            const float3 A = f3cross(Fv, G), B = f3cross(H, G);
            const float A2 = f3dot(A, A), B2 = f3dot(B, B), gn = sqrtf(f3dot(G, G));
            float ca = 0.f, cb = 0.f;  // grad = ca A + cb B
            if (role == 0) {
                ca = -gn / A2;
            } else if (role == 3) {
                cb = gn / B2;
            } else {
                const float FG = f3dot(Fv, G) / (A2 * gn), HG = f3dot(H, G) / (B2 * gn);
                if (role == 1) {
                    ca = gn / A2 + FG;
                    cb = -HG;
                } else {
                    ca = -FG;
                    cb = -gn / B2 + HG;
                }
            }
            const float dE = c.esc[e].y;
            fx -= dE * (ca * A.x + cb * B.x);
            fy -= dE * (ca * A.y + cb * B.y);
            fz -= dE * (ca * A.z + cb * B.z);
        }
    }

    // Morse pairs: F_i = (dU/dr)/r R, R = X_j - X_i
    for (int s = c.mor_off[v]; s < c.mor_off[v + 1]; ++s) {
        const int2 pr2 = c.mor[s];
        const float sc = c.msc[pr2.y];
        const float3 R = X.rel(pr2.x, v);
        fx += sc * R.x;
        fy += sc * R.y;
        fz += sc * R.z;
    }

    // wall repulsion on surface nodes (Section 3.4.1)
    if (c.is_mem[v] && P.rep_F0 != 0.f) {
        const float eps = fmaxf((c.xh[2 * n + v] - P.z_wall) + c.xl[2 * n + v], P.rep_eps_min);
        fz += P.rep_F0 * P.rep_tau / expm1f(P.rep_tau * eps);
    }
    F[v] = fx;
    F[n + v] = fy;
    F[2 * n + v] = fz;
}

int launch_scalars(MemCtx* c, const double* X, cudaStream_t s)
{
    const int nsplit = 3 * c->n > 2 * c->nplt ? 3 * c->n : 2 * c->nplt;
    k_mem_split<<<(nsplit + 255) / 256, 256, 0, s>>>(X, c->n, c->xh, c->xl, c->acc, 2 * c->nplt);
    int rc = check_launch("membrane: split positions");
    if (rc) return rc;
    const int nel = c->ne + c->nt + c->np;
    if (nel > 0) {
        k_mem_elements<<<(nel + 255) / 256, 256, 0, s>>>(*c);
        rc = check_launch("membrane: element scalars");
    }
    return rc;
}

}  // namespace

int launch_membrane_forces(MemCtx* c, const double* X, float* F, cudaStream_t s)
{
    int rc = launch_scalars(c, X, s);
    if (rc) return rc;
    k_mem_nodes<<<(c->n + 127) / 128, 128, 0, s>>>(F, *c);
    return check_launch("membrane_forces");
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
    const Layout L = make_layout(n_nodes, n_tri, (int)T.edge.size(), n_pairs, n_plt, T.spr.size(),
                                 T.trl.size(), T.dih.size(), 2 * (size_t)n_pairs);
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
    const Layout L = make_layout(n, nt, ne, np, nplt, T.spr.size(), T.trl.size(), T.dih.size(), T.mor.size());
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
    if (!rc) rc = up(S_SPR_OFF, T.spr_off.data(), sizeof(int) * (n + 1));
    if (!rc) rc = up(S_SPR, T.spr.data(), sizeof(int2) * T.spr.size());
    if (!rc) rc = up(S_TRI_OFF, T.tri_off.data(), sizeof(int) * (n + 1));
    if (!rc) rc = up(S_TRL, T.trl.data(), sizeof(int4) * T.trl.size());
    if (!rc) rc = up(S_DIH_OFF, T.dih_off.data(), sizeof(int) * (n + 1));
    if (!rc) rc = up(S_DIH, T.dih.data(), sizeof(int) * T.dih.size());
    if (!rc) rc = up(S_MOR_OFF, T.mor_off.data(), sizeof(int) * (n + 1));
    if (!rc) rc = up(S_MOR, T.mor.data(), sizeof(int2) * T.mor.size());
    if (!rc) rc = up(S_NODE_PLT, node_plt, sizeof(int) * n);
    if (!rc) rc = up(S_IS_MEM, mem_v.data(), n);
    if (!rc) rc = up(S_PLT_REST, plt_rest.data(), sizeof(double) * plt_rest.size());
    if (!rc) rc = up(S_PLT_ANCHOR, anchor.data(), sizeof(int) * nplt);
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
    c->spr_off = reinterpret_cast<const int*>(at(S_SPR_OFF));
    c->spr = reinterpret_cast<const int2*>(at(S_SPR));
    c->tri_off = reinterpret_cast<const int*>(at(S_TRI_OFF));
    c->trl = reinterpret_cast<const int4*>(at(S_TRL));
    c->dih_off = reinterpret_cast<const int*>(at(S_DIH_OFF));
    c->dih = reinterpret_cast<const int*>(at(S_DIH));
    c->mor_off = reinterpret_cast<const int*>(at(S_MOR_OFF));
    c->mor = reinterpret_cast<const int2*>(at(S_MOR));
    c->node_plt = reinterpret_cast<const int*>(at(S_NODE_PLT));
    c->is_mem = reinterpret_cast<const uint8_t*>(at(S_IS_MEM));
    c->plt_rest = reinterpret_cast<const double*>(at(S_PLT_REST));
    c->plt_anchor = reinterpret_cast<const int*>(at(S_PLT_ANCHOR));
    c->acc = reinterpret_cast<double*>(at(S_ACC));
    c->xh = reinterpret_cast<float*>(at(S_XH));
    c->xl = reinterpret_cast<float*>(at(S_XL));
    c->esc = reinterpret_cast<float2*>(at(S_ESC));
    c->tsc = reinterpret_cast<float*>(at(S_TSC));
    c->msc = reinterpret_cast<float*>(at(S_MSC));
    *out = c;
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
    if (!c || !X || !F) return set_error(PFSI_ERR_ARG, "membrane_forces: null argument");
    if (!aligned(X, 8) || !aligned(F, 4)) return set_error(PFSI_ERR_ARG, "membrane_forces: misaligned arrays");
    return launch_membrane_forces(c, X, F, as_stream(stream));
}

extern "C" int membrane_measure(mem_ctx* c, const double* X, double* out_host, void* stream)
{
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
