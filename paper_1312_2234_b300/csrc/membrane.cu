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
// Design: a node-parallel gather (one thread per node walks its own lists of
// springs, triangles, dihedral roles and Morse partners), so every node's
// force is written once, without atomics, in a fixed order.  Positions are
// FP64 (they accumulate tiny displacements over many steps); each neighbour
// is taken relative to the node in FP64 and rounded once to FP32, after which
// all geometry is FP32.  The per-platelet totals S and V come first from a
// triangle-parallel reduction accumulated in FP64.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

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
struct Layout {
    size_t off[24];
    size_t total;
};
enum Slice {
    S_TRI, S_TRI_PLT, S_TRI_S0, S_EDGE, S_EDGE_L0, S_EDGE_CS0, S_PAIR_R0, S_SPR_OFF, S_SPR,
    S_TRI_OFF, S_TRL, S_DIH_OFF, S_DIH, S_MOR_OFF, S_MOR, S_NODE_PLT, S_IS_MEM, S_PLT_S0,
    S_PLT_V0, S_PLT_ANCHOR, S_ACC, S_COUNT
};

Layout make_layout(int n, int nt, int ne, int np, int nplt, size_t n_spr, size_t n_trl,
                   size_t n_dih, size_t n_mor)
{
    const size_t bytes[S_COUNT] = {
        sizeof(int) * 3 * (size_t)nt, sizeof(int) * (size_t)nt, sizeof(float) * (size_t)nt,
        sizeof(int4) * (size_t)ne, sizeof(float) * (size_t)ne, sizeof(float2) * (size_t)ne,
        sizeof(float) * (size_t)np, sizeof(int) * (size_t)(n + 1), sizeof(int2) * n_spr,
        sizeof(int) * (size_t)(n + 1), sizeof(int4) * n_trl, sizeof(int) * (size_t)(n + 1),
        sizeof(int) * n_dih, sizeof(int) * (size_t)(n + 1), sizeof(int2) * n_mor,
        sizeof(int) * (size_t)n, (size_t)n, sizeof(double) * (size_t)nplt,
        sizeof(double) * (size_t)nplt, sizeof(int) * (size_t)nplt, sizeof(double) * 2 * (size_t)nplt};
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

// ------------------------------------------------------------------ device helpers
__device__ __forceinline__ float3 rel(const double* __restrict__ X, int n, int v, double xi,
                                      double yi, double zi)
{
    return make_float3((float)(X[v] - xi), (float)(X[n + v] - yi), (float)(X[2 * n + v] - zi));
}
__device__ __forceinline__ float3 f3sub(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 f3cross(float3 a, float3 b)
{
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float f3dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// Per-platelet total area and volume, FP64 accumulation.  Triangles of one
// platelet are contiguous, so a warp is almost always uniform in platelet.
__global__ void __launch_bounds__(256) k_mem_reduce(const double* __restrict__ X, int n, int nt,
                                                    const int* __restrict__ tri,
                                                    const int* __restrict__ tri_plt,
                                                    const int* __restrict__ anchor,
                                                    double* __restrict__ acc)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double S = 0.0, V = 0.0;
    int p = -1;
    if (t < nt) {
        p = tri_plt[t];
        const int a = tri[3 * t], b = tri[3 * t + 1], c = tri[3 * t + 2], o = anchor[p];
        const double ox = X[o], oy = X[n + o], oz = X[2 * n + o];
        const float3 pa = rel(X, n, a, ox, oy, oz);
        const float3 pb = rel(X, n, b, ox, oy, oz);
        const float3 pc = rel(X, n, c, ox, oy, oz);
        const float3 nn = f3cross(f3sub(pb, pa), f3sub(pc, pa));
        S = 0.5 * (double)sqrtf(f3dot(nn, nn));
        V = (double)f3dot(pa, f3cross(pb, pc)) * (1.0 / 6.0);
    }
    const int p0 = __shfl_sync(0xffffffffu, p, 0);
    if (__all_sync(0xffffffffu, p == p0) && p0 >= 0) {
        for (int o = 16; o > 0; o >>= 1) {
            S += __shfl_down_sync(0xffffffffu, S, o);
            V += __shfl_down_sync(0xffffffffu, V, o);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&acc[2 * p0], S);
            atomicAdd(&acc[2 * p0 + 1], V);
        }
    } else if (p >= 0) {
        atomicAdd(&acc[2 * p], S);
        atomicAdd(&acc[2 * p + 1], V);
    }
}

__global__ void k_zero(double* __restrict__ a, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = 0.0;
}

__global__ void __launch_bounds__(128) k_mem_forces(const double* __restrict__ X, float* __restrict__ F,
                                                    MemCtx c)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= c.n) return;
    const int n = c.n;
    const double xi = X[v], yi = X[n + v], zi = X[2 * n + v];
    const mem_params P = c.p;
    float fx = 0.f, fy = 0.f, fz = 0.f;

    // Eq. 3 springs: F_i = k (|R| - L0) R/|R|, R = X_j - X_i
    for (int s = c.spr_off[v]; s < c.spr_off[v + 1]; ++s) {
        const int2 e = c.spr[s];
        const float3 R = rel(X, n, e.x, xi, yi, zi);
        const float r = sqrtf(f3dot(R, R));
        const float sc = P.k_spring * (r - c.edge_L0[e.y]) / r;
        fx += sc * R.x;
        fy += sc * R.y;
        fz += sc * R.z;
    }

    // Eq. 4-5 area and volume: dS_t/dX_i = (1/2) nhat x (X_b - X_a) for the
    // outward triangle (i, a, b); dV/dX_i = (1/6) sum (X_a - X_i) x (X_b - X_i)
    // (the fan sum does not depend on the origin on a closed surface).
    const int plt = c.node_plt[v];
    const double Sp = c.acc[2 * plt], Vp = c.acc[2 * plt + 1];
    const float cSg = P.k_s != 0.f ? (float)((double)P.k_s * (Sp - c.plt_S0[plt]) / c.plt_S0[plt]) : 0.f;
    const float cV = P.k_v != 0.f ? (float)((double)P.k_v * (Vp - c.plt_V0[plt]) / c.plt_V0[plt]) : 0.f;
    for (int s = c.tri_off[v]; s < c.tri_off[v + 1]; ++s) {
        const int4 t = c.trl[s];
        const float3 e1 = rel(X, n, t.x, xi, yi, zi);
        const float3 e2 = rel(X, n, t.y, xi, yi, zi);
        const float3 nn = f3cross(e1, e2);
        const float len = sqrtf(f3dot(nn, nn));
        const float inv = 1.0f / len;
        const float3 nh = make_float3(nn.x * inv, nn.y * inv, nn.z * inv);
        const float3 gS = f3cross(nh, f3sub(e2, e1));  // 2 dS_t/dX_i
        const float S0 = c.tri_S0[t.z];
        const float cS = (P.k_t != 0.f ? P.k_t * (0.5f * len - S0) / S0 : 0.f) + cSg;
        fx -= 0.5f * cS * gS.x + cV * nn.x * (1.0f / 6.0f);
        fy -= 0.5f * cS * gS.y + cV * nn.y * (1.0f / 6.0f);
        fz -= 0.5f * cS * gS.z + cV * nn.z * (1.0f / 6.0f);
    }

    // bending: E = k_b (1 - cos(phi - phi0)), dE/dphi = k_b (sin phi cos phi0 -
    // cos phi sin phi0); torsion gradient of the chain r1-r2-r3-r4 = k-i-j-l
    // (Blondel and Karplus 1996).
    if (P.k_b != 0.f) {
        for (int s = c.dih_off[v]; s < c.dih_off[v + 1]; ++s) {
            const int code = c.dih[s];
            const int e = code >> 2, role = code & 3;
            const int4 q = c.edge[e];
            const float3 r1 = rel(X, n, q.z, xi, yi, zi);
            const float3 r2 = rel(X, n, q.x, xi, yi, zi);
            const float3 r3 = rel(X, n, q.y, xi, yi, zi);
            const float3 r4 = rel(X, n, q.w, xi, yi, zi);
            const float3 Fv = f3sub(r1, r2), G = f3sub(r2, r3), H = f3sub(r4, r3);
            const float3 A = f3cross(Fv, G), B = f3cross(H, G);
            const float A2 = f3dot(A, A), B2 = f3dot(B, B), gn = sqrtf(f3dot(G, G));
            const float iAB = rsqrtf(A2 * B2);
            const float cphi = f3dot(A, B) * iAB;
            const float sphi = f3dot(f3cross(B, A), G) * iAB / gn;
            const float2 cs0 = c.edge_cs0[e];
            const float dE = P.k_b * (sphi * cs0.x - cphi * cs0.y);
            float ca = 0.f, cb = 0.f;  // gradient = ca * A + cb * B
            if (role == 0) {
                ca = -gn / A2;
            } else if (role == 3) {
                cb = gn / B2;
            } else {
                const float FG = f3dot(Fv, G), HG = f3dot(H, G);
                if (role == 1) {
                    ca = gn / A2 + FG / (A2 * gn);
                    cb = -HG / (B2 * gn);
                } else {
                    ca = -FG / (A2 * gn);
                    cb = -gn / B2 + HG / (B2 * gn);
                }
            }
            fx -= dE * (ca * A.x + cb * B.x);
            fy -= dE * (ca * A.y + cb * B.y);
            fz -= dE * (ca * A.z + cb * B.z);
        }
    }

    // Morse pairs: F_i = 2 D a (1 - e^{-a d}) e^{-a d} R/|R|, d = |R| - r0
    if (P.morse_D != 0.f) {
        for (int s = c.mor_off[v]; s < c.mor_off[v + 1]; ++s) {
            const int2 pr = c.mor[s];
            const float3 R = rel(X, n, pr.x, xi, yi, zi);
            const float r = sqrtf(f3dot(R, R));
            const float ad = P.morse_a * (r - c.pair_r0[pr.y]);
            const float ex = expf(-ad);
            const float sc = 2.0f * P.morse_D * P.morse_a * (-expm1f(-ad)) * ex / r;
            fx += sc * R.x;
            fy += sc * R.y;
            fz += sc * R.z;
        }
    }

    // wall repulsion on surface nodes (Section 3.4.1)
    if (c.is_mem[v] && P.rep_F0 != 0.f) {
        const float eps = fmaxf((float)(zi - (double)P.z_wall), P.rep_eps_min);
        fz += P.rep_F0 * P.rep_tau / expm1f(P.rep_tau * eps);
    }
    F[v] = fx;
    F[n + v] = fy;
    F[2 * n + v] = fz;
}

int launch_reduce(MemCtx* c, const double* X, cudaStream_t s)
{
    k_zero<<<(2 * c->nplt + 127) / 128, 128, 0, s>>>(c->acc, 2 * c->nplt);
    int rc = check_launch("membrane: zero accumulators");
    if (rc) return rc;
    if (c->nt > 0) {
        k_mem_reduce<<<(c->nt + 255) / 256, 256, 0, s>>>(X, c->n, c->nt, c->tri, c->tri_plt,
                                                         c->plt_anchor, c->acc);
        rc = check_launch("membrane: area/volume reduction");
    }
    return rc;
}

}  // namespace

int launch_membrane_forces(MemCtx* c, const double* X, float* F, cudaStream_t s)
{
    int rc = launch_reduce(c, X, s);
    if (rc) return rc;
    if (c->n == 0) return PFSI_OK;
    k_mem_forces<<<(c->n + 127) / 128, 128, 0, s>>>(X, F, *c);
    return check_launch("membrane_forces");
}

}  // namespace pfsi

using namespace pfsi;

extern "C" int membrane_query_workspace(int n_nodes, int n_tri, const int* tri, int n_pairs, int n_plt,
                                        size_t* bytes)
{
    if (!bytes || n_nodes < 0 || n_tri < 0 || n_pairs < 0 || n_plt < 1 || (n_tri > 0 && !tri))
        return set_error(PFSI_ERR_ARG, "membrane_query_workspace: bad argument");
    // the pair list is not needed for the sizes (two entries per pair)
    std::vector<int> no_pairs;
    Topology T;
    std::string err;
    int rc = build_topology(n_nodes, n_tri, tri, 0, no_pairs.data(), T, err);
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

    auto pos = [&](int v, double* r) {
        r[0] = X0[v];
        r[1] = X0[n + v];
        r[2] = X0[2 * n + v];
    };
    // rest state in FP64 on the host
    std::vector<int> tri_plt(nt);
    std::vector<float> tri_S0(nt);
    for (int t = 0; t < nt; ++t) {
        double a[3], b[3], cc[3], e1[3], e2[3], nn[3];
        pos(tri[3 * t], a);
        pos(tri[3 * t + 1], b);
        pos(tri[3 * t + 2], cc);
        dsub(b, a, e1);
        dsub(cc, a, e2);
        dcross(e1, e2, nn);
        tri_S0[t] = (float)(0.5 * std::sqrt(ddot(nn, nn)));
        tri_plt[t] = node_plt[tri[3 * t]];
        if (!(tri_S0[t] > 0.f)) return set_error(PFSI_ERR_ARG, "membrane_create: zero-area rest triangle");
    }
    std::vector<float> L0(ne);
    std::vector<float2> cs0(ne);
    for (int e = 0; e < ne; ++e) {
        const int4 q = T.edge[e];
        double ri[3], rj[3], R[3];
        pos(q.x, ri);
        pos(q.y, rj);
        dsub(rj, ri, R);
        L0[e] = (float)std::sqrt(ddot(R, R));
        cs0[e] = make_float2(1.f, 0.f);
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
            const double nAB = std::sqrt(ddot(A, A) * ddot(B, B));
            const double cphi = ddot(A, B) / nAB;
            const double sphi = ddot(BxA, G) / (nAB * std::sqrt(ddot(G, G)));
            const double phi = std::atan2(sphi, cphi);
            cs0[e] = make_float2((float)std::cos(phi), (float)std::sin(phi));
        }
    }
    std::vector<float> r0(np);
    for (int s = 0; s < np; ++s) {
        double a[3], b[3], R[3];
        pos(pairs[2 * s], a);
        pos(pairs[2 * s + 1], b);
        dsub(b, a, R);
        r0[s] = (float)std::sqrt(ddot(R, R));
    }
    std::vector<int> anchor(nplt, -1);
    for (int v = 0; v < n; ++v)
        if (is_membrane[v] && anchor[node_plt[v]] < 0) anchor[node_plt[v]] = v;
    for (int q = 0; q < nplt; ++q)
        if (anchor[q] < 0) anchor[q] = 0;
    std::vector<double> S0(nplt, 0.0), V0(nplt, 0.0);
    for (int t = 0; t < nt; ++t) {
        const int q = tri_plt[t];
        double o[3], a[3], b[3], cc[3], bc[3];
        pos(anchor[q], o);
        pos(tri[3 * t], a);
        pos(tri[3 * t + 1], b);
        pos(tri[3 * t + 2], cc);
        dsub(a, o, a);
        dsub(b, o, b);
        dsub(cc, o, cc);
        dcross(b, cc, bc);
        S0[q] += tri_S0[t];
        V0[q] += ddot(a, bc) / 6.0;
    }
    for (int q = 0; q < nplt; ++q)
        if (p->k_s != 0.f && !(S0[q] > 0.0))
            return set_error(PFSI_ERR_ARG, "membrane_create: platelet without surface area");
    std::vector<int> nplt_v(node_plt, node_plt + n);
    std::vector<uint8_t> mem_v(is_membrane, is_membrane + n);

    char* base = static_cast<char*>(ws);
    auto up = [&](int slice, const void* src, size_t bytes) -> int {
        if (bytes == 0) return PFSI_OK;
        return check_cuda(cudaMemcpy(base + L.off[slice], src, bytes, cudaMemcpyHostToDevice),
                          "membrane_create: upload");
    };
    rc = up(S_TRI, tri, sizeof(int) * 3 * (size_t)nt);
    if (!rc) rc = up(S_TRI_PLT, tri_plt.data(), sizeof(int) * nt);
    if (!rc) rc = up(S_TRI_S0, tri_S0.data(), sizeof(float) * nt);
    if (!rc) rc = up(S_EDGE, T.edge.data(), sizeof(int4) * ne);
    if (!rc) rc = up(S_EDGE_L0, L0.data(), sizeof(float) * ne);
    if (!rc) rc = up(S_EDGE_CS0, cs0.data(), sizeof(float2) * ne);
    if (!rc) rc = up(S_PAIR_R0, r0.data(), sizeof(float) * np);
    if (!rc) rc = up(S_SPR_OFF, T.spr_off.data(), sizeof(int) * (n + 1));
    if (!rc) rc = up(S_SPR, T.spr.data(), sizeof(int2) * T.spr.size());
    if (!rc) rc = up(S_TRI_OFF, T.tri_off.data(), sizeof(int) * (n + 1));
    if (!rc) rc = up(S_TRL, T.trl.data(), sizeof(int4) * T.trl.size());
    if (!rc) rc = up(S_DIH_OFF, T.dih_off.data(), sizeof(int) * (n + 1));
    if (!rc) rc = up(S_DIH, T.dih.data(), sizeof(int) * T.dih.size());
    if (!rc) rc = up(S_MOR_OFF, T.mor_off.data(), sizeof(int) * (n + 1));
    if (!rc) rc = up(S_MOR, T.mor.data(), sizeof(int2) * T.mor.size());
    if (!rc) rc = up(S_NODE_PLT, nplt_v.data(), sizeof(int) * n);
    if (!rc) rc = up(S_IS_MEM, mem_v.data(), n);
    if (!rc) rc = up(S_PLT_S0, S0.data(), sizeof(double) * nplt);
    if (!rc) rc = up(S_PLT_V0, V0.data(), sizeof(double) * nplt);
    if (!rc) rc = up(S_PLT_ANCHOR, anchor.data(), sizeof(int) * nplt);
    if (rc) return rc;

    mem_ctx* c = new mem_ctx();
    c->p = *p;
    c->n = n;
    c->nt = nt;
    c->ne = ne;
    c->np = np;
    c->nplt = nplt;
    c->tri = reinterpret_cast<const int*>(base + L.off[S_TRI]);
    c->tri_plt = reinterpret_cast<const int*>(base + L.off[S_TRI_PLT]);
    c->tri_S0 = reinterpret_cast<const float*>(base + L.off[S_TRI_S0]);
    c->edge = reinterpret_cast<const int4*>(base + L.off[S_EDGE]);
    c->edge_L0 = reinterpret_cast<const float*>(base + L.off[S_EDGE_L0]);
    c->edge_cs0 = reinterpret_cast<const float2*>(base + L.off[S_EDGE_CS0]);
    c->pair_r0 = reinterpret_cast<const float*>(base + L.off[S_PAIR_R0]);
    c->spr_off = reinterpret_cast<const int*>(base + L.off[S_SPR_OFF]);
    c->spr = reinterpret_cast<const int2*>(base + L.off[S_SPR]);
    c->tri_off = reinterpret_cast<const int*>(base + L.off[S_TRI_OFF]);
    c->trl = reinterpret_cast<const int4*>(base + L.off[S_TRL]);
    c->dih_off = reinterpret_cast<const int*>(base + L.off[S_DIH_OFF]);
    c->dih = reinterpret_cast<const int*>(base + L.off[S_DIH]);
    c->mor_off = reinterpret_cast<const int*>(base + L.off[S_MOR_OFF]);
    c->mor = reinterpret_cast<const int2*>(base + L.off[S_MOR]);
    c->node_plt = reinterpret_cast<const int*>(base + L.off[S_NODE_PLT]);
    c->is_mem = reinterpret_cast<const uint8_t*>(base + L.off[S_IS_MEM]);
    c->plt_S0 = reinterpret_cast<const double*>(base + L.off[S_PLT_S0]);
    c->plt_V0 = reinterpret_cast<const double*>(base + L.off[S_PLT_V0]);
    c->plt_anchor = reinterpret_cast<const int*>(base + L.off[S_PLT_ANCHOR]);
    c->acc = reinterpret_cast<double*>(base + L.off[S_ACC]);
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
    int rc = launch_reduce(c, X, s);
    if (rc) return rc;
    rc = check_cuda(cudaMemcpyAsync(out_host, c->acc, sizeof(double) * 2 * c->nplt, cudaMemcpyDeviceToHost, s),
                    "membrane_measure: copy");
    if (rc) return rc;
    return check_cuda(cudaStreamSynchronize(s), "membrane_measure: synchronise");
}
