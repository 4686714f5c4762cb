// fem.cu -- finite-element bending of the hybrid membrane (Section 3.1,
// Eq. 6-10): curvature from quadratic six-node triangles and the normal
// bending force that follows from the energy of Eq. 6.
//
// The surface is covered by six-node elements (corners at parametric
// (0,0), (1,0), (0,1), then the midpoints of edges 0-1, 1-2, 2-0); a nodal
// field is interpolated on an element with the quadratic basis of Eq. 7.
// One force evaluation is four element passes, each followed by a node pass
// that averages the element values over the elements sharing the node (a
// fixed-order gather through a node -> element-node list, no atomics):
//
//   pass 0  unit normal dX/dxi x dX/deta at every element node, and the
//           node's share (one third) of the flat sub-triangles touching it;
//           node: normals summed and normalised, areas summed;
//   pass 1  Eq. 9: kappa solves [dX/dxi; dX/deta; n] kappa =
//           [dn/dxi; dn/deta; 0] with n the nodal normals interpolated by
//           Eq. 7.  With c0 = (a_eta x n)/det, c1 = (n x a_xi)/det (the first
//           two columns of the inverse of the row matrix), kappa =
//           c0 (x) dn/dxi + c1 (x) dn/deta, so K = tr(kappa)/2 (Eq. 10) and
//           K_G = (c0.dn_xi)(c1.dn_eta) - (c0.dn_eta)(c1.dn_xi);
//           node: means of K and K_G;
//   pass 2  surface gradient of K: g = c0 dK/dxi + c1 dK/deta; node: mean;
//   pass 3  surface divergence of g: c0.dg/dxi + c1.dg/deta; node: mean
//           (= Lap_S K), then F_i = A_i (k0/2)(Lap_S K + 2K(K^2 - K_G)) n_i.
//
// Positions are FP64, read as hi/lo float pairs (x = hi + lo, as the
// membrane pass splits them; a split pass runs first when no split is
// given).  Every element works in coordinates relative to its first corner,
// (hi_k - hi_0) + (lo_k - lo_0) in FP32, which keeps the digits the absolute
// position would lose and uses no FP64 arithmetic (a scarce pipe on this
// part).
#include <cuda_runtime.h>

#include <vector>

#include "pfsi_internal.cuh"

namespace pfsi {

struct FemCtx {
    int n, ne;
    const int* off;     // [n+1] node -> element-node list
    const int* list;    // [6 ne] entries 6 e + j
    const int* elem;    // [6 ne]
    float4* slot;       // [6 ne] per element-node values of the current pass
    float4* nrm;        // [n] (unit normal, area)
    float4* curv;       // [n] (K, K_G, Lap_S K, -)
    float4* grad;       // [n] (surface gradient of K, -)
    float* xh;          // [3n] own split of the positions (standalone calls)
    float* xl;
};

namespace {

constexpr int kFemThreads = 256;

__device__ __forceinline__ float3 f3(float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b)
{
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// d/dxi and d/deta of the six quadratic basis functions of Eq. 7 at element
// node j (parametric (0,0), (1,0), (0,1), (1/2,0), (1/2,1/2), (0,1/2)).
__device__ __forceinline__ void basis_derivatives(int j, float dxi[6], float deta[6])
{
    const float xi = (j == 1 || j == 3 || j == 4) ? (j == 1 ? 1.0f : 0.5f) : 0.0f;
    const float eta = (j == 2 || j == 4 || j == 5) ? (j == 2 ? 1.0f : 0.5f) : 0.0f;
    const float z = 1.0f - xi - eta;
    dxi[0] = 1.0f - 4.0f * z;
    dxi[1] = 4.0f * xi - 1.0f;
    dxi[2] = 0.0f;
    dxi[3] = 4.0f * (z - xi);
    dxi[4] = 4.0f * eta;
    dxi[5] = -4.0f * eta;
    deta[0] = 1.0f - 4.0f * z;
    deta[1] = 0.0f;
    deta[2] = 4.0f * eta - 1.0f;
    deta[3] = -4.0f * xi;
    deta[4] = 4.0f * xi;
    deta[5] = 4.0f * (z - eta);
}

__device__ __forceinline__ float tri_area(float3 a, float3 b, float3 c)
{
    const float3 n = cross3(b - a, c - a);
    return 0.5f * sqrtf(dot3(n, n));
}

// Columns c0, c1 of the inverse of the row matrix [a_xi; a_eta; n].
__device__ __forceinline__ void tangential_inverse(float3 a_xi, float3 a_eta, float3 n, float3& c0, float3& c1)
{
    const float3 en = cross3(a_eta, n);
    const float inv = 1.0f / dot3(a_xi, en);
    c0 = inv * en;
    c1 = inv * cross3(n, a_xi);
}

// x = hi + lo, hi the FP32 rounding of x (one coordinate per thread).
__global__ void k_fem_split(int n, const double* __restrict__ X, float* __restrict__ xh, float* __restrict__ xl)
{
    pdl_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * n) return;
    const double x = X[i];
    const float h = (float)x;
    xh[i] = h;
    xl[i] = (float)(x - (double)h);
}

// One thread per element: loads its six nodes once and writes the values of
// all six element nodes (the loop over j is unrolled, so the basis
// derivatives at node j are constants).
template <int Pass>
__global__ void __launch_bounds__(kFemThreads)
    k_fem_elem(FemCtx c, const float* __restrict__ xh, const float* __restrict__ xl)
{
    pdl_wait();
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= c.ne) return;
    const int n = c.n;
    int idx[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) idx[k] = __ldg(c.elem + 6 * e + k);
    // positions relative to corner 0: (hi_k - hi_0) + (lo_k - lo_0)
    float3 d[6];
    {
        const int i0 = idx[0];
        const float h0x = __ldg(xh + i0), h0y = __ldg(xh + n + i0), h0z = __ldg(xh + 2 * n + i0);
        const float l0x = __ldg(xl + i0), l0y = __ldg(xl + n + i0), l0z = __ldg(xl + 2 * n + i0);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int i = idx[k];
            d[k] = make_float3((__ldg(xh + i) - h0x) + (__ldg(xl + i) - l0x),
                               (__ldg(xh + n + i) - h0y) + (__ldg(xl + n + i) - l0y),
                               (__ldg(xh + 2 * n + i) - h0z) + (__ldg(xl + 2 * n + i) - l0z));
        }
    }
    // nodal values of the previous node pass
    float3 nrm[6], val[6];
    float kv[6];
    if (Pass >= 1) {
#pragma unroll
        for (int k = 0; k < 6; ++k) nrm[k] = f3(c.nrm[idx[k]]);
    }
    if (Pass == 2) {
#pragma unroll
        for (int k = 0; k < 6; ++k) kv[k] = c.curv[idx[k]].x;
    }
    if (Pass == 3) {
#pragma unroll
        for (int k = 0; k < 6; ++k) val[k] = f3(c.grad[idx[k]]);
    }
    float area[4];
    if (Pass == 0) {
        // sub-triangles (0,3,5), (3,1,4), (5,4,2), (3,4,5)
        area[0] = tri_area(d[0], d[3], d[5]);
        area[1] = tri_area(d[3], d[1], d[4]);
        area[2] = tri_area(d[5], d[4], d[2]);
        area[3] = tri_area(d[3], d[4], d[5]);
    }
    float4* out = c.slot + 6 * (size_t)e;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        float dxi[6], deta[6];
        basis_derivatives(j, dxi, deta);
        float3 a_xi = make_float3(0.f, 0.f, 0.f), a_eta = a_xi;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            a_xi = a_xi + dxi[k] * d[k];
            a_eta = a_eta + deta[k] * d[k];
        }
        float4 o;
        if (Pass == 0) {
            float3 nv = cross3(a_xi, a_eta);
            nv = rsqrtf(dot3(nv, nv)) * nv;
            // corners touch one sub-triangle, midpoints three
            const float a = j == 0   ? area[0]
                            : j == 1 ? area[1]
                            : j == 2 ? area[2]
                            : j == 3 ? area[0] + area[1] + area[3]
                            : j == 4 ? area[1] + area[2] + area[3]
                                     : area[0] + area[2] + area[3];
            o = make_float4(nv.x, nv.y, nv.z, a * (1.0f / 3.0f));
        } else {
            float3 c0, c1;
            tangential_inverse(a_xi, a_eta, nrm[j], c0, c1);
            if (Pass == 1) {
                float3 dn_xi = make_float3(0.f, 0.f, 0.f), dn_eta = dn_xi;
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    dn_xi = dn_xi + dxi[k] * nrm[k];
                    dn_eta = dn_eta + deta[k] * nrm[k];
                }
                const float p = dot3(c0, dn_xi), q = dot3(c1, dn_eta);
                const float r = dot3(c0, dn_eta), s = dot3(c1, dn_xi);
                o = make_float4(0.5f * (p + q), p * q - r * s, 0.f, 0.f);
            } else if (Pass == 2) {
                float k_xi = 0.f, k_eta = 0.f;
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    k_xi += dxi[k] * kv[k];
                    k_eta += deta[k] * kv[k];
                }
                const float3 g = k_xi * c0 + k_eta * c1;
                o = make_float4(g.x, g.y, g.z, 0.f);
            } else {
                float3 g_xi = make_float3(0.f, 0.f, 0.f), g_eta = g_xi;
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    g_xi = g_xi + dxi[k] * val[k];
                    g_eta = g_eta + deta[k] * val[k];
                }
                o = make_float4(dot3(c0, g_xi) + dot3(c1, g_eta), 0.f, 0.f, 0.f);
            }
        }
        out[j] = o;
    }
}

// Node pass: fixed-order sum over the node's element nodes.  Pass 3 also
// writes the force (F [3][n], added if `accumulate`) and, if `fields` is
// non-null, the nodal fields [7][n]: n_x, n_y, n_z, A, K, K_G, Lap_S K.
template <int Pass>
__global__ void __launch_bounds__(kFemThreads)
    k_fem_node(FemCtx c, float k0, float* __restrict__ F, int accumulate, float* __restrict__ fields)
{
    pdl_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.n) return;
    const int b = __ldg(c.off + i), en = __ldg(c.off + i + 1);
    // a vertex lies in ~6 elements, an edge midpoint in 2: the first six list
    // entries, then their slots, are loaded together; sums in list order
    constexpr int kPre = 6;
    int li[kPre];
#pragma unroll
    for (int u = 0; u < kPre; ++u) li[u] = b + u < en ? __ldg(c.list + b + u) : -1;
    float4 pv[kPre];
#pragma unroll
    for (int u = 0; u < kPre; ++u) pv[u] = li[u] >= 0 ? c.slot[li[u]] : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int u = 0; u < kPre; ++u)
        if (li[u] >= 0) {
            s.x += pv[u].x;
            s.y += pv[u].y;
            s.z += pv[u].z;
            s.w += pv[u].w;
        }
    for (int k = b + kPre; k < en; ++k) {
        const float4 v = c.slot[__ldg(c.list + k)];
        s.x += v.x;
        s.y += v.y;
        s.z += v.z;
        s.w += v.w;
    }
    const int cnt = en - b;
    const float inv = cnt > 0 ? 1.0f / (float)cnt : 0.f;
    if (Pass == 0) {
        const float L2 = s.x * s.x + s.y * s.y + s.z * s.z;
        const float r = L2 > 0.f ? rsqrtf(L2) : 0.f;
        c.nrm[i] = make_float4(r * s.x, r * s.y, r * s.z, s.w);
    } else if (Pass == 1) {
        c.curv[i] = make_float4(inv * s.x, inv * s.y, 0.f, 0.f);
    } else if (Pass == 2) {
        c.grad[i] = make_float4(inv * s.x, inv * s.y, inv * s.z, 0.f);
    } else {
        const float lap = inv * s.x;
        const float4 kv = c.curv[i];
        const float4 nv = c.nrm[i];
        const float K = kv.x, KG = kv.y;
        const float m = cnt > 0 ? nv.w * 0.5f * k0 * (lap + 2.0f * K * (K * K - KG)) : 0.f;
        if (F) {
            const float fx = m * nv.x, fy = m * nv.y, fz = m * nv.z;
            if (accumulate) {
                F[i] += fx;
                F[c.n + i] += fy;
                F[2 * c.n + i] += fz;
            } else {
                F[i] = fx;
                F[c.n + i] = fy;
                F[2 * c.n + i] = fz;
            }
        }
        if (fields) {
            const size_t n = (size_t)c.n;
            fields[i] = nv.x;
            fields[n + i] = nv.y;
            fields[2 * n + i] = nv.z;
            fields[3 * n + i] = nv.w;
            fields[4 * n + i] = K;
            fields[5 * n + i] = KG;
            fields[6 * n + i] = lap;
        }
    }
}

struct FemLayout {
    size_t off, list, elem, slot, nrm, curv, grad, xh, xl, total;
};

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

FemLayout fem_layout(int n, int ne)
{
    FemLayout L;
    size_t o = 0;
    L.off = o;
    o += up256(4 * (size_t)(n + 1));
    L.list = o;
    o += up256(4 * 6 * (size_t)ne);
    L.elem = o;
    o += up256(4 * 6 * (size_t)ne);
    L.slot = o;
    o += up256(16 * 6 * (size_t)ne);
    L.nrm = o;
    o += up256(16 * (size_t)n);
    L.curv = o;
    o += up256(16 * (size_t)n);
    L.grad = o;
    o += up256(16 * (size_t)n);
    L.xh = o;
    o += up256(12 * (size_t)n);
    L.xl = o;
    o += up256(12 * (size_t)n);
    L.total = o;
    return L;
}

}  // namespace

int launch_fem_forces(FemCtx* c, float k0, const double* X, const float* xh, const float* xl, float* F,
                      int accumulate, float* fields, cudaStream_t s)
{
    const int ge = (c->ne + kFemThreads - 1) / kFemThreads;
    const int gn = (c->n + kFemThreads - 1) / kFemThreads;
    const FemCtx v = *c;
    int rc = PFSI_OK;
    if (!xh || !xl) {
        rc = check_cuda(launch_pdl(k_fem_split, dim3((3 * c->n + kFemThreads - 1) / kFemThreads), dim3(kFemThreads), 0, s,
                                   c->n, X, c->xh, c->xl),
                        "fem bending: split");
        xh = c->xh;
        xl = c->xl;
    }
    if (!rc) rc = check_cuda(launch_pdl(k_fem_elem<0>, dim3(ge), dim3(kFemThreads), 0, s, v, xh, xl), "fem bending");
    if (!rc)
        rc = check_cuda(launch_pdl(k_fem_node<0>, dim3(gn), dim3(kFemThreads), 0, s, v, k0, (float*)nullptr, 0,
                                   (float*)nullptr),
                        "fem bending");
    if (!rc) rc = check_cuda(launch_pdl(k_fem_elem<1>, dim3(ge), dim3(kFemThreads), 0, s, v, xh, xl), "fem bending");
    if (!rc)
        rc = check_cuda(launch_pdl(k_fem_node<1>, dim3(gn), dim3(kFemThreads), 0, s, v, k0, (float*)nullptr, 0,
                                   (float*)nullptr),
                        "fem bending");
    if (!rc) rc = check_cuda(launch_pdl(k_fem_elem<2>, dim3(ge), dim3(kFemThreads), 0, s, v, xh, xl), "fem bending");
    if (!rc)
        rc = check_cuda(launch_pdl(k_fem_node<2>, dim3(gn), dim3(kFemThreads), 0, s, v, k0, (float*)nullptr, 0,
                                   (float*)nullptr),
                        "fem bending");
    if (!rc) rc = check_cuda(launch_pdl(k_fem_elem<3>, dim3(ge), dim3(kFemThreads), 0, s, v, xh, xl), "fem bending");
    if (!rc)
        rc = check_cuda(launch_pdl(k_fem_node<3>, dim3(gn), dim3(kFemThreads), 0, s, v, k0, F, accumulate, fields),
                        "fem bending");
    if (rc) return rc;
    return check_launch("fem bending");
}

}  // namespace pfsi

using namespace pfsi;

struct fem_ctx {
    FemCtx d;
    void* ws;
};

namespace pfsi {
FemCtx* fem_internal(fem_ctx* c) { return c ? &c->d : nullptr; }
int fem_node_count(const FemCtx* c) { return c->n; }
}

extern "C" int fem_query_workspace(int n_nodes, int n_elem, size_t* bytes)
{
    if (!bytes || n_nodes < 1 || n_elem < 1) return set_error(PFSI_ERR_ARG, "fem_query_workspace: bad argument");
    *bytes = fem_layout(n_nodes, n_elem).total;
    return PFSI_OK;
}

extern "C" int fem_create(int n_nodes, int n_elem, const int* elem6, void* ws, size_t ws_bytes, fem_ctx** out)
{
    if (!out || n_nodes < 1 || n_elem < 1 || !elem6 || !ws) return set_error(PFSI_ERR_ARG, "fem_create: bad argument");
    if (!aligned(ws, 256)) return set_error(PFSI_ERR_ARG, "fem_create: workspace must be 256-byte aligned");
    const FemLayout L = fem_layout(n_nodes, n_elem);
    if (ws_bytes < L.total) return set_error(PFSI_ERR_ARG, "fem_create: workspace too small");
    std::vector<int> off(n_nodes + 1, 0), list(6 * (size_t)n_elem);
    for (int e = 0; e < n_elem; ++e) {
        for (int j = 0; j < 6; ++j) {
            const int i = elem6[6 * e + j];
            if (i < 0 || i >= n_nodes) return set_error(PFSI_ERR_ARG, "fem_create: node index out of range");
            for (int k = 0; k < j; ++k)
                if (elem6[6 * e + k] == i) return set_error(PFSI_ERR_ARG, "fem_create: repeated node in an element");
            off[i + 1] += 1;
        }
    }
    for (int i = 0; i < n_nodes; ++i) off[i + 1] += off[i];
    std::vector<int> fill(off.begin(), off.end() - 1);
    for (int t = 0; t < 6 * n_elem; ++t) list[fill[elem6[t]]++] = t;   // ascending element-node order per node
    char* b = (char*)ws;
    int rc = check_cuda(cudaMemset(ws, 0, L.total), "fem_create: clear");
    if (!rc) rc = check_cuda(cudaMemcpy(b + L.off, off.data(), 4 * off.size(), cudaMemcpyHostToDevice), "fem_create");
    if (!rc) rc = check_cuda(cudaMemcpy(b + L.list, list.data(), 4 * list.size(), cudaMemcpyHostToDevice), "fem_create");
    if (!rc) rc = check_cuda(cudaMemcpy(b + L.elem, elem6, 4 * 6 * (size_t)n_elem, cudaMemcpyHostToDevice), "fem_create");
    if (rc) return rc;
    fem_ctx* c = new fem_ctx();
    c->d = FemCtx{n_nodes, n_elem, (const int*)(b + L.off), (const int*)(b + L.list), (const int*)(b + L.elem),
                  (float4*)(b + L.slot), (float4*)(b + L.nrm), (float4*)(b + L.curv), (float4*)(b + L.grad),
                  (float*)(b + L.xh), (float*)(b + L.xl)};
    c->ws = ws;
    *out = c;
    return PFSI_OK;
}

extern "C" int fem_destroy(fem_ctx* c)
{
    delete c;
    return PFSI_OK;
}

extern "C" int fem_bending_forces(fem_ctx* c, float k0, const double* X, float* F, int accumulate, void* stream)
{
    NvtxRange nvtx_range("fem_bending_forces");
    if (!c || !X || !F) return set_error(PFSI_ERR_ARG, "fem_bending_forces: bad argument");
    if (!aligned(X, 8) || !aligned(F, 4)) return set_error(PFSI_ERR_ARG, "fem_bending_forces: misaligned buffer");
    return launch_fem_forces(&c->d, k0, X, nullptr, nullptr, F, accumulate ? 1 : 0, nullptr, as_stream(stream));
}

extern "C" int fem_fields(fem_ctx* c, const double* X, float* fields, void* stream)
{
    NvtxRange nvtx_range("fem_fields");
    if (!c || !X || !fields) return set_error(PFSI_ERR_ARG, "fem_fields: bad argument");
    if (!aligned(X, 8) || !aligned(fields, 4)) return set_error(PFSI_ERR_ARG, "fem_fields: misaligned buffer");
    return launch_fem_forces(&c->d, 0.0f, X, nullptr, nullptr, nullptr, 0, fields, as_stream(stream));
}
