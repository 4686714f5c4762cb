// ib.cu -- immersed-boundary coupling (Section 3.4.2, Eq. 31-36) for sm_103a.
//
// Both kernels run one thread per Lagrangian node over the node's 4x4x4
// support of the cosine kernel phi(r) = (1 + cos(pi r / 2)) / 4 (Eq. 36,
// h = 1).  With r measured from the cell below-left of the node, the four
// offsets of each axis are -1 - t, -t, 1 - t, 2 - t (t in [0,1)), all inside
// |r| <= 2, so the weights need no branch.  The support wraps in x and y and
// is cut at the walls (cells with k outside [0, nz) are skipped) so that
// spreading and interpolation stay adjoint.
//
// Spreading adds F_m * w into the float4 force field with one vector
// reduction per support cell (red.global.add.v4.f32) and marks the rows
// (j, k) it touched; interpolation gathers the float4 velocity written by
// the lattice step in exactly those rows and clears their marks.
#include "pfsi_internal.cuh"

namespace pfsi {

namespace {

__device__ __forceinline__ float phi4(float r) { return 0.25f * (1.0f + cospif(0.5f * r)); }

struct Support {
    int ix[4], jy[4], kz0;
    float wx[4], wy[4], wz[4];
};

__device__ __forceinline__ void support(double x, double y, double z, int nx, int ny, Support& s)
{
    const double fx = floor(x), fy = floor(y), fz = floor(z);
    const float tx = (float)(x - fx), ty = (float)(y - fy), tz = (float)(z - fz);
    int bx = (int)fx - 1, by = (int)fy - 1;
    s.kz0 = (int)fz - 1;
    bx %= nx;
    if (bx < 0) bx += nx;
    by %= ny;
    if (by < 0) by += ny;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        s.wx[a] = phi4((float)(a - 1) - tx);
        s.wy[a] = phi4((float)(a - 1) - ty);
        s.wz[a] = phi4((float)(a - 1) - tz);
        int ii = bx + a, jj = by + a;
        while (ii >= nx) ii -= nx;   // at most three passes (narrow grids)
        while (jj >= ny) jj -= ny;
        s.ix[a] = ii;
        s.jy[a] = jj;
    }
}

__global__ void __launch_bounds__(256) k_ib_spread(const double* __restrict__ X,
                                                   const float* __restrict__ F, int M,
                                                   float4* __restrict__ g,
                                                   uint32_t* __restrict__ flags, int nx, int ny,
                                                   int nz)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    Support s;
    support(X[m], X[M + m], X[2 * M + m], nx, ny, s);
    const float fx = F[m], fy = F[M + m], fz = F[2 * M + m];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int k = s.kz0 + c;
        if (k < 0 || k >= nz) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int row = k * ny + s.jy[b];
            flags[row] = 1u;
            const float wyz = s.wy[b] * s.wz[c];
            float4* base = g + (size_t)row * nx;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const float w = s.wx[a] * wyz;
                atomicAdd(base + s.ix[a], make_float4(fx * w, fy * w, fz * w, 0.0f));
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_ib_interp(double* __restrict__ X, float* __restrict__ U,
                                                   int M, const float4* __restrict__ v,
                                                   uint32_t* __restrict__ flags, int nx, int ny,
                                                   int nz, int advect)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const double x = X[m], y = X[M + m], z = X[2 * M + m];
    Support s;
    support(x, y, z, nx, ny, s);
    float ux = 0.f, uy = 0.f, uz = 0.f;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int k = s.kz0 + c;
        if (k < 0 || k >= nz) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int row = k * ny + s.jy[b];
            const float wyz = s.wy[b] * s.wz[c];
            const float4* base = v + (size_t)row * nx;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const float w = s.wx[a] * wyz;
                const float4 vv = base[s.ix[a]];
                ux += w * vv.x;
                uy += w * vv.y;
                uz += w * vv.z;
            }
            flags[row] = 0u;
        }
    }
    U[m] = ux;
    U[M + m] = uy;
    U[2 * M + m] = uz;
    if (advect) {
        X[m] = x + (double)ux;
        X[M + m] = y + (double)uy;
        X[2 * M + m] = z + (double)uz;
    }
}

inline int blocks_for(int n, int t) { return (n + t - 1) / t; }

}  // namespace

int launch_ib_spread(LbCtx* c, const double* X, const float* F, int M, cudaStream_t s)
{
    if (M == 0) return PFSI_OK;
    k_ib_spread<<<blocks_for(M, 256), 256, 0, s>>>(X, F, M, c->g, c->flags, c->p.nx, c->p.ny, c->p.nz);
    return check_launch("ib_spread");
}

int launch_ib_interp(LbCtx* c, double* X, float* U, int M, int advect, cudaStream_t s)
{
    if (M == 0) return PFSI_OK;
    k_ib_interp<<<blocks_for(M, 256), 256, 0, s>>>(X, U, M, c->v, c->flags, c->p.nx, c->p.ny, c->p.nz,
                                                   advect);
    return check_launch("ib_interp");
}

}  // namespace pfsi

using namespace pfsi;

extern "C" int ib_spread(lb_ctx* c, const double* X, const float* F, int M, void* stream)
{
    if (!c || M < 0 || (M > 0 && (!X || !F))) return set_error(PFSI_ERR_ARG, "ib_spread: bad argument");
    if (!aligned(X, 8) || !aligned(F, 4)) return set_error(PFSI_ERR_ARG, "ib_spread: misaligned arrays");
    return launch_ib_spread(c, X, F, M, as_stream(stream));
}

extern "C" int ib_interp(lb_ctx* c, double* X, float* U, int M, int advect, void* stream)
{
    if (!c || M < 0 || (M > 0 && (!X || !U))) return set_error(PFSI_ERR_ARG, "ib_interp: bad argument");
    if (!aligned(X, 8) || !aligned(U, 4)) return set_error(PFSI_ERR_ARG, "ib_interp: misaligned arrays");
    return launch_ib_interp(c, X, U, M, advect, as_stream(stream));
}
