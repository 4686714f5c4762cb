// ib.cu -- immersed-boundary coupling (Section 3.4.2, Eq. 31-36) for sm_103a.
//
// Kernel: phi(r) = (1 + cos(pi r / 2)) / 4 (Eq. 36, h = 1).  With r measured
// from the cell below-left of the node, the four offsets of each axis are
// -1 - t, -t, 1 - t, 2 - t (t in [0,1)), all inside |r| <= 2, so the weights
// need no branch.  The support wraps in x and y and is cut at the walls
// (cells with k outside [0, nz) are skipped), so spreading and interpolation
// stay adjoint.
//
// Blocking: a block takes a chunk of 256 consecutive nodes (consecutive nodes
// of a platelet mesh lie close together) and the bounding box of their 4x4x4
// supports.  When the box fits the shared-memory tile (4096 cells):
//   spreading  accumulates the chunk's F_m * w in the tile with shared
//              atomics, then adds each nonzero tile cell to the float4 force
//              field with one vector reduction (red.global.add.v4.f32): ~10
//              global reductions per node instead of 64;
//   interp     loads the velocity of the box into the tile once and gathers
//              every node's 64 weights from shared memory.
// Otherwise the block falls back to per-node global reductions / gathers.
// Both kernels take the same decision for the same positions, and flag /
// clear the same rows: every row of the box (a superset of the support rows),
// so the lattice step writes the velocity wherever interpolation will read.
#include <climits>

#include "pfsi_internal.cuh"

namespace pfsi {

namespace {

constexpr int kChunk = 256;
constexpr int kTileCells = 4096;
constexpr size_t kTileBytes = kTileCells * sizeof(float4);

__device__ __forceinline__ float phi4(float r) { return 0.25f * (1.0f + cospif(0.5f * r)); }

__device__ __forceinline__ int wrap(int i, int n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

struct Node {
    int bx, by, bz;              // unwrapped cell of support offset 0 on each axis
    float wx[4], wy[4], wz[4];
};

__device__ __forceinline__ void node_support(double x, double y, double z, Node& s)
{
    const double fx = floor(x), fy = floor(y), fz = floor(z);
    const float tx = (float)(x - fx), ty = (float)(y - fy), tz = (float)(z - fz);
    s.bx = (int)fx - 1;
    s.by = (int)fy - 1;
    s.bz = (int)fz - 1;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        s.wx[a] = phi4((float)(a - 1) - tx);
        s.wy[a] = phi4((float)(a - 1) - ty);
        s.wz[a] = phi4((float)(a - 1) - tz);
    }
}

struct Box {
    int x0, y0, z0;   // unwrapped origin; z0 clipped to the walls
    int ex, ey, ez;   // extents (ez after clipping, may be <= 0)
    bool tiled;
};

// Bounding box of the supports of the block's active nodes.
__device__ Box block_box(const Node& s, bool active, int nz)
{
    __shared__ int red[6][kChunk / 32];
    __shared__ Box box;
    int v[6] = {active ? s.bx : INT_MAX, active ? s.by : INT_MAX, active ? s.bz : INT_MAX,
                active ? s.bx : INT_MIN, active ? s.by : INT_MIN, active ? s.bz : INT_MIN};
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        v[k] = __reduce_min_sync(0xffffffffu, v[k]);
        v[k + 3] = __reduce_max_sync(0xffffffffu, v[k + 3]);
    }
    if (lane == 0)
        for (int k = 0; k < 6; ++k) red[k][warp] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        int r[6] = {INT_MAX, INT_MAX, INT_MAX, INT_MIN, INT_MIN, INT_MIN};
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            for (int k = 0; k < 3; ++k) r[k] = min(r[k], red[k][w]);
            for (int k = 3; k < 6; ++k) r[k] = max(r[k], red[k][w]);
        }
        Box b;
        b.x0 = r[0];
        b.y0 = r[1];
        const int z0 = max(r[2], 0), z1 = min(r[5] + 3, nz - 1);
        b.z0 = z0;
        b.ex = r[3] + 4 - r[0];
        b.ey = r[4] + 4 - r[1];
        b.ez = z1 - z0 + 1;
        b.tiled = b.ez > 0 && (long long)b.ex * b.ey * b.ez <= kTileCells;
        box = b;
    }
    __syncthreads();
    return box;
}

__global__ void __launch_bounds__(kChunk) k_ib_spread(const double* __restrict__ X, const float* __restrict__ F,
                                                      int M, float4* __restrict__ g,
                                                      uint32_t* __restrict__ flags, int nx, int ny, int nz)
{
    extern __shared__ float4 tile[];
    const int m = blockIdx.x * kChunk + threadIdx.x;
    const bool active = m < M;
    Node s;
    float fx = 0.f, fy = 0.f, fz = 0.f;
    if (active) {
        node_support(X[m], X[M + m], X[2 * M + m], s);
        fx = F[m];
        fy = F[M + m];
        fz = F[2 * M + m];
    }
    const Box b = block_box(s, active, nz);
    if (b.tiled) {
        const int cells = b.ex * b.ey * b.ez;
        for (int i = threadIdx.x; i < cells; i += kChunk) tile[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();
        if (active) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int k = s.bz + c - b.z0;
                if (k < 0 || k >= b.ez) continue;
#pragma unroll
                for (int bb = 0; bb < 4; ++bb) {
                    const float wyz = s.wy[bb] * s.wz[c];
                    float* row = reinterpret_cast<float*>(tile + ((size_t)k * b.ey + (s.by + bb - b.y0)) * b.ex +
                                                          (s.bx - b.x0));
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        const float w = s.wx[a] * wyz;
                        atomicAdd(row + 4 * a + 0, fx * w);
                        atomicAdd(row + 4 * a + 1, fy * w);
                        atomicAdd(row + 4 * a + 2, fz * w);
                    }
                }
            }
        }
        __syncthreads();
        const int x0 = wrap(b.x0, nx), y0 = wrap(b.y0, ny);
        for (int i = threadIdx.x; i < cells; i += kChunk) {
            const float4 val = tile[i];
            const int a = i % b.ex, rest = i / b.ex, bb = rest % b.ey, c = rest / b.ey;
            if (a == 0) flags[(b.z0 + c) * ny + wrap(y0 + bb, ny)] = 1u;
            if (val.x != 0.f || val.y != 0.f || val.z != 0.f) {
                const int gi = wrap(x0 + a, nx), gj = wrap(y0 + bb, ny);
                atomicAdd(g + ((size_t)(b.z0 + c) * ny + gj) * nx + gi, val);
            }
        }
        return;
    }
    if (!active) return;
    // fallback: per-node global reductions
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int k = s.bz + c;
        if (k < 0 || k >= nz) continue;
#pragma unroll
        for (int bb = 0; bb < 4; ++bb) {
            const int row = k * ny + wrap(s.by + bb, ny);
            flags[row] = 1u;
            const float wyz = s.wy[bb] * s.wz[c];
            float4* base = g + (size_t)row * nx;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const float w = s.wx[a] * wyz;
                atomicAdd(base + wrap(s.bx + a, nx), make_float4(fx * w, fy * w, fz * w, 0.0f));
            }
        }
    }
}

__global__ void __launch_bounds__(kChunk) k_ib_interp(double* __restrict__ X, float* __restrict__ U, int M,
                                                      const float4* __restrict__ v,
                                                      uint32_t* __restrict__ flags, int nx, int ny, int nz,
                                                      int advect)
{
    extern __shared__ float4 tile[];
    const int m = blockIdx.x * kChunk + threadIdx.x;
    const bool active = m < M;
    Node s;
    double x = 0.0, y = 0.0, z = 0.0;
    if (active) {
        x = X[m];
        y = X[M + m];
        z = X[2 * M + m];
        node_support(x, y, z, s);
    }
    const Box b = block_box(s, active, nz);
    float ux = 0.f, uy = 0.f, uz = 0.f;
    if (b.tiled) {
        const int cells = b.ex * b.ey * b.ez;
        const int x0 = wrap(b.x0, nx), y0 = wrap(b.y0, ny);
        for (int i = threadIdx.x; i < cells; i += kChunk) {
            const int a = i % b.ex, rest = i / b.ex, bb = rest % b.ey, c = rest / b.ey;
            const int row = (b.z0 + c) * ny + wrap(y0 + bb, ny);
            tile[i] = v[(size_t)row * nx + wrap(x0 + a, nx)];
        }
        __syncthreads();
        for (int i = threadIdx.x; i < b.ey * b.ez; i += kChunk)
            flags[(b.z0 + i / b.ey) * ny + wrap(y0 + i % b.ey, ny)] = 0u;
        if (!active) return;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int k = s.bz + c - b.z0;
            if (k < 0 || k >= b.ez) continue;
#pragma unroll
            for (int bb = 0; bb < 4; ++bb) {
                const float wyz = s.wy[bb] * s.wz[c];
                const float4* row = tile + ((size_t)k * b.ey + (s.by + bb - b.y0)) * b.ex + (s.bx - b.x0);
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const float w = s.wx[a] * wyz;
                    const float4 vv = row[a];
                    ux += w * vv.x;
                    uy += w * vv.y;
                    uz += w * vv.z;
                }
            }
        }
    } else {
        if (!active) return;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int k = s.bz + c;
            if (k < 0 || k >= nz) continue;
#pragma unroll
            for (int bb = 0; bb < 4; ++bb) {
                const int row = k * ny + wrap(s.by + bb, ny);
                const float wyz = s.wy[bb] * s.wz[c];
                const float4* base = v + (size_t)row * nx;
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const float w = s.wx[a] * wyz;
                    const float4 vv = base[wrap(s.bx + a, nx)];
                    ux += w * vv.x;
                    uy += w * vv.y;
                    uz += w * vv.z;
                }
                flags[row] = 0u;
            }
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

}  // namespace

int ib_prepare()
{
    int rc = check_cuda(cudaFuncSetAttribute(k_ib_spread, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileBytes),
                        "ib: shared memory size");
    if (!rc)
        rc = check_cuda(cudaFuncSetAttribute(k_ib_interp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileBytes),
                        "ib: shared memory size");
    return rc;
}

int launch_ib_spread(LbCtx* c, const double* X, const float* F, int M, cudaStream_t s)
{
    if (M == 0) return PFSI_OK;
    k_ib_spread<<<(M + kChunk - 1) / kChunk, kChunk, kTileBytes, s>>>(X, F, M, c->g, c->flags, c->p.nx, c->p.ny,
                                                                       c->p.nz);
    return check_launch("ib_spread");
}

int launch_ib_interp(LbCtx* c, double* X, float* U, int M, int advect, cudaStream_t s)
{
    if (M == 0) return PFSI_OK;
    k_ib_interp<<<(M + kChunk - 1) / kChunk, kChunk, kTileBytes, s>>>(X, U, M, c->v, c->flags, c->p.nx, c->p.ny,
                                                                       c->p.nz, advect);
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
