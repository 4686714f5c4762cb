// ib.cu -- immersed-boundary coupling (Section 3.4.2, Eq. 31-36) for sm_103a.
//
// Kernel: phi(r) = (1 + cos(pi r / 2)) / 4 (Eq. 36, h = 1).  With r measured
// from the cell below-left of the node, the four offsets of each axis are
// -1 - t, -t, 1 - t, 2 - t (t in [0,1)), all inside |r| <= 2, so the weights
// need no branch.  The support wraps in x and y and is cut at the walls
// (cells with k outside [0, nz) are skipped), so spreading and interpolation
// stay adjoint.
//
// Blocking: a block of 512 threads takes a chunk of up to 256 consecutive
// nodes (consecutive nodes of a platelet mesh lie close together; the coupled
// step passes chunks that never straddle two platelets, the public calls use
// fixed chunks of 256).  Each thread of
// the first half stages one node (support origin, weights, force); then each
// warp walks its share of the chunk one node at a time with lane l on support
// cell (a, b, c) = (l & 3, (l >> 2) & 3, (l >> 4) + {0, 2}), so one
// instruction touches 32 distinct cells.  When the bounding box of the
// chunk's supports fits the shared tile (three float planes of 4096 cells):
//   spreading  accumulates in the tile with shared atomics, then adds every
//              nonzero tile cell to the float4 force field with one vector
//              reduction (red.global.add.v4.f32): ~4 global reductions per
//              node of a platelet instead of 64;
//   interp     loads the box's velocity into the tile once; each node's 64
//              weighted values are summed across the warp with shuffles and
//              the staging threads write U (and advance X) afterwards.
// Otherwise (e.g. a chunk that straddles two platelets) the block works on the
// global arrays directly, with the same lane-per-cell mapping.  Both kernels
// take the same decision for the same positions and flag / clear the same
// rows: every row of the box (a superset of the support rows), so the lattice
// step writes the velocity wherever interpolation will read it.
#include <climits>

#include "pfsi_internal.cuh"

namespace pfsi {

namespace {

constexpr int kChunk = 256;                 // nodes per block
constexpr int kThreads = 512;               // threads per block
constexpr int kWarps = kThreads / 32;
constexpr int kTileFloats = 3 * 4096;       // three planes of up to 4096 cells
constexpr size_t kTileBytes = kTileFloats * sizeof(float);

__device__ __forceinline__ float phi4(float r) { return 0.25f * (1.0f + cospif(0.5f * r)); }

__device__ __forceinline__ int wrap(int i, int n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

struct Stage {
    int bx[kChunk], by[kChunk], bz[kChunk];
    float w[12][kChunk];  // wx[0..3], wy[0..3], wz[0..3]
    float f[3][kChunk];
};

__device__ __forceinline__ void stage_node(Stage& st, int j, double x, double y, double z)
{
    const double fx = floor(x), fy = floor(y), fz = floor(z);
    const float tx = (float)(x - fx), ty = (float)(y - fy), tz = (float)(z - fz);
    st.bx[j] = (int)fx - 1;
    st.by[j] = (int)fy - 1;
    st.bz[j] = (int)fz - 1;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        st.w[a][j] = phi4((float)(a - 1) - tx);
        st.w[4 + a][j] = phi4((float)(a - 1) - ty);
        st.w[8 + a][j] = phi4((float)(a - 1) - tz);
    }
}

struct Box {
    int x0, y0, z0;    // unwrapped origin; z0 clipped to the walls
    int ex, ey, ez;    // extents (ez after clipping, may be <= 0)
    int sx, sy;        // x stride and y extent of the tile
    bool tiled;
};

// Bounding box of the staged supports (nodes [0, nodes)); also a barrier for
// the staging writes.
__device__ Box block_box(const Stage& st, int nodes, int nz)
{
    __shared__ int red[6][kWarps];
    __shared__ Box box;
    const int j = threadIdx.x;
    const bool on = j < nodes;
    int v[6] = {on ? st.bx[j] : INT_MAX, on ? st.by[j] : INT_MAX, on ? st.bz[j] : INT_MAX,
                on ? st.bx[j] : INT_MIN, on ? st.by[j] : INT_MIN, on ? st.bz[j] : INT_MIN};
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
        for (int w = 0; w < kWarps; ++w) {
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
        b.sx = b.ex;
        b.sy = b.ey;
        b.tiled = b.ez > 0 && b.ex <= 4096 && b.ey <= 4096 && (long long)b.ex * b.ey * b.ez * 3 <= kTileFloats;
        box = b;
    }
    __syncthreads();
    return box;
}

// chunk of the block: from the table (start, count) or the fixed 256-node split
__device__ __forceinline__ int2 block_chunk(const int2* __restrict__ chunks, int M)
{
    if (chunks) return chunks[blockIdx.x];
    const int m0 = blockIdx.x * kChunk;
    return make_int2(m0, min(kChunk, M - m0));
}

__global__ void __launch_bounds__(kThreads) k_ib_spread(const double* __restrict__ X, const float* __restrict__ F,
                                                        int M, const int2* __restrict__ chunks,
                                                        float4* __restrict__ g, uint32_t* __restrict__ flags,
                                                        int nx, int ny, int nz)
{
    extern __shared__ float tile[];
    __shared__ Stage st;
    const int2 ch = block_chunk(chunks, M);
    const int m0 = ch.x, nodes = ch.y;
    if (threadIdx.x < nodes) {
        const int m = m0 + threadIdx.x;
        stage_node(st, threadIdx.x, X[m], X[M + m], X[2 * M + m]);
        st.f[0][threadIdx.x] = F[m];
        st.f[1][threadIdx.x] = F[M + m];
        st.f[2][threadIdx.x] = F[2 * M + m];
    }
    const Box b = block_box(st, nodes, nz);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int la = lane & 3, lb = (lane >> 2) & 3, lc = lane >> 4;
    const int plane = b.sx * b.sy * b.ez;
    if (b.tiled) {
        for (int i = threadIdx.x; i < 3 * plane; i += kThreads) tile[i] = 0.f;
        __syncthreads();
    }
    for (int j = warp; j < nodes; j += kWarps) {
        const float fx = st.f[0][j], fy = st.f[1][j], fz = st.f[2][j];
        const float wxy = st.w[la][j] * st.w[4 + lb][j];
        const int bx = st.bx[j], by = st.by[j], bz = st.bz[j];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = lc + 2 * h;
            const float w = wxy * st.w[8 + c][j];
            if (b.tiled) {
                const int k = bz + c - b.z0;
                if (k < 0 || k >= b.ez) continue;
                const int i = (k * b.sy + (by + lb - b.y0)) * b.sx + (bx + la - b.x0);
                atomicAdd(tile + i, fx * w);
                atomicAdd(tile + plane + i, fy * w);
                atomicAdd(tile + 2 * plane + i, fz * w);
            } else {
                const int k = bz + c;
                if (k < 0 || k >= nz) continue;
                const int row = k * ny + wrap(by + lb, ny);
                if (la == 0) flags[row] = 1u;
                atomicAdd(g + (size_t)row * nx + wrap(bx + la, nx), make_float4(fx * w, fy * w, fz * w, 0.0f));
            }
        }
    }
    if (!b.tiled) return;
    __syncthreads();
    // flush: one warp per tile row
    const int x0 = wrap(b.x0, nx), y0 = wrap(b.y0, ny);
    for (int r = warp; r < b.ey * b.ez; r += kWarps) {
        const int bb = r % b.ey, c = r / b.ey;
        const int grow = (b.z0 + c) * ny + wrap(y0 + bb, ny);
        if (lane == 0) flags[grow] = 1u;
        const int base = (c * b.sy + bb) * b.sx;
        for (int a = lane; a < b.ex; a += 32) {
            const float4 val = make_float4(tile[base + a], tile[plane + base + a], tile[2 * plane + base + a], 0.f);
            if (val.x != 0.f || val.y != 0.f || val.z != 0.f)
                atomicAdd(g + (size_t)grow * nx + wrap(x0 + a, nx), val);
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_ib_interp(double* __restrict__ X, float* __restrict__ U, int M,
                                                        const int2* __restrict__ chunks,
                                                        const float4* __restrict__ v,
                                                        uint32_t* __restrict__ flags, int nx, int ny, int nz,
                                                        int advect)
{
    extern __shared__ float tile[];
    __shared__ Stage st;
    __shared__ float su[3][kChunk];
    const int2 ch = block_chunk(chunks, M);
    const int m0 = ch.x, nodes = ch.y;
    if (threadIdx.x < nodes) {
        const int m = m0 + threadIdx.x;
        stage_node(st, threadIdx.x, X[m], X[M + m], X[2 * M + m]);
    }
    const Box b = block_box(st, nodes, nz);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int la = lane & 3, lb = (lane >> 2) & 3, lc = lane >> 4;
    const int plane = b.sx * b.sy * b.ez;
    if (b.tiled) {
        // fill: one warp per tile row; clear the rows' flags
        const int x0 = wrap(b.x0, nx), y0 = wrap(b.y0, ny);
        for (int r = warp; r < b.ey * b.ez; r += kWarps) {
            const int bb = r % b.ey, c = r / b.ey;
            const int grow = (b.z0 + c) * ny + wrap(y0 + bb, ny);
            const int base = (c * b.sy + bb) * b.sx;
            for (int a = lane; a < b.ex; a += 32) {
                const float4 val = v[(size_t)grow * nx + wrap(x0 + a, nx)];
                tile[base + a] = val.x;
                tile[plane + base + a] = val.y;
                tile[2 * plane + base + a] = val.z;
            }
            if (lane == 0) flags[grow] = 0u;
        }
        __syncthreads();
    }
    for (int j = warp; j < nodes; j += kWarps) {
        const float wxy = st.w[la][j] * st.w[4 + lb][j];
        const int bx = st.bx[j], by = st.by[j], bz = st.bz[j];
        float ux = 0.f, uy = 0.f, uz = 0.f;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = lc + 2 * h;
            const float w = wxy * st.w[8 + c][j];
            if (b.tiled) {
                const int k = bz + c - b.z0;
                if (k < 0 || k >= b.ez) continue;
                const int i = (k * b.sy + (by + lb - b.y0)) * b.sx + (bx + la - b.x0);
                ux += w * tile[i];
                uy += w * tile[plane + i];
                uz += w * tile[2 * plane + i];
            } else {
                const int k = bz + c;
                if (k < 0 || k >= nz) continue;
                const int row = k * ny + wrap(by + lb, ny);
                const float4 vv = v[(size_t)row * nx + wrap(bx + la, nx)];
                ux += w * vv.x;
                uy += w * vv.y;
                uz += w * vv.z;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ux += __shfl_xor_sync(0xffffffffu, ux, o);
            uy += __shfl_xor_sync(0xffffffffu, uy, o);
            uz += __shfl_xor_sync(0xffffffffu, uz, o);
        }
        if (lane == 0) {
            su[0][j] = ux;
            su[1][j] = uy;
            su[2][j] = uz;
        }
    }
    __syncthreads();
    if (threadIdx.x < nodes) {
        const int j = threadIdx.x, m = m0 + j;
        const float ux = su[0][j], uy = su[1][j], uz = su[2][j];
        U[m] = ux;
        U[M + m] = uy;
        U[2 * M + m] = uz;
        if (advect) {
            X[m] += (double)ux;
            X[M + m] += (double)uy;
            X[2 * M + m] += (double)uz;
        }
    }
    // fallback path: clear the support rows (after every warp has read them)
    for (int j = warp; j < nodes; j += kWarps) {
        if (la != 0) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = st.bz[j] + lc + 2 * h;
            if (k >= 0 && k < nz) flags[k * ny + wrap(st.by[j] + lb, ny)] = 0u;
        }
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

int launch_ib_spread(LbCtx* c, const double* X, const float* F, int M, const int2* chunks, int n_chunks,
                     cudaStream_t s)
{
    if (M == 0) return PFSI_OK;
    const int blocks = chunks ? n_chunks : (M + kChunk - 1) / kChunk;
    k_ib_spread<<<blocks, kThreads, kTileBytes, s>>>(X, F, M, chunks, c->g, c->flags, c->p.nx, c->p.ny, c->p.nz);
    return check_launch("ib_spread");
}

int launch_ib_interp(LbCtx* c, double* X, float* U, int M, int advect, const int2* chunks, int n_chunks,
                     cudaStream_t s)
{
    if (M == 0) return PFSI_OK;
    const int blocks = chunks ? n_chunks : (M + kChunk - 1) / kChunk;
    k_ib_interp<<<blocks, kThreads, kTileBytes, s>>>(X, U, M, chunks, c->v, c->flags, c->p.nx, c->p.ny, c->p.nz,
                                                     advect);
    return check_launch("ib_interp");
}

}  // namespace pfsi

using namespace pfsi;

extern "C" int ib_spread(lb_ctx* c, const double* X, const float* F, int M, void* stream)
{
    if (!c || M < 0 || (M > 0 && (!X || !F))) return set_error(PFSI_ERR_ARG, "ib_spread: bad argument");
    if (!aligned(X, 8) || !aligned(F, 4)) return set_error(PFSI_ERR_ARG, "ib_spread: misaligned arrays");
    return launch_ib_spread(c, X, F, M, nullptr, 0, as_stream(stream));
}

extern "C" int ib_interp(lb_ctx* c, double* X, float* U, int M, int advect, void* stream)
{
    if (!c || M < 0 || (M > 0 && (!X || !U))) return set_error(PFSI_ERR_ARG, "ib_interp: bad argument");
    if (!aligned(X, 8) || !aligned(U, 4)) return set_error(PFSI_ERR_ARG, "ib_interp: misaligned arrays");
    return launch_ib_interp(c, X, U, M, advect, nullptr, 0, as_stream(stream));
}
