// ib.cu -- immersed-boundary coupling (Section 3.4.2, Eq. 31-36) for sm_103a.
//
// Kernel: phi(r) = (1 + cos(pi r / 2)) / 4 (Eq. 36, h = 1).  With r measured
// from the cell below-left of the node, the four offsets of each axis are
// -1 - t, -t, 1 - t, 2 - t (t in [0,1)), all inside |r| <= 2.  With
// theta = pi t / 2 the four cosines are -sin, cos, sin, -cos of theta, so
// one sincospi per axis gives the weights
//   (1 - sin)/4, (1 + cos)/4, (1 + sin)/4, (1 - cos)/4.
// The support wraps in x and y and is cut at the walls (cells with k outside
// [0, nz) are skipped), so spreading and interpolation stay adjoint.
//
// Blocking: a block of 64 threads takes a chunk of up to 64 consecutive
// nodes, one thread per node (consecutive nodes of a platelet mesh lie close
// together; the coupled step passes chunks that never straddle two
// platelets, the public calls use fixed chunks of 64).  When the bounding
// box of the chunk's supports fits the shared tile (768 cells, no wider than
// the grid):
//   spreading  accumulates F_m * w in the tile in 32-bit fixed point (shared
//              integer atomics run several times faster than shared float
//              atomics on this part), scaled per block by 2^33 / (64 max|F|):
//              every weight is at most 1/8, so no cell sum can reach 2^30,
//              and the rounding stays below ~1e-7 of the block's largest
//              force.  Each lane starts its 16 support rows at a
//              lane-dependent row so that neighbouring nodes seldom hit one
//              address in the same instruction.  The tile is then added to
//              the float4 force field with one vector reduction
//              (red.global.add.v4.f32) per nonzero cell: ~6 per node
//              instead of 64.  Within a block the sum is order-independent.
//   interp     loads the box's velocity into a float4 tile (four coalesced
//              loads in flight per thread) and gathers each node's 64
//              weighted values from it.
// Otherwise the block works on the global arrays directly.  Both kernels take
// the same decision for the same positions and flag / clear the same rows:
// every row of the box (a superset of the support rows), so the lattice step
// writes the velocity wherever interpolation will read it.
#include <climits>

#include "pfsi_internal.cuh"

namespace pfsi {

namespace {

constexpr int kChunk = kIbChunk;            // nodes (= threads) per block
constexpr int kWarps = kChunk / 32;
// 3 int planes (spread) or float4 cells (interp).  Chunks of 128 nodes in
// Morton order of the platelet's rest shape have boxes of ~340 cells on
// average (largest ~1200 on the 500-platelet channel); a 1536-cell tile let
// 8-9 blocks share an SM where a 4096-cell tile held 3.  Chunks of 64 nodes
// with a 768-cell tile (9 KB spreading, 12 KB interpolation) make the
// full-scale step 1.590 -> 1.570 ms (512 cells the same; 64 nodes with 1024
// cells 1.578, 32 nodes with 640 cells 1.598, 256 nodes with 3072 cells 1.623).
constexpr int kTileCells = 768;
constexpr int kMaxRows = kTileCells / 4;    // a box is at least 4 cells wide
constexpr size_t kTileBytes = kTileCells * sizeof(float4);

__device__ __forceinline__ int wrap(int i, int n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

// A node takes part only if all its coordinates lie within +-kFarCoord
// lattice units (false for NaN): the integer cell indices of its support then
// cannot overflow.  A run that blew up leaves such nodes out (no force
// spread; its velocity reads NaN and its position is not advected) instead of
// indexing outside the grid; sim_check reports the state.
__device__ __forceinline__ bool in_range(double x, double y, double z)
{
    return coord_in_range(x) && coord_in_range(y) && coord_in_range(z);
}

struct Node {
    int bx, by, bz;                 // unwrapped cell of support offset 0 on each axis
    float wx[4], wy[4], wz[4];
};

__device__ __forceinline__ void weights(double x, int& b, float* w)
{
    const double f = floor(x);
    b = (int)f - 1;
    float s, c;
    sincospif(0.5f * (float)(x - f), &s, &c);
    w[0] = 0.25f * (1.0f - s);
    w[1] = 0.25f * (1.0f + c);
    w[2] = 0.25f * (1.0f + s);
    w[3] = 0.25f * (1.0f - c);
}

__device__ __forceinline__ void node_support(double x, double y, double z, Node& s)
{
    weights(x, s.bx, s.wx);
    weights(y, s.by, s.wy);
    weights(z, s.bz, s.wz);
}

struct Box {
    int x0, y0, z0;    // unwrapped origin; z0 clipped to the walls
    int ex, ey, ez;    // extents (ez after clipping, may be <= 0)
    bool tiled;
};

// Bounding box of the block's supports (all threads take part).
__device__ Box block_box(const Node& s, bool on, int nx, int ny, int nz)
{
    __shared__ int red[6][kWarps];
    __shared__ Box box;
    int v[6] = {on ? s.bx : INT_MAX, on ? s.by : INT_MAX, on ? s.bz : INT_MAX,
                on ? s.bx : INT_MIN, on ? s.by : INT_MIN, on ? s.bz : INT_MIN};
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
        b.tiled = b.ez > 0 && b.ex <= nx && b.ey <= ny && (long long)b.ex * b.ey * b.ez <= kTileCells;
        box = b;
    }
    __syncthreads();
    return box;
}

__device__ __forceinline__ int2 block_chunk(const int2* __restrict__ chunks, int M, int bx)
{
    if (chunks) return chunks[bx];
    const int m0 = bx * kChunk;
    return make_int2(m0, min(kChunk, M - m0));
}

// Linear index of the first cell of every tile row (bb, c) in the grid.
__device__ __forceinline__ void row_table(const Box& b, int nx, int ny, int* rowbase)
{
    const int y0 = wrap(b.y0, ny);
    for (int r = threadIdx.x; r < b.ey * b.ez; r += kChunk) {
        const int bb = r % b.ey, c = r / b.ey;
        int gy = y0 + bb;
        if (gy >= ny) gy -= ny;
        rowbase[r] = ((b.z0 + c) * ny + gy) * nx;
    }
}

__device__ __forceinline__ void ib_spread_block(const double* __restrict__ X, const float* __restrict__ F, int M,
                                                const int2* __restrict__ chunks, const int* __restrict__ perm,
                                                float4* __restrict__ g, uint32_t* __restrict__ flags, int nx, int ny,
                                                int nz, int bx)
{
    extern __shared__ int itile[];
    __shared__ float swy[4][kChunk], swz[4][kChunk];
    __shared__ float wmax[kWarps];
    __shared__ int rowbase[kMaxRows];
    const int2 ch = block_chunk(chunks, M, bx);
    const bool in_chunk = (int)threadIdx.x < ch.y;
    const int m = in_chunk && perm ? perm[ch.x + threadIdx.x] : ch.x + threadIdx.x;
    Node s;
    float fx = 0.f, fy = 0.f, fz = 0.f;
    bool on = false;
    if (in_chunk) {
        const double x = X[m], y = X[M + m], z = X[2 * M + m];
        on = in_range(x, y, z);
        if (on) node_support(x, y, z, s);
    }
    if (on) {
        fx = F[m];
        fy = F[M + m];
        fz = F[2 * M + m];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            swy[a][threadIdx.x] = s.wy[a];
            swz[a][threadIdx.x] = s.wz[a];
        }
    }
    const int lane = threadIdx.x & 31;
    float fm = fmaxf(fabsf(fx), fmaxf(fabsf(fy), fabsf(fz)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) fm = fmaxf(fm, __shfl_xor_sync(0xffffffffu, fm, o));
    if (lane == 0) wmax[threadIdx.x >> 5] = fm;
    const Box b = block_box(s, on, nx, ny, nz);
    if (b.tiled) {
        float fmax = 0.f;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) fmax = fmaxf(fmax, wmax[w]);
        const float scale = fmax > 0.f ? 8589934592.0f / ((float)kChunk * fmax) : 0.f;  // 2^33 / (kChunk max|F|)
        const int plane = b.ex * b.ey * b.ez;
        for (int i = threadIdx.x; i < 3 * plane; i += kChunk) itile[i] = 0;
        row_table(b, nx, ny, rowbase);
        __syncthreads();
        if (on && scale > 0.f) {
            const int ox = s.bx - b.x0, oy = s.by - b.y0, oz = s.bz - b.z0;
            const float sx = fx * scale, sy = fy * scale, sz = fz * scale;
            for (int q = 0; q < 16; ++q) {
                const int rr = (q + lane) & 15;           // lane-rotated support row
                const int bb = rr & 3, c = rr >> 2;
                const int k = oz + c;
                if (k < 0 || k >= b.ez) continue;
                const float wyz = swy[bb][threadIdx.x] * swz[c][threadIdx.x];
                int* row = itile + (k * b.ey + oy + bb) * b.ex + ox;
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const float w = s.wx[a] * wyz;
                    atomicAdd(row + a, __float2int_rn(sx * w));
                    atomicAdd(row + plane + a, __float2int_rn(sy * w));
                    atomicAdd(row + 2 * plane + a, __float2int_rn(sz * w));
                }
            }
        }
        __syncthreads();
        // flush: cell i = (a, row r), advanced incrementally
        const float inv = scale > 0.f ? 1.0f / scale : 0.f;
        const int x0 = wrap(b.x0, nx);
        const int da = kChunk % b.ex, dr = kChunk / b.ex;
        int a = threadIdx.x % b.ex, r = threadIdx.x / b.ex;
        for (int i = threadIdx.x; i < plane; i += kChunk) {
            if (a == 0) flags[rowbase[r] / nx] = 1u;
            const int vx = itile[i], vy = itile[plane + i], vz = itile[2 * plane + i];
            if (vx | vy | vz) {
                int gx = x0 + a;
                if (gx >= nx) gx -= nx;
                atomicAdd(g + rowbase[r] + gx, make_float4(vx * inv, vy * inv, vz * inv, 0.f));
            }
            a += da;
            r += dr;
            if (a >= b.ex) {
                a -= b.ex;
                ++r;
            }
        }
        return;
    }
    if (!on) return;
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

__global__ void __launch_bounds__(kChunk) k_ib_spread(const double* __restrict__ X, const float* __restrict__ F,
                                                      int M, const int2* __restrict__ chunks,
                                                      const int* __restrict__ perm, float4* __restrict__ g,
                                                      uint32_t* __restrict__ flags, int nx, int ny, int nz)
{
    pdl_wait();
    ib_spread_block(X, F, M, chunks, perm, g, flags, nx, ny, nz, blockIdx.x);
}

// kPart: also write the block's sum of the advected X (next.part)
template <bool kPart>
__device__ __forceinline__ void ib_interp_block(double* __restrict__ X, float* __restrict__ U, int M,
                                                const int2* __restrict__ chunks, const int* __restrict__ perm,
                                                const float4* __restrict__ v, uint32_t* __restrict__ flags, int nx,
                                                int ny, int nz, int advect, const NextSplit& next, int bx)
{
    if (next.acc) {   // the next membrane pass accumulates into cleared sums
        const int t = bx * blockDim.x + threadIdx.x;
        if (t < next.nacc) next.acc[t] = 0.0;
    }
    extern __shared__ float4 tile4[];
    __shared__ int rowbase[kMaxRows];
    const int2 ch = block_chunk(chunks, M, bx);
    const bool in_chunk = (int)threadIdx.x < ch.y;
    const int m = in_chunk && perm ? perm[ch.x + threadIdx.x] : ch.x + threadIdx.x;
    Node s;
    double x = 0.0, y = 0.0, z = 0.0;
    bool on = false;
    if (in_chunk) {
        x = X[m];
        y = X[M + m];
        z = X[2 * M + m];
        on = in_range(x, y, z);
        if (on) node_support(x, y, z, s);
    }
    const Box b = block_box(s, on, nx, ny, nz);
    float ux = 0.f, uy = 0.f, uz = 0.f;
    if (b.tiled) {
        row_table(b, nx, ny, rowbase);
        __syncthreads();
        const int cells = b.ex * b.ey * b.ez;
        const int x0 = wrap(b.x0, nx);
        const int da = kChunk % b.ex, dr = kChunk / b.ex;
        int a = threadIdx.x % b.ex, r = threadIdx.x / b.ex;
        constexpr int kInFlight = 4;
        for (int i0 = threadIdx.x; i0 < cells; i0 += kInFlight * kChunk) {
            float4 val[kInFlight];
#pragma unroll
            for (int u = 0; u < kInFlight; ++u) {
                if (i0 + u * kChunk < cells) {
                    int gx = x0 + a;
                    if (gx >= nx) gx -= nx;
                    val[u] = v[rowbase[r] + gx];
                    if (a == 0) flags[rowbase[r] / nx] = 0u;
                }
                a += da;
                r += dr;
                if (a >= b.ex) {
                    a -= b.ex;
                    ++r;
                }
            }
#pragma unroll
            for (int u = 0; u < kInFlight; ++u)
                if (i0 + u * kChunk < cells) tile4[i0 + u * kChunk] = val[u];
        }
        __syncthreads();
        if (on) {
            const int ox = s.bx - b.x0, oy = s.by - b.y0, oz = s.bz - b.z0;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int k = oz + c;
                if (k < 0 || k >= b.ez) continue;
#pragma unroll
                for (int bb = 0; bb < 4; ++bb) {
                    const float wyz = s.wy[bb] * s.wz[c];
                    const float4* row = tile4 + (k * b.ey + oy + bb) * b.ex + ox;
#pragma unroll
                    for (int aa = 0; aa < 4; ++aa) {
                        const float w = s.wx[aa] * wyz;
                        const float4 vv = row[aa];
                        ux += w * vv.x;
                        uy += w * vv.y;
                        uz += w * vv.z;
                    }
                }
            }
        }
    } else if (on) {
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
                for (int aa = 0; aa < 4; ++aa) {
                    const float w = s.wx[aa] * wyz;
                    const float4 vv = base[wrap(s.bx + aa, nx)];
                    ux += w * vv.x;
                    uy += w * vv.y;
                    uz += w * vv.z;
                }
                flags[row] = 0u;
            }
        }
    }
    double xn[3] = {0.0, 0.0, 0.0};
    if (in_chunk && !on) {
        // left out: its velocity reads NaN and its position stays as it is
        // (also in the split and the block's position sum), so that neither
        // U nor a platelet centroid looks valid; sim_check counts it
        const float qnan = __int_as_float(0x7fffffff);
        U[m] = qnan;
        U[M + m] = qnan;
        U[2 * M + m] = qnan;
        if (advect) {
            xn[0] = x;
            xn[1] = y;
            xn[2] = z;
            if (next.h) {
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const float h = __double2float_rn(xn[d]);
                    next.h[d * M + m] = h;
                    next.l[d * M + m] = __double2float_rn(xn[d] - (double)h);
                }
            }
        }
    }
    if (on) {
        U[m] = ux;
        U[M + m] = uy;
        U[2 * M + m] = uz;
        if (advect) {
            xn[0] = x + widen(ux);
            xn[1] = y + widen(uy);
            xn[2] = z + widen(uz);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                X[d * M + m] = xn[d];
                if (next.h) {   // the hi/lo split the membrane pass would form from X
                    const float h = __double2float_rn(xn[d]);
                    next.h[d * M + m] = h;
                    next.l[d * M + m] = __double2float_rn(xn[d] - (double)h);
                }
            }
        }
    }
    if (kPart && advect) {   // the block's sum of the advected X, fixed order
        __shared__ double wsum[kWarps][3];
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double t = xn[d];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            if (lane == 0) wsum[warp][d] = t;
        }
        __syncthreads();
        if (threadIdx.x < 3) {
            double t = 0.0;
            for (int w = 0; w < kWarps; ++w) t += wsum[w][threadIdx.x];
            next.part[3 * bx + threadIdx.x] = t;
        }
    }
}

// 14 blocks per SM (at most 72 registers, 12 bytes spilled) where the 80
// registers the compiler picks unbounded allow 12: the shared tiles allow 14
// (full-scale step 1.5265 -> 1.5232 ms; 64 registers, 16 blocks, spill 28
// bytes and run 1.537 ms).
template <bool kPart>
__global__ void __launch_bounds__(kChunk, 14) k_ib_interp(double* __restrict__ X, float* __restrict__ U, int M,
                                                      const int2* __restrict__ chunks,
                                                      const int* __restrict__ perm,
                                                      const float4* __restrict__ v,
                                                      uint32_t* __restrict__ flags, int nx, int ny, int nz,
                                                      int advect, const __grid_constant__ NextSplit next)
{
    pdl_wait();
    ib_interp_block<kPart>(X, U, M, chunks, perm, v, flags, nx, ny, nz, advect, next, blockIdx.x);
}

// Spreading and interpolation over several chambers, one launch each (see
// Multi): each chamber's share of the grid takes its nodes' chunks on its
// own lattice.
struct SpreadArgs {
    const double* X;
    const float* F;
    int M;
    const int2* chunks;
    const int* perm;
    float4* g;
    uint32_t* flags;
    int nx, ny, nz;
};
struct InterpArgs {
    double* X;
    float* U;
    int M;
    const int2* chunks;
    const int* perm;
    const float4* v;
    uint32_t* flags;
    int nx, ny, nz;
};

__global__ void __launch_bounds__(kChunk) k_ib_spread_multi(const __grid_constant__ Multi<SpreadArgs> t)
{
    pdl_wait();
    const int e = multi_entry(t, blockIdx.x);
    const SpreadArgs& a = t.a[e];
    ib_spread_block(a.X, a.F, a.M, a.chunks, a.perm, a.g, a.flags, a.nx, a.ny, a.nz, blockIdx.x - t.first[e]);
}

__global__ void __launch_bounds__(kChunk) k_ib_interp_multi(const __grid_constant__ Multi<InterpArgs> t)
{
    pdl_wait();
    const int e = multi_entry(t, blockIdx.x);
    const InterpArgs& a = t.a[e];
    const NextSplit none;
    ib_interp_block<false>(a.X, a.U, a.M, a.chunks, a.perm, a.v, a.flags, a.nx, a.ny, a.nz, 1, none,
                           blockIdx.x - t.first[e]);
}

}  // namespace

int ib_prepare()
{
    int rc = check_cuda(cudaFuncSetAttribute(k_ib_spread, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileBytes),
                        "ib: shared memory size");
    if (!rc)
        rc = check_cuda(cudaFuncSetAttribute(k_ib_interp<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kTileBytes),
                        "ib: shared memory size");
    if (!rc)
        rc = check_cuda(cudaFuncSetAttribute(k_ib_interp<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kTileBytes),
                        "ib: shared memory size");
    if (!rc)
        rc = check_cuda(cudaFuncSetAttribute(k_ib_spread_multi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kTileBytes),
                        "ib: shared memory size");
    if (!rc)
        rc = check_cuda(cudaFuncSetAttribute(k_ib_interp_multi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kTileBytes),
                        "ib: shared memory size");
    return rc;
}

int launch_ib_spread(LbCtx* c, const double* X, const float* F, int M, const int2* chunks, const int* perm, int n_chunks,
                     cudaStream_t s)
{
    if (M == 0) return PFSI_OK;
    const int blocks = chunks ? n_chunks : (M + kChunk - 1) / kChunk;
    return check_cuda(launch_pdl(k_ib_spread, dim3(blocks), dim3(kChunk), 3 * kTileCells * sizeof(int), s, X, F, M, chunks,
                                 perm, c->g, c->flags, c->p.nx, c->p.ny, c->p.nz),
                      "ib_spread");
}

int launch_ib_interp(LbCtx* c, double* X, float* U, int M, int advect, const int2* chunks, const int* perm, int n_chunks,
                     cudaStream_t s, NextSplit next)
{
    if (M == 0) return PFSI_OK;
    const int blocks = chunks ? n_chunks : (M + kChunk - 1) / kChunk;
    if (next.acc && (long long)blocks * kChunk < next.nacc)
        return set_error(PFSI_ERR_ARG, "ib_interp: fewer threads than per-platelet sums to clear");
    if (next.part && !chunks)
        return set_error(PFSI_ERR_ARG, "ib_interp: chunk sums need the chunk table");
    return check_cuda(launch_pdl(next.part ? k_ib_interp<true> : k_ib_interp<false>, dim3(blocks), dim3(kChunk), kTileBytes,
                                 s, X, U, M, chunks, perm, (const float4*)velocity_field(c), c->flags, c->p.nx, c->p.ny,
                                 c->p.nz, advect, next),
                      "ib_interp");
}

int launch_ib_spread_multi(const Chamber* ch, int n, cudaStream_t s)
{
    std::vector<Multi<SpreadArgs>> lists;
    for (int i = 0; i < n; ++i) {
        const LbCtx* c = ch[i].lb;
        const MemCtx* m = ch[i].mem;
        multi_push(lists, SpreadArgs{ch[i].X, ch[i].F, ch[i].M, m->chunks, m->perm, c->g, c->flags, c->p.nx, c->p.ny,
                                     c->p.nz},
                   ch[i].M > 0 ? m->n_chunks : 0);
    }
    int rc = PFSI_OK;
    for (const auto& t : lists)
        if (!rc)
            rc = check_cuda(launch_pdl(k_ib_spread_multi, dim3(t.blocks()), dim3(kChunk), 3 * kTileCells * sizeof(int), s, t),
                            "ib_spread");
    return rc;
}

int launch_ib_interp_multi(const Chamber* ch, int n, cudaStream_t s)
{
    std::vector<Multi<InterpArgs>> lists;
    for (int i = 0; i < n; ++i) {
        const LbCtx* c = ch[i].lb;
        const MemCtx* m = ch[i].mem;
        multi_push(lists, InterpArgs{ch[i].X, ch[i].U, ch[i].M, m->chunks, m->perm, velocity_field(c), c->flags,
                                     c->p.nx, c->p.ny, c->p.nz},
                   ch[i].M > 0 ? m->n_chunks : 0);
    }
    int rc = PFSI_OK;
    for (const auto& t : lists)
        if (!rc)
            rc = check_cuda(launch_pdl(k_ib_interp_multi, dim3(t.blocks()), dim3(kChunk), kTileBytes, s, t), "ib_interp");
    return rc;
}

}  // namespace pfsi

using namespace pfsi;

extern "C" int ib_spread(lb_ctx* c, const double* X, const float* F, int M, void* stream)
{
    NvtxRange nvtx_range("ib_spread");
    if (!c || M < 0 || (M > 0 && (!X || !F))) return set_error(PFSI_ERR_ARG, "ib_spread: bad argument");
    if (!aligned(X, 8) || !aligned(F, 4)) return set_error(PFSI_ERR_ARG, "ib_spread: misaligned arrays");
    return launch_ib_spread(c, X, F, M, nullptr, nullptr, 0, as_stream(stream));
}

extern "C" int ib_interp(lb_ctx* c, double* X, float* U, int M, int advect, void* stream)
{
    NvtxRange nvtx_range("ib_interp");
    if (!c || M < 0 || (M > 0 && (!X || !U))) return set_error(PFSI_ERR_ARG, "ib_interp: bad argument");
    if (!aligned(X, 8) || !aligned(U, 4)) return set_error(PFSI_ERR_ARG, "ib_interp: misaligned arrays");
    return launch_ib_interp(c, X, U, M, advect, nullptr, nullptr, 0, as_stream(stream));
}
