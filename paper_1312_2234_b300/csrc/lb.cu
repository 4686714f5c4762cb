// lb.cu -- D3Q19 lattice Boltzmann step (Section 3.3, Eq. 16-21) for sm_103a.
//
// One fused kernel per step: pull streaming from the post-collision buffer
// (periodic x, y; halfway bounce-back at the z walls with the moving-wall
// term at the top), moments (Eq. 17-18), force-corrected velocity
// v = u + F/(2 rho), BGK relaxation to the equilibrium of Eq. 20 and Guo's
// source (Eq. 19 with the (c c^T - c_s^2 I) tensor), written to the other
// buffer.  Populations are stored shifted, f~ = f - w_q, so that FP32 keeps
// the small deviations from rest that carry the flow (|u| ~ 1e-5..1e-3).
//
// Layout: structure of arrays f[q][cell], x fastest; one thread per cell, a
// block covers a run of one (j, k) row so that the wall branch and the row's
// force flag are uniform across the block.  Traffic per cell: 19 float
// loads + 19 float stores (152 B), plus, in rows marked by the spreading
// kernel, the force (16 B read, 16 B cleared) and the velocity (16 B).
//
// Mixed storage keeps, per cell, the post-collision non-equilibrium part
// f*neq_q = f*_q - E_q(m) in 16 bits and m = (v, rho - 1) in FP32 (108 B per
// cell per step), E_q the split of pfsi_internal.cuh (the equilibrium of
// Eq. 20 up to w_q rho (1 - rho) (3 c.v)^2 / 2).  The state is the same as
// the FP32 one up to the rounding of f*neq: a pulling cell rebuilds f*_q of
// its source cell as E_q(m of the source) + f*neq_q, collides in FP32 exactly
// as above and stores its own f*neq and m.  The 18 neighbour moments a cell
// reads are shared with its neighbours; only the own cell's m travels from
// DRAM.  lb_tma.cu holds the TMA-staged kernel of this storage; the kernel
// here serves grids whose rows do not start on 16-byte boundaries.
#include <algorithm>
#include <climits>
#include <string>
#include <utility>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "pfsi_internal.cuh"

namespace pfsi {

namespace {

constexpr int kRowBlock = 128;     // default threads per block along x (FP32 kernel)
constexpr int kMaxRowBlock = 256;

// Stream-collide of cell (i, j, k) with FP32 shifted populations: the body
// of k_lb_step and of the batched k_lb_step_batch.
__device__ __forceinline__ void fp32_cell(const float* __restrict__ fin, float* __restrict__ fout,
                                          float4* __restrict__ g, float4* __restrict__ vout,
                                          const uint32_t* __restrict__ flags, int nx, int ny, int nz, int i, int j,
                                          int k, float omega, float guo, float3 body, float3 utop, int onsite)
{
    const int N = nx * ny * nz;
    const int row = k * ny + j;
    const int cell = row * nx + i;
    const int xm = (i == 0) ? nx - 1 : i - 1;       // source column for c_x = +1
    const int xp = (i == nx - 1) ? 0 : i + 1;       // source column for c_x = -1
    const int ym = (j == 0) ? ny - 1 : j - 1;
    const int yp = (j == ny - 1) ? 0 : j + 1;

    float f[19];
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        const int sx = cxq(q) == 1 ? xm : (cxq(q) == -1 ? xp : i);
        const int sy = cyq(q) == 1 ? ym : (cyq(q) == -1 ? yp : j);
        const int sk = k - czq(q);
        if (czq(q) == 1 && k == 0) {
            f[q] = fin[oppq(q) * N + cell];                         // still bottom wall
        } else if (czq(q) == -1 && k == nz - 1) {
            const float cu = cxq(q) * utop.x + cyq(q) * utop.y;     // moving top wall,
            f[q] = fin[oppq(q) * N + cell] + 6.0f * wq(q) * cu;     // rho_w = 1
        } else {
            f[q] = fin[q * N + (sk * ny + sy) * nx + sx];
        }
    }
    if (onsite) {   // on-site walls replace the bounce-back values of the entering populations
        if (k == 0) onsite_wall<1>(f, make_float3(0.f, 0.f, 0.f));
        if (k == nz - 1) onsite_wall<-1>(f, utop);
    }

    float drho = 0.f, mx = 0.f, my = 0.f, mz = 0.f;
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        drho += f[q];
        if (cxq(q)) mx += cxq(q) * f[q];
        if (cyq(q)) my += cyq(q) * f[q];
        if (czq(q)) mz += czq(q) * f[q];
    }
    const float rho = 1.0f + drho;
    float Fx = body.x, Fy = body.y, Fz = body.z;
    const bool forced = flags[row] != 0u;
    if (forced) {
        const float4 gg = g[cell];
        Fx += gg.x;
        Fy += gg.y;
        Fz += gg.z;
    }
    const float irho = 1.0f / rho;
    const float vx = (mx + 0.5f * Fx) * irho;
    const float vy = (my + 0.5f * Fy) * irho;
    const float vz = (mz + 0.5f * Fz) * irho;
    const float vv = fmaf(vx, vx, fmaf(vy, vy, vz * vz));
    const float vF = fmaf(vx, Fx, fmaf(vy, Fy, vz * Fz));

    // f~' = (1 - omega) f~ + omega (f^eq - w) + S with the equilibrium of
    // Eq. 20 and Guo's source w (1 - 1/2tau) [3 c.F + 9 (c.v)(c.F) - 3 v.F]
    // (Eq. 19), taken per pair of opposite directions: with
    //   a = w 3 omega rho (c.v),  b = w 3 guo (c.F),
    //   A0 = omega (drho - 1.5 rho v.v) - 3 guo v.F,
    // the part even in c is w A0 + 1.5 (c.v)(a + 2b) and the odd part a + b.
    const float keep = 1.0f - omega;
    const float R3 = 3.0f * omega * rho;
    const float G3 = 3.0f * guo;
    const float A0 = fmaf(omega, fmaf(-1.5f * rho, vv, drho), -G3 * vF);
    fout[18 * N + cell] = fmaf(keep, f[18], wq(18) * A0);
#pragma unroll
    for (int q = 0; q < 18; ++q) {
        if (oppq(q) < q) continue;
        const int o = oppq(q);
        float cv = 0.f, cF = 0.f;
        if (cxq(q)) { cv += cxq(q) * vx; cF += cxq(q) * Fx; }
        if (cyq(q)) { cv += cyq(q) * vy; cF += cyq(q) * Fy; }
        if (czq(q)) { cv += czq(q) * vz; cF += czq(q) * Fz; }
        const float a = (wq(q) * R3) * cv;
        const float b = (wq(q) * G3) * cF;
        const float odd = fmaf(wq(q) * R3, cv, b);
        const float even = fmaf(1.5f * cv, fmaf(2.0f, b, a), wq(q) * A0);
        fout[q * N + cell] = fmaf(keep, f[q], even + odd);
        fout[o * N + cell] = fmaf(keep, f[o], even - odd);
    }
    if (forced) {
        vout[cell] = make_float4(vx, vy, vz, rho);
        g[cell] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

__global__ void __launch_bounds__(kMaxRowBlock) k_lb_step(
    const float* __restrict__ fin, float* __restrict__ fout, float4* __restrict__ g,
    float4* __restrict__ vout, const uint32_t* __restrict__ flags, int nx, int ny, int nz,
    float omega, float guo, float3 body, float3 utop, int onsite)
{
    pdl_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx) return;
    fp32_cell(fin, fout, g, vout, flags, nx, ny, nz, i, blockIdx.y, blockIdx.z, omega, guo, body, utop, onsite);
}

// 16-bit encodings of f*neq: BF16 as is, FP16 scaled by 2^s (get takes
// 2^-s, put takes 2^s; both exact powers of two).
template <int kMode>
struct Neq;
template <>
struct Neq<PFSI_LB_BF16> {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ float get(T h, float) { return __bfloat162float(h); }
    static __device__ __forceinline__ T put(float x, float) { return __float2bfloat16_rn(x); }
};
template <>
struct Neq<PFSI_LB_FP16> {
    using T = __half;
    static __device__ __forceinline__ float get(T h, float inv_scale) { return __half2float(h) * inv_scale; }
    static __device__ __forceinline__ T put(float x, float scale) { return __float2half_rn(x * scale); }
};

// Mixed kernel blocking: a block takes a 32 x 8 (x, y) column of cells and
// marches it through kz consecutive planes.  The moments of the column plus
// a one-cell halo are kept for the planes k - 1, k, k + 1 in a shared ring
// of four slots (the fourth takes plane k + 2 while k computes, so one
// barrier per plane suffices); each moment comes from L2
// ~(340 / 256)(kz + 2) / kz times per step instead of 19 times through L1.
// A warp is one tile row.
//
// The ring holds each cell's record in the form the rebuild wants, (P, J)
// of split_record, so that E_q costs three operations per pulled
// population.
template <int TX_, int TY_>
struct Tile {
    static constexpr int TX = TX_, TY = TY_;
    static constexpr int HX = TX + 2, HY = TY + 2;
    static constexpr int Plane = HX * HY;
    static constexpr int Threads = TX * TY;
    static constexpr int Halo = (Plane + Threads - 1) / Threads;
};
constexpr int kSlots = 4;

template <class T>
struct Ring {
    float4 pj[kSlots][T::Plane];   // (P, Jx, Jy, Jz)
};

template <class T>
__device__ __forceinline__ void halo_load(const float4* __restrict__ m, int k, int plane_cells, const int* off,
                                          float4* r)
{
    const float4* plane = m + (size_t)k * plane_cells;
#pragma unroll
    for (int u = 0; u < T::Halo; ++u)
        if (off[u] >= 0) r[u] = plane[off[u]];
}

// Ring position of halo cell h (row-major over the tile plus halo).  The
// two-cell tiles (PairTile) keep each row's odd-x and even-x halo cells in
// two halves (odd first): a thread's two cells are x-adjacent, so with a
// row-major ring the 32 lanes of a warp would read records 32 bytes apart
// (twice the shared-memory wavefronts); split by parity, the lanes read
// consecutive records for every direction.
template <int TY_>
struct PairTile;
template <class T>
struct IsPairTile {
    static constexpr bool value = false;
};
template <int TY>
struct IsPairTile<PairTile<TY>> {
    static constexpr bool value = true;
};
template <class T>
__device__ __forceinline__ int ring_pos(int h)
{
    if constexpr (IsPairTile<T>::value) {
        const int hy = h / T::HX, hx = h - hy * T::HX;
        return hy * T::HX + ((hx & 1) ? (hx >> 1) : T::HX / 2 + (hx >> 1));
    } else {
        return h;
    }
}

template <class T>
__device__ __forceinline__ void halo_store(Ring<T>& ring, int slot, const float4* r)
{
#pragma unroll
    for (int u = 0; u < T::Halo; ++u) {
        const int h = threadIdx.x + u * T::Threads;
        if (h < T::Plane) ring.pj[slot][ring_pos<T>(h)] = split_record(r[u]);
    }
}

// f[q] += E_q of the source cell (bounce-back: the own cell's opposite
// population, plus the moving-wall term at the top).  sm, s0, sp: ring slots
// of the planes k - 1, k, k + 1.
template <int q, class T>
__device__ __forceinline__ void add_feq(float* f, const Ring<T>& ring, int sm, int s0, int sp, int own, int k,
                                        int nz, float3 utop)
{
    if (czq(q) == 1 && k == 0) {
        f[q] = fmaf(wq(q), split_eq<oppq(q)>(ring.pj[s0][own]), f[q]);
    } else if (czq(q) == -1 && k == nz - 1) {
        const float cu = cxq(q) * utop.x + cyq(q) * utop.y;
        f[q] = fmaf(wq(q), split_eq<oppq(q)>(ring.pj[s0][own]), fmaf(6.0f * wq(q), cu, f[q]));
    } else {
        f[q] = fmaf(wq(q), split_eq<q>(ring.pj[czq(q) == 1 ? sm : (czq(q) == -1 ? sp : s0)][own - cyq(q) * T::HX - cxq(q)]),
                    f[q]);
    }
}

template <class T, int... Q>
__device__ __forceinline__ void add_feq_all(std::integer_sequence<int, Q...>, float* f, const Ring<T>& ring, int sm,
                                            int s0, int sp, int own, int k, int nz, float3 utop)
{
    (add_feq<Q>(f, ring, sm, s0, sp, own, k, nz, utop), ...);
}

// Raw 16-bit f*neq a cell of plane k pulls (bounce-back: its own opposite).
__device__ __forceinline__ void load_neq(const uint16_t* __restrict__ nin, uint32_t* raw, int N, int k, int nz,
                                         int nx, int ny, int i, int j, int xm, int xp, int ym, int yp)
{
    const int cell = (k * ny + j) * nx + i;
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        if ((czq(q) == 1 && k == 0) || (czq(q) == -1 && k == nz - 1)) {
            raw[q] = nin[nslot(oppq(q)) * N + cell];
        } else {
            const int sx = cxq(q) == 1 ? xm : (cxq(q) == -1 ? xp : i);
            const int sy = cyq(q) == 1 ? ym : (cyq(q) == -1 ? yp : j);
            raw[q] = nin[nslot(q) * N + ((k - czq(q)) * ny + sy) * nx + sx];
        }
    }
}

template <int kMode>
__device__ __forceinline__ float neq_value(uint32_t raw, float inv_scale)
{
    if (kMode == PFSI_LB_BF16) return __uint_as_float(raw << 16);
    return __half2float(__ushort_as_half((unsigned short)raw)) * inv_scale;
}

// Stored values of the pair (q, opposite of q) of one cell: the part even
// in c is w E0 + cv (h + b), the odd part a + b (see mixed_column).
template <int kMode, int q>
__device__ __forceinline__ void store_pair(typename Neq<kMode>::T* __restrict__ nout, int N, int cell, const float* f,
                                           float vx, float vy, float vz, float3 F3, float rk, float rh, float keep,
                                           float E0, float guo, float scale)
{
    if (q == 18 || oppq(q) < q) return;
    const float cv = cdot<q>(vx, vy, vz), cF = cdot<q>(F3.x, F3.y, F3.z);
    const float wcv = wq(q) * cv;
    const float b = (wq(q) * guo) * cF;
    const float odd = fmaf(rk, wcv, b);
    const float even = fmaf(cv, fmaf(rh, wcv, b), wq(q) * E0);
    nout[nslot(q) * N + cell] = Neq<kMode>::put(fmaf(keep, f[q], even + odd), scale);
    nout[nslot(oppq(q)) * N + cell] = Neq<kMode>::put(fmaf(keep, f[oppq(q)], even - odd), scale);
}

template <int kMode, int... Q>
__device__ __forceinline__ void store_pairs(std::integer_sequence<int, Q...>, typename Neq<kMode>::T* __restrict__ nout,
                                            int N, int cell, const float* f, float vx, float vy, float vz, float3 F3,
                                            float rk, float rh, float keep, float E0, float guo, float scale)
{
    (store_pair<kMode, Q>(nout, N, cell, f, vx, vy, vz, F3, rk, rh, keep, E0, guo, scale), ...);
}

// One column of the mixed step: the (x, y) tile at (x0, y0) marched through
// the planes z0 <= k < z1 (the body of k_lb_step_mixed and of the batched
// k_lb_step_batch_mixed).  The ring is free again when it returns.
template <int kMode, class T>
__device__ __forceinline__ void mixed_column(Ring<T>& ring, const uint16_t* __restrict__ nin,
                                             typename Neq<kMode>::T* __restrict__ nout,
                                             const float4* __restrict__ min_, float4* __restrict__ mout,
                                             float4* __restrict__ g, const uint32_t* __restrict__ flags, int nx,
                                             int ny, int nz, int x0, int y0, int z0, int z1, float omega, float guo,
                                             float3 body, float3 utop, float inv_scale, int onsite)
{
    const int tx = threadIdx.x % T::TX, ty = threadIdx.x / T::TX;
    const int i = x0 + tx, j = y0 + ty;
    const bool live = i < nx && j < ny;
    const int N = nx * ny * nz;
    const int plane_cells = nx * ny;
    const int xm = (i == 0) ? nx - 1 : i - 1;
    const int xp = (i >= nx - 1) ? 0 : i + 1;
    const int ym = (j == 0) ? ny - 1 : j - 1;
    const int yp = (j >= ny - 1) ? 0 : j + 1;
    const float keep = 1.0f - omega;
    const float scale = 1.0f / inv_scale;
    const int own = (ty + 1) * T::HX + tx + 1;

    // in-plane offsets of this thread's halo cells (wrapped in x and y)
    int off[T::Halo];
#pragma unroll
    for (int u = 0; u < T::Halo; ++u) {
        const int h = threadIdx.x + u * T::Threads;
        const int hy = h / T::HX, hx = h - hy * T::HX;
        int gx = x0 + hx - 1, gy = y0 + hy - 1;
        gx = gx < 0 ? gx + nx : (gx >= nx ? gx % nx : gx);
        gy = gy < 0 ? gy + ny : (gy >= ny ? gy % ny : gy);
        off[u] = h < T::Plane ? gy * nx + gx : -1;
    }

    float4 r[T::Halo];
    for (int p = max(z0 - 1, 0); p <= min(z0 + 1, nz - 1); ++p) {
        halo_load<T>(min_, p, plane_cells, off, r);
        halo_store<T>(ring, p & 3, r);
    }
    __syncthreads();

    const float3 F3b = make_float3(3.0f * body.x, 3.0f * body.y, 3.0f * body.z);
    for (int k = z0; k < z1; ++k) {
        const bool pre = k + 2 < nz && k + 2 <= z1;
        if (pre) halo_load<T>(min_, k + 2, plane_cells, off, r);
        if (live) {
            const int cell = (k * ny + j) * nx + i;
            uint32_t raw[19];
            load_neq(nin, raw, N, k, nz, nx, ny, i, j, xm, xp, ym, yp);
            float f[19];
#pragma unroll
            for (int q = 0; q < 19; ++q) f[q] = neq_value<kMode>(raw[q], inv_scale);
            add_feq_all(std::make_integer_sequence<int, 19>{}, f, ring, (k + 3) & 3, k & 3, (k + 1) & 3, own, k,
                        nz, utop);
            if (onsite) {
                if (k == 0) onsite_wall<1>(f, make_float3(0.f, 0.f, 0.f));
                if (k == nz - 1) onsite_wall<-1>(f, utop);
            }

            // moments per pair of opposite directions (the order every
            // 16-bit kernel uses, so that they agree bit for bit)
            float drho = f[18], mx = 0.f, my = 0.f, mz = 0.f;
#pragma unroll
            for (int q = 0; q < 18; ++q) {
                if (oppq(q) < q) continue;
                const float s = f[q] + f[oppq(q)], d = f[q] - f[oppq(q)];
                drho += s;
                if (cxq(q)) mx = cxq(q) > 0 ? mx + d : mx - d;
                if (cyq(q)) my = cyq(q) > 0 ? my + d : my - d;
                if (czq(q)) mz = czq(q) > 0 ? mz + d : mz - d;
            }
            const float rho = 1.0f + drho;
            float3 F3 = F3b;
            const bool forced = flags[k * ny + j] != 0u;
            if (forced) {
                const float4 gg = g[cell];
                F3.x = fmaf(3.0f, gg.x, F3.x);
                F3.y = fmaf(3.0f, gg.y, F3.y);
                F3.z = fmaf(3.0f, gg.z, F3.z);
            }
            // V = 3v = 3 (m + F/2) / rho; F3 = 3F
            const float i3rho = __fdividef(3.0f, rho);   // fast division (~2 ulp), as every 16-bit kernel
            const float vx = fmaf(F3.x, 1.0f / 6.0f, mx) * i3rho;
            const float vy = fmaf(F3.y, 1.0f / 6.0f, my) * i3rho;
            const float vz = fmaf(F3.z, 1.0f / 6.0f, mz) * i3rho;
            const float VV = fmaf(vx, vx, fmaf(vy, vy, vz * vz));                   // 9 v.v
            const float P0 = fmaf(rho * (-1.0f / 6.0f), VV, drho);                   // drho - 1.5 rho v.v
            const float vF3 = fmaf(vx, F3.x, fmaf(vy, F3.y, vz * F3.z)) * (1.0f / 3.0f);  // 3 v.F
            // stored f* - E = (1 - omega)(f - f^eq) + S + (f^eq - E), with
            // (f^eq - w)/w = P0 + rho (cv + cv^2/2), S/(w guo) = cF (1 + cv) - vF3
            // and (f^eq - E)/w = rho (1 - rho) cv^2 / 2 (cv = 3 c.v, cF = 3 c.F),
            // per pair of opposite directions: with
            //   a = -keep w rho cv,  h = w rho cv (omega - rho) / 2,  b = w guo cF,
            //   E0 = -keep P0 - guo vF3,
            // the part even in c is w E0 + cv (h + b), the odd part a + b.
            const float E0 = fmaf(-keep, P0, -guo * vF3);
            const float rh = 0.5f * rho * (omega - rho);
            nout[nslot(18) * N + cell] = Neq<kMode>::put(fmaf(keep, f[18], wq(18) * E0), scale);
            store_pairs<kMode>(std::make_integer_sequence<int, 18>{}, nout, N, cell, f, vx, vy, vz, F3,
                               -keep * rho, rh, keep, E0, guo, scale);
            mout[cell] = make_float4(vx * (1.0f / 3.0f), vy * (1.0f / 3.0f), vz * (1.0f / 3.0f), drho);
            if (forced) g[cell] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (pre) halo_store<T>(ring, (k + 2) & 3, r);   // slot of plane k - 2: no longer read
        __syncthreads();
    }
}

template <int kMode, class T>
__global__ void __launch_bounds__(T::Threads, 768 / T::Threads) k_lb_step_mixed(
    const uint16_t* __restrict__ nin, typename Neq<kMode>::T* __restrict__ nout, const float4* __restrict__ min_,
    float4* __restrict__ mout, float4* __restrict__ g, const uint32_t* __restrict__ flags, int nx, int ny, int nz,
    int kz, float omega, float guo, float3 body, float3 utop, float inv_scale, int onsite)
{
    pdl_wait();
    __shared__ Ring<T> ring;
    const int z0 = blockIdx.z * kz;
    mixed_column<kMode, T>(ring, nin, nout, min_, mout, g, flags, nx, ny, nz, blockIdx.x * T::TX, blockIdx.y * T::TY,
                           z0, min(z0 + kz, nz), omega, guo, body, utop, inv_scale, onsite);
}

// ---------------------------------------------------------------------------
// Pair kernel of the mixed storage: a thread takes two x-adjacent cells of a
// row, (x0 + 2 tx, x0 + 2 tx + 1) of a 64 x TY tile marched through kz
// planes like the kernel above (same ring of moment records, 32 x TY
// threads).  The two cells share their address arithmetic (the second
// cell's values sit 2 bytes after the first's), with an even nx their
// 16-bit values along x move as one 32-bit word per direction, and each
// floating-point operation of the step runs on both cells as one packed
// FP32x2 instruction (add, mul, fma .rn .f32x2: per lane the rounding of
// the scalar operation).  Every lane follows the operation sequence of
// mixed_column exactly, so the two kernels give bit-identical populations.
template <int TY_>
struct PairTile {
    static constexpr int TX = 64, TY = TY_;
    static constexpr int HX = TX + 2, HY = TY + 2;   // HX even: the parity halves of a ring row are equal
    static constexpr int Plane = HX * HY;
    static constexpr int Threads = 32 * TY;
    static constexpr int Halo = (Plane + Threads - 1) / Threads;
};

__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b as one fma with the exact product -1 b: the rounding of a - b, and
// no separate negation of the packed operand
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return fma2(dup2(-1.0f), b, a); }

// s a + t b for s, t = +-1 (the products exact): the rounding of the sum
template <int s, int t>
__device__ __forceinline__ float2 signed_sum2(float2 a, float2 b)
{
    if (s > 0) return t > 0 ? add2(a, b) : sub2(a, b);
    if (t > 0) return sub2(b, a);
    return sub2(mul2(dup2(-1.0f), a), b);   // (-a) + (-b), signed zeros included
}
template <int s>
__device__ __forceinline__ float2 signed2(float2 a)
{
    return s > 0 ? a : mul2(dup2(-1.0f), a);
}

// c_q . (x, y, z) of both cells: per lane the value of cdot
template <int q>
__device__ __forceinline__ float2 cdot2(float2 x, float2 y, float2 z)
{
    constexpr int cx = cxq(q), cy = cyq(q), cz = czq(q);
    if (cx != 0 && cy != 0) return signed_sum2<cx, cy>(x, y);
    if (cx != 0 && cz != 0) return signed_sum2<cx, cz>(x, z);
    if (cy != 0 && cz != 0) return signed_sum2<cy, cz>(y, z);
    if (cx != 0) return signed2<cx>(x);
    if (cy != 0) return signed2<cy>(y);
    if (cz != 0) return signed2<cz>(z);
    return dup2(0.f);
}

// f*neq of direction q that the two cells of plane k pull, as floats
// (bounce-back at k = 0 and nz - 1: the own cells' opposite slot).  kWord: the two
// values along x sit in one aligned 32-bit word (even nx; i1 = i0 + 1 in
// the same row).
template <int kMode, int q, bool kWord>
__device__ __forceinline__ float2 pull_pair(const uint16_t* __restrict__ nin, int N, int k, int nz, int nx, int ny,
                                            int j, int ym, int yp, int i0, int i1, int xm0, int xm1, int xp0,
                                            int xp1, float inv_scale)
{
    const bool bounce = (czq(q) == 1 && k == 0) || (czq(q) == -1 && k == nz - 1);
    const int sy = cyq(q) == 1 ? ym : (cyq(q) == -1 ? yp : j);
    const uint16_t* row = bounce ? nin + nslot(oppq(q)) * N + (k * ny + j) * nx
                                 : nin + nslot(q) * N + ((k - czq(q)) * ny + sy) * nx;
    const bool straight = bounce || cxq(q) == 0;   // both sources at i0, i1
    if (kWord && straight) {   // (kWord: i0 even, the word aligned)
        const uint32_t w = *reinterpret_cast<const uint32_t*>(row + i0);
        if constexpr (kMode == PFSI_LB_BF16)
            return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
        return mul2(__half22float2(*reinterpret_cast<const __half2*>(&w)), dup2(inv_scale));
    }
    const int a = straight ? i0 : (cxq(q) == 1 ? xm0 : xp0);
    const int b = straight ? i1 : (cxq(q) == 1 ? xm1 : xp1);
    const uint32_t r0 = row[a], r1 = row[b];
    if constexpr (kMode == PFSI_LB_BF16) return make_float2(__uint_as_float(r0 << 16), __uint_as_float(r1 << 16));
    return mul2(make_float2(__half2float(__ushort_as_half((unsigned short)r0)),
                            __half2float(__ushort_as_half((unsigned short)r1))),
                dup2(inv_scale));
}

// Offset in the parity-split ring row of the halo cell dx cells right of a
// thread's first cell (halo x = 2 tx + 1 + dx, dx in -1..2), from the
// thread's base (ty + 1) HX + tx.
template <class T, int dx>
__device__ __forceinline__ constexpr int pair_off()
{
    return ((1 + dx) & 1) ? ((1 + dx) >> 1) : T::HX / 2 + ((1 + dx) >> 1);
}

// F += E_q of the source cells (as add_feq, both cells; own = the thread's
// ring base (ty + 1) HX + tx)
template <int q, class T>
__device__ __forceinline__ void add_feq2(float2& F, const Ring<T>& ring, int sm, int s0, int sp, int own, int k,
                                         int nz, float3 utop)
{
    if (czq(q) == 1 && k == 0) {
        const float4 a = ring.pj[s0][own + pair_off<T, 0>()], b = ring.pj[s0][own + pair_off<T, 1>()];
        F = fma2(dup2(wq(q)), make_float2(split_eq<oppq(q)>(a), split_eq<oppq(q)>(b)), F);
    } else if (czq(q) == -1 && k == nz - 1) {
        const float cu = cxq(q) * utop.x + cyq(q) * utop.y;
        const float4 a = ring.pj[s0][own + pair_off<T, 0>()], b = ring.pj[s0][own + pair_off<T, 1>()];
        F = fma2(dup2(wq(q)), make_float2(split_eq<oppq(q)>(a), split_eq<oppq(q)>(b)),
                 fma2(dup2(6.0f * wq(q)), dup2(cu), F));
    } else {
        const int slot = czq(q) == 1 ? sm : (czq(q) == -1 ? sp : s0);
        const int src = own - cyq(q) * T::HX;
        const float4 a = ring.pj[slot][src + pair_off<T, -cxq(q)>()],
                     b = ring.pj[slot][src + pair_off<T, 1 - cxq(q)>()];
        // E / w = P + cj (1 + cj / 2), both cells at once
        const float2 cj = make_float2(cdot<q>(a.y, a.z, a.w), cdot<q>(b.y, b.z, b.w));
        const float2 e = fma2(cj, fma2(cj, dup2(0.5f), dup2(1.0f)), make_float2(a.x, b.x));
        F = fma2(dup2(wq(q)), e, F);
    }
}

template <int kMode, bool kWord, class T, int... Q>
__device__ __forceinline__ void pull_all2(std::integer_sequence<int, Q...>, float2* F, const uint16_t* __restrict__ nin,
                                          int N, int k, int nz, int nx, int ny, int j, int ym, int yp, int i0,
                                          int i1, int xm0, int xm1, int xp0, int xp1, float inv_scale,
                                          const Ring<T>& ring, int sm, int s0, int sp, int own, float3 utop)
{
    ((F[Q] = pull_pair<kMode, Q, kWord>(nin, N, k, nz, nx, ny, j, ym, yp, i0, i1, xm0, xm1, xp0, xp1, inv_scale)),
     ...);
    (add_feq2<Q, T>(F[Q], ring, sm, s0, sp, own, k, nz, utop), ...);
}

// Staged windows of the 16-bit values (k_lb_step_staged): per slot (slot
// order) the TY source rows of its direction (y0 - c_y .. y0 - c_y + TY - 1,
// wrapped) of kWinX values starting 8 cells left of the column
// (x0 - 8 .. x0 + 71, wrapped per 16-byte chunk).
constexpr int kWinX = 80;
constexpr int kWinChunks = kWinX / 8;

// f*neq of direction q that the two cells pull on an interior plane, from
// the window: the cells' sources sit at row ty, values 8 + 2 tx - c_x and
// 9 + 2 tx - c_x of the direction's slot (win already points at row ty,
// value 2 tx).
template <int kMode, int q, int TY>
__device__ __forceinline__ float2 pull_staged(const uint16_t* __restrict__ win, float inv_scale)
{
    const uint16_t* p = win + nslot(q) * TY * kWinX + 8 - cxq(q);
    uint32_t r0, r1;
    if (cxq(q) == 0) {   // an aligned word
        const uint32_t w = *reinterpret_cast<const uint32_t*>(p);
        if constexpr (kMode == PFSI_LB_BF16)
            return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
        r0 = w & 0xffffu;
        r1 = w >> 16;
    } else {
        r0 = p[0];
        r1 = p[1];
    }
    if constexpr (kMode == PFSI_LB_BF16) return make_float2(__uint_as_float(r0 << 16), __uint_as_float(r1 << 16));
    return mul2(make_float2(__half2float(__ushort_as_half((unsigned short)r0)),
                            __half2float(__ushort_as_half((unsigned short)r1))),
                dup2(inv_scale));
}

template <int kMode, class T, int... Q>
__device__ __forceinline__ void pull_all_staged(std::integer_sequence<int, Q...>, float2* F,
                                                const uint16_t* __restrict__ win, float inv_scale,
                                                const Ring<T>& ring, int sm, int s0, int sp, int own, float3 utop)
{
    ((F[Q] = pull_staged<kMode, Q, T::TY>(win, inv_scale)), ...);
    (add_feq2<Q, T>(F[Q], ring, sm, s0, sp, own, 1, 3, utop), ...);   // an interior plane
}

// Stores the two cells' values of one slot (a 32-bit word when kWord).
template <int kMode, bool kWord>
__device__ __forceinline__ void put_pair(typename Neq<kMode>::T* __restrict__ out, int i0, int i1, bool live1,
                                         float2 x, float scale)
{
    uint32_t w;
    if constexpr (kMode == PFSI_LB_BF16) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(x.x, x.y);
        w = *reinterpret_cast<const uint32_t*>(&h);
    } else {
        const float2 y = mul2(x, dup2(scale));
        const __half2 h = __floats2half2_rn(y.x, y.y);
        w = *reinterpret_cast<const uint32_t*>(&h);
    }
    uint16_t* o = reinterpret_cast<uint16_t*>(out);
    if constexpr (kWord) {
        *reinterpret_cast<uint32_t*>(o + i0) = w;
    } else {
        o[i0] = (uint16_t)(w & 0xffffu);
        if (live1) o[i1] = (uint16_t)(w >> 16);
    }
}

// Stored values of the pair (q, opposite of q) of both cells (store_pair).
template <int kMode, bool kWord, int q>
__device__ __forceinline__ void store_pair2(typename Neq<kMode>::T* __restrict__ nout, int N, int base, int i0, int i1,
                                            bool live1, const float2* F, float2 vx, float2 vy, float2 vz, float2 Fx,
                                            float2 Fy, float2 Fz, float2 rk, float2 rh, float2 keep, float2 E0,
                                            float guo, float scale)
{
    if (q == 18 || oppq(q) < q) return;
    const float2 cv = cdot2<q>(vx, vy, vz), cF = cdot2<q>(Fx, Fy, Fz);
    const float2 wcv = mul2(dup2(wq(q)), cv);
    const float2 b = mul2(dup2(wq(q) * guo), cF);
    const float2 odd = fma2(rk, wcv, b);
    const float2 even = fma2(cv, fma2(rh, wcv, b), mul2(dup2(wq(q)), E0));
    put_pair<kMode, kWord>(nout + nslot(q) * N + base, i0, i1, live1, fma2(keep, F[q], add2(even, odd)), scale);
    put_pair<kMode, kWord>(nout + nslot(oppq(q)) * N + base, i0, i1, live1, fma2(keep, F[oppq(q)], sub2(even, odd)),
                           scale);
}

template <int kMode, bool kWord, int... Q>
__device__ __forceinline__ void store_pairs2(std::integer_sequence<int, Q...>, typename Neq<kMode>::T* __restrict__ nout,
                                             int N, int base, int i0, int i1, bool live1, const float2* F, float2 vx,
                                             float2 vy, float2 vz, float2 Fx, float2 Fy, float2 Fz, float2 rk,
                                             float2 rh, float2 keep, float2 E0, float guo, float scale)
{
    (store_pair2<kMode, kWord, Q>(nout, N, base, i0, i1, live1, F, vx, vy, vz, Fx, Fy, Fz, rk, rh, keep, E0, guo,
                                  scale),
     ...);
}

// One plane k of the pair kernel's column (both cells live or the second
// repeating the first); the walls are the planes k = 0 and nz - 1.  (With
// the wall a template argument, one body per kind of plane, the compiler
// hoists the interior body's loads and spills some 700 bytes a thread;
// passed as a wall code computed from k it made the kernel half again
// slower.)  kStaged: an interior plane pulled from the staged window.
template <int kMode, bool kWord, class T, bool kStaged = false>
__device__ __forceinline__ void pair_plane(const Ring<T>& ring, const uint16_t* __restrict__ nin,
                                           typename Neq<kMode>::T* __restrict__ nout, float4* __restrict__ mout,
                                           float4* __restrict__ g, const uint32_t* __restrict__ flags, int N, int nx,
                                           int ny, int k, int j, int ym, int yp, int i0, int i1, bool live1, int xm0,
                                           int xm1, int xp0, int xp1, int own, float omega, float keep, float guo,
                                           float3 F3b, float3 utop, float inv_scale, float scale, int onsite,
                                           int nz, uint32_t row_flag, const uint16_t* __restrict__ win = nullptr)
{
    const int row = k * ny + j;
    const int base = row * nx;   // the cells are base + i0, base + i1
    float2 F[19];
    if constexpr (kStaged)   // an interior plane (wall == 0), pulled from the staged window
        pull_all_staged<kMode, T>(std::make_integer_sequence<int, 19>{}, F, win, inv_scale, ring, (k + 3) & 3, k & 3,
                                  (k + 1) & 3, own, utop);
    else
        pull_all2<kMode, kWord, T>(std::make_integer_sequence<int, 19>{}, F, nin, N, k, nz, nx, ny, j, ym, yp, i0,
                                   i1, xm0, xm1, xp0, xp1, inv_scale, ring, (k + 3) & 3, k & 3, (k + 1) & 3, own,
                                   utop);
    if (onsite && (k == 0 || k == nz - 1)) {
        float fa[19], fb[19];
#pragma unroll
        for (int q = 0; q < 19; ++q) {
            fa[q] = F[q].x;
            fb[q] = F[q].y;
        }
        if (k == 0) {
            onsite_wall<1>(fa, make_float3(0.f, 0.f, 0.f));
            onsite_wall<1>(fb, make_float3(0.f, 0.f, 0.f));
        } else {
            onsite_wall<-1>(fa, utop);
            onsite_wall<-1>(fb, utop);
        }
#pragma unroll
        for (int q = 0; q < 19; ++q) F[q] = make_float2(fa[q], fb[q]);
    }

    // moments per pair of opposite directions (mixed_column's order)
    float2 drho = F[18], mx = dup2(0.f), my = dup2(0.f), mz = dup2(0.f);
#pragma unroll
    for (int q = 0; q < 18; ++q) {
        if (oppq(q) < q) continue;
        const float2 sq = add2(F[q], F[oppq(q)]), d = sub2(F[q], F[oppq(q)]);
        drho = add2(drho, sq);
        if (cxq(q)) mx = cxq(q) > 0 ? add2(mx, d) : sub2(mx, d);
        if (cyq(q)) my = cyq(q) > 0 ? add2(my, d) : sub2(my, d);
        if (czq(q)) mz = czq(q) > 0 ? add2(mz, d) : sub2(mz, d);
    }
    const float2 rho = add2(dup2(1.0f), drho);
    float2 Fx = dup2(F3b.x), Fy = dup2(F3b.y), Fz = dup2(F3b.z);
    const bool forced = row_flag != 0u;   // flags[row], loaded a plane ahead by the caller
    float4 g0, g1;
    if (forced) {
        g0 = g[base + i0];
        g1 = g[base + i1];
        Fx = fma2(dup2(3.0f), make_float2(g0.x, g1.x), Fx);
        Fy = fma2(dup2(3.0f), make_float2(g0.y, g1.y), Fy);
        Fz = fma2(dup2(3.0f), make_float2(g0.z, g1.z), Fz);
    }
    const float2 i3rho = make_float2(__fdividef(3.0f, rho.x), __fdividef(3.0f, rho.y));   // fast division (~2 ulp), as every 16-bit kernel
    const float2 vx = mul2(fma2(Fx, dup2(1.0f / 6.0f), mx), i3rho);
    const float2 vy = mul2(fma2(Fy, dup2(1.0f / 6.0f), my), i3rho);
    const float2 vz = mul2(fma2(Fz, dup2(1.0f / 6.0f), mz), i3rho);
    const float2 VV = fma2(vx, vx, fma2(vy, vy, mul2(vz, vz)));
    const float2 P0 = fma2(mul2(rho, dup2(-1.0f / 6.0f)), VV, drho);
    const float2 vF3 = mul2(fma2(vx, Fx, fma2(vy, Fy, mul2(vz, Fz))), dup2(1.0f / 3.0f));
    const float2 E0 = fma2(dup2(-keep), P0, mul2(dup2(-guo), vF3));
    const float2 rh = mul2(mul2(dup2(0.5f), rho), sub2(dup2(omega), rho));
    const float2 rk = mul2(dup2(-keep), rho);
    put_pair<kMode, kWord>(nout + nslot(18) * N + base, i0, i1, live1,
                           fma2(dup2(keep), F[18], mul2(dup2(wq(18)), E0)), scale);
    store_pairs2<kMode, kWord>(std::make_integer_sequence<int, 18>{}, nout, N, base, i0, i1, live1, F, vx, vy,
                               vz, Fx, Fy, Fz, rk, rh, dup2(keep), E0, guo, scale);
    const float2 third = dup2(1.0f / 3.0f);
    const float2 ux = mul2(vx, third), uy = mul2(vy, third), uz = mul2(vz, third);
    mout[base + i0] = make_float4(ux.x, uy.x, uz.x, drho.x);
    if (live1) mout[base + i1] = make_float4(ux.y, uy.y, uz.y, drho.y);
    if (forced) {
        g[base + i0] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (live1) g[base + i1] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

template <int kMode, bool kWord, class T>
__device__ __forceinline__ void mixed_pair_column(Ring<T>& ring, const uint16_t* __restrict__ nin,
                                                  typename Neq<kMode>::T* __restrict__ nout,
                                                  const float4* __restrict__ min_, float4* __restrict__ mout,
                                                  float4* __restrict__ g, const uint32_t* __restrict__ flags, int nx,
                                                  int ny, int nz, int x0, int y0, int z0, int z1, float omega,
                                                  float guo, float3 body, float3 utop, float inv_scale, int onsite)
{
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int j = y0 + ty;
    const int i0 = x0 + 2 * tx;
    const bool live0 = i0 < nx && j < ny;
    const bool live1 = i0 + 1 < nx && j < ny;
    const int i1 = live1 ? i0 + 1 : i0;   // a missing second cell repeats the first (nothing stored)
    const int N = nx * ny * nz;
    const int plane_cells = nx * ny;
    const int xm0 = (i0 == 0) ? nx - 1 : i0 - 1, xm1 = (i1 == 0) ? nx - 1 : i1 - 1;
    const int xp0 = (i0 >= nx - 1) ? 0 : i0 + 1, xp1 = (i1 >= nx - 1) ? 0 : i1 + 1;
    const int ym = (j == 0) ? ny - 1 : j - 1;
    const int yp = (j >= ny - 1) ? 0 : j + 1;
    const float keep = 1.0f - omega;
    const float scale = 1.0f / inv_scale;
    const int own = (ty + 1) * T::HX + tx;   // ring base of the thread's cells (parity-split rows)

    int off[T::Halo];
#pragma unroll
    for (int u = 0; u < T::Halo; ++u) {
        const int h = threadIdx.x + u * T::Threads;
        const int hy = h / T::HX, hx = h - hy * T::HX;
        int gx = x0 + hx - 1, gy = y0 + hy - 1;
        gx = gx < 0 ? gx + nx : (gx >= nx ? gx % nx : gx);
        gy = gy < 0 ? gy + ny : (gy >= ny ? gy % ny : gy);
        off[u] = h < T::Plane ? gy * nx + gx : -1;
    }

    float4 r[T::Halo];
    for (int p = max(z0 - 1, 0); p <= min(z0 + 1, nz - 1); ++p) {
        halo_load<T>(min_, p, plane_cells, off, r);
        halo_store<T>(ring, p & 3, r);
    }
    __syncthreads();

    const float3 F3b = make_float3(3.0f * body.x, 3.0f * body.y, 3.0f * body.z);
    // the row flag of the next plane is loaded one plane ahead
    uint32_t flag_next = live0 ? flags[z0 * ny + j] : 0u;
    for (int k = z0; k < z1; ++k) {
        const uint32_t flag = flag_next;
        if (live0 && k + 1 < z1) flag_next = flags[(k + 1) * ny + j];
        const bool pre = k + 2 < nz && k + 2 <= z1;
        if (pre) halo_load<T>(min_, k + 2, plane_cells, off, r);
        if (live0)
            pair_plane<kMode, kWord, T>(ring, nin, nout, mout, g, flags, N, nx, ny, k, j, ym, yp, i0, i1, live1, xm0,
                                        xm1, xp0, xp1, own, omega, keep, guo, F3b, utop, inv_scale, scale, onsite,
                                        nz, flag);
        if (pre) halo_store<T>(ring, (k + 2) & 3, r);   // slot of plane k - 2: no longer read
        __syncthreads();
    }
}

// At most 128 registers a thread (two blocks of 256 threads per SM, four of
// 128): unbounded, the compiler takes up to 168 and leaves one block per SM.
template <int kMode, bool kWord, class T>
__global__ void __launch_bounds__(T::Threads, 512 / T::Threads) k_lb_step_pair(
    const uint16_t* __restrict__ nin, typename Neq<kMode>::T* __restrict__ nout, const float4* __restrict__ min_,
    float4* __restrict__ mout, float4* __restrict__ g, const uint32_t* __restrict__ flags, int nx, int ny, int nz,
    int kz, float omega, float guo, float3 body, float3 utop, float inv_scale, int onsite)
{
    pdl_wait();
    __shared__ Ring<T> ring;
    const int z0 = blockIdx.z * kz;
    mixed_pair_column<kMode, kWord, T>(ring, nin, nout, min_, mout, g, flags, nx, ny, nz, blockIdx.x * T::TX,
                                       blockIdx.y * T::TY, z0, min(z0 + kz, nz), omega, guo, body, utop, inv_scale,
                                       onsite);
}

// Staged pair kernel (nx a multiple of 8): the pair kernel's column with the
// 16-bit values of each interior plane copied to shared memory first.  The
// window of plane k + 1 (slots with c_z = 0 from plane k + 1, c_z = +1 from
// k, c_z = -1 from k + 2; each slot the TY rows its direction pulls from) is
// copied with cp.async (16-byte chunks, wrapped periodically per chunk in x
// and per row in y) while plane k computes, so
// the pulls become shared-memory loads at compile-time offsets and the
// per-direction address arithmetic and wall selects of the global pulls go
// away.  The two wall planes take the global pulls (bounce-back).  Every
// lane runs the operation sequence of mixed_column.
template <int TY>
__host__ __device__ constexpr int staged_copies()
{
    return 19 * TY * kWinChunks;
}
template <class T>
__host__ __device__ constexpr size_t staged_smem()
{
    return sizeof(Ring<T>) + 2 * (size_t)staged_copies<T::TY>() * 16;   // ring, two windows
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <int kMode, class T>
__device__ __forceinline__ void mixed_staged_column(char* smem, const uint16_t* __restrict__ nin,
                                                    typename Neq<kMode>::T* __restrict__ nout,
                                                    const float4* __restrict__ min_, float4* __restrict__ mout,
                                                    float4* __restrict__ g, const uint32_t* __restrict__ flags,
                                                    int nx, int ny, int nz, int x0, int y0, int z0, int z1,
                                                    float omega, float guo, float3 body, float3 utop,
                                                    float inv_scale, int onsite)
{
    Ring<T>& ring = *reinterpret_cast<Ring<T>*>(smem);
    uint16_t* winbuf = reinterpret_cast<uint16_t*>(smem + sizeof(Ring<T>));
    constexpr int kCopies = (staged_copies<T::TY>() + T::Threads - 1) / T::Threads;
    constexpr int kWinElems = staged_copies<T::TY>() * 8;   // values per buffer
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int j = y0 + ty;
    const int i0 = x0 + 2 * tx;
    const bool live0 = i0 < nx && j < ny;
    const bool live1 = live0;   // nx even: i0 + 1 < nx whenever i0 < nx
    const int i1 = i0 + 1;
    const int N = nx * ny * nz;
    const int plane_cells = nx * ny;
    const int xm0 = (i0 == 0) ? nx - 1 : i0 - 1, xm1 = i0;
    const int xp0 = i1, xp1 = (i1 >= nx - 1) ? 0 : i1 + 1;
    const int ym = (j == 0) ? ny - 1 : j - 1;
    const int yp = (j >= ny - 1) ? 0 : j + 1;
    const float keep = 1.0f - omega;
    const float scale = 1.0f / inv_scale;
    const int own = (ty + 1) * T::HX + tx;   // ring base of the thread's cells (parity-split rows)

    // this thread's window chunks: value offsets without the plane term
    // (copy u = threadIdx.x + m Threads is slot s, row r, chunk c; the
    // chunks of a buffer are laid out in u order)
    int coff[kCopies];
    const int cx0 = (x0 >> 3) - 1, nchunk = nx >> 3;
#pragma unroll
    for (int m = 0; m < kCopies; ++m) {
        const int u = threadIdx.x + m * T::Threads;
        const int sl = u / (T::TY * kWinChunks), rc = u - sl * T::TY * kWinChunks;
        const int r = rc / kWinChunks, c = rc - r * kWinChunks;
        int cy = 0;   // c_y of the slot's direction
#pragma unroll
        for (int q = 0; q < 19; ++q)
            if (nslot(q) == sl) cy = cyq(q);
        int gy = y0 - cy + r;
        gy = gy < 0 ? gy + ny : (gy >= ny ? gy % ny : gy);
        int gc = cx0 + c;
        gc = gc < 0 ? gc + nchunk : (gc >= nchunk ? gc % nchunk : gc);
        const int dz = sl < 9 ? 0 : (sl < 14 ? -1 : 1);   // slot groups c_z = 0, +1, -1
        coff[m] = u < staged_copies<T::TY>() ? sl * N + dz * plane_cells + gy * nx + gc * 8 : -1;
    }
    // copies of the window of plane kk (interior) into buffer b
    auto stage = [&](int kk, int b) {
        uint16_t* dst = winbuf + b * kWinElems;
#pragma unroll
        for (int m = 0; m < kCopies; ++m)
            if (coff[m] >= 0)
                cp_async16(dst + (threadIdx.x + m * T::Threads) * 8, nin + coff[m] + kk * plane_cells);
        cp_async_commit();
    };
    const bool interior0 = z0 > 0 && z0 < nz - 1;
    if (interior0) stage(z0, z0 & 1);

    int off[T::Halo];
#pragma unroll
    for (int u = 0; u < T::Halo; ++u) {
        const int h = threadIdx.x + u * T::Threads;
        const int hy = h / T::HX, hx = h - hy * T::HX;
        int gx = x0 + hx - 1, gy = y0 + hy - 1;
        gx = gx < 0 ? gx + nx : (gx >= nx ? gx % nx : gx);
        gy = gy < 0 ? gy + ny : (gy >= ny ? gy % ny : gy);
        off[u] = h < T::Plane ? gy * nx + gx : -1;
    }
    float4 r[T::Halo];
    for (int p = max(z0 - 1, 0); p <= min(z0 + 1, nz - 1); ++p) {
        halo_load<T>(min_, p, plane_cells, off, r);
        halo_store<T>(ring, p & 3, r);
    }
    cp_async_wait_all();
    __syncthreads();

    const float3 F3b = make_float3(3.0f * body.x, 3.0f * body.y, 3.0f * body.z);
    // the row flag of the next plane is loaded one plane ahead
    uint32_t flag_next = live0 ? flags[z0 * ny + j] : 0u;
    for (int k = z0; k < z1; ++k) {
        const uint32_t flag = flag_next;
        if (live0 && k + 1 < z1) flag_next = flags[(k + 1) * ny + j];
        // the next plane's window: its buffer was last read by plane k - 1,
        // which every thread has finished (barrier at the end of k - 1)
        if (k + 1 < z1 && k + 1 < nz - 1) stage(k + 1, (k + 1) & 1);
        const bool pre = k + 2 < nz && k + 2 <= z1;
        if (pre) halo_load<T>(min_, k + 2, plane_cells, off, r);
        if (live0) {
            if (k != 0 && k != nz - 1)
                pair_plane<kMode, true, T, true>(ring, nin, nout, mout, g, flags, N, nx, ny, k, j, ym, yp, i0, i1,
                                                 live1, xm0, xm1, xp0, xp1, own, omega, keep, guo, F3b, utop,
                                                 inv_scale, scale, 0, 3, flag,
                                                 winbuf + (k & 1) * kWinElems + ty * kWinX + 2 * tx);
            else
                pair_plane<kMode, true, T>(ring, nin, nout, mout, g, flags, N, nx, ny, k, j, ym, yp, i0, i1, live1,
                                           xm0, xm1, xp0, xp1, own, omega, keep, guo, F3b, utop, inv_scale, scale,
                                           onsite, nz, flag);
        }
        if (pre) halo_store<T>(ring, (k + 2) & 3, r);   // slot of plane k - 2: no longer read
        cp_async_wait_all();   // the next plane's window has landed (this thread's copies)
        __syncthreads();       // ... and everyone's
    }
}

template <int kMode, class T>
__global__ void __launch_bounds__(T::Threads, 512 / T::Threads) k_lb_step_staged(
    const uint16_t* __restrict__ nin, typename Neq<kMode>::T* __restrict__ nout, const float4* __restrict__ min_,
    float4* __restrict__ mout, float4* __restrict__ g, const uint32_t* __restrict__ flags, int nx, int ny, int nz,
    int kz, float omega, float guo, float3 body, float3 utop, float inv_scale, int onsite)
{
    pdl_wait();
    extern __shared__ __align__(16) char staged_sm[];
    const int z0 = blockIdx.z * kz;
    mixed_staged_column<kMode, T>(staged_sm, nin, nout, min_, mout, g, flags, nx, ny, nz, blockIdx.x * T::TX,
                                  blockIdx.y * T::TY, z0, min(z0 + kz, nz), omega, guo, body, utop, inv_scale,
                                  onsite);
}

template <int kMode, int q>
__device__ __forceinline__ void export_q(const typename Neq<kMode>::T* __restrict__ nin, float4 m,
                                         float* __restrict__ fout, int N, int cell, float inv_scale)
{
    fout[q * N + cell] = wq(q) * split_eq<q>(split_record(m)) + Neq<kMode>::get(nin[nslot(q) * N + cell], inv_scale);
}

template <int kMode, int... Q>
__global__ void k_lb_export_mixed(std::integer_sequence<int, Q...>, const typename Neq<kMode>::T* __restrict__ nin,
                                  const float4* __restrict__ min_, float* __restrict__ fout, int N, float inv_scale)
{
    for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < N; cell += gridDim.x * blockDim.x) {
        const float4 m = min_[cell];
        (export_q<kMode, Q>(nin, m, fout, N, cell, inv_scale), ...);
    }
}

// Developed shear profile, post-collision, shifted by w_q; evaluated in FP64.
// onsite: walls on the end layers (profile u_top k/(nz - 1)); otherwise half
// a link outside them (u_top (k + 1/2)/nz).
__global__ void k_lb_init_shear(float* __restrict__ f, int nx, int ny, int nz, double tau,
                                double ux_top, double uy_top, int onsite)
{
    // The profile depends on the height k = blockIdx.y alone: the block's
    // first 19 threads evaluate the plane's populations in FP64 once, then the
    // block streams them to its share of the plane's cells.
    __shared__ float val[19];
    const int N = nx * ny * nz, plane = nx * ny;
    const int k = blockIdx.y;
    if (threadIdx.x < 19) {
        const int q = threadIdx.x;
        const double H = onsite ? (double)(nz - 1) : (double)nz, z0 = onsite ? 0.0 : 0.5;
        const double dux = ux_top / H, duy = uy_top / H;
        const double ux = dux * (k + z0), uy = duy * (k + z0);
        const double uu = ux * ux + uy * uy;
        const double w = q < 6 ? 1.0 / 18.0 : (q < 18 ? 1.0 / 36.0 : 1.0 / 3.0);
        const double cu = cxq(q) * ux + cyq(q) * uy;
        const double feq = w * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
        const double qgrad = (double)czq(q) * (cxq(q) * dux + cyq(q) * duy);
        const double fneq_post = -(tau - 1.0) * w * 3.0 * qgrad;
        val[q] = (float)(feq + fneq_post);
    }
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < plane; i += gridDim.x * blockDim.x) {
        const int cell = k * plane + i;
#pragma unroll
        for (int q = 0; q < 19; ++q) f[q * N + cell] = val[q];
    }
}

// FP64 sums of rho and rho*u of the current state.
__global__ void k_lb_moments(const float* __restrict__ f, int N, double* __restrict__ acc)
{
    double s[4] = {0, 0, 0, 0};
    for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < N; cell += gridDim.x * blockDim.x) {
        double d = 0, mx = 0, my = 0, mz = 0;
#pragma unroll
        for (int q = 0; q < 19; ++q) {
            const double fq = (double)f[q * N + cell];
            d += fq;
            mx += cxq(q) * fq;
            my += cyq(q) * fq;
            mz += czq(q) * fq;
        }
        s[0] += 1.0 + d;
        s[1] += mx;
        s[2] += my;
        s[3] += mz;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        double x = s[c];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(&acc[c], x);
    }
}

// Mixed storage: the same developed profile as (v, 0) and the first-order
// non-equilibrium part, evaluated in FP64.
template <int kMode>
__global__ void k_lb_init_shear_mixed(typename Neq<kMode>::T* __restrict__ nout, float4* __restrict__ mout, int nx,
                                      int ny, int nz, double tau, double ux_top, double uy_top, float inv_scale,
                                      int onsite)
{
    // per plane k = blockIdx.y, as k_lb_init_shear
    __shared__ typename Neq<kMode>::T val[19];
    const int N = nx * ny * nz, plane = nx * ny;
    const int k = blockIdx.y;
    const double H = onsite ? (double)(nz - 1) : (double)nz, z0 = onsite ? 0.0 : 0.5;
    const double dux = ux_top / H, duy = uy_top / H;
    if (threadIdx.x < 19) {
        const int q = threadIdx.x;
        const double w = q < 6 ? 1.0 / 18.0 : (q < 18 ? 1.0 / 36.0 : 1.0 / 3.0);
        const double qgrad = (double)czq(q) * (cxq(q) * dux + cyq(q) * duy);
        val[q] = Neq<kMode>::put((float)(-(tau - 1.0) * w * 3.0 * qgrad), 1.0f / inv_scale);
    }
    const float4 m = make_float4((float)(dux * (k + z0)), (float)(duy * (k + z0)), 0.f, 0.f);
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < plane; i += gridDim.x * blockDim.x) {
        const int cell = k * plane + i;
        mout[cell] = m;
#pragma unroll
        for (int q = 0; q < 19; ++q) nout[nslot(q) * N + cell] = val[q];
    }
}

// FP64 sums of rho and rho*u of the current mixed state, from the rebuilt
// post-collision populations.
template <int kMode>
__global__ void k_lb_moments_mixed(const typename Neq<kMode>::T* __restrict__ nin, const float4* __restrict__ min_,
                                   int N, double* __restrict__ acc, float inv_scale)
{
    double s[4] = {0, 0, 0, 0};
    for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < N; cell += gridDim.x * blockDim.x) {
        const float4 m = min_[cell];
        const double vx = m.x, vy = m.y, vz = m.z, d = m.w;
        const double vv = vx * vx + vy * vy + vz * vz;
        double sd = 0, mx = 0, my = 0, mz = 0;
#pragma unroll
        for (int q = 0; q < 19; ++q) {
            // E_q of the split (pfsi_internal.cuh) in FP64: P + c.J + (c.J)^2 / 2
            const double w = q < 6 ? 1.0 / 18.0 : (q < 18 ? 1.0 / 36.0 : 1.0 / 3.0);
            const double cj = 3.0 * (1.0 + d) * (cxq(q) * vx + cyq(q) * vy + czq(q) * vz);
            const double fq = w * (d - 1.5 * (1.0 + d) * vv + cj + 0.5 * cj * cj) +
                              (double)Neq<kMode>::get(nin[nslot(q) * N + cell], inv_scale);
            sd += fq;
            mx += cxq(q) * fq;
            my += cyq(q) * fq;
            mz += czq(q) * fq;
        }
        s[0] += 1.0 + sd;
        s[1] += mx;
        s[2] += my;
        s[3] += mz;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        double x = s[c];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(&acc[c], x);
    }
}

float inv_scale_of(const lb_params& p) { return p.storage == PFSI_LB_FP16 ? ldexpf(1.0f, -p.fp16_exponent) : 1.0f; }

template <int kMode>
using NeqT = typename Neq<kMode>::T;

// Launch shapes (chosen by lb_set_shape / lb_autotune): FP32, threads per
// block along x; mixed storage, the (x, y) column tile of the marching kernel.
constexpr int kFp32Block[PFSI_LB_SHAPES] = {kRowBlock, 32, 64, 256};

template <int kMode, class T>
cudaError_t launch_mixed(LbCtx* c, cudaStream_t s, float omega, float guo, float3 body, float3 utop, float inv_scale)
{
    const lb_params& p = c->p;
    const int a = c->cur, b = c->cur ^ 1;
    // columns march through kz planes; kz is picked so that the grid has
    // about eight blocks of 256 threads per SM (fewer halo planes per cell on
    // large grids, enough blocks on small ones)
    const int tiles = ((p.nx + T::TX - 1) / T::TX) * ((p.ny + T::TY - 1) / T::TY);
    const long long want = 148LL * 8 * 256 / T::Threads;
    const int kz = (int)std::min<long long>(32, std::max<long long>(2, ((long long)tiles * p.nz + want - 1) / want));
    const dim3 grid((p.nx + T::TX - 1) / T::TX, (p.ny + T::TY - 1) / T::TY, (p.nz + kz - 1) / kz);
    return launch_pdl(k_lb_step_mixed<kMode, T>, grid, dim3(T::Threads), 0, s, (const uint16_t*)c->f[a],
                      (NeqT<kMode>*)c->f[b], (const float4*)c->m[a], c->m[b], c->g, (const uint32_t*)c->flags, p.nx, p.ny,
                      p.nz, kz, omega, guo, body, utop, inv_scale, p.walls);
}

template <int kMode, class T>
cudaError_t launch_pair(LbCtx* c, cudaStream_t s, float omega, float guo, float3 body, float3 utop, float inv_scale)
{
    const lb_params& p = c->p;
    const int a = c->cur, b = c->cur ^ 1;
    const int tiles = ((p.nx + T::TX - 1) / T::TX) * ((p.ny + T::TY - 1) / T::TY);
    const long long want = 148LL * 8 * 256 / T::Threads;
    const int kz = (int)std::min<long long>(32, std::max<long long>(2, ((long long)tiles * p.nz + want - 1) / want));
    const dim3 grid((p.nx + T::TX - 1) / T::TX, (p.ny + T::TY - 1) / T::TY, (p.nz + kz - 1) / kz);
    auto kernel = p.nx % 2 == 0 ? k_lb_step_pair<kMode, true, T> : k_lb_step_pair<kMode, false, T>;
    return launch_pdl(kernel, grid, dim3(T::Threads), 0, s, (const uint16_t*)c->f[a], (NeqT<kMode>*)c->f[b],
                      (const float4*)c->m[a], c->m[b], c->g, (const uint32_t*)c->flags, p.nx, p.ny, p.nz, kz, omega,
                      guo, body, utop, inv_scale, p.walls);
}

template <int kMode, class T>
cudaError_t launch_staged(LbCtx* c, cudaStream_t s, float omega, float guo, float3 body, float3 utop, float inv_scale)
{
    const lb_params& p = c->p;
    const int a = c->cur, b = c->cur ^ 1;
    const int tiles = ((p.nx + T::TX - 1) / T::TX) * ((p.ny + T::TY - 1) / T::TY);
    const long long want = 148LL * 8 * 256 / T::Threads;
    const int kz = (int)std::min<long long>(32, std::max<long long>(2, ((long long)tiles * p.nz + want - 1) / want));
    const dim3 grid((p.nx + T::TX - 1) / T::TX, (p.ny + T::TY - 1) / T::TY, (p.nz + kz - 1) / kz);
    return launch_pdl(k_lb_step_staged<kMode, T>, grid, dim3(T::Threads), staged_smem<T>(), s,
                      (const uint16_t*)c->f[a], (NeqT<kMode>*)c->f[b], (const float4*)c->m[a], c->m[b], c->g,
                      (const uint32_t*)c->flags, p.nx, p.ny, p.nz, kz, omega, guo, body, utop, inv_scale, p.walls);
}

// The staged kernels' dynamic shared memory limit (above the 48 KB default),
// set for the current device when a mixed-storage context is created.
int staged_prepare()
{
    int rc = check_cuda(cudaFuncSetAttribute(k_lb_step_staged<PFSI_LB_BF16, PairTile<4>>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)staged_smem<PairTile<4>>()),
                        "lb: staged kernel shared memory");
    if (!rc)
        rc = check_cuda(cudaFuncSetAttribute(k_lb_step_staged<PFSI_LB_FP16, PairTile<4>>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)staged_smem<PairTile<4>>()),
                        "lb: staged kernel shared memory");
    return rc;
}

template <int kMode>
cudaError_t launch_mixed_shape(LbCtx* c, cudaStream_t s, float omega, float guo, float3 body, float3 utop,
                               float inv_scale)
{
    // nx a multiple of 8: shape 0 the staged pair kernel (64 x 4 columns),
    // 1 the pair kernel (64 x 4), 2 the one-cell kernel (32 x 8), 3 the
    // TMA-staged kernel (32 x 8) where its tensor maps exist, else the
    // one-cell kernel (32 x 4).  Otherwise: 0, 1 the pair kernel (64 x 4,
    // 64 x 8), 2, 3 the one-cell kernel (32 x 8, 32 x 4).
    const bool staged = c->p.nx % 8 == 0;
    switch (c->shape) {
    case 0:
        if (staged) return launch_staged<kMode, PairTile<4>>(c, s, omega, guo, body, utop, inv_scale);
        return launch_pair<kMode, PairTile<4>>(c, s, omega, guo, body, utop, inv_scale);
    case 1:
        if (staged) return launch_pair<kMode, PairTile<4>>(c, s, omega, guo, body, utop, inv_scale);
        return launch_pair<kMode, PairTile<8>>(c, s, omega, guo, body, utop, inv_scale);
    case 2: return launch_mixed<kMode, Tile<32, 8>>(c, s, omega, guo, body, utop, inv_scale);
    default:
        if (c->tma) return lb_tma_launch(c, c->tma, 0, s, omega, guo, body, utop, inv_scale);
        return launch_mixed<kMode, Tile<32, 4>>(c, s, omega, guo, body, utop, inv_scale);
    }
}

// ---------------------------------------------------------------------------
// Batched step: one launch per storage kind steps every chamber of a batch.
// The chambers' cells are cut into tiles listed chamber after chamber; a
// persistent grid (as many blocks as fit on the GPU at once) walks the list,
// block b taking tiles b, b + grid, b + 2 grid, ...  Each tile is computed by
// the same per-cell code as the single-chamber kernels, so a chamber stepped
// in a batch gets bit-identical populations.  The list travels as a kernel
// parameter (__grid_constant__): its block-uniform fields are read from the
// constant bank as the single-chamber kernels read theirs, instead of
// occupying registers.

// Tile list entry of one chamber: its buffers for one lattice-buffer parity,
// its parameters and its place in the list.
struct LbChamber {
    const void* fin;       // populations read (FP32 shifted f, or 16-bit f*neq)
    void* fout;            // populations written
    const float4* min;     // mixed: moment records read
    float4* mout;          // mixed: moment records written; FP32: (v, rho) of the forced rows
    float4* g;
    const uint32_t* flags;
    float3 body, utop;
    float omega, guo, inv_scale;
    int nx, ny, nz, onsite;
    int tile0;             // first tile of the chamber in the list
    int shape;             // mixed: column tile (kBatchTX x kBatchTY)
    int tiles_x, tiles_y;  // mixed: columns along x and along y
    int kz;                // mixed: planes per column
};

// Chambers per launch: a kind with more chambers takes several launches.
constexpr int kTableMax = 128;

struct LbTable {
    int n, ntiles;
    LbChamber ch[kTableMax];
};
static_assert(sizeof(LbTable) <= 32000, "the tile list must fit the kernel parameter space");

constexpr int kBatchThreads = 256;                 // FP32 blocks
constexpr int kBatchFp32Tile = kBatchThreads;      // FP32: consecutive cells (flat order) per tile
constexpr int kBatchMixedThreads = 128;            // mixed-storage blocks
// mixed column tiles of 128 threads: the pair kernel's 64 x 4 (two cells a
// thread), the one-cell kernel's 32 x 4 and 16 x 8
constexpr int kBatchShapes = 3;
constexpr int kBatchTX[kBatchShapes] = {64, 32, 16};
constexpr int kBatchTY[kBatchShapes] = {4, 4, 8};
constexpr int kBatchKz = 16;                        // mixed: planes per column
constexpr int kBatchPlane = 66 * 6;                 // largest ring plane of the three shapes (64 x 4)
static_assert(PairTile<4>::Plane <= kBatchPlane && Tile<32, 4>::Plane <= kBatchPlane &&
                  Tile<16, 8>::Plane <= kBatchPlane && PairTile<4>::Threads == kBatchMixedThreads &&
                  Tile<32, 4>::Threads == kBatchMixedThreads && Tile<16, 8>::Threads == kBatchMixedThreads,
              "ring storage must hold every shape's plane; every shape takes the block");

// Chamber of tile t: the list is sorted by tile0 and a block's tiles only
// grow, so the search moves forward from the previous tile's chamber.
__device__ __forceinline__ int chamber_of(const LbTable& tab, int t, int c)
{
    while (c + 1 < tab.n && tab.ch[c + 1].tile0 <= t) ++c;
    return c;
}

__global__ void __launch_bounds__(kBatchThreads) k_lb_step_batch(const __grid_constant__ LbTable tab)
{
    int c = 0;
    for (int t = blockIdx.x; t < tab.ntiles; t += gridDim.x) {
        c = chamber_of(tab, t, c);
        const LbChamber& ch = tab.ch[c];
        const int nx = ch.nx, plane = nx * ch.ny;
        const int cell = (t - ch.tile0) * kBatchFp32Tile + (int)threadIdx.x;
        if (cell >= plane * ch.nz) continue;
        const int k = cell / plane, r = cell - k * plane;
        const int j = r / nx, i = r - j * nx;
        fp32_cell((const float*)ch.fin, (float*)ch.fout, ch.g, ch.mout, ch.flags, nx, ch.ny, ch.nz, i, j, k,
                  ch.omega, ch.guo, ch.body, ch.utop, ch.onsite);
    }
}

template <int kMode, int S>
__device__ __forceinline__ void batch_column(float4* ring_mem, const LbChamber& ch, int tx, int ty, int z0)
{
    const int z1 = min(z0 + ch.kz, ch.nz);
    if constexpr (S == 0) {
        using T = PairTile<4>;
        auto& ring = *reinterpret_cast<Ring<T>*>(ring_mem);
        if (ch.nx % 2 == 0)
            mixed_pair_column<kMode, true, T>(ring, (const uint16_t*)ch.fin, (typename Neq<kMode>::T*)ch.fout, ch.min,
                                              ch.mout, ch.g, ch.flags, ch.nx, ch.ny, ch.nz, tx * T::TX, ty * T::TY,
                                              z0, z1, ch.omega, ch.guo, ch.body, ch.utop, ch.inv_scale, ch.onsite);
        else
            mixed_pair_column<kMode, false, T>(ring, (const uint16_t*)ch.fin, (typename Neq<kMode>::T*)ch.fout,
                                               ch.min, ch.mout, ch.g, ch.flags, ch.nx, ch.ny, ch.nz, tx * T::TX,
                                               ty * T::TY, z0, z1, ch.omega, ch.guo, ch.body, ch.utop, ch.inv_scale,
                                               ch.onsite);
    } else {
        using T = Tile<kBatchTX[S], kBatchTY[S]>;
        mixed_column<kMode, T>(*reinterpret_cast<Ring<T>*>(ring_mem), (const uint16_t*)ch.fin,
                               (typename Neq<kMode>::T*)ch.fout, ch.min, ch.mout, ch.g, ch.flags, ch.nx, ch.ny, ch.nz,
                               tx * T::TX, ty * T::TY, z0, z1, ch.omega, ch.guo, ch.body, ch.utop, ch.inv_scale,
                               ch.onsite);
    }
}

// At most 128 registers (four blocks of 128 threads per SM), the pair
// kernel's budget.
template <int kMode>
__global__ void __launch_bounds__(kBatchMixedThreads, 4) k_lb_step_batch_mixed(const __grid_constant__ LbTable tab)
{
    __shared__ float4 ring_mem[kSlots * kBatchPlane];
    int c = 0;
    for (int t = blockIdx.x; t < tab.ntiles; t += gridDim.x) {
        c = chamber_of(tab, t, c);
        const LbChamber& ch = tab.ch[c];
        // tiles of a chamber: x fastest, then y, then the column's plane range
        const int u = t - ch.tile0, per_range = ch.tiles_x * ch.tiles_y;
        const int tz = u / per_range, r = u - tz * per_range;
        const int ty = r / ch.tiles_x, tx = r - ty * ch.tiles_x;
        switch (ch.shape) {   // uniform over the block
        case 1: batch_column<kMode, 1>(ring_mem, ch, tx, ty, tz * ch.kz); break;
        case 2: batch_column<kMode, 2>(ring_mem, ch, tx, ty, tz * ch.kz); break;
        default: batch_column<kMode, 0>(ring_mem, ch, tx, ty, tz * ch.kz);
        }
    }
}

}  // namespace

int launch_lb_step(LbCtx* c, cudaStream_t s)
{
    const lb_params& p = c->p;
    const float omega = 1.0f / p.tau;
    const float guo = 1.0f - 0.5f / p.tau;
    const float3 body = make_float3(p.body[0], p.body[1], p.body[2]);
    const float3 utop = make_float3(p.u_top[0], p.u_top[1], p.u_top[2]);
    switch (p.storage) {
    case PFSI_LB_BF16: {
        const int rc = check_cuda(launch_mixed_shape<PFSI_LB_BF16>(c, s, omega, guo, body, utop, 1.0f), "lb_step");
        if (rc) return rc;
        break;
    }
    case PFSI_LB_FP16: {
        const int rc = check_cuda(launch_mixed_shape<PFSI_LB_FP16>(c, s, omega, guo, body, utop, inv_scale_of(p)),
                                  "lb_step");
        if (rc) return rc;
        break;
    }
    default: {
        const int want = kFp32Block[c->shape];
        const int cap = ((p.nx + 31) / 32) * 32;
        const int bx = want < cap ? want : cap;
        const dim3 grid((p.nx + bx - 1) / bx, p.ny, p.nz);
        const int rc = check_cuda(launch_pdl(k_lb_step, grid, dim3(bx), 0, s, (const float*)c->f[c->cur],
                                             (float*)c->f[c->cur ^ 1], c->g, c->v, (const uint32_t*)c->flags, p.nx, p.ny,
                                             p.nz, omega, guo, body, utop, p.walls),
                                  "lb_step");
        if (rc) return rc;
    }
    }
    c->cur ^= 1;
    return check_launch("lb_step");
}

// Host side of a batch: per storage kind, the tile lists of its chambers for
// each lattice-buffer parity (one list per launch of up to kTableMax
// chambers).
struct LbBatch {
    std::vector<LbCtx*> lat;
    struct Kind {
        std::vector<int> members;          // indices into lat, in list order
        std::vector<int> shapes;           // mixed: column shape per member
        std::vector<LbTable> tab[2];       // per parity of the buffers read
        int sms = 0, per_sm = 0;           // SMs, resident blocks of the kernel per SM
        int tuned = 0;                     // blocks per SM the autotuner picked (0: none)
        int grid = 0;                      // blocks of the persistent grid
    } kind[3];                             // PFSI_LB_FP32, PFSI_LB_BF16, PFSI_LB_FP16
    int blocks_per_sm = 0;                 // grid: this many blocks per SM (0: every resident block)
    int priority = 0;                      // launch priority (cudaLaunchAttributePriority)
};

namespace {

// Columns of a mixed chamber for a batch shape, and the shape the batch
// starts from before tuning: the least work per chamber counting idle cells
// in ragged columns (a pair-kernel thread takes two) and a quarter of a
// cell per ring record.
long long batch_cost(const lb_params& p, int shape)
{
    const long long tx = (p.nx + kBatchTX[shape] - 1) / kBatchTX[shape];
    const long long ty = (p.ny + kBatchTY[shape] - 1) / kBatchTY[shape];
    return tx * ty * (4 * kBatchMixedThreads * (shape == 0 ? 2 : 1) + (kBatchTX[shape] + 2) * (kBatchTY[shape] + 2));
}

int batch_default_shape(const lb_params& p)
{
    int best = 0;
    for (int s = 1; s < kBatchShapes; ++s)
        if (batch_cost(p, s) < batch_cost(p, best)) best = s;
    return best;
}

LbChamber chamber_entry(const LbCtx* c, int parity, int shape)
{
    const lb_params& p = c->p;
    LbChamber e = {};
    e.fin = c->f[parity];
    e.fout = c->f[parity ^ 1];
    e.min = p.storage ? c->m[parity] : nullptr;
    e.mout = p.storage ? c->m[parity ^ 1] : c->v;
    e.g = c->g;
    e.flags = c->flags;
    e.body = make_float3(p.body[0], p.body[1], p.body[2]);
    e.utop = make_float3(p.u_top[0], p.u_top[1], p.u_top[2]);
    e.omega = 1.0f / p.tau;
    e.guo = 1.0f - 0.5f / p.tau;
    e.inv_scale = inv_scale_of(p);
    e.nx = p.nx;
    e.ny = p.ny;
    e.nz = p.nz;
    e.onsite = p.walls;
    e.shape = shape;
    if (p.storage) {
        e.tiles_x = (p.nx + kBatchTX[shape] - 1) / kBatchTX[shape];
        e.tiles_y = (p.ny + kBatchTY[shape] - 1) / kBatchTY[shape];
        e.kz = std::min(kBatchKz, p.nz);
    }
    return e;
}

long long chamber_tiles(const LbChamber& e, int mode)
{
    if (mode == PFSI_LB_FP32) return ((long long)e.nx * e.ny * e.nz + kBatchFp32Tile - 1) / kBatchFp32Tile;
    return (long long)e.tiles_x * e.tiles_y * ((e.nz + e.kz - 1) / e.kz);
}

// Rebuilds both parities' lists of one kind from the chambers' shapes.
int batch_upload(LbBatch* b, int mode, const std::vector<int>& shapes)
{
    LbBatch::Kind& K = b->kind[mode];
    K.shapes = shapes;
    for (int par = 0; par < 2; ++par) {
        K.tab[par].clear();
        for (size_t u = 0; u < K.members.size(); ++u) {
            if (u % kTableMax == 0) {
                K.tab[par].emplace_back();
                K.tab[par].back().n = 0;
                K.tab[par].back().ntiles = 0;
            }
            LbTable& T = K.tab[par].back();
            LbChamber e = chamber_entry(b->lat[K.members[u]], par, shapes[u]);
            e.tile0 = T.ntiles;
            const long long tiles = (long long)T.ntiles + chamber_tiles(e, mode);
            if (tiles > INT_MAX) return set_error(PFSI_ERR_ARG, "lb_batch: too many tiles for one launch");
            T.ch[T.n++] = e;
            T.ntiles = (int)tiles;
        }
    }
    return PFSI_OK;
}

template <typename K>
int resident_blocks(K kernel, int threads, LbBatch::Kind& kind)
{
    int dev = 0;
    int rc = check_cuda(cudaGetDevice(&dev), "lb_batch: device");
    if (!rc) rc = check_cuda(cudaDeviceGetAttribute(&kind.sms, cudaDevAttrMultiProcessorCount, dev), "lb_batch: SMs");
    if (!rc)
        rc = check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&kind.per_sm, kernel, threads, 0),
                        "lb_batch: occupancy");
    kind.per_sm = std::max(kind.per_sm, 1);
    return rc;
}

void size_grids(LbBatch* b)
{
    for (auto& K : b->kind) {
        const int want = K.tuned > 0 ? K.tuned : b->blocks_per_sm;
        K.grid = K.sms * (want > 0 ? std::min(want, K.per_sm) : K.per_sm);
    }
}

// One launch of kind `mode` over the list `tab` (no parity flip), at the
// batch's launch priority.
cudaError_t batch_launch_kind(const LbBatch* b, const LbBatch::Kind& K, int mode, const LbTable& tab,
                              cudaStream_t s)
{
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributePriority;
    attr[0].val.priority = b->priority;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(std::max(1, std::min(K.grid, tab.ntiles)));
    cfg.blockDim = dim3(mode == PFSI_LB_FP32 ? kBatchThreads : kBatchMixedThreads);
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    switch (mode) {
    case PFSI_LB_BF16: return cudaLaunchKernelEx(&cfg, k_lb_step_batch_mixed<PFSI_LB_BF16>, tab);
    case PFSI_LB_FP16: return cudaLaunchKernelEx(&cfg, k_lb_step_batch_mixed<PFSI_LB_FP16>, tab);
    default: return cudaLaunchKernelEx(&cfg, k_lb_step_batch, tab);
    }
}

}  // namespace

void lb_batch_free(LbBatch* b) { delete b; }

int lb_batch_build(LbCtx* const* lat, int n, LbBatch** out)
{
    if (!lat || n < 1 || !out) return set_error(PFSI_ERR_ARG, "lb_batch: bad argument");
    for (int i = 0; i < n; ++i) {
        if (!lat[i]) return set_error(PFSI_ERR_ARG, "lb_batch: null lattice");
        if (lat[i]->cur != lat[0]->cur)
            return set_error(PFSI_ERR_ARG, "lb_batch: lattices must be at the same buffer parity");
        for (int j = 0; j < i; ++j)
            if (lat[j] == lat[i]) return set_error(PFSI_ERR_ARG, "lb_batch: a lattice appears twice");
    }
    LbBatch* b = new LbBatch();
    b->lat.assign(lat, lat + n);
    int rc = PFSI_OK;
    for (int mode = 0; mode < 3 && !rc; ++mode) {
        LbBatch::Kind& K = b->kind[mode];
        std::vector<int> shapes;
        for (int i = 0; i < n; ++i)
            if (lat[i]->p.storage == mode) {
                K.members.push_back(i);
                shapes.push_back(mode ? batch_default_shape(lat[i]->p) : 0);
            }
        if (K.members.empty()) continue;
        rc = batch_upload(b, mode, shapes);
        if (!rc)
            rc = mode == PFSI_LB_BF16   ? resident_blocks(k_lb_step_batch_mixed<PFSI_LB_BF16>, kBatchMixedThreads, K)
                 : mode == PFSI_LB_FP16 ? resident_blocks(k_lb_step_batch_mixed<PFSI_LB_FP16>, kBatchMixedThreads, K)
                                        : resident_blocks(k_lb_step_batch, kBatchThreads, K);
    }
    size_grids(b);
    if (rc) {
        lb_batch_free(b);
        return rc;
    }
    *out = b;
    return PFSI_OK;
}

int launch_lb_batch(LbBatch* b, cudaStream_t s)
{
    const int parity = b->lat[0]->cur;
    for (const LbCtx* c : b->lat)
        if (c->cur != parity) return set_error(PFSI_ERR_ARG, "lb_batch: lattices are at different buffer parities");
    for (int mode = 0; mode < 3; ++mode)
        for (const LbTable& T : b->kind[mode].tab[parity]) {
            const int rc = check_cuda(batch_launch_kind(b, b->kind[mode], mode, T, s), "lb_batch: launch");
            if (rc) return rc;
        }
    for (LbCtx* c : b->lat) c->cur ^= 1;
    return PFSI_OK;
}

// Per mixed chamber, times each column shape on that chamber alone and
// keeps the fastest; then, per storage kind, times the batched launch with
// 1 .. (resident blocks) blocks per SM and keeps the fastest grid.  The launches read
// the current buffers and write the others without taking the parity
// forward, so the state is unchanged provided no spread force is pending
// (g is zero between coupled steps: the step that consumes it clears it).
int lb_batch_tune(LbBatch* b, int reps, cudaStream_t s, float* ms_out)
{
    if (!b || reps < 1) return set_error(PFSI_ERR_ARG, "lb_batch_tune: bad argument");
    const int parity = b->lat[0]->cur;
    for (const LbCtx* c : b->lat)
        if (c->cur != parity) return set_error(PFSI_ERR_ARG, "lb_batch: lattices are at different buffer parities");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = check_cuda(cudaEventCreate(&e0), "lb_batch_tune: event");
    if (!rc) rc = check_cuda(cudaEventCreate(&e1), "lb_batch_tune: event");
    // mean time of `reps` launches of the lists after one warm-up
    auto time_launches = [&](const LbBatch::Kind& K, int mode, const std::vector<LbTable>& tabs, float* ms) {
        int r = PFSI_OK;
        for (const LbTable& T : tabs)
            if (!r) r = check_cuda(batch_launch_kind(b, K, mode, T, s), "lb_batch_tune: launch");
        if (!r) r = check_cuda(cudaEventRecord(e0, s), "lb_batch_tune: record");
        for (int k = 0; k < reps && !r; ++k)
            for (const LbTable& T : tabs)
                if (!r) r = check_cuda(batch_launch_kind(b, K, mode, T, s), "lb_batch_tune: launch");
        if (!r) r = check_cuda(cudaEventRecord(e1, s), "lb_batch_tune: record");
        if (!r) r = check_cuda(cudaEventSynchronize(e1), "lb_batch_tune: synchronise");
        if (!r) r = check_cuda(cudaEventElapsedTime(ms, e0, e1), "lb_batch_tune: elapsed");
        *ms /= reps;
        return r;
    };
    std::vector<LbTable> one(1);
    for (int mode = 1; mode < 3 && !rc; ++mode) {
        LbBatch::Kind& K = b->kind[mode];
        std::vector<int> shapes;
        for (size_t u = 0; u < K.members.size() && !rc; ++u) {
            const LbCtx* c = b->lat[K.members[u]];
            int best = 0;
            float best_ms = 0.f;
            for (int shape = 0; shape < kBatchShapes && !rc; ++shape) {
                LbChamber e = chamber_entry(c, parity, shape);
                e.tile0 = 0;
                one[0].n = 1;
                one[0].ntiles = (int)chamber_tiles(e, mode);
                one[0].ch[0] = e;
                float ms = 0.f;
                rc = time_launches(K, mode, one, &ms);
                if (!rc && (shape == 0 || ms < best_ms)) {
                    best = shape;
                    best_ms = ms;
                }
            }
            shapes.push_back(best);
        }
        if (!rc && !K.members.empty()) rc = batch_upload(b, mode, shapes);
    }
    // then the grid of each kind: 1 .. resident blocks per SM
    float total = 0.f;
    for (int mode = 0; mode < 3 && !rc; ++mode) {
        LbBatch::Kind& K = b->kind[mode];
        if (K.members.empty()) continue;
        int best = 0;
        float best_ms = 0.f;
        for (int per = K.per_sm; per >= 1 && !rc; --per) {
            K.tuned = per;
            size_grids(b);
            float ms = 0.f;
            rc = time_launches(K, mode, K.tab[parity], &ms);
            if (!rc && (best == 0 || ms < best_ms)) {
                best = per;
                best_ms = ms;
            }
        }
        K.tuned = best;
        size_grids(b);
        total += best_ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (!rc && ms_out) *ms_out = total;
    return rc;
}

int lb_batch_assign_shapes(LbBatch* b, const int* shapes)
{
    for (size_t i = 0; i < b->lat.size(); ++i)
        if (b->lat[i]->p.storage && (shapes[i] < 0 || shapes[i] >= kBatchShapes))
            return set_error(PFSI_ERR_ARG, "lb_batch_set_shapes: shape out of range");
    for (int mode = 1; mode < 3; ++mode) {
        const LbBatch::Kind& K = b->kind[mode];
        if (K.members.empty()) continue;
        std::vector<int> s;
        for (int i : K.members) s.push_back(shapes[i]);
        const int rc = batch_upload(b, mode, s);
        if (rc) return rc;
    }
    return PFSI_OK;
}

int lb_batch_configure_grid(LbBatch* b, int blocks_per_sm, int priority)
{
    if (blocks_per_sm < 0) return set_error(PFSI_ERR_ARG, "lb_batch_set_grid: negative blocks per SM");
    b->blocks_per_sm = blocks_per_sm;
    b->priority = priority;
    for (auto& K : b->kind) K.tuned = 0;
    size_grids(b);
    return PFSI_OK;
}

int lb_batch_shapes(const LbBatch* b, int* shapes)
{
    for (size_t i = 0; i < b->lat.size(); ++i) shapes[i] = -1;
    for (int mode = 1; mode < 3; ++mode) {
        const LbBatch::Kind& K = b->kind[mode];
        for (size_t u = 0; u < K.members.size(); ++u) shapes[K.members[u]] = K.shapes[u];
    }
    return PFSI_OK;
}

}  // namespace pfsi

using namespace pfsi;

extern "C" int lb_query_sizes(const lb_params* p, lb_sizes* out)
{
    if (!p || !out) return set_error(PFSI_ERR_ARG, "lb_query_sizes: null argument");
    if (p->nx < 1 || p->ny < 1 || p->nz < 2)
        return set_error(PFSI_ERR_ARG, "lb_query_sizes: need nx, ny >= 1 and nz >= 2");
    const long long N = (long long)p->nx * p->ny * p->nz;
    if (N * 19 > (long long)INT_MAX)
        return set_error(PFSI_ERR_ARG, "lb_query_sizes: grid too large (19 * cells must fit in int32)");
    if (p->storage != PFSI_LB_FP32 && p->storage != PFSI_LB_BF16 && p->storage != PFSI_LB_FP16)
        return set_error(PFSI_ERR_ARG, "lb_query_sizes: unknown storage mode");
    if (p->storage == PFSI_LB_FP16 && (p->fp16_exponent < -60 || p->fp16_exponent > 60))
        return set_error(PFSI_ERR_ARG, "lb_query_sizes: fp16_exponent outside -60..60");
    if (p->walls != PFSI_WALLS_BOUNCEBACK && p->walls != PFSI_WALLS_ONSITE)
        return set_error(PFSI_ERR_ARG, "lb_query_sizes: unknown wall mode");
    out->n_cells = N;
    out->f_bytes = (size_t)N * 19 * (p->storage == PFSI_LB_FP32 ? sizeof(float) : sizeof(uint16_t));
    out->g_bytes = (size_t)N * sizeof(float4);
    out->v_bytes = (size_t)N * sizeof(float4);
    out->flag_bytes = (size_t)p->ny * p->nz * sizeof(uint32_t);
    return PFSI_OK;
}

namespace {

int create_common(const char* who, const lb_params* p, void* f_a, void* f_b, float* m_a, float* m_b, float* g,
                  float* v, uint32_t* row_flags, lb_ctx** out)
{
    lb_sizes sz;
    int rc = lb_query_sizes(p, &sz);
    if (rc) return rc;
    if (!(p->tau > 0.5f)) return set_error(PFSI_ERR_ARG, std::string(who) + ": tau must exceed 1/2");
    if (p->u_top[2] != 0.0f) return set_error(PFSI_ERR_ARG, std::string(who) + ": the top wall cannot move along z");
    if (!aligned(f_a, 16) || !aligned(f_b, 16) || !aligned(g, 16) || !aligned(v, 16) || !aligned(m_a, 16) ||
        !aligned(m_b, 16) || !aligned(row_flags, 4))
        return set_error(PFSI_ERR_ARG, std::string(who) + ": buffers must be 16-byte aligned");
    rc = ib_prepare();
    if (!rc && p->storage != PFSI_LB_FP32) rc = staged_prepare();
    if (rc) return rc;
    lb_ctx* c = new lb_ctx();
    c->p = *p;
    c->N = sz.n_cells;
    c->f[0] = f_a;
    c->f[1] = f_b;
    c->cur = 0;
    c->g = reinterpret_cast<float4*>(g);
    c->v = reinterpret_cast<float4*>(v);
    c->m[0] = reinterpret_cast<float4*>(m_a);
    c->m[1] = reinterpret_cast<float4*>(m_b);
    c->flags = row_flags;
    c->tma = nullptr;
    if (p->storage != PFSI_LB_FP32) c->tma = lb_tma_create(c);
    rc = check_cuda(cudaMemsetAsync(c->g, 0, sz.g_bytes, 0), "lb_create: clear g");
    if (!rc) rc = check_cuda(cudaMemsetAsync(c->flags, 0, sz.flag_bytes, 0), "lb_create: clear flags");
    if (!rc) rc = check_cuda(cudaStreamSynchronize(0), "lb_create: synchronise");
    if (rc) {
        lb_tma_destroy(c->tma);
        delete c;
        return rc;
    }
    *out = c;
    return PFSI_OK;
}

}  // namespace

extern "C" int lb_create(const lb_params* p, float* f_a, float* f_b, float* g, float* v,
                         uint32_t* row_flags, lb_ctx** out)
{
    if (!p || !out || !f_a || !f_b || !g || !v || !row_flags)
        return set_error(PFSI_ERR_ARG, "lb_create: null argument");
    if (p->storage != PFSI_LB_FP32) return set_error(PFSI_ERR_ARG, "lb_create: storage must be PFSI_LB_FP32");
    return create_common("lb_create", p, f_a, f_b, nullptr, nullptr, g, v, row_flags, out);
}

extern "C" int lb_create_mixed(const lb_params* p, void* fneq_a, void* fneq_b, float* m_a, float* m_b, float* g,
                               uint32_t* row_flags, lb_ctx** out)
{
    if (!p || !out || !fneq_a || !fneq_b || !m_a || !m_b || !g || !row_flags)
        return set_error(PFSI_ERR_ARG, "lb_create_mixed: null argument");
    if (p->storage != PFSI_LB_BF16 && p->storage != PFSI_LB_FP16)
        return set_error(PFSI_ERR_ARG, "lb_create_mixed: storage must be PFSI_LB_BF16 or PFSI_LB_FP16");
    return create_common("lb_create_mixed", p, fneq_a, fneq_b, m_a, m_b, g, nullptr, row_flags, out);
}

extern "C" int lb_destroy(lb_ctx* ctx)
{
    if (ctx) lb_tma_destroy(ctx->tma);
    delete ctx;
    return PFSI_OK;
}

extern "C" int lb_init_shear(lb_ctx* c, void* stream)
{
    NvtxRange nvtx_range("lb_init_shear");
    if (!c) return set_error(PFSI_ERR_ARG, "lb_init_shear: null context");
    const lb_params& p = c->p;
    const int plane = p.nx * p.ny;
    const dim3 blocks((plane + 255) / 256 < 32 ? (plane + 255) / 256 : 32, p.nz);
    cudaStream_t s = as_stream(stream);
    const double tau = p.tau, ux = p.u_top[0], uy = p.u_top[1];
    switch (p.storage) {
    case PFSI_LB_BF16:
        k_lb_init_shear_mixed<PFSI_LB_BF16><<<blocks, 256, 0, s>>>((NeqT<PFSI_LB_BF16>*)c->f[c->cur], c->m[c->cur],
                                                                   p.nx, p.ny, p.nz, tau, ux, uy, 1.0f, p.walls);
        break;
    case PFSI_LB_FP16:
        k_lb_init_shear_mixed<PFSI_LB_FP16><<<blocks, 256, 0, s>>>((NeqT<PFSI_LB_FP16>*)c->f[c->cur], c->m[c->cur],
                                                                   p.nx, p.ny, p.nz, tau, ux, uy, inv_scale_of(p),
                                                                   p.walls);
        break;
    default:
        k_lb_init_shear<<<blocks, 256, 0, s>>>((float*)c->f[c->cur], p.nx, p.ny, p.nz, tau, ux, uy, p.walls);
    }
    return check_launch("lb_init_shear");
}

extern "C" int lb_step(lb_ctx* c, int nsteps, void* stream)
{
    NvtxRange nvtx_range("lb_step");
    if (!c) return set_error(PFSI_ERR_ARG, "lb_step: null context");
    if (nsteps < 0) return set_error(PFSI_ERR_ARG, "lb_step: negative step count");
    for (int s = 0; s < nsteps; ++s) {
        const int rc = launch_lb_step(c, as_stream(stream));
        if (rc) return rc;
    }
    return PFSI_OK;
}

extern "C" int lb_current(const lb_ctx* c, float** f)
{
    if (!c || !f) return set_error(PFSI_ERR_ARG, "lb_current: null argument");
    if (c->p.storage != PFSI_LB_FP32)
        return set_error(PFSI_ERR_ARG, "lb_current: mixed storage holds no FP32 populations (use lb_export)");
    *f = (float*)c->f[c->cur];
    return PFSI_OK;
}

extern "C" int lb_set_shape(lb_ctx* c, int shape)
{
    if (!c || shape < 0 || shape >= PFSI_LB_SHAPES) return set_error(PFSI_ERR_ARG, "lb_set_shape: bad argument");
    c->shape = shape;
    return PFSI_OK;
}

extern "C" int lb_get_shape(const lb_ctx* c, int* shape)
{
    if (!c || !shape) return set_error(PFSI_ERR_ARG, "lb_get_shape: null argument");
    *shape = c->shape;
    return PFSI_OK;
}

extern "C" int lb_autotune(lb_ctx* c, int reps, void* stream, float* best_ms)
{
    NvtxRange nvtx_range("lb_autotune");
    if (!c || reps < 1) return set_error(PFSI_ERR_ARG, "lb_autotune: bad argument");
    cudaStream_t s = as_stream(stream);
    cudaEvent_t e0, e1;
    int rc = check_cuda(cudaEventCreate(&e0), "lb_autotune: event");
    if (rc) return rc;
    rc = check_cuda(cudaEventCreate(&e1), "lb_autotune: event");
    if (rc) {
        cudaEventDestroy(e0);
        return rc;
    }
    int best = 0;
    float best_t = 0.f;
    for (int shape = 0; shape < PFSI_LB_SHAPES && !rc; ++shape) {
        c->shape = shape;
        rc = launch_lb_step(c, s);
        if (!rc) rc = check_cuda(cudaEventRecord(e0, s), "lb_autotune: record");
        for (int r = 0; r < reps && !rc; ++r) rc = launch_lb_step(c, s);
        if (!rc) rc = check_cuda(cudaEventRecord(e1, s), "lb_autotune: record");
        if (!rc) rc = check_cuda(cudaEventSynchronize(e1), "lb_autotune: synchronise");
        float ms = 0.f;
        if (!rc) rc = check_cuda(cudaEventElapsedTime(&ms, e0, e1), "lb_autotune: elapsed");
        ms /= reps;
        if (!rc && (shape == 0 || ms < best_t)) {
            best = shape;
            best_t = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->shape = best;
    if (!rc && best_ms) *best_ms = best_t;
    return rc;
}

struct lb_batch {
    pfsi::LbBatch* impl;
};

extern "C" int lb_batch_create(lb_ctx* const* lattices, int n, lb_batch** out)
{
    if (!lattices || !out) return set_error(PFSI_ERR_ARG, "lb_batch_create: null argument");
    std::vector<LbCtx*> lat(lattices, lattices + std::max(n, 0));
    LbBatch* impl = nullptr;
    const int rc = lb_batch_build(lat.data(), n, &impl);
    if (rc) return rc;
    *out = new lb_batch{impl};
    return PFSI_OK;
}

extern "C" int lb_batch_step(lb_batch* b, int nsteps, void* stream)
{
    NvtxRange nvtx_range("lb_batch_step");
    if (!b || nsteps < 0) return set_error(PFSI_ERR_ARG, "lb_batch_step: bad argument");
    for (int k = 0; k < nsteps; ++k) {
        const int rc = launch_lb_batch(b->impl, as_stream(stream));
        if (rc) return rc;
    }
    return PFSI_OK;
}

extern "C" int lb_batch_autotune(lb_batch* b, int reps, void* stream, float* ms_per_step)
{
    NvtxRange nvtx_range("lb_batch_autotune");
    if (!b) return set_error(PFSI_ERR_ARG, "lb_batch_autotune: null batch");
    return lb_batch_tune(b->impl, reps, as_stream(stream), ms_per_step);
}

extern "C" int lb_batch_get_shapes(const lb_batch* b, int* shapes)
{
    if (!b || !shapes) return set_error(PFSI_ERR_ARG, "lb_batch_get_shapes: null argument");
    return lb_batch_shapes(b->impl, shapes);
}

extern "C" int lb_batch_set_shapes(lb_batch* b, const int* shapes)
{
    if (!b || !shapes) return set_error(PFSI_ERR_ARG, "lb_batch_set_shapes: null argument");
    return lb_batch_assign_shapes(b->impl, shapes);
}

extern "C" int lb_batch_set_grid(lb_batch* b, int blocks_per_sm)
{
    if (!b) return set_error(PFSI_ERR_ARG, "lb_batch_set_grid: null batch");
    return lb_batch_configure_grid(b->impl, blocks_per_sm, b->impl->priority);
}

extern "C" int lb_batch_destroy(lb_batch* b)
{
    if (!b) return PFSI_OK;
    lb_batch_free(b->impl);
    delete b;
    return PFSI_OK;
}

extern "C" int lb_velocity(const lb_ctx* c, float** v)
{
    if (!c || !v) return set_error(PFSI_ERR_ARG, "lb_velocity: null argument");
    *v = reinterpret_cast<float*>(velocity_field(c));
    return PFSI_OK;
}

extern "C" int lb_export(lb_ctx* c, float* f_out, void* stream)
{
    NvtxRange nvtx_range("lb_export");
    if (!c || !f_out) return set_error(PFSI_ERR_ARG, "lb_export: null argument");
    if (!aligned(f_out, 4)) return set_error(PFSI_ERR_ARG, "lb_export: misaligned output");
    cudaStream_t s = as_stream(stream);
    const int N = (int)c->N;
    const lb_params& p = c->p;
    if (p.storage == PFSI_LB_FP32)
        return check_cuda(cudaMemcpyAsync(f_out, c->f[c->cur], (size_t)N * 19 * sizeof(float),
                                          cudaMemcpyDeviceToDevice, s),
                          "lb_export: copy");
    const int blocks = (N + 255) / 256 < 148 * 8 ? (N + 255) / 256 : 148 * 8;
    if (p.storage == PFSI_LB_BF16)
        k_lb_export_mixed<PFSI_LB_BF16><<<blocks, 256, 0, s>>>(std::make_integer_sequence<int, 19>{},
                                                               (const NeqT<PFSI_LB_BF16>*)c->f[c->cur],
                                                               c->m[c->cur], f_out, N, 1.0f);
    else
        k_lb_export_mixed<PFSI_LB_FP16><<<blocks, 256, 0, s>>>(std::make_integer_sequence<int, 19>{},
                                                               (const NeqT<PFSI_LB_FP16>*)c->f[c->cur],
                                                               c->m[c->cur], f_out, N, inv_scale_of(p));
    return check_launch("lb_export");
}

namespace pfsi {
namespace {

// Counts of the instability check: cnt[0] non-finite, cnt[1] rho <= 0,
// cnt[2] |u| > u_max (one atomic per thread that found something).
__device__ __forceinline__ void check_cell(float rho, float ux, float uy, float uz, float u_max2, bool bad_store,
                                           unsigned long long* c)
{
    const bool nf = bad_store || !isfinite(rho) || !isfinite(ux) || !isfinite(uy) || !isfinite(uz);
    c[0] += nf;
    c[1] += !nf && rho <= 0.0f;
    c[2] += !nf && (ux * ux + uy * uy + uz * uz) > u_max2;
}

__device__ __forceinline__ void flush_counts(const unsigned long long* c, unsigned long long* cnt)
{
    for (int k = 0; k < 3; ++k)
        if (c[k]) atomicAdd(&cnt[k], c[k]);
}

__global__ void k_lb_check(const float* __restrict__ f, int N, float u_max2, unsigned long long* __restrict__ cnt)
{
    unsigned long long c[3] = {0, 0, 0};
    for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < N; cell += gridDim.x * blockDim.x) {
        float d = 0.f, mx = 0.f, my = 0.f, mz = 0.f;
#pragma unroll
        for (int q = 0; q < 19; ++q) {
            const float fq = f[q * N + cell];
            d += fq;
            if (cxq(q)) mx += cxq(q) * fq;
            if (cyq(q)) my += cyq(q) * fq;
            if (czq(q)) mz += czq(q) * fq;
        }
        const float rho = 1.0f + d, inv = 1.0f / rho;
        check_cell(rho, mx * inv, my * inv, mz * inv, u_max2, false, c);
    }
    flush_counts(c, cnt);
}

template <int kMode>
__global__ void k_lb_check_mixed(const uint16_t* __restrict__ neq, const float4* __restrict__ m, int N, float u_max2,
                                 unsigned long long* __restrict__ cnt)
{
    // an all-ones exponent field marks a non-finite 16-bit value
    constexpr uint16_t kExp = kMode == PFSI_LB_BF16 ? 0x7f80u : 0x7c00u;
    unsigned long long c[3] = {0, 0, 0};
    for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < N; cell += gridDim.x * blockDim.x) {
        bool bad = false;
#pragma unroll
        for (int q = 0; q < 19; ++q) bad |= (neq[q * N + cell] & kExp) == kExp;
        const float4 v = m[cell];
        check_cell(1.0f + v.w, v.x, v.y, v.z, u_max2, bad, c);
    }
    flush_counts(c, cnt);
}

}  // namespace
}  // namespace pfsi

extern "C" int lb_check(lb_ctx* c, float u_max, unsigned long long* dev_scratch4, long long* out_host, void* stream)
{
    NvtxRange nvtx_range("lb_check");
    if (!c || !dev_scratch4 || !out_host || !(u_max > 0.0f)) return set_error(PFSI_ERR_ARG, "lb_check: bad argument");
    if (!aligned(dev_scratch4, 8)) return set_error(PFSI_ERR_ARG, "lb_check: scratch must be 8-byte aligned");
    cudaStream_t s = as_stream(stream);
    int rc = check_cuda(cudaMemsetAsync(dev_scratch4, 0, 4 * sizeof(unsigned long long), s), "lb_check: clear");
    if (rc) return rc;
    const int N = (int)c->N;
    const int blocks = (N + 255) / 256 < 148 * 8 ? (N + 255) / 256 : 148 * 8;
    const float u2 = u_max * u_max;
    switch (c->p.storage) {
    case PFSI_LB_BF16:
        k_lb_check_mixed<PFSI_LB_BF16><<<blocks, 256, 0, s>>>((const uint16_t*)c->f[c->cur], c->m[c->cur], N, u2,
                                                              dev_scratch4);
        break;
    case PFSI_LB_FP16:
        k_lb_check_mixed<PFSI_LB_FP16><<<blocks, 256, 0, s>>>((const uint16_t*)c->f[c->cur], c->m[c->cur], N, u2,
                                                              dev_scratch4);
        break;
    default:
        k_lb_check<<<blocks, 256, 0, s>>>((const float*)c->f[c->cur], N, u2, dev_scratch4);
    }
    if ((rc = check_launch("lb_check"))) return rc;
    unsigned long long h[4];
    rc = check_cuda(cudaMemcpyAsync(h, dev_scratch4, sizeof(h), cudaMemcpyDeviceToHost, s), "lb_check: copy");
    if (!rc) rc = check_cuda(cudaStreamSynchronize(s), "lb_check: synchronise");
    if (rc) return rc;
    for (int k = 0; k < 3; ++k) out_host[k] = (long long)h[k];
    if (h[0] || h[1] || h[2])
        return set_error(PFSI_ERR_UNSTABLE, "lb_check: " + std::to_string(h[0]) + " non-finite cells, " +
                                                std::to_string(h[1]) + " with rho <= 0, " + std::to_string(h[2]) +
                                                " faster than u_max");
    return PFSI_OK;
}

extern "C" int lb_moments_fp64(lb_ctx* c, double* dev_scratch4, double* out_host, void* stream)
{
    NvtxRange nvtx_range("lb_moments_fp64");
    if (!c || !dev_scratch4 || !out_host) return set_error(PFSI_ERR_ARG, "lb_moments_fp64: null argument");
    if (!aligned(dev_scratch4, 8)) return set_error(PFSI_ERR_ARG, "lb_moments_fp64: scratch must be 8-byte aligned");
    cudaStream_t s = as_stream(stream);
    int rc = check_cuda(cudaMemsetAsync(dev_scratch4, 0, 4 * sizeof(double), s), "lb_moments_fp64: clear");
    if (rc) return rc;
    const int N = (int)c->N;
    const int blocks = (N + 255) / 256 < 148 * 8 ? (N + 255) / 256 : 148 * 8;
    switch (c->p.storage) {
    case PFSI_LB_BF16:
        k_lb_moments_mixed<PFSI_LB_BF16><<<blocks, 256, 0, s>>>((const NeqT<PFSI_LB_BF16>*)c->f[c->cur],
                                                                c->m[c->cur], N, dev_scratch4, 1.0f);
        break;
    case PFSI_LB_FP16:
        k_lb_moments_mixed<PFSI_LB_FP16><<<blocks, 256, 0, s>>>((const NeqT<PFSI_LB_FP16>*)c->f[c->cur],
                                                                c->m[c->cur], N, dev_scratch4, inv_scale_of(c->p));
        break;
    default:
        k_lb_moments<<<blocks, 256, 0, s>>>((const float*)c->f[c->cur], N, dev_scratch4);
    }
    rc = check_launch("lb_moments_fp64");
    if (rc) return rc;
    rc = check_cuda(cudaMemcpyAsync(out_host, dev_scratch4, 4 * sizeof(double), cudaMemcpyDeviceToHost, s),
                    "lb_moments_fp64: copy");
    if (rc) return rc;
    return check_cuda(cudaStreamSynchronize(s), "lb_moments_fp64: synchronise");
}
