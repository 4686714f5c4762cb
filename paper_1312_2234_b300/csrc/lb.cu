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

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "pfsi_internal.cuh"

namespace pfsi {

namespace {

constexpr int kRowBlock = 128;     // default threads per block along x (FP32 kernel)
constexpr int kMaxRowBlock = 256;

__global__ void __launch_bounds__(kMaxRowBlock) k_lb_step(
    const float* __restrict__ fin, float* __restrict__ fout, float4* __restrict__ g,
    float4* __restrict__ vout, const uint32_t* __restrict__ flags, int nx, int ny, int nz,
    float omega, float guo, float3 body, float3 utop, int onsite)
{
    pdl_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y, k = blockIdx.z;
    if (i >= nx) return;
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
    const float vv = vx * vx + vy * vy + vz * vz;
    const float vF = vx * Fx + vy * Fy + vz * Fz;

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
        const float odd = a + b;
        const float even = fmaf(1.5f * cv, fmaf(2.0f, b, a), wq(q) * A0);
        fout[q * N + cell] = fmaf(keep, f[q], even + odd);
        fout[o * N + cell] = fmaf(keep, f[o], even - odd);
    }
    if (forced) {
        vout[cell] = make_float4(vx, vy, vz, rho);
        g[cell] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
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

template <class T>
__device__ __forceinline__ void halo_store(Ring<T>& ring, int slot, const float4* r)
{
#pragma unroll
    for (int u = 0; u < T::Halo; ++u) {
        const int h = threadIdx.x + u * T::Threads;
        if (h < T::Plane) ring.pj[slot][h] = split_record(r[u]);
    }
}

// E_q of a ring cell, for direction q.
template <int q, class T>
__device__ __forceinline__ float feq_ring(const Ring<T>& ring, int slot, int h)
{
    return wq(q) * split_eq<q>(ring.pj[slot][h]);
}

// f[q] += E_q of the source cell (bounce-back: the own cell's opposite
// population, plus the moving-wall term at the top).  sm, s0, sp: ring slots
// of the planes k - 1, k, k + 1.
template <int q, class T>
__device__ __forceinline__ void add_feq(float* f, const Ring<T>& ring, int sm, int s0, int sp, int own, int k,
                                        int nz, float3 utop)
{
    if (czq(q) == 1 && k == 0) {
        f[q] += feq_ring<oppq(q)>(ring, s0, own);
    } else if (czq(q) == -1 && k == nz - 1) {
        const float cu = cxq(q) * utop.x + cyq(q) * utop.y;
        f[q] += feq_ring<oppq(q)>(ring, s0, own) + 6.0f * wq(q) * cu;
    } else {
        f[q] += feq_ring<q>(ring, czq(q) == 1 ? sm : (czq(q) == -1 ? sp : s0), own - cyq(q) * T::HX - cxq(q));
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
// in c is w E0 + cv (h + b), the odd part a + b (see k_lb_step_mixed).
template <int kMode, int q>
__device__ __forceinline__ void store_pair(typename Neq<kMode>::T* __restrict__ nout, int N, int cell, const float* f,
                                           float vx, float vy, float vz, float3 F3, float rk, float rh, float keep,
                                           float E0, float guo, float scale)
{
    if (q == 18 || oppq(q) < q) return;
    const float cv = cdot<q>(vx, vy, vz), cF = cdot<q>(F3.x, F3.y, F3.z);
    const float wcv = wq(q) * cv;
    const float a = rk * wcv;
    const float b = (wq(q) * guo) * cF;
    const float odd = a + b;
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

template <int kMode, class T>
__global__ void __launch_bounds__(T::Threads, 768 / T::Threads) k_lb_step_mixed(
    const uint16_t* __restrict__ nin, typename Neq<kMode>::T* __restrict__ nout, const float4* __restrict__ min_,
    float4* __restrict__ mout, float4* __restrict__ g, const uint32_t* __restrict__ flags, int nx, int ny, int nz,
    int kz, float omega, float guo, float3 body, float3 utop, float inv_scale, int onsite)
{
    pdl_wait();
    __shared__ Ring<T> ring;
    const int tx = threadIdx.x % T::TX, ty = threadIdx.x / T::TX;
    const int x0 = blockIdx.x * T::TX, y0 = blockIdx.y * T::TY;
    const int z0 = blockIdx.z * kz, z1 = min(z0 + kz, nz);
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

            float drho = 0.f, mx = 0.f, my = 0.f, mz = 0.f;
#pragma unroll
            for (int q = 0; q < 19; ++q) {
                drho += f[q];
                if (cxq(q)) mx += cxq(q) * f[q];
                if (cyq(q)) my += cyq(q) * f[q];
                if (czq(q)) mz += czq(q) * f[q];
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
            const float i3rho = 3.0f / rho;
            const float vx = fmaf(F3.x, 1.0f / 6.0f, mx) * i3rho;
            const float vy = fmaf(F3.y, 1.0f / 6.0f, my) * i3rho;
            const float vz = fmaf(F3.z, 1.0f / 6.0f, mz) * i3rho;
            const float VV = vx * vx + vy * vy + vz * vz;                           // 9 v.v
            const float P0 = fmaf(-rho / 6.0f, VV, drho);                            // drho - 1.5 rho v.v
            const float vF3 = (vx * F3.x + vy * F3.y + vz * F3.z) * (1.0f / 3.0f);  // 3 v.F
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

template <int kMode>
cudaError_t launch_mixed_shape(LbCtx* c, cudaStream_t s, float omega, float guo, float3 body, float3 utop,
                               float inv_scale)
{
    if (c->tma) {
        // shapes 0, 1: this kernel with 32 x 4 or 32 x 8 columns (the faster
        // on B300); 2, 3: the TMA-staged kernel with 32 x 8 or 32 x 4 columns
        switch (c->shape) {
        case 0: return launch_mixed<kMode, Tile<32, 4>>(c, s, omega, guo, body, utop, inv_scale);
        case 1: return launch_mixed<kMode, Tile<32, 8>>(c, s, omega, guo, body, utop, inv_scale);
        case 2: return lb_tma_launch(c, c->tma, 0, s, omega, guo, body, utop, inv_scale);
        default: return lb_tma_launch(c, c->tma, 1, s, omega, guo, body, utop, inv_scale);
        }
    }
    switch (c->shape) {
    case 1: return launch_mixed<kMode, Tile<32, 4>>(c, s, omega, guo, body, utop, inv_scale);
    case 2: return launch_mixed<kMode, Tile<64, 4>>(c, s, omega, guo, body, utop, inv_scale);
    case 3: return launch_mixed<kMode, Tile<16, 8>>(c, s, omega, guo, body, utop, inv_scale);
    default: return launch_mixed<kMode, Tile<32, 8>>(c, s, omega, guo, body, utop, inv_scale);
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
