// lb_tma.cu -- D3Q19 lattice Boltzmann step on 16-bit f*neq storage (Section
// 3.3, Eq. 16-21) with the tiles moved by the Tensor Memory Accelerator, for
// sm_103a.
//
// The state is that of the mixed storage of lb.cu: per cell the post-collision
// non-equilibrium parts in 16 bits (BF16, or FP16 scaled by 2^s) and the FP32
// moment record m = (v, rho - 1).  The step is the same operation: pull
// streaming (periodic x, y; halfway bounce-back at the z walls, moving top
// wall), moments (Eq. 17-18), v = u + F/(2 rho), BGK relaxation to the
// equilibrium of Eq. 20 with Guo's source (Eq. 19).
//
// Split of a population into its stored 16 bits and its rebuilt part.  A
// pulling cell rebuilds f*_q of its source cell as E_q(source) + stored_q,
// E_q = w_q (P + c.J + (c.J)^2 / 2) with J = 3 rho v and P = rho - 1 -
// 1.5 rho v.v, four numbers per cell held in a shared-memory ring of
// planes.  E_q differs from the equilibrium of Eq. 20 only by
// w_q rho (1 - rho) (3 c.v)^2 / 2; the writer stores f*_q - E_q (its
// collision carries that difference in the part even in c), so the pair
// rebuilds f*_q exactly up to the rounding of the stored value, at three
// FP32 operations per pulled population.
//
// Data movement.  A block owns a TX x TY column of cells and marches it
// through kz planes.  Plane k pulls, per direction q, the stored values of
// the source plane k - c_z over the column plus a one-cell halo.  The stored
// array holds the directions in slot order grouped by c_z (nslot), so the
// three groups of a plane are three TMA boxes: the nine c_z = 0 slots of
// plane k, the five c_z = +1 slots of plane k - 1 and the five c_z = -1
// slots of plane k + 1, each 48 x (TY + 2) cells starting 8 cells left of
// the column so that the copy starts on a 16-byte boundary (at a wall plane
// the group that would come from outside is the own plane's opposite
// group: bounce-back).  One more box brings the moment records of plane
// k + 1 plus halo.  The copies for plane k + 2 are in flight while plane k
// computes (three stage buffers, one mbarrier each).  The 19 output tiles
// are staged in shared memory and written by one TMA store; the moment
// record of a cell is stored by its thread.  The periodic halo of columns
// on the x and y edges of the domain lies outside the tensor, where TMA
// fills zeros; the threads of those blocks patch the wrapped entries with
// plain loads after the copy has landed.
//
// Every mbarrier wait is bounded; a wait that gives up sets bit 0 of the
// status word, waits (bounded) for the block's copies in flight and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>
#include <string>

#include "pfsi_internal.cuh"

namespace pfsi {

namespace {

constexpr int kStages = 3;           // stage buffers (copies for two planes ahead in flight)
constexpr int kSuspendNs = 1000000;   // suspend hint of one try (1 ms)
constexpr int kTries = 4096;          // tries before a wait gives up (~4 s)

__device__ unsigned int g_lb_tma_status;   // bit 0: a bounded wait gave up

constexpr int kRing = 5;             // ring slots of moment planes (k - 2 .. k + 3 in play)

template <int TX_, int TY_>
struct TmaTile {
    static constexpr int TX = TX_, TY = TY_;
    static constexpr int Threads = TX * TY;          // compute threads: one per cell of the column
    static constexpr int Warps = Threads / 32;
    static constexpr int Block = Threads + 32;       // plus one producer warp
    static constexpr int WX = TX + 16;               // box width of a direction tile (x0 - 8 .. x0 + TX + 8)
    static constexpr int HY = TY + 2, HX = TX + 2;   // halo extents
    static constexpr int QB = HY * WX * 2;           // bytes of one direction tile (dense within a group box)
    static constexpr int G0 = 0;                                  // slots 0..8
    static constexpr int GP = ((G0 + 9 * QB + 127) / 128) * 128;  // slots 9..13
    static constexpr int GM = ((GP + 5 * QB + 127) / 128) * 128;  // slots 14..18
    static constexpr int StageBytes = ((GM + 5 * QB + 127) / 128) * 128;
    static constexpr int RingCells = HY * HX;
    static constexpr int RingBoxBytes = RingCells * 16;
    static constexpr int RingSlotBytes = ((RingBoxBytes + 127) / 128) * 128;
    static constexpr int OutNeqBytes = TX * TY * 2;  // one direction
    static constexpr int OutBytes = 19 * OutNeqBytes;
    static constexpr int OffStage = 0;
    static constexpr int OffRing = kStages * StageBytes;
    static constexpr int OffOut = OffRing + kRing * RingSlotBytes;   // two output buffers
    static constexpr int OffBar = OffOut + 2 * OutBytes;
    // mbarriers: full[3], empty[3], out-full[2], out-empty[2]
    static constexpr int SmemBytes = OffBar + 8 * 10 + 128;   // + alignment slack
    static_assert(OutBytes % 128 == 0, "TMA store tiles must stay 128-byte aligned");
    // resident blocks per SM that the registers are sized for: as many as the
    // shared memory holds, at most 512 compute threads per SM
    static constexpr int MinBlocks = (512 / Threads) < (233472 / (SmemBytes + 1024)) ? (512 / Threads)
                                                                                      : (233472 / (SmemBytes + 1024));
    static_assert(Threads % 32 == 0, "whole warps of cells");
    // byte offset of slot s's tile within a stage
    static __host__ __device__ constexpr int tile(int s)
    {
        return s < 9 ? G0 + s * QB : (s < 14 ? GP + (s - 9) * QB : GM + (s - 14) * QB);
    }
};

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// One bounded try: the thread sleeps until the phase completes or about
// kSuspendNs have passed.
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "n"(kSuspendNs)
        : "memory");
    return ok != 0;
}
// Bounded wait for phase `parity` of the mbarrier (at most kTries tries, a
// few seconds); false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    for (int i = 0; i < kTries; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_load4(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                          uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(dst),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tma_store4(const CUtensorMap* map, uint32_t src, int c0, int c1, int c2, int c3)
{
    asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(map),
                 "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(src)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16-bit stored value -> FP32 (BF16 as is; FP16 times 2^-s) and back.
template <int kMode>
__device__ __forceinline__ float neq_get(uint16_t raw, float inv_scale)
{
    if (kMode == PFSI_LB_BF16) return __uint_as_float((uint32_t)raw << 16);
    return __half2float(__ushort_as_half(raw)) * inv_scale;
}
template <int kMode>
__device__ __forceinline__ uint16_t neq_put(float x, float scale)
{
    if (kMode == PFSI_LB_BF16) return __bfloat16_as_ushort(__float2bfloat16_rn(x));
    return __half_as_ushort(__float2half_rn(x * scale));
}

struct StepArgs {
    const uint16_t* nin;      // current stored values (wrapped halo patches)
    const float4* min_;       // current moment records (wrapped halo patches)
    float4* mout;             // next moment records
    float4* g;
    const uint32_t* flags;
    int nx, ny, nz, kz;
    float omega, guo, inv_scale;
    float3 body, utop;
    int onsite;
};

// Copies of plane k's stage (thread 0): the three slot groups (at a wall
// plane the group from outside the domain is replaced by the own plane's
// opposite group: bounce-back) and the moment records of the planes in
// [p0, p1] into their ring slots.
template <class T>
__device__ __forceinline__ void issue_stage(const StepArgs& a, const CUtensorMap* tm9, const CUtensorMap* tm5,
                                            const CUtensorMap* tm_m, char* smem, int buf, int k, int p0, int p1,
                                            int x0, int y0)
{
    const uint32_t bar = smem_u32(smem + T::OffBar + 8 * buf);
    int planes = 0;
    for (int p = p0; p <= p1; ++p) planes += (p >= 0 && p < a.nz);
    mbar_expect_tx(bar, 19u * T::QB + (uint32_t)planes * T::RingBoxBytes);
    const uint32_t st = smem_u32(smem + T::OffStage + buf * T::StageBytes);
    tma_load4(st + T::G0, tm9, x0 - 8, y0 - 1, k, 0, bar);
    if (k == 0)
        tma_load4(st + T::GP, tm5, x0 - 8, y0 - 1, k, 14, bar);
    else
        tma_load4(st + T::GP, tm5, x0 - 8, y0 - 1, k - 1, 9, bar);
    if (k == a.nz - 1)
        tma_load4(st + T::GM, tm5, x0 - 8, y0 - 1, k, 9, bar);
    else
        tma_load4(st + T::GM, tm5, x0 - 8, y0 - 1, k + 1, 14, bar);
    for (int p = p0; p <= p1; ++p)
        if (p >= 0 && p < a.nz)
            tma_load4(smem_u32(smem + T::OffRing + (p % kRing) * T::RingSlotBytes), tm_m, 0, x0 - 1, y0 - 1, p, bar);
}

// Edge blocks: the direction tiles' entries outside the domain in x or y
// (zero-filled by TMA) that live cells pull, replaced by their periodic
// images.  The entries form one list -- the x halo columns of the five
// directions with c_x = +1 (left edge) and c_x = -1 (right edge), the y
// halo rows of the five with c_y = +1 (bottom) and c_y = -1 (top) -- of
// which every compute thread takes its share.  The values are the previous
// step's state in global memory, so a thread loads them early (while it
// computes the plane before) and writes them once the copy has landed.
__constant__ int kDirEdge[4][5] = {{0, 6, 7, 8, 9}, {1, 10, 11, 12, 13}, {2, 6, 10, 14, 15}, {3, 7, 11, 16, 17}};

template <class T>
struct Patch {
    static constexpr int Per = (10 * T::HY + 10 * T::HX + T::Threads - 1) / T::Threads;
    int idx[Per];          // uint16 index in the stage buffer, or -1
    int q[Per];            // direction
    int off[Per];          // wrapped in-plane cell offset gy nx + gx
    uint16_t v[Per];
};

// The thread's entries of the list (the same for every plane of the column).
template <class T>
__device__ __forceinline__ void patch_plan(Patch<T>& pt, const StepArgs& a, int x0, int y0)
{
    const int xr = min(a.nx - x0, T::TX), yr = min(a.ny - y0, T::TY);   // live extent of the column
    const bool side[4] = {x0 == 0, x0 + T::TX >= a.nx, y0 == 0, y0 + T::TY >= a.ny};
    constexpr int kLen[4] = {5 * T::HY, 5 * T::HY, 5 * T::HX, 5 * T::HX};
#pragma unroll
    for (int u = 0; u < Patch<T>::Per; ++u) {
        pt.idx[u] = -1;
        int e = threadIdx.x + u * T::Threads;
        for (int kind = 0; kind < 4; ++kind) {
            if (!side[kind]) continue;
            if (e >= kLen[kind]) {
                e -= kLen[kind];
                continue;
            }
            const int per = kind < 2 ? T::HY : T::HX;
            const int d = e / per, r = e - d * per;
            const int q = kDirEdge[kind][d];
            const int bx = kind == 0 ? 7 : (kind == 1 ? 8 + xr : 7 + r);
            const int by = kind < 2 ? r : (kind == 2 ? 0 : 1 + yr);
            int gx = x0 - 8 + bx, gy = y0 - 1 + by;
            if (gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny) break;   // inside: TMA has it
            if (gx < -1 || gx > a.nx || gy < -1 || gy > a.ny) break;     // read by no live cell
            gx = gx < 0 ? gx + a.nx : (gx >= a.nx ? gx - a.nx : gx);
            gy = gy < 0 ? gy + a.ny : (gy >= a.ny ? gy - a.ny : gy);
            pt.idx[u] = T::tile(nslot(q)) / 2 + by * T::WX + bx;
            pt.q[u] = q;
            pt.off[u] = gy * a.nx + gx;
            break;
        }
    }
}

// Loads the thread's entries of plane k's stage (early: the previous
// step's state), skipping the groups that bounce back from the own plane.
template <class T>
__device__ __forceinline__ void patch_gather(Patch<T>& pt, const StepArgs& a, int k)
{
    const long long N = (long long)a.nx * a.ny * a.nz, plane = (long long)a.nx * a.ny;
#pragma unroll
    for (int u = 0; u < Patch<T>::Per; ++u) {
        if (pt.idx[u] < 0) continue;
        const int q = pt.q[u], cz = czq(q);
        if ((cz == 1 && k == 0) || (cz == -1 && k == a.nz - 1)) continue;
        pt.v[u] = a.nin[(long long)nslot(q) * N + (long long)(k - cz) * plane + pt.off[u]];
    }
}

template <class T>
__device__ __forceinline__ void patch_scatter(const Patch<T>& pt, const StepArgs& a, char* smem, int buf, int k)
{
    uint16_t* st = reinterpret_cast<uint16_t*>(smem + T::OffStage + buf * T::StageBytes);
#pragma unroll
    for (int u = 0; u < Patch<T>::Per; ++u) {
        if (pt.idx[u] < 0) continue;
        const int cz = czq(pt.q[u]);
        if ((cz == 1 && k == 0) || (cz == -1 && k == a.nz - 1)) continue;
        st[pt.idx[u]] = pt.v[u];
    }
}

// The records (v, rho - 1) of a plane's ring cells -> (P, J), every compute
// thread its share; the wrapped halo of edge blocks comes from global memory
// (loaded early by ring_gather).
template <class T>
struct RingHalo {
    static constexpr int Per = (T::RingCells + T::Threads - 1) / T::Threads;
    int off[Per];          // wrapped in-plane offset of an edge block's outside ring cell, or -1
    bool wrapped[Per];
    float4 m[Per];
};

template <class T>
__device__ __forceinline__ void ring_plan(RingHalo<T>& rh, const StepArgs& a, int x0, int y0, bool edge)
{
#pragma unroll
    for (int u = 0; u < RingHalo<T>::Per; ++u) {
        rh.off[u] = -1;
        const int h = threadIdx.x + u * T::Threads;
        if (!edge || h >= T::RingCells) continue;
        const int hy = h / T::HX, hx = h - hy * T::HX;
        int gx = x0 - 1 + hx, gy = y0 - 1 + hy;
        if ((gx < 0 || gx >= a.nx || gy < 0 || gy >= a.ny) && gx <= a.nx && gy <= a.ny) {
            gx = gx < 0 ? gx + a.nx : (gx >= a.nx ? gx - a.nx : gx);
            gy = gy < 0 ? gy + a.ny : (gy >= a.ny ? gy - a.ny : gy);
            rh.off[u] = gy * a.nx + gx;
        }
    }
}

// Loads the thread's outside ring cells of plane p (early).
template <class T>
__device__ __forceinline__ void ring_gather(RingHalo<T>& rh, const StepArgs& a, int p)
{
#pragma unroll
    for (int u = 0; u < RingHalo<T>::Per; ++u) {
        rh.wrapped[u] = rh.off[u] >= 0 && p >= 0 && p < a.nz;
        if (rh.wrapped[u]) rh.m[u] = a.min_[(long long)p * a.ny * a.nx + rh.off[u]];
    }
}

template <class T>
__device__ __forceinline__ void ring_convert(const RingHalo<T>& rh, char* smem, int p)
{
    float4* r = reinterpret_cast<float4*>(smem + T::OffRing + (p % kRing) * T::RingSlotBytes);
#pragma unroll
    for (int u = 0; u < RingHalo<T>::Per; ++u) {
        const int h = threadIdx.x + u * T::Threads;
        if (h < T::RingCells) r[h] = split_record(rh.wrapped[u] ? rh.m[u] : r[h]);
    }
}

// Named barrier of the compute warps alone (the producer warp runs on).
template <class T>
__device__ __forceinline__ void compute_sync()
{
    asm volatile("bar.sync 1, %0;" ::"n"(T::Threads) : "memory");
}

// f[q] = E_q(source) + stored_q(source) for one direction.  kWall: 0 bulk
// plane, 1 bottom plane, 2 top plane (bounce-back from the own cell).
// Ring offsets (float4 units) of the planes k - 1, k, k + 1: rm, r0, rp.
template <int kMode, class T, int kWall, int q>
__device__ __forceinline__ void pull(float* f, const uint16_t* st, const float4* ring, int rm, int r0, int rp,
                                     int tx, int ty, float inv_scale, float3 utop)
{
    const uint16_t* tile = st + T::tile(nslot(q)) / 2;
    const bool bb = (kWall == 1 && czq(q) == 1) || (kWall == 2 && czq(q) == -1);
    if (bb) {
        const float4 rec = ring[r0 + (ty + 1) * T::HX + tx + 1];
        const uint16_t raw = tile[(ty + 1) * T::WX + tx + 8];
        float e = neq_get<kMode>(raw, inv_scale);
        if (kWall == 2) e = fmaf(6.0f * wq(q), cxq(q) * utop.x + cyq(q) * utop.y, e);
        f[q] = fmaf(wq(oppq(q)), split_eq<oppq(q)>(rec), e);
    } else {
        const int slot = czq(q) == 1 ? rm : (czq(q) == -1 ? rp : r0);
        const float4 rec = ring[slot + (ty + 1 - cyq(q)) * T::HX + tx + 1 - cxq(q)];
        const uint16_t raw = tile[(ty + 1 - cyq(q)) * T::WX + tx + 8 - cxq(q)];
        f[q] = fmaf(wq(q), split_eq<q>(rec), neq_get<kMode>(raw, inv_scale));
    }
}

template <int kMode, class T, int kWall, int... Q>
__device__ __forceinline__ void pull_all(std::integer_sequence<int, Q...>, float* f, const uint16_t* st,
                                         const float4* ring, int rm, int r0, int rp, int tx, int ty, float inv_scale,
                                         float3 utop)
{
    (pull<kMode, T, kWall, Q>(f, st, ring, rm, r0, rp, tx, ty, inv_scale, utop), ...);
}

// Stored values of the pair (q, opposite of q): with cv = 3 c.v, cF = 3 c.F
// (see cell_step) the part even in c is w E0 + cv (h + b), the odd part
// a + b.
template <int kMode, class T, int q>
__device__ __forceinline__ void pair_out(uint16_t* out, int o, const float* f, float vx, float vy, float vz, float3 F3,
                                         float rk, float rh, float keep, float E0, float guo, float scale)
{
    if (q == 18 || oppq(q) < q) return;
    const float cv = cdot<q>(vx, vy, vz), cF = cdot<q>(F3.x, F3.y, F3.z);
    const float wcv = wq(q) * cv;
    const float b = (wq(q) * guo) * cF;
    const float odd = fmaf(rk, wcv, b);
    const float even = fmaf(cv, fmaf(rh, wcv, b), wq(q) * E0);
    out[nslot(q) * (T::OutNeqBytes / 2) + o] = neq_put<kMode>(fmaf(keep, f[q], even + odd), scale);
    out[nslot(oppq(q)) * (T::OutNeqBytes / 2) + o] = neq_put<kMode>(fmaf(keep, f[oppq(q)], even - odd), scale);
}

template <int kMode, class T, int... Q>
__device__ __forceinline__ void pair_all(std::integer_sequence<int, Q...>, uint16_t* out, int o, const float* f,
                                         float vx, float vy, float vz, float3 F3, float rk, float rh, float keep,
                                         float E0, float guo, float scale)
{
    (pair_out<kMode, T, Q>(out, o, f, vx, vy, vz, F3, rk, rh, keep, E0, guo, scale), ...);
}

// One cell of plane k: pull, collide, stage the stored values in output
// buffer ob and write the moment record.  forced: the row's flag; gg its
// force (valid if forced).
template <int kMode, class T, int kWall>
__device__ __forceinline__ void cell_step(const StepArgs& a, char* smem, int buf, int ob, int k, int tx, int ty,
                                          long long cell, bool forced, float4 gg)
{
    const uint16_t* st = reinterpret_cast<const uint16_t*>(smem + T::OffStage + buf * T::StageBytes);
    const float4* ring = reinterpret_cast<const float4*>(smem + T::OffRing);
    constexpr int kSlot = T::RingSlotBytes / 16;
    const int rm = ((k + kRing - 1) % kRing) * kSlot, r0 = (k % kRing) * kSlot, rp = ((k + 1) % kRing) * kSlot;
    float f[19];
    pull_all<kMode, T, kWall>(std::make_integer_sequence<int, 19>{}, f, st, ring, rm, r0, rp, tx, ty, a.inv_scale,
                              a.utop);
    if (kWall && a.onsite) {
        if (kWall == 1) onsite_wall<1>(f, make_float3(0.f, 0.f, 0.f));
        if (kWall == 2) onsite_wall<-1>(f, a.utop);
    }

    // moments per pair of opposite directions (the order of every 16-bit kernel)
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
    float3 F3 = make_float3(3.0f * a.body.x, 3.0f * a.body.y, 3.0f * a.body.z);
    if (forced) {
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
    const float keep = 1.0f - a.omega;
    // stored = f* - E = (1 - omega)(f - f^eq) + S + (f^eq - E): per pair of
    // opposite directions, with cv = 3 c.v, cF = 3 c.F,
    //   a = -keep w rho cv (odd), h = w rho cv (omega - rho) / 2 (even; the
    //   -keep of the relaxation plus the 1 - rho of f^eq - E), b = w guo cF,
    //   E0 = -keep P0 - guo vF3,
    // even part w E0 + cv (h + b), odd part a + b.
    const float E0 = fmaf(-keep, P0, -a.guo * vF3);
    const float rk = -keep * rho, rh = 0.5f * rho * (a.omega - rho);
    const float scale = 1.0f / a.inv_scale;
    uint16_t* out = reinterpret_cast<uint16_t*>(smem + T::OffOut + ob * T::OutBytes);
    const int o = ty * T::TX + tx;
    out[nslot(18) * (T::OutNeqBytes / 2) + o] = neq_put<kMode>(fmaf(keep, f[18], wq(18) * E0), scale);
    pair_all<kMode, T>(std::make_integer_sequence<int, 18>{}, out, o, f, vx, vy, vz, F3, rk, rh, keep, E0, a.guo,
                       scale);
    a.mout[cell] = make_float4(vx * (1.0f / 3.0f), vy * (1.0f / 3.0f), vz * (1.0f / 3.0f), drho);
    if (forced) a.g[cell] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Plane loop of one column, warp-specialised.  The compute warps (one
// thread per cell) pull, collide and write plane k's outputs, then prepare
// plane k + 1 (patch its wrapped halo, split the records of plane k + 2);
// the producer warp only moves data:
//   full[s]    the TMA copies of stage s have landed (expect_tx)
//   empty[s]   the compute warps are done with stage s (one arrival each)
//   ofull[b]   the compute warps have written output buffer b (one each)
//   oempty[b]  the TMA store that last read output buffer b is done with it
// Per plane k (iteration it) the producer (lane 0) frees output buffer
// it & 1, stores plane k - 1 and issues the copies of stage it + 2 once the
// compute warps have released their buffers.
template <int kMode, class T>
__global__ void __launch_bounds__(T::Block, T::MinBlocks) k_lb_step_tma(
    const __grid_constant__ CUtensorMap tm9, const __grid_constant__ CUtensorMap tm5,
    const __grid_constant__ CUtensorMap tm_out, const __grid_constant__ CUtensorMap tm_m, StepArgs a)
{
    extern __shared__ char smem_raw[];
    char* smem = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x0 = blockIdx.x * T::TX, y0 = blockIdx.y * T::TY;
    const int z0 = blockIdx.z * a.kz, z1 = min(z0 + a.kz, a.nz);
    const int n_it = z1 - z0;
    const bool edge = x0 == 0 || x0 + T::TX >= a.nx || y0 == 0 || y0 + T::TY >= a.ny;
    const uint32_t bars = smem_u32(smem + T::OffBar);
    auto full = [&](int s) { return bars + 8 * s; };
    auto empty = [&](int s) { return bars + 8 * (3 + s); };
    auto ofull = [&](int b) { return bars + 8 * (6 + b); };
    auto oempty = [&](int b) { return bars + 8 * (8 + b); };

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), T::Warps);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(ofull(b), T::Warps);
            mbar_init(oempty(b), 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    pdl_wait();

    if (warp == T::Warps) {
        // ------------------------------------------------ producer warp
        if (lane != 0) return;
        issue_stage<T>(a, &tm9, &tm5, &tm_m, smem, 0, z0, z0 - 1, z0 + 1, x0, y0);
        if (n_it > 1) issue_stage<T>(a, &tm9, &tm5, &tm_m, smem, 1, z0 + 1, z0 + 2, z0 + 2, x0, y0);
        int issued = n_it > 1 ? 2 : 1;
        bool ok = true;
        for (int it = 0; it < n_it && ok; ++it) {
            const int k = z0 + it;
            // output buffer it & 1: the store issued in the previous
            // iteration (plane k - 2) has read it
            asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
            mbar_arrive(oempty(it & 1));
            if (it > 0) {
                ok = mbar_wait(ofull((it - 1) & 1), (uint32_t)(((it - 1) >> 1) & 1));
                if (!ok) break;
                tma_store4(&tm_out, smem_u32(smem + T::OffOut + ((it - 1) & 1) * T::OutBytes), x0, y0, k - 1, 0);
                bulk_commit();
            }
            if (issued < n_it) {
                // stage it + 2 reuses the buffers of iteration it - 1
                if (it > 0) ok = mbar_wait(empty((it - 1) % kStages), (uint32_t)(((it - 1) / kStages) & 1));
                if (!ok) break;
                fence_async_smem();
                const int kn = z0 + issued;
                issue_stage<T>(a, &tm9, &tm5, &tm_m, smem, issued % kStages, kn, kn + 1, kn + 1, x0, y0);
                ++issued;
            }
        }
        if (ok && n_it > 0) ok = mbar_wait(ofull((n_it - 1) & 1), (uint32_t)(((n_it - 1) >> 1) & 1));
        if (ok && n_it > 0) {
            tma_store4(&tm_out, smem_u32(smem + T::OffOut + ((n_it - 1) & 1) * T::OutBytes), x0, y0, z1 - 1, 0);
            bulk_commit();
        }
        if (!ok) {
            atomicOr(&g_lb_tma_status, 1u);
            // wait (bounded) for every copy issued into this block's buffers
            for (int it = 0; it < issued; ++it) mbar_wait(full(it % kStages), (uint32_t)((it / kStages) & 1));
        }
        bulk_wait_all();
        return;
    }

    // ------------------------------------------------ compute warps
    const int tx = threadIdx.x % T::TX, ty = threadIdx.x / T::TX;
    const int i = x0 + tx, j = y0 + ty;
    const bool live = i < a.nx && j < a.ny;
    Patch<T> pt;
    RingHalo<T> rh;
    if (edge) patch_plan<T>(pt, a, x0, y0);
    ring_plan<T>(rh, a, x0, y0, edge);
    // plane z0: its stage's wrapped halo and the records of z0 - 1 .. z0 + 1;
    // its force row
    bool forced = false;
    float4 gg = make_float4(0.f, 0.f, 0.f, 0.f);
    if (live && n_it > 0) {
        forced = a.flags[z0 * a.ny + j] != 0u;
        if (forced) gg = a.g[((long long)z0 * a.ny + j) * a.nx + i];
    }
    if (edge) patch_gather<T>(pt, a, z0);
    bool ok = n_it == 0 || mbar_wait(full(0), 0u);
    if (ok && n_it > 0) {
        if (edge) patch_scatter<T>(pt, a, smem, 0, z0);
        for (int p = z0 - 1; p <= z0 + 1; ++p) {
            if (p < 0 || p >= a.nz) continue;
            ring_gather<T>(rh, a, p);
            ring_convert<T>(rh, smem, p);
        }
    }
    for (int it = 0; it < n_it; ++it) {
        const int k = z0 + it, s = it % kStages, b = it & 1;
        ok = __all_sync(0xffffffffu, ok);
        compute_sync<T>();
        if (!ok) {
            if (lane == 0) atomicOr(&g_lb_tma_status, 1u);
            break;
        }
        // early loads for the next plane: its force flag, its stage's wrapped
        // halo, the outside records of plane k + 2
        const bool next = it + 1 < n_it;
        const bool fnext = live && next && a.flags[(k + 1) * a.ny + j] != 0u;
        if (next) {
            if (edge) patch_gather<T>(pt, a, k + 1);
            ring_gather<T>(rh, a, k + 2);
        }
        const long long cell = ((long long)k * a.ny + j) * a.nx + i;
        ok = mbar_wait(oempty(b), (uint32_t)((it >> 1) & 1));
        if (ok && live) {
            if (k == 0)
                cell_step<kMode, T, 1>(a, smem, s, b, k, tx, ty, cell, forced, gg);
            else if (k == a.nz - 1)
                cell_step<kMode, T, 2>(a, smem, s, b, k, tx, ty, cell, forced, gg);
            else
                cell_step<kMode, T, 0>(a, smem, s, b, k, tx, ty, cell, forced, gg);
        }
        fence_async_smem();   // the output tile is read by the TMA store
        __syncwarp();
        if (lane == 0) {
            mbar_arrive(empty(s));
            mbar_arrive(ofull(b));
        }
        // the next plane's force, read now and used in the next iteration
        forced = fnext;
        if (forced) gg = a.g[cell + (long long)a.ny * a.nx];
        // prepare plane k + 1: its stage's wrapped halo, the records of k + 2
        if (ok && next) {
            ok = mbar_wait(full((it + 1) % kStages), (uint32_t)(((it + 1) / kStages) & 1));
            if (ok) {
                if (edge) patch_scatter<T>(pt, a, smem, (it + 1) % kStages, k + 1);
                if (k + 2 < a.nz) ring_convert<T>(rh, smem, k + 2);
            }
        }
    }
}

using Tile32x8 = TmaTile<32, 8>;
using Tile32x4 = TmaTile<32, 4>;

// ---------------------------------------------------------------- host side
typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn()
{
    static EncodeTiled fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    }
    return fn;
}

// Tensor maps of the two ping-pong buffers, for each tile shape:
// [buffer] x {stored-value tiles with halo (load), stored-value tiles
// (store), records with halo (load)}.
struct TmaMaps {
    // per buffer: nine-slot and five-slot group boxes with halo (loads), the
    // 19 output tiles (store), the records with halo (load)
    CUtensorMap n9[2], n5[2], n_store[2], m_load[2];
};
}  // namespace

struct LbTma {
    TmaMaps set[2];   // 0: 32 x 8 columns, 1: 32 x 4
};

namespace {

template <class T>
bool encode_maps(TmaMaps* t, const LbCtx* c)
{
    EncodeTiled enc = encode_fn();
    if (!enc) return false;
    const lb_params& p = c->p;
    const cuuint64_t nx = p.nx, ny = p.ny, nz = p.nz;
    const cuuint32_t es[4] = {1, 1, 1, 1};
    auto ok = [](CUresult r) { return r == CUDA_SUCCESS; };
    for (int b = 0; b < 2; ++b) {
        const cuuint64_t dims[4] = {nx, ny, nz, 19};
        const cuuint64_t strides[3] = {nx * 2, nx * ny * 2, nx * ny * nz * 2};
        const cuuint32_t box9[4] = {(cuuint32_t)T::WX, (cuuint32_t)T::HY, 1, 9};
        const cuuint32_t box5[4] = {(cuuint32_t)T::WX, (cuuint32_t)T::HY, 1, 5};
        const cuuint32_t box_s[4] = {(cuuint32_t)T::TX, (cuuint32_t)T::TY, 1, 19};
        if (!ok(enc(&t->n9[b], CU_TENSOR_MAP_DATA_TYPE_UINT16, 4, c->f[b], dims, strides, box9, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE)) ||
            !ok(enc(&t->n5[b], CU_TENSOR_MAP_DATA_TYPE_UINT16, 4, c->f[b], dims, strides, box5, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE)) ||
            !ok(enc(&t->n_store[b], CU_TENSOR_MAP_DATA_TYPE_UINT16, 4, c->f[b], dims, strides, box_s, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE)))
            return false;
        const cuuint64_t mdims[4] = {4, nx, ny, nz};
        const cuuint64_t mstrides[3] = {16, nx * 16, nx * ny * 16};
        const cuuint32_t mbox[4] = {4, (cuuint32_t)T::HX, (cuuint32_t)T::HY, 1};
        if (!ok(enc(&t->m_load[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, c->m[b], mdims, mstrides, mbox, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE)))
            return false;
    }
    return true;
}

template <int kMode, class T>
cudaError_t launch_tma(const LbCtx* c, const TmaMaps* t, cudaStream_t s, float omega, float guo, float3 body,
                       float3 utop, float inv_scale)
{
    const lb_params& p = c->p;
    const int a = c->cur, b = c->cur ^ 1;
    static bool attr_set = false;   // one attribute per instantiation
    if (!attr_set) {
        const cudaError_t e = cudaFuncSetAttribute(k_lb_step_tma<kMode, T>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, T::SmemBytes);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int tiles = ((p.nx + T::TX - 1) / T::TX) * ((p.ny + T::TY - 1) / T::TY);
    // columns march through kz planes: about eight waves of the resident
    // blocks, so that the last wave is short and the copies of a column's
    // first planes are paid once per kz planes
    const long long resident = 148LL * T::MinBlocks;
    const long long want = resident * 8;
    int kz = (int)std::max<long long>(2, ((long long)tiles * p.nz + want - 1) / want);
    kz = std::min(kz, p.nz);
    StepArgs args;
    args.nin = (const uint16_t*)c->f[a];
    args.min_ = c->m[a];
    args.mout = c->m[b];
    args.g = c->g;
    args.flags = c->flags;
    args.nx = p.nx;
    args.ny = p.ny;
    args.nz = p.nz;
    args.kz = kz;
    args.omega = omega;
    args.guo = guo;
    args.inv_scale = inv_scale;
    args.body = body;
    args.utop = utop;
    args.onsite = p.walls;
    const dim3 grid((p.nx + T::TX - 1) / T::TX, (p.ny + T::TY - 1) / T::TY, (p.nz + kz - 1) / kz);
    return launch_pdl(k_lb_step_tma<kMode, T>, grid, dim3(T::Block), (size_t)T::SmemBytes, s, t->n9[a], t->n5[a],
                      t->n_store[b], t->m_load[a], args);
}

}  // namespace

bool lb_tma_supported(const LbCtx* c)
{
    const lb_params& p = c->p;
    // TMA rows start on 16-byte boundaries: the row pitch of the 16-bit
    // tensor (2 nx bytes) must be a multiple of 16
    return (p.storage == PFSI_LB_BF16 || p.storage == PFSI_LB_FP16) && p.nx % 8 == 0 && p.nx >= 8 && p.ny >= 2 &&
           p.nz >= 3;
}

LbTma* lb_tma_create(const LbCtx* c)
{
    if (!lb_tma_supported(c)) return nullptr;
    LbTma* t = new LbTma();
    std::memset(t, 0, sizeof(LbTma));
    if (!encode_maps<Tile32x8>(&t->set[0], c) || !encode_maps<Tile32x4>(&t->set[1], c)) {
        delete t;
        return nullptr;
    }
    return t;
}

void lb_tma_destroy(LbTma* t) { delete t; }

cudaError_t lb_tma_launch(const LbCtx* c, const LbTma* t, int tile, cudaStream_t s, float omega, float guo,
                          float3 body, float3 utop, float inv_scale)
{
    const bool bf16 = c->p.storage == PFSI_LB_BF16;
    if (tile == 1)
        return bf16 ? launch_tma<PFSI_LB_BF16, Tile32x4>(c, &t->set[1], s, omega, guo, body, utop, inv_scale)
                    : launch_tma<PFSI_LB_FP16, Tile32x4>(c, &t->set[1], s, omega, guo, body, utop, inv_scale);
    return bf16 ? launch_tma<PFSI_LB_BF16, Tile32x8>(c, &t->set[0], s, omega, guo, body, utop, inv_scale)
                : launch_tma<PFSI_LB_FP16, Tile32x8>(c, &t->set[0], s, omega, guo, body, utop, inv_scale);
}

int lb_tma_status(unsigned int* out, bool clear)
{
    int rc = check_cuda(cudaMemcpyFromSymbol(out, g_lb_tma_status, sizeof(unsigned int)), "lb_tma_status: copy");
    if (!rc && clear) {
        const unsigned int zero = 0;
        rc = check_cuda(cudaMemcpyToSymbol(g_lb_tma_status, &zero, sizeof(zero)), "lb_tma_status: clear");
    }
    return rc;
}

}  // namespace pfsi
