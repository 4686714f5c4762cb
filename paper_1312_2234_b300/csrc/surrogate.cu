// surrogate.cu -- learned membrane-force surrogate for sm_103a (no paper
// counterpart: a 42 -> 128 -> 128 -> 18 GELU network that sets the element
// stresses of the local membrane terms of Section 3.1, springs Eq. 2-3, local
// area Eq. 4, bending).
//
// The local energy is split into node shares: membrane node i owns, per
// one-ring slot k, half the spring of its spoke (i, n_k), a third of the area
// term of its fan triangle (i, n_k, n_{k+1}) and half the bending of its
// spoke (torsion of n_{k+1} - i - n_k - n_{k-1}).  One thread per node gathers
// the one-ring (split hi/lo positions), forms the 18 element strains
// (stretch (L - L0)/L0, area (S - S0)/S0, bending angle phi - phi0) from
// small quantities only (the edge change d = e - e0 from the split positions,
// L^2 - L0^2 = d.(2 e0 + d), |c|^2 - |c0|^2 = dc.(2 c0 + dc)), and feeds the
// network their direction and the slot's rest descriptors.  The output sets
// the stresses y = x * m * out_scale * o (m = L0^2, S0, 1), and the node's
// force contributions y dx/dX (exact strain gradients: spoke unit vectors,
// triangle area gradients, torsion gradients) go to the node and its
// one-ring by atomic adds.
//
// Dense layers: one tcgen05 kernel, C = A B^T with both operands BF16 and
// K-contiguous in global memory (every layer of the forward and backward pass
// and every weight gradient is such a product; the backward pass keeps
// transposed copies of the activations for that).  A CTA of 128 threads owns
// a 128-row tile and all N <= 128 columns, stages 64-wide K chunks of A and B
// in shared memory in the no-swizzle K-major core-matrix layout (8 rows x 16
// bytes per core matrix, LBO = 128 B along K, SBO = 1024 B along rows), one
// elected thread issues the kind::f16 MMAs into an FP32 TMEM accumulator and
// commits them to an mbarrier per stage (two stages: the next chunk loads
// while the tensor core works), and every thread then reads its row back
// with tcgen05.ld and applies a fused epilogue (bias + GELU, GELU' product,
// output layer, or a split-K partial).  Waits on the mbarriers are bounded;
// a timeout sets an error flag and the CTA frees its TMEM and returns.
//
// Inference inside the coupled step is one persistent kernel per step: each
// CTA keeps W1, W2, W3 in shared memory and, per 128-node tile, computes the
// strains and inputs into a shared input tile, runs the three layers through
// TMEM (the GELU epilogues write BF16 activations back to shared memory for
// the next MMA) and scatters the stress forces.
//
// An FP32 check path runs the same layer sequence with the same epilogues on
// CUDA cores (plain dot products, FP32 activations), so the training pipeline
// can be compared with the FP64 reference at FP32 precision.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "ff.cuh"
#include "pfsi_internal.cuh"

namespace pfsi {

namespace {

using bf16 = __nv_bfloat16;

constexpr int kIn = PFSI_SG_IN, kInPad = PFSI_SG_IN_PAD, kHid = PFSI_SG_HID, kOut = PFSI_SG_OUT,
              kOutPad = PFSI_SG_OUT_PAD;
constexpr int kTile = 128;     // rows per CTA (MMA M)
constexpr int kChunkK = 64;    // K per shared-memory stage
constexpr int kMaxSplit = 148;

static_assert(PFSI_SG_W1 == 0 && PFSI_SG_B1 == PFSI_SG_W1 + kHid * kInPad && PFSI_SG_W2 == PFSI_SG_B1 + kHid &&
                  PFSI_SG_B2 == PFSI_SG_W2 + kHid * kHid && PFSI_SG_W3 == PFSI_SG_B2 + kHid &&
                  PFSI_SG_B3 == PFSI_SG_W3 + kOutPad * kHid && PFSI_SG_N_TRAINED == PFSI_SG_B3 + kOutPad &&
                  PFSI_SG_IN_SHIFT == PFSI_SG_N_TRAINED && PFSI_SG_IN_SCALE == PFSI_SG_IN_SHIFT + kInPad &&
                  PFSI_SG_OUT_SCALE == PFSI_SG_IN_SCALE + kInPad && PFSI_SG_TGT_SCALE == PFSI_SG_OUT_SCALE + kOutPad &&
                  PFSI_SG_N_FLOATS == PFSI_SG_TGT_SCALE + kOutPad,
              "parameter layout");
constexpr int kStrain = 18;    // element strains per row (= outputs)
constexpr int kTgt = 2 * kStrain;
static_assert(kOut == kStrain && kIn == kStrain + 24 && kIn < kInPad, "input layout");
constexpr size_t kShadowOff = ((size_t)PFSI_SG_N_FLOATS * 4 + 255) / 256 * 256;
constexpr int hW1 = 0, hW2 = hW1 + kHid * kInPad, hW3 = hW2 + kHid * kHid, hW2t = hW3 + kOutPad * kHid,
              hW3t = hW2t + kHid * kHid, nShadow = hW3t + kHid * kOutPad;
static_assert(kShadowOff + (size_t)nShadow * 2 == PFSI_SG_PARAM_BYTES, "parameter buffer size");

struct Params {
    const float* p;      // FP32 master block
    const bf16* h;       // BF16 shadows
};
inline Params params_of(const void* buf)
{
    return {reinterpret_cast<const float*>(buf),
            reinterpret_cast<const bf16*>(reinterpret_cast<const char*>(buf) + kShadowOff)};
}

// ------------------------------------------------------------------ GELU (tanh form)
// kFast: the hardware tanh approximation (BF16 mode, where every activation is
// rounded to BF16 right after); otherwise tanhf (FP32 check mode).
template <bool kFast>
__device__ __forceinline__ float tanh_t(float u)
{
    if (kFast) {
        float t;
        asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(u));
        return t;
    }
    return tanhf(u);
}
template <bool kFast>
__device__ __forceinline__ float gelu_f(float z)
{
    const float u = 0.7978845608028654f * fmaf(0.044715f * z, z * z, z);
    return 0.5f * z * (1.0f + tanh_t<kFast>(u));
}
template <bool kFast>
__device__ __forceinline__ float gelu_grad_f(float z)
{
    const float u = 0.7978845608028654f * fmaf(0.044715f * z, z * z, z);
    const float t = tanh_t<kFast>(u);
    const float du = 0.7978845608028654f * fmaf(3.0f * 0.044715f, z * z, 1.0f);
    return 0.5f * (1.0f + t) + 0.5f * z * (1.0f - t * t) * du;
}

// GELU of 16 pre-activations into 8 BF16 pairs: u = z (c1 + c3 z^2),
// g = h + h tanh(u) with h = z / 2 (hardware tanh; the result is rounded to
// BF16 right after).
__device__ __forceinline__ void gelu16_bf16(const float* z, uint32_t* out)
{
    // the same operations as gelu_f's fast form, two activations per packed
    // f32x2 instruction (each lane is one correctly rounded operation)
    constexpr float c1 = 0.7978845608028654f, c3 = 0.7978845608028654f * 0.044715f;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float2 x = make_float2(z[2 * q], z[2 * q + 1]);
        const float2 u = __fmul2_rn(x, __ffma2_rn(make_float2(c3, c3), __fmul2_rn(x, x), make_float2(c1, c1)));
        float2 t;
        asm("tanh.approx.f32 %0, %1;" : "=f"(t.x) : "f"(u.x));
        asm("tanh.approx.f32 %0, %1;" : "=f"(t.y) : "f"(u.y));
        const float2 h = __fmul2_rn(make_float2(0.5f, 0.5f), x);
        const float2 g = __ffma2_rn(h, t, h);
        const __nv_bfloat162 b = __float22bfloat162_rn(g);
        out[q] = *reinterpret_cast<const uint32_t*>(&b);
    }
}

template <class T>
__device__ __forceinline__ T to_t(float x);
template <>
__device__ __forceinline__ float to_t<float>(float x) { return x; }
template <>
__device__ __forceinline__ bf16 to_t<bf16>(float x) { return __float2bfloat16_rn(x); }
__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(bf16 x) { return __bfloat162float(x); }

// 16 consecutive values of a row, stored with 16-byte vector stores.
__device__ __forceinline__ void store16(float* dst, const float* v)
{
#pragma unroll
    for (int q = 0; q < 4; ++q)
        reinterpret_cast<float4*>(dst)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}
__device__ __forceinline__ void store16(bf16* dst, const float* v)
{
    uint32_t w[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
        w[q] = *reinterpret_cast<const uint32_t*>(&h);
    }
    reinterpret_cast<uint4*>(dst)[0] = make_uint4(w[0], w[1], w[2], w[3]);
    reinterpret_cast<uint4*>(dst)[1] = make_uint4(w[4], w[5], w[6], w[7]);
}
__device__ __forceinline__ void load16(const float* src, float* v)
{
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 a = reinterpret_cast<const float4*>(src)[q];
        v[4 * q] = a.x;
        v[4 * q + 1] = a.y;
        v[4 * q + 2] = a.z;
        v[4 * q + 3] = a.w;
    }
}

// ------------------------------------------------------------------ epilogues
// operator() is applied to one accumulator element (row, column n) of
// C = A B^T (FP32 path); row16 to 16 consecutive columns n0.. of a row
// (tensor-core path, vector stores).  `split` is the K-split index.

// hidden layer: z = acc + b; h = gelu(z)
template <class T>
struct EpiHidden {
    static constexpr bool kFast = sizeof(T) == 2;
    const float* bias;
    float* Z;    // [rows][128] pre-activations (null: not kept)
    T* H;        // [rows][128]
    T* Ht;       // [128][ldt] (null: no transposed copy)
    int ldt;
    __device__ void operator()(int row, int n, float acc, int) const
    {
        const float z = acc + bias[n];
        if (Z) Z[(size_t)row * kHid + n] = z;
        const float h = gelu_f<kFast>(z);
        H[(size_t)row * kHid + n] = to_t<T>(h);
        if (Ht) Ht[(size_t)n * ldt + row] = to_t<T>(h);
    }
    __device__ void row16(int row, int n0, const float* v, int) const
    {
        float z[16], h[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            z[j] = v[j] + bias[n0 + j];
            h[j] = gelu_f<kFast>(z[j]);
        }
        if (Z) store16(Z + (size_t)row * kHid + n0, z);
        store16(H + (size_t)row * kHid + n0, h);
        if (Ht)
#pragma unroll
            for (int j = 0; j < 16; ++j) Ht[(size_t)(n0 + j) * ldt + row] = to_t<T>(h[j]);
    }
};

// output layer: o = acc + b3
struct EpiOut {
    const float* bias;
    float* O;    // [rows][16]
    __device__ void operator()(int row, int n, float acc, int) const { O[(size_t)row * kOutPad + n] = acc + bias[n]; }
    __device__ void row16(int row, int n0, const float* v, int) const
    {
        float o[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) o[j] = v[j] + bias[n0 + j];
        store16(O + (size_t)row * kOutPad + n0, o);
    }
};

// backward through a hidden layer: dz = acc * gelu'(z)
template <class T>
struct EpiBack {
    static constexpr bool kFast = sizeof(T) == 2;
    const float* Z;
    T* D;        // [rows][128] (null: not kept)
    T* Dt;       // [128][ldt]
    int ldt;
    __device__ void operator()(int row, int n, float acc, int) const
    {
        const float d = acc * gelu_grad_f<kFast>(Z[(size_t)row * kHid + n]);
        if (D) D[(size_t)row * kHid + n] = to_t<T>(d);
        Dt[(size_t)n * ldt + row] = to_t<T>(d);
    }
    __device__ void row16(int row, int n0, const float* v, int) const
    {
        float z[16], d[16];
        load16(Z + (size_t)row * kHid + n0, z);
#pragma unroll
        for (int j = 0; j < 16; ++j) d[j] = v[j] * gelu_grad_f<kFast>(z[j]);
        if (D) store16(D + (size_t)row * kHid + n0, d);
#pragma unroll
        for (int j = 0; j < 16; ++j) Dt[(size_t)(n0 + j) * ldt + row] = to_t<T>(d[j]);
    }
};

// split-K partial of a weight gradient G (ld floats per row, size floats):
// G[row][n] = acc, or G[n][row] = acc when transposed
struct EpiPartial {
    float* part;
    int ld, size;
    bool transpose;
    __device__ void operator()(int row, int n, float acc, int split) const
    {
        float* P = part + (size_t)split * size;
        if (transpose)
            P[(size_t)n * ld + row] = acc;
        else
            P[(size_t)row * ld + n] = acc;
    }
    __device__ void row16(int row, int n0, const float* v, int split) const
    {
        float* P = part + (size_t)split * size;
        if (transpose) {
#pragma unroll
            for (int j = 0; j < 16; ++j) P[(size_t)(n0 + j) * ld + row] = v[j];
        } else {
            store16(P + (size_t)row * ld + n0, v);
        }
    }
};

// ------------------------------------------------------------------ tcgen05 / mbarrier helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the completion of the phase with the given parity: false
// after `limit` polls (the callers then record an error and stop).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int limit = 1 << 22)
{
    for (int it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void fence_barrier_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Shared-memory matrix descriptor: no swizzle, K-major core matrices.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version bits 46-48 = 0b001
    return d;                  // base offset 0, relative LBO, swizzle none
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, M = 128, N given.
__host__ __device__ constexpr uint32_t idesc_bf16(int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kTile >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// Copy rows [0, nrows) x K range [k0, k0 + kc) of a row-major BF16 matrix
// into the core-matrix layout of one stage (kc a multiple of 16).
__device__ __forceinline__ void stage_fill(uint8_t* dst, const bf16* __restrict__ src, int ld, int row0, int nrows,
                                           int k0, int kc)
{
    const int cpr = kc >> 3;   // 16-byte chunks per row
    for (int q = threadIdx.x; q < nrows * cpr; q += kTile) {
        const int r = q / cpr, kg = q - r * cpr;
        const uint4 val = *reinterpret_cast<const uint4*>(src + (size_t)(row0 + r) * ld + k0 + 8 * kg);
        *reinterpret_cast<uint4*>(dst + (((r >> 3) * (kChunkK / 8) + kg) << 7) + ((r & 7) << 4)) = val;
    }
}

// C[rows x N] = A[rows x K] B[N x K]^T; grid (rows / 128, splits); each CTA
// takes K range [split * k_per, min(K, (split + 1) * k_per)).
template <int N, class Epi>
__global__ void __launch_bounds__(kTile) k_gemm_tc(const bf16* __restrict__ A, int lda, const bf16* __restrict__ B,
                                                   int ldb, int K, int k_per, Epi epi, int* __restrict__ err)
{
    static_assert(N == 16 || N == 32 || N == 64 || N == 128, "N");
    constexpr uint32_t kCols = N < 32 ? 32 : N;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* sA = smem;                                 // 2 stages x 16 KB
    uint8_t* sB = smem + 2 * kTile * kChunkK * 2;       // 2 stages x N * 128 B
    __shared__ uint64_t bar[2];
    __shared__ uint32_t tmem_sh;

    const int m0 = blockIdx.x * kTile;
    const int kb = blockIdx.y * k_per, ke = min(K, kb + k_per);
    const int nchunks = ke > kb ? (ke - kb + kChunkK - 1) / kChunkK : 0;
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_barrier_init();
    }
    if (threadIdx.x < 32) tmem_alloc(&tmem_sh, kCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_sh;

    bool ok = true;
    for (int c = 0; c < nchunks && ok; ++c) {
        const int s = c & 1;
        if (c >= 2) {   // stage s free again (one thread polls)
            ok = __syncthreads_and(threadIdx.x == 0 ? mbar_wait(&bar[s], ((c - 2) >> 1) & 1) : true) != 0;
            if (!ok) break;
        }
        const int k0 = kb + c * kChunkK, kc = min(kChunkK, ke - k0);
        stage_fill(sA + s * kTile * kChunkK * 2, A, lda, m0, kTile, k0, kc);
        stage_fill(sB + s * N * kChunkK * 2, B, ldb, 0, N, k0, kc);
        fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(sA + s * kTile * kChunkK * 2), b0 = smem_u32(sB + s * N * kChunkK * 2);
            for (int j = 0; j < kc / 16; ++j)
                mma_bf16(tmem, smem_desc(a0 + 256 * j, 128, 1024), smem_desc(b0 + 256 * j, 128, 1024), idesc_bf16(N),
                         (c > 0 || j > 0) ? 1u : 0u);
            mma_commit(&bar[s]);
        }
    }
    if (ok && nchunks > 0)
        ok = __syncthreads_and(threadIdx.x == 0 ? mbar_wait(&bar[(nchunks - 1) & 1], ((nchunks - 1) >> 1) & 1)
                                                : true) != 0;
    tc_fence_after();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = m0 + warp * 32 + lane;
    if (ok) {
#pragma unroll 1
        for (int n0 = 0; n0 < N; n0 += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)n0, v);
            if (nchunks == 0)
                for (int j = 0; j < 16; ++j) v[j] = 0.f;
            epi.row16(row, n0, v, blockIdx.y);
        }
    } else if (lane == 0) {
        atomicExch(err, 1);
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) {
        tc_fence_after();
        tmem_dealloc(tmem, kCols);
    }
}

// FP32 check path: one thread per output element, A(row, k) = A[row*sar + k*sak],
// B(n, k) = B[n*sbn + k*sbk]; K range per split as in the tensor-core kernel.
template <class Epi>
__global__ void k_gemm_f32(const float* __restrict__ A, long long sar, long long sak, const float* __restrict__ B,
                           long long sbn, long long sbk, int rows, int N, int K, int k_per, Epi epi)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)rows * N) return;
    const int row = (int)(t / N), n = (int)(t % N);
    const int kb = blockIdx.y * k_per, ke = min(K, kb + k_per);
    float acc = 0.f;
    for (int k = kb; k < ke; ++k) acc = fmaf(A[row * sar + k * sak], B[n * sbn + k * sbk], acc);
    epi(row, n, acc, blockIdx.y);
}

// ------------------------------------------------------------------ loss, reductions, Adam
// Stress error per output: e = a o - b (target row: a[18], b[18]);
// dO = 2 a e / (18 B) in columns 0..17 (zero in 18..31), row-major and
// transposed; loss += sum e^2 / (18 B).
template <class T>
__global__ void k_sg_loss(const float* __restrict__ O, const float* __restrict__ target, int B, int rows,
                          T* __restrict__ dO, T* __restrict__ dOt, double* __restrict__ loss)
{
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    double sq = 0.0;
    if (row < rows) {
        for (int n = 0; n < kOutPad; ++n) {
            float d = 0.f;
            if (n < kOut && row < B) {
                const float a = target[(size_t)row * kTgt + n], b = target[(size_t)row * kTgt + kStrain + n];
                const float e = fmaf(a, O[(size_t)row * kOutPad + n], -b);
                d = 2.0f * a * e / ((float)kOut * (float)B);
                sq += (double)e * (double)e;
            }
            dO[(size_t)row * kOutPad + n] = to_t<T>(d);
            dOt[(size_t)n * rows + row] = to_t<T>(d);
        }
    }
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, o);
    if ((threadIdx.x & 31) == 0 && sq != 0.0) atomicAdd(loss, sq / ((double)kOut * (double)B));
}

// out[r] = sum over c < cols of M[r * ld + c] (one warp per row, fixed order)
template <class T>
__global__ void k_rowsum(const T* __restrict__ M, int rows, int cols, int ld, float* __restrict__ out)
{
    const int r = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (r >= rows) return;
    float s = 0.f;
    for (int c = threadIdx.x & 31; c < cols; c += 32) s += to_f(M[(size_t)r * ld + c]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) out[r] = s;
}

__global__ void k_reduce_splits(const float* __restrict__ part, int splits, int count, float* __restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    float s = 0.f;
    for (int k = 0; k < splits; ++k) s += part[(size_t)k * count + i];
    out[i] = s;
}

// inputs [rows][64] -> transposed copy [64][rows]
template <class T>
__global__ void k_transpose_in(const T* __restrict__ X, int rows, T* __restrict__ Xt)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= rows * kInPad) return;
    const int c = t / rows, r = t - c * rows;
    Xt[t] = X[(size_t)r * kInPad + c];
}

__global__ void k_sg_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                          float* __restrict__ v, int count, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float gi = g[i];
    const float mi = fmaf(b1, m[i], (1.0f - b1) * gi);
    const float vi = fmaf(b2, v[i], (1.0f - b2) * gi * gi);
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void k_sg_shadows(const float* __restrict__ p, bf16* __restrict__ h)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kHid * kInPad) h[hW1 + i] = __float2bfloat16_rn(p[PFSI_SG_W1 + i]);
    if (i < kHid * kHid) {
        h[hW2 + i] = __float2bfloat16_rn(p[PFSI_SG_W2 + i]);
        const int r = i / kHid, c = i % kHid;   // W2t[c][r] = W2[r][c]
        h[hW2t + c * kHid + r] = __float2bfloat16_rn(p[PFSI_SG_W2 + i]);
    }
    if (i < kOutPad * kHid) {
        h[hW3 + i] = __float2bfloat16_rn(p[PFSI_SG_W3 + i]);
        const int r = i / kHid, c = i % kHid;   // W3t[c][r] = W3[r][c]
        h[hW3t + c * kOutPad + r] = __float2bfloat16_rn(p[PFSI_SG_W3 + i]);
    }
}

// ------------------------------------------------------------------ features
struct SgDev {
    int n_nodes;          // mesh nodes
    int rows;             // surrogate nodes
    int rows_pad;         // multiple of 128
    const int* node;      // [rows_pad] (-1 padding)
    const int* ring;      // [rows][6] (-1 padding)
    const float* rest;    // [rows][64]: rest record (see build_rings)
};

__device__ __forceinline__ float3 f3(const float* p) { return make_float3(p[0], p[1], p[2]); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b)
{
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 add3(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 sub3(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 scale3(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }

// a[i] for a runtime i in [0, 6) (selects: the array stays in registers)
__device__ __forceinline__ float3 pick6(const float3 (&a)[6], int i)
{
    float3 r = a[0];
#pragma unroll
    for (int j = 1; j < 6; ++j)
        if (i == j) r = a[j];
    return r;
}
__device__ __forceinline__ void sub_at6(float3 (&a)[6], int i, float3 v)
{
#pragma unroll
    for (int j = 0; j < 6; ++j)
        if (i == j) a[j] = sub3(a[j], v);
}

// One row's one-ring: node, neighbours (-1 beyond the degree), degree and
// the current spoke vectors e_k = X[n_k] - X[v].
struct RowRing {
    int v, deg;
    int nb[6];
    float3 e[6];
};

// Torsion of the chain r1 - 0 - r3 - r4 (points relative to the second):
// F = r1, G = -r3, H = r4 - r3, A = F x G, B = H x G,
// cos = A.B / (|A||B|), sin = (B x A).G / (|A||B||G|).
// (The surrogate's geometry uses the hardware reciprocal square root and the
// fast division intrinsic, ~2 ulp each.)
__device__ __forceinline__ void torsion_cs(float3 r1, float3 r3, float3 r4, float& c, float& s)
{
    const float3 G = scale3(-1.f, r3), H = sub3(r4, r3);
    const float3 A = cross3(r1, G), B = cross3(H, G);
    const float iab = rsqrtf(dot3(A, A) * dot3(B, B));
    c = dot3(A, B) * iab;
    s = dot3(cross3(B, A), G) * iab * rsqrtf(dot3(G, G));
}

// Its gradient with respect to the four points (Blondel and Karplus 1996).
__device__ __forceinline__ void torsion_grad(float3 r1, float3 r3, float3 r4, float3 g[4])
{
    const float3 G = scale3(-1.f, r3), H = sub3(r4, r3);
    const float3 A = cross3(r1, G), B = cross3(H, G);
    const float G2 = dot3(G, G), rg = rsqrtf(G2), gn = G2 * rg;
    const float iA = __fdividef(1.0f, dot3(A, A)), iB = __fdividef(1.0f, dot3(B, B));
    const float FG = dot3(r1, G) * iA * rg, HG = dot3(H, G) * iB * rg;
    const float ka = gn * iA, kb = gn * iB;
    g[0] = scale3(-ka, A);
    g[3] = scale3(kb, B);
    g[1] = sub3(scale3(ka + FG, A), scale3(HG, B));
    g[2] = add3(scale3(-FG, A), scale3(HG - kb, B));
}

// Element strains x[18] of surrogate row r (stretch, area strain and bending
// angle of slots 0..5; zero for empty slots), its one-ring, and the rest
// values of its slots.  xa, xb: positions split into hi/lo floats, [n] (x, y,
// z, 0).
//
// The strains are small differences of O(1) quantities, so they are formed
// from small quantities only: d_k = e_k - e0_k from the split positions and
// the split rest edge (exact to ~1e-7 of |d_k|), L^2 - L0^2 = d.(2 e0 + d),
// and for the fan triangle (c = e_k x e_{k+1}) |c|^2 - |c0|^2 = dc.(2 c0 + dc)
// with dc = d_k x e0_{k+1} + e0_k x d_{k+1} + d_k x d_{k+1}.  The bending
// angle is atan2 of sin and cos of phi - phi0 (absolute error ~1e-7).
__device__ __forceinline__ void row_strains(const float4* __restrict__ xa, const float4* __restrict__ xb,
                                            const SgDev& d, int r, RowRing& g, float* x, float* L0, float* S0,
                                            float* cph, float* sph, float& inv_l)
{
    const int v = d.node[r];
    const float4 vh = xa[v], vl = xb[v];
    float rest[64];
#pragma unroll
    for (int q = 0; q < 4; ++q) load16(d.rest + 64 * (size_t)r + 16 * q, rest + 16 * q);
    float3 dk[6], e0[6];
    int deg = 0;
    g.v = v;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const int nb = d.ring[6 * r + k];
        g.nb[k] = nb;
        e0[k] = f3(rest + 3 * k);
        if (nb >= 0) {
            const float4 uh = xa[nb], ul = xb[nb];
            const ff ex = ff_diff(uh.x, ul.x, vh.x, vl.x), ey = ff_diff(uh.y, ul.y, vh.y, vl.y),
                     ez = ff_diff(uh.z, ul.z, vh.z, vl.z);
            dk[k] = make_float3((ex.h - rest[3 * k]) + (ex.l - rest[18 + 3 * k]),
                                (ey.h - rest[3 * k + 1]) + (ey.l - rest[18 + 3 * k + 1]),
                                (ez.h - rest[3 * k + 2]) + (ez.l - rest[18 + 3 * k + 2]));
            deg = k + 1;
        } else {
            dk[k] = make_float3(0.f, 0.f, 0.f);
        }
        g.e[k] = add3(e0[k], dk[k]);
        cph[k] = rest[36 + k];
        sph[k] = rest[42 + k];
        L0[k] = rest[48 + k];
        S0[k] = rest[54 + k];
    }
    g.deg = deg;
    inv_l = rest[60];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        if (k < deg) {
            // stretch of spoke k
            const float dl2 = dot3(dk[k], add3(scale3(2.f, e0[k]), dk[k]));
            const float L2 = dot3(g.e[k], g.e[k]);
            const float L = L2 * rsqrtf(L2);
            x[k] = __fdividef(dl2, (L + L0[k]) * L0[k]);
            // area strain of the fan triangle (v, n_k, n_{k+1}); static
            // indices for the cyclic successor keep the arrays in registers
            const bool last = !(k < 5 && k + 1 < deg);
            const float3 e0n = last ? e0[0] : e0[k < 5 ? k + 1 : 0];
            const float3 dn = last ? dk[0] : dk[k < 5 ? k + 1 : 0];
            const float3 c0 = cross3(e0[k], e0n);
            const float3 dc = add3(add3(cross3(dk[k], e0n), cross3(e0[k], dn)), cross3(dk[k], dn));
            const float dS2 = dot3(dc, add3(scale3(2.f, c0), dc));
            const float3 cc = add3(c0, dc);
            const float c2 = dot3(cc, cc);
            const float S = 0.5f * c2 * rsqrtf(c2);
            x[6 + k] = __fdividef(dS2, 4.0f * (S + S0[k]) * S0[k]);
            // bending angle of spoke k: chain n_{k+1} - v - n_k - n_{k-1}
            const float3 en = last ? g.e[0] : g.e[k < 5 ? k + 1 : 0];
            const float3 ep = k > 0 ? g.e[k > 0 ? k - 1 : 0] : pick6(g.e, deg - 1);
            float c, s;
            torsion_cs(en, g.e[k], ep, c, s);
            x[12 + k] = atan2f(fmaf(s, cph[k], -c * sph[k]), fmaf(c, cph[k], s * sph[k]));
        } else {
            x[k] = x[6 + k] = x[12 + k] = 0.f;
        }
    }
}

// Network inputs f[64] of a row: the strain direction x s / |x s| (inputs
// 0..17) and the slots' rest descriptors L0/l, S0/l^2, cos phi0, sin phi0
// ((r - shift) * scale, inputs 18..41), zero for empty slots and beyond 41.
__device__ __forceinline__ void row_inputs(const float* x, int deg, const float* L0, const float* S0,
                                           const float* cph, const float* sph, float inv_l,
                                           const float* __restrict__ shift, const float* __restrict__ scale, float* f)
{
    float mm = 0.f;
#pragma unroll
    for (int j = 0; j < kStrain; ++j) {
        f[j] = x[j] * scale[j];
        mm = fmaf(f[j], f[j], mm);
    }
    const float inv = mm > 0.f ? rsqrtf(mm) : 0.f;
#pragma unroll
    for (int j = 0; j < kStrain; ++j) f[j] *= inv;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const float raw[4] = {L0[k] * inv_l, S0[k] * inv_l * inv_l, cph[k], sph[k]};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = kStrain + 6 * q + k;
            f[j] = k < deg ? (raw[q] - shift[j]) * scale[j] : 0.f;
        }
    }
#pragma unroll
    for (int j = kIn; j < kInPad; ++j) f[j] = 0.f;
}

// Factors q of the stresses' strain gradients: y_j dx_j/dX = (q_j o_j) G_j
// with G = e/L (spring, at n_k), the area gradient (area), the torsion
// gradient (bending): q_s = x_s L0 out_s (y_s / L0), q_a = x_a out_a
// (y_a / S0), q_b = x_b out_b.
__device__ __forceinline__ void stress_factors(const float* x, const float* L0, const float* __restrict__ out,
                                               float* q)
{
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        q[k] = x[k] * L0[k] * out[k];
        q[6 + k] = x[6 + k] * out[6 + k];
        q[12 + k] = x[12 + k] * out[12 + k];
    }
}

// The exact global area and volume terms of a row's own node: the platelet's
// coefficients cS = k_s (S - S0)/S0, cV = k_v (V - V0)/V0 and the node's
// position relative to the platelet's anchor (Eq. 4-5: F_v -= cS dS/dX_v +
// cV dV/dX_v, summed over the node's fan triangles).
struct RowGlobal {
    float cS, cV;
    float3 r;
    float wall;     // z force of the wall repulsion (Section 3.4.1) when the surrogate applies it, else 0
};

// The membrane context's data the global terms read.
struct GlobalArgs {
    const float2* coef;     // [nplt] (cS, cV)
    const int* node_plt;    // [n]
    const int* anchor;      // [nplt]
    int wall;               // nonzero: add the wall repulsion (a mesh without Morse pairs)
    float rep_F0, rep_tau, rep_eps_min, z_wall;
};

__device__ __forceinline__ RowGlobal row_global(const float4* __restrict__ xa, const float4* __restrict__ xb,
                                                const GlobalArgs& ga, int v)
{
    const int q = ga.node_plt[v];
    const float2 cf = ga.coef[q];
    const int o = ga.anchor[q];
    const float4 vh = xa[v], vl = xb[v], oh = xa[o], ol = xb[o];
    const ff dx = ff_diff(vh.x, vl.x, oh.x, ol.x), dy = ff_diff(vh.y, vl.y, oh.y, ol.y),
             dz = ff_diff(vh.z, vl.z, oh.z, ol.z);
    float wall = 0.f;
    if (ga.wall && ga.rep_F0 != 0.f) {   // the plain nodes pass's term, F0 tau / (e^{tau eps} - 1)
        const float eps = fmaxf((vh.z - ga.z_wall) + vl.z, ga.rep_eps_min);
        wall = ga.rep_F0 * ga.rep_tau / expm1f(ga.rep_tau * eps);
    }
    return {cf.x, cf.y, make_float3(dx.h + dx.l, dy.h + dy.l, dz.h + dz.l), wall};
}

// F -= sum_j p_j G_j of one row (p = q o), added to the node and its
// one-ring with atomic adds, plus the node's global area and volume terms.
// Area gradient of corner a of the fan triangle (v, n_k, n_{k+1}):
// (1/2) nhat x (P_{a+2} - P_{a+1}); volume gradient of corner v:
// (1/6) (P_{n_k} - o) x (P_{n_{k+1}} - o) = (1/6) (c + r x (e_{k+1} - e_k)).
__device__ __forceinline__ void row_scatter(const RowRing& g, const float* p, const RowGlobal& gl,
                                            float* __restrict__ F, int n)
{
    float3 Fi = make_float3(0.f, 0.f, 0.f);
    float3 Fn[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) Fn[k] = make_float3(0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        if (k < g.deg) {
            const bool last = !(k < 5 && k + 1 < g.deg);
            const int kn = last ? 0 : k + 1;
            const int kp = k > 0 ? k - 1 : g.deg - 1;
            const float3 ek = g.e[k];
            const float3 en = last ? g.e[0] : g.e[k < 5 ? k + 1 : 0];
            const float3 ep = k > 0 ? g.e[k > 0 ? k - 1 : 0] : pick6(g.e, g.deg - 1);
            // spring: -y_s dx_s/dX_{n_k} = -q_s o_s e/L, the opposite at v
            const float3 fs = scale3(p[k] * rsqrtf(dot3(ek, ek)), ek);
            Fn[k] = sub3(Fn[k], fs);
            Fi = add3(Fi, fs);
            // area: nhat x (.) / 2 with nhat = c / |c| (the own corner also
            // takes the global area coefficient), and the own volume term
            const float3 c = cross3(ek, en);
            const float ic = rsqrtf(dot3(c, c));
            const float h = 0.5f * p[6 + k] * ic;
            const float3 de = sub3(en, ek);
            Fi = sub3(Fi, scale3(0.5f * (p[6 + k] + gl.cS) * ic, cross3(c, de)));
            Fi = sub3(Fi, scale3(gl.cV * (1.0f / 6.0f), add3(c, cross3(gl.r, de))));
            Fn[k] = add3(Fn[k], scale3(h, cross3(c, en)));
            sub_at6(Fn, kn, scale3(h, cross3(c, ek)));
            // bending: chain n_{k+1} - v - n_k - n_{k-1}
            float3 tg[4];
            torsion_grad(en, ek, ep, tg);
            const float pb = p[12 + k];
            sub_at6(Fn, kn, scale3(pb, tg[0]));
            Fi = sub3(Fi, scale3(pb, tg[1]));
            Fn[k] = sub3(Fn[k], scale3(pb, tg[2]));
            sub_at6(Fn, kp, scale3(pb, tg[3]));
        }
    }
    atomicAdd(F + g.v, Fi.x);
    atomicAdd(F + n + g.v, Fi.y);
    atomicAdd(F + 2 * n + g.v, Fi.z + gl.wall);
#pragma unroll
    for (int k = 0; k < 6; ++k)
        if (k < g.deg) {
            const int u = g.nb[k];
            atomicAdd(F + u, Fn[k].x);
            atomicAdd(F + n + u, Fn[k].y);
            atomicAdd(F + 2 * n + u, Fn[k].z);
        }
}

// FP64 positions -> hi/lo float split, [3][n] each
__global__ void k_sg_split(const double* __restrict__ X, int n3, float* __restrict__ xh, float* __restrict__ xl)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n3) {
        const double x = X[t];
        const float h = __double2float_rn(x);
        xh[t] = h;
        xl[t] = __double2float_rn(x - (double)h);
    }
}

// hi/lo split positions [3][n] -> per-node float4 pairs (x, y, z, 0)
__global__ void k_sg_pack(const float* __restrict__ xh, const float* __restrict__ xl, int n, float4* __restrict__ xa,
                          float4* __restrict__ xb)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    xa[t] = make_float4(xh[t], xh[n + t], xh[2 * n + t], 0.f);
    xb[t] = make_float4(xl[t], xl[n + t], xl[2 * n + t], 0.f);
}

// Inputs (feat [rows][64]), strains (xs [rows][18]) and rest moduli scales
// (ms [rows][18]: L0^2, S0, 1; zero for empty slots) of every row.
template <class T>
__global__ void k_sg_features(const float4* __restrict__ xa, const float4* __restrict__ xb, SgDev d,
                              const float* __restrict__ P, T* __restrict__ feat, float* __restrict__ xs,
                              float* __restrict__ ms)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= d.rows) return;
    RowRing g;
    float x[kStrain], L0[6], S0[6], cph[6], sph[6], inv_l;
    row_strains(xa, xb, d, r, g, x, L0, S0, cph, sph, inv_l);
    float f[kInPad];
    row_inputs(x, g.deg, L0, S0, cph, sph, inv_l, P + PFSI_SG_IN_SHIFT, P + PFSI_SG_IN_SCALE, f);
#pragma unroll
    for (int q = 0; q < kInPad / 16; ++q) store16(feat + (size_t)r * kInPad + 16 * q, f + 16 * q);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const bool on = k < g.deg;
        xs[(size_t)kStrain * r + k] = x[k];
        xs[(size_t)kStrain * r + 6 + k] = x[6 + k];
        xs[(size_t)kStrain * r + 12 + k] = x[12 + k];
        ms[(size_t)kStrain * r + k] = on ? L0[k] * L0[k] : 0.f;
        ms[(size_t)kStrain * r + 6 + k] = on ? S0[k] : 0.f;
        ms[(size_t)kStrain * r + 12 + k] = on ? 1.f : 0.f;
    }
}

// Training record of every row: the exact stresses y (cs m x, ca m x,
// cb sin x) give a = x m t and b = y t / out_scale.
__global__ void k_sg_targets(SgDev d, const float* __restrict__ P, float cs, float ca, float cb,
                             const float* __restrict__ xs, const float* __restrict__ ms, float* __restrict__ target)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= d.rows) return;
    const float* out = P + PFSI_SG_OUT_SCALE;
    const float* tg = P + PFSI_SG_TGT_SCALE;
    for (int j = 0; j < kStrain; ++j) {
        const float x = xs[(size_t)kStrain * r + j], m = ms[(size_t)kStrain * r + j];
        const float y = j < 6 ? cs * m * x : (j < 12 ? ca * m * x : cb * m * sinf(x));
        target[(size_t)kTgt * r + j] = x * m * tg[j];
        target[(size_t)kTgt * r + kStrain + j] = y * tg[j] / out[j];
    }
}

// FP32 check path, output layer and forces: o = W3 h2 + b3 (CUDA cores),
// then the row's stress forces.
__global__ void k_sg_f32_forces(const float4* __restrict__ xa, const float4* __restrict__ xb, SgDev d,
                                const float* __restrict__ P, const float* __restrict__ H2, GlobalArgs ga,
                                float* __restrict__ F)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= d.rows) return;
    RowRing g;
    float x[kStrain], L0[6], S0[6], cph[6], sph[6], inv_l, q[kStrain];
    row_strains(xa, xb, d, r, g, x, L0, S0, cph, sph, inv_l);
    stress_factors(x, L0, P + PFSI_SG_OUT_SCALE, q);
    for (int j = 0; j < kStrain; ++j) {
        float acc = P[PFSI_SG_B3 + j];
        for (int k = 0; k < kHid; ++k) acc = fmaf(H2[(size_t)r * kHid + k], P[PFSI_SG_W3 + j * kHid + k], acc);
        q[j] *= acc;
    }
    row_scatter(g, q, row_global(xa, xb, ga, g.v), F, d.n_nodes);
}

// ------------------------------------------------------------------ fused inference
// Persistent kernel, one CTA of four warpgroups per SM.  Each warpgroup is an
// independent pipeline over 128-row tiles: it computes the tile's strains and
// inputs into its shared input tile A0 (128 x 64), runs the three layers
// through its 128 TMEM columns (each layer's accumulator overwrites the
// previous one once the GELU epilogue has read it back; the epilogue writes
// the BF16 activations into its shared hidden tile A1, 128 x 144, for the
// next MMA) and scatters the stress forces of its rows.  W1, W2, W3 sit once
// per CTA in shared memory in the core-matrix layout, with the biases folded
// in as an extra K column (the input tile carries a 1 in column 42, the
// hidden tile in column 128; K of the hidden layers is padded to 144), so the
// epilogue is the GELU alone.  Four pipelines per SM keep the tensor core
// busy while the others gather their rows or run their epilogues.
constexpr int kInferWG = 4;
constexpr int kKb = kHid + 16;                 // hidden K with the bias column (128) and zero padding
constexpr int kInferW1 = 0;
constexpr int kInferW2 = kInferW1 + kHid * kInPad * 2;
constexpr int kInferW3 = kInferW2 + kHid * kKb * 2;
constexpr int kInferPipe = kInferW3 + kOutPad * kKb * 2;            // first pipeline's tile
constexpr int kInferPipeBytes = kTile * kKb * 2;                     // A1; A0 aliases its first 8 KB
constexpr int kInferSmem = kInferPipe + kInferWG * kInferPipeBytes;
static_assert(kInferSmem <= 227 * 1024, "fused inference shared memory");

// rows x (8 * kgroups) BF16 row-major (leading dimension ld) -> core-matrix
// layout with dst_kgroups >= kgroups 16-byte groups per 8-row block
__device__ __forceinline__ void load_core(uint8_t* dst, const bf16* __restrict__ src, int ld, int rows, int kgroups,
                                          int dst_kgroups)
{
    for (int q = threadIdx.x; q < rows * kgroups; q += blockDim.x) {
        const int r = q / kgroups, kg = q - r * kgroups;
        *reinterpret_cast<uint4*>(dst + (((r >> 3) * dst_kgroups + kg) << 7) + ((r & 7) << 4)) =
            *reinterpret_cast<const uint4*>(src + (size_t)r * ld + 8 * kg);
    }
}

// Folded bias: K group `kg` of row r (layout with kgroups per block) holds
// (b, 0, ..., 0); the group after it, if `tail`, zeros.
__device__ __forceinline__ void put_bias_group(uint8_t* tile, int kgroups, int r, int kg, float b, bool tail)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(b, 0.f);
    uint8_t* base = tile + (((r >> 3) * kgroups + kg) << 7) + ((r & 7) << 4);
    *reinterpret_cast<uint4*>(base) = make_uint4(*reinterpret_cast<const uint32_t*>(&h), 0u, 0u, 0u);
    if (tail) *reinterpret_cast<uint4*>(base + 128) = make_uint4(0u, 0u, 0u, 0u);
}

// 16 values of a row into a core-matrix tile (kgroups per 8-row block)
__device__ __forceinline__ void put_row16(uint8_t* tile, int kgroups, int row, int n0, const float* v)
{
    uint32_t w[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
        w[q] = *reinterpret_cast<const uint32_t*>(&h);
    }
    uint8_t* base = tile + (((row >> 3) * kgroups + (n0 >> 3)) << 7) + ((row & 7) << 4);
    *reinterpret_cast<uint4*>(base) = make_uint4(w[0], w[1], w[2], w[3]);
    *reinterpret_cast<uint4*>(base + 128) = make_uint4(w[4], w[5], w[6], w[7]);
}

// barrier and AND-vote over the 128 threads of one warpgroup (named barrier id)
__device__ __forceinline__ void wg_sync(int id) { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }
__device__ __forceinline__ bool wg_and(bool v, int id)
{
    uint32_t r;
    asm volatile(
        "{\n"
        ".reg .pred p, q;\n"
        "setp.ne.u32 p, %1, 0;\n"
        "bar.red.and.pred q, %2, 128, p;\n"
        "selp.u32 %0, 1, 0, q;\n"
        "}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id)
        : "memory");
    return r != 0;
}

__global__ void __launch_bounds__(kInferWG * kTile, 1) k_sg_infer(const float4* __restrict__ xa,
                                                                  const float4* __restrict__ xb, SgDev d, Params P,
                                                                  GlobalArgs ga, float* __restrict__ F,
                                                                  int* __restrict__ err)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t bars[kInferWG];
    __shared__ uint32_t tmem_sh;
    // input shift and scale, output scale (read by every row)
    __shared__ float s_shift[kInPad], s_scale[kInPad], s_out[kOutPad];
    for (int i = threadIdx.x; i < kInPad; i += blockDim.x) {
        s_shift[i] = P.p[PFSI_SG_IN_SHIFT + i];
        s_scale[i] = P.p[PFSI_SG_IN_SCALE + i];
    }
    for (int i = threadIdx.x; i < kOutPad; i += blockDim.x) s_out[i] = P.p[PFSI_SG_OUT_SCALE + i];
    const int wg = threadIdx.x >> 7, t = threadIdx.x & (kTile - 1);
    const int bar_id = 1 + wg;
    uint64_t* bar = &bars[wg];
    if (threadIdx.x == 0) {
        for (int k = 0; k < kInferWG; ++k) mbar_init(&bars[k], 1);
        fence_barrier_init();
    }
    if (threadIdx.x < 32) tmem_alloc(&tmem_sh, 512);
    // weights with the biases folded in: input 42 of A0 and column 128 of the
    // hidden tile are 1, so W1[:, 42] = b1, W2[:, 128] = b2, W3[:, 128] = b3
    load_core(smem + kInferW1, P.h + hW1, kInPad, kHid, kInPad / 8, kInPad / 8);
    load_core(smem + kInferW2, P.h + hW2, kHid, kHid, kHid / 8, kKb / 8);
    load_core(smem + kInferW3, P.h + hW3, kHid, kOutPad, kHid / 8, kKb / 8);
    __syncthreads();
    if (threadIdx.x < kHid) {
        const int r = threadIdx.x;
        reinterpret_cast<bf16*>(smem + kInferW1 + (((r >> 3) * (kInPad / 8) + (kIn >> 3)) << 7) +
                                ((r & 7) << 4))[kIn & 7] = __float2bfloat16_rn(P.p[PFSI_SG_B1 + r]);
        put_bias_group(smem + kInferW2, kKb / 8, r, kHid / 8, P.p[PFSI_SG_B2 + r], true);
        if (r < kOutPad) put_bias_group(smem + kInferW3, kKb / 8, r, kHid / 8, P.p[PFSI_SG_B3 + r], true);
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // this warpgroup's 128 TMEM columns; a warp reads the 32 lanes of its rows
    const uint32_t tmem = tmem_sh + (uint32_t)(wg * 128);
    const uint32_t lanes = tmem + ((uint32_t)((t >> 5) * 32) << 16);
    uint8_t* A1 = smem + kInferPipe + wg * kInferPipeBytes;
    uint8_t* A0 = A1;   // the input tile lives in the hidden tile until layer 1 has read it
    const uint32_t sW1 = smem_u32(smem + kInferW1), sW2 = smem_u32(smem + kInferW2), sW3 = smem_u32(smem + kInferW3);
    const uint32_t sA0 = smem_u32(A0), sA1 = smem_u32(A1);
    uint32_t phase = 0;
    bool ok = true;
    const int n_tiles = d.rows_pad / kTile;
    for (int tile = blockIdx.x * kInferWG + wg; tile < n_tiles; tile += gridDim.x * kInferWG) {
        const int row = tile * kTile + t;
        float f[kInPad], q[kStrain];
        RowRing g;
        g.deg = 0;
        if (row < d.rows) {
            float x[kStrain], L0[6], S0[6], cph[6], sph[6], inv_l;
            row_strains(xa, xb, d, row, g, x, L0, S0, cph, sph, inv_l);
            row_inputs(x, g.deg, L0, S0, cph, sph, inv_l, s_shift, s_scale, f);
            stress_factors(x, L0, s_out, q);
        } else {
#pragma unroll
            for (int k = 0; k < kInPad; ++k) f[k] = 0.f;
#pragma unroll
            for (int k = 0; k < kStrain; ++k) q[k] = 0.f;
        }
        f[kIn] = 1.0f;   // bias input
#pragma unroll
        for (int c = 0; c < kInPad / 16; ++c) put_row16(A0, kInPad / 8, t, 16 * c, f + 16 * c);
        for (int layer = 0; layer < 3; ++layer) {
            fence_proxy_async();
            tc_fence_before();
            wg_sync(bar_id);
            if (t == 0) {
                tc_fence_after();
                if (layer == 0) {
                    for (int j = 0; j < kInPad / 16; ++j)
                        mma_bf16(tmem, smem_desc(sA0 + 256 * j, 128, 128 * (kInPad / 8)),
                                 smem_desc(sW1 + 256 * j, 128, 128 * (kInPad / 8)), idesc_bf16(kHid), j > 0 ? 1u : 0u);
                } else {
                    const uint32_t sW = layer == 1 ? sW2 : sW3;
                    const uint32_t idesc = idesc_bf16(layer == 1 ? kHid : kOutPad);
                    for (int j = 0; j < kKb / 16; ++j)
                        mma_bf16(tmem, smem_desc(sA1 + 256 * j, 128, 128 * (kKb / 8)),
                                 smem_desc(sW + 256 * j, 128, 128 * (kKb / 8)), idesc, j > 0 ? 1u : 0u);
                }
                mma_commit(bar);
            }
            // one thread polls the barrier; the others sleep in bar.red and
            // leave the issue slots to the other pipelines
            ok = wg_and(t == 0 ? mbar_wait(bar, phase) : true, bar_id);
            phase ^= 1u;
            tc_fence_after();
            if (!ok || layer == 2) break;
            // GELU epilogue: accumulator (bias included) -> BF16 activations in
            // A1 (the MMA that read this tile has completed)
#pragma unroll 1
            for (int n0 = 0; n0 < kHid; n0 += 16) {
                float v[16];
                tmem_ld16(lanes + (uint32_t)n0, v);
                uint32_t w[8];
                gelu16_bf16(v, w);
                uint8_t* base = A1 + (((t >> 3) * (kKb / 8) + (n0 >> 3)) << 7) + ((t & 7) << 4);
                *reinterpret_cast<uint4*>(base) = make_uint4(w[0], w[1], w[2], w[3]);
                *reinterpret_cast<uint4*>(base + 128) = make_uint4(w[4], w[5], w[6], w[7]);
            }
            if (layer == 0) put_bias_group(A1, kKb / 8, t, kHid / 8, 1.0f, true);
        }
        if (!ok) break;
        // output o (bias included) -> stresses -> forces of the tile's rows
        {
            float o[16];
            tmem_ld16(lanes, o);
#pragma unroll
            for (int j = 0; j < 16; ++j) q[j] *= o[j];
            tmem_ld16(lanes + 16u, o);
#pragma unroll
            for (int j = 16; j < kStrain; ++j) q[j] *= o[j - 16];
        }
        if (row < d.rows) row_scatter(g, q, row_global(xa, xb, ga, g.v), F, d.n_nodes);
    }
    if (!ok && t == 0) atomicExch(err, 1);
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) {
        tc_fence_after();
        tmem_dealloc(tmem_sh, 512);
    }
}

// ------------------------------------------------------------------ host side
template <int N>
constexpr size_t gemm_smem() { return 2 * kTile * kChunkK * 2 + 2 * N * kChunkK * 2; }

template <int N, class Epi>
int smem_attr()
{
    return check_cuda(cudaFuncSetAttribute(k_gemm_tc<N, Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)gemm_smem<N>()),
                      "surrogate: gemm shared memory");
}

// Kernel attributes, set before any launch (and outside graph capture).
int prepare_tc()
{
    int rc = smem_attr<128, EpiHidden<bf16>>();
    if (!rc) rc = smem_attr<128, EpiBack<bf16>>();
    if (!rc) rc = smem_attr<128, EpiPartial>();
    if (!rc) rc = smem_attr<kOutPad, EpiOut>();
    if (!rc) rc = smem_attr<kOutPad, EpiPartial>();
    if (!rc) rc = smem_attr<kInPad, EpiPartial>();
    if (!rc)
        rc = check_cuda(cudaFuncSetAttribute(k_sg_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, kInferSmem),
                        "surrogate: shared memory");
    return rc;
}

template <int N, class Epi>
int gemm_tc(const bf16* A, int lda, const bf16* B, int ldb, int rows, int K, int splits, Epi epi, int* err,
            cudaStream_t s)
{
    const int k_per = ((K + splits - 1) / splits + kChunkK - 1) / kChunkK * kChunkK;
    const int used = (K + k_per - 1) / k_per;
    k_gemm_tc<N, Epi><<<dim3(rows / kTile, used), kTile, gemm_smem<N>(), s>>>(A, lda, B, ldb, K, k_per, epi, err);
    return check_launch("surrogate: tensor-core layer");
}

template <class Epi>
int gemm_f32(const float* A, long long sar, long long sak, const float* B, long long sbn, long long sbk, int rows,
             int N, int K, int splits, Epi epi, cudaStream_t s)
{
    const int k_per = (K + splits - 1) / splits;
    const int used = (K + k_per - 1) / k_per;
    const long long total = (long long)rows * N;
    k_gemm_f32<Epi><<<dim3((unsigned)((total + 255) / 256), used), 256, 0, s>>>(A, sar, sak, B, sbn, sbk, rows, N, K,
                                                                                k_per, epi);
    return check_launch("surrogate: FP32 layer");
}

int splits_for(int K) { return std::max(1, std::min(kMaxSplit, K / 256)); }
int used_splits(int K, int splits)
{
    const int k_per = ((K + splits - 1) / splits + kChunkK - 1) / kChunkK * kChunkK;
    return (K + k_per - 1) / k_per;
}

// Training workspace for a batch of `rows` (multiple of 128) samples.
struct Work {
    void* Xt;       // [64][rows]
    float* Z1;      // [rows][128]
    float* Z2;
    void* H1;       // [rows][128]
    void* H2;
    void* H1t;      // [128][rows]
    void* H2t;
    float* O;       // [rows][32]
    void* dO;       // [rows][32]
    void* dOt;      // [32][rows]
    void* dZ2;      // [rows][128]
    void* dZ2t;     // [128][rows]
    void* dZ1t;     // [128][rows]
    float* part;    // [kMaxSplit][128][128]
    double* loss;
    int* err;
    size_t total;
};

Work work_layout(void* base, int rows)
{
    const size_t R = rows;
    const size_t sizes[] = {4 * kInPad * R, 4 * 128 * R, 4 * 128 * R, 4 * 128 * R, 4 * 128 * R, 4 * 128 * R,
                            4 * 128 * R, 4 * kOutPad * R, 4 * kOutPad * R, 4 * kOutPad * R, 4 * 128 * R, 4 * 128 * R,
                            4 * 128 * R, 4 * (size_t)kMaxSplit * 128 * 128, 8, 4};
    void* ptr[16];
    size_t o = 0;
    for (int i = 0; i < 16; ++i) {
        ptr[i] = base ? (char*)base + o : nullptr;
        o += (sizes[i] + 255) / 256 * 256;
    }
    Work w;
    w.Xt = ptr[0];
    w.Z1 = (float*)ptr[1];
    w.Z2 = (float*)ptr[2];
    w.H1 = ptr[3];
    w.H2 = ptr[4];
    w.H1t = ptr[5];
    w.H2t = ptr[6];
    w.O = (float*)ptr[7];
    w.dO = ptr[8];
    w.dOt = ptr[9];
    w.dZ2 = ptr[10];
    w.dZ2t = ptr[11];
    w.dZ1t = ptr[12];
    w.part = (float*)ptr[13];
    w.loss = (double*)ptr[14];
    w.err = (int*)ptr[15];
    w.total = o;
    return w;
}

// Forward + backward on a batch; gradients into g (trained-parameter layout).
int grad_bf16(Params P, const bf16* X, const float* target, int B, int rows, float* g, Work& w, cudaStream_t s)
{
    bf16 *Xt = (bf16*)w.Xt, *H1 = (bf16*)w.H1, *H2 = (bf16*)w.H2, *H1t = (bf16*)w.H1t, *H2t = (bf16*)w.H2t;
    bf16 *dO = (bf16*)w.dO, *dOt = (bf16*)w.dOt, *dZ2 = (bf16*)w.dZ2, *dZ2t = (bf16*)w.dZ2t, *dZ1t = (bf16*)w.dZ1t;
    int rc = PFSI_OK;
    k_transpose_in<bf16><<<(rows * kInPad + 255) / 256, 256, 0, s>>>(X, rows, Xt);
    if ((rc = check_launch("surrogate: transpose"))) return rc;
    if ((rc = gemm_tc<128>(X, kInPad, P.h + hW1, kInPad, rows, kInPad, 1,
                           EpiHidden<bf16>{P.p + PFSI_SG_B1, w.Z1, H1, H1t, rows}, w.err, s)))
        return rc;
    if ((rc = gemm_tc<128>(H1, kHid, P.h + hW2, kHid, rows, kHid, 1,
                           EpiHidden<bf16>{P.p + PFSI_SG_B2, w.Z2, H2, H2t, rows}, w.err, s)))
        return rc;
    if ((rc = gemm_tc<kOutPad>(H2, kHid, P.h + hW3, kHid, rows, kHid, 1, EpiOut{P.p + PFSI_SG_B3, w.O}, w.err, s)))
        return rc;
    if ((rc = check_cuda(cudaMemsetAsync(w.loss, 0, sizeof(double), s), "surrogate: clear loss"))) return rc;
    k_sg_loss<bf16><<<(rows + 127) / 128, 128, 0, s>>>(w.O, target, B, rows, dO, dOt, w.loss);
    if ((rc = check_launch("surrogate: loss"))) return rc;
    // dZ2 = (dO W3) * gelu'(Z2); dZ1 = (dZ2 W2) * gelu'(Z1)
    if ((rc = gemm_tc<128>(dO, kOutPad, P.h + hW3t, kOutPad, rows, kOutPad, 1,
                           EpiBack<bf16>{w.Z2, dZ2, dZ2t, rows}, w.err, s)))
        return rc;
    if ((rc = gemm_tc<128>(dZ2, kHid, P.h + hW2t, kHid, rows, kHid, 1, EpiBack<bf16>{w.Z1, nullptr, dZ1t, rows},
                           w.err, s)))
        return rc;
    // weight gradients, split over the batch
    const int sp = splits_for(rows);
    const int u = used_splits(rows, sp);
    if ((rc = gemm_tc<kOutPad>(H2t, rows, dOt, rows, kHid, rows, sp, EpiPartial{w.part, kHid, kOutPad * kHid, true},
                               w.err, s)))
        return rc;
    k_reduce_splits<<<(kOutPad * kHid + 255) / 256, 256, 0, s>>>(w.part, u, kOutPad * kHid, g + PFSI_SG_W3);
    if ((rc = check_launch("surrogate: reduce"))) return rc;
    if ((rc = gemm_tc<128>(dZ2t, rows, H1t, rows, kHid, rows, sp, EpiPartial{w.part, kHid, kHid * kHid, false}, w.err, s)))
        return rc;
    k_reduce_splits<<<(kHid * kHid + 255) / 256, 256, 0, s>>>(w.part, u, kHid * kHid, g + PFSI_SG_W2);
    if ((rc = check_launch("surrogate: reduce"))) return rc;
    if ((rc = gemm_tc<kInPad>(dZ1t, rows, Xt, rows, kHid, rows, sp, EpiPartial{w.part, kInPad, kHid * kInPad, false},
                              w.err, s)))
        return rc;
    k_reduce_splits<<<(kHid * kInPad + 255) / 256, 256, 0, s>>>(w.part, u, kHid * kInPad, g + PFSI_SG_W1);
    if ((rc = check_launch("surrogate: reduce"))) return rc;
    k_rowsum<bf16><<<(kHid + 7) / 8, 256, 0, s>>>(dZ1t, kHid, rows, rows, g + PFSI_SG_B1);
    k_rowsum<bf16><<<(kHid + 7) / 8, 256, 0, s>>>(dZ2t, kHid, rows, rows, g + PFSI_SG_B2);
    k_rowsum<bf16><<<(kOutPad + 7) / 8, 256, 0, s>>>(dOt, kOutPad, rows, rows, g + PFSI_SG_B3);
    return check_launch("surrogate: bias gradients");
}

int grad_f32(Params P, const float* X, const float* target, int B, int rows, float* g, Work& w, cudaStream_t s)
{
    float *Xt = (float*)w.Xt, *H1 = (float*)w.H1, *H2 = (float*)w.H2, *H1t = (float*)w.H1t, *H2t = (float*)w.H2t;
    float *dO = (float*)w.dO, *dOt = (float*)w.dOt, *dZ2 = (float*)w.dZ2, *dZ2t = (float*)w.dZ2t,
          *dZ1t = (float*)w.dZ1t;
    const float* W1 = P.p + PFSI_SG_W1;
    const float* W2 = P.p + PFSI_SG_W2;
    const float* W3 = P.p + PFSI_SG_W3;
    int rc = PFSI_OK;
    k_transpose_in<float><<<(rows * kInPad + 255) / 256, 256, 0, s>>>(X, rows, Xt);
    if ((rc = check_launch("surrogate: transpose"))) return rc;
    if ((rc = gemm_f32(X, kInPad, 1, W1, kInPad, 1, rows, kHid, kInPad, 1,
                       EpiHidden<float>{P.p + PFSI_SG_B1, w.Z1, H1, H1t, rows}, s)))
        return rc;
    if ((rc = gemm_f32(H1, kHid, 1, W2, kHid, 1, rows, kHid, kHid, 1,
                       EpiHidden<float>{P.p + PFSI_SG_B2, w.Z2, H2, H2t, rows}, s)))
        return rc;
    if ((rc = gemm_f32(H2, kHid, 1, W3, kHid, 1, rows, kOutPad, kHid, 1, EpiOut{P.p + PFSI_SG_B3, w.O}, s)))
        return rc;
    if ((rc = check_cuda(cudaMemsetAsync(w.loss, 0, sizeof(double), s), "surrogate: clear loss"))) return rc;
    k_sg_loss<float><<<(rows + 127) / 128, 128, 0, s>>>(w.O, target, B, rows, dO, dOt, w.loss);
    if ((rc = check_launch("surrogate: loss"))) return rc;
    // B(n, k) = W3[k][n] (transposed view), W2[k][n]
    if ((rc = gemm_f32(dO, kOutPad, 1, W3, 1, kHid, rows, kHid, kOutPad, 1, EpiBack<float>{w.Z2, dZ2, dZ2t, rows},
                       s)))
        return rc;
    if ((rc = gemm_f32(dZ2, kHid, 1, W2, 1, kHid, rows, kHid, kHid, 1, EpiBack<float>{w.Z1, nullptr, dZ1t, rows},
                       s)))
        return rc;
    const int sp = splits_for(rows);
    const int k_per = (rows + sp - 1) / sp;
    const int u = (rows + k_per - 1) / k_per;
    if ((rc = gemm_f32(H2t, rows, 1, dOt, rows, 1, kHid, kOutPad, rows, sp, EpiPartial{w.part, kHid, kOutPad * kHid, true},
                       s)))
        return rc;
    k_reduce_splits<<<(kOutPad * kHid + 255) / 256, 256, 0, s>>>(w.part, u, kOutPad * kHid, g + PFSI_SG_W3);
    if ((rc = check_launch("surrogate: reduce"))) return rc;
    if ((rc = gemm_f32(dZ2t, rows, 1, H1t, rows, 1, kHid, kHid, rows, sp, EpiPartial{w.part, kHid, kHid * kHid, false}, s)))
        return rc;
    k_reduce_splits<<<(kHid * kHid + 255) / 256, 256, 0, s>>>(w.part, u, kHid * kHid, g + PFSI_SG_W2);
    if ((rc = check_launch("surrogate: reduce"))) return rc;
    if ((rc = gemm_f32(dZ1t, rows, 1, Xt, rows, 1, kHid, kInPad, rows, sp, EpiPartial{w.part, kInPad, kHid * kInPad, false},
                       s)))
        return rc;
    k_reduce_splits<<<(kHid * kInPad + 255) / 256, 256, 0, s>>>(w.part, u, kHid * kInPad, g + PFSI_SG_W1);
    if ((rc = check_launch("surrogate: reduce"))) return rc;
    k_rowsum<float><<<(kHid + 7) / 8, 256, 0, s>>>(dZ1t, kHid, rows, rows, g + PFSI_SG_B1);
    k_rowsum<float><<<(kHid + 7) / 8, 256, 0, s>>>(dZ2t, kHid, rows, rows, g + PFSI_SG_B2);
    k_rowsum<float><<<(kOutPad + 7) / 8, 256, 0, s>>>(dOt, kOutPad, rows, rows, g + PFSI_SG_B3);
    return check_launch("surrogate: bias gradients");
}

// ------------------------------------------------------------------ mesh context (host build)
struct Rest {
    std::vector<int> node, ring;
    std::vector<float> rest;
};

int build_rings(int n, int nt, const int* tri, const double* X0, const unsigned char* is_mem, Rest& R,
                std::string& err)
{
    // around node i, the face (i, a, b) (counter-clockwise) makes b follow a
    std::vector<std::vector<std::pair<int, int>>> nxt(n);
    for (int t = 0; t < nt; ++t) {
        const int v[3] = {tri[3 * t], tri[3 * t + 1], tri[3 * t + 2]};
        for (int c = 0; c < 3; ++c) {
            if (v[c] < 0 || v[c] >= n) {
                err = "triangle vertex index out of range";
                return PFSI_ERR_ARG;
            }
            nxt[v[c]].push_back({v[(c + 1) % 3], v[(c + 2) % 3]});
        }
    }
    auto P = [&](int v, int c) { return X0[(size_t)c * n + v]; };
    for (int i = 0; i < n; ++i) {
        if (nxt[i].empty() || (is_mem && !is_mem[i])) continue;
        const int d = (int)nxt[i].size();
        if (d < 3 || d > 6) {
            err = "a membrane node needs 3 to 6 neighbours";
            return PFSI_ERR_ARG;
        }
        int start = nxt[i][0].first;
        for (auto& pr : nxt[i]) start = std::min(start, pr.first);
        int ring[6] = {-1, -1, -1, -1, -1, -1};
        int cur = start, k = 0;
        do {
            if (k >= d) {
                err = "open or non-manifold one-ring";
                return PFSI_ERR_ARG;
            }
            ring[k++] = cur;
            int nx = -1;
            for (auto& pr : nxt[i])
                if (pr.first == cur) nx = pr.second;
            if (nx < 0) {
                err = "open one-ring";
                return PFSI_ERR_ARG;
            }
            cur = nx;
        } while (cur != start);
        if (k != d) {
            err = "one-ring does not close";
            return PFSI_ERR_ARG;
        }
        // rest record (FP64 geometry): e0_k split hi/lo (0..35), cos and sin of
        // the rest bending angle of each spoke (36..47), L0_k (48..53), S0_k
        // of the fan triangles (54..59), 1/l with l the mean L0 (60)
        double e[6][3];
        for (int q = 0; q < d; ++q)
            for (int c = 0; c < 3; ++c) e[q][c] = P(ring[q], c) - P(i, c);
        auto cross = [](const double* a, const double* b, double* r) {
            r[0] = a[1] * b[2] - a[2] * b[1];
            r[1] = a[2] * b[0] - a[0] * b[2];
            r[2] = a[0] * b[1] - a[1] * b[0];
        };
        auto dot = [](const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; };
        float r64[64] = {};
        double ell = 0;
        for (int q = 0; q < d; ++q) {
            const double* en = e[(q + 1) % d];
            const double* ep = e[(q + d - 1) % d];
            const double L = std::sqrt(dot(e[q], e[q]));
            double cc[3];
            cross(e[q], en, cc);
            const double S = 0.5 * std::sqrt(dot(cc, cc));
            if (!(L > 0) || !(S > 0)) {
                err = "degenerate rest one-ring";
                return PFSI_ERR_ARG;
            }
            // torsion of n_{q+1} - i - n_q - n_{q-1}, points relative to i:
            // F = e_{q+1}, G = -e_q, H = e_{q-1} - e_q
            double G[3], H[3], A[3], B[3], BA[3];
            for (int c = 0; c < 3; ++c) {
                G[c] = -e[q][c];
                H[c] = ep[c] - e[q][c];
            }
            cross(en, G, A);
            cross(H, G, B);
            cross(B, A, BA);
            const double ab = std::sqrt(dot(A, A) * dot(B, B));
            if (!(ab > 0)) {
                err = "degenerate rest one-ring";
                return PFSI_ERR_ARG;
            }
            const double cphi = dot(A, B) / ab, sphi = dot(BA, G) / (ab * L);
            const double phi = std::atan2(sphi, cphi);
            for (int c = 0; c < 3; ++c) {
                const float h = (float)e[q][c];
                r64[3 * q + c] = h;
                r64[18 + 3 * q + c] = (float)(e[q][c] - (double)h);
            }
            r64[36 + q] = (float)std::cos(phi);
            r64[42 + q] = (float)std::sin(phi);
            r64[48 + q] = (float)L;
            r64[54 + q] = (float)S;
            ell += L / d;
        }
        r64[60] = (float)(1.0 / ell);
        R.node.push_back(i);
        for (int q = 0; q < 6; ++q) R.ring.push_back(ring[q]);
        R.rest.insert(R.rest.end(), r64, r64 + 64);
    }
    if (R.node.empty()) {
        err = "no membrane node with a closed one-ring";
        return PFSI_ERR_ARG;
    }
    return PFSI_OK;
}

struct SgLayout {
    size_t node, ring, rest, feat, xs, ms, h1, h2, xh, xl, xa, xb, err, total;
};
// rows: surrogate rows; n: mesh nodes
SgLayout sg_layout(int rows, int n)
{
    const size_t Rp = ((size_t)rows + kTile - 1) / kTile * kTile;
    const size_t sizes[] = {4 * Rp, 4 * 6 * Rp, 4 * 64 * Rp, 4 * kInPad * Rp, 4 * kStrain * Rp, 4 * kStrain * Rp,
                            4 * 128 * Rp, 4 * 128 * Rp, 12 * (size_t)n, 12 * (size_t)n, 16 * (size_t)n,
                            16 * (size_t)n, 4};
    constexpr int kParts = sizeof(sizes) / sizeof(sizes[0]);
    size_t off[kParts], o = 0;
    for (int i = 0; i < kParts; ++i) {
        off[i] = o;
        o += (sizes[i] + 255) / 256 * 256;
    }
    return {off[0], off[1], off[2], off[3], off[4], off[5], off[6], off[7], off[8], off[9], off[10], off[11], off[12], o};
}

}  // namespace

struct SgCtx {
    SgDev d;
    int mode;
    void* ws;
    SgLayout L;
    bf16* feat;       // [rows_pad][64] (BF16 mode) / float (FP32 mode)
    float* xs;        // [rows_pad][18] element strains
    float* ms;        // [rows_pad][18] rest moduli scales
    float* xh;        // [3][n] split positions (standalone feature calls)
    float* xl;
    float4* xa;       // [n] split positions per node (hi, lo)
    float4* xb;
    void* h1;         // [rows_pad][128]
    void* h2;
    int* err;
};

// Surrogate forces added to F (the exact global terms must already be in F).
int launch_surrogate_forces(SgCtx* c, const void* params, const MemCtx* mem, float* F, cudaStream_t s)
{
    const Params P = params_of(params);
    const int rows = c->d.rows_pad;
    const GlobalArgs ga{mem->coef,       mem->node_plt,       mem->plt_anchor,     mem->np == 0 ? 1 : 0,
                        mem->p.rep_F0, mem->p.rep_tau, mem->p.rep_eps_min, mem->p.z_wall};
    k_sg_pack<<<(c->d.n_nodes + 255) / 256, 256, 0, s>>>(mem->xh, mem->xl, c->d.n_nodes, c->xa, c->xb);
    int rc = check_launch("surrogate: positions");
    if (rc) return rc;
    if (c->mode == PFSI_SG_FP32) {
        k_sg_features<float><<<(c->d.rows + 127) / 128, 128, 0, s>>>(c->xa, c->xb, c->d, P.p, (float*)c->feat,
                                                                     c->xs, c->ms);
        if ((rc = check_launch("surrogate: features"))) return rc;
        float *H1 = (float*)c->h1, *H2 = (float*)c->h2;
        if ((rc = gemm_f32((const float*)c->feat, kInPad, 1, P.p + PFSI_SG_W1, kInPad, 1, rows, kHid, kInPad, 1,
                           EpiHidden<float>{P.p + PFSI_SG_B1, nullptr, H1, nullptr, 0}, s)))
            return rc;
        if ((rc = gemm_f32(H1, kHid, 1, P.p + PFSI_SG_W2, kHid, 1, rows, kHid, kHid, 1,
                           EpiHidden<float>{P.p + PFSI_SG_B2, nullptr, H2, nullptr, 0}, s)))
            return rc;
        k_sg_f32_forces<<<(c->d.rows + 127) / 128, 128, 0, s>>>(c->xa, c->xb, c->d, P.p, H2, ga, F);
        return check_launch("surrogate: FP32 output layer and forces");
    }
    const int tiles = rows / kTile;
    const int want = (tiles + kInferWG - 1) / kInferWG;
    const int grid = want < 148 ? want : 148;
    k_sg_infer<<<grid, kInferWG * kTile, kInferSmem, s>>>(c->xa, c->xb, c->d, P, ga, F, c->err);
    return check_launch("surrogate: fused inference");
}

}  // namespace pfsi

using namespace pfsi;

struct sg_ctx : pfsi::SgCtx {};

namespace pfsi {
SgCtx* sg_internal(sg_ctx* c) { return c; }
int sg_node_count(const SgCtx* c) { return c->d.n_nodes; }
}  // namespace pfsi

extern "C" int sg_params_bytes(size_t* bytes)
{
    if (!bytes) return set_error(PFSI_ERR_ARG, "sg_params_bytes: null argument");
    *bytes = PFSI_SG_PARAM_BYTES;
    return PFSI_OK;
}

extern "C" int sg_sync_shadows(void* params, void* stream)
{
    if (!params || !aligned(params, 256)) return set_error(PFSI_ERR_ARG, "sg_sync_shadows: bad parameter buffer");
    const Params P = params_of(params);
    k_sg_shadows<<<(kHid * kHid + 255) / 256, 256, 0, as_stream(stream)>>>(P.p, const_cast<bf16*>(P.h));
    return check_launch("sg_sync_shadows");
}

extern "C" int sg_query_work(int batch, size_t* bytes)
{
    if (!bytes || batch < 1) return set_error(PFSI_ERR_ARG, "sg_query_work: bad argument");
    const int rows = (batch + kTile - 1) / kTile * kTile;
    *bytes = work_layout(nullptr, rows).total;
    return PFSI_OK;
}

extern "C" int sg_grad(const void* params, const void* feat, const float* target, int batch, int mode, float* grad,
                       double* loss, void* work, size_t work_bytes, void* stream)
{
    NvtxRange nvtx_range("sg_grad");
    if (!params || !feat || !target || !grad || !work || batch < 1 || (mode != PFSI_SG_BF16 && mode != PFSI_SG_FP32))
        return set_error(PFSI_ERR_ARG, "sg_grad: bad argument");
    if (batch % kTile) return set_error(PFSI_ERR_ARG, "sg_grad: batch must be a multiple of 128 (pad the rows)");
    if (!aligned(params, 256) || !aligned(work, 256) || !aligned(feat, 16))
        return set_error(PFSI_ERR_ARG, "sg_grad: misaligned buffer");
    Work w = work_layout(work, batch);
    if (work_bytes < w.total) return set_error(PFSI_ERR_ARG, "sg_grad: workspace too small");
    cudaStream_t s = as_stream(stream);
    int rc = mode == PFSI_SG_BF16 ? prepare_tc() : PFSI_OK;
    if (!rc) rc = check_cuda(cudaMemsetAsync(w.err, 0, sizeof(int), s), "sg_grad: clear flag");
    if (rc) return rc;
    const Params P = params_of(params);
    rc = mode == PFSI_SG_BF16 ? grad_bf16(P, (const bf16*)feat, target, batch, batch, grad, w, s)
                              : grad_f32(P, (const float*)feat, target, batch, batch, grad, w, s);
    if (rc) return rc;
    if (loss) rc = check_cuda(cudaMemcpyAsync(loss, w.loss, sizeof(double), cudaMemcpyDeviceToDevice, s), "sg_grad");
    return rc;
}

extern "C" int sg_work_status(void* work, int batch, int* flag)
{
    if (!work || !flag || batch < 1) return set_error(PFSI_ERR_ARG, "sg_work_status: bad argument");
    const int rows = (batch + kTile - 1) / kTile * kTile;
    Work w = work_layout(work, rows);
    return check_cuda(cudaMemcpy(flag, w.err, sizeof(int), cudaMemcpyDeviceToHost), "sg_work_status");
}

extern "C" int sg_adam(void* params, const float* grad, float* m, float* v, float lr, float beta1, float beta2,
                       float eps, int t, void* stream)
{
    NvtxRange nvtx_range("sg_adam");
    if (!params || !grad || !m || !v || t < 1 || !(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) ||
        !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
        return set_error(PFSI_ERR_ARG, "sg_adam: bad argument");
    if (!aligned(params, 256)) return set_error(PFSI_ERR_ARG, "sg_adam: misaligned parameter buffer");
    cudaStream_t s = as_stream(stream);
    const float c1 = (float)(1.0 - std::pow((double)beta1, t)), c2 = (float)(1.0 - std::pow((double)beta2, t));
    k_sg_adam<<<(PFSI_SG_N_TRAINED + 255) / 256, 256, 0, s>>>((float*)params, grad, m, v, PFSI_SG_N_TRAINED, lr, beta1,
                                                             beta2, eps, c1, c2);
    int rc = check_launch("sg_adam");
    if (rc) return rc;
    return sg_sync_shadows(params, stream);
}

extern "C" int sg_query_workspace(int n_nodes, size_t* bytes)
{
    if (!bytes || n_nodes < 1) return set_error(PFSI_ERR_ARG, "sg_query_workspace: bad argument");
    *bytes = sg_layout(n_nodes, n_nodes).total;
    return PFSI_OK;
}

extern "C" int sg_create(int n_nodes, int n_tri, const int* tri, const double* X0, const unsigned char* is_membrane,
                         int mode, void* ws, size_t ws_bytes, sg_ctx** out)
{
    if (!out || n_nodes < 1 || n_tri < 1 || !tri || !X0 || !ws || (mode != PFSI_SG_BF16 && mode != PFSI_SG_FP32))
        return set_error(PFSI_ERR_ARG, "sg_create: bad argument");
    if (!aligned(ws, 256)) return set_error(PFSI_ERR_ARG, "sg_create: workspace must be 256-byte aligned");
    Rest R;
    std::string err;
    int rc = build_rings(n_nodes, n_tri, tri, X0, is_membrane, R, err);
    if (!rc && mode == PFSI_SG_BF16) rc = prepare_tc();
    if (rc) return set_error(rc, "sg_create: " + err);
    const int rows = (int)R.node.size();
    const SgLayout L = sg_layout(rows, n_nodes);
    if (ws_bytes < sg_layout(n_nodes, n_nodes).total) return set_error(PFSI_ERR_ARG, "sg_create: workspace too small");
    const int rows_pad = (rows + kTile - 1) / kTile * kTile;
    R.node.resize(rows_pad, -1);
    char* b = (char*)ws;
    rc = check_cuda(cudaMemset(ws, 0, L.total), "sg_create: clear");
    if (!rc) rc = check_cuda(cudaMemcpy(b + L.node, R.node.data(), 4 * R.node.size(), cudaMemcpyHostToDevice), "sg_create");
    if (!rc) rc = check_cuda(cudaMemcpy(b + L.ring, R.ring.data(), 4 * R.ring.size(), cudaMemcpyHostToDevice), "sg_create");
    if (!rc) rc = check_cuda(cudaMemcpy(b + L.rest, R.rest.data(), 4 * R.rest.size(), cudaMemcpyHostToDevice), "sg_create");
    if (rc) return rc;
    sg_ctx* c = new sg_ctx();
    c->d = SgDev{n_nodes, rows, rows_pad, (const int*)(b + L.node), (const int*)(b + L.ring),
                 (const float*)(b + L.rest)};
    c->mode = mode;
    c->ws = ws;
    c->L = L;
    c->feat = (bf16*)(b + L.feat);
    c->xs = (float*)(b + L.xs);
    c->ms = (float*)(b + L.ms);
    c->xh = (float*)(b + L.xh);
    c->xl = (float*)(b + L.xl);
    c->xa = (float4*)(b + L.xa);
    c->xb = (float4*)(b + L.xb);
    c->h1 = b + L.h1;
    c->h2 = b + L.h2;
    c->err = (int*)(b + L.err);
    *out = c;
    return PFSI_OK;
}

extern "C" int sg_destroy(sg_ctx* c)
{
    delete c;
    return PFSI_OK;
}

extern "C" int sg_rows(const sg_ctx* c, int* rows, const int** node)
{
    if (!c || !rows) return set_error(PFSI_ERR_ARG, "sg_rows: null argument");
    *rows = c->d.rows;
    if (node) *node = c->d.node;
    return PFSI_OK;
}

extern "C" int sg_features(sg_ctx* c, const void* params, const double* X, void* feat, float* xs, float* ms,
                           void* stream)
{
    NvtxRange nvtx_range("sg_features");
    if (!c || !params || !X) return set_error(PFSI_ERR_ARG, "sg_features: null argument");
    const Params P = params_of(params);
    cudaStream_t s = as_stream(stream);
    const int n3 = 3 * c->d.n_nodes;
    k_sg_split<<<(n3 + 255) / 256, 256, 0, s>>>(X, n3, c->xh, c->xl);
    int rc = check_launch("sg_features: split");
    if (rc) return rc;
    k_sg_pack<<<(c->d.n_nodes + 255) / 256, 256, 0, s>>>(c->xh, c->xl, c->d.n_nodes, c->xa, c->xb);
    if ((rc = check_launch("sg_features: positions"))) return rc;
    float* x = xs ? xs : c->xs;
    float* m = ms ? ms : c->ms;
    if (c->mode == PFSI_SG_FP32) {
        k_sg_features<float><<<(c->d.rows + 127) / 128, 128, 0, s>>>(c->xa, c->xb, c->d, P.p,
                                                                     feat ? (float*)feat : (float*)c->feat, x, m);
    } else {
        k_sg_features<bf16><<<(c->d.rows + 127) / 128, 128, 0, s>>>(c->xa, c->xb, c->d, P.p,
                                                                    feat ? (bf16*)feat : c->feat, x, m);
    }
    return check_launch("sg_features");
}

extern "C" int sg_membrane_forces(sg_ctx* c, const void* params, mem_ctx* mem, const double* X, float* F,
                                  void* stream)
{
    NvtxRange nvtx_range("sg_membrane_forces");
    if (!c || !params || !mem || !X || !F) return set_error(PFSI_ERR_ARG, "sg_membrane_forces: null argument");
    if (mem->n != c->d.n_nodes) return set_error(PFSI_ERR_ARG, "sg_membrane_forces: node count differs");
    cudaStream_t s = as_stream(stream);
    int rc = launch_membrane_remainder(mem, X, F, s);   // also splits X into mem->xh, mem->xl
    if (rc) return rc;
    return launch_surrogate_forces(c, params, mem, F, s);
}

extern "C" int sg_targets(const sg_ctx* c, const void* params, float k_spring, float k_t, float k_b, const float* xs,
                          const float* ms, float* target, void* stream)
{
    NvtxRange nvtx_range("sg_targets");
    if (!c || !params || !target) return set_error(PFSI_ERR_ARG, "sg_targets: null argument");
    const Params P = params_of(params);
    k_sg_targets<<<(c->d.rows + 127) / 128, 128, 0, as_stream(stream)>>>(
        c->d, P.p, 0.5f * k_spring, k_t / 3.0f, 0.5f * k_b, xs ? xs : c->xs, ms ? ms : c->ms, target);
    return check_launch("sg_targets");
}

extern "C" int sg_status(const sg_ctx* c, int* flag)
{
    if (!c || !flag) return set_error(PFSI_ERR_ARG, "sg_status: null argument");
    return check_cuda(cudaMemcpy(flag, c->err, sizeof(int), cudaMemcpyDeviceToHost), "sg_status");
}

namespace pfsi {
namespace {
// One thread waits, with `limit` polls, for the first phase of an mbarrier
// that expects one arrival nobody makes; out[0] = 1 if the phase completed.
__global__ void k_wait_selftest(int limit, int* out)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
        out[0] = mbar_wait(&bar, 0u, limit) ? 1 : 0;
    }
}
}  // namespace
}  // namespace pfsi

extern "C" int pfsi_wait_selftest(int limit, int* dev_word, void* stream)
{
    if (limit < 1 || !dev_word) return set_error(PFSI_ERR_ARG, "pfsi_wait_selftest: bad argument");
    cudaStream_t s = as_stream(stream);
    k_wait_selftest<<<1, 32, 0, s>>>(limit, dev_word);
    int rc = check_launch("pfsi_wait_selftest");
    int h = -1;
    if (!rc) rc = check_cuda(cudaMemcpyAsync(&h, dev_word, sizeof(int), cudaMemcpyDeviceToHost, s), "pfsi_wait_selftest");
    if (!rc) rc = check_cuda(cudaStreamSynchronize(s), "pfsi_wait_selftest");
    if (rc) return rc;
    return h == 1 ? PFSI_OK : set_error(PFSI_ERR_TIMEOUT, "pfsi_wait_selftest: the wait gave up after the limit");
}
