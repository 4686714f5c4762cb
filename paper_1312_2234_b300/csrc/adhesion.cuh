// adhesion.cuh -- FP64 receptor-site geometry shared by the wall bonds
// (bonds.cu) and the platelet-platelet bridges (bridges.cu), Section 3.2.
// Every operation is explicitly rounded in the order of the plain
// restatement, so that a stochastic decision differs from it only when a
// uniform lands within an ulp of its probability.
#pragma once

#include "pfsi_internal.cuh"

namespace pfsi {

// w0 X_a + w1 X_b + (1 - w0 - w1) X_c, component d
__device__ __forceinline__ double site_coord(const double* __restrict__ X, int M, int d, int a, int b, int c,
                                            double w0, double w1)
{
    const double w2 = __dsub_rn(__dsub_rn(1.0, w0), w1);
    return __dadd_rn(__dadd_rn(__dmul_rn(w0, X[d * M + a]), __dmul_rn(w1, X[d * M + b])),
                     __dmul_rn(w2, X[d * M + c]));
}

__device__ __forceinline__ double min_image(double d, int L)
{
    const double Ld = (double)L;
    return __dsub_rn(d, __dmul_rn(Ld, floor(__dadd_rn(__ddiv_rn(d, Ld), 0.5))));
}

__device__ __forceinline__ double norm3_rn(double a, double b, double c)
{
    return __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b)), __dmul_rn(c, c)));
}

struct SitePos {
    double x, y, z;
};

// Receptor site s: barycentric point of triangle site_tri[s].
__device__ __forceinline__ SitePos site_pos(const int* __restrict__ site_tri, const double* __restrict__ site_w,
                                            const int* __restrict__ tri, const double* __restrict__ X, int M, int s)
{
    const int t = site_tri[s];
    const int a = tri[3 * t], b = tri[3 * t + 1], cc = tri[3 * t + 2];
    const double w0 = site_w[2 * s], w1 = site_w[2 * s + 1];
    return {site_coord(X, M, 0, a, b, cc, w0, w1), site_coord(X, M, 1, a, b, cc, w0, w1),
            site_coord(X, M, 2, a, b, cc, w0, w1)};
}

// Adds f * (w0, w1, 1 - w0 - w1) to the three nodes of site s's triangle.
__device__ __forceinline__ void site_add_force(const int* __restrict__ site_tri, const double* __restrict__ site_w,
                                               const int* __restrict__ tri, float* __restrict__ F, int M, int s,
                                               const double f[3])
{
    const int t = site_tri[s];
    const double w0 = site_w[2 * s], w1 = site_w[2 * s + 1];
    const float w[3] = {(float)w0, (float)w1, (float)(1.0 - w0 - w1)};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int node = tri[3 * t + k];
#pragma unroll
        for (int dd = 0; dd < 3; ++dd) atomicAdd(&F[dd * M + node], w[k] * (float)f[dd]);
    }
}

__device__ __forceinline__ uint64_t current_step(const unsigned long long* step_dev, uint64_t step_host)
{
    return step_dev ? (uint64_t)*step_dev : step_host;
}

}  // namespace pfsi
