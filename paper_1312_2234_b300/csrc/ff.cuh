// ff.cuh -- double-float ("float-float") arithmetic on the FP32 pipes.
//
// A value is an unevaluated sum h + l of two floats with |l| <= ulp(h)/2,
// about 48 significant bits.  Built from the error-free transformations of
// Knuth (two-sum), Dekker (fast two-sum) and the FMA product; errors are
// bounded in absolute terms by ~2^-47 of the operands' magnitudes, which is
// what the cancelling differences of the membrane model need (a strain of
// 1e-6 still keeps ~7 significant digits).  B300's FP64 rate is a small
// fraction of its FP32 rate, so these few dozen FP32 operations are cheaper
// than the equivalent FP64 ones.  The compiler must not reassociate (no
// fast-math flags are used on this library).
#pragma once

#include <cmath>

#ifdef __CUDA_ARCH__
#define PFSI_FMAF(a, b, c) __fmaf_rn(a, b, c)
#else
#define PFSI_FMAF(a, b, c) std::fma(a, b, c)
#endif

namespace pfsi {

struct ff {
    float h, l;
};
struct ff3 {
    ff x, y, z;
};

__host__ __device__ __forceinline__ ff ff_two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__host__ __device__ __forceinline__ ff ff_fast(float a, float b)  // requires |a| >= |b| (or a == 0)
{
    const float s = a + b;
    return {s, b - (s - a)};
}
__host__ __device__ __forceinline__ ff ff_prod(float a, float b)
{
    const float p = a * b;
    return {p, PFSI_FMAF(a, b, -p)};
}
__host__ __device__ __forceinline__ ff ff_add(ff a, ff b)
{
    const ff s = ff_two_sum(a.h, b.h);
    return ff_fast(s.h, s.l + (a.l + b.l));
}
__host__ __device__ __forceinline__ ff ff_neg(ff a) { return {-a.h, -a.l}; }
__host__ __device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }
__host__ __device__ __forceinline__ ff ff_mul(ff a, ff b)
{
    const ff p = ff_prod(a.h, b.h);
    return ff_fast(p.h, p.l + (a.h * b.l + a.l * b.h));
}
__host__ __device__ __forceinline__ ff ff_sqrt(ff a)
{
    if (!(a.h > 0.f)) return {0.f, 0.f};
    const float h = sqrtf(a.h);
    const ff r = ff_prod(h, h);
    return ff_fast(h, ((a.h - r.h) - r.l + a.l) / (2.f * h));
}
__host__ __device__ __forceinline__ float ff_float(ff a) { return a.h + a.l; }

// (a - b) of two split coordinates (h, l), exactly up to the rounding of the
// low parts.
__host__ __device__ __forceinline__ ff ff_diff(float ah, float al, float bh, float bl)
{
    const ff s = ff_two_sum(ah, -bh);
    return ff_fast(s.h, s.l + (al - bl));
}

__host__ __device__ __forceinline__ ff3 ff3_neg(ff3 a) { return {ff_neg(a.x), ff_neg(a.y), ff_neg(a.z)}; }
__host__ __device__ __forceinline__ ff ff3_dot(ff3 a, ff3 b)
{
    return ff_add(ff_add(ff_mul(a.x, b.x), ff_mul(a.y, b.y)), ff_mul(a.z, b.z));
}
__host__ __device__ __forceinline__ ff3 ff3_cross(ff3 a, ff3 b)
{
    return {ff_sub(ff_mul(a.y, b.z), ff_mul(a.z, b.y)), ff_sub(ff_mul(a.z, b.x), ff_mul(a.x, b.z)),
            ff_sub(ff_mul(a.x, b.y), ff_mul(a.y, b.x))};
}

// |d|^2 - C for a short vector d (double-float) and a constant C close to
// |d|^2: the leading difference is exact (Sterbenz) and the tails are summed
// separately, so the result is accurate to ~2^-46 |d|^2 absolute.
__host__ __device__ __forceinline__ float ff3_sqnorm_minus(ff3 d, ff C)
{
    const ff p0 = ff_prod(d.x.h, d.x.h), p1 = ff_prod(d.y.h, d.y.h), p2 = ff_prod(d.z.h, d.z.h);
    const ff s = ff_two_sum(p0.h, p1.h);
    const ff t = ff_two_sum(s.h, p2.h);
    const float lead = t.h - C.h;
    const float cross = 2.f * (d.x.h * d.x.l + d.y.h * d.y.l + d.z.h * d.z.l);
    const float tail = ((s.l + t.l) + (p0.l + p1.l + p2.l)) + cross - C.l;
    return lead + tail;
}

// a . b - C, same scheme (C close to a . b, or the result not small).
__host__ __device__ __forceinline__ float ff3_dot_minus(ff3 a, ff3 b, ff C)
{
    const ff p0 = ff_prod(a.x.h, b.x.h), p1 = ff_prod(a.y.h, b.y.h), p2 = ff_prod(a.z.h, b.z.h);
    const ff s = ff_two_sum(p0.h, p1.h);
    const ff t = ff_two_sum(s.h, p2.h);
    const ff lead = ff_two_sum(t.h, -C.h);
    const float cross = (a.x.h * b.x.l + a.x.l * b.x.h) + (a.y.h * b.y.l + a.y.l * b.y.h) +
                        (a.z.h * b.z.l + a.z.l * b.z.h);
    const float tail = ((s.l + t.l) + (p0.l + p1.l + p2.l)) + cross - C.l;
    return lead.h + (lead.l + tail);
}

}  // namespace pfsi
