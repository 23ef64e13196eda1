// Double-float ("df") arithmetic on the FP32 pipes: a value is the unevaluated
// sum h + l of two floats with |l| <= ulp(h)/2, about 48 significant bits.
// Error-free transformations: Knuth's TwoSum and Dekker's TwoProduct (with a
// fused multiply-add for the exact product error); the operations follow the
// double-double algorithms of Dekker (1971) and Hida, Li & Bailey (2001) in
// their "sloppy" forms, whose error is a few units of 2^-44 of the operands.
// Used where FP64 accuracy is needed at FP32 throughput (GB300: 64 FP32 lanes
// per FP64 lane).  Products and sums inside the transformations use the
// __fmul_rn / __fadd_rn intrinsics, which the compiler never contracts into
// a fused multiply-add (contraction would break the exactness).
#pragma once
#include <cuda_runtime.h>

namespace am {

struct df {
    float h, l;
};

__device__ __forceinline__ df df_make(float h, float l) { return df{h, l}; }

// split of a double into a df (exact to 2^-48 relative)
__device__ __forceinline__ df df_from(double x) {
    const float h = (float)x;
    return df{h, (float)(x - (double)h)};
}
__device__ __forceinline__ double df_to(df x) { return (double)x.h + (double)x.l; }

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float v = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
    return df{s, e};
}
// s + e = a + b exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return df{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df df_add(df x, df y) {
    const df s = two_sum(x.h, y.h);
    return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(x.l, y.l)));
}
__device__ __forceinline__ df df_neg(df x) { return df{-x.h, -x.l}; }
__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df_neg(y)); }

// x * y: exact product of the heads by FMA, cross terms, renormalised
__device__ __forceinline__ df df_mul(df x, df y) {
    const float p = __fmul_rn(x.h, y.h);
    float e = fmaf(x.h, y.h, -p);
    e = fmaf(x.h, y.l, e);
    e = fmaf(x.l, y.h, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ df df_mul_f(df x, float c) {
    const float p = __fmul_rn(x.h, c);
    const float e = fmaf(x.l, c, fmaf(x.h, c, -p));
    return fast_two_sum(p, e);
}
// exact scaling by a power of two
__device__ __forceinline__ df df_scale2(df x, float pow2) { return df{x.h * pow2, x.l * pow2}; }

// x * y + z with one renormalisation
__device__ __forceinline__ df df_fma(df x, df y, df z) {
    const float p = __fmul_rn(x.h, y.h);
    const float pe = fmaf(x.h, y.h, -p);
    const df s = two_sum(p, z.h);
    const float t = fmaf(x.h, y.l, fmaf(x.l, y.h, z.l));
    return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(pe, t)));
}

// 1 / sqrt(x) for x > 0: the FP32 estimate refined by one Newton step for
// the inverse square root, y1 = y0 + y0 (1 - x y0^2) / 2, with x y0^2
// formed in df; the step's quadratic convergence takes the estimate's
// relative error e to about e^2 (the FP32 estimate is good to a few units
// of 2^-23).
__device__ __forceinline__ df df_rsqrt(df x) {
    const float y0 = rsqrtf(x.h);
    const float y0y0 = __fmul_rn(y0, y0);
    const df y2 = df{y0y0, fmaf(y0, y0, -y0y0)};
    const df t = df_mul(x, y2);  // close to 1
    const float e = __fsub_rn(__fsub_rn(1.0f, t.h), t.l);  // 1 - t.h exact (Sterbenz)
    return fast_two_sum(y0, __fmul_rn(0.5f * y0, e));
}

// sign of x - y (exact comparison of the represented values)
__device__ __forceinline__ bool df_ge(df x, df y) {
    return __fadd_rn(__fsub_rn(x.h, y.h), __fsub_rn(x.l, y.l)) >= 0.0f;
}

}  // namespace am
