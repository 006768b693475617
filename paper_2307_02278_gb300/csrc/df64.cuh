// Double-float ("df64") arithmetic: a value is the unevaluated sum hi + lo of
// two FP32 numbers, about 48 significant bits.  Error-free transformations:
// TwoSum (Knuth, TAOCP vol. 2), QuickTwoSum and the FMA-based TwoProduct
// (Dekker 1971; Hida, Li & Bailey, double-double/quad-double library 2001).
// Used where a long chain of dependent scalar operations would otherwise issue
// on the FP64 pipe, whose per-instruction cost on this GPU is about 64 times
// that of an FP32 instruction.
#pragma once

namespace mbd {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_from(double x) {
    const float h = (float)x;
    return df{h, (float)(x - (double)h)};
}
__device__ __forceinline__ double df_to(df a) { return (double)a.hi + (double)a.lo; }

// s + e == a + b exactly
__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return df{s, e};
}
// s + e == a + b exactly, requires |a| >= |b| (or a == 0)
__device__ __forceinline__ df quick_two_sum(float a, float b) {
    const float s = a + b;
    return df{s, b - (s - a)};
}
__device__ __forceinline__ df df_add(df a, df b) {
    const df s = two_sum(a.hi, b.hi);
    const df t = two_sum(a.lo, b.lo);
    df u = quick_two_sum(s.hi, s.lo + t.hi);
    return quick_two_sum(u.hi, u.lo + t.lo);
}
__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ df df_mul(df a, df b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return quick_two_sum(p, e);
}
__device__ __forceinline__ df df_mulf(df a, float b) {
    const float p = a.hi * b;
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return quick_two_sum(p, e);
}
// 1/sqrt(x), x > 0: FP32 seed, two Newton-Raphson steps y <- y (3 - x y^2) / 2
__device__ __forceinline__ df df_rsqrt(df x) {
    df y = df{rsqrtf(x.hi), 0.0f};
    for (int it = 0; it < 2; ++it) {
        const df xy2 = df_mul(x, df_mul(y, y));
        const df t = df_sub(df{1.5f, 0.0f}, df_mulf(xy2, 0.5f));
        y = df_mul(y, t);
    }
    return y;
}
// a / b: FP32 reciprocal seed, two Newton-Raphson steps y <- y (2 - b y), then a y
__device__ __forceinline__ df df_div(df a, df b) {
    df y = df{1.0f / b.hi, 0.0f};
    for (int it = 0; it < 2; ++it) y = df_mul(y, df_sub(df{2.0f, 0.0f}, df_mul(b, y)));
    return df_mul(a, y);
}
__device__ __forceinline__ float df_abs_hi(df a) { return a.hi < 0.0f ? -a.hi : a.hi; }

}  // namespace mbd
