// Implicit QL with Wilkinson shifts for a symmetric tridiagonal matrix
// (Bowdler, Martin, Reinsch & Wilkinson 1968, the "tql" algorithm; Gauss
// weights from the first row of the eigenvector matrix, Golub & Welsch 1969),
// in FP64 (double) and in double-float arithmetic (df, 48-bit significand).
// Split into the pieces the quadrature kernel runs: find_split, ql_sweep (the
// scalar chain of one sweep, recording its plane rotations) and
// apply_rotations (one row of U).
#pragma once

#include "df64.cuh"

namespace mbd {

// deflation threshold for 48-bit arithmetic
constexpr float kQLEps = 1.42e-14f;

// First m >= l with a negligible off-diagonal e[m] (or n - 1).  Called by
// all 32 lanes of a warp: lane t tests m = l + t, l + t + 32, ...
__device__ __forceinline__ bool negligible(const df *d, const df *e, int m) {
    return df_abs_hi(e[m]) <= kQLEps * (df_abs_hi(d[m]) + df_abs_hi(d[m + 1]));
}
__device__ __forceinline__ bool negligible(const double *d, const double *e, int m) {
    return fabs(e[m]) <= 2.220446049250313e-16 * (fabs(d[m]) + fabs(d[m + 1]));
}
template <class S> __device__ __forceinline__ int find_split(const S *d, const S *e, int l, int n) {
    const int lane = threadIdx.x & 31;
    for (int base = l; base < n - 1; base += 32) {
        const int m = base + lane;
        const unsigned hit = __ballot_sync(0xffffffffu, m < n - 1 && negligible(d, e, m));
        if (hit) return base + __ffs(hit) - 1;
    }
    return n - 1;
}

// One implicit QL sweep on the block l..mm (Wilkinson shift); records the
// rotation (c, s) of index i in cs[i], sn[i] for i = mm-1 down to mm-nrot.
// Returns nrot.
__device__ __forceinline__ int ql_sweep(df *d, df *e, df *cs, df *sn, int l, int mm) {
    df g = df_div(df_sub(d[l + 1], d[l]), df_mulf(e[l], 2.0f));
    df rr;
    if (df_abs_hi(g) > 1e18f) {
        rr = g.hi < 0.0f ? df_neg(g) : g;
    } else {
        const df x = df_add(df_mul(g, g), df{1.0f, 0.0f});
        rr = df_mul(x, df_rsqrt(x));
    }
    const df den = g.hi < 0.0f ? df_sub(g, rr) : df_add(g, rr);
    g = df_add(df_sub(d[mm], d[l]), df_div(e[l], den));
    df s = df{1.0f, 0.0f}, c = df{1.0f, 0.0f}, p = df{0.0f, 0.0f};
    int nrot = 0;
    for (int i = mm - 1; i >= l; --i) {
        const df f = df_mul(s, e[i]);
        const df b = df_mul(c, e[i]);
        const df x = df_add(df_mul(f, f), df_mul(g, g));
        if (x.hi == 0.0f) {                 // exact split
            e[i + 1] = df{0.0f, 0.0f};
            d[i + 1] = df_sub(d[i + 1], p);
            e[mm] = df{0.0f, 0.0f};
            return -(nrot + 1);
        }
        const df inv = df_rsqrt(x);
        rr = df_mul(x, inv);
        e[i + 1] = rr;
        s = df_mul(f, inv);
        c = df_mul(g, inv);
        g = df_sub(d[i + 1], p);
        rr = df_add(df_mul(df_sub(d[i], g), s), df_mulf(df_mul(c, b), 2.0f));
        p = df_mul(s, rr);
        d[i + 1] = df_add(g, p);
        g = df_sub(df_mul(c, rr), b);
        cs[i] = c;
        sn[i] = s;
        ++nrot;
    }
    d[l] = df_sub(d[l], p);
    e[l] = g;
    e[mm] = df{0.0f, 0.0f};
    return nrot;
}

// Apply the sweep's rotations (columns i, i+1 for i = mm-1 down) to one row of U.
__device__ __forceinline__ void apply_rotations(df *zr, const df *cs, const df *sn, int mm, int nrot) {
    for (int t = 0; t < nrot; ++t) {
        const int i = mm - 1 - t;
        const df zf = zr[i + 1];
        const df zi = zr[i];
        zr[i + 1] = df_add(df_mul(sn[i], zi), df_mul(cs[i], zf));
        zr[i] = df_sub(df_mul(cs[i], zi), df_mul(sn[i], zf));
    }
}

// ---------------------------------------------------------------- FP64

__device__ __forceinline__ int ql_sweep(double *d, double *e, double *cs, double *sn, int l, int mm) {
    double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
    double rr = sqrt(g * g + 1.0);
    g = d[mm] - d[l] + e[l] / (g + copysign(rr, g));
    double s = 1.0, c = 1.0, p = 0.0;
    int nrot = 0;
    // FP64 operations have a long latency on this part: the chain from one
    // reciprocal square root to the next is kept to five dependent operations.
    for (int i = mm - 1; i >= l; --i) {
        const double f = s * e[i];
        const double b = c * e[i];
        const double b2 = b + b;
        // r = |(f, g)|, s = f / r, c = g / r with one reciprocal square root
        const double x = fma(g, g, f * f);
        if (x == 0.0) {
            e[i + 1] = 0.0;
            d[i + 1] -= p;
            e[mm] = 0.0;
            return -(nrot + 1);
        }
        const double inv = rsqrt(x);
        rr = x * inv;
        e[i + 1] = rr;
        s = f * inv;
        c = g * inv;
        g = d[i + 1] - p;
        rr = fma(d[i] - g, s, c * b2);
        p = s * rr;
        d[i + 1] = g + p;
        g = fma(c, rr, -b);
        cs[i] = c;
        sn[i] = s;
        ++nrot;
    }
    d[l] -= p;
    e[l] = g;
    e[mm] = 0.0;
    return nrot;
}

__device__ __forceinline__ void apply_rotations(double *zr, const double *cs, const double *sn, int mm, int nrot) {
    for (int t = 0; t < nrot; ++t) {
        const int i = mm - 1 - t;
        const double zf = zr[i + 1];
        const double zi = zr[i];
        zr[i + 1] = sn[i] * zi + cs[i] * zf;
        zr[i] = cs[i] * zi - sn[i] * zf;
    }
}

__device__ __forceinline__ void to_scalar(double x, double &y) { y = x; }
__device__ __forceinline__ void to_scalar(double x, df &y) { y = df_from(x); }
__device__ __forceinline__ double from_scalar(double x) { return x; }
__device__ __forceinline__ double from_scalar(df x) { return df_to(x); }

}  // namespace mbd
