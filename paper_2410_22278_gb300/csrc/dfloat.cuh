// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// floats with |lo| <= ulp(hi), about 44 significant bits.  Error-free
// transformations (Knuth's two-sum, Dekker's fast two-sum, the FMA
// two-product) run on the FP32 pipe, which on this GPU has 64 times the
// throughput of the FP64 pipe.  Used by the mixed-precision structure
// factors, whose accuracy target (relative 1e-11 on a structure factor)
// sits between FP32 and FP64.
//
// Every function is __host__ __device__ so the host can check the same
// arithmetic against extended precision; fmaf is correctly rounded on both.
#pragma once
#include <cmath>
#include <cuda_runtime.h>

namespace jk {

struct dfl {
    float hi, lo;
};

// s + e = a + b exactly (any a, b)
__host__ __device__ __forceinline__ dfl two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

// s + e = a + b exactly when |a| >= |b| (or a == 0)
__host__ __device__ __forceinline__ dfl fast_two_sum(float a, float b)
{
    const float s = a + b;
    const float e = b - (s - a);
    return {s, e};
}

__host__ __device__ __forceinline__ dfl df_add(dfl a, dfl b)
{
    dfl s = two_sum(a.hi, b.hi);
    s.lo += a.lo + b.lo;
    return fast_two_sum(s.hi, s.lo);
}

__host__ __device__ __forceinline__ dfl df_neg(dfl a) { return {-a.hi, -a.lo}; }

__host__ __device__ __forceinline__ dfl df_sub(dfl a, dfl b) { return df_add(a, df_neg(b)); }

__host__ __device__ __forceinline__ dfl df_mul(dfl a, dfl b)
{
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}

// a * f for a plain float f
__host__ __device__ __forceinline__ dfl df_mulf(dfl a, float f)
{
    const float p = a.hi * f;
    float e = fmaf(a.hi, f, -p);
    e = fmaf(a.lo, f, e);
    return fast_two_sum(p, e);
}

// split of a double into hi + lo (host side and table set-up)
__host__ __device__ __forceinline__ dfl dfl_split(double x)
{
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}

__host__ __device__ __forceinline__ double dfl_value(dfl a) { return (double)a.hi + (double)a.lo; }

// 2 pi as a double-float
constexpr float kTwoPiHi = 6.28318548202514648f;      // float nearest 2 pi
constexpr float kTwoPiLo = -1.74845553146951440e-7f;  // 2 pi - kTwoPiHi

// The phase of e^{-iG.P} in turns, reduced exactly.  With G = sum_k n_k b_k
// (b_k the reciprocal vectors, integer n_k) and f_k the fractional
// coordinates of P, G.P = 2 pi sum_k n_k f_k, and only sum_k n_k f_k mod 1
// matters.  Each f_k (already reduced to [-1/2, 1/2]) comes as three floats
// f1 + f2 + f3: f1 on the grid 2^-16, f2 on the grid 2^-33 (|f2| <= 2^-17),
// f3 the rest (|f3| <= 2^-34).  For |n_k| <= 64 the sums u1 = sum n_k f1_k
// and u2 = sum n_k f2_k are exact in float (at most 23 significant bits), so
// u1 - j/1024 with j = rint(1024 (u1 + u2)) is exact too, and the remainder
// w = (u1 - j/1024) + u2 + u3 (|w| <= 2^-11 + 2^-18) comes out as a
// double-float with absolute error below 1e-15 turns.  Returns j (the index
// into a 1024-entry table of (cos, sin)(2 pi j / 1024)) and w.
__host__ __device__ __forceinline__ int df_turns(float n1, float n2, float n3, const float f1[3], const float f2[3], const float f3[3],
                                                 dfl &w)
{
    const float u1 = fmaf(n3, f1[2], fmaf(n2, f1[1], n1 * f1[0]));
    const float u2 = fmaf(n3, f2[2], fmaf(n2, f2[1], n1 * f2[0]));
    const float u3 = fmaf(n3, f3[2], fmaf(n2, f3[1], n1 * f3[0]));
    const float jf = rintf((u1 + u2) * 1024.0f);
    const float ua = u1 - jf * (1.0f / 1024.0f);
    dfl s = two_sum(ua, u2);
    w = fast_two_sum(s.hi, s.lo + u3);
    return (int)jf;
}

// cos and sin of 2 pi (j/1024 + w) from the table entry
// t = (cos hi, cos lo, sin hi, sin lo) of 2 pi j / 1024 and the remainder w
// (|w| <= 2^-11 + 2^-18 turns): e = 2 pi w (|e| <= 3.1e-3) by Taylor series,
// sin e = e - e^3/6 + e^5/120 (next term < 5e-22) and
// cos e = 1 - e^2/2 + e^4/24 (next term < 2e-18), the small terms in float;
// then the angle-addition formulas in double-float.
__host__ __device__ __forceinline__ void df_sincos_turns(dfl w, float4 t, dfl &c, dfl &s)
{
    const dfl e = df_mul(w, dfl{kTwoPiHi, kTwoPiLo});
    // e^2 as a double-float
    const float p = e.hi * e.hi;
    const float pe = fmaf(2.0f * e.hi, e.lo, fmaf(e.hi, e.hi, -p));
    const dfl e2 = fast_two_sum(p, pe);
    const float e2f = e2.hi;
    // sin e
    const float c3 = e.hi * e2f * fmaf(e2f, 1.0f / 120.0f, -1.0f / 6.0f);
    const dfl se = fast_two_sum(e.hi, e.lo + c3);
    // cos e = (1 - e2/2) + e2^2/24
    const float h = 0.5f * e2.hi;
    const float chi = 1.0f - h;
    const float clo = ((1.0f - chi) - h) - 0.5f * e2.lo + e2f * e2f * (1.0f / 24.0f);
    const dfl ce = fast_two_sum(chi, clo);
    const dfl ca{t.x, t.y}, sa{t.z, t.w};
    c = df_sub(df_mul(ca, ce), df_mul(sa, se));
    s = df_add(df_mul(sa, ce), df_mul(ca, se));
}

// Host: a fractional coordinate reduced to [-1/2, 1/2] and split into the
// three floats df_turns expects (grid 2^-16, grid 2^-33, rest).
inline void frac_split3(long double f, float out[3])
{
    f -= rintl(f);
    const long double f1 = rintl(f * 65536.0L) / 65536.0L;
    const long double f2 = rintl((f - f1) * 8589934592.0L) / 8589934592.0L;
    out[0] = (float)f1;
    out[1] = (float)f2;
    out[2] = (float)(f - f1 - f2);
}

}  // namespace jk
