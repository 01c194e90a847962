// Device-side McMurchie-Davidson machinery (Section 2.2 and 2.3 of
// arXiv:2410.22278): Cartesian-to-Hermite coefficients E (Eqs.
// E_recursion_i, E_recursion_j, E_recursion_out), Hermite Coulomb
// integrals R (Eq. R_recursion) and the Boys function.  Everything is
// templated on the angular momenta so that loops unroll and the small
// arrays live in registers.
#pragma once
#include <cuda_runtime.h>

#include "jk_internal.h"

namespace jk {

__host__ __device__ constexpr int ncart(int l) { return (l + 1) * (l + 2) / 2; }
__host__ __device__ constexpr int nherm(int L) { return (L + 1) * (L + 2) * (L + 3) / 6; }

// Cartesian exponent of component k of a shell of momentum l along axis ax,
// order lx descending then ly descending.
__host__ __device__ constexpr int cexp(int l, int k, int ax)
{
    int n = 0;
    for (int lx = l; lx >= 0; --lx)
        for (int ly = l - lx; ly >= 0; --ly) {
            if (n == k) return ax == 0 ? lx : (ax == 1 ? ly : l - lx - ly);
            ++n;
        }
    return 0;
}

// E^{ij}_t for one axis, stored E[(i*(LB+1)+j)*(LA+LB+1)+t].  The Gaussian
// factor of Eq. E_recursion_0 is carried by the pair prefactor K, so E^{00}_0 = 1.
template <int LA, int LB, typename T>
__device__ __forceinline__ void herm_E(T PA, T PB, T oo2p, T *E)
{
    constexpr int NT = LA + LB + 1;
#pragma unroll
    for (int k = 0; k < (LA + 1) * (LB + 1) * NT; ++k) E[k] = T(0);
    E[0] = T(1);
#pragma unroll
    for (int i = 0; i <= LA; ++i)
#pragma unroll
        for (int j = 0; j <= LB; ++j) {
            if (i == 0 && j == 0) continue;
#pragma unroll
            for (int t = 0; t <= i + j; ++t) {
                T v;
                if (i > 0) {
                    const int b = ((i - 1) * (LB + 1) + j) * NT;
                    v = PA * E[b + t];
                    if (t > 0) v += oo2p * E[b + t - 1];
                    if (t + 1 <= i - 1 + j) v += T(t + 1) * E[b + t + 1];
                } else {
                    const int b = (i * (LB + 1) + j - 1) * NT;
                    v = PB * E[b + t];
                    if (t > 0) v += oo2p * E[b + t - 1];
                    if (t + 1 <= i + j - 1) v += T(t + 1) * E[b + t + 1];
                }
                E[(i * (LB + 1) + j) * NT + t] = v;
            }
        }
}

// R^0_{tuv} for t+u+v <= L from R^m_000 = s[m], in place in one dense
// (L+1)^3 buffer B[(t*(L+1)+u)*(L+1)+v]: for m = L-1 .. 0 the levels
// n = L-m .. 1 are overwritten from the R^{m+1} values still held at levels
// n-1 and n-2, then B[0] = s[m].
template <int L, typename T>
__device__ __forceinline__ void herm_R(const T *s, T X, T Y, T Z, T *B)
{
    constexpr int D = L + 1;
    B[0] = s[L];
#pragma unroll
    for (int m = L - 1; m >= 0; --m) {
#pragma unroll
        for (int n = L - m; n >= 1; --n) {
#pragma unroll
            for (int t = n; t >= 0; --t) {
#pragma unroll
                for (int u = n - t; u >= 0; --u) {
                    const int v = n - t - u;
                    T r;
                    if (t > 0) {
                        r = X * B[((t - 1) * D + u) * D + v];
                        if (t > 1) r += T(t - 1) * B[((t - 2) * D + u) * D + v];
                    } else if (u > 0) {
                        r = Y * B[(t * D + u - 1) * D + v];
                        if (u > 1) r += T(u - 1) * B[(t * D + u - 2) * D + v];
                    } else {
                        r = Z * B[(t * D + u) * D + v - 1];
                        if (v > 1) r += T(v - 1) * B[(t * D + u) * D + v - 2];
                    }
                    B[(t * D + u) * D + v] = r;
                }
            }
        }
        B[0] = s[m];
    }
}

// Boys function F_m(T), m = 0..L (Eq. boys_function_erf_form for F_0 at
// large T).  Below JK_BOYS_TMAX: a 7-term Taylor expansion of F_L about the
// nearest table point, F_L(T) = sum_j F_{L+j}(T_k) (T_k - T)^j / j!, then
// downward recursion F_m = (2T F_{m+1} + e^{-T}) / (2m+1).  Above: F_0 =
// (1/2) sqrt(pi/T) (erf(sqrt T) is 1 to double precision there) and upward
// recursion F_{m+1} = ((2m+1) F_m - e^{-T}) / (2T), stable for T > m.
template <int L>
__device__ __forceinline__ void boys(double T, const double *__restrict__ tab, double *F)
{
    if (T < JK_BOYS_TMAX) {
        const int k = __double2int_rn(T * JK_BOYS_INV_STEP);
        const double d = k * (1.0 / JK_BOYS_INV_STEP) - T;
        const double *row = tab + k * JK_BOYS_MCOL + L;
        double f = __ldg(row + 6) * (1.0 / 720.0);
        f = f * d + __ldg(row + 5) * (1.0 / 120.0);
        f = f * d + __ldg(row + 4) * (1.0 / 24.0);
        f = f * d + __ldg(row + 3) * (1.0 / 6.0);
        f = f * d + __ldg(row + 2) * 0.5;
        f = f * d + __ldg(row + 1);
        f = f * d + __ldg(row + 0);
        F[L] = f;
        if (L > 0) {
            const double e = exp(-T);
#pragma unroll
            for (int m = L - 1; m >= 0; --m) F[m] = (2.0 * T * F[m + 1] + e) * (1.0 / (2 * m + 1));
        }
    } else {
        const double e = exp(-T);
        const double oo2t = 0.5 / T;
        F[0] = 0.88622692545275801365 * rsqrt(T);  // sqrt(pi)/2 / sqrt(T)
#pragma unroll
        for (int m = 0; m < L; ++m) F[m + 1] = ((2 * m + 1) * F[m] - e) * oo2t;
    }
}

// Single-precision variant (5 Taylor terms; spacing 1/32 keeps the
// truncation near 1e-11 relative, well below float rounding).
template <int L>
__device__ __forceinline__ void boys(float T, const float *__restrict__ tab, float *F)
{
    if (T < float(JK_BOYS_TMAX)) {
        const int k = __float2int_rn(T * float(JK_BOYS_INV_STEP));
        const float d = k * (1.0f / JK_BOYS_INV_STEP) - T;
        const float *row = tab + k * JK_BOYS_MCOL + L;
        float f = __ldg(row + 4) * (1.0f / 24.0f);
        f = fmaf(f, d, __ldg(row + 3) * (1.0f / 6.0f));
        f = fmaf(f, d, __ldg(row + 2) * 0.5f);
        f = fmaf(f, d, __ldg(row + 1));
        f = fmaf(f, d, __ldg(row + 0));
        F[L] = f;
        if (L > 0) {
            const float e = __expf(-T);
#pragma unroll
            for (int m = L - 1; m >= 0; --m) F[m] = (2.0f * T * F[m + 1] + e) * (1.0f / (2 * m + 1));
        }
    } else {
        const float e = __expf(-T);
        const float oo2t = 0.5f / T;
        F[0] = 0.88622692545275801365f * rsqrtf(T);
#pragma unroll
        for (int m = 0; m < L; ++m) F[m + 1] = ((2 * m + 1) * F[m] - e) * oo2t;
    }
}

// Top order only: F_L(T) for T < JK_BOYS_TMAX by the 7-term (double) or
// 5-term (float) Taylor expansion about the nearest table point.
template <int L>
__device__ __forceinline__ double boys_top(double T, const double *__restrict__ tab)
{
    const int k = __double2int_rn(T * JK_BOYS_INV_STEP);
    const double d = k * (1.0 / JK_BOYS_INV_STEP) - T;
    const double *row = tab + k * JK_BOYS_MCOL + L;
    double f = __ldg(row + 6) * (1.0 / 720.0);
    f = f * d + __ldg(row + 5) * (1.0 / 120.0);
    f = f * d + __ldg(row + 4) * (1.0 / 24.0);
    f = f * d + __ldg(row + 3) * (1.0 / 6.0);
    f = f * d + __ldg(row + 2) * 0.5;
    f = f * d + __ldg(row + 1);
    return f * d + __ldg(row + 0);
}
template <int L>
__device__ __forceinline__ float boys_top(float T, const float *__restrict__ tab)
{
    const int k = __float2int_rn(T * float(JK_BOYS_INV_STEP));
    const float d = k * (1.0f / JK_BOYS_INV_STEP) - T;
    const float *row = tab + k * JK_BOYS_MCOL + L;
    float f = __ldg(row + 4) * (1.0f / 24.0f);
    f = fmaf(f, d, __ldg(row + 3) * (1.0f / 6.0f));
    f = fmaf(f, d, __ldg(row + 2) * 0.5f);
    f = fmaf(f, d, __ldg(row + 1));
    return fmaf(f, d, __ldg(row + 0));
}

// Screening arithmetic in single precision (it decides which terms to form,
// not their values): approximate reciprocal, quotient and square root (within
// 2 ulp; the radii carry margins far wider).  The terms themselves use the
// correctly rounded operations.
__device__ __forceinline__ float frcp_fast(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ float fdiv_fast(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ float fsqrt_fast(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ double erfc_(double x) { return erfc(x); }
__device__ __forceinline__ float erfc_(float x) { return erfcf(x); }
__device__ __forceinline__ double exp_(double x) { return exp(x); }
__device__ __forceinline__ float exp_(float x) { return expf(x); }

// Range-separated Boys integrals G_m(T, c) = int_c^1 t^{2m} e^{-T t^2} dt,
// m = 0..L.  The erfc-attenuated seed of the real-space sum is
//   (-2a)^m F_m(aX^2) - c_w (-2a_w)^m F_m(a_w X^2) = (-2a)^m G_m(aX^2, c_w)
// (substitute t -> t c_w in the second Boys integral), so the difference of
// two nearly equal Boys values never has to be formed.  Integration by parts
// gives (2m+1) G_m - 2T G_{m+1} = e^{-T} - c^{2m+1} e^{-c^2 T}:
//   small T: G_L = F_L(T) - c^{2L+1} F_L(c^2 T) from the table, downward;
//   large T: G_0 = sqrt(pi)/(2 sqrt T) (erfc(c sqrt T) - erfc(sqrt T)), upward.
template <int L, typename T>
__device__ __forceinline__ void boys_attenuated(T Tt, T c, const T *__restrict__ tab, T *G)
{
    const T c2 = c * c;
    const T e1 = exp_(-Tt), e2 = exp_(-c2 * Tt);
    if (Tt < T(L) + T(1.5)) {
        T cp = c;  // c^{2m+1}
#pragma unroll
        for (int m = 0; m < L; ++m) cp *= c2;
        G[L] = boys_top<L>(Tt, tab) - cp * boys_top<L>(c2 * Tt, tab);
#pragma unroll
        for (int m = L - 1; m >= 0; --m) {
            cp /= c2;
            G[m] = (T(2) * Tt * G[m + 1] + e1 - cp * e2) * (T(1) / T(2 * m + 1));
        }
    } else {
        const T s = sqrt(Tt);
        // erfc(s) < 2.2e-17 for s >= 6: below the rounding of erfc(c s) in
        // every term that passes screening, and an erfc saved
        T es = T(0);
        if (s < T(6)) es = erfc_(s);
        G[0] = T(0.88622692545275801365) / s * (erfc_(c * s) - es);
        T cp = c;
        const T h = T(0.5) / Tt;
#pragma unroll
        for (int m = 0; m < L; ++m) {
            G[m + 1] = (T(2 * m + 1) * G[m] - e1 + cp * e2) * h;
            cp *= c2;
        }
    }
}

}  // namespace jk
