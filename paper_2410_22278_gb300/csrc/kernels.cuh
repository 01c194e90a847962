// Quartet-class kernels of the J/K build.
//
// Real space (erfc part of Eq. pbc_eri_general_final): one thread per
// unique pair of shell-pair images (bra, ket); the thread contracts the
// Cartesian block over the primitive pairs of both images and over the R1
// lattice images inside the sphere of Eq. pbc_eri_real_cutoff_implementation,
// then digests the block into the J and K accumulators with the weights of
// the 8-element permutation orbit.  The 32 lanes of a warp hold 32 bras and
// walk the same ket, so the ket-side Coulomb term is reduced with warp
// shuffles before one atomic per element.
//
// Reciprocal space (erf part): per unique shell pair and reciprocal vector,
// the Bloch-summed pair-density structure factor
//   rho_ab(G) = sum_R sum_prims K (pi/p)^{3/2} e^{-G^2/4p} e^{-iG.P}
//               prod_axis sum_t E^{ab}_t (-iG)^t,
// scaled by sqrt(8 pi w(G) / V), written into a dense complex n x n slab.
#pragma once
#include <cuda_runtime.h>

#include "dfloat.cuh"
#include "jk_internal.h"
#include "flops.h"
#include "md.cuh"

namespace jk {

constexpr double kPi = 3.14159265358979323846;
constexpr double kTwoPi52 = 34.986836655249725;  // 2 pi^{5/2}
constexpr int kRealThreads = 128;


__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) { return warp_sum(v); }

// Running sum over the ket loop: plain in double; in float a compensated
// (two-sum) pair, so the per-lane Coulomb partial keeps ~48 bits.
template <typename T>
struct Acc;
template <>
struct Acc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double v) { s += v; }
    __device__ __forceinline__ double value() const { return s; }
};
template <>
struct Acc<float> {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add(float v)
    {
        const float t = hi + v;
        const float bp = t - hi;
        lo += (hi - (t - bp)) + (v - bp);
        hi = t;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Attenuated seeds s_m = (-2 alpha)^m F_m(alpha X^2) - c_w (-2 alpha_w)^m F_m(alpha_w X^2)
// = (-2 alpha)^m G_m(alpha X^2, c_w)  (see boys_attenuated).
template <int L>
__device__ __forceinline__ void seeds(double x2, double alpha, double aw, double cw, const PlanDev &pl, double *s)
{
    (void)aw;
    double G[L + 1];
    boys_attenuated<L, double>(alpha * x2, cw, pl.boys, G);
    double f = 1.0;
#pragma unroll
    for (int m = 0; m <= L; ++m) {
        s[m] = f * G[m];
        f *= -2.0 * alpha;
    }
}
// Single precision unless c_w is close to 1 (the integration interval
// [c_w, 1] is short and the table branch would lose bits), where the seed is
// formed in double and rounded once.
// Single precision throughout.  The mixed path sends every quartet whose
// largest c_w exceeds 0.85 (the integration interval [c_w, 1] is short and
// the table branch would lose bits) to the FP64 list instead (k_real, mode
// 2), so this form never sees such a seed.
template <int L>
__device__ __forceinline__ void seeds(float x2, float alpha, float aw, float cw, const PlanDev &pl, float *s)
{
    (void)aw;
    float G[L + 1];
    boys_attenuated<L, float>(alpha * x2, cw, pl.boys_f, G);
    float f = 1.0f;
#pragma unroll
    for (int m = 0; m <= L; ++m) {
        s[m] = f * G[m];
        f *= -2.0f * alpha;
    }
}

// Exact float -> double with integer operations only, for the FP64
// digestion atomics of the FP32 kernels: a conversion instruction would run
// on the FP64 pipe, which here has 1/64 of the FP32 rate.  Zero and
// subnormal floats (below 1.2e-38, far under any digested term) give 0.
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x)
{
    const unsigned u = __float_as_uint(x);
    const unsigned e = (u >> 23) & 0xffu;
    const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3);
    const unsigned lo = u << 29;
    return e ? __hiloint2double((int)hi, (int)lo) : 0.0;
}

// Pair data in the kernel's working precision.
template <typename T>
struct PairT {
    T P[3], PA[3], PB[3], p, ip, K;
};
__device__ __forceinline__ void load_pair(const PlanDev &pl, int k, const PpiF &, PairT<double> &o)
{
    const PpiRec x = pl.ppi[k];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        o.P[a] = x.P[a];
        o.PA[a] = x.PA[a];
        o.PB[a] = x.PB[a];
    }
    o.p = x.p;
    o.ip = x.pad;
    o.K = x.K;
}
__device__ __forceinline__ void load_pair(const PlanDev &, int, const PpiF &f, PairT<float> &o)
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        o.P[a] = f.P[a];
        o.PA[a] = f.PA[a];
        o.PB[a] = f.PB[a];
    }
    o.p = f.p;
    o.ip = f.pad;
    o.K = f.K;
}
__device__ __forceinline__ double latc(const double *d, const float *, int k, double) { return d[k]; }
__device__ __forceinline__ float latc(const double *, const float *f, int k, float) { return f[k]; }
__device__ __forceinline__ double lat_at(const PlanDev &pl, int k, double) { return pl.r1[k]; }
__device__ __forceinline__ float lat_at(const PlanDev &pl, int k, float) { return pl.r1f[k]; }

// Contracted real-space block V[((a*NB+b)*NC+c)*ND+d] of one pair of
// shell-pair images.  The sphere of Eq. pbc_eri_real_cutoff_implementation
// and the R1 candidate tests are evaluated in single precision for both
// kernels (they only decide which terms to form); the terms themselves are
// formed in T.
template <int LA, int LB, int LC, int LD, typename T>
__device__ __forceinline__ void quartet_block(const PlanDev &pl, const SpiRec &sb, const SpiRec &sk, T *V, Tally &tl)
{
    constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
    constexpr int L = LA + LB + LC + LD, LAB = LA + LB, LCD = LC + LD;
    constexpr int NTA = LAB + 1, NTC = LCD + 1, D = L + 1;
    // classes of total momentum >= 6 (d shells) keep their component loops
    // rolled: full unrolling there only bloats code and compile time
    constexpr int UNR = L >= 6 ? 1 : 64;
    const float iw2 = pl.inv_omega2f;
    // primitive pairs are in descending order of B = |K| p^{-5/4}: the loops
    // end at the first pair whose bound B_i B_j falls below the threshold
    const float Bk0 = __ldg(pl.ppB + sk.pp0);
    for (int i = 0; i < sb.npp; ++i) {
        const float Bi = __ldg(pl.ppB + sb.pp0 + i);
        if (Bi * Bk0 < pl.mag_thr) break;
        const PpiF xf = pl.ppf[sb.pp0 + i];
        PairT<T> x;
        load_pair(pl, sb.pp0 + i, xf, x);
        T Ea[3][(LA + 1) * (LB + 1) * NTA];
        const T oo2p = T(0.5) * x.ip;
        ++tl.brap;
#pragma unroll
        for (int k = 0; k < 3; ++k) herm_E<LA, LB, T>(x.PA[k], x.PB[k], oo2p, Ea[k]);
        for (int j = 0; j < sk.npp; ++j) {
            if (Bi * __ldg(pl.ppB + sk.pp0 + j) < pl.mag_thr) break;
            const PpiF yf = pl.ppf[sk.pp0 + j];
            // ---- screening, single precision
            const float ipf = xf.pad, iqf = yf.pad;
            const float awf = frcp_fast(ipf + iqf + iw2);
            const float cwf = fsqrt_fast(awf * (ipf + iqf));
            const float preff = 34.986836655249725f * xf.K * yf.K * ipf * iqf * rsqrtf(xf.p + yf.p);
            ++tl.screen;

            const float lg = __logf(fabsf(preff) * (1.0f - cwf)) - pl.log_ewald_R;
            if (!(lg > 0.0f)) continue;
            ++tl.radius;
            float r = fsqrt_fast(fdiv_fast(lg, awf));
            if (L > 0) {
                r = fsqrt_fast(fdiv_fast(lg + L * __logf(1.0f + 2.0f * awf * r), awf));
                r = fsqrt_fast(fdiv_fast(lg + L * __logf(1.0f + 2.0f * awf * r), awf));
                // the Gaussian bound is derived for s functions; widen for L > 0
                r += 0.5f + 0.25f * L;
            }
            const float r2 = r * r;
            PairT<T> y;
            load_pair(pl, sk.pp0 + j, yf, y);
            // minimum image of P - Q (Eq. lattice_image_min_norm), working precision
            T X0[3] = {x.P[0] - y.P[0], x.P[1] - y.P[1], x.P[2] - y.P[2]};
            {
                T f[3];
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    f[a] = rint(latc(pl.Finv, pl.Finvf, 3 * a, T(0)) * X0[0] + latc(pl.Finv, pl.Finvf, 3 * a + 1, T(0)) * X0[1] +
                                latc(pl.Finv, pl.Finvf, 3 * a + 2, T(0)) * X0[2]);
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    X0[a] -= f[0] * latc(pl.L, pl.Lf, a, T(0)) + f[1] * latc(pl.L, pl.Lf, 3 + a, T(0)) + f[2] * latc(pl.L, pl.Lf, 6 + a, T(0));
            }
            const float x0n = fsqrt_fast((float)(X0[0] * X0[0] + X0[1] * X0[1] + X0[2] * X0[2]));
            T Rs[D * D * D];
#pragma unroll
            for (int k = 0; k < D * D * D; ++k) Rs[k] = T(0);
            bool any = false;
            const T ip = x.ip, iq = y.ip;
            const T aw = T(1) / (ip + iq + latc(&pl.inv_omega2, &pl.inv_omega2f, 0, T(0)));
            const T alpha = T(1) / (ip + iq);
            const T cw = sqrt(aw * (ip + iq));
            for (int c = 0; c < pl.nr1; ++c) {
                if (pl.r1f[4 * c + 3] - x0n >= r) break;
                ++tl.cand;
                const T Xx = X0[0] - lat_at(pl, 4 * c, T(0)), Xy = X0[1] - lat_at(pl, 4 * c + 1, T(0)),
                        Xz = X0[2] - lat_at(pl, 4 * c + 2, T(0));
                const T x2 = Xx * Xx + Xy * Xy + Xz * Xz;
                if ((float)x2 >= r2) continue;
                any = true;
                ++tl.img;
                T s[L + 1];
                seeds<L>(x2, alpha, aw, cw, pl, s);
                T B[D * D * D];
                herm_R<L, T>(s, Xx, Xy, Xz, B);
#pragma unroll
                for (int t = 0; t <= L; ++t)
#pragma unroll
                    for (int u = 0; u <= L - t; ++u)
#pragma unroll
                        for (int v = 0; v <= L - t - u; ++v) Rs[(t * D + u) * D + v] += B[(t * D + u) * D + v];
            }
            if (!any) continue;
            ++tl.term;
            T Ec[3][(LC + 1) * (LD + 1) * NTC];
            const T oo2q = T(0.5) * iq;
#pragma unroll
            for (int k = 0; k < 3; ++k) herm_E<LC, LD, T>(y.PA[k], y.PB[k], oo2q, Ec[k]);
            const T tp = T(kTwoPi52) * x.K * y.K * ip * iq / sqrt(x.p + y.p);
#pragma unroll UNR
            for (int c = 0; c < NC; ++c)
#pragma unroll UNR
                for (int d = 0; d < ND; ++d) {
                    const int cx = cexp(LC, c, 0), cy = cexp(LC, c, 1), cz = cexp(LC, c, 2);
                    const int dx = cexp(LD, d, 0), dy = cexp(LD, d, 1), dz = cexp(LD, d, 2);
                    T W[NTA * NTA * NTA];
#pragma unroll
                    for (int tx = 0; tx <= LAB; ++tx)
#pragma unroll
                        for (int ty = 0; ty <= LAB - tx; ++ty)
#pragma unroll
                            for (int tz = 0; tz <= LAB - tx - ty; ++tz) {
                                T acc = T(0);
#pragma unroll
                                for (int sx = 0; sx <= cx + dx; ++sx)
#pragma unroll
                                    for (int sy = 0; sy <= cy + dy; ++sy)
#pragma unroll
                                        for (int sz = 0; sz <= cz + dz; ++sz) {
                                            const T e = Ec[0][(cx * (LD + 1) + dx) * NTC + sx] * Ec[1][(cy * (LD + 1) + dy) * NTC + sy] *
                                                        Ec[2][(cz * (LD + 1) + dz) * NTC + sz];
                                            const T rv = Rs[((tx + sx) * D + ty + sy) * D + tz + sz];
                                            if ((sx + sy + sz) & 1)
                                                acc -= e * rv;
                                            else
                                                acc += e * rv;
                                        }
                                W[(tx * NTA + ty) * NTA + tz] = acc;
                            }
#pragma unroll UNR
                    for (int a = 0; a < NA; ++a)
#pragma unroll UNR
                        for (int b = 0; b < NB; ++b) {
                            const int ax = cexp(LA, a, 0), ay = cexp(LA, a, 1), az = cexp(LA, a, 2);
                            const int bx = cexp(LB, b, 0), by = cexp(LB, b, 1), bz = cexp(LB, b, 2);
                            T v = T(0);
#pragma unroll
                            for (int tx = 0; tx <= ax + bx; ++tx)
#pragma unroll
                                for (int ty = 0; ty <= ay + by; ++ty)
#pragma unroll
                                    for (int tz = 0; tz <= az + bz; ++tz)
                                        v += Ea[0][(ax * (LB + 1) + bx) * NTA + tx] * Ea[1][(ay * (LB + 1) + by) * NTA + ty] *
                                             Ea[2][(az * (LB + 1) + bz) * NTA + tz] * W[(tx * NTA + ty) * NTA + tz];
                            V[((a * NB + b) * NC + c) * ND + d] += tp * v;
                        }
                }
        }
    }
}

// Quartet-level real-space bound: false only if no primitive quartet of the
// pair of images can have an image term inside its screening sphere, so the
// quartet contributes nothing and its primitive loop can be skipped.  Every
// primitive prefactor 2 pi^{5/2} |K_i K_j| / (p q sqrt(p+q)) is at most
// 2 pi^{5/2} 2^{-1/2} |K_i| p^{-5/4} |K_j| q^{-5/4} (p + q >= 2 sqrt(pq)), so
// sum-free B0 = 2 pi^{5/2} 2^{-1/2} S_bra S_ket bounds each of them; the
// screening radius grows with the prefactor and, through both terms of its
// fixed-point form, shrinks as alpha_w grows, so the radius from (B0, the
// smallest alpha_w) dominates every primitive radius.  The distance is a
// lower bound on |P_i - Q_j - R1| over all lattice vectors R1: the distance
// from the image centres' difference to the lattice (exact minimum image for
// orthogonal cells, else the largest plane-spacing projection) less both
// extents.
template <int L>
__device__ __forceinline__ bool reaches(const PlanDev &pl, const SpiRec &sb, float kx, float ky, float kz, float kext, float kS,
                                        float kpmin)
{
    const float B0 = 24.7394241f * sb.S * kS * 1.001f;  // 2 pi^{5/2} / sqrt 2
    const float lg = __logf(B0) - pl.log_ewald_R;
    if (!(lg > 0.0f)) return false;
    const float aw = frcp_fast(frcp_fast(sb.pmin) + frcp_fast(kpmin) + pl.inv_omega2f);
    float r = fsqrt_fast(fdiv_fast(lg, aw));
    if (L > 0) {
        r = fsqrt_fast(fdiv_fast(lg + L * __logf(1.0f + 2.0f * aw * r), aw));
        r = fsqrt_fast(fdiv_fast(lg + L * __logf(1.0f + 2.0f * aw * r), aw));
    }
    r = r * 1.0001f + (L > 0 ? 0.5f + 0.25f * L : 0.0f) + sb.ext + kext + 1e-3f;
    const float X[3] = {sb.Pc[0] - kx, sb.Pc[1] - ky, sb.Pc[2] - kz};
    float f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        f[a] = pl.Finvf[3 * a] * X[0] + pl.Finvf[3 * a + 1] * X[1] + pl.Finvf[3 * a + 2] * X[2];
        f[a] -= rintf(f[a]);
    }
    float d2;
    if (pl.orth) {
        float Y[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) Y[a] = f[0] * pl.Lf[a] + f[1] * pl.Lf[3 + a] + f[2] * pl.Lf[6 + a];
        d2 = Y[0] * Y[0] + Y[1] * Y[1] + Y[2] * Y[2];
    } else {
        const float d = fmaxf(fmaxf(pl.hplane[0] * fabsf(f[0]), pl.hplane[1] * fabsf(f[1])), pl.hplane[2] * fabsf(f[2]));
        d2 = d * d;
    }
    return d2 < r * r;
}
template <int L>
__device__ __forceinline__ bool quartet_reaches(const PlanDev &pl, const SpiRec &sb, const SpiRec &sk)
{
    return reaches<L>(pl, sb, sk.Pc[0], sk.Pc[1], sk.Pc[2], sk.ext, sk.S, sk.pmin);
}
// The same bound for a block of 32 consecutive ket images: the block's
// sphere contains every member's centre shifted next to the first member
// (the lattice distance to a bra does not change under that shift) plus its
// extent, and its S and exponent bound every member's, so a bra that cannot
// reach the block cannot reach any of its images.
template <int L>
__device__ __forceinline__ bool block_reaches(const PlanDev &pl, const SpiRec &sb, int blk)
{
    const float4 c = __ldg(pl.kblk + blk);
    const float2 t = __ldg(pl.kblk2 + blk);
    return reaches<L>(pl, sb, c.x, c.y, c.z, c.w, t.x, t.y);
}

// Size estimate of the real-space block of a pair of images, for the
// precision switch (not for screening): the sum over primitive quartets of
// the Gaussian bound behind Eq. pbc_eri_real_cutoff_definition,
// 2 pi^{5/2}/(pq sqrt(p+q)) |K K| (1 - c_w) exp(-alpha_w d^2), at the
// distance d between the images' centres less their extents.
__device__ __forceinline__ float quartet_estimate(const PlanDev &pl, const SpiRec &sb, const SpiRec &sk)
{
    float X[3] = {sb.Pc[0] - sk.Pc[0], sb.Pc[1] - sk.Pc[1], sb.Pc[2] - sk.Pc[2]};
    float f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) f[a] = rintf(pl.Finvf[3 * a] * X[0] + pl.Finvf[3 * a + 1] * X[1] + pl.Finvf[3 * a + 2] * X[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) X[a] -= f[0] * pl.Lf[a] + f[1] * pl.Lf[3 + a] + f[2] * pl.Lf[6 + a];
    const float d = fmaxf(0.0f, fsqrt_fast(X[0] * X[0] + X[1] * X[1] + X[2] * X[2]) - sb.ext - sk.ext);
    const float d2 = d * d, iw2 = pl.inv_omega2f;
    float est = 0.0f;
    for (int i = 0; i < sb.npp; ++i) {
        const PpiF x = pl.ppf[sb.pp0 + i];
        for (int j = 0; j < sk.npp; ++j) {
            const PpiF y = pl.ppf[sk.pp0 + j];
            const float aw = frcp_fast(x.pad + y.pad + iw2);
            const float cw = fsqrt_fast(aw * (x.pad + y.pad));
            est += 34.986836655249725f * fabsf(x.K * y.K) * x.pad * y.pad * rsqrtf(x.p + y.p) * (1.0f - cw) * __expf(-aw * d2);
        }
    }
    return est;
}

// max |D'| over the six shell blocks an image quartet (ij|kl) digests into
// (FP32 shell-block maxima; exact, so every caller gets the same value)
__device__ __forceinline__ float quartet_dmax(const float *__restrict__ dm, int nsh, const SpiRec &sb, const SpiRec &sk)
{
    const float a = fmaxf(fmaxf(dm[sb.I * nsh + sb.J], dm[sk.I * nsh + sk.J]), fmaxf(dm[sb.J * nsh + sk.I], dm[sb.I * nsh + sk.I]));
    return fmaxf(a, fmaxf(dm[sb.J * nsh + sk.J], dm[sb.I * nsh + sk.J]));
}

// O(1) upper bound of quartet_estimate (same distance d; each primitive term
// bounded as in quartet_reaches, with 1 - c_w <= 1 and the smallest alpha_w):
// quartets below tau by this bound need no per-primitive estimate.
__device__ __forceinline__ float quartet_estimate_bound(const PlanDev &pl, const SpiRec &sb, const SpiRec &sk)
{
    float X[3] = {sb.Pc[0] - sk.Pc[0], sb.Pc[1] - sk.Pc[1], sb.Pc[2] - sk.Pc[2]};
    float f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) f[a] = rintf(pl.Finvf[3 * a] * X[0] + pl.Finvf[3 * a + 1] * X[1] + pl.Finvf[3 * a + 2] * X[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) X[a] -= f[0] * pl.Lf[a] + f[1] * pl.Lf[3 + a] + f[2] * pl.Lf[6 + a];
    const float d = fmaxf(0.0f, fsqrt_fast(X[0] * X[0] + X[1] * X[1] + X[2] * X[2]) - sb.ext - sk.ext);
    const float aw = frcp_fast(frcp_fast(sb.pmin) + frcp_fast(sk.pmin) + pl.inv_omega2f);
    return 24.7394241f * 1.001f * sb.S * sk.S * __expf(-aw * d * d);
}

// mode 0: every quartet in this kernel's precision.  mode 2 (mixed
// precision, T = float): quartets whose density-weighted size estimate is
// >= tau are appended to the compact list `big` (processed afterwards in
// FP64 by k_real_list) instead of being evaluated here; if the list is full
// the quartet is evaluated here and counted in ovf.  *cnt counts the image
// quartets this launch evaluated.
template <int LA, int LB, int LC, int LD, typename T>
__global__ void __launch_bounds__(kRealThreads) k_real(PlanDev pl, int b0, int b1, int k0, int k1, int same, int kchunk, int mode,
                                                        double tau, const T *__restrict__ Dp, const T *__restrict__ dmax,
                                                        double *__restrict__ X, double *__restrict__ Y,
                                                        unsigned long long *__restrict__ cnt, int2 *__restrict__ big,
                                                        unsigned *__restrict__ nbig, unsigned cap, unsigned *__restrict__ ovf)
{
    constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
    constexpr int DUNR = LA + LB + LC + LD >= 6 ? 1 : 64;
    const int tile0 = b0 + blockIdx.x * kRealThreads;
    const int bra = tile0 + threadIdx.x;
    int kbeg = k0 + blockIdx.y * kchunk;
    const int kend = min(k1, kbeg + kchunk);
    if (same) kbeg = max(kbeg, tile0);
    if (kbeg >= kend) return;
    const bool act = bra < b1;
    const SpiRec sb = pl.spi[act ? bra : b0];
    const int n = pl.nbf, nsh = pl.nshell;
    const int aoI = pl.shells[sb.I].ao, aoJ = pl.shells[sb.J].ao;
    T Dij[NA * NB];
    Acc<T> jb[NA * NB];
#pragma unroll
    for (int a = 0; a < NA; ++a)
#pragma unroll
        for (int b = 0; b < NB; ++b) Dij[a * NB + b] = __ldg(Dp + (size_t)(aoI + a) * n + aoJ + b);
    const float tauf = (float)tau;
    unsigned nq = 0;
    Tally tl;  // event counts (flops.h)
    for (int kt = kbeg; kt < kend; ++kt) {
        // one bound per block of 32 kets for the whole warp first
        if (kt == kbeg || (kt & 31) == 0) {
            if (!__any_sync(0xffffffffu, act && block_reaches<LA + LB + LC + LD>(pl, sb, kt >> 5))) {
                kt = min(kend, ((kt >> 5) + 1) << 5) - 1;
                continue;
            }
        }
        const SpiRec sk = pl.spi[kt];
        bool valid = act && (!same || kt >= bra);
        valid = valid && quartet_reaches<LA + LB + LC + LD>(pl, sb, sk);
        if (!__any_sync(0xffffffffu, valid)) continue;  // no lane of the warp has work for this ket
        // mixed precision (mode 2, FP32 kernel): a quartet whose size estimate
        // reaches tau, or whose [c_w, 1] interval is short, is listed for the
        // FP64 pass instead of being evaluated here
        if (sizeof(T) == 4 && valid && mode) {
            const float dm = quartet_dmax(reinterpret_cast<const float *>(dmax), nsh, sb, sk);
            const float est = quartet_estimate_bound(pl, sb, sk) * dm >= tauf ? quartet_estimate(pl, sb, sk) * dm : 0.0f;
            // largest c_w^2 = (1/p + 1/q) / (1/p + 1/q + 1/w^2) over the quartet's primitives
            const float ipq = frcp_fast(sb.pmin) + frcp_fast(sk.pmin);
            if (est >= tauf || ipq > 0.7225f * (ipq + pl.inv_omega2f)) {
                const unsigned slot = atomicAdd(nbig, 1u);
                if (slot < cap) {
                    big[slot] = make_int2(bra, kt);
                    valid = false;
                } else {
                    atomicAdd(ovf, 1u);
                }
            }
        }
        T V[NA * NB * NC * ND];
#pragma unroll
        for (int k = 0; k < NA * NB * NC * ND; ++k) V[k] = T(0);
        if (valid) quartet_block<LA, LB, LC, LD, T>(pl, sb, sk, V, tl);
        nq += valid;
        tl.quart += valid;
        // orbit weight, exact in either precision
        const T w = valid ? T(sb.w) * T(sk.w) * ((same && kt == bra) ? T(0.5) : T(1)) : T(0);
        const int aoK = pl.shells[sk.I].ao, aoL = pl.shells[sk.J].ao;
        // Coulomb, bra side: X_ij += 2w sum_kl V D_kl (held over the ket loop)
        T Dkl[NC * ND];
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int d = 0; d < ND; ++d) Dkl[c * ND + d] = __ldg(Dp + (size_t)(aoK + c) * n + aoL + d);
#pragma unroll
        for (int ab = 0; ab < NA * NB; ++ab) {
            T s = T(0);
#pragma unroll
            for (int cd = 0; cd < NC * ND; ++cd) s += V[ab * NC * ND + cd] * Dkl[cd];
            jb[ab].add(T(2) * w * s);
        }
        // Coulomb, ket side: X_kl += 2w sum_ij V D_ij, summed over the warp's bras
#pragma unroll
        for (int cd = 0; cd < NC * ND; ++cd) {
            T s = T(0);
#pragma unroll
            for (int ab = 0; ab < NA * NB; ++ab) s += V[ab * NC * ND + cd] * Dij[ab];
            s = warp_sum_t(T(2) * w * s);
            if ((threadIdx.x & 31) == 0 && s != T(0)) atomicAdd(X + (size_t)(aoK + cd / ND) * n + aoL + cd % ND, to_f64(s));
        }
        // exchange: the four index assignments of the orbit (the other four are transposes)
        if (valid && Y) {
#pragma unroll DUNR
            for (int a = 0; a < NA; ++a)
#pragma unroll DUNR
                for (int d = 0; d < ND; ++d) {  // K_il += w V_ijkl D_jk
                    T s = T(0);
#pragma unroll
                    for (int b = 0; b < NB; ++b)
#pragma unroll
                        for (int c = 0; c < NC; ++c) s += V[((a * NB + b) * NC + c) * ND + d] * __ldg(Dp + (size_t)(aoJ + b) * n + aoK + c);
                    atomicAdd(Y + (size_t)(aoI + a) * n + aoL + d, to_f64(w * s));
                }
#pragma unroll DUNR
            for (int b = 0; b < NB; ++b)
#pragma unroll DUNR
                for (int d = 0; d < ND; ++d) {  // K_jl += w V_ijkl D_ik
                    T s = T(0);
#pragma unroll
                    for (int a = 0; a < NA; ++a)
#pragma unroll
                        for (int c = 0; c < NC; ++c) s += V[((a * NB + b) * NC + c) * ND + d] * __ldg(Dp + (size_t)(aoI + a) * n + aoK + c);
                    atomicAdd(Y + (size_t)(aoJ + b) * n + aoL + d, to_f64(w * s));
                }
#pragma unroll DUNR
            for (int a = 0; a < NA; ++a)
#pragma unroll DUNR
                for (int c = 0; c < NC; ++c) {  // K_ik += w V_ijkl D_jl
                    T s = T(0);
#pragma unroll
                    for (int b = 0; b < NB; ++b)
#pragma unroll
                        for (int d = 0; d < ND; ++d) s += V[((a * NB + b) * NC + c) * ND + d] * __ldg(Dp + (size_t)(aoJ + b) * n + aoL + d);
                    atomicAdd(Y + (size_t)(aoI + a) * n + aoK + c, to_f64(w * s));
                }
#pragma unroll DUNR
            for (int b = 0; b < NB; ++b)
#pragma unroll DUNR
                for (int c = 0; c < NC; ++c) {  // K_jk += w V_ijkl D_il
                    T s = T(0);
#pragma unroll
                    for (int a = 0; a < NA; ++a)
#pragma unroll
                        for (int d = 0; d < ND; ++d) s += V[((a * NB + b) * NC + c) * ND + d] * __ldg(Dp + (size_t)(aoI + a) * n + aoL + d);
                    atomicAdd(Y + (size_t)(aoJ + b) * n + aoK + c, to_f64(w * s));
                }
        }
    }
    if (act) {
#pragma unroll DUNR
        for (int a = 0; a < NA; ++a)
#pragma unroll DUNR
            for (int b = 0; b < NB; ++b) {
                const double v = jb[a * NB + b].value();
                if (v != 0.0) atomicAdd(X + (size_t)(aoI + a) * n + aoJ + b, v);
            }
    }
    // warp-aggregated counts of the image quartets this launch evaluated and
    // of their algorithmic flops (cnt[4])
    unsigned tot = nq;
    unsigned long long fl = tally_alg<LA, LB, LC, LD>(tl), fs = tally_screen<LA, LB, LC, LD>(tl);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        tot += __shfl_xor_sync(0xffffffffu, tot, o);
        fl += __shfl_xor_sync(0xffffffffu, fl, o);
        fs += __shfl_xor_sync(0xffffffffu, fs, o);
    }
    if ((threadIdx.x & 31) == 0 && tot) atomicAdd(cnt, (unsigned long long)tot);
    if ((threadIdx.x & 31) == 0 && fl) atomicAdd(cnt + 4, fl);
    if ((threadIdx.x & 31) == 0 && fs) atomicAdd(cnt + 8, fs);
}

// FP64 pass over the compact list of large quartets collected by the
// mixed-precision kernel of the same class pair (grid-stride; each entry is
// one unique pair of images, digested with the same orbit weights).
template <int LA, int LB, int LC, int LD>
__global__ void __launch_bounds__(kRealThreads) k_real_list(PlanDev pl, const int2 *__restrict__ big, const unsigned *__restrict__ nbig,
                                                             unsigned cap, int same, const double *__restrict__ Dp, double *__restrict__ X,
                                                             double *__restrict__ Y, unsigned long long *__restrict__ cnt)
{
    constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
    constexpr int DUNR = LA + LB + LC + LD >= 6 ? 1 : 64;
    const unsigned total = min(*nbig, cap);
    const int n = pl.nbf;
    unsigned done = 0;
    Tally tl;
    for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int2 q = big[e];
        const SpiRec sb = pl.spi[q.x], sk = pl.spi[q.y];
        double V[NA * NB * NC * ND];
#pragma unroll
        for (int k = 0; k < NA * NB * NC * ND; ++k) V[k] = 0.0;
        quartet_block<LA, LB, LC, LD, double>(pl, sb, sk, V, tl);
        ++tl.quart;
        ++done;
        const double w = double(sb.w) * double(sk.w) * ((same && q.x == q.y) ? 0.5 : 1.0);
        const int aoI = pl.shells[sb.I].ao, aoJ = pl.shells[sb.J].ao, aoK = pl.shells[sk.I].ao, aoL = pl.shells[sk.J].ao;
        auto Dd = [&](int r, int c) { return __ldg(Dp + (size_t)r * n + c); };
#pragma unroll DUNR
        for (int a = 0; a < NA; ++a)
#pragma unroll DUNR
            for (int b = 0; b < NB; ++b) {
                double s = 0;
#pragma unroll
                for (int c = 0; c < NC; ++c)
#pragma unroll
                    for (int d = 0; d < ND; ++d) s += V[((a * NB + b) * NC + c) * ND + d] * Dd(aoK + c, aoL + d);
                atomicAdd(X + (size_t)(aoI + a) * n + aoJ + b, 2.0 * w * s);
            }
#pragma unroll DUNR
        for (int c = 0; c < NC; ++c)
#pragma unroll DUNR
            for (int d = 0; d < ND; ++d) {
                double s = 0;
#pragma unroll
                for (int a = 0; a < NA; ++a)
#pragma unroll
                    for (int b = 0; b < NB; ++b) s += V[((a * NB + b) * NC + c) * ND + d] * Dd(aoI + a, aoJ + b);
                atomicAdd(X + (size_t)(aoK + c) * n + aoL + d, 2.0 * w * s);
            }
        if (!Y) continue;  // a Coulomb-only build
#pragma unroll DUNR
        for (int a = 0; a < NA; ++a)
#pragma unroll DUNR
            for (int d = 0; d < ND; ++d) {
                double s = 0;
#pragma unroll
                for (int b = 0; b < NB; ++b)
#pragma unroll
                    for (int c = 0; c < NC; ++c) s += V[((a * NB + b) * NC + c) * ND + d] * Dd(aoJ + b, aoK + c);
                atomicAdd(Y + (size_t)(aoI + a) * n + aoL + d, w * s);
            }
#pragma unroll DUNR
        for (int b = 0; b < NB; ++b)
#pragma unroll DUNR
            for (int d = 0; d < ND; ++d) {
                double s = 0;
#pragma unroll
                for (int a = 0; a < NA; ++a)
#pragma unroll
                    for (int c = 0; c < NC; ++c) s += V[((a * NB + b) * NC + c) * ND + d] * Dd(aoI + a, aoK + c);
                atomicAdd(Y + (size_t)(aoJ + b) * n + aoL + d, w * s);
            }
#pragma unroll DUNR
        for (int a = 0; a < NA; ++a)
#pragma unroll DUNR
            for (int c = 0; c < NC; ++c) {
                double s = 0;
#pragma unroll
                for (int b = 0; b < NB; ++b)
#pragma unroll
                    for (int d = 0; d < ND; ++d) s += V[((a * NB + b) * NC + c) * ND + d] * Dd(aoJ + b, aoL + d);
                atomicAdd(Y + (size_t)(aoI + a) * n + aoK + c, w * s);
            }
#pragma unroll DUNR
        for (int b = 0; b < NB; ++b)
#pragma unroll DUNR
            for (int c = 0; c < NC; ++c) {
                double s = 0;
#pragma unroll
                for (int a = 0; a < NA; ++a)
#pragma unroll
                    for (int d = 0; d < ND; ++d) s += V[((a * NB + b) * NC + c) * ND + d] * Dd(aoI + a, aoL + d);
                atomicAdd(Y + (size_t)(aoJ + b) * n + aoK + c, w * s);
            }
    }
    unsigned tot = done;
    unsigned long long fl = tally_alg<LA, LB, LC, LD>(tl), fs = tally_screen<LA, LB, LC, LD>(tl);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        tot += __shfl_xor_sync(0xffffffffu, tot, o);
        fl += __shfl_xor_sync(0xffffffffu, fl, o);
        fs += __shfl_xor_sync(0xffffffffu, fs, o);
    }
    if ((threadIdx.x & 31) == 0 && tot) atomicAdd(cnt, (unsigned long long)tot);
    if ((threadIdx.x & 31) == 0 && fl) atomicAdd(cnt + 4, fl);
    if ((threadIdx.x & 31) == 0 && fs) atomicAdd(cnt + 8, fs);
}

// sin and cos of a phase in FP64 by table and angle addition: theta =
// k (2 pi / 1024) + e with k = rint(theta 1024 / 2 pi), reduced with the
// step split in two (a 32-bit head, so k * head is exact for |k| < 2^21, and
// the remainder); |e| <= pi/1024 + rounding, where seven-term sine and
// eight-term cosine Taylor series are exact to double rounding; then
// sin(a + e) = sin a cos e + cos a sin e, cos(a + e) = cos a cos e - sin a sin e
// with (cos a, sin a) from the 1024-entry table.
__device__ __forceinline__ void phase_sincos(double th, const double2 *__restrict__ tab, double &s, double &c)
{
    const double kd = rint(th * 162.97466172610083);  // 1024 / (2 pi)
    double e = fma(-kd, 0.006135923151305178, th);  // 2 pi / 1024, head
    e = fma(-kd, 2.3738673853539813e-13, e);        // tail
    const double2 t = __ldg(tab + ((int)kd & 1023));
    const double e2 = e * e;
    const double se = e * (1.0 + e2 * (-1.0 / 6.0 + e2 * (1.0 / 120.0 - e2 * (1.0 / 5040.0))));
    const double ce = 1.0 + e2 * (-0.5 + e2 * (1.0 / 24.0 + e2 * (-1.0 / 720.0 + e2 * (1.0 / 40320.0))));
    s = t.y * ce + t.x * se;
    c = t.x * ce - t.y * se;
}

// Structure factors of one class of unique shell pairs for a chunk of G.
// Thread (shell pair, g) with g fastest.  M layout: [2*gcur][n][n], part 0
// real, part 1 imaginary, both scaled by sqrt(8 pi w(G)/V) (gv[4g+3]).
template <int LA, int LB>
__global__ void __launch_bounds__(128) k_sfac(PlanDev pl, int sp0, int sp1, const double *__restrict__ gv, int g0, int gcur,
                                              const double *__restrict__ gtab, double *__restrict__ M)
{
    constexpr int NA = ncart(LA), NB = ncart(LB), NT = LA + LB + 1;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int gi = (int)(idx % gcur);
    const int sp = sp0 + (int)(idx / gcur);
    if (sp >= sp1) return;
    const SpairRec rec = pl.spair[sp];
    const double Gx = gv[4 * (g0 + gi)], Gy = gv[4 * (g0 + gi) + 1], Gz = gv[4 * (g0 + gi) + 2], sw = gv[4 * (g0 + gi) + 3];
    const double Gv[3] = {Gx, Gy, Gz};
    double re[NA * NB], im[NA * NB];
#pragma unroll
    for (int k = 0; k < NA * NB; ++k) re[k] = im[k] = 0.0;
    const bool diag = rec.I == rec.J;
    for (int s = 0; s < rec.nspi; ++s) {
        const SpiRec si = pl.spi[pl.spi_order[rec.spi0 + s]];
        const bool rzero = si.n[0] == 0 && si.n[1] == 0 && si.n[2] == 0;
        for (int pp = 0; pp < si.npp; ++pp) {
            const PpiRec x = pl.ppi[si.pp0 + pp];
            // K (pi/p)^{3/2} e^{-G^2/4p}, the Gaussian factor from the chunk's table
            const double amp = x.K * __ldg(gtab + (size_t)__ldg(pl.ppi_pidx + si.pp0 + pp) * gcur + gi);
            double sn, cs;
            phase_sincos(Gx * x.P[0] + Gy * x.P[1] + Gz * x.P[2], pl.phase, sn, cs);
            const double pr = amp * cs, pim = -amp * sn;  // amp * e^{-iG.P}
            // per-axis polynomials h[ax][i][j] = sum_t E^{ij}_t (-i G)^t  (complex)
            double hr[3][(LA + 1) * (LB + 1)], hi[3][(LA + 1) * (LB + 1)];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                double E[(LA + 1) * (LB + 1) * NT];
                herm_E<LA, LB, double>(x.PA[k], x.PB[k], 0.5 / x.p, E);
                const double g = Gv[k];
                // (-iG)^t: 1, -iG, -G^2, iG^3, G^4
                const double pw_r[5] = {1.0, 0.0, -g * g, 0.0, g * g * g * g};
                const double pw_i[5] = {0.0, -g, 0.0, g * g * g, 0.0};
#pragma unroll
                for (int i = 0; i <= LA; ++i)
#pragma unroll
                    for (int j = 0; j <= LB; ++j) {
                        double ar = 0, ai = 0;
#pragma unroll
                        for (int t = 0; t <= i + j; ++t) {
                            ar += E[(i * (LB + 1) + j) * NT + t] * pw_r[t];
                            ai += E[(i * (LB + 1) + j) * NT + t] * pw_i[t];
                        }
                        hr[k][i * (LB + 1) + j] = ar;
                        hi[k][i * (LB + 1) + j] = ai;
                    }
            }
#pragma unroll
            for (int a = 0; a < NA; ++a)
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    const int ix = cexp(LA, a, 0) * (LB + 1) + cexp(LB, b, 0);
                    const int iy = cexp(LA, a, 1) * (LB + 1) + cexp(LB, b, 1);
                    const int iz = cexp(LA, a, 2) * (LB + 1) + cexp(LB, b, 2);
                    double tr = hr[0][ix] * hr[1][iy] - hi[0][ix] * hi[1][iy];
                    double ti = hr[0][ix] * hi[1][iy] + hi[0][ix] * hr[1][iy];
                    const double ur = tr * hr[2][iz] - ti * hi[2][iz];
                    const double ui = tr * hi[2][iz] + ti * hr[2][iz];
                    const double vr = ur * pr - ui * pim, vi = ur * pim + ui * pr;
                    re[a * NB + b] += vr;
                    im[a * NB + b] += vi;
                    if (diag && !rzero) {  // the image (I, I, -R) is the transposed block
                        re[b * NB + a] += vr;
                        im[b * NB + a] += vi;
                    }
                }
        }
    }
    const int n = pl.nbf;
    const int aoI = pl.shells[rec.I].ao, aoJ = pl.shells[rec.J].ao;
    double *Mr = M + (size_t)(2 * gi) * n * n;
    double *Mi = Mr + (size_t)n * n;
#pragma unroll
    for (int a = 0; a < NA; ++a)
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const size_t o = (size_t)(aoI + a) * n + aoJ + b;
            Mr[o] = sw * re[a * NB + b];
            Mi[o] = sw * im[a * NB + b];
            if (!diag) {
                const size_t ot = (size_t)(aoJ + b) * n + aoI + a;
                Mr[ot] = sw * re[a * NB + b];
                Mi[ot] = sw * im[a * NB + b];
            }
        }
}


// E^{ij}_t for one axis in double-float (the recursion of herm_E with
// E^{00}_0 = 1 folded in at compile time); entries with t > i + j are never
// read.
template <int LA, int LB>
__host__ __device__ __forceinline__ void herm_E_df(dfl PA, dfl PB, dfl oo2p, dfl *E)
{
    constexpr int NT = LA + LB + 1;
#pragma unroll
    for (int i = 0; i <= LA; ++i)
#pragma unroll
        for (int j = 0; j <= LB; ++j) {
            if (i == 0 && j == 0) continue;
            const int b = i > 0 ? ((i - 1) * (LB + 1) + j) * NT : (i * (LB + 1) + j - 1) * NT;
            const int top = i + j - 1;  // highest t of the level below
            const dfl X = i > 0 ? PA : PB;
#pragma unroll
            for (int t = 0; t <= i + j; ++t) {
                dfl v{0.0f, 0.0f};
                bool any = false;
                if (t <= top) {
                    v = (b + t == 0) ? X : df_mul(X, E[b + t]);
                    any = true;
                }
                if (t > 0) {
                    const dfl u = (b + t - 1 == 0) ? oo2p : df_mul(oo2p, E[b + t - 1]);
                    v = any ? df_add(v, u) : u;
                    any = true;
                }
                if (t + 1 <= top) v = df_add(v, df_mulf(E[b + t + 1], (float)(t + 1)));
                E[(i * (LB + 1) + j) * NT + t] = v;
            }
        }
}

__host__ __device__ __forceinline__ void df_cmul(dfl &xr, dfl &xi, dfl yr, dfl yi)
{
    const dfl r = df_sub(df_mul(xr, yr), df_mul(xi, yi));
    const dfl i = df_add(df_mul(xr, yi), df_mul(xi, yr));
    xr = r;
    xi = i;
}

// One primitive pair's contribution to the Cartesian block of a structure
// factor, in double-float: with the phase and Gaussian factor (pr, pim)
// already formed, multiply by the per-axis Hermite polynomials
// h_k = sum_t E^{ij}_t (-iG_k)^t (Gp[k][t] = G_k^t) and accumulate into
// re/im; twice adds the transposed block as well (the image (I, I, -R)).
template <int LA, int LB>
__host__ __device__ __forceinline__ void sfac_df_poly(const dfl PA[3], const dfl PB[3], dfl oo2p, const dfl (*Gp)[LA + LB + 1], dfl pr,
                                                      dfl pim, bool twice, dfl *re, dfl *im)
{
    constexpr int NA = ncart(LA), NB = ncart(LB), NT = LA + LB + 1;
    dfl hr[3][(LA + 1) * (LB + 1)], hi[3][(LA + 1) * (LB + 1)];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        dfl E[(LA + 1) * (LB + 1) * NT];
        herm_E_df<LA, LB>(PA[k], PB[k], oo2p, E);
#pragma unroll
        for (int i = 0; i <= LA; ++i)
#pragma unroll
            for (int j = 0; j <= LB; ++j) {
                if (i == 0 && j == 0) continue;
                const int e0 = (i * (LB + 1) + j) * NT;
                // (-iG)^t: 1, -iG, -G^2, iG^3, G^4
                dfl ar = E[e0], ai{0.0f, 0.0f};
#pragma unroll
                for (int t = 1; t <= i + j; ++t) {
                    const dfl term = df_mul(E[e0 + t], Gp[k][t]);
                    if (t == 1) ai = df_neg(term);
                    else if (t == 2) ar = df_sub(ar, term);
                    else if (t == 3) ai = df_add(ai, term);
                    else ar = df_add(ar, term);
                }
                hr[k][i * (LB + 1) + j] = ar;
                hi[k][i * (LB + 1) + j] = ai;
            }
    }
#pragma unroll
    for (int a = 0; a < NA; ++a)
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            dfl vr = pr, vi = pim;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int ia = cexp(LA, a, k), jb = cexp(LB, b, k);
                if (ia == 0 && jb == 0) continue;
                df_cmul(vr, vi, hr[k][ia * (LB + 1) + jb], hi[k][ia * (LB + 1) + jb]);
            }
            re[a * NB + b] = df_add(re[a * NB + b], vr);
            im[a * NB + b] = df_add(im[a * NB + b], vi);
            if (twice) {
                re[b * NB + a] = df_add(re[b * NB + a], vr);
                im[b * NB + a] = df_add(im[b * NB + a], vi);
            }
        }
}

// Structure factors of one class of unique shell pairs for a chunk of G, as
// k_sfac, in double-float arithmetic on the FP32 pipe (mixed precision): the
// phase from the integer coordinates of G and the split fractional
// coordinates of P (df_turns, exact reduction mod 2 pi), sin and cos by table
// and Taylor series, the Gaussian factor from the chunk's double-float table,
// the Hermite polynomials and the Cartesian products in double-float.
// Relative accuracy about 1e-14 per term; the result is rounded to FP64.
// gtab already carries the weight sqrt(8 pi w(G) / V).
template <int LA, int LB>
__global__ void __launch_bounds__(128) k_sfac_df(PlanDev pl, int sp0, int sp1, int g0, int gcur, const float2 *__restrict__ gtab,
                                                 double *__restrict__ M)
{
    constexpr int NA = ncart(LA), NB = ncart(LB), L = LA + LB;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int gi = (int)(idx % gcur);
    const int sp = sp0 + (int)(idx / gcur);
    if (sp >= sp1) return;
    const SpairRec rec = pl.spair[sp];
    const float4 gn = __ldg(pl.gdf + 3 * (size_t)(g0 + gi));
    dfl Gp[3][L + 1];  // powers of G_k, [k][t] = G_k^t, t >= 1
    if constexpr (L > 0) {
        const float4 g1 = __ldg(pl.gdf + 3 * (size_t)(g0 + gi) + 1), g2 = __ldg(pl.gdf + 3 * (size_t)(g0 + gi) + 2);
        const dfl Gk[3] = {{g1.x, g1.y}, {g1.z, g1.w}, {g2.x, g2.y}};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            Gp[k][0] = dfl{1.0f, 0.0f};
            Gp[k][1] = Gk[k];
#pragma unroll
            for (int t = 2; t <= L; ++t) Gp[k][t] = df_mul(Gp[k][t - 1], Gk[k]);
        }
    }
    dfl re[NA * NB], im[NA * NB];
#pragma unroll
    for (int k = 0; k < NA * NB; ++k) re[k] = im[k] = dfl{0.0f, 0.0f};
    const bool diag = rec.I == rec.J;
    for (int s = 0; s < rec.nspi; ++s) {
        const SpiRec si = pl.spi[pl.spi_order[rec.spi0 + s]];
        const bool rzero = si.n[0] == 0 && si.n[1] == 0 && si.n[2] == 0;
        const bool twice = diag && !rzero;  // the image (I, I, -R) is the transposed block
        for (int pp = 0; pp < si.npp; ++pp) {
            const PpiDF *q = pl.ppdf + si.pp0 + pp;
            const float4 qa = __ldg(&q->a), qb = __ldg(&q->b), qc = __ldg(&q->c);
            const float f1[3] = {qa.x, qa.y, qa.z}, f2[3] = {qb.x, qb.y, qb.z}, f3[3] = {qc.x, qc.y, qc.z};
            dfl w, cs, sn;
            const int j = df_turns(gn.x, gn.y, gn.z, f1, f2, f3, w);
            df_sincos_turns(w, __ldg(pl.phasef + (j & 1023)), cs, sn);
            // K (pi/p)^{3/2} e^{-G^2/4p} sqrt(8 pi w(G) / V) e^{-iG.P}
            const float2 gt = __ldg(gtab + (size_t)__float_as_int(qc.w) * gcur + gi);
            const dfl amp = df_mul(dfl{qa.w, qb.w}, dfl{gt.x, gt.y});
            const dfl pr = df_mul(amp, cs), pim = df_neg(df_mul(amp, sn));
            if constexpr (L == 0) {
                const float f = twice ? 2.0f : 1.0f;  // s-s: the transposed block is the same element
                re[0] = df_add(re[0], dfl{f * pr.hi, f * pr.lo});
                im[0] = df_add(im[0], dfl{f * pim.hi, f * pim.lo});
            } else {
                const float4 qd = __ldg(&q->d), qe = __ldg(&q->e), qf = __ldg(&q->f), qg = __ldg(&q->g);
                const dfl PA[3] = {{qd.x, qd.y}, {qd.z, qd.w}, {qe.x, qe.y}};
                const dfl PB[3] = {{qe.z, qe.w}, {qf.x, qf.y}, {qf.z, qf.w}};
                sfac_df_poly<LA, LB>(PA, PB, dfl{qg.x, qg.y}, Gp, pr, pim, twice, re, im);
            }
        }
    }
    const int n = pl.nbf;
    const int aoI = pl.shells[rec.I].ao, aoJ = pl.shells[rec.J].ao;
    double *Mr = M + (size_t)(2 * gi) * n * n;
    double *Mi = Mr + (size_t)n * n;
#pragma unroll
    for (int a = 0; a < NA; ++a)
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            // hi + lo in FP64, the conversions by integer operations (one FP64 add each)
            const double vr = to_f64(re[a * NB + b].hi) + to_f64(re[a * NB + b].lo);
            const double vi = to_f64(im[a * NB + b].hi) + to_f64(im[a * NB + b].lo);
            const size_t o = (size_t)(aoI + a) * n + aoJ + b;
            Mr[o] = vr;
            Mi[o] = vi;
            if (!diag) {
                const size_t ot = (size_t)(aoJ + b) * n + aoI + a;
                Mr[ot] = vr;
                Mi[ot] = vi;
            }
        }
}

}  // namespace jk
