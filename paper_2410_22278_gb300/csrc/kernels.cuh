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

#include "jk_internal.h"
#include "md.cuh"

namespace jk {

constexpr double kPi = 3.14159265358979323846;
constexpr double kTwoPi52 = 34.986836655249725;  // 2 pi^{5/2}
constexpr int kRealThreads = 128;

template <typename T>
struct Prec;
template <>
struct Prec<double> {
    __device__ static const double *tab(const PlanDev &pl) { return pl.boys; }
};
template <>
struct Prec<float> {
    __device__ static const float *tab(const PlanDev &pl) { return pl.boys_f; }
};

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Attenuated seeds s_m = (-2 alpha)^m F_m(alpha X^2) - c_w (-2 alpha_w)^m F_m(alpha_w X^2).
template <int L>
__device__ __forceinline__ void seeds(double x2, double alpha, double aw, double cw, const PlanDev &pl, double *s)
{
    double F1[L + 1], F2[L + 1];
    boys<L>(alpha * x2, pl.boys, F1);
    boys<L>(aw * x2, pl.boys, F2);
    double f1 = 1.0, f2 = cw;
#pragma unroll
    for (int m = 0; m <= L; ++m) {
        s[m] = f1 * F1[m] - f2 * F2[m];
        f1 *= -2.0 * alpha;
        f2 *= -2.0 * aw;
    }
}
// Single precision unless the two terms nearly cancel (c_w close to 1),
// where the seed is formed in double and rounded once.
template <int L>
__device__ __forceinline__ void seeds(double x2, double alpha, double aw, double cw, const PlanDev &pl, float *s)
{
    if (cw > 0.85) {
        double sd[L + 1];
        seeds<L>(x2, alpha, aw, cw, pl, sd);
#pragma unroll
        for (int m = 0; m <= L; ++m) s[m] = (float)sd[m];
        return;
    }
    float F1[L + 1], F2[L + 1];
    boys<L>((float)(alpha * x2), pl.boys_f, F1);
    boys<L>((float)(aw * x2), pl.boys_f, F2);
    float f1 = 1.0f, f2 = (float)cw;
    const float ma = (float)(-2.0 * alpha), mw = (float)(-2.0 * aw);
#pragma unroll
    for (int m = 0; m <= L; ++m) {
        s[m] = f1 * F1[m] - f2 * F2[m];
        f1 *= ma;
        f2 *= mw;
    }
}

// Contracted real-space block V[((a*NB+b)*NC+c)*ND+d] of one pair of shell-pair images.
template <int LA, int LB, int LC, int LD, typename T>
__device__ __forceinline__ void quartet_block(const PlanDev &pl, const SpiRec &sb, const SpiRec &sk, T *V)
{
    constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
    constexpr int L = LA + LB + LC + LD, LAB = LA + LB, LCD = LC + LD;
    constexpr int NTA = LAB + 1, NTC = LCD + 1, D = L + 1;
    for (int i = 0; i < sb.npp; ++i) {
        const PpiRec x = pl.ppi[sb.pp0 + i];
        T Ea[3][(LA + 1) * (LB + 1) * NTA];
        const T oo2p = T(0.5 / x.p);
#pragma unroll
        for (int k = 0; k < 3; ++k) herm_E<LA, LB, T>(T(x.PA[k]), T(x.PB[k]), oo2p, Ea[k]);
        for (int j = 0; j < sk.npp; ++j) {
            const PpiRec y = pl.ppi[sk.pp0 + j];
            const double p = x.p, q = y.p;
            const double alpha = p * q / (p + q);
            const double aw = 1.0 / (1.0 / p + 1.0 / q + pl.inv_omega2);
            const double cw = sqrt(aw / alpha);
            const double pref = kTwoPi52 / (p * q * sqrt(p + q)) * x.K * y.K;
            // Eq. pbc_eri_real_cutoff_implementation with the Hermite growth margin
            const double lg = log(fabs(pref) * (1.0 - cw) / pl.ewald_R);
            if (lg <= 0.0) continue;
            double r = sqrt(lg / aw);
            r = sqrt((lg + L * log1p(2.0 * aw * r)) / aw);
            r = sqrt((lg + L * log1p(2.0 * aw * r)) / aw);
            const double r2 = r * r;
            // minimum image of P - Q (Eq. lattice_image_min_norm)
            double X0[3] = {x.P[0] - y.P[0], x.P[1] - y.P[1], x.P[2] - y.P[2]};
            {
                double f[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) f[a] = rint(pl.Finv[3 * a] * X0[0] + pl.Finv[3 * a + 1] * X0[1] + pl.Finv[3 * a + 2] * X0[2]);
#pragma unroll
                for (int a = 0; a < 3; ++a) X0[a] -= f[0] * pl.L[a] + f[1] * pl.L[3 + a] + f[2] * pl.L[6 + a];
            }
            const double x0n = sqrt(X0[0] * X0[0] + X0[1] * X0[1] + X0[2] * X0[2]);
            T Rs[D * D * D];
#pragma unroll
            for (int k = 0; k < D * D * D; ++k) Rs[k] = T(0);
            bool any = false;
            for (int c = 0; c < pl.nr1; ++c) {
                const double4 rc = reinterpret_cast<const double4 *>(pl.r1)[c];
                if (rc.w - x0n >= r) break;
                const double Xx = X0[0] - rc.x, Xy = X0[1] - rc.y, Xz = X0[2] - rc.z;
                const double x2 = Xx * Xx + Xy * Xy + Xz * Xz;
                if (x2 >= r2) continue;
                any = true;
                T s[L + 1];
                seeds<L>(x2, alpha, aw, cw, pl, s);
                T B[D * D * D];
                herm_R<L, T>(s, T(Xx), T(Xy), T(Xz), B);
#pragma unroll
                for (int t = 0; t <= L; ++t)
#pragma unroll
                    for (int u = 0; u <= L - t; ++u)
#pragma unroll
                        for (int v = 0; v <= L - t - u; ++v) Rs[(t * D + u) * D + v] += B[(t * D + u) * D + v];
            }
            if (!any) continue;
            T Ec[3][(LC + 1) * (LD + 1) * NTC];
            const T oo2q = T(0.5 / q);
#pragma unroll
            for (int k = 0; k < 3; ++k) herm_E<LC, LD, T>(T(y.PA[k]), T(y.PB[k]), oo2q, Ec[k]);
            const T tp = T(pref);
#pragma unroll
            for (int c = 0; c < NC; ++c)
#pragma unroll
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
#pragma unroll
                    for (int a = 0; a < NA; ++a)
#pragma unroll
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

// mode: 0 every quartet; 1 only quartets whose density-weighted Schwarz
// estimate is >= tau; 2 only those below tau.
template <int LA, int LB, int LC, int LD, typename T>
__global__ void __launch_bounds__(kRealThreads) k_real(PlanDev pl, int b0, int b1, int k0, int k1, int same, int kchunk, int mode,
                                                        double tau, const double *__restrict__ Dp, const double *__restrict__ dmax,
                                                        double *__restrict__ X, double *__restrict__ Y)
{
    constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
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
    double Dij[NA * NB], jb[NA * NB];
#pragma unroll
    for (int a = 0; a < NA; ++a)
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            Dij[a * NB + b] = __ldg(Dp + (size_t)(aoI + a) * n + aoJ + b);
            jb[a * NB + b] = 0.0;
        }
    const double dIJ = mode ? dmax[sb.I * nsh + sb.J] : 0.0;
    for (int kt = kbeg; kt < kend; ++kt) {
        const SpiRec sk = pl.spi[kt];
        bool valid = act && (!same || kt >= bra);
        if (valid && mode) {
            double dm = fmax(fmax(dIJ, dmax[sk.I * nsh + sk.J]), fmax(dmax[sb.J * nsh + sk.I], dmax[sb.I * nsh + sk.I]));
            dm = fmax(dm, fmax(dmax[sb.J * nsh + sk.J], dmax[sb.I * nsh + sk.J]));
            const double bound = sb.Q * sk.Q * dm;
            valid = (mode == 1) ? (bound >= tau) : (bound < tau);
        }
        T V[NA * NB * NC * ND];
#pragma unroll
        for (int k = 0; k < NA * NB * NC * ND; ++k) V[k] = T(0);
        if (valid) quartet_block<LA, LB, LC, LD, T>(pl, sb, sk, V);
        const double w = valid ? double(sb.w) * double(sk.w) * ((same && kt == bra) ? 0.5 : 1.0) : 0.0;
        const int aoK = pl.shells[sk.I].ao, aoL = pl.shells[sk.J].ao;
        // Coulomb, bra side: X_ij += 2w sum_kl V D_kl (held in registers over the ket loop)
        double Dkl[NC * ND];
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int d = 0; d < ND; ++d) Dkl[c * ND + d] = __ldg(Dp + (size_t)(aoK + c) * n + aoL + d);
#pragma unroll
        for (int ab = 0; ab < NA * NB; ++ab) {
            double s = 0.0;
#pragma unroll
            for (int cd = 0; cd < NC * ND; ++cd) s += double(V[ab * NC * ND + cd]) * Dkl[cd];
            jb[ab] += 2.0 * w * s;
        }
        // Coulomb, ket side: X_kl += 2w sum_ij V D_ij, summed over the warp's bras
#pragma unroll
        for (int cd = 0; cd < NC * ND; ++cd) {
            double s = 0.0;
#pragma unroll
            for (int ab = 0; ab < NA * NB; ++ab) s += double(V[ab * NC * ND + cd]) * Dij[ab];
            s = warp_sum(2.0 * w * s);
            if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(X + (size_t)(aoK + cd / ND) * n + aoL + cd % ND, s);
        }
        // exchange: the four index assignments of the orbit (the other four are transposes)
        if (valid) {
#pragma unroll
            for (int a = 0; a < NA; ++a)
#pragma unroll
                for (int d = 0; d < ND; ++d) {  // K_il += w V_ijkl D_jk
                    double s = 0.0;
#pragma unroll
                    for (int b = 0; b < NB; ++b)
#pragma unroll
                        for (int c = 0; c < NC; ++c) s += double(V[((a * NB + b) * NC + c) * ND + d]) * __ldg(Dp + (size_t)(aoJ + b) * n + aoK + c);
                    atomicAdd(Y + (size_t)(aoI + a) * n + aoL + d, w * s);
                }
#pragma unroll
            for (int b = 0; b < NB; ++b)
#pragma unroll
                for (int d = 0; d < ND; ++d) {  // K_jl += w V_ijkl D_ik
                    double s = 0.0;
#pragma unroll
                    for (int a = 0; a < NA; ++a)
#pragma unroll
                        for (int c = 0; c < NC; ++c) s += double(V[((a * NB + b) * NC + c) * ND + d]) * __ldg(Dp + (size_t)(aoI + a) * n + aoK + c);
                    atomicAdd(Y + (size_t)(aoJ + b) * n + aoL + d, w * s);
                }
#pragma unroll
            for (int a = 0; a < NA; ++a)
#pragma unroll
                for (int c = 0; c < NC; ++c) {  // K_ik += w V_ijkl D_jl
                    double s = 0.0;
#pragma unroll
                    for (int b = 0; b < NB; ++b)
#pragma unroll
                        for (int d = 0; d < ND; ++d) s += double(V[((a * NB + b) * NC + c) * ND + d]) * __ldg(Dp + (size_t)(aoJ + b) * n + aoL + d);
                    atomicAdd(Y + (size_t)(aoI + a) * n + aoK + c, w * s);
                }
#pragma unroll
            for (int b = 0; b < NB; ++b)
#pragma unroll
                for (int c = 0; c < NC; ++c) {  // K_jk += w V_ijkl D_il
                    double s = 0.0;
#pragma unroll
                    for (int a = 0; a < NA; ++a)
#pragma unroll
                        for (int d = 0; d < ND; ++d) s += double(V[((a * NB + b) * NC + c) * ND + d]) * __ldg(Dp + (size_t)(aoI + a) * n + aoL + d);
                    atomicAdd(Y + (size_t)(aoJ + b) * n + aoK + c, w * s);
                }
        }
    }
    if (act) {
#pragma unroll
        for (int a = 0; a < NA; ++a)
#pragma unroll
            for (int b = 0; b < NB; ++b)
                if (jb[a * NB + b] != 0.0) atomicAdd(X + (size_t)(aoI + a) * n + aoJ + b, jb[a * NB + b]);
    }
}

// Structure factors of one class of unique shell pairs for a chunk of G.
// Thread (shell pair, g) with g fastest.  M layout: [2*gcur][n][n], part 0
// real, part 1 imaginary, both scaled by sqrt(8 pi w(G)/V) (gv[4g+3]).
template <int LA, int LB>
__global__ void __launch_bounds__(128) k_sfac(PlanDev pl, int sp0, int sp1, const double *__restrict__ gv, int g0, int gcur,
                                              double *__restrict__ M)
{
    constexpr int NA = ncart(LA), NB = ncart(LB), NT = LA + LB + 1;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int gi = (int)(idx % gcur);
    const int sp = sp0 + (int)(idx / gcur);
    if (sp >= sp1) return;
    const SpairRec rec = pl.spair[sp];
    const double Gx = gv[4 * (g0 + gi)], Gy = gv[4 * (g0 + gi) + 1], Gz = gv[4 * (g0 + gi) + 2], sw = gv[4 * (g0 + gi) + 3];
    const double G2 = Gx * Gx + Gy * Gy + Gz * Gz;
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
            const double amp = x.K * (kPi / x.p) * sqrt(kPi / x.p) * exp(-G2 / (4.0 * x.p));
            double sn, cs;
            sincos(Gx * x.P[0] + Gy * x.P[1] + Gz * x.P[2], &sn, &cs);
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

}  // namespace jk
