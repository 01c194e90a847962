// Coulomb-only real-space path in the Hermite basis (the J-engine of Section
// 3.2 and Eqs. pbc_j_split_1 .. pbc_j_split_4), used by builds that ask for J
// alone (K == NULL).
//
//   1. Hermite ket density of every local primitive pair p of an image
//      (I, J, R):  Dh_p[s] = sum_{a in I, b in J} E^{ab}_s D'_ab  (N_H(l_I+l_J)
//      values, Eq. pbc_j_split_1);
//   2. per primitive quartet (bra pair i, ket pair j) and lattice image R1:
//      the bra side J_ab += 2w pref sum_t E^{ab,i}_t sum_s (-1)^{|s|}
//      R_{t+s} Dh_j[s] (Cartesian, in registers, over the ket loop), and the
//      ket side JH_j[s] += 2w pref (-1)^{|s|} sum_t R_{t+s} Dh_i[t] (Hermite,
//      summed over the bra primitives and the warp's 32 bras, one atomic
//      per element into the per-primitive-pair accumulator JH);
//   3. back to Cartesian: X_cd += sum_s E^{cd,j}_s JH_j[s] for every local
//      primitive pair (Eq. pbc_j_split_3).
// No Cartesian ERI block is formed: for a (dd|dd) quartet the contraction
// is N_H(4)^2 = 35 x 35 Hermite products instead of the 1296-element block.
#pragma once
#include "kernels.cuh"

namespace jk {

// position of the Hermite index (tx, ty, tz) inside the simplex of total
// order <= L: levels n = tx + ty + tz in turn, tx then ty descending
__host__ __device__ constexpr int hpos(int tx, int ty, int tz)
{
    const int n = tx + ty + tz;
    return (n > 0 ? nherm(n - 1) : 0) + (n - tx) * (n - tx + 1) / 2 + (n - tx - ty);
}

// Hermite density of one primitive pair from its E tables and the D' block
template <int LA, int LB, typename T>
__device__ __forceinline__ void hermite_density(const T (*E)[(LA + 1) * (LB + 1) * (LA + LB + 1)], const T *Dab, T *Dh)
{
    constexpr int NA = ncart(LA), NB = ncart(LB), L = LA + LB, NT = L + 1;
#pragma unroll
    for (int q = 0; q < nherm(L); ++q) Dh[q] = T(0);
#pragma unroll
    for (int a = 0; a < NA; ++a)
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int ax = cexp(LA, a, 0), ay = cexp(LA, a, 1), az = cexp(LA, a, 2);
            const int bx = cexp(LB, b, 0), by = cexp(LB, b, 1), bz = cexp(LB, b, 2);
            const T d = Dab[a * NB + b];
#pragma unroll
            for (int tx = 0; tx <= ax + bx; ++tx)
#pragma unroll
                for (int ty = 0; ty <= ay + by; ++ty)
#pragma unroll
                    for (int tz = 0; tz <= az + bz; ++tz)
                        Dh[hpos(tx, ty, tz)] += d * E[0][(ax * (LB + 1) + bx) * NT + tx] * E[1][(ay * (LB + 1) + by) * NT + ty] *
                                                E[2][(az * (LB + 1) + bz) * NT + tz];
        }
}

// Hermite densities of the local primitive pairs of the images [b0, b1) of
// one class (l_I, l_J) = (LA, LB): one thread per image.  Dh has a stride of
// hs values per primitive pair; written in FP64 and, if Dhf is given, FP32.
template <int LA, int LB>
__global__ void k_hermite_density(PlanDev pl, int b0, int b1, const double *__restrict__ Dp, int hs, double *__restrict__ Dh,
                                  float *__restrict__ Dhf)
{
    constexpr int NA = ncart(LA), NB = ncart(LB), NH = nherm(LA + LB);
    const int im = b0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (im >= b1) return;
    const SpiRec s = pl.spi[im];
    const int n = pl.nbf, aoI = pl.shells[s.I].ao, aoJ = pl.shells[s.J].ao;
    double Dab[NA * NB];
#pragma unroll
    for (int a = 0; a < NA; ++a)
#pragma unroll
        for (int b = 0; b < NB; ++b) Dab[a * NB + b] = Dp[(size_t)(aoI + a) * n + aoJ + b];
    for (int p = s.pp0; p < s.pp0 + s.npp; ++p) {
        const PpiRec x = pl.ppi[p];
        double E[3][(LA + 1) * (LB + 1) * (LA + LB + 1)];
#pragma unroll
        for (int k = 0; k < 3; ++k) herm_E<LA, LB, double>(x.PA[k], x.PB[k], 0.5 * x.pad, E[k]);
        double h[NH];
        hermite_density<LA, LB, double>(E, Dab, h);
#pragma unroll
        for (int q = 0; q < NH; ++q) {
            Dh[(size_t)p * hs + q] = h[q];
            if (Dhf) Dhf[(size_t)p * hs + q] = (float)h[q];
        }
    }
}

// X_cd += sum_s E^{cd}_s JH_p[s] over the local primitive pairs of the
// images [b0, b1) of one class: one thread per image, one atomic per element.
template <int LA, int LB>
__global__ void k_hermite_back(PlanDev pl, int b0, int b1, int hs, const double *__restrict__ JH, double *__restrict__ X)
{
    constexpr int NA = ncart(LA), NB = ncart(LB), L = LA + LB, NT = L + 1;
    const int im = b0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (im >= b1) return;
    const SpiRec s = pl.spi[im];
    const int n = pl.nbf, aoI = pl.shells[s.I].ao, aoJ = pl.shells[s.J].ao;
    double out[NA * NB];
#pragma unroll
    for (int q = 0; q < NA * NB; ++q) out[q] = 0.0;
    for (int p = s.pp0; p < s.pp0 + s.npp; ++p) {
        const PpiRec x = pl.ppi[p];
        double E[3][(LA + 1) * (LB + 1) * (LA + LB + 1)];
#pragma unroll
        for (int k = 0; k < 3; ++k) herm_E<LA, LB, double>(x.PA[k], x.PB[k], 0.5 * x.pad, E[k]);
        const double *h = JH + (size_t)p * hs;
#pragma unroll
        for (int a = 0; a < NA; ++a)
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const int ax = cexp(LA, a, 0), ay = cexp(LA, a, 1), az = cexp(LA, a, 2);
                const int bx = cexp(LB, b, 0), by = cexp(LB, b, 1), bz = cexp(LB, b, 2);
                double v = 0.0;
#pragma unroll
                for (int tx = 0; tx <= ax + bx; ++tx)
#pragma unroll
                    for (int ty = 0; ty <= ay + by; ++ty)
#pragma unroll
                        for (int tz = 0; tz <= az + bz; ++tz)
                            v += E[0][(ax * (LB + 1) + bx) * NT + tx] * E[1][(ay * (LB + 1) + by) * NT + ty] *
                                 E[2][(az * (LB + 1) + bz) * NT + tz] * h[hpos(tx, ty, tz)];
                out[a * NB + b] += v;
            }
    }
#pragma unroll
    for (int a = 0; a < NA; ++a)
#pragma unroll
        for (int b = 0; b < NB; ++b)
            if (out[a * NB + b] != 0.0) atomicAdd(X + (size_t)(aoI + a) * n + aoJ + b, out[a * NB + b]);
}

// J-engine tile kernel of one class pair: lanes hold 32 bra images, the
// warp walks the kets of its chunk (quartet-level bounds and the mixed
// policy as in k_real, large quartets to the FP64 list); for every ket
// primitive pair the warp loops its bra primitives, evaluates the lattice
// images of each primitive quartet into the R table, adds the bra side to
// the lane's Cartesian J accumulator and the ket side to a Hermite
// accumulator that is summed over the warp and added to JH once per ket
// primitive pair.  Dh: Hermite densities (stride hs) in the kernel's
// precision.
template <int LA, int LB, int LC, int LD, typename T>
__global__ void __launch_bounds__(kRealThreads) k_jeng(PlanDev pl, int b0, int b1, int k0, int k1, int same, int kchunk, int mode,
                                                        double tau, const T *__restrict__ dmax, const T *__restrict__ Dh, int hs,
                                                        double *__restrict__ X, double *__restrict__ JH, unsigned long long *__restrict__ cnt,
                                                        int2 *__restrict__ big, unsigned *__restrict__ nbig, unsigned cap,
                                                        unsigned *__restrict__ ovf)
{
    constexpr int NA = ncart(LA), NB = ncart(LB);
    constexpr int L = LA + LB + LC + LD, LAB = LA + LB, LCD = LC + LD, D = L + 1, NTA = LAB + 1;
    constexpr int NHA = nherm(LAB), NHC = nherm(LCD);
    const int tile0 = b0 + blockIdx.x * kRealThreads;
    const int bra = tile0 + threadIdx.x;
    int kbeg = k0 + blockIdx.y * kchunk;
    const int kend = min(k1, kbeg + kchunk);
    if (same) kbeg = max(kbeg, tile0);
    if (kbeg >= kend) return;
    const bool act = bra < b1;
    const SpiRec sb = pl.spi[act ? bra : b0];
    const int n = pl.nbf, nsh = pl.nshell;
    Acc<T> jb[NA * NB];
    const float tauf = (float)tau;
    unsigned nq = 0;
    Tally tl;
    for (int kt = kbeg; kt < kend; ++kt) {
        if (kt == kbeg || (kt & 31) == 0) {
            if (!__any_sync(0xffffffffu, act && block_reaches<L>(pl, sb, kt >> 5))) {
                kt = min(kend, ((kt >> 5) + 1) << 5) - 1;
                continue;
            }
        }
        const SpiRec sk = pl.spi[kt];
        bool valid = act && (!same || kt >= bra);
        valid = valid && quartet_reaches<L>(pl, sb, sk);
        if (!__any_sync(0xffffffffu, valid)) continue;
        if (sizeof(T) == 4 && valid && mode) {
            const float dm = quartet_dmax(reinterpret_cast<const float *>(dmax), nsh, sb, sk);
            const float est = quartet_estimate_bound(pl, sb, sk) * dm >= tauf ? quartet_estimate(pl, sb, sk) * dm : 0.0f;
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
        nq += valid;
        tl.quart += valid;
        const T w2 = valid ? T(2) * T(sb.w) * T(sk.w) * ((same && kt == bra) ? T(0.5) : T(1)) : T(0);
        // ket primitive pairs in turn (the same for every lane of the warp)
        for (int j = 0; j < sk.npp; ++j) {
            const int kp = sk.pp0 + j;
            const PpiF yf = pl.ppf[kp];
            PairT<T> y;
            load_pair(pl, kp, yf, y);
            T Dk[NHC], Jk[NHC];
#pragma unroll
            for (int q = 0; q < NHC; ++q) {
                Dk[q] = __ldg(Dh + (size_t)kp * hs + q);
                Jk[q] = T(0);
            }
            const float Bk = __ldg(pl.ppB + kp);
            if (valid)
                for (int i = 0; i < sb.npp; ++i) {
                    if (__ldg(pl.ppB + sb.pp0 + i) * Bk < pl.mag_thr) break;
                    const int bp = sb.pp0 + i;
                    const PpiF xf = pl.ppf[bp];
                    // screening radius (single precision), as in quartet_block
                    const float ipf = xf.pad, iqf = yf.pad;
                    const float awf = frcp_fast(ipf + iqf + pl.inv_omega2f);
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
                        r += 0.5f + 0.25f * L;
                    }
                    const float r2 = r * r;
                    PairT<T> x;
                    load_pair(pl, bp, xf, x);
                    T X0[3] = {x.P[0] - y.P[0], x.P[1] - y.P[1], x.P[2] - y.P[2]};
                    {
                        T f[3];
#pragma unroll
                        for (int a = 0; a < 3; ++a)
                            f[a] = rint(latc(pl.Finv, pl.Finvf, 3 * a, T(0)) * X0[0] + latc(pl.Finv, pl.Finvf, 3 * a + 1, T(0)) * X0[1] +
                                        latc(pl.Finv, pl.Finvf, 3 * a + 2, T(0)) * X0[2]);
#pragma unroll
                        for (int a = 0; a < 3; ++a)
                            X0[a] -= f[0] * latc(pl.L, pl.Lf, a, T(0)) + f[1] * latc(pl.L, pl.Lf, 3 + a, T(0)) +
                                     f[2] * latc(pl.L, pl.Lf, 6 + a, T(0));
                    }
                    const float x0n = fsqrt_fast((float)(X0[0] * X0[0] + X0[1] * X0[1] + X0[2] * X0[2]));
                    T Rs[D * D * D];
#pragma unroll
                    for (int q = 0; q < D * D * D; ++q) Rs[q] = T(0);
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
                        T sd[L + 1];
                        seeds<L>(x2, alpha, aw, cw, pl, sd);
                        T Bt[D * D * D];
                        herm_R<L, T>(sd, Xx, Xy, Xz, Bt);
#pragma unroll
                        for (int t = 0; t <= L; ++t)
#pragma unroll
                            for (int u = 0; u <= L - t; ++u)
#pragma unroll
                                for (int v = 0; v <= L - t - u; ++v) Rs[(t * D + u) * D + v] += Bt[(t * D + u) * D + v];
                    }
                    if (!any) continue;
                    ++tl.term;
                    const T pref = w2 * T(kTwoPi52) * x.K * y.K * ip * iq / sqrt(x.p + y.p);
                    // bra side: h_t = sum_s (-1)^|s| R_{t+s} Dk_s, then J_ab += pref sum_t E^{ab}_t h_t
                    T h[NHA];
#pragma unroll
                    for (int tx = 0; tx <= LAB; ++tx)
#pragma unroll
                        for (int ty = 0; ty <= LAB - tx; ++ty)
#pragma unroll
                            for (int tz = 0; tz <= LAB - tx - ty; ++tz) {
                                T acc = T(0);
#pragma unroll
                                for (int sx = 0; sx <= LCD; ++sx)
#pragma unroll
                                    for (int sy = 0; sy <= LCD - sx; ++sy)
#pragma unroll
                                        for (int sz = 0; sz <= LCD - sx - sy; ++sz) {
                                            const T term = Rs[((tx + sx) * D + ty + sy) * D + tz + sz] * Dk[hpos(sx, sy, sz)];
                                            acc += ((sx + sy + sz) & 1) ? -term : term;
                                        }
                                h[hpos(tx, ty, tz)] = acc;
                            }
                    T Ea[3][(LA + 1) * (LB + 1) * NTA];
                    const T oo2p = T(0.5) * ip;
#pragma unroll
                    for (int k = 0; k < 3; ++k) herm_E<LA, LB, T>(x.PA[k], x.PB[k], oo2p, Ea[k]);
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
                                             Ea[2][(az * (LB + 1) + bz) * NTA + tz] * h[hpos(tx, ty, tz)];
                            jb[a * NB + b].add(pref * v);
                        }
                    // ket side: Jk_s += pref (-1)^|s| sum_t R_{t+s} Db_t
                    T Db[NHA];
#pragma unroll
                    for (int q = 0; q < NHA; ++q) Db[q] = __ldg(Dh + (size_t)bp * hs + q);
#pragma unroll
                    for (int sx = 0; sx <= LCD; ++sx)
#pragma unroll
                        for (int sy = 0; sy <= LCD - sx; ++sy)
#pragma unroll
                            for (int sz = 0; sz <= LCD - sx - sy; ++sz) {
                                T acc = T(0);
#pragma unroll
                                for (int tx = 0; tx <= LAB; ++tx)
#pragma unroll
                                    for (int ty = 0; ty <= LAB - tx; ++ty)
#pragma unroll
                                        for (int tz = 0; tz <= LAB - tx - ty; ++tz)
                                            acc += Rs[((tx + sx) * D + ty + sy) * D + tz + sz] * Db[hpos(tx, ty, tz)];
                                Jk[hpos(sx, sy, sz)] += ((sx + sy + sz) & 1) ? -pref * acc : pref * acc;
                            }
                }
            // the ket side of this ket primitive pair, summed over the warp's bras
#pragma unroll
            for (int q = 0; q < NHC; ++q) {
                const T v = warp_sum_t(Jk[q]);
                if ((threadIdx.x & 31) == 0 && v != T(0)) atomicAdd(JH + (size_t)kp * hs + q, to_f64(v));
            }
        }
    }
    if (act) {
        const int aoI = pl.shells[sb.I].ao, aoJ = pl.shells[sb.J].ao;
#pragma unroll
        for (int a = 0; a < NA; ++a)
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const double v = jb[a * NB + b].value();
                if (v != 0.0) atomicAdd(X + (size_t)(aoI + a) * n + aoJ + b, v);
            }
    }
    // algorithmic count of the Hermite contraction: per term 2 N_H(LAB) N_H(LCD)
    // flops on each side plus the bra back-transform, in place of the
    // Cartesian block (the tally's term cost is the Cartesian one; here the
    // images and terms are counted with the J-engine's own term cost below)
    unsigned long long fl = (unsigned long long)tl.img * (flops::per_image(L) - 8) +
                            (unsigned long long)tl.term * (8 + 4ull * NHA * NHC + 3 * flops::herm_E(LA, LB) + 2ull * NA * NB * NHA) +
                            (unsigned long long)tl.quart * 2ull * NHC,
                       fs = tally_screen<LA, LB, LC, LD>(tl);
    unsigned tot = nq;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        tot += __shfl_xor_sync(0xffffffffu, tot, o);
        fl += __shfl_xor_sync(0xffffffffu, fl, o);
        fs += __shfl_xor_sync(0xffffffffu, fs, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (tot) atomicAdd(cnt, (unsigned long long)tot);
        if (fl) atomicAdd(cnt + 4, fl);
        if (fs) atomicAdd(cnt + 8, fs);
    }
}

}  // namespace jk
