// Warp-cooperative real-space quartet kernels (erfc part of Eq.
// pbc_eri_general_final) for the classes of s and p shells.
//
// The lane-per-bra tile kernel of kernels.cuh lets the 32 lanes of a warp
// walk one ket with 32 different bras; lanes whose bra cannot reach the ket,
// or whose primitive quartet is screened out, idle while the others work.
// Here one warp owns one bra image and a range of kets:
//   1. the 32 lanes test 32 kets at once (block bound, quartet-level bound,
//      precision policy) and the kets that pass are compacted with a ballot;
//   2. the primitive pairs of those kets are laid out one per lane (the
//      local primitive pairs of consecutive images are contiguous), so every
//      lane evaluates the bra primitives against its own ket primitive;
//   3. the partial Cartesian blocks of lanes that hold the same ket are
//      summed by a segmented warp reduction, and the first lane of each ket
//      digests the block into J and K (FP64 atomics); the bra-side Coulomb
//      term stays in registers until the end.
// Primitive pairs are stored in descending order of B = |K| p^{-5/4}: every
// primitive prefactor 2 pi^{5/2} |K_i K_j| / (pq sqrt(p+q)) is at most
// 2 pi^{5/2} 2^{-1/2} B_i B_j (p + q >= 2 sqrt(pq)), so a loop over
// primitives ends at the first pair whose B_i B_j lies below the
// per-term threshold (PlanDev::mag_thr): the magnitude test of Eq.
// pbc_eri_real_cutoff_implementation fails for it and for every later one.
// Which kernel family (this one, the lane-per-bra one of kernels.cuh or the
// pair-queue one below) runs a class pair is chosen by the autotuner.
// The FP64 pass over the large quartets of the mixed path likewise gives one
// list entry to a whole warp: its primitive quartets are screened 32 at a
// time, queued, evaluated one per lane and summed by a full warp reduction.
#pragma once
#include "kernels.cuh"

namespace jk {

// Pair data plus its Hermite coefficients in the kernel's precision.
template <int LA, int LB, typename T>
struct PrimE {
    PairT<T> x;
    T E[3][(LA + 1) * (LB + 1) * (LA + LB + 1)];
};

template <int LA, int LB, typename T>
__device__ __forceinline__ void load_prim(const PlanDev &pl, int k, PrimE<LA, LB, T> &o, PpiF &f)
{
    f = pl.ppf[k];
    load_pair(pl, k, f, o.x);
    const T oo2p = T(0.5) * o.x.ip;
#pragma unroll
    for (int a = 0; a < 3; ++a) herm_E<LA, LB, T>(o.x.PA[a], o.x.PB[a], oo2p, o.E[a]);
}

// Screening of one primitive quartet, all in single precision: true if some
// lattice image of P - Q lies inside the sphere of Eq.
// pbc_eri_real_cutoff_implementation (the same radius and image test as
// prim_term).  The minimum image decides at once when it lies inside; else
// no other image can, unless the shortest non-zero candidate vector is
// shorter than |X0| + r (|X0 - R1| >= |R1| - |X0|).
template <int L>
__device__ __forceinline__ bool prim_reaches(const PlanDev &pl, const PpiF &bf, const PpiF &kf)
{
    const float ipf = bf.pad, iqf = kf.pad;
    const float awf = frcp_fast(ipf + iqf + pl.inv_omega2f);
    const float cwf = fsqrt_fast(awf * (ipf + iqf));
    const float preff = 34.986836655249725f * bf.K * kf.K * ipf * iqf * rsqrtf(bf.p + kf.p);
    const float lg = __logf(fabsf(preff) * (1.0f - cwf)) - pl.log_ewald_R;
    if (!(lg > 0.0f)) return false;
    float r = fsqrt_fast(fdiv_fast(lg, awf));
    if (L > 0) {
        r = fsqrt_fast(fdiv_fast(lg + L * __logf(1.0f + 2.0f * awf * r), awf));
        r = fsqrt_fast(fdiv_fast(lg + L * __logf(1.0f + 2.0f * awf * r), awf));
        r += 0.5f + 0.25f * L;
    }
    float X0[3] = {bf.P[0] - kf.P[0], bf.P[1] - kf.P[1], bf.P[2] - kf.P[2]};
    float f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) f[a] = rintf(pl.Finvf[3 * a] * X0[0] + pl.Finvf[3 * a + 1] * X0[1] + pl.Finvf[3 * a + 2] * X0[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) X0[a] -= f[0] * pl.Lf[a] + f[1] * pl.Lf[3 + a] + f[2] * pl.Lf[6 + a];
    const float x2 = X0[0] * X0[0] + X0[1] * X0[1] + X0[2] * X0[2];
    const float r2 = r * r;
    if (x2 < r2) return true;
    const float x0n = fsqrt_fast(x2);
    for (int c = 1; c < pl.nr1; ++c) {
        if (pl.r1f[4 * c + 3] - x0n >= r) return false;
        const float Xx = X0[0] - pl.r1f[4 * c], Xy = X0[1] - pl.r1f[4 * c + 1], Xz = X0[2] - pl.r1f[4 * c + 2];
        if (Xx * Xx + Xy * Xy + Xz * Xz < r2) return true;
    }
    return false;
}

// One primitive quartet (bra pair xb, ket pair xk): screening radius of Eq.
// pbc_eri_real_cutoff_implementation (single precision), minimum image,
// the R1 images inside the sphere, seeds and the Hermite R table, then the
// contraction with both E tables into the Cartesian block V; the events go
// to the lane's tally (flops.h).
template <int LA, int LB, int LC, int LD, typename T>
__device__ __forceinline__ void prim_term(const PlanDev &pl, const PrimE<LA, LB, T> &b, const PpiF &bf, const PrimE<LC, LD, T> &k,
                                          const PpiF &kf, T *V, Tally &tl)
{
    constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
    constexpr int L = LA + LB + LC + LD, LAB = LA + LB, LCD = LC + LD;
    constexpr int NTA = LAB + 1, NTC = LCD + 1, D = L + 1;
    const float iw2 = pl.inv_omega2f;
    const float ipf = bf.pad, iqf = kf.pad;
    const float awf = frcp_fast(ipf + iqf + iw2);
    const float cwf = fsqrt_fast(awf * (ipf + iqf));
    const float preff = 34.986836655249725f * bf.K * kf.K * ipf * iqf * rsqrtf(bf.p + kf.p);
    ++tl.screen;
    const float lg = __logf(fabsf(preff) * (1.0f - cwf)) - pl.log_ewald_R;
    if (!(lg > 0.0f)) return;
    float r = fsqrt_fast(fdiv_fast(lg, awf));
    if (L > 0) {
        r = fsqrt_fast(fdiv_fast(lg + L * __logf(1.0f + 2.0f * awf * r), awf));
        r = fsqrt_fast(fdiv_fast(lg + L * __logf(1.0f + 2.0f * awf * r), awf));
        r += 0.5f + 0.25f * L;  // the Gaussian bound is derived for s functions; widen for L > 0
    }
    const float r2 = r * r;
    const PairT<T> &x = b.x, &y = k.x;
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
    ++tl.radius;
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
        const T Xx = X0[0] - lat_at(pl, 4 * c, T(0)), Xy = X0[1] - lat_at(pl, 4 * c + 1, T(0)), Xz = X0[2] - lat_at(pl, 4 * c + 2, T(0));
        const T x2 = Xx * Xx + Xy * Xy + Xz * Xz;
        ++tl.cand;
        if ((float)x2 >= r2) continue;
        any = true;
        ++tl.img;
        T s[L + 1];
        seeds<L>(x2, alpha, aw, cw, pl, s);
        T Bt[D * D * D];
        herm_R<L, T>(s, Xx, Xy, Xz, Bt);
#pragma unroll
        for (int t = 0; t <= L; ++t)
#pragma unroll
            for (int u = 0; u <= L - t; ++u)
#pragma unroll
                for (int v = 0; v <= L - t - u; ++v) Rs[(t * D + u) * D + v] += Bt[(t * D + u) * D + v];
    }
    if (!any) return;
    ++tl.term;
    const T tp = T(kTwoPi52) * x.K * y.K * ip * iq / sqrt(x.p + y.p);
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
                                    const T e = k.E[0][(cx * (LD + 1) + dx) * NTC + sx] * k.E[1][(cy * (LD + 1) + dy) * NTC + sy] *
                                                k.E[2][(cz * (LD + 1) + dz) * NTC + sz];
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
                for (int bb = 0; bb < NB; ++bb) {
                    const int ax = cexp(LA, a, 0), ay = cexp(LA, a, 1), az = cexp(LA, a, 2);
                    const int bx = cexp(LB, bb, 0), by = cexp(LB, bb, 1), bz = cexp(LB, bb, 2);
                    T v = T(0);
#pragma unroll
                    for (int tx = 0; tx <= ax + bx; ++tx)
#pragma unroll
                        for (int ty = 0; ty <= ay + by; ++ty)
#pragma unroll
                            for (int tz = 0; tz <= az + bz; ++tz)
                                v += b.E[0][(ax * (LB + 1) + bx) * NTA + tx] * b.E[1][(ay * (LB + 1) + by) * NTA + ty] *
                                     b.E[2][(az * (LB + 1) + bz) * NTA + tz] * W[(tx * NTA + ty) * NTA + tz];
                    V[((a * NB + bb) * NC + c) * ND + d] += tp * v;
                }
        }
}

// Digest the block V of the image quartet (bra sb, ket sk) with orbit weight
// w: ket-side Coulomb X_kl += 2w sum_ij V D_ij (atomics), exchange in its
// four index assignments (the other four of the orbit are transposes, added
// at assembly), and the bra-side Coulomb term into the lane's jb.
template <int LA, int LB, int LC, int LD, typename T>
__device__ __forceinline__ void digest(const PlanDev &pl, const SpiRec &sb, const SpiRec &sk, const T *V, T w, const T *__restrict__ Dp,
                                       const T *Dij, Acc<T> *jb, double *__restrict__ X, double *__restrict__ Y)
{
    constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
    const int n = pl.nbf;
    const int aoI = pl.shells[sb.I].ao, aoJ = pl.shells[sb.J].ao, aoK = pl.shells[sk.I].ao, aoL = pl.shells[sk.J].ao;
    auto Dd = [&](int r, int c) { return __ldg(Dp + (size_t)r * n + c); };
#pragma unroll
    for (int ab = 0; ab < NA * NB; ++ab) {
        T s = T(0);
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int d = 0; d < ND; ++d) s += V[ab * NC * ND + c * ND + d] * Dd(aoK + c, aoL + d);
        jb[ab].add(T(2) * w * s);
    }
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            T s = T(0);
#pragma unroll
            for (int ab = 0; ab < NA * NB; ++ab) s += V[ab * NC * ND + c * ND + d] * Dij[ab];
            atomicAdd(X + (size_t)(aoK + c) * n + aoL + d, to_f64(T(2) * w * s));
        }
    if (!Y) return;  // a Coulomb-only build
#pragma unroll
    for (int a = 0; a < NA; ++a)
#pragma unroll
        for (int d = 0; d < ND; ++d) {  // K_il += w V_ijkl D_jk
            T s = T(0);
#pragma unroll
            for (int b = 0; b < NB; ++b)
#pragma unroll
                for (int c = 0; c < NC; ++c) s += V[((a * NB + b) * NC + c) * ND + d] * Dd(aoJ + b, aoK + c);
            atomicAdd(Y + (size_t)(aoI + a) * n + aoL + d, to_f64(w * s));
        }
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int d = 0; d < ND; ++d) {  // K_jl += w V_ijkl D_ik
            T s = T(0);
#pragma unroll
            for (int a = 0; a < NA; ++a)
#pragma unroll
                for (int c = 0; c < NC; ++c) s += V[((a * NB + b) * NC + c) * ND + d] * Dd(aoI + a, aoK + c);
            atomicAdd(Y + (size_t)(aoJ + b) * n + aoL + d, to_f64(w * s));
        }
#pragma unroll
    for (int a = 0; a < NA; ++a)
#pragma unroll
        for (int c = 0; c < NC; ++c) {  // K_ik += w V_ijkl D_jl
            T s = T(0);
#pragma unroll
            for (int b = 0; b < NB; ++b)
#pragma unroll
                for (int d = 0; d < ND; ++d) s += V[((a * NB + b) * NC + c) * ND + d] * Dd(aoJ + b, aoL + d);
            atomicAdd(Y + (size_t)(aoI + a) * n + aoK + c, to_f64(w * s));
        }
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int c = 0; c < NC; ++c) {  // K_jk += w V_ijkl D_il
            T s = T(0);
#pragma unroll
            for (int a = 0; a < NA; ++a)
#pragma unroll
                for (int d = 0; d < ND; ++d) s += V[((a * NB + b) * NC + c) * ND + d] * Dd(aoI + a, aoL + d);
            atomicAdd(Y + (size_t)(aoJ + b) * n + aoK + c, to_f64(w * s));
        }
}

constexpr int kWarpsPerBlock = 4;

// Warp-per-bra tile kernel.  Block = 4 warps = 4 consecutive bras, one chunk
// of kchunk kets (blockIdx.y).  mode and the FP64 list as in k_real.
// Counters (cnt, one precision's base): [0] image quartets evaluated, [4]
// algorithmic flops, [8] screening and bookkeeping flops, [12] lane-terms
// processed and [14] lane slots offered in the primitive loop (their ratio
// is the lane occupancy).
template <int LA, int LB, int LC, int LD, typename T>
__global__ void __launch_bounds__(32 * kWarpsPerBlock) k_real_w(PlanDev pl, int b0, int b1, int k0, int k1, int same, int kchunk, int mode,
                                                                double tau, const T *__restrict__ Dp, const T *__restrict__ dmax,
                                                                double *__restrict__ X, double *__restrict__ Y,
                                                                unsigned long long *__restrict__ cnt, int2 *__restrict__ big,
                                                                unsigned *__restrict__ nbig, unsigned cap, unsigned *__restrict__ ovf)
{
    constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD), NV = NA * NB * NC * ND;
    constexpr int L = LA + LB + LC + LD;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int bra = b0 + blockIdx.x * kWarpsPerBlock + wid;
    if (bra >= b1) return;  // whole warp; no block-wide barrier below
    int kbeg = k0 + blockIdx.y * kchunk;
    const int kend = min(k1, kbeg + kchunk);
    if (same) kbeg = max(kbeg, bra);
    if (kbeg >= kend) return;
    const SpiRec sb = pl.spi[bra];
    const int n = pl.nbf, nsh = pl.nshell;
    const int aoI = pl.shells[sb.I].ao, aoJ = pl.shells[sb.J].ao;
    T Dij[NA * NB];
    Acc<T> jb[NA * NB];
#pragma unroll
    for (int a = 0; a < NA; ++a)
#pragma unroll
        for (int b = 0; b < NB; ++b) Dij[a * NB + b] = __ldg(Dp + (size_t)(aoI + a) * n + aoJ + b);
    const float tauf = (float)tau;
    Tally tl;
    unsigned used = 0, slots = 0;  // lane-terms processed and lane slots offered
    unsigned nq = 0;
    for (int kb = kbeg & ~31; kb < kend; kb += 32) {
        const int kt = kb + lane;
        bool valid = kt >= kbeg && kt < kend;
        // one bound for the 32-image block (the same for every lane)
        if (!__any_sync(0xffffffffu, valid) || !block_reaches<L>(pl, sb, kb >> 5)) continue;
        SpiRec sk{};
        if (valid) {
            sk = pl.spi[kt];
            valid = quartet_reaches<L>(pl, sb, sk);
        }
        if (sizeof(T) == 4 && valid && mode) {
            // precision policy: large quartets (and short [c_w, 1] intervals) go to the FP64 list
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
        const unsigned vmask = __ballot_sync(0xffffffffu, valid);
        if (!vmask) continue;
        nq += lane == 0 ? __popc(vmask) : 0;
        // lay the primitive pairs of the valid kets out one per lane
        const int np = valid ? sk.npp : 0;
        int incl = np;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        const int excl = incl - np;
        for (int e0 = 0; e0 < total; e0 += 32) {
            const int e = e0 + lane;
            const bool act = e < total;
            // owner lane: the first lane whose inclusive prefix exceeds e
            int own = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int probe = own + step - 1;
                const int v = __shfl_sync(0xffffffffu, incl, probe);
                if (v <= e) own += step;
            }
            if (!act) own = 32 + lane;  // a segment of its own
            const int src = own & 31;
            const int okt = __shfl_sync(0xffffffffu, kt, src);
            const int oex = __shfl_sync(0xffffffffu, excl, src);
            const int opp0 = __shfl_sync(0xffffffffu, sk.pp0, src);
            T V[NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) V[q] = T(0);
            if (act) {
                const int kpp = opp0 + (e - oex);
                PrimE<LC, LD, T> kp;
                PpiF kf;
                load_prim<LC, LD, T>(pl, kpp, kp, kf);
                ++tl.ketp;
                const float Bk = __ldg(pl.ppB + kpp);
                // bra primitives in descending order of their bound B: the
                // first one whose B_i B_k is below the magnitude threshold ends
                // the loop (every later term is smaller still)
                for (int i = 0; i < sb.npp; ++i) {
                    if (__ldg(pl.ppB + sb.pp0 + i) * Bk < pl.mag_thr) break;
                    PrimE<LA, LB, T> bp;
                    PpiF bf;
                    load_prim<LA, LB, T>(pl, sb.pp0 + i, bp, bf);
                    ++tl.brap;  // recomputed per lane: bookkeeping
                    prim_term<LA, LB, LC, LD, T>(pl, bp, bf, kp, kf, V, tl);
                    ++used;
                }
            }
            slots += (lane == 0) ? 32u * sb.npp : 0u;
            // segmented sum over the lanes holding the same ket (contiguous)
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int oo = __shfl_down_sync(0xffffffffu, own, o);
                const bool add = lane + o < 32 && oo == own;
#pragma unroll
                for (int q = 0; q < NV; ++q) {
                    const T t = __shfl_down_sync(0xffffffffu, V[q], o);
                    if (add) V[q] += t;
                }
            }
            const int prev = __shfl_up_sync(0xffffffffu, own, 1);
            const bool head = act && (lane == 0 || prev != own);
            if (head) {
                const SpiRec skh = pl.spi[okt];
                const T w = T(sb.w) * T(skh.w) * ((same && okt == bra) ? T(0.5) : T(1));
                digest<LA, LB, LC, LD, T>(pl, sb, skh, V, w, Dp, Dij, jb, X, Y);
                ++tl.quart;
            }
        }
    }
    // bra-side Coulomb: one atomic per element for the warp
#pragma unroll
    for (int a = 0; a < NA; ++a)
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const double v = warp_sum(jb[a * NB + b].value());
            if (lane == 0 && v != 0.0) atomicAdd(X + (size_t)(aoI + a) * n + aoJ + b, v);
        }
    unsigned long long fl = tally_alg<LA, LB, LC, LD>(tl), fs = tally_screen<LA, LB, LC, LD>(tl), u64 = used, s64 = slots;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        fl += __shfl_xor_sync(0xffffffffu, fl, o);
        fs += __shfl_xor_sync(0xffffffffu, fs, o);
        u64 += __shfl_xor_sync(0xffffffffu, u64, o);
        s64 += __shfl_xor_sync(0xffffffffu, s64, o);
    }
    if (lane == 0) {
        if (nq) atomicAdd(cnt, (unsigned long long)nq);
        if (fl) atomicAdd(cnt + 4, fl);
        if (fs) atomicAdd(cnt + 8, fs);
        if (u64) atomicAdd(cnt + 12, u64);
        if (s64) atomicAdd(cnt + 14, s64);
    }
}

// Pair-queue tile kernel (third family for s and p class pairs): as the
// lane-per-bra kernel, a warp holds 32 consecutive bras and walks the kets of
// its chunk; but every (bra, ket) image pair that passes the quartet-level
// bound goes into a per-warp queue in shared memory, and the queue is
// evaluated 32 pairs at a time, one pair per lane, so lanes whose own bra
// misses a ket do not idle while the others work.  The pairs of one batch
// are ordered by ket, so the ket-side Coulomb term is summed over the lanes
// of a ket by a segmented warp reduction; the bra-side term is added to the
// bra's FP64 partial in shared memory; exchange as in the other kernels.
template <int LA, int LB, int LC, int LD, typename T>
__global__ void __launch_bounds__(kRealThreads) k_real_q(PlanDev pl, int b0, int b1, int k0, int k1, int same, int kchunk, int mode,
                                                          double tau, const T *__restrict__ Dp, const T *__restrict__ dmax,
                                                          double *__restrict__ X, double *__restrict__ Y,
                                                          unsigned long long *__restrict__ cnt, int2 *__restrict__ big,
                                                          unsigned *__restrict__ nbig, unsigned cap, unsigned *__restrict__ ovf)
{
    constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD), NV = NA * NB * NC * ND;
    constexpr int L = LA + LB + LC + LD;
    constexpr int NW = kRealThreads / 32;
    __shared__ int qall[NW][64];
    __shared__ double jball[NW][32 * NA * NB];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int *qb = qall[wid];
    double *jbs = jball[wid];
    const int wbra0 = b0 + blockIdx.x * kRealThreads + 32 * wid;  // the warp's first bra
    const int bra = wbra0 + lane;
    int kbeg = k0 + blockIdx.y * kchunk;
    const int kend = min(k1, kbeg + kchunk);
    if (same) kbeg = max(kbeg, wbra0);
    if (kbeg >= kend || wbra0 >= b1) return;  // whole warp; no block-wide barrier below
    const bool act = bra < b1;
    const SpiRec sb = pl.spi[act ? bra : b0];
    const int n = pl.nbf, nsh = pl.nshell;
#pragma unroll
    for (int q = 0; q < NA * NB; ++q) jbs[lane * NA * NB + q] = 0.0;
    __syncwarp();
    const float tauf = (float)tau;
    unsigned nq = 0, qn = 0, qd = 0;
    Tally tl;
    // evaluate `count` queued pairs, one per lane
    auto process = [&](unsigned count) {
        const bool on = lane < count;
        int o = 0, kt = 0;
        if (on) {
            const int item = qb[(qd + lane) & 63];
            o = item & 31;
            kt = item >> 5;
        }
        T V[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) V[q] = T(0);
        SpiRec sbo{}, sk{};
        if (on) {
            sbo = pl.spi[wbra0 + o];
            sk = pl.spi[kt];
            quartet_block<LA, LB, LC, LD, T>(pl, sbo, sk, V, tl);
            ++tl.quart;
            ++nq;
        }
        const T w = on ? T(sbo.w) * T(sk.w) * ((same && kt == wbra0 + o) ? T(0.5) : T(1)) : T(0);
        const int aoI = pl.shells[on ? sbo.I : sb.I].ao, aoJ = pl.shells[on ? sbo.J : sb.J].ao;
        const int aoK = pl.shells[on ? sk.I : sb.I].ao, aoL = pl.shells[on ? sk.J : sb.J].ao;
        auto Dd = [&](int r, int c) { return __ldg(Dp + (size_t)r * n + c); };
        // bra-side Coulomb: the bra's FP64 partial in shared memory
        if (on) {
#pragma unroll
            for (int ab = 0; ab < NA * NB; ++ab) {
                T s2 = T(0);
#pragma unroll
                for (int c = 0; c < NC; ++c)
#pragma unroll
                    for (int d = 0; d < ND; ++d) s2 += V[ab * NC * ND + c * ND + d] * Dd(aoK + c, aoL + d);
                if (s2 != T(0)) atomicAdd(jbs + o * NA * NB + ab, to_f64(T(2) * w * s2));
            }
        }
        // ket-side Coulomb: segmented sum over the lanes of one ket (the batch is ordered by ket)
        const int key = on ? kt : -1 - lane;
#pragma unroll
        for (int cd = 0; cd < NC * ND; ++cd) {
            T s2 = T(0);
            if (on) {
                T Dij[NA * NB];
#pragma unroll
                for (int a = 0; a < NA; ++a)
#pragma unroll
                    for (int b = 0; b < NB; ++b) Dij[a * NB + b] = Dd(aoI + a, aoJ + b);
#pragma unroll
                for (int ab = 0; ab < NA * NB; ++ab) s2 += V[ab * NC * ND + cd] * Dij[ab];
                s2 *= T(2) * w;
            }
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int ok2 = __shfl_down_sync(0xffffffffu, key, off);
                const T t2 = __shfl_down_sync(0xffffffffu, s2, off);
                if (lane + off < 32 && ok2 == key) s2 += t2;
            }
            const int prevk = __shfl_up_sync(0xffffffffu, key, 1);
            if (on && (lane == 0 || prevk != key) && s2 != T(0))
                atomicAdd(X + (size_t)(aoK + cd / ND) * n + aoL + cd % ND, to_f64(s2));
        }
        // exchange: the four index assignments of the orbit (the other four are transposes)
        if (on && Y) {
#pragma unroll
            for (int a = 0; a < NA; ++a)
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    T s2 = T(0);
#pragma unroll
                    for (int b = 0; b < NB; ++b)
#pragma unroll
                        for (int c = 0; c < NC; ++c) s2 += V[((a * NB + b) * NC + c) * ND + d] * Dd(aoJ + b, aoK + c);
                    atomicAdd(Y + (size_t)(aoI + a) * n + aoL + d, to_f64(w * s2));
                }
#pragma unroll
            for (int b = 0; b < NB; ++b)
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    T s2 = T(0);
#pragma unroll
                    for (int a = 0; a < NA; ++a)
#pragma unroll
                        for (int c = 0; c < NC; ++c) s2 += V[((a * NB + b) * NC + c) * ND + d] * Dd(aoI + a, aoK + c);
                    atomicAdd(Y + (size_t)(aoJ + b) * n + aoL + d, to_f64(w * s2));
                }
#pragma unroll
            for (int a = 0; a < NA; ++a)
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    T s2 = T(0);
#pragma unroll
                    for (int b = 0; b < NB; ++b)
#pragma unroll
                        for (int d = 0; d < ND; ++d) s2 += V[((a * NB + b) * NC + c) * ND + d] * Dd(aoJ + b, aoL + d);
                    atomicAdd(Y + (size_t)(aoI + a) * n + aoK + c, to_f64(w * s2));
                }
#pragma unroll
            for (int b = 0; b < NB; ++b)
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    T s2 = T(0);
#pragma unroll
                    for (int a = 0; a < NA; ++a)
#pragma unroll
                        for (int d = 0; d < ND; ++d) s2 += V[((a * NB + b) * NC + c) * ND + d] * Dd(aoI + a, aoL + d);
                    atomicAdd(Y + (size_t)(aoJ + b) * n + aoK + c, to_f64(w * s2));
                }
        }
        qd += count;
        __syncwarp();
    };
    for (int kt = kbeg; kt < kend; ++kt) {
        // one bound per block of 32 kets for the whole warp first
        if (kt == kbeg || (kt & 31) == 0) {
            if (!__any_sync(0xffffffffu, act && block_reaches<L>(pl, sb, kt >> 5))) {
                kt = min(kend, ((kt >> 5) + 1) << 5) - 1;
                continue;
            }
        }
        const SpiRec sk = pl.spi[kt];
        bool valid = act && (!same || kt >= bra) && quartet_reaches<L>(pl, sb, sk);
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
        const unsigned m = __ballot_sync(0xffffffffu, valid);
        if (!m) continue;
        if (valid) qb[(qn + __popc(m & ((1u << lane) - 1u))) & 63] = (kt << 5) | lane;
        qn += __popc(m);
        __syncwarp();
        if (qn - qd >= 32) process(32);
    }
    while (qn > qd) process(min(32u, qn - qd));
    // the bra-side Coulomb partials of the warp's bras
    if (act) {
        const int aoI = pl.shells[sb.I].ao, aoJ = pl.shells[sb.J].ao;
#pragma unroll
        for (int a = 0; a < NA; ++a)
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const double v = jbs[lane * NA * NB + a * NB + b];
                if (v != 0.0) atomicAdd(X + (size_t)(aoI + a) * n + aoJ + b, v);
            }
    }
    unsigned long long fl = tally_alg<LA, LB, LC, LD>(tl), fs = tally_screen<LA, LB, LC, LD>(tl);
    unsigned tot = nq;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        tot += __shfl_xor_sync(0xffffffffu, tot, o);
        fl += __shfl_xor_sync(0xffffffffu, fl, o);
        fs += __shfl_xor_sync(0xffffffffu, fs, o);
    }
    if (lane == 0) {
        if (tot) atomicAdd(cnt, (unsigned long long)tot);
        if (fl) atomicAdd(cnt + 4, fl);
        if (fs) atomicAdd(cnt + 8, fs);
    }
}

// FP64 pass over the listed large quartets: one warp per list entry.  The
// entry's npp_bra x npp_ket primitive quartets are screened 32 at a time in
// single precision, the ones that pass go into a per-warp queue (shared
// memory) and are evaluated in FP64 one per lane, 32 at a time, into the
// lane's block; the block is summed over the warp and digested by lane 0.
// Counters as k_real_w (cnt points at the FP64 slots).
template <int LA, int LB, int LC, int LD>
__global__ void __launch_bounds__(32 * kWarpsPerBlock) k_real_list_w(PlanDev pl, const int2 *__restrict__ big, const unsigned *__restrict__ nbig,
                                                                     unsigned cap, int same, const double *__restrict__ Dp,
                                                                     double *__restrict__ X, double *__restrict__ Y,
                                                                     unsigned long long *__restrict__ cnt)
{
    constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD), NV = NA * NB * NC * ND;
    constexpr int L = LA + LB + LC + LD;
    __shared__ int qall[kWarpsPerBlock][64];
    const int lane = threadIdx.x & 31;
    int *qbuf = qall[threadIdx.x >> 5];
    const unsigned total = min(*nbig, cap);
    const int n = pl.nbf;
    Tally tl;
    unsigned used = 0, slots = 0;
    unsigned done = 0;
    const unsigned nwarps = gridDim.x * kWarpsPerBlock;
    for (unsigned q = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5); q < total; q += nwarps) {
        const int2 pr = big[q];
        const SpiRec sb = pl.spi[pr.x], sk = pl.spi[pr.y];
        const int nterm = sb.npp * sk.npp;
        double V[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) V[k] = 0.0;
        unsigned qn = 0, qd = 0;
        auto drain = [&](unsigned count) {
            if (lane < count) {
                const int t = qbuf[(qd + lane) & 63];
                const int i = t / sk.npp, j = t - i * sk.npp;
                PrimE<LA, LB, double> bp;
                PrimE<LC, LD, double> kp;
                PpiF bf, kf;
                load_prim<LA, LB, double>(pl, sb.pp0 + i, bp, bf);
                load_prim<LC, LD, double>(pl, sk.pp0 + j, kp, kf);
                ++tl.brap;
                ++tl.ketp;
                prim_term<LA, LB, LC, LD, double>(pl, bp, bf, kp, kf, V, tl);
                ++used;
            }
            if (lane == 0) slots += 32;
            qd += count;
            __syncwarp();
        };
        for (int t0 = 0; t0 < nterm; t0 += 32) {
            const int t = t0 + lane;
            bool pass = false;
            if (t < nterm) {
                const int i = t / sk.npp, j = t - i * sk.npp;
                pass = __ldg(pl.ppB + sb.pp0 + i) * __ldg(pl.ppB + sk.pp0 + j) >= pl.mag_thr &&
                       prim_reaches<L>(pl, pl.ppf[sb.pp0 + i], pl.ppf[sk.pp0 + j]);
                ++tl.screen;
            }
            const unsigned m = __ballot_sync(0xffffffffu, pass);
            if (pass) qbuf[(qn + __popc(m & ((1u << lane) - 1u))) & 63] = t;
            qn += __popc(m);
            __syncwarp();
            if (qn - qd >= 32) drain(32);
        }
        while (qn > qd) drain(min(32u, qn - qd));
#pragma unroll
        for (int k = 0; k < NV; ++k) V[k] = warp_sum(V[k]);
        if (lane == 0) {
            ++done;
            Acc<double> jb[NA * NB];
            double Dij[NA * NB];
            const int aoI = pl.shells[sb.I].ao, aoJ = pl.shells[sb.J].ao;
#pragma unroll
            for (int a = 0; a < NA; ++a)
#pragma unroll
                for (int b = 0; b < NB; ++b) Dij[a * NB + b] = __ldg(Dp + (size_t)(aoI + a) * n + aoJ + b);
            const double w = double(sb.w) * double(sk.w) * ((same && pr.x == pr.y) ? 0.5 : 1.0);
            digest<LA, LB, LC, LD, double>(pl, sb, sk, V, w, Dp, Dij, jb, X, Y);
            ++tl.quart;
#pragma unroll
            for (int a = 0; a < NA; ++a)
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    const double v = jb[a * NB + b].value();
                    if (v != 0.0) atomicAdd(X + (size_t)(aoI + a) * n + aoJ + b, v);
                }
        }
        __syncwarp();
    }
    unsigned long long fl = tally_alg<LA, LB, LC, LD>(tl), fs = tally_screen<LA, LB, LC, LD>(tl), u64 = used, s64 = slots;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        fl += __shfl_xor_sync(0xffffffffu, fl, o);
        fs += __shfl_xor_sync(0xffffffffu, fs, o);
        u64 += __shfl_xor_sync(0xffffffffu, u64, o);
        s64 += __shfl_xor_sync(0xffffffffu, s64, o);
    }
    if (lane == 0) {
        if (done) atomicAdd(cnt, (unsigned long long)done);
        if (fl) atomicAdd(cnt + 4, fl);
        if (fs) atomicAdd(cnt + 8, fs);
        if (u64) atomicAdd(cnt + 12, u64);
        if (s64) atomicAdd(cnt + 14, s64);
    }
}

}  // namespace jk
