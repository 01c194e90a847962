// Split-precision GEMMs on the BF16 tensor cores for the reciprocal
// exchange contraction K_LR = sum_b M_b D M_b (b runs over the real and
// imaginary parts of the structure-factor slab of each G).
//
// Each FP64 operand row r is scaled by 2^{-sigma_r} (sigma_r from the
// largest exponent in the row) and cut into S slices of balanced signed
// digits, x ~ 2^{sigma_r} sum_s d_s 2^{-7-8s} with d_s in [-128, 128]
// (exact in BF16, whose significand holds 8 bits): the first digit carries
// 8 bits including the sign and every further digit 8 more, about 8S - 1
// significant bits per operand.  The digits come from integer arithmetic on
// the IEEE significand, so slicing costs no FP64 arithmetic.  A slice
// product over K <= 1024 terms sums integers of magnitude at most 2^14, so
// its sum stays within 2^24 and is exact in the FP32 accumulator of the
// tensor-core MMA; the products with s + t <= S - 1 (0-based) are combined
// with their power-of-two scales in a compensated single-precision pair.
// This is the error-free splitting of Ozaki, Ogita, Oishi and Rump (Numer.
// Algorithms 59, 2012) with digits sized to the FP32 accumulator.  The
// GEMMs run on the tcgen05 tensor cores (TMA operand tiles, accumulators
// and the compensated pairs in tensor memory; k_ozaki_tc below).
//
// Two factorisations of the contraction:
//   dense:    Zt_b = (D M_b)^T, then K += sum_b M_b Z_b;
//   low rank: D = C+ C+^T - C- C-^T from the device-side pivoted LDL^T of
//             dense.cu (a closed-shell SCF density has rank n_occ), then
//             Y_b = M_b [C+ C-] and K += sum_b Y+_b Y+_b^T - Y-_b Y-_b^T.
// Which form a build takes is decided on the device: the launches of both
// are enqueued, and each kernel reads the factorisation's status array
// (TcArgs::dyn) and returns at once when its form was not chosen.
// M_b is symmetric, so its row slices serve as the A operand of one GEMM
// and the B operand (B^T rows) of the other; the K GEMMs form only tiles on
// or above the diagonal and mirror them.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "plan.h"
#include "tc.cuh"

namespace jk {

namespace {

constexpr int KFLUSH = 1024;  // exactness bound of the FP32 accumulator

__device__ __forceinline__ void two_sum_add(float &hi, float &lo, float x)
{
    const float t = hi + x;
    const float bp = t - hi;
    lo += (hi - (t - bp)) + (x - bp);
    hi = t;
}

}  // namespace

// Slices of a batch of rows x cols FP64 matrices (row-major, leading dim ld,
// batch stride bstride elements): one warp per row.  sigma = E_max - 1022
// with E_max the largest biased exponent in the row (so |x| < 2^sigma);
// V = x 2^{62 - sigma} (|V| < 2^62) is formed exactly as a signed 64-bit
// integer by shifting the 53-bit significand, and the digits are taken from
// the top by rounding to nearest: d_s = round(V_s / 2^{55 - 8s}),
// V_{s+1} = V_s - d_s 2^{55 - 8s}, so |V_{s+1}| <= 2^{54 - 8s} and the next
// digit again lies in [-128, 128].  S <= 7.  Output:
// out[((b*S + s)*rows_pad + r)*cols_pad + k] (zero outside rows x cols),
// ex[b*rows_pad + r].
__global__ void k_ozaki_slice(const double *__restrict__ X, int rows, int cols, int ld, long long bstride, int rows_pad, int cols_pad,
                              int S, int B, __nv_bfloat16 *__restrict__ out, int *__restrict__ ex)
{
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= (long long)B * rows_pad) return;
    const int b = (int)(warp / rows_pad), r = (int)(warp % rows_pad);
    const unsigned long long *row = reinterpret_cast<const unsigned long long *>(X + (size_t)b * bstride + (size_t)r * ld);
    int emax = 0;
    if (r < rows)
        for (int k = lane; k < cols; k += 32) emax = max(emax, (int)((row[k] >> 52) & 0x7ff));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    const int sigma = emax > 0 ? emax - 1022 : 0;
    if (lane == 0) ex[(size_t)b * rows_pad + r] = sigma;
    __nv_bfloat16 *o = out + ((size_t)b * S * rows_pad + r) * cols_pad;
    const size_t sstride = (size_t)rows_pad * cols_pad;
    auto scaled = [&](int k) -> long long {
        if (r >= rows || k >= cols) return 0;
        const unsigned long long bits = row[k];
        const int E = (int)((bits >> 52) & 0x7ff);
        if (E == 0) return 0;  // zero; subnormals flush to zero
        const unsigned long long M = (bits & 0xfffffffffffffull) | (1ull << 52);
        const int sh = E - 1013 - sigma;  // <= 9, so F < 2^62
        const unsigned long long F = sh >= 0 ? (M << sh) : (sh > -64 ? (M >> (-sh)) : 0ull);
        return (bits >> 63) ? -(long long)F : (long long)F;
    };
    // two adjacent columns per lane, stored as one bf16 pair per slice
    // (cols_pad and the slice stride are even)
    for (int k = 2 * lane; k < cols_pad; k += 64) {
        long long V0 = scaled(k), V1 = scaled(k + 1);
        for (int s = 0; s < S; ++s) {
            const int shift = 55 - 8 * s;
            const long long d0 = (V0 + (1LL << (shift - 1))) >> shift;  // arithmetic shift: floor
            const long long d1 = (V1 + (1LL << (shift - 1))) >> shift;
            V0 -= d0 * (1LL << shift);
            V1 -= d1 * (1LL << shift);
            *reinterpret_cast<__nv_bfloat162 *>(o + s * sstride + k) = __floats2bfloat162_rn((float)d0, (float)d1);
        }
    }
}

// ---------------------------------------------------------------------------
// The split-precision GEMMs on the tcgen05 tensor cores.  One CTA per
// 128 x 128 output tile and range of batches: thread 256 (warp 8) issues
// the TMA loads of the operand slices (4-stage ring of 128 x 64 BF16 tiles
// per operand, 128-byte swizzle) and the tcgen05.mma instructions (M = N =
// 128, K = 16) into one of two FP32 accumulators in tensor memory; warps 0-7
// (two per TMEM lane quadrant, 64 columns each, one output row per thread)
// fold each exact slice product into a compensated FP32 pair (hi, lo) kept
// in tensor memory.  TMEM columns: accumulators 0-127 and 128-255, hi
// 256-383, lo 384-511.  The epilogue does no FP64 arithmetic: MODE 0 writes
// (hi, lo) float pairs (read by the pair slicer), MODE 1 adds them into
// float-pair partial sums with FP32 two-sums.
struct TcArgs {
    int a_batch_rows, a_slice_rows;  // TMA row of A slice s, batch b: a_row0 + b*a_batch_rows + s*a_slice_rows + row
    int b_batch_rows, b_slice_rows;
    int a_row0, b_row0;              // first row of the operand in its tensor map (a chunk of the reciprocal cache)
    const int *Aex;
    int a_exb;  // exponents of batch b at Aex[b * a_exb] (a_exb = 0: shared)
    const int *Bex;
    int b_exb;
    int koff, klen;  // K range, multiples of 64
    int S, nb, bsplit, ntm, ntn;
    float2 *out;  // MODE 0: per-batch output as (hi, lo) pairs
    int out_rows, out_cols;
    long long o_bstride;
    int ldo, transpose;
    float2 *part;  // MODE 1: (hi, lo) partial sums, split z at part + z * part_stride (upper tiles only)
    long long part_stride;
    int ldp;
    float sign;
    unsigned *err;
    // device status of the low-rank factorisation (dyn[0] low rank chosen,
    // dyn[1] rows of C+, dyn[2] rows of C-) and what this launch computes:
    // 0 always, 1 dense form only, 2 Y = M [C+ C-] (column tiles up to
    // dyn[1] + dyn[2]), 3 K += Y+ Y+^T (K range [0, dyn[1])), 4 K -= Y- Y-^T
    // (K range [dyn[1], dyn[1] + dyn[2]))
    const int *dyn;
    int dyn_mode;
};

constexpr int TC_BM = 128, TC_BN = 128, TC_BK = 64, TC_ST = 4, TC_KCH = KFLUSH / TC_BK;
constexpr int TC_EPI_WARPS = 8, TC_THREADS = 32 * (TC_EPI_WARPS + 1), TC_PROD = 32 * TC_EPI_WARPS;
constexpr uint32_t TC_TILE_BYTES = TC_BM * TC_BK * 2;  // 16 KB per operand tile
constexpr size_t TC_SMEM = (size_t)TC_ST * 2 * TC_TILE_BYTES + 1024;
constexpr uint64_t TC_WAIT_NS = 2000000000ull;

// 2^e as a float for the slice scales, 0 below the normal range (such a term
// is below 2^-126 and negligible against the entries it is added to)
__device__ __forceinline__ float pow2f(int e) { return __int_as_float(max(e + 127, 0) << 23); }

// (h, l) += (x, y), all float pairs with |l| <= ulp(h)/2 (double-float addition)
__device__ __forceinline__ void pair_add(float &h, float &l, float x, float y)
{
    const float s = h + x;
    const float bp = s - h;
    float e = (h - (s - bp)) + (x - bp);
    e += l + y;
    h = s + e;
    l = e - (h - s);
}

// Position in the work sequence of one CTA: batch b, slice pair (s, t) with
// s + t < S, K block kb.
struct TcCursor {
    int b, s, t, kb;
    bool done;
};
__device__ __forceinline__ void tc_advance(TcCursor &c, int nk, int S, int b1)
{
    if (++c.kb < nk) return;
    c.kb = 0;
    if (c.s + ++c.t < S) return;
    c.t = 0;
    if (++c.s < S) return;
    c.s = 0;
    if (++c.b >= b1) c.done = true;
}

template <int MODE>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_ozaki_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcArgs g)
{
    extern __shared__ uint8_t tc_dsm[];
    __shared__ __align__(8) uint64_t full[TC_ST], empty[TC_ST], acc_full[2], acc_empty[2];
    __shared__ __align__(16) int cex_s[TC_EPI_WARPS][64];  // column exponents of the current batch, per epilogue warp
    __shared__ uint32_t tmem_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sbase = tc::smem_u32(tc_dsm);
    const uint32_t tiles = (sbase + 1023u) & ~1023u;  // 1024-byte aligned operand ring (shared address)
    uint8_t *tiles_gen = tc_dsm + (tiles - sbase);

    int mi, nj;
    if (MODE == 0) {
        mi = blockIdx.x % g.ntm;
        nj = blockIdx.x / g.ntm;
    } else {
        int t = blockIdx.x;
        mi = 0;
        while (t >= g.ntm - mi) {
            t -= g.ntm - mi;
            ++mi;
        }
        nj = mi + t;
    }
    // form selected on the device: a CTA with no work returns before it
    // touches barriers or tensor memory (the test is uniform over the CTA)
    int koff = g.koff, klen = g.klen;
    if (g.dyn_mode) {
        const int low = g.dyn[0], rp = g.dyn[1], rn = g.dyn[2];
        if (g.dyn_mode == 1 && low) return;
        if (g.dyn_mode == 2 && (!low || nj * TC_BN >= rp + rn)) return;
        if (g.dyn_mode == 3) {
            if (!low || rp == 0) return;
            koff = 0;
            klen = rp;
        }
        if (g.dyn_mode == 4) {
            if (!low || rn == 0) return;
            koff = rp;
            klen = rn;
        }
    }
    const int per = (g.nb + g.bsplit - 1) / g.bsplit;
    const int b0 = blockIdx.z * per, b1 = min(g.nb, b0 + per);
    const int row0 = mi * TC_BM, col0 = nj * TC_BN;
    const int nk = klen / TC_BK, nkc = (nk + TC_KCH - 1) / TC_KCH;

    if (tid == TC_PROD) {
        for (int i = 0; i < TC_ST; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&acc_full[i], 1);
            tc::mbar_init(&acc_empty[i], 32 * TC_EPI_WARPS);
        }
        tc::fence_mbar_init();
        tc::prefetch_tmap(&tmA);
        tc::prefetch_tmap(&tmB);
    }
    if (warp == 0) {
        tc::tmem_alloc(&tmem_s, 512);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_s;
    bool ok = b0 < b1;

    if (warp == TC_EPI_WARPS) {
        if (lane == 0 && ok) {
            const uint32_t idesc = tc::idesc_bf16_f32(TC_BM, TC_BN);
            TcCursor mc{b0, 0, 0, 0, false}, lc{b0, 0, 0, 0, false};
            long long m = 0, j = 0;  // loads consumed by MMAs, loads issued
            int c = 0;                // accumulator chunks completed
            auto issue = [&](const TcCursor &q, int slot) {
                uint8_t *a = tiles_gen + (size_t)slot * 2 * TC_TILE_BYTES;
                const int x = koff + q.kb * TC_BK;
                tc::mbar_expect_tx(&full[slot], 2 * TC_TILE_BYTES);
                tc::tma_load_2d(a, &tmA, &full[slot], x, g.a_row0 + q.b * g.a_batch_rows + q.s * g.a_slice_rows + row0);
                tc::tma_load_2d(a + TC_TILE_BYTES, &tmB, &full[slot], x, g.b_row0 + q.b * g.b_batch_rows + q.t * g.b_slice_rows + col0);
            };
            for (; j < TC_ST - 1 && !lc.done; ++j) {
                issue(lc, (int)(j % TC_ST));
                tc_advance(lc, nk, g.S, b1);
            }
            while (!mc.done && ok) {
                const bool first = mc.kb % TC_KCH == 0, last = (mc.kb % TC_KCH == TC_KCH - 1) || mc.kb == nk - 1;
                const int buf = c & 1, use = c >> 1;
                if (first && use >= 1 && !tc::mbar_wait(&acc_empty[buf], (use - 1) & 1, TC_WAIT_NS)) {
                    ok = false;
                    break;
                }
                const int slot = (int)(m % TC_ST);
                if (!tc::mbar_wait(&full[slot], (uint32_t)((m / TC_ST) & 1), TC_WAIT_NS)) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t a = tiles + (uint32_t)slot * 2 * TC_TILE_BYTES, bb = a + TC_TILE_BYTES;
                const uint64_t ad = tc::sdesc_k128(a), bd = tc::sdesc_k128(bb);
#pragma unroll
                for (int k = 0; k < TC_BK / 16; ++k)
                    tc::mma_bf16(tmem + (uint32_t)buf * TC_BN, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), idesc,
                                 (!first || k > 0) ? 1u : 0u);
                tc::mma_commit(&empty[slot]);
                if (last) {
                    tc::mma_commit(&acc_full[buf]);
                    ++c;
                }
                ++m;
                tc_advance(mc, nk, g.S, b1);
                if (!lc.done) {
                    const int s2 = (int)(j % TC_ST);
                    if (j >= TC_ST && !tc::mbar_wait(&empty[s2], (uint32_t)(((j / TC_ST) - 1) & 1), TC_WAIT_NS)) {
                        ok = false;
                        break;
                    }
                    issue(lc, s2);
                    tc_advance(lc, nk, g.S, b1);
                    ++j;
                }
            }
            // drain: every issued load has landed and every MMA has completed
            // before the CTA releases its shared and tensor memory
            for (long long q = m; q < j; ++q) tc::mbar_wait(&full[q % TC_ST], (uint32_t)((q / TC_ST) & 1), TC_WAIT_NS);
            for (long long q = (m > TC_ST ? m - TC_ST : 0); q < m; ++q)
                tc::mbar_wait(&empty[q % TC_ST], (uint32_t)((q / TC_ST) & 1), TC_WAIT_NS);
            if (!ok) atomicOr(g.err, 2u);
        }
    } else if (ok) {
        // epilogue: warp w serves TMEM lanes 32 (w % 4) .. + 31 (output rows)
        // and columns 64 (w / 4) .. + 63.  Waits are made warp-uniform
        // (tcgen05.ld/st are warp-collective) and no barrier spans the
        // epilogue warps, so a wait that runs out ends this warp's work
        // without stranding another thread.
        const int quad = warp & 3, half = warp >> 2;
        const int rl = 32 * quad + lane, r = row0 + rl;
        const uint32_t lane_addr = tmem + ((uint32_t)(32 * quad) << 16);
        int c = 0;
        bool fresh = true;
        for (int b = b0; b < b1 && ok; ++b) {
            const int rex = g.Aex[(size_t)(g.a_exb ? b : 0) * g.a_exb + r];
            // the warp's 64 column exponents of this batch, staged once in
            // shared memory (read back as broadcasts for every slice product)
            {
                const int *cex = g.Bex + (size_t)(g.b_exb ? b : 0) * g.b_exb + col0 + 64 * half;
                __syncwarp();
                cex_s[warp][lane] = __ldg(cex + lane);
                cex_s[warp][32 + lane] = __ldg(cex + 32 + lane);
                __syncwarp();
            }
            const int4 *cex4 = reinterpret_cast<const int4 *>(cex_s[warp]);
            if (MODE == 0) fresh = true;
            for (int s = 0; s < g.S && ok; ++s)
                for (int t = 0; s + t < g.S && ok; ++t)
                    for (int kc = 0; kc < nkc && ok; ++kc) {
                        const int buf = c & 1, use = c >> 1;
                        ok = __all_sync(0xffffffffu, tc::mbar_wait(&acc_full[buf], use & 1, TC_WAIT_NS));
                        if (!ok) break;
                        tc::fence_after_sync();
                        const bool fin = (s == g.S - 1 && t == 0 && kc == nkc - 1) && (MODE == 0 || b == b1 - 1);
                        const int base = rex - 14 - 8 * (s + t);
#pragma unroll 1
                        for (int q = 0; q < 2; ++q) {
                            const int cq = 64 * half + 32 * q;  // first column of this group within the tile
                            float av[32], hv[32], lv[32];
                            int ce[32];
#pragma unroll
                            for (int i = 0; i < 8; ++i) {
                                const int4 v = cex4[8 * q + i];
                                ce[4 * i] = v.x;
                                ce[4 * i + 1] = v.y;
                                ce[4 * i + 2] = v.z;
                                ce[4 * i + 3] = v.w;
                            }
                            tc::tmem_ld32(lane_addr + (uint32_t)(buf * TC_BN + cq), av);
                            if (!fresh) {
                                tc::tmem_ld32(lane_addr + (uint32_t)(256 + cq), hv);
                                tc::tmem_ld32(lane_addr + (uint32_t)(384 + cq), lv);
                            }
                            tc::tmem_ld_wait();
#pragma unroll
                            for (int e = 0; e < 32; ++e) {
                                const float v = av[e] * pow2f(base + ce[e]);
                                if (fresh) {
                                    hv[e] = v;
                                    lv[e] = 0.f;
                                } else {
                                    two_sum_add(hv[e], lv[e], v);
                                }
                            }
                            if (fin) {
                                if (MODE == 0) {
                                    float2 *O = g.out + (size_t)b * g.o_bstride;
                                    if (r < g.out_rows)
#pragma unroll
                                        for (int e = 0; e < 32; ++e) {
                                            const int cc = col0 + cq + e;
                                            if (cc < g.out_cols)
                                                O[g.transpose ? (size_t)cc * g.ldo + r : (size_t)r * g.ldo + cc] = make_float2(hv[e], lv[e]);
                                        }
                                } else {
                                    float2 *Pz = g.part + (size_t)blockIdx.z * g.part_stride + (size_t)r * g.ldp;
                                    if (r < g.out_rows)
#pragma unroll
                                        for (int e = 0; e < 32; ++e) {
                                            const int cc = col0 + cq + e;
                                            if (cc < g.out_cols) {
                                                float2 p = Pz[cc];
                                                pair_add(p.x, p.y, g.sign * hv[e], g.sign * lv[e]);
                                                Pz[cc] = p;
                                            }
                                        }
                                }
                            } else {
                                tc::tmem_st32(lane_addr + (uint32_t)(256 + cq), hv);
                                tc::tmem_st32(lane_addr + (uint32_t)(384 + cq), lv);
                            }
                        }
                        tc::tmem_st_wait();
                        tc::fence_before_sync();
                        tc::mbar_arrive(&acc_empty[buf]);
                        fresh = false;
                        ++c;
                    }
        }
        if (!ok) atomicOr(g.err, 4u);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, 512);
    }
}

// K_LR[i][j] += sum_z part_z[min-tile][max-tile]: the (hi, lo) partial sums
// hold the tiles on or above the diagonal; the lower tiles are their
// transposes.
__global__ void k_kpart_reduce(int n, int ldp, int splits, long long pstride, const float2 *__restrict__ part, double *__restrict__ KLR)
{
    const long long n2 = (long long)n * n;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n2; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        const bool up = (i / TC_BM) <= (j / TC_BN);
        const size_t idx = up ? (size_t)i * ldp + j : (size_t)j * ldp + i;
        double v = 0;
        for (int z = 0; z < splits; ++z) {
            const float2 p = part[(size_t)z * pstride + idx];
            v += (double)p.x + (double)p.y;
        }
        KLR[e] += v;
    }
}

// Slices (as k_ozaki_slice) of rows given as (hi, lo) float pairs x = hi + lo
// with |lo| <= ulp(hi)/2: sigma = E_max - 126 from the largest float exponent
// of hi in the row (so |x| < 2^sigma), and V = x 2^{62 - sigma} is formed
// exactly from the two significands as a signed 64-bit integer (bits of lo
// below 2^0 are dropped).
__global__ void k_ozaki_slice_pair(const float2 *__restrict__ X, int rows, int cols, int ld, long long bstride, int rows_pad,
                                   int cols_pad, int S, int B, __nv_bfloat16 *__restrict__ out, int *__restrict__ ex,
                                   const int *__restrict__ dyn, int dyn_mode)
{
    // dyn_mode 1: dense form only; 2: low-rank Y, whose first dyn[1] + dyn[2] columns are live
    if (dyn_mode == 1 && dyn[0]) return;
    if (dyn_mode == 2) {
        if (!dyn[0]) return;
        cols = min(cols, dyn[1] + dyn[2]);
    }
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= (long long)B * rows_pad) return;
    const int b = (int)(warp / rows_pad), r = (int)(warp % rows_pad);
    const float2 *row = X + (size_t)b * bstride + (size_t)r * ld;
    int emax = 0;
    if (r < rows)
        for (int k = lane; k < cols; k += 32) emax = max(emax, (int)((__float_as_uint(row[k].x) >> 23) & 0xff));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    const int sigma = emax > 0 ? emax - 126 : 0;
    if (lane == 0) ex[(size_t)b * rows_pad + r] = sigma;
    __nv_bfloat16 *o = out + ((size_t)b * S * rows_pad + r) * cols_pad;
    const size_t sstride = (size_t)rows_pad * cols_pad;
    auto part = [&](float f) -> long long {
        const unsigned u = __float_as_uint(f);
        const int E = (int)((u >> 23) & 0xff);
        if (E == 0) return 0;  // zero or subnormal
        const unsigned long long M = (u & 0x7fffffu) | 0x800000u;
        const int sh = E - 88 - sigma;  // <= 38 for hi, so |term| < 2^62
        const unsigned long long F = sh >= 0 ? (M << sh) : (sh > -64 ? (M >> (-sh)) : 0ull);
        return (u >> 31) ? -(long long)F : (long long)F;
    };
    // the low-rank Y is read by the GEMMs up to its live columns (a multiple
    // of 128); the dense form through cols_pad
    const int cend = dyn_mode == 2 ? min(cols_pad, (cols + 127) / 128 * 128) : cols_pad;
    // two adjacent columns per lane, stored as one bf16 pair per slice
    // (cols_pad and the slice stride are even)
    for (int k = 2 * lane; k < cend; k += 64) {
        long long V0 = 0, V1 = 0;
        if (r < rows) {
            if (k < cols) {
                const float2 x = row[k];
                V0 = part(x.x) + part(x.y);
            }
            if (k + 1 < cols) {
                const float2 x = row[k + 1];
                V1 = part(x.x) + part(x.y);
            }
        }
        for (int s = 0; s < S; ++s) {
            const int shift = 55 - 8 * s;
            const long long d0 = (V0 + (1LL << (shift - 1))) >> shift;  // arithmetic shift: floor
            const long long d1 = (V1 + (1LL << (shift - 1))) >> shift;
            V0 -= d0 * (1LL << shift);
            V1 -= d1 * (1LL << shift);
            *reinterpret_cast<__nv_bfloat162 *>(o + s * sstride + k) = __floats2bfloat162_rn((float)d0, (float)d1);
        }
    }
}

static unsigned blocks_for_rows(long long rows) { return (unsigned)((rows * 32 + 255) / 256); }

static void slice(const double *X, int rows, int cols, int ld, long long bstride, int rows_pad, int cols_pad, int S, int B,
                  __nv_bfloat16 *out, int *ex, cudaStream_t st)
{
    k_ozaki_slice<<<blocks_for_rows((long long)B * rows_pad), 256, 0, st>>>(X, rows, cols, ld, bstride, rows_pad, cols_pad, S, B, out, ex);
}

static void slice_pair(const float2 *X, int rows, int cols, int ld, long long bstride, int rows_pad, int cols_pad, int S, int B,
                       __nv_bfloat16 *out, int *ex, const int *dyn, int dyn_mode, cudaStream_t st)
{
    k_ozaki_slice_pair<<<blocks_for_rows((long long)B * rows_pad), 256, 0, st>>>(X, rows, cols, ld, bstride, rows_pad, cols_pad, S, B, out,
                                                                                  ex, dyn, dyn_mode);
}

// batches per CTA of a tcgen05 GEMM launch: about two waves of CTAs
static int tc_splits(int tiles, int nb) { return std::max(1, std::min(nb, (2 * 152 + tiles / 2) / std::max(1, tiles))); }

static int check(const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(JK_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return JK_OK;
}

// ---- tcgen05 form: tensor maps, launch helpers --------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *, const cuuint64_t *,
                                  const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

// Tensor map of a slice buffer viewed as `rows` K-major rows of kpad BF16
// (kpad a multiple of 64, base 16-byte aligned), 64 x 128 boxes, 128-byte swizzle.
static bool slice_map(CUtensorMap *m, const __nv_bfloat16 *base, long long rows, int kpad)
{
    EncodeTiledFn f = encode_tiled();
    if (!f || kpad % TC_BK || ((uintptr_t)base & 15)) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)kpad * 2};
    const cuuint32_t box[2] = {TC_BK, TC_BM};
    const cuuint32_t es[2] = {1, 1};
    return f(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Called once per plan after the mixed workspace exists: tensor maps of the
// fixed slice buffers (the low-rank Y slices use a fixed K extent of rcap
// columns, of which a build uses its rank's share), the exchange partial
// sums, the kernels' shared memory.
int ozaki_setup_tc(Plan *P)
{
    Workspace &w = P->ws;
    w.tc = false;
    const int npad = w.npad, n = P->nbf, S = w.oz_slices;
    const long long big_rows = 2LL * w.gc * S * npad;
    if (!slice_map(&w.tm_Ms, w.Ms, big_rows, npad) || !slice_map(&w.tm_Zd, w.Zs, big_rows, npad) ||
        !slice_map(&w.tm_Ds, w.Ds, (long long)S * npad, npad) || !slice_map(&w.tm_Cs, w.Cs, (long long)S * npad, npad) ||
        (w.lr.rcap > 0 && !slice_map(&w.tm_Zl, w.Zs, big_rows, w.lr.rcap)))
        return fail(JK_ERR_CUDA, "cuTensorMapEncodeTiled failed for the exchange slice buffers");
    const int nt = npad / TC_BM, ntri = nt * (nt + 1) / 2;
    w.kpart_splits = std::max(1, std::min(32, (4 * 152 + ntri / 2) / ntri));
    const size_t bytes = (size_t)w.kpart_splits * n * n * sizeof(double);
    if (cudaMalloc((void **)&w.Kpart, bytes) != cudaSuccess) return fail(JK_ERR_OOM, "cudaMalloc failed for exchange partial sums");
    w.bytes += bytes;
    if (cudaFuncSetAttribute(k_ozaki_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(k_ozaki_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM) != cudaSuccess)
        return fail(JK_ERR_CUDA, "cudaFuncSetAttribute failed for the tensor-core GEMM");
    w.tc = true;
    return JK_OK;
}

static void launch_tc(int mode, const CUtensorMap &A, const CUtensorMap &B, const TcArgs &a, dim3 grid, cudaStream_t st)
{
    if (mode == 0) k_ozaki_tc<0><<<grid, TC_THREADS, TC_SMEM, st>>>(A, B, a);
    else k_ozaki_tc<1><<<grid, TC_THREADS, TC_SMEM, st>>>(A, B, a);
}

// End of the reciprocal exchange: fold the per-split partial sums into K_LR.
int ozaki_finish(Plan *P, cudaStream_t st)
{
    Workspace &w = P->ws;
    if (!w.tc) return JK_OK;
    const int n = P->nbf;
    k_kpart_reduce<<<152 * 8, 256, 0, st>>>(n, n, w.kpart_splits, (long long)n * n, w.Kpart, w.KLR);
    return check("exchange partial-sum reduction");
}

// Start of a build (mixed precision): slices of D' for the dense form, the
// pivoted LDL^T of D' on the device (rank and form in w.lr.dyn) and the
// slices of its packed factor rows.  Nothing here waits for the device.
int ozaki_begin(Plan *P, cudaStream_t st)
{
    Workspace &w = P->ws;
    const int n = P->nbf;
    w.chunk_log.clear();
    slice(w.Dp, n, n, n, 0, w.npad, w.npad, w.oz_slices, 1, w.Ds, w.Dex, st);
    cudaMemsetAsync(w.Kpart, 0, (size_t)w.kpart_splits * n * n * sizeof(double), st);
    int rc = lowrank_factor(w.Dp, n, w.lr.rcap, 1e-12, w.lr, w.err, st);
    if (rc) return rc;
    if (w.lr.rcap > 0) slice(w.lr.Ct, w.lr.rcap, n, n, 0, w.lr.rcap, w.npad, w.oz_slices, 1, w.Cs, w.Cex, st);
    return check("density slices and low-rank factor");
}

// K_LR += sum_b M_b D M_b for the m2 slabs of one G chunk, with S slices
// per operand (the density or low-rank factor slices, cut once with
// oz_slices, are used through their first S slices: a balanced-digit
// expansion truncated after S digits).  Both forms are enqueued; the
// kernels of the form the factorisation did not choose return at once.
int ozaki_exchange_chunk(Plan *P, int chunk, const double *Mc, int m2, int S, cudaStream_t st)
{
    Workspace &w = P->ws;
    const int n = P->nbf, npad = w.npad;
    if (S < 1 || S > w.oz_slices) return fail(JK_ERR_INVALID, "slice count outside 1..oz_slices");
    const int nt = npad / TC_BM, ntri = nt * (nt + 1) / 2;
    PhaseTimer &tm = P->timer;
    w.chunk_log.push_back({m2, S});
    const int *dyn = w.lr.dyn;
    // the slab's slices: in the chunk buffer, or in the reciprocal cache
    // (cut once, by the build that fills it)
    RecipCache &cc = P->cache;
    const bool cached = cc.on && cc.Ms;
    __nv_bfloat16 *Ms = cached ? cc.Ms + (size_t)cc.row0[chunk] * npad : w.Ms;
    int *Mex = cached ? cc.Mex + cc.ex0[chunk] : w.Mex;
    const CUtensorMap &tmM = cached ? cc.tm_Ms : w.tm_Ms;
    const int mrow0 = cached ? (int)cc.row0[chunk] : 0;
    int ev = tm.start(8);
    if (!cached || !cc.s_valid) slice(Mc, n, n, n, (long long)n * n, npad, npad, S, m2, Ms, Mex, st);
    tm.stop(8, ev, 1);
    {
        // dense form: Zt_b = (D M_b)^T, as (hi, lo) pairs ...
        TcArgs t{};
        t.a_batch_rows = 0; t.a_slice_rows = npad; t.b_batch_rows = S * npad; t.b_slice_rows = npad;
        t.Aex = w.Dex; t.a_exb = 0; t.Bex = Mex; t.b_exb = npad; t.b_row0 = mrow0;
        t.koff = 0; t.klen = npad; t.S = S; t.nb = m2; t.ntm = nt; t.ntn = nt;
        t.out = reinterpret_cast<float2 *>(w.Z); t.out_rows = n; t.out_cols = n; t.o_bstride = (long long)n * n; t.ldo = n;
        t.transpose = 1; t.err = w.err; t.bsplit = tc_splits(nt * nt, m2);
        t.dyn = dyn; t.dyn_mode = 1;
        ev = tm.start(7);
        launch_tc(0, w.tm_Ds, tmM, t, dim3(nt * nt, 1, t.bsplit), st);
        tm.stop(7, ev, 1);
        ev = tm.start(8);
        slice_pair(reinterpret_cast<const float2 *>(w.Z), n, n, n, (long long)n * n, npad, npad, S, m2, w.Zs, w.Zex, dyn, 1, st);
        tm.stop(8, ev, 1);
        // ... then K += sum_b M_b Z_b, upper tiles into the float-pair partials
        TcArgs k{};
        k.a_batch_rows = S * npad; k.a_slice_rows = npad; k.b_batch_rows = S * npad; k.b_slice_rows = npad;
        k.Aex = Mex; k.a_exb = npad; k.Bex = w.Zex; k.b_exb = npad; k.a_row0 = mrow0;
        k.koff = 0; k.klen = npad; k.S = S; k.nb = m2; k.bsplit = std::min(w.kpart_splits, m2); k.ntm = nt; k.ntn = nt;
        k.part = w.Kpart; k.part_stride = (long long)n * n; k.ldp = n; k.out_rows = n; k.out_cols = n; k.sign = 1.f;
        k.err = w.err; k.dyn = dyn; k.dyn_mode = 1;
        ev = tm.start(7);
        launch_tc(1, tmM, w.tm_Zd, k, dim3(ntri, 1, k.bsplit), st);
        tm.stop(7, ev, 1);
    }
    const int rcap = w.lr.rcap;
    if (rcap > 0) {
        // low-rank form: Y_b = M_b [C+ C-]  (n x rcap, row-major, (hi, lo) pairs; live columns up to the rank)
        TcArgs y{};
        y.a_batch_rows = S * npad; y.a_slice_rows = npad; y.b_batch_rows = 0; y.b_slice_rows = rcap;
        y.Aex = Mex; y.a_exb = npad; y.Bex = w.Cex; y.b_exb = 0; y.a_row0 = mrow0;
        y.koff = 0; y.klen = npad; y.S = S; y.nb = m2; y.ntm = nt; y.ntn = rcap / TC_BN;
        y.out = reinterpret_cast<float2 *>(w.Z); y.out_rows = n; y.out_cols = rcap; y.o_bstride = (long long)n * rcap; y.ldo = rcap;
        y.transpose = 0; y.err = w.err; y.bsplit = tc_splits(nt * (rcap / TC_BN), m2);
        y.dyn = dyn; y.dyn_mode = 2;
        ev = tm.start(7);
        launch_tc(0, tmM, w.tm_Cs, y, dim3(nt * (rcap / TC_BN), 1, y.bsplit), st);
        tm.stop(7, ev, 1);
        ev = tm.start(8);
        slice_pair(reinterpret_cast<const float2 *>(w.Z), n, rcap, rcap, (long long)n * rcap, npad, rcap, S, m2, w.Zs, w.Zex, dyn, 2, st);
        tm.stop(8, ev, 1);
        // K += sum_b Y+_b Y+_b^T - Y-_b Y-_b^T  (symmetric, K range per group)
        for (int grp = 0; grp < 2; ++grp) {
            TcArgs k{};
            k.a_batch_rows = S * npad; k.a_slice_rows = npad; k.b_batch_rows = S * npad; k.b_slice_rows = npad;
            k.Aex = w.Zex; k.a_exb = npad; k.Bex = w.Zex; k.b_exb = npad;
            k.koff = 0; k.klen = 0; k.S = S; k.nb = m2; k.bsplit = std::min(w.kpart_splits, m2); k.ntm = nt;
            k.ntn = nt;
            k.part = w.Kpart; k.part_stride = (long long)n * n; k.ldp = n; k.out_rows = n; k.out_cols = n;
            k.sign = grp == 0 ? 1.f : -1.f;
            k.err = w.err; k.dyn = dyn; k.dyn_mode = grp == 0 ? 3 : 4;
            ev = tm.start(7);
            launch_tc(1, w.tm_Zl, w.tm_Zl, k, dim3(ntri, 1, k.bsplit), st);
            tm.stop(7, ev, 1);
        }
    }
    return check("split-precision exchange GEMM");
}

// Reciprocal cache: every chunk's structure-factor slab (FP64) and, for
// mixed plans, its slices and row exponents, if the total fits max_bytes.
// The caller holds the plan's lock and has waited for its last build.
void release_cache(Plan *P)
{
    RecipCache &c = P->cache;
    if (c.M) cudaFree(c.M);
    if (c.Ms) cudaFree(c.Ms);
    if (c.Mex) cudaFree(c.Mex);
    c = RecipCache{};
}

int cache_reciprocal(Plan *P, size_t max_bytes)
{
    release_cache(P);
    if (max_bytes == 0) return JK_OK;
    Workspace &w = P->ws;
    const int ng = (int)(P->gvec.size() / 4);
    const size_t n2 = (size_t)P->nbf * P->nbf;
    RecipCache &c = P->cache;
    // mixed plans keep the structure factors as packed upper triangles
    const size_t npk = (size_t)P->nbf * (P->nbf + 1) / 2;
    size_t bM = 2 * (size_t)ng * (P->precision == JK_MIXED ? npk : n2) * sizeof(double), bS = 0, bX = 0;
    long long rows = 0, ex = 0;
    const bool mixed = P->precision == JK_MIXED;
    if (mixed) {
        for (int g0 = 0, ch = 0; g0 < ng; g0 += w.gc, ++ch) {
            const int m2 = 2 * std::min(w.gc, ng - g0), S = w.chunk_slices[ch];
            c.row0.push_back(rows);
            c.ex0.push_back(ex);
            rows += (long long)m2 * S * w.npad;
            ex += (long long)m2 * w.npad;
        }
        bS = (size_t)rows * w.npad * sizeof(__nv_bfloat16);
        bX = (size_t)ex * sizeof(int);
        if (rows >= (1LL << 31)) {
            c = RecipCache{};
            return fail(JK_ERR_OOM, "reciprocal cache: too many slice rows for one tensor map");
        }
    }
    const size_t need = bM + bS + bX;
    if (need > max_bytes) {
        c = RecipCache{};
        return fail(JK_ERR_OOM, "reciprocal cache needs " + std::to_string(need) + " bytes, above the limit given");
    }
    if (cudaMalloc((void **)&c.M, bM) != cudaSuccess || (mixed && cudaMalloc((void **)&c.Ms, bS) != cudaSuccess) ||
        (mixed && cudaMalloc((void **)&c.Mex, bX) != cudaSuccess)) {
        cudaGetLastError();
        release_cache(P);
        return fail(JK_ERR_OOM, "cudaMalloc failed for the reciprocal cache");
    }
    // entries of shell pairs without images are never written
    if (cudaMemset(c.M, 0, bM) != cudaSuccess) {
        release_cache(P);
        return fail(JK_ERR_CUDA, "cudaMemset failed for the reciprocal cache");
    }
    if (mixed && !slice_map(&c.tm_Ms, c.Ms, rows, w.npad)) {
        release_cache(P);
        return fail(JK_ERR_CUDA, "cuTensorMapEncodeTiled failed for the reciprocal cache");
    }
    c.on = true;
    c.bytes = need;
    return JK_OK;
}

// BF16 MMA flops the exchange GEMMs of the last build issued, from its chunk
// log and the form and rank the device chose (dyn read back after the build).
double ozaki_mma_flops(const Plan *P, const int dyn[3])
{
    const Workspace &w = P->ws;
    const int npad = w.npad, nt = npad / TC_BM, ntri = nt * (nt + 1) / 2;
    double f = 0;
    for (auto &c : w.chunk_log) {
        const int m2 = c.first, S = c.second;
        const double prods = S * (S + 1) / 2.0;
        if (!dyn[0]) {
            f += prods * 2.0 * npad * (double)npad * npad * m2;
            f += prods * 2.0 * TC_BM * (double)TC_BN * npad * ntri * m2;
        } else {
            f += prods * 2.0 * npad * (double)(dyn[1] + dyn[2]) * npad * m2;
            f += prods * 2.0 * TC_BM * (double)TC_BN * (dyn[1] + dyn[2]) * ntri * m2;
        }
    }
    return f;
}

}  // namespace jk
