// Split-precision GEMMs on the BF16 tensor cores for the reciprocal
// exchange contraction K_LR = sum_b M_b D M_b (b runs over the real and
// imaginary parts of the structure-factor slab of each G).
//
// Each FP64 operand row r is scaled by 2^{-sigma_r} (sigma_r from the
// largest exponent in the row) and cut into S slices of 7-bit digits,
// x = sign(x) 2^{sigma_r} sum_s d_s 2^{-7(s+1)}, d_s in [0, 127] (exact in
// BF16).  The digits are read straight from the IEEE bit pattern (integer
// shifts), so slicing costs no FP64 arithmetic.  A slice product over K <=
// 1024 terms sums integers below 2^14, so it is exact in the FP32
// accumulator of the tensor-core MMA; the products with s + t <= S - 1
// (0-based) are combined with their power-of-two scales in a compensated
// single-precision pair.  This is the error-free splitting of Ozaki, Ogita,
// Oishi and Rump (Numer. Algorithms 59, 2012) with digits sized to the FP32
// accumulator.
//
// Two factorisations of the contraction:
//   dense:    Zt_b = (D M_b)^T, then K += sum_b M_b Z_b;
//   low rank: D = C+ C+^T - C- C-^T from the eigenvalues of D kept above a
//             relative 1e-10 (a closed-shell SCF density has rank n_occ), then
//             Y_b = M_b [C+ C-] and K += sum_b Y+_b Y+_b^T - Y-_b Y-_b^T.
// M_b is symmetric, so its row slices serve as the A operand of one GEMM
// and the B operand (B^T rows) of the other; the K GEMMs form only tiles on
// or above the diagonal and mirror them.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cusolverDn.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "plan.h"

namespace jk {

namespace {

constexpr int BM = 128, BN = 128, BK = 32, LDS = BK + 8;  // smem row stride in bf16
constexpr int KFLUSH = 1024;                               // exactness bound of the FP32 accumulator

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void mma_bf16(float *c, const uint32_t *a, const uint32_t *b)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

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
// F = floor(|x| 2^{64 - sigma}) is formed by shifting the 53-bit significand,
// and digit s is bits [63 - 7s, 57 - 7s] of F.  Output:
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
    for (int k = lane; k < cols_pad; k += 32) {
        unsigned long long F = 0;
        bool neg = false;
        if (r < rows && k < cols) {
            const unsigned long long bits = row[k];
            const int E = (int)((bits >> 52) & 0x7ff);
            if (E > 0) {  // subnormals flush to zero
                const unsigned long long M = (bits & 0xfffffffffffffull) | (1ull << 52);
                const int sh = E - 1011 - sigma;  // <= 11
                F = sh >= 0 ? (M << sh) : (sh > -64 ? (M >> (-sh)) : 0ull);
                neg = (bits >> 63) != 0;
            }
        }
        for (int s = 0; s < S; ++s) {
            const int d = (int)((F >> (57 - 7 * s)) & 127ull);
            o[s * sstride + k] = __float2bfloat16_rn((float)(neg ? -d : d));
        }
    }
}

struct GemmArgs {
    const __nv_bfloat16 *A;
    const int *Aex;
    long long a_bstride;  // elements between batches (0: shared operand)
    int a_exb;            // exponents between batches
    int a_rows_pad;       // rows per slice block
    const __nv_bfloat16 *B;
    const int *Bex;
    long long b_bstride;
    int b_exb;
    int b_rows_pad;
    int kpad;             // row length (K stride) of both operands
    int koff, klen;       // K range used
    int S, nb, bsplit, ntm, ntn;
    double *out;
    int out_rows, out_cols;
    long long o_bstride;
    int ldo, transpose;
    float sign;
};

// MODE 0: blockIdx.z = b; out_b = A_b B_b (A may be shared), written as FP64
// (transposed if requested).  MODE 1: blockIdx.z = split index over b;
// out += sign sum_b A_b B_b over upper tiles (ntm == ntn), FP64 atomics,
// mirrored below the diagonal.
template <int MODE>
__global__ void __launch_bounds__(256, 1) k_ozaki_gemm(GemmArgs g)
{
    __shared__ __align__(16) __nv_bfloat16 sA[2][BM * LDS];
    __shared__ __align__(16) __nv_bfloat16 sB[2][BN * LDS];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gi = lane >> 2, tig = lane & 3;
    const int wm = warp >> 2, wn = warp & 3;
    int mi, nj, b0, b1;
    if (MODE == 0) {
        mi = blockIdx.x % g.ntm;
        nj = blockIdx.x / g.ntm;
        b0 = blockIdx.z;
        b1 = b0 + 1;
    } else {
        int t = blockIdx.x;
        mi = 0;
        while (t >= g.ntm - mi) {
            t -= g.ntm - mi;
            ++mi;
        }
        nj = mi + t;
        const int per = (g.nb + g.bsplit - 1) / g.bsplit;
        b0 = blockIdx.z * per;
        b1 = min(g.nb, b0 + per);
    }
    const int row0 = mi * BM, col0 = nj * BN;
    float hi[4][4][4], lo[4][4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int e = 0; e < 4; ++e) hi[a][c][e] = lo[a][c][e] = 0.f;

    for (int b = b0; b < b1; ++b) {
        const __nv_bfloat16 *Ab = g.A + (size_t)b * g.a_bstride;
        const int *Aeb = g.Aex + (size_t)(g.a_bstride ? b : 0) * g.a_exb;
        const __nv_bfloat16 *Bb = g.B + (size_t)b * g.b_bstride;
        const int *Beb = g.Bex + (size_t)(g.b_bstride ? b : 0) * g.b_exb;
        int rex[4][2], cex[4][2];
#pragma unroll
        for (int mt = 0; mt < 4; ++mt) {
            rex[mt][0] = Aeb[row0 + wm * 64 + mt * 16 + gi];
            rex[mt][1] = Aeb[row0 + wm * 64 + mt * 16 + gi + 8];
        }
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            cex[nt][0] = Beb[col0 + wn * 32 + nt * 8 + 2 * tig];
            cex[nt][1] = Beb[col0 + wn * 32 + nt * 8 + 2 * tig + 1];
        }
        for (int s = 0; s < g.S; ++s)
            for (int t = 0; s + t < g.S; ++t) {
                const __nv_bfloat16 *A = Ab + ((size_t)s * g.a_rows_pad + row0) * g.kpad;
                const __nv_bfloat16 *Bt = Bb + ((size_t)t * g.b_rows_pad + col0) * g.kpad;
                for (int kc = g.koff; kc < g.koff + g.klen; kc += KFLUSH) {
                    const int kend = min(g.koff + g.klen, kc + KFLUSH);
                    float acc[4][4][4];
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int c = 0; c < 4; ++c)
#pragma unroll
                            for (int e = 0; e < 4; ++e) acc[a][c][e] = 0.f;
                    auto load_stage = [&](int buf, int k0) {
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
                            const int chunk = tid + q * 256;
                            const int r = chunk >> 2, c8 = (chunk & 3) * 8;
                            cp_async16(&sA[buf][r * LDS + c8], A + (size_t)r * g.kpad + k0 + c8);
                            cp_async16(&sB[buf][r * LDS + c8], Bt + (size_t)r * g.kpad + k0 + c8);
                        }
                        cp_async_commit();
                    };
                    load_stage(0, kc);
                    const int nk = (kend - kc) / BK;
                    for (int kt = 0; kt < nk; ++kt) {
                        if (kt + 1 < nk) {
                            load_stage((kt + 1) & 1, kc + (kt + 1) * BK);
                            cp_async_wait<1>();
                        } else {
                            cp_async_wait<0>();
                        }
                        __syncthreads();
                        const __nv_bfloat16 *a_s = sA[kt & 1], *b_s = sB[kt & 1];
#pragma unroll
                        for (int kk = 0; kk < BK; kk += 16) {
                            uint32_t af[4][4], bf[4][2];
#pragma unroll
                            for (int mt = 0; mt < 4; ++mt) {
                                const int r = wm * 64 + mt * 16 + gi;
                                af[mt][0] = *reinterpret_cast<const uint32_t *>(&a_s[r * LDS + kk + 2 * tig]);
                                af[mt][1] = *reinterpret_cast<const uint32_t *>(&a_s[(r + 8) * LDS + kk + 2 * tig]);
                                af[mt][2] = *reinterpret_cast<const uint32_t *>(&a_s[r * LDS + kk + 8 + 2 * tig]);
                                af[mt][3] = *reinterpret_cast<const uint32_t *>(&a_s[(r + 8) * LDS + kk + 8 + 2 * tig]);
                            }
#pragma unroll
                            for (int nt = 0; nt < 4; ++nt) {
                                const int c = wn * 32 + nt * 8 + gi;
                                bf[nt][0] = *reinterpret_cast<const uint32_t *>(&b_s[c * LDS + kk + 2 * tig]);
                                bf[nt][1] = *reinterpret_cast<const uint32_t *>(&b_s[c * LDS + kk + 8 + 2 * tig]);
                            }
#pragma unroll
                            for (int mt = 0; mt < 4; ++mt)
#pragma unroll
                                for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[mt][nt], af[mt], bf[nt]);
                        }
                        __syncthreads();
                    }
#pragma unroll
                    for (int mt = 0; mt < 4; ++mt)
#pragma unroll
                        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const int sh = rex[mt][e >> 1] + cex[nt][e & 1] - 7 * (s + t + 2);
                                two_sum_add(hi[mt][nt][e], lo[mt][nt][e], ldexpf(acc[mt][nt][e], sh));
                            }
                }
            }
        if (MODE == 0) {
            double *O = g.out + (size_t)b * g.o_bstride;
#pragma unroll
            for (int mt = 0; mt < 4; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int i = row0 + wm * 64 + mt * 16 + gi + (e >> 1) * 8;
                        const int j = col0 + wn * 32 + nt * 8 + 2 * tig + (e & 1);
                        if (i < g.out_rows && j < g.out_cols)
                            O[g.transpose ? (size_t)j * g.ldo + i : (size_t)i * g.ldo + j] =
                                (double)hi[mt][nt][e] + (double)lo[mt][nt][e];
                        hi[mt][nt][e] = lo[mt][nt][e] = 0.f;
                    }
        }
    }
    if (MODE == 1) {
#pragma unroll
        for (int mt = 0; mt < 4; ++mt)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int i = row0 + wm * 64 + mt * 16 + gi + (e >> 1) * 8;
                    const int j = col0 + wn * 32 + nt * 8 + 2 * tig + (e & 1);
                    const double v = (double)g.sign * ((double)hi[mt][nt][e] + (double)lo[mt][nt][e]);
                    if (i < g.out_rows && j < g.out_cols && v != 0.0) {
                        atomicAdd(g.out + (size_t)i * g.ldo + j, v);
                        if (mi != nj) atomicAdd(g.out + (size_t)j * g.ldo + i, v);
                    }
                }
    }
}

// C^T of the low-rank factor: row k' of Ct is eigenvector idx[k'] times
// sqrt|lambda|; rows beyond r are zero.  V column-major (column = vector).
__global__ void k_lowrank_factor(int n, const double *__restrict__ V, const double *__restrict__ W, const int *__restrict__ idx, int r,
                                 int rpad, double *__restrict__ Ct)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)rpad * n) return;
    const int kr = (int)(e / n), i = (int)(e % n);
    double v = 0.0;
    if (kr < r) {
        const int j = idx[kr];
        v = V[(size_t)j * n + i] * sqrt(fabs(W[j]));
    }
    Ct[e] = v;
}

static unsigned blocks_for_rows(long long rows) { return (unsigned)((rows * 32 + 255) / 256); }

static void slice(const double *X, int rows, int cols, int ld, long long bstride, int rows_pad, int cols_pad, int S, int B,
                  __nv_bfloat16 *out, int *ex, cudaStream_t st)
{
    k_ozaki_slice<<<blocks_for_rows((long long)B * rows_pad), 256, 0, st>>>(X, rows, cols, ld, bstride, rows_pad, cols_pad, S, B, out, ex);
}

static int check(const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(JK_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return JK_OK;
}

// Start of a build (mixed precision): slices of D' for the dense form and,
// when the plan has a solver, the eigendecomposition of D' whose eigenvalues
// are copied to pinned host memory (read back later by ozaki_prepare_lowrank,
// after the real-space kernels, so the copy never stalls the stream).
int ozaki_begin(Plan *P, cudaStream_t st)
{
    Workspace &w = P->ws;
    const int n = P->nbf;
    slice(w.Dp, n, n, n, 0, w.npad, w.npad, w.oz_slices, 1, w.Ds, w.Dex, st);
    w.lowrank = false;
    if (!w.solver) return check("density slices");
    if (cusolverDnSetStream(w.solver, st) != CUSOLVER_STATUS_SUCCESS) return fail(JK_ERR_CUDA, "cusolverDnSetStream failed");
    cudaMemcpyAsync(w.eigV, w.Dp, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, st);
    if (cusolverDnDsyevd(w.solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, w.eigV, n, w.eigW, w.eigWork, w.eigLwork,
                         w.eigInfo) != CUSOLVER_STATUS_SUCCESS)
        return fail(JK_ERR_CUDA, "cusolverDnDsyevd failed");
    cudaMemcpyAsync(w.eigW_host, w.eigW, sizeof(double) * n, cudaMemcpyDeviceToHost, st);
    cudaEventRecord(w.eig_done, st);
    return check("eigendecomposition of D");
}

// After the real-space phase: decide between the dense and the low-rank form
// from the eigenvalues and, for low rank, form C^T and its slices.
int ozaki_prepare_lowrank(Plan *P, cudaStream_t st)
{
    Workspace &w = P->ws;
    w.lowrank = false;
    if (!w.solver) return JK_OK;
    if (cudaEventSynchronize(w.eig_done) != cudaSuccess) return fail(JK_ERR_CUDA, "eigendecomposition failed");
    const int n = P->nbf;
    double wmax = 0;
    for (int i = 0; i < n; ++i) wmax = std::max(wmax, std::fabs(w.eigW_host[i]));
    std::vector<int> pos, neg;
    for (int i = n - 1; i >= 0; --i)
        if (w.eigW_host[i] > 1e-10 * wmax) pos.push_back(i);
    for (int i = 0; i < n; ++i)
        if (w.eigW_host[i] < -1e-10 * wmax) neg.push_back(i);
    const int rp = ((int)pos.size() + BN - 1) / BN * BN, rn = ((int)neg.size() + BN - 1) / BN * BN;
    if (wmax == 0 || rp + rn > (6 * w.npad) / 10) return JK_OK;  // not worth it: dense form
    std::vector<int> idx(rp + rn, 0);
    for (size_t k = 0; k < pos.size(); ++k) idx[k] = pos[k];
    for (size_t k = 0; k < neg.size(); ++k) idx[rp + k] = neg[k];
    cudaMemcpyAsync(w.eigIdx, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice, st);
    // the two column groups share one C^T buffer: rows [0, rp) and [rp, rp + rn)
    const long long e1 = (long long)rp * n, e2 = (long long)rn * n;
    if (rp) k_lowrank_factor<<<(unsigned)((e1 + 255) / 256), 256, 0, st>>>(n, w.eigV, w.eigW, w.eigIdx, (int)pos.size(), rp, w.Ct);
    if (rn)
        k_lowrank_factor<<<(unsigned)((e2 + 255) / 256), 256, 0, st>>>(n, w.eigV, w.eigW, w.eigIdx + rp, (int)neg.size(), rn, w.Ct + e1);
    slice(w.Ct, rp + rn, n, n, 0, rp + rn, w.npad, w.oz_slices, 1, w.Cs, w.Cex, st);
    cudaStreamSynchronize(st);  // idx is a host vector that must outlive the copy
    w.lowrank = true;
    w.rpos = rp;
    w.rneg = rn;
    return check("low-rank factor");
}

// K_LR += sum_b M_b D M_b for the m2 slabs of one G chunk.
int ozaki_exchange_chunk(Plan *P, int m2, cudaStream_t st)
{
    Workspace &w = P->ws;
    const int n = P->nbf, npad = w.npad, S = w.oz_slices;
    const int nt = npad / BM;
    PhaseTimer &tm = P->timer;
    const double prods = S * (S + 1) / 2.0;
    int ev = tm.start(8);
    slice(w.M, n, n, n, (long long)n * n, npad, npad, S, m2, w.Ms, w.Mex, st);
    tm.stop(8, ev, 1);
    const long long ms_b = (long long)S * npad * npad;
    if (!w.lowrank) {
        // Zt_b = (D M_b)^T
        GemmArgs z{};
        z.A = w.Ds; z.Aex = w.Dex; z.a_bstride = 0; z.a_exb = 0; z.a_rows_pad = npad;
        z.B = w.Ms; z.Bex = w.Mex; z.b_bstride = ms_b; z.b_exb = npad; z.b_rows_pad = npad;
        z.kpad = npad; z.koff = 0; z.klen = npad; z.S = S; z.nb = m2; z.bsplit = 1; z.ntm = nt; z.ntn = nt;
        z.out = w.Z; z.out_rows = n; z.out_cols = n; z.o_bstride = (long long)n * n; z.ldo = n; z.transpose = 1; z.sign = 1.f;
        ev = tm.start(7);
        k_ozaki_gemm<0><<<dim3(nt * nt, 1, m2), 256, 0, st>>>(z);
        tm.stop(7, ev, 1);
        w.mma_flops += prods * 2.0 * npad * (double)npad * npad * m2;
        ev = tm.start(8);
        slice(w.Z, n, n, n, (long long)n * n, npad, npad, S, m2, w.Zs, w.Zex, st);
        tm.stop(8, ev, 1);
        // K += sum_b M_b Z_b
        GemmArgs k{};
        k.A = w.Ms; k.Aex = w.Mex; k.a_bstride = ms_b; k.a_exb = npad; k.a_rows_pad = npad;
        k.B = w.Zs; k.Bex = w.Zex; k.b_bstride = ms_b; k.b_exb = npad; k.b_rows_pad = npad;
        k.kpad = npad; k.koff = 0; k.klen = npad; k.S = S; k.nb = m2; k.ntm = nt; k.ntn = nt;
        const int ntri = nt * (nt + 1) / 2;
        k.bsplit = std::max(1, std::min((152 * 2 + ntri - 1) / ntri, m2));
        k.out = w.KLR; k.out_rows = n; k.out_cols = n; k.ldo = n; k.sign = 1.f;
        ev = tm.start(7);
        k_ozaki_gemm<1><<<dim3(ntri, 1, k.bsplit), 256, 0, st>>>(k);
        tm.stop(7, ev, 1);
        w.mma_flops += prods * 2.0 * BM * (double)BN * npad * ntri * m2;
        return check("split-precision exchange GEMM (dense)");
    }
    const int rt = w.rpos + w.rneg;
    // Y_b = M_b [C+ C-]  (n x rt, row-major)
    GemmArgs y{};
    y.A = w.Ms; y.Aex = w.Mex; y.a_bstride = ms_b; y.a_exb = npad; y.a_rows_pad = npad;
    y.B = w.Cs; y.Bex = w.Cex; y.b_bstride = 0; y.b_exb = 0; y.b_rows_pad = rt;
    y.kpad = npad; y.koff = 0; y.klen = npad; y.S = S; y.nb = m2; y.bsplit = 1; y.ntm = nt; y.ntn = rt / BN;
    y.out = w.Z; y.out_rows = n; y.out_cols = rt; y.o_bstride = (long long)n * rt; y.ldo = rt; y.transpose = 0; y.sign = 1.f;
    ev = tm.start(7);
    k_ozaki_gemm<0><<<dim3(nt * (rt / BN), 1, m2), 256, 0, st>>>(y);
    tm.stop(7, ev, 1);
    w.mma_flops += prods * 2.0 * npad * (double)rt * npad * m2;
    ev = tm.start(8);
    slice(w.Z, n, rt, rt, (long long)n * rt, npad, rt, S, m2, w.Zs, w.Zex, st);
    tm.stop(8, ev, 1);
    // K += sum_b Y+_b Y+_b^T - Y-_b Y-_b^T  (symmetric, K range per group)
    const long long ys_b = (long long)S * npad * rt;
    const int ntri = nt * (nt + 1) / 2;
    for (int grp = 0; grp < 2; ++grp) {
        const int klen = grp == 0 ? w.rpos : w.rneg;
        if (!klen) continue;
        GemmArgs k{};
        k.A = w.Zs; k.Aex = w.Zex; k.a_bstride = ys_b; k.a_exb = npad; k.a_rows_pad = npad;
        k.B = w.Zs; k.Bex = w.Zex; k.b_bstride = ys_b; k.b_exb = npad; k.b_rows_pad = npad;
        k.kpad = rt; k.koff = grp == 0 ? 0 : w.rpos; k.klen = klen; k.S = S; k.nb = m2; k.ntm = nt; k.ntn = nt;
        k.bsplit = std::max(1, std::min((152 * 2 + ntri - 1) / ntri, m2));
        k.out = w.KLR; k.out_rows = n; k.out_cols = n; k.ldo = n; k.sign = grp == 0 ? 1.f : -1.f;
        ev = tm.start(7);
        k_ozaki_gemm<1><<<dim3(ntri, 1, k.bsplit), 256, 0, st>>>(k);
        tm.stop(7, ev, 1);
        w.mma_flops += prods * 2.0 * BM * (double)BN * klen * ntri * m2;
    }
    return check("split-precision exchange GEMM (low rank)");
}

}  // namespace jk
