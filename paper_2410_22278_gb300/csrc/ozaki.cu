// Split-precision GEMMs on the BF16 tensor cores for the reciprocal
// exchange contraction K_LR = sum_b M_b D M_b (b runs over the real and
// imaginary parts of the structure-factor slab of each G).
//
// Each FP64 operand row r is scaled by 2^{-sigma_r} (sigma_r the exponent
// of the row's largest magnitude) and cut into S slices of 7-bit signed
// integers, x = 2^{sigma_r} sum_s d_s 2^{-7 s}, d_s in [-128, 128] (exact in
// BF16).  A slice product d_s^A . d_t^B over K <= 1024 terms is a sum of
// integers below 2^14 each, so it is exact in the FP32 accumulator of the
// tensor-core MMA; the products with s + t <= S + 1 are then combined with
// their power-of-two scales in a compensated single-precision pair (about
// 48 bits).  This is the error-free splitting of Ozaki, Ogita, Oishi and Rump
// (Numer. Algorithms 59, 2012), here with 7-bit slices sized to the FP32
// accumulator.
//
// Operand layouts (all row-major, K contiguous, rows padded to npad):
//   GEMM "Z":  Zt_b = (D M_b)^T, A = slices of D, B^T = slices of M_b (M_b is
//              symmetric, so its rows are the columns B needs);
//   GEMM "K":  K += sum_b M_b Z_b with A = slices of M_b and B^T = slices of
//              Zt_b; only tiles on or above the diagonal are formed (the sum
//              is symmetric) and mirrored on output.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

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

// compensated accumulation hi + lo += x
__device__ __forceinline__ void two_sum_add(float &hi, float &lo, float x)
{
    const float t = hi + x;
    const float bp = t - hi;
    lo += (hi - (t - bp)) + (x - bp);
    hi = t;
}

}  // namespace

// Slices of a batch of n x n FP64 matrices (row-major, stride n*n): one
// warp per row; sigma = ilogb(max|x|) + 1; slices written to
// out[((b*S + s)*npad + r)*npad + k] (zero beyond n), exponents to
// ex[b*npad + r] (0 for empty and padding rows).
__global__ void k_ozaki_slice(const double *__restrict__ X, int n, int npad, int S, int B, __nv_bfloat16 *__restrict__ out,
                              int *__restrict__ ex)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const long long rows = (long long)B * npad;
    if (warp >= rows) return;
    const int b = (int)(warp / npad), r = (int)(warp % npad);
    const double *row = X + ((size_t)b * n + r) * n;
    double amax = 0;
    if (r < n)
        for (int k = lane; k < n; k += 32) amax = fmax(amax, fabs(row[k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    const int sigma = amax > 0 ? ilogb(amax) + 1 : 0;
    if (lane == 0) ex[(size_t)b * npad + r] = sigma;
    for (int k = lane; k < npad; k += 32) {
        double v = (r < n && k < n) ? ldexp(row[k], -sigma) : 0.0;
        for (int s = 0; s < S; ++s) {
            v *= 128.0;
            const double d = rint(v);
            v -= d;
            out[(((size_t)b * S + s) * npad + r) * npad + k] = __float2bfloat16_rn((float)d);
        }
    }
}

// MODE 0 ("Z"): blockIdx.z = b; C_b = A B_b with A = slices of one matrix
// (batch stride 0), written transposed as FP64 to Zt[b][j][i].
// MODE 1 ("K"): blockIdx.z = split index over b; C = sum_b A_b B_b
// accumulated with FP64 atomics into Kout[i][j] and Kout[j][i].
template <int MODE>
__global__ void __launch_bounds__(256, 1)
    k_ozaki_gemm(const __nv_bfloat16 *__restrict__ As, const int *__restrict__ Aex, long long a_bstride, int a_exstride,
                 const __nv_bfloat16 *__restrict__ Bs, const int *__restrict__ Bex, int n, int npad, int S, int nb, int bsplit,
                 double *__restrict__ out)
{
    __shared__ __align__(16) __nv_bfloat16 sA[2][BM * LDS];
    __shared__ __align__(16) __nv_bfloat16 sB[2][BN * LDS];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, tig = lane & 3;
    const int wm = warp >> 2, wn = warp & 3;
    const int ntile = npad / BM;
    int mi, nj, b0, b1;
    if (MODE == 0) {
        mi = blockIdx.x % ntile;
        nj = blockIdx.x / ntile;
        b0 = blockIdx.z;
        b1 = b0 + 1;
    } else {
        // upper-triangular tile index -> (mi, nj) with mi <= nj
        int t = blockIdx.x;
        mi = 0;
        while (t >= ntile - mi) {
            t -= ntile - mi;
            ++mi;
        }
        nj = mi + t;
        const int per = (nb + bsplit - 1) / bsplit;
        b0 = blockIdx.z * per;
        b1 = min(nb, b0 + per);
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
        const __nv_bfloat16 *Ab = As + (size_t)(MODE == 0 ? 0 : b) * a_bstride;
        const int *Aeb = Aex + (size_t)(MODE == 0 ? 0 : b) * a_exstride;
        const __nv_bfloat16 *Bb = Bs + (size_t)b * S * (size_t)npad * npad;
        const int *Beb = Bex + (size_t)b * npad;
        // per-thread row and column exponents of the fragments it owns
        int rex[4][2], cex[4][2];
#pragma unroll
        for (int mt = 0; mt < 4; ++mt) {
            rex[mt][0] = Aeb[row0 + wm * 64 + mt * 16 + g];
            rex[mt][1] = Aeb[row0 + wm * 64 + mt * 16 + g + 8];
        }
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            cex[nt][0] = Beb[col0 + wn * 32 + nt * 8 + 2 * tig];
            cex[nt][1] = Beb[col0 + wn * 32 + nt * 8 + 2 * tig + 1];
        }
        for (int s = 0; s < S; ++s)
            for (int t = 0; s + t < S; ++t) {  // s + t <= S + 1 in 1-based slice numbers
                const __nv_bfloat16 *A = Ab + ((size_t)s * npad + row0) * npad;
                const __nv_bfloat16 *Bt = Bb + ((size_t)t * npad + col0) * npad;
                for (int kc = 0; kc < npad; kc += KFLUSH) {
                    const int kend = min(npad, kc + KFLUSH);
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
                            const int chunk = tid + q * 256;  // 512 chunks of 16 B per operand tile
                            const int r = chunk >> 2, c8 = (chunk & 3) * 8;
                            cp_async16(&sA[buf][r * LDS + c8], A + (size_t)r * npad + k0 + c8);
                            cp_async16(&sB[buf][r * LDS + c8], Bt + (size_t)r * npad + k0 + c8);
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
                                const int r = wm * 64 + mt * 16 + g;
                                af[mt][0] = *reinterpret_cast<const uint32_t *>(&a_s[r * LDS + kk + 2 * tig]);
                                af[mt][1] = *reinterpret_cast<const uint32_t *>(&a_s[(r + 8) * LDS + kk + 2 * tig]);
                                af[mt][2] = *reinterpret_cast<const uint32_t *>(&a_s[r * LDS + kk + 8 + 2 * tig]);
                                af[mt][3] = *reinterpret_cast<const uint32_t *>(&a_s[(r + 8) * LDS + kk + 8 + 2 * tig]);
                            }
#pragma unroll
                            for (int nt = 0; nt < 4; ++nt) {
                                const int c = wn * 32 + nt * 8 + g;
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
                    // exact integer sums -> scaled compensated accumulation
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
            double *Zt = out + (size_t)b * n * n;
#pragma unroll
            for (int mt = 0; mt < 4; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int i = row0 + wm * 64 + mt * 16 + g + (e >> 1) * 8;
                        const int j = col0 + wn * 32 + nt * 8 + 2 * tig + (e & 1);
                        if (i < n && j < n) Zt[(size_t)j * n + i] = (double)hi[mt][nt][e] + (double)lo[mt][nt][e];
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
                    const int i = row0 + wm * 64 + mt * 16 + g + (e >> 1) * 8;
                    const int j = col0 + wn * 32 + nt * 8 + 2 * tig + (e & 1);
                    const double v = (double)hi[mt][nt][e] + (double)lo[mt][nt][e];
                    if (i < n && j < n && v != 0.0) {
                        atomicAdd(out + (size_t)i * n + j, v);
                        if (mi != nj) atomicAdd(out + (size_t)j * n + i, v);
                    }
                }
    }
}

// K_LR += sum_b M_b D M_b for the 2*gcur slabs of one G chunk, with the D
// slices (Ds, Dex) prepared once per build.
int ozaki_exchange_chunk(Plan *P, int m2, const __nv_bfloat16 *Ds, const int *Dex, cudaStream_t st)
{
    Workspace &w = P->ws;
    const int n = P->nbf, npad = w.npad, S = w.oz_slices;
    const int ntile = npad / BM;
    // slices of the structure-factor slabs
    {
        const long long rows = (long long)m2 * npad;
        k_ozaki_slice<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, st>>>(w.M, n, npad, S, m2, w.Ms, w.Mex);
    }
    // Zt_b = (D M_b)^T
    {
        dim3 grid(ntile * ntile, 1, m2);
        k_ozaki_gemm<0><<<grid, 256, 0, st>>>(Ds, Dex, 0, 0, w.Ms, w.Mex, n, npad, S, m2, 1, w.Z);
    }
    {
        const long long rows = (long long)m2 * npad;
        k_ozaki_slice<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, st>>>(w.Z, n, npad, S, m2, w.Zs, w.Zex);
    }
    // K_LR += sum_b M_b Z_b (upper tiles, mirrored); split over b to fill the GPU
    {
        const int ntri = ntile * (ntile + 1) / 2;
        int split = (152 * 2 + ntri - 1) / ntri;
        split = std::max(1, std::min(split, m2));
        dim3 grid(ntri, 1, split);
        k_ozaki_gemm<1><<<grid, 256, 0, st>>>(w.Ms, w.Mex, (long long)S * npad * npad, npad, w.Zs, w.Zex, n, npad, S, m2, split, w.KLR);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(JK_ERR_CUDA, std::string("split-precision exchange GEMM: ") + cudaGetErrorString(e));
    return JK_OK;
}

int ozaki_slice_density(Plan *P, cudaStream_t st)
{
    Workspace &w = P->ws;
    const long long rows = w.npad;
    k_ozaki_slice<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, st>>>(w.Dp, P->nbf, w.npad, w.oz_slices, 1, w.Ds, w.Dex);
    return JK_OK;
}

}  // namespace jk
