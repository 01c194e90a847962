// Dense FP64 kernels of the reciprocal-space and background contractions
// (Sections 2.5 and 2.6 of arXiv:2410.22278 with k = 0; Section 3.2 puts the
// reciprocal part on the GPU):
//
//   * the slab passes of the reciprocal Coulomb term: rho_D = M^T vec(D'),
//     then J_LR += M rho_D, where M holds one column per real or imaginary
//     part of a G vector's pair structure factors (k_slab_dot, k_slab_axpy);
//   * a batched FP64 GEMM (k_dgemm) for the background S D' S and the FP64
//     form of the reciprocal exchange K_LR += sum_b M_b D' M_b;
//   * a rank-revealing pivoted LDL^T factorisation of D' on the device
//     (k_ldlt_pivoted), D' ~ sum_j s_j v_j v_j^T with s_j = +-1, which
//     gives the low-rank form of the exchange contraction: a closed-shell
//     SCF density D = 2 C C^T has rank n_occ, so K_LR = sum_b Y+_b Y+_b^T -
//     Y-_b Y-_b^T with Y_b = M_b [C+ C-] costs 3 n^2 r instead of 4 n^3 per
//     slab.  The rank and the choice between the dense and the low-rank
//     form are decided on the device and published in a small status array
//     that the exchange kernels read, so the host never waits for them.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "dense.h"
#include "plan.h"

namespace jk {

// ---------------------------------------------------------------------------
// Reciprocal Coulomb slab passes.  M is [m2][n2] (one structure-factor column
// per row of M here, n2 = n*n contiguous values each).

// rho[b] = sum_i M[b][i] x[i] in two passes: block (s, b) sums the s-th of
// `splits` ranges of i (four independent accumulators per thread, so each
// thread keeps four loads in flight) into part[b * splits + s]; then
// k_slab_dot_final adds the parts in a fixed order (deterministic).
__global__ void __launch_bounds__(256) k_slab_dot(const double *__restrict__ M, long long n2, int m2, const double *__restrict__ x,
                                                  int splits, double *__restrict__ part)
{
    __shared__ double sh[8];
    const int b = blockIdx.y, sidx = blockIdx.x;
    const long long per = (n2 + splits - 1) / splits;
    const long long i0 = sidx * per, i1 = min(n2, i0 + per);
    const double *row = M + (size_t)b * n2;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    long long i = i0 + threadIdx.x;
    for (; i + 3 * 256 < i1; i += 4 * 256) {
        a0 = fma(__ldg(row + i), __ldg(x + i), a0);
        a1 = fma(__ldg(row + i + 256), __ldg(x + i + 256), a1);
        a2 = fma(__ldg(row + i + 512), __ldg(x + i + 512), a2);
        a3 = fma(__ldg(row + i + 768), __ldg(x + i + 768), a3);
    }
    for (; i < i1; i += 256) a0 = fma(__ldg(row + i), __ldg(x + i), a0);
    double s = (a0 + a1) + (a2 + a3);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += sh[w];
        part[(size_t)b * splits + sidx] = t;
    }
}

__global__ void k_slab_dot_final(int m2, int splits, const double *__restrict__ part, double *__restrict__ rho)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= m2) return;
    double t = 0.0;
    for (int k = 0; k < splits; ++k) t += part[(size_t)b * splits + k];
    rho[b] = t;
}

// y[i] += alpha sum_b M[b][i] rho[b]; threads over i (coalesced per b),
// eight independent accumulators (eight loads in flight per thread), rho
// staged through shared memory.
__global__ void __launch_bounds__(256) k_slab_axpy(const double *__restrict__ M, long long n2, int m2, const double *__restrict__ rho,
                                                   double alpha, double *__restrict__ y)
{
    __shared__ double r[1024];
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b0 = 0; b0 < m2; b0 += 1024) {
        const int nb = min(1024, m2 - b0);
        __syncthreads();
        for (int k = threadIdx.x; k < nb; k += blockDim.x) r[k] = rho[b0 + k];
        __syncthreads();
        if (i < n2) {
            const double *col = M + (size_t)b0 * n2 + i;
            int k = 0;
            for (; k + 7 < nb; k += 8) {
#pragma unroll
                for (int u = 0; u < 8; ++u) acc[u] = fma(__ldg(col + (size_t)(k + u) * n2), r[k + u], acc[u]);
            }
            for (; k < nb; ++k) acc[0] = fma(__ldg(col + (size_t)k * n2), r[k], acc[0]);
        }
    }
    if (i < n2) y[i] += alpha * (((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7])));
}

int slab_dot_splits(long long n2, int m2)
{
    // about eight blocks per SM in total (a chunk of one G vector has only two
    // slabs), at least 4096 elements per block
    const long long want = std::max(1LL, (152LL * 8 + m2 - 1) / std::max(1, m2));
    return (int)std::max(1LL, std::min({want, (n2 + 4095) / 4096, (long long)kSlabSplitsMax}));
}

void slab_gemv_t(const double *M, long long n2, int m2, const double *x, double *part, double *rho, cudaStream_t st)
{
    if (m2 <= 0) return;
    const int splits = slab_dot_splits(n2, m2);
    k_slab_dot<<<dim3(splits, m2), 256, 0, st>>>(M, n2, m2, x, splits, part);
    k_slab_dot_final<<<(m2 + 127) / 128, 128, 0, st>>>(m2, splits, part, rho);
}

void slab_gemv_n(const double *M, long long n2, int m2, const double *rho, double alpha, double *y, cudaStream_t st)
{
    if (m2 <= 0 || n2 <= 0) return;
    k_slab_axpy<<<(unsigned)((n2 + 255) / 256), 256, 0, st>>>(M, n2, m2, rho, alpha, y);
}

// ---------------------------------------------------------------------------
// Batched FP64 GEMM, row-major: for batch b,
//   C_b (= or +=) alpha A_b B_b,   A_b: m x k (row stride lda, batch stride sa),
//                                  B_b: k x n (ldb, sb), C_b: m x n (ldc, sc).
// sc = 0 means "batch reduce": every batch adds into the one C with FP64
// atomics, the batch range split over blockIdx.z; otherwise blockIdx.z runs
// over the batches and C_b = alpha A_b B_b + beta C_b.  upper != 0 forms only
// the output tiles on or above the diagonal (symmetric results; the caller
// mirrors them).  64 x 64 tiles, 16-deep K steps through shared memory, 256
// threads with 4 x 4 outputs each (rows ty + 16 i, columns tx + 16 j); the
// kernel is bound by the FP64 pipe, so one such tile keeps it busy.
constexpr int DG_BM = 64, DG_BN = 64, DG_BK = 16;

__global__ void __launch_bounds__(256) k_dgemm(int m, int n, int k, const double *__restrict__ A, long long lda, long long sa,
                                               const double *__restrict__ B, long long ldb, long long sb, double *__restrict__ C,
                                               long long ldc, long long sc, int nbatch, int per, double alpha, double beta, int upper)
{
    __shared__ double As[DG_BK][DG_BM + 1];
    __shared__ double Bs[DG_BK][DG_BN];
    const int tiles_n = (n + DG_BN - 1) / DG_BN;
    const int tm = blockIdx.x / tiles_n, tn = blockIdx.x % tiles_n;
    if (upper && tm > tn) return;
    const int row0 = tm * DG_BM, col0 = tn * DG_BN;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int b0 = sc ? (int)blockIdx.z : (int)blockIdx.z * per;
    const int b1 = sc ? b0 + 1 : min(nbatch, b0 + per);
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int b = b0; b < b1; ++b) {
        const double *Ab = A + (size_t)b * sa, *Bb = B + (size_t)b * sb;
        for (int kk = 0; kk < k; kk += DG_BK) {
            // A tile: 64 rows x 16 columns, 4 per thread (consecutive threads
            // along k for coalescing); B tile: 16 rows x 64 columns
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int e = threadIdx.x + 256 * q;
                const int ar = e >> 4, ac = e & 15;
                const int gr = row0 + ar, gc = kk + ac;
                As[ac][ar] = (gr < m && gc < k) ? __ldg(Ab + (size_t)gr * lda + gc) : 0.0;
                const int br = e >> 6, bc = e & 63;
                const int hr = kk + br, hc = col0 + bc;
                Bs[br][bc] = (hr < k && hc < n) ? __ldg(Bb + (size_t)hr * ldb + hc) : 0.0;
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < DG_BK; ++q) {
                double a[4], bv[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) a[i] = As[q][ty + 16 * i];
#pragma unroll
                for (int j = 0; j < 4; ++j) bv[j] = Bs[q][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bv[j], acc[i][j]);
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = row0 + ty + 16 * i, c = col0 + tx + 16 * j;
            if (r >= m || c >= n) continue;
            if (sc) {
                double *p = C + (size_t)b0 * sc + (size_t)r * ldc + c;
                *p = alpha * acc[i][j] + (beta != 0.0 ? beta * *p : 0.0);
            } else if (b0 < b1) {
                atomicAdd(C + (size_t)r * ldc + c, alpha * acc[i][j]);
            }
        }
}

void dgemm_batched(int m, int n, int k, const double *A, long long lda, long long sa, const double *B, long long ldb, long long sb,
                   double *C, long long ldc, long long sc, int nbatch, double alpha, double beta, bool upper, cudaStream_t st)
{
    if (m <= 0 || n <= 0 || nbatch <= 0) return;
    const int tiles = ((m + DG_BM - 1) / DG_BM) * ((n + DG_BN - 1) / DG_BN);
    int per = 1, nz = nbatch;
    if (!sc) {
        // batch reduce: about four waves of blocks over the SMs
        const int want = std::max(1, (152 * 4 + tiles - 1) / tiles);
        nz = std::min(nbatch, want);
        per = (nbatch + nz - 1) / nz;
        nz = (nbatch + per - 1) / per;
    }
    k_dgemm<<<dim3(tiles, 1, nz), 256, 0, st>>>(m, n, k, A, lda, sa, B, ldb, sb, C, ldc, sc, nbatch, per, alpha, beta, upper ? 1 : 0);
}

// Mirror the tiles below the diagonal from those above (64-row tiles of an
// n x n row-major matrix filled by an upper-tile GEMM).
__global__ void k_mirror_upper(int n, double *__restrict__ C)
{
    const long long n2 = (long long)n * n;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n2; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        if (i / DG_BM > j / DG_BN) C[e] = C[(size_t)j * n + i];
    }
}

void mirror_upper(int n, double *C, cudaStream_t st)
{
    const long long n2 = (long long)n * n;
    k_mirror_upper<<<(unsigned)std::min<long long>((n2 + 255) / 256, 152 * 16), 256, 0, st>>>(n, C);
}

// ---------------------------------------------------------------------------
// Rank-revealing pivoted LDL^T of the symmetric D' on the device.
//
// Left-looking symmetric elimination with diagonal pivoting: at step k the
// pivot p is the row with the largest |residual diagonal| d_p, and
//   v_k[i] = (D'[i][p] - sum_{j<k} s_j v_j[i] v_j[p]) / sqrt|d_p|,  s_k = sign d_p,
//   residual diagonal d_i -= s_k v_k[i]^2,
// so D' = sum_k s_k v_k v_k^T + residual.  It stops when the largest
// |residual diagonal| falls to tol times the largest initial one (for a
// positive semidefinite residual every entry is bounded by its largest
// diagonal), or gives up -- the dense form is then used -- when the rank
// passes rcap or an entry grows beyond 1e6 sqrt(max |D'_ii|) (an indefinite
// matrix whose diagonal pivots are small against its off-diagonal entries).
//
// One cooperative launch: every block picks the same pivot from the shared
// residual diagonal, updates the rows it owns (one warp per row, lanes over
// j), and meets the others at a grid barrier.  Vt is [n][rcap] so that the
// dot products over j read contiguous memory.  Values written by other
// blocks are read through L2 (ld.global.cg).
struct LdltArgs {
    const double *A;
    int n, rcap;
    double tol;
    double *Vt;        // [n][rcap]
    double *diag;      // [n]
    int *done_row;     // [n]
    double *sgn;       // [rcap]
    int *rowmap;       // [rcap]: factor index of packed row r', or -1
    int *dyn;          // [8]: lowrank, rp (padded to 128), rn (padded), rank, reason (0 ok, 1 rank, 2 growth, 3 sign split, 4 barrier)
    unsigned *bar;     // grid barrier counter (zeroed before the launch)
    unsigned *err;     // check word of the build
};

__device__ __forceinline__ double ldcg(const double *p) { return __ldcg(p); }

// Grid barrier over gridDim.x blocks (co-resident by the cooperative launch).
// Waits are bounded by the global timer (2 s); a block that gives up reports
// false and sets the build's check word.
__device__ bool grid_barrier(unsigned *bar, unsigned target, unsigned *err)
{
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok_s = 1;
        __threadfence();
        atomicAdd(bar, 1u);
        unsigned long long t0;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
        while (true) {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
            if (v >= target) break;
            unsigned long long t1;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
            if (t1 - t0 > 2000000000ull) {
                ok_s = 0;
                atomicOr(err, 8u);
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
    }
    __syncthreads();
    return ok_s != 0;
}

__global__ void __launch_bounds__(256) k_ldlt_pivoted(LdltArgs a)
{
    const int n = a.n, nb = gridDim.x;
    const int per = (n + nb - 1) / nb;
    const int r0 = blockIdx.x * per, r1 = min(n, r0 + per);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    __shared__ double red_v[8];
    __shared__ int red_i[8];
    __shared__ double s_d, s_dmax0;
    __shared__ int s_p, s_stop, s_fail;
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        a.diag[i] = a.A[(size_t)i * n + i];
        a.done_row[i] = 0;
    }
    unsigned target = nb;
    bool ok = grid_barrier(a.bar, target, a.err);
    int k = 0, reason = ok ? 0 : 4;
    if (threadIdx.x == 0) s_fail = 0;
    while (ok) {
        // pivot: the largest |residual diagonal| (ties to the lower index)
        double bv = -1.0;
        int bi = n;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const double v = fabs(ldcg(a.diag + i));
            if (v > bv || (v == bv && i < bi)) {
                bv = v;
                bi = i;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > bv || (ov == bv && oi < bi)) {
                bv = ov;
                bi = oi;
            }
        }
        if (lane == 0) {
            red_v[warp] = bv;
            red_i[warp] = bi;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < nwarp; ++w)
                if (red_v[w] > bv || (red_v[w] == bv && red_i[w] < bi)) {
                    bv = red_v[w];
                    bi = red_i[w];
                }
            if (k == 0) s_dmax0 = bv;
            s_p = bi;
            s_d = bi < n ? ldcg(a.diag + bi) : 0.0;
            s_stop = !(bv > a.tol * s_dmax0) || s_dmax0 == 0.0 || bi >= n;
        }
        __syncthreads();
        if (s_stop) break;
        if (k >= a.rcap) {
            reason = 1;
            break;
        }
        const int p = s_p;
        const double d = s_d, sd = sqrt(fabs(d)), s = d > 0.0 ? 1.0 : -1.0;
        const double glim = 1e6 * sqrt(s_dmax0);
        const double *vp = a.Vt + (size_t)p * a.rcap;
        for (int i = r0 + warp; i < r1; i += nwarp) {
            double v = 0.0;
            if (!a.done_row[i]) {
                const double *vi = a.Vt + (size_t)i * a.rcap;
                double t = 0.0;
                for (int j = lane; j < k; j += 32) t = fma(ldcg(a.sgn + j) * ldcg(vi + j), ldcg(vp + j), t);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
                v = (a.A[(size_t)i * n + p] - t) / sd;
            }
            if (lane == 0) {
                a.Vt[(size_t)i * a.rcap + k] = v;
                if (i == p) {
                    a.diag[i] = 0.0;
                    a.done_row[i] = 1;
                } else if (!a.done_row[i]) {
                    a.diag[i] -= s * v * v;
                }
                if (!(fabs(v) <= glim)) s_fail = 1;
            }
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) a.sgn[k] = s;
        ++k;
        target += nb;
        __syncthreads();
        if (threadIdx.x == 0 && s_fail) atomicOr(reinterpret_cast<unsigned *>(a.dyn + 7), 1u);
        if (!(ok = grid_barrier(a.bar, target, a.err))) {
            reason = 4;
            break;
        }
        // growth in any block ends the factorisation for every block
        if (__ldcg(a.dyn + 7)) {
            reason = 2;
            break;
        }
    }
    // block 0 publishes the outcome and the packed row order (positives,
    // padded to 128 rows, then negatives)
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int np = 0, nn = 0;
        if (!reason)
            for (int j = 0; j < k; ++j) (ldcg(a.sgn + j) > 0 ? np : nn) += 1;
        const int rp = (np + 127) / 128 * 128, rn = (nn + 127) / 128 * 128;
        if (!reason && rp + rn > a.rcap) reason = 3;
        const bool low = !reason && k > 0;
        for (int r = 0; r < a.rcap; ++r) a.rowmap[r] = -1;
        if (low) {
            int ip = 0, in = rp;
            for (int j = 0; j < k; ++j) a.rowmap[ldcg(a.sgn + j) > 0 ? ip++ : in++] = j;
        }
        a.dyn[0] = low ? 1 : 0;
        a.dyn[1] = low ? rp : 0;
        a.dyn[2] = low ? rn : 0;
        a.dyn[3] = k;
        a.dyn[4] = reason;
    }
}

// Ct[r'][i] = v_{rowmap[r']}[i] (zero rows where rowmap is -1), r' < rcap.
__global__ void k_lowrank_pack(int n, int rcap, const double *__restrict__ Vt, const int *__restrict__ rowmap, const int *__restrict__ dyn,
                               double *__restrict__ Ct)
{
    if (!dyn[0]) return;
    const long long tot = (long long)rcap * n;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / n), i = (int)(e % n);
        const int j = rowmap[r];
        Ct[e] = j >= 0 ? Vt[(size_t)i * rcap + j] : 0.0;
    }
}

int lowrank_factor(const double *A, int n, int rcap, double tol, LowRankWs &w, unsigned *err, cudaStream_t st)
{
    cudaMemsetAsync(w.dyn, 0, 8 * sizeof(int), st);
    if (rcap <= 0) return JK_OK;  // too small for the low-rank form: dyn[0] = 0 selects the dense one
    cudaMemsetAsync(w.bar, 0, sizeof(unsigned), st);
    int dev = 0, nsm = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_ldlt_pivoted, 256, 0);
    if (occ < 1) return fail(JK_ERR_CUDA, "factorisation kernel cannot be resident");
    const int nb = std::max(1, std::min(nsm, (n + 7) / 8));
    LdltArgs a{A, n, rcap, tol, w.Vt, w.diag, w.done_row, w.sgn, w.rowmap, w.dyn, w.bar, err};
    void *args[] = {&a};
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_ldlt_pivoted, dim3(nb), dim3(256), args, 0, st);
    if (e != cudaSuccess) return fail(JK_ERR_CUDA, std::string("factorisation launch: ") + cudaGetErrorString(e));
    const long long tot = (long long)rcap * n;
    k_lowrank_pack<<<(unsigned)std::min<long long>((tot + 255) / 256, 152 * 8), 256, 0, st>>>(n, rcap, w.Vt, w.rowmap, w.dyn, w.Ct);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(JK_ERR_CUDA, std::string("low-rank pack: ") + cudaGetErrorString(e));
    return JK_OK;
}

}  // namespace jk
