// Dense FP64 kernels of the reciprocal-space and background contractions and
// the device-side low-rank factorisation of the density (dense.cu).
#pragma once
#include <cuda_runtime.h>

namespace jk {

// Workspace of the rank-revealing factorisation D' ~ sum_j s_j v_j v_j^T.
struct LowRankWs {
    int rcap = 0;              // largest padded rank (rp + rn) the low-rank form accepts
    double *Vt = nullptr;      // [n][rcap]
    double *diag = nullptr;    // [n]
    int *done_row = nullptr;   // [n]
    double *sgn = nullptr;     // [rcap]
    int *rowmap = nullptr;     // [rcap]
    int *dyn = nullptr;        // [8] device status: lowrank, rp, rn, rank, reason, -, -, growth flag
    unsigned *bar = nullptr;   // grid barrier counter
    double *Ct = nullptr;      // [rcap][n] packed factor rows: C+ (rp rows) then C- (rn rows)
};

// rho[b] = sum_i M[b][i] x[i] for b < m2 (M is [m2][n2]); part holds
// m2 * kSlabSplitsMax partial sums.
constexpr int kSlabSplitsMax = 1024;
void slab_gemv_t(const double *M, long long n2, int m2, const double *x, double *part, double *rho, cudaStream_t st);
// y[i] += alpha sum_b M[b][i] rho[b].
void slab_gemv_n(const double *M, long long n2, int m2, const double *rho, double alpha, double *y, cudaStream_t st);
// Row-major batched FP64 GEMM; sc = 0 reduces every batch into one C (atomics).
void dgemm_batched(int m, int n, int k, const double *A, long long lda, long long sa, const double *B, long long ldb, long long sb,
                   double *C, long long ldc, long long sc, int nbatch, double alpha, double beta, bool upper, cudaStream_t st);
// Copy the 64-row tiles above the diagonal of C (n x n) to their mirror images.
void mirror_upper(int n, double *C, cudaStream_t st);
// Pivoted LDL^T of A (n x n, symmetric, device) with relative stopping
// tolerance tol; rank and form published in w.dyn, factor rows in w.Ct.
int lowrank_factor(const double *A, int n, int rcap, double tol, LowRankWs &w, unsigned *err, cudaStream_t st);

}  // namespace jk
