// Build orchestration for one J/K evaluation (Sections 2.5, 2.6 and 3.2 of
// arXiv:2410.22278) and the small bandwidth-bound kernels around it.
//
// Step order on the caller's stream:
//   1. D' = F o D with F_mn = f_m f_n the Cartesian component factors of
//      Eq. local_normalization, so every kernel works on raw Cartesian
//      functions; per-shell-block max |D'| for the precision policy.
//   2. real-space (erfc) quartet kernels per class pair -> X (Coulomb), Y
//      (exchange) accumulators, FP64 atomics.
//   3. reciprocal (erf) part per chunk of G: structure-factor slab M,
//      rho_D = M^T vec(D') and J_LR += M rho_D (Coulomb), Z = D' M per G and
//      K_LR += [M_1 .. M_g] [Z_1; ..; Z_g] (exchange).
//   4. removed K = 0 term in closed form: -(pi/(V w^2)) Tr(D'S) S and
//      -(pi/(V w^2)) S D' S.
//   5. J = F o (X + X^T + J_LR + J_bg), K = F o (Y + Y^T + K_LR + K_bg).
#include <algorithm>
#include <cstdio>
#include <map>
#include <string>

#include "kernels.cuh"
#include "launch.h"
#include "plan.h"
#include "real_units.h"

namespace jk {

__global__ void k_scale(int n, const double *__restrict__ f, const double *__restrict__ A, double *__restrict__ B)
{
    const size_t n2 = (size_t)n * n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x)
        B[i] = f[i / n] * f[i % n] * A[i];
}

__global__ void k_to_float(size_t n, const double *__restrict__ a, float *__restrict__ b)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) b[i] = (float)a[i];
}

__global__ void k_dmax(PlanDev pl, const double *__restrict__ Dp, double *__restrict__ dmax)
{
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int nsh = pl.nshell;
    if (idx >= (long long)nsh * nsh) return;
    const int I = (int)(idx / nsh), J = (int)(idx % nsh);
    const ShellRec a = pl.shells[I], b = pl.shells[J];
    double m = 0;
    for (int i = 0; i < ncart(a.l); ++i)
        for (int j = 0; j < ncart(b.l); ++j) m = fmax(m, fabs(Dp[(size_t)(a.ao + i) * pl.nbf + b.ao + j]));
    dmax[idx] = m;
}

// out[k] += sum_i A_k[i] * B[i] for k = 0, 1 (two traces in one pass)
__global__ void k_dot2(size_t n2, const double *__restrict__ B, const double *__restrict__ A0, const double *__restrict__ A1,
                       double *__restrict__ out)
{
    double s0 = 0, s1 = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x) {
        if (A0) s0 += A0[i] * B[i];
        if (A1) s1 += A1[i] * B[i];
    }
    __shared__ double sh[2][32];
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = s0;
        sh[1][threadIdx.x >> 5] = s1;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const int nw = blockDim.x >> 5;
        s0 = threadIdx.x < nw ? sh[0][threadIdx.x] : 0.0;
        s1 = threadIdx.x < nw ? sh[1][threadIdx.x] : 0.0;
        s0 = warp_sum(s0);
        s1 = warp_sum(s1);
        if (threadIdx.x == 0) {
            atomicAdd(out, s0);
            atomicAdd(out + 1, s1);
        }
    }
}

// J = F o (X + X^T + JLR + c tr S), K = F o (Y + Y^T + KLR + c SDS)
__global__ void k_final(int n, const double *__restrict__ f, const double *__restrict__ X, const double *__restrict__ Y,
                        const double *__restrict__ JLR, const double *__restrict__ KLR, const double *__restrict__ S,
                        const double *__restrict__ SDS, const double *__restrict__ trDS, double c, const unsigned *__restrict__ err,
                        double *__restrict__ J, double *__restrict__ K)
{
    const size_t n2 = (size_t)n * n;
    const double tr = *trDS;
    // a wait of a tensor-core GEMM ran out: the result is not trusted
    const double poison = *err ? __longlong_as_double(0x7ff8000000000000ll) : 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x) {
        const size_t r = i / n, cidx = i % n, t = cidx * n + r;
        const double ff = f[r] * f[cidx];
        if (J) J[i] = ff * (X[i] + X[t] + 0.5 * (JLR[i] + JLR[t]) + c * tr * S[i]) + poison;
        if (K) K[i] = ff * (Y[i] + Y[t] + 0.5 * (KLR[i] + KLR[t]) + c * 0.5 * (SDS[i] + SDS[t])) + poison;
    }
}

template <int LA, int LB>
static void sfac_go(const PlanDev &pl, int sp0, int sp1, const double *gv, int g0, int gcur, const double *gtab, double *M,
                    cudaStream_t st)
{
    const long long nt = (long long)(sp1 - sp0) * gcur;
    if (nt <= 0) return;
    k_sfac<LA, LB><<<(unsigned)((nt + 127) / 128), 128, 0, st>>>(pl, sp0, sp1, gv, g0, gcur, gtab, M);
}

void launch_sfac(int cls, const PlanDev &pl, int sp0, int sp1, const double *gv, int g0, int gcur, const double *gtab, double *M,
                 cudaStream_t st)
{
    switch (cls) {
    case 0: sfac_go<0, 0>(pl, sp0, sp1, gv, g0, gcur, gtab, M, st); break;
    case 1: sfac_go<1, 0>(pl, sp0, sp1, gv, g0, gcur, gtab, M, st); break;
    case 2: sfac_go<1, 1>(pl, sp0, sp1, gv, g0, gcur, gtab, M, st); break;
    case 3: sfac_go<2, 0>(pl, sp0, sp1, gv, g0, gcur, gtab, M, st); break;
    case 4: sfac_go<2, 1>(pl, sp0, sp1, gv, g0, gcur, gtab, M, st); break;
    case 5: sfac_go<2, 2>(pl, sp0, sp1, gv, g0, gcur, gtab, M, st); break;
    default: break;
    }
}

template <int LA, int LB>
static void sfac_df_go(const PlanDev &pl, int sp0, int sp1, int g0, int gcur, const float2 *gtab, double *M, cudaStream_t st)
{
    const long long nt = (long long)(sp1 - sp0) * gcur;
    if (nt <= 0) return;
    k_sfac_df<LA, LB><<<(unsigned)((nt + 127) / 128), 128, 0, st>>>(pl, sp0, sp1, g0, gcur, gtab, M);
}

static void launch_sfac_df(int cls, const PlanDev &pl, int sp0, int sp1, int g0, int gcur, const float2 *gtab, double *M, cudaStream_t st)
{
    switch (cls) {
    case 0: sfac_df_go<0, 0>(pl, sp0, sp1, g0, gcur, gtab, M, st); break;
    case 1: sfac_df_go<1, 0>(pl, sp0, sp1, g0, gcur, gtab, M, st); break;
    case 2: sfac_df_go<1, 1>(pl, sp0, sp1, g0, gcur, gtab, M, st); break;
    case 3: sfac_df_go<2, 0>(pl, sp0, sp1, g0, gcur, gtab, M, st); break;
    case 4: sfac_df_go<2, 1>(pl, sp0, sp1, g0, gcur, gtab, M, st); break;
    case 5: sfac_df_go<2, 2>(pl, sp0, sp1, g0, gcur, gtab, M, st); break;
    default: break;
    }
}

// (pi/p)^{3/2} e^{-G^2/4p} for every distinct pair exponent p and every G of
// a chunk, laid out [p][g] (consecutive threads of the structure-factor
// kernel read consecutive g); into tab (FP64) or, when tab2 is given, into
// tab2 as double-floats times the weight sqrt(8 pi w(G) / V) of the G
__global__ void k_gauss_table(int npv, const double *__restrict__ pv, const double *__restrict__ gv, int g0, int gcur,
                              double *__restrict__ tab, float2 *__restrict__ tab2)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)npv * gcur) return;
    const int ip = (int)(e / gcur), gi = (int)(e % gcur);
    const double *g = gv + 4 * (size_t)(g0 + gi);
    const double G2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2], p = pv[ip];
    const double v = (kPi / p) * sqrt(kPi / p) * exp(-G2 / (4.0 * p));
    if (tab2) {
        const dfl d = dfl_split(v * g[3]);
        tab2[e] = make_float2(d.hi, d.lo);
    } else {
        tab[e] = v;
    }
}

void launch_gauss_table(const Plan *P, int g0, int gcur, double *tab, cudaStream_t st)
{
    const long long ne = (long long)P->pvals.size() * gcur;
    if (ne > 0) k_gauss_table<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>((int)P->pvals.size(), P->d_pvals, P->d_gvec, g0, gcur, tab, nullptr);
}

static int grid_for(size_t n) { return (int)std::min<size_t>((n + 255) / 256, 152 * 16); }

static int cuda_check(const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(JK_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return JK_OK;
}

int compute_overlap_raw(Plan *P, cudaStream_t st)
{
    PlanDev pl = P->dev();
    for (int c = 0; c < JK_NCLASS_MAX; ++c)
        launch_sfac(c, pl, P->spair_class_off[c], P->spair_class_off[c + 1], P->d_g0, 0, 1, P->d_gtab0, P->ws.M, st);
    cudaMemcpyAsync(P->d_S, P->ws.M, sizeof(double) * P->nbf * P->nbf, cudaMemcpyDeviceToDevice, st);
    return cuda_check("overlap");
}

void PhaseTimer::begin(cudaStream_t s)
{
    st = s;
    next = 0;
    marks.clear();
    for (int i = 0; i < kPhases; ++i) launches[i] = 0;
}
int PhaseTimer::start(int phase)
{
    (void)phase;
    if (next >= (int)pool.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        pool.push_back(e);
    }
    cudaEventRecord(pool[next], st);
    return next++;
}
void PhaseTimer::stop(int phase, int ev_start, int nlaunch)
{
    int e = start(phase);
    marks.push_back({phase, {ev_start, e}});
    launches[phase] += nlaunch;
}
void PhaseTimer::destroy()
{
    for (auto e : pool) cudaEventDestroy(e);
    pool.clear();
}

#define BLAS_OK(x)                                                                       \
    do {                                                                                 \
        if ((x) != CUBLAS_STATUS_SUCCESS) return fail(JK_ERR_CUDA, "cuBLAS call failed: " #x); \
    } while (0)

int run_build(Plan *P, const double *D, double *J, double *K, cudaStream_t st)
{
    std::lock_guard<std::mutex> guard(P->build_mu);
    if (cudaSetDevice(P->device) != cudaSuccess) return fail(JK_ERR_CUDA, "cudaSetDevice failed");
    const int n = P->nbf;
    const size_t n2 = (size_t)n * n;
    PlanDev pl = P->dev();
    Workspace &w = P->ws;
    BLAS_OK(cublasSetStream(P->blas, st));
    BLAS_OK(cublasSetPointerMode(P->blas, CUBLAS_POINTER_MODE_HOST));
    const bool mixed = P->precision == JK_MIXED;
    PhaseTimer &tm = P->timer;
    tm.begin(st);
    w.mma_flops = 0;
    const int ev_all = tm.start(6);
    int ev = tm.start(0);

    k_scale<<<grid_for(n2), 256, 0, st>>>(n, P->d_compf, D, w.Dp);
    if (mixed) {
        const long long ns2 = (long long)P->nshell * P->nshell;
        k_dmax<<<(unsigned)((ns2 + 255) / 256), 256, 0, st>>>(pl, w.Dp, w.dmax);
        k_to_float<<<grid_for(n2), 256, 0, st>>>(n2, w.Dp, w.Dpf);
        k_to_float<<<grid_for((size_t)ns2), 256, 0, st>>>((size_t)ns2, w.dmax, w.dmaxf);
    }
    cudaMemsetAsync(w.X, 0, n2 * sizeof(double), st);
    cudaMemsetAsync(w.Y, 0, n2 * sizeof(double), st);
    cudaMemsetAsync(w.JLR, 0, n2 * sizeof(double), st);
    cudaMemsetAsync(w.KLR, 0, n2 * sizeof(double), st);
    cudaMemsetAsync(w.scal, 0, 16 * sizeof(double), st);
    cudaMemsetAsync(w.cnt, 0, 8 * sizeof(unsigned long long), st);
    if (w.nbig) cudaMemsetAsync(w.nbig, 0, 2 * sizeof(unsigned), st);
    int rc;
    if ((rc = cuda_check("prologue"))) return rc;
    // mixed precision: slices of D' and the eigendecomposition of D' for the
    // exchange contraction, enqueued now so they overlap nothing and are
    // ready when the reciprocal phase needs them
    if (mixed && K && (rc = ozaki_begin(P, st))) return rc;
    tm.stop(0, ev, mixed ? 4 : 1);

    // ---- real space
    ev = tm.start(1);
    int nreal = 0;
    for (int cb = 0; cb < JK_NCLASS_MAX; ++cb)
        for (int ck = cb; ck < JK_NCLASS_MAX; ++ck) {
            const ClassRange &B = P->classes[cb], &Kc = P->classes[ck];
            if (B.b1 <= B.b0 || Kc.b1 <= Kc.b0) continue;
            RealLaunch a{};
            a.pl = pl;
            a.b0 = B.b0;
            a.b1 = B.b1;
            a.k0 = Kc.b0;
            a.k1 = Kc.b1;
            a.same = cb == ck;
            a.kchunk = P->kchunk[cb][ck];
            a.tau = P->mixed_tau;
            a.Dp = w.Dp;
            a.dmax = w.dmax;
            a.Dpf = w.Dpf;
            a.dmaxf = w.dmaxf;
            a.X = w.X;
            a.Y = w.Y;
            a.st = st;
            if (!mixed) {
                a.mode = 0;
                a.fp32 = false;
                a.cnt = w.cnt;
                launch_real(cb, ck, a);
                nreal += 1;
            } else {
                // FP32 pass over every quartet, collecting the large ones ...
                cudaMemsetAsync(w.nbig, 0, sizeof(unsigned), st);
                a.mode = 2;
                a.fp32 = true;
                a.cnt = w.cnt + 1;
                a.big = w.big;
                a.nbig = w.nbig;
                a.ovf = w.nbig + 1;
                a.cap = w.cap;
                launch_real(cb, ck, a);
                // ... then FP64 over the compact list
                a.list_pass = true;
                a.cnt64 = w.cnt;
                const int el = tm.start(9);
                launch_real(cb, ck, a);
                tm.stop(9, el, 1);
                nreal += 2;
            }
            if ((rc = cuda_check("real-space kernel"))) return rc;
        }

    tm.stop(1, ev, nreal);

    // ---- reciprocal space
    const int ng = (int)(P->gvec.size() / 4);
    // mixed precision: structure factors in double-float on the FP32 pipe
    const bool sfac_df = mixed && P->sfac_df && w.gtab2;
    if (mixed && K && (rc = ozaki_prepare_lowrank(P, st))) return rc;
    for (int g0 = 0; g0 < ng; g0 += w.gc) {
        const int gcur = std::min(w.gc, ng - g0);
        ev = tm.start(2);
        int nsf = 0;
        {
            const long long ne = (long long)P->pvals.size() * gcur;
            k_gauss_table<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>((int)P->pvals.size(), P->d_pvals, P->d_gvec, g0, gcur, w.gtab,
                                                                         sfac_df ? w.gtab2 : nullptr);
        }
        for (int c = 0; c < JK_NCLASS_MAX; ++c) {
            if (sfac_df)
                launch_sfac_df(c, pl, P->spair_class_off[c], P->spair_class_off[c + 1], g0, gcur, w.gtab2, w.M, st);
            else
                launch_sfac(c, pl, P->spair_class_off[c], P->spair_class_off[c + 1], P->d_gvec, g0, gcur, w.gtab, w.M, st);
            nsf += P->spair_class_off[c + 1] > P->spair_class_off[c];
        }
        if ((rc = cuda_check("structure factors"))) return rc;
        tm.stop(2, ev, nsf);
        const double one = 1.0, zero = 0.0;
        const int m2 = 2 * gcur;
        if (J) {
            ev = tm.start(3);
            BLAS_OK(cublasDgemv(P->blas, CUBLAS_OP_T, (int)n2, m2, &one, w.M, (int)n2, w.Dp, 1, &zero, w.rho, 1));
            BLAS_OK(cublasDgemv(P->blas, CUBLAS_OP_N, (int)n2, m2, &one, w.M, (int)n2, w.rho, 1, &one, w.JLR, 1));
            tm.stop(3, ev, 2);
        }
        if (K) {
            ev = tm.start(4);
            if (mixed) {
                // split-precision BF16 tensor-core GEMMs, slices per chunk from its G bound
                if ((rc = ozaki_exchange_chunk(P, m2, w.chunk_slices[g0 / w.gc], st))) return rc;
                tm.stop(4, ev, 4);
            } else {
                // the plain FP64 form: K_LR += [M_1 .. M_2g] [Z_1; ..; Z_2g], Z_b = D' M_b (native DGEMM)
                BLAS_OK(cublasDgemmStridedBatched(P->blas, CUBLAS_OP_N, CUBLAS_OP_N, n, n, n, &one, w.Dp, n, 0, w.M, n, (long long)n2,
                                                  &zero, w.Z, m2 * n, n, m2));
                BLAS_OK(cublasDgemm(P->blas, CUBLAS_OP_N, CUBLAS_OP_N, n, n, m2 * n, &one, w.M, n, w.Z, m2 * n, &one, w.KLR, n));
                tm.stop(4, ev, 2);
            }
        }
    }
    if (mixed && K) {
        ev = tm.start(4);
        if ((rc = ozaki_finish(P, st))) return rc;
        tm.stop(4, ev, 1);
    }
    ev = tm.start(5);

    // ---- removed K = 0 term: c = -pi / (V w^2)
    const double cbg = -kPi / (P->volume * P->omega * P->omega);
    k_dot2<<<grid_for(n2), 256, 0, st>>>(n2, P->d_S, w.Dp, nullptr, w.scal);
    if (K) {
        const double one = 1.0, zero = 0.0;
        BLAS_OK(cublasDgemm(P->blas, CUBLAS_OP_N, CUBLAS_OP_N, n, n, n, &one, w.Dp, n, P->d_S, n, &zero, w.T1, n));
        BLAS_OK(cublasDgemm(P->blas, CUBLAS_OP_N, CUBLAS_OP_N, n, n, n, &one, P->d_S, n, w.T1, n, &zero, w.T2, n));
    }
    k_final<<<grid_for(n2), 256, 0, st>>>(n, P->d_compf, w.X, w.Y, w.JLR, w.KLR, P->d_S, w.T2, w.scal, cbg, w.err, J, K);
    tm.stop(5, ev, K ? 4 : 2);
    tm.stop(6, ev_all, 0);
    return cuda_check("epilogue");
}

// Autotuner: for every class pair with work, time the real-space tile
// kernel of the plan's precision over a sub-range of at most 4096 bras
// against all kets, for ket-chunk sizes {8, 16, 32, 64, 128}, and keep the
// fastest.  Results are cached in a text file (one line per GPU name,
// precision, class pair and size bucket) when cache_path is given.
int autotune(Plan *P, const double *D, cudaStream_t st, const char *cache_path, int *chosen)
{
    std::lock_guard<std::mutex> guard(P->build_mu);
    if (cudaSetDevice(P->device) != cudaSuccess) return fail(JK_ERR_CUDA, "cudaSetDevice failed");
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, P->device);
    const bool mixed = P->precision == JK_MIXED;
    const int n = P->nbf;
    const size_t n2 = (size_t)n * n;
    Workspace &w = P->ws;
    PlanDev pl = P->dev();
    k_scale<<<grid_for(n2), 256, 0, st>>>(n, P->d_compf, D, w.Dp);
    if (mixed) k_to_float<<<grid_for(n2), 256, 0, st>>>(n2, w.Dp, w.Dpf);
    // existing cache entries
    std::map<std::string, int> cache;
    if (cache_path) {
        FILE *f = fopen(cache_path, "r");
        if (f) {
            char key[512];
            int v;
            while (fscanf(f, "%511s %d", key, &v) == 2) cache[key] = v;
            fclose(f);
        }
    }
    auto bucket = [](int x) { int b = 0; while ((1 << b) < x) ++b; return b; };
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int cands[] = {8, 16, 32, 64, 128};
    int k = 0;
    bool dirty = false;
    for (int cb = 0; cb < JK_NCLASS_MAX; ++cb)
        for (int ck = cb; ck < JK_NCLASS_MAX; ++ck) {
            const ClassRange &B = P->classes[cb], &Kc = P->classes[ck];
            if (B.b1 <= B.b0 || Kc.b1 <= Kc.b0) continue;
            char key[512];
            snprintf(key, sizeof key, "%s|%s|%d%d|%d|%d", prop.name, mixed ? "mixed" : "fp64", cb, ck, bucket(B.b1 - B.b0),
                     bucket(Kc.b1 - Kc.b0));
            for (char *q = key; *q; ++q)
                if (*q == ' ') *q = '_';
            int best = -1;
            auto it = cache.find(key);
            if (it != cache.end()) {
                best = it->second;
            } else {
                float best_ms = 1e30f;
                for (int c : cands) {
                    RealLaunch a{};
                    a.pl = pl;
                    a.b0 = B.b0;
                    a.b1 = std::min(B.b1, B.b0 + 4096);
                    a.k0 = Kc.b0;
                    a.k1 = Kc.b1;
                    a.same = cb == ck;
                    a.kchunk = c;
                    a.mode = 0;
                    a.fp32 = mixed;
                    a.Dp = w.Dp;
                    a.dmax = w.dmax;
                    a.Dpf = w.Dpf;
                    a.dmaxf = w.dmaxf;
                    a.X = w.X;
                    a.Y = w.Y;
                    a.cnt = w.cnt;
                    a.st = st;
                    cudaEventRecord(e0, st);
                    launch_real(cb, ck, a);
                    cudaEventRecord(e1, st);
                    if (cudaEventSynchronize(e1) != cudaSuccess) {
                        cudaEventDestroy(e0);
                        cudaEventDestroy(e1);
                        return fail(JK_ERR_CUDA, "autotune launch failed");
                    }
                    float ms = 0;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (ms < best_ms) {
                        best_ms = ms;
                        best = c;
                    }
                }
                cache[key] = best;
                dirty = true;
            }
            P->kchunk[cb][ck] = best;
            if (chosen && k < 36) chosen[k] = best;
            ++k;
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cache_path && dirty) {
        FILE *f = fopen(cache_path, "w");
        if (f) {
            for (auto &kv : cache) fprintf(f, "%s %d\n", kv.first.c_str(), kv.second);
            fclose(f);
        }
    }
    P->tuned = true;
    return cuda_check("autotune");
}

int build_counts(Plan *P, long long *counts, int n)
{
    unsigned long long h[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    unsigned hb[2] = {0, 0};
    if (P->timer.next > 0 && cudaEventSynchronize(P->timer.pool[P->timer.next - 1]) != cudaSuccess)
        return fail(JK_ERR_CUDA, "build did not finish");
    if (cudaMemcpy(h, P->ws.cnt, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess) return fail(JK_ERR_CUDA, "count copy failed");
    if (P->ws.nbig && cudaMemcpy(hb, P->ws.nbig, sizeof hb, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(JK_ERR_CUDA, "count copy failed");
    h[2] = hb[1];
    h[3] = 0;
    for (int i = 0; i < n && i < 6; ++i) counts[i] = (long long)h[i];
    unsigned e = 0;
    if (cudaMemcpy(&e, P->ws.err, sizeof e, cudaMemcpyDeviceToHost) != cudaSuccess) return fail(JK_ERR_CUDA, "check word copy failed");
    if (e) return fail(JK_ERR_TIMEOUT, "a bounded wait in a tensor-core GEMM ran out; J and K of that build are NaN");
    return JK_OK;
}

int build_times(Plan *P, double *ms, int *launches, int n)
{
    PhaseTimer &tm = P->timer;
    for (int i = 0; i < n; ++i) {
        if (ms) ms[i] = 0;
        if (launches) launches[i] = 0;
    }
    if (tm.marks.empty()) return JK_OK;
    if (cudaEventSynchronize(tm.pool[tm.next - 1]) != cudaSuccess) return fail(JK_ERR_CUDA, "build did not finish");
    for (auto &m : tm.marks) {
        float t = 0;
        cudaEventElapsedTime(&t, tm.pool[m.second.first], tm.pool[m.second.second]);
        if (m.first < n && ms) ms[m.first] += t;
    }
    for (int i = 0; i < n && i < PhaseTimer::kPhases; ++i)
        if (launches) launches[i] = tm.launches[i];
    int tot = 0;
    for (int i = 0; i < 6; ++i) tot += tm.launches[i];
    if (launches && n > 6) launches[6] = tot;
    if (ms && n > 10) ms[10] = P->ws.mma_flops;  // slot 10: BF16 MMA flops issued (for the tensor roofline)
    return JK_OK;
}

}  // namespace jk
