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

#include "jeng.cuh"
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

// Packed upper triangles (row-major, i <= j): entry (i, j) at
// i n - i (i - 1) / 2 + j - i.  The structure factors M_b are symmetric in
// their two basis indices (each unique shell pair writes both blocks), so
// the Coulomb contraction needs one triangle: rho_b = sum_{i<=j} M_b(ij)
// Ds(ij) with Ds the symmetrised density (D'_ij + D'_ji off the diagonal),
// and J_LR(ij) = J_LR(ji) = sum_b M_b(ij) rho_b.
__device__ __forceinline__ long long tri_index(long long n, long long i, long long j) { return i * n - i * (i - 1) / 2 + j - i; }

// Ap[b] = upper triangle of A[b] for nb matrices n x n
__global__ void k_pack_upper(int n, long long npk, int nb, const double *__restrict__ A, double *__restrict__ Ap)
{
    const long long n2 = (long long)n * n, tot = n2 * nb;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < tot; idx += (long long)gridDim.x * blockDim.x) {
        const long long b = idx / n2, r = idx - b * n2, i = r / n, j = r - i * n;
        if (j >= i) Ap[b * npk + tri_index(n, i, j)] = A[idx];
    }
}

// Ds = packed D + D^T off the diagonal, D on it
__global__ void k_sym_density(int n, const double *__restrict__ D, double *__restrict__ Ds)
{
    const long long n2 = (long long)n * n;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n2; idx += (long long)gridDim.x * blockDim.x) {
        const long long i = idx / n, j = idx - i * n;
        if (j > i) Ds[tri_index(n, i, j)] = D[idx] + D[j * n + i];
        else if (j == i) Ds[tri_index(n, i, i)] = D[idx];
    }
}

// J (n x n) = the symmetric matrix of the packed Jp
__global__ void k_unpack_sym(int n, const double *__restrict__ Jp, double *__restrict__ J)
{
    const long long n2 = (long long)n * n;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n2; idx += (long long)gridDim.x * blockDim.x) {
        const long long i = idx / n, j = idx - i * n;
        J[idx] = Jp[i <= j ? tri_index(n, i, j) : tri_index(n, j, i)];
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

// Hermite densities (back = false) or the Hermite-to-Cartesian step (back =
// true) of the J-engine for the images of class cls (l_I >= l_J)
template <int LA, int LB>
static void hermite_go(bool back, const PlanDev &pl, int b0, int b1, const Workspace &w, const double *Dp, bool f32, double *X,
                       cudaStream_t st)
{
    if (b1 <= b0) return;
    const unsigned g = (unsigned)((b1 - b0 + 127) / 128);
    if (back)
        k_hermite_back<LA, LB><<<g, 128, 0, st>>>(pl, b0, b1, w.hs, w.JH, X);
    else
        k_hermite_density<LA, LB><<<g, 128, 0, st>>>(pl, b0, b1, Dp, w.hs, w.DhD, f32 ? w.DhF : nullptr);
}

static void launch_hermite(int cls, bool back, const PlanDev &pl, int b0, int b1, const Workspace &w, const double *Dp, bool f32,
                           double *X, cudaStream_t st)
{
    switch (cls) {
    case 0: hermite_go<0, 0>(back, pl, b0, b1, w, Dp, f32, X, st); break;
    case 1: hermite_go<1, 0>(back, pl, b0, b1, w, Dp, f32, X, st); break;
    case 2: hermite_go<1, 1>(back, pl, b0, b1, w, Dp, f32, X, st); break;
    case 3: hermite_go<2, 0>(back, pl, b0, b1, w, Dp, f32, X, st); break;
    case 4: hermite_go<2, 1>(back, pl, b0, b1, w, Dp, f32, X, st); break;
    case 5: hermite_go<2, 2>(back, pl, b0, b1, w, Dp, f32, X, st); break;
    default: break;
    }
}

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
    st = cur = s;
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
    cudaEventRecord(pool[next], cur);
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

// Reciprocal (erf) part of the build on stream st: structure factors (or
// the cache), the Coulomb slab passes and the exchange contraction, chunk
// by chunk of G.  Enqueued on its own stream, concurrent with real space.
static int reciprocal_phase(Plan *P, double *J, double *K, cudaStream_t st)
{
    const int n = P->nbf;
    const size_t n2 = (size_t)n * n;
    PlanDev pl = P->dev();
    Workspace &w = P->ws;
    const bool mixed = P->precision == JK_MIXED;
    PhaseTimer &tm = P->timer;
    int ev, rc;
    const int ng = (int)(P->gvec.size() / 4);
    // mixed precision: structure factors in double-float on the FP32 pipe
    const bool sfac_df = mixed && P->sfac_df && w.gtab2;
    // the D-independent structure factors (and their exchange slices) come
    // from the reciprocal cache once a build has filled it; a mixed plan
    // caches them as packed upper triangles for the Coulomb contraction (the
    // exchange reads its BF16 slices), an FP64 plan in full
    RecipCache &cache = P->cache;
    const bool packed = cache.on && mixed;
    const long long npk = (long long)n * (n + 1) / 2;
    if (J && packed) {
        // symmetrised density and the packed J_LR accumulator in the
        // epilogue's scratch (free until the epilogue)
        k_sym_density<<<grid_for(n2), 256, 0, st>>>(n, w.Dp, w.T1);
        cudaMemsetAsync(w.T2, 0, npk * sizeof(double), st);
    }
    for (int g0 = 0, chunk = 0; g0 < ng; g0 += w.gc, ++chunk) {
        const int gcur = std::min(w.gc, ng - g0);
        // Mf: full structure factors of the chunk (formed here when needed);
        // Mc: what the Coulomb contraction reads
        double *Mf = w.M, *Mc = w.M;
        bool form = true;
        if (cache.on && !mixed) {
            Mf = Mc = cache.M + 2 * (size_t)g0 * n2;
            form = !cache.m_valid;
        } else if (packed) {
            Mc = cache.M + 2 * (size_t)g0 * npk;
            form = !cache.m_valid || (K && !cache.s_valid);  // the exchange slices are cut from the full form
        }
        if (form) {
            ev = tm.start(2);
            int nsf = 0;
            const long long ne = (long long)P->pvals.size() * gcur;
            k_gauss_table<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>((int)P->pvals.size(), P->d_pvals, P->d_gvec, g0, gcur, w.gtab,
                                                                         sfac_df ? w.gtab2 : nullptr);
            for (int c = 0; c < JK_NCLASS_MAX; ++c) {
                if (sfac_df)
                    launch_sfac_df(c, pl, P->spair_class_off[c], P->spair_class_off[c + 1], g0, gcur, w.gtab2, Mf, st);
                else
                    launch_sfac(c, pl, P->spair_class_off[c], P->spair_class_off[c + 1], P->d_gvec, g0, gcur, w.gtab, Mf, st);
                nsf += P->spair_class_off[c + 1] > P->spair_class_off[c];
            }
            if (packed && !cache.m_valid) {
                k_pack_upper<<<152 * 16, 256, 0, st>>>(n, npk, 2 * gcur, Mf, Mc);
                ++nsf;
            }
            if ((rc = cuda_check("structure factors"))) return rc;
            tm.stop(2, ev, nsf + 1);
        }
        const int m2 = 2 * gcur;
        if (J) {
            // rho_D = M^T vec(D'), J_LR += M rho_D (two passes over the slab)
            ev = tm.start(3);
            if (packed) {
                slab_gemv_t(Mc, npk, m2, w.T1, w.rho_part, w.rho, st);
                slab_gemv_n(Mc, npk, m2, w.rho, 1.0, w.T2, st);
            } else {
                slab_gemv_t(Mc, (long long)n2, m2, w.Dp, w.rho_part, w.rho, st);
                slab_gemv_n(Mc, (long long)n2, m2, w.rho, 1.0, w.JLR, st);
            }
            tm.stop(3, ev, 3);
        }
        if (K) {
            ev = tm.start(4);
            if (mixed) {
                // split-precision BF16 tensor-core GEMMs, slices per chunk from its G bound
                if ((rc = ozaki_exchange_chunk(P, chunk, Mf, m2, w.chunk_slices[chunk], st))) return rc;
                tm.stop(4, ev, 4);
            } else {
                // the plain FP64 form: Z_b = D' M_b, then K_LR += sum_b M_b Z_b
                // (upper tiles; the product is symmetric), FP64 GEMMs
                dgemm_batched(n, n, n, w.Dp, n, 0, Mf, n, (long long)n2, w.Z, n, (long long)n2, m2, 1.0, 0.0, false, st);
                dgemm_batched(n, n, n, Mf, n, (long long)n2, w.Z, n, (long long)n2, w.KLR, n, 0, m2, 1.0, 0.0, true, st);
                tm.stop(4, ev, 2);
            }
        }
    }
    // filled in stream order: later builds on this plan are ordered after this one
    if (J && packed) k_unpack_sym<<<grid_for(n2), 256, 0, st>>>(n, w.T2, w.JLR);
    if (cache.on) {
        cache.m_valid = true;
        if (mixed && K) cache.s_valid = true;
    }
    if (mixed && K) {
        ev = tm.start(4);
        if ((rc = ozaki_finish(P, st))) return rc;
        tm.stop(4, ev, 1);
    } else if (K && ng > 0) {
        mirror_upper(n, w.KLR, st);
    }
    return cuda_check("reciprocal phase");
}

// The caller holds P->build_mu (jk_build), so the stream ordering against
// the previous build on this plan and the use of its workspace are one
// critical section.
int run_build(Plan *P, const double *D, double *J, double *K, cudaStream_t st)
{
    if (cudaSetDevice(P->device) != cudaSuccess) return fail(JK_ERR_CUDA, "cudaSetDevice failed");
    const int n = P->nbf;
    const size_t n2 = (size_t)n * n;
    PlanDev pl = P->dev();
    Workspace &w = P->ws;
    const bool mixed = P->precision == JK_MIXED;
    PhaseTimer &tm = P->timer;
    tm.begin(st);
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
    cudaMemsetAsync(w.cnt, 0, kCounters * sizeof(unsigned long long), st);
    if (w.nbig) cudaMemsetAsync(w.nbig, 0, 2 * sizeof(unsigned), st);
    int rc;
    if ((rc = cuda_check("prologue"))) return rc;
    // mixed precision: slices of D' and its low-rank factorisation for the
    // exchange contraction (decided on the device; nothing waits for it)
    if (mixed && K && (rc = ozaki_begin(P, st))) return rc;
    tm.stop(0, ev, mixed ? (K ? 8 : 4) : 1);

    // Coulomb-only build: the J-engine (Hermite densities in, Hermite J out)
    // (only the classes with a d shell, l_I = 2, take part: kJengClass)
    constexpr int kJengClass = 3;
    bool have_d = false;
    for (int c = kJengClass; c < JK_NCLASS_MAX; ++c) have_d = have_d || P->classes[c].b1 > P->classes[c].b0;
    const bool jeng = J && !K && have_d;
    if (jeng) {
        const int eh = tm.start(0);
        cudaMemsetAsync(w.JH, 0, std::max<size_t>(1, P->ppi.size()) * w.hs * sizeof(double), st);
        for (int c = kJengClass; c < JK_NCLASS_MAX; ++c)
            launch_hermite(c, false, pl, P->classes[c].b0, P->classes[c].b1, w, w.Dp, mixed, nullptr, st);
        tm.stop(0, eh, JK_NCLASS_MAX - kJengClass + 1);
    }

    // ---- real space (the phases run one after another on the caller's
    // stream: run on streams of their own they gained nothing on the water
    // box -- the tile kernels fill every SM, and the tensor-core GEMMs, which
    // need a whole SM each, only start as the tile grids drain)
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
            a.variant = P->kvariant[cb][ck];
            a.tau = P->mixed_tau;
            a.Dp = w.Dp;
            a.dmax = w.dmax;
            a.Dpf = w.Dpf;
            a.dmaxf = w.dmaxf;
            a.X = w.X;
            a.Y = K ? w.Y : nullptr;
            a.st = st;
            a.DhD = w.DhD;
            a.DhF = w.DhF;
            a.JH = w.JH;
            a.hs = w.hs;
            // Coulomb-only builds take the J-engine for class pairs with a d
            // shell on both sides, where the Hermite contraction is smaller
            // than the Cartesian block (measured: for s and p classes the
            // Cartesian kernels with the exchange digestion skipped are
            // faster); its tiles are lane-per-bra: kets per tile as tuned for
            // that family, else 32
            const bool use_jeng = jeng && cb >= kJengClass && ck >= kJengClass;
            if (use_jeng && a.variant != 0) a.kchunk = 32;
            if (use_jeng && !mixed) {
                a.mode = 0;
                a.fp32 = false;
                a.cnt = w.cnt;
                const int et = tm.start(10);
                launch_jeng(cb, ck, a);
                tm.stop(10, et, 1);
                nreal += 1;
            } else if (use_jeng) {
                cudaMemsetAsync(w.nbig, 0, sizeof(unsigned), st);
                a.mode = 2;
                a.fp32 = true;
                a.cnt = w.cnt + 1;
                a.big = w.big;
                a.nbig = w.nbig;
                a.ovf = w.nbig + 1;
                a.cap = w.cap;
                const int et = tm.start(10);
                launch_jeng(cb, ck, a);
                tm.stop(10, et, 1);
                // the listed large quartets: the Cartesian FP64 pass, Coulomb only
                a.list_pass = true;
                a.cnt64 = w.cnt;
                const int el = tm.start(9);
                launch_real(cb, ck, a);
                tm.stop(9, el, 1);
                nreal += 2;
            } else if (!mixed) {
                a.mode = 0;
                a.fp32 = false;
                a.cnt = w.cnt;
                const int et = tm.start(10);
                launch_real(cb, ck, a);
                tm.stop(10, et, 1);
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
                const int et = tm.start(10);
                launch_real(cb, ck, a);
                tm.stop(10, et, 1);
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
    if (jeng) {
        // Hermite J of every primitive pair back to Cartesian, into X
        for (int c = kJengClass; c < JK_NCLASS_MAX; ++c)
            launch_hermite(c, true, pl, P->classes[c].b0, P->classes[c].b1, w, nullptr, false, w.X, st);
        nreal += JK_NCLASS_MAX - kJengClass;
    }
    tm.stop(1, ev, nreal);

    // ---- reciprocal space
    if ((rc = reciprocal_phase(P, J, K, st))) return rc;

    ev = tm.start(5);

    // ---- removed K = 0 term: c = -pi / (V w^2)
    const double cbg = -kPi / (P->volume * P->omega * P->omega);
    k_dot2<<<grid_for(n2), 256, 0, st>>>(n2, P->d_S, w.Dp, nullptr, w.scal);
    if (K) {
        // S D' S (both factors symmetric; FP64 GEMMs)
        dgemm_batched(n, n, n, w.Dp, n, 0, P->d_S, n, 0, w.T1, n, (long long)n2, 1, 1.0, 0.0, false, st);
        dgemm_batched(n, n, n, P->d_S, n, 0, w.T1, n, 0, w.T2, n, (long long)n2, 1, 1.0, 0.0, false, st);
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
    float part_ms = 0;
    // candidates (family, kets per tile): lane-per-bra kernels with 8 .. 128
    // kets per tile, and for s and p class pairs the warp kernels with
    // 128 .. 2048 kets per warp and the pair-queue kernels with 32 .. 512
    // kets per tile; a choice is stored as family * 65536 + kets
    std::vector<int> cands_t = {8, 16, 32, 64, 128}, cands_w;
    for (int c : {128, 256, 512, 1024, 2048}) cands_w.push_back(65536 + c);   // warp kernels
    for (int c : {32, 64, 128, 256, 512}) cands_w.push_back(2 * 65536 + c);   // pair-queue kernels
    int k = 0;
    bool dirty = false;
    for (int cb = 0; cb < JK_NCLASS_MAX; ++cb)
        for (int ck = cb; ck < JK_NCLASS_MAX; ++ck, ++k) {
            const ClassRange &B = P->classes[cb], &Kc = P->classes[ck];
            if (chosen) {
                chosen[2 * k] = P->kvariant[cb][ck];
                chosen[2 * k + 1] = P->kchunk[cb][ck];
            }
            if (B.b1 <= B.b0 || Kc.b1 <= Kc.b0) continue;
            char key[512];
            snprintf(key, sizeof key, "%s|%s|v3|%d%d|%d|%d", prop.name, mixed ? "mixed" : "fp64", cb, ck, bucket(B.b1 - B.b0),
                     bucket(Kc.b1 - Kc.b0));
            for (char *q = key; *q; ++q)
                if (*q == ' ') *q = '_';
            int best = -1;
            auto it = cache.find(key);
            if (it != cache.end()) {
                best = it->second;
            } else {
                float best_ms = 1e30f;
                std::vector<int> cands = cands_t;
                if (real_has_warp_kernel(cb, ck)) cands.insert(cands.end(), cands_w.begin(), cands_w.end());
                // two sub-ranges of at most 2048 bras (the class is sorted by
                // primitive count, so the start and the middle differ)
                const int nbc = B.b1 - B.b0, mid = B.b0 + nbc / 2;
                for (int c : cands)
                    for (int part = 0; part < 2; ++part) {
                        RealLaunch a{};
                        a.pl = pl;
                        a.b0 = part == 0 ? B.b0 : std::max(B.b0 + std::min(nbc, 2048), mid);
                        a.b1 = std::min(B.b1, a.b0 + 2048);
                        if (a.b1 <= a.b0) continue;
                        a.k0 = Kc.b0;
                        a.k1 = Kc.b1;
                        a.same = cb == ck;
                        a.kchunk = c & 65535;
                        a.variant = c >> 16;
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
                        if (part == 0) part_ms = ms;
                        else part_ms += ms;
                        if (part == 1 || nbc <= 2048) {
                            if (part_ms < best_ms) {
                                best_ms = part_ms;
                                best = c;
                            }
                    }
                }
                cache[key] = best;
                dirty = true;
            }
            P->kchunk[cb][ck] = best & 65535;
            P->kvariant[cb][ck] = best >> 16;
            if (chosen) {
                chosen[2 * k] = best >> 16;
                chosen[2 * k + 1] = best & 65535;
            }
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

// Real-space schedule given by the caller: (family, kets per tile) per
// class pair in the order of jk_autotune's output.
int set_schedule(Plan *P, const int *sched, int n)
{
    int k = 0;
    for (int cb = 0; cb < JK_NCLASS_MAX; ++cb)
        for (int ck = cb; ck < JK_NCLASS_MAX; ++ck, ++k) {
            if (k >= n) return JK_OK;
            const int fam = sched[2 * k], kets = sched[2 * k + 1];
            if (fam < 0 || fam > 2 || (fam >= 1 && !real_has_warp_kernel(cb, ck)) || kets < 1 || kets > 65535)
                return fail(JK_ERR_INVALID, "schedule entry " + std::to_string(k) + " out of range");
        }
    k = 0;
    for (int cb = 0; cb < JK_NCLASS_MAX; ++cb)
        for (int ck = cb; ck < JK_NCLASS_MAX && k < n; ++ck, ++k) {
            P->kvariant[cb][ck] = sched[2 * k];
            P->kchunk[cb][ck] = sched[2 * k + 1];
        }
    return JK_OK;
}

int build_counts(Plan *P, long long *counts, int n)
{
    unsigned long long h[kCounters] = {};
    unsigned hb[2] = {0, 0};
    if (P->timer.next > 0 && cudaEventSynchronize(P->timer.pool[P->timer.next - 1]) != cudaSuccess)
        return fail(JK_ERR_CUDA, "build did not finish");
    if (cudaMemcpy(h, P->ws.cnt, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess) return fail(JK_ERR_CUDA, "count copy failed");
    if (P->ws.nbig && cudaMemcpy(hb, P->ws.nbig, sizeof hb, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(JK_ERR_CUDA, "count copy failed");
    // rank and form of the density factorisation (mixed builds with K)
    int dyn[4] = {0, 0, 0, 0};
    if (P->precision == JK_MIXED && P->ws.lr.dyn && cudaMemcpy(dyn, P->ws.lr.dyn, sizeof dyn, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(JK_ERR_CUDA, "status copy failed");
    // public layout (jk_build_counts)
    const long long out[13] = {(long long)h[0], (long long)h[1], (long long)hb[1], dyn[3], (long long)h[4], (long long)h[5], dyn[0],
                               (long long)h[8], (long long)h[9], (long long)h[12], (long long)h[14], (long long)h[13], (long long)h[15]};
    for (int i = 0; i < n && i < 13; ++i) counts[i] = out[i];
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
    if (ms && n > 11) {
        // slot 11: BF16 MMA flops issued (for the tensor roofline), from the
        // form and rank the device chose
        int dyn[3] = {0, 0, 0};
        if (P->precision == JK_MIXED && P->ws.lr.dyn &&
            cudaMemcpy(dyn, P->ws.lr.dyn, sizeof dyn, cudaMemcpyDeviceToHost) != cudaSuccess)
            return fail(JK_ERR_CUDA, "status copy failed");
        ms[11] = P->precision == JK_MIXED ? ozaki_mma_flops(P, dyn) : 0.0;
    }
    return JK_OK;
}

}  // namespace jk
