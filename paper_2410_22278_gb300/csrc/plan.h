// Host-side plan: built once per geometry (Section 3.1), then immutable.
#pragma once
#include <cmath>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/jk.h"
#include "dense.h"
#include "jk_internal.h"

namespace jk {

// thread-local last error; returns the status for convenience
int fail(int status, const std::string &msg);

struct ClassRange {
    int la, lb;
    int b0, b1;  // spi index range
};

// Device counters of a build: per precision (base 0 FP64, 1 FP32) image
// quartets [base], algorithmic flops [4 + base], screening and bookkeeping
// flops [8 + base], lane-terms [12 + base] and lane slots [14 + base] of the
// primitive loops.
constexpr int kCounters = 16;

struct Workspace {
    double *Dp = nullptr;     // D scaled by component factors
    double *X = nullptr;      // real-space J accumulator
    double *Y = nullptr;      // real-space K accumulator
    double *JLR = nullptr;    // reciprocal J (raw components)
    double *KLR = nullptr;    // reciprocal K (raw components)
    double *T1 = nullptr;     // n x n temporaries
    double *T2 = nullptr;
    double *M = nullptr;      // structure-factor chunk [2*gc][n][n]
    double *Z = nullptr;      // D * M chunk, stacked
    double *rho = nullptr;    // [2*gc] density structure factors
    double *rho_part = nullptr;  // [2*gc][kSlabSplitsMax] their partial sums
    double *dmax = nullptr;   // [nshell*nshell] max |D'| per shell block
    float *Dpf = nullptr;     // single-precision copies for the FP32 kernels (mixed precision)
    float *dmaxf = nullptr;
    double *scal = nullptr;   // small scalars (traces, energies)
    // Coulomb-only builds (J-engine): per local primitive pair, hs Hermite
    // density values (FP64 and FP32) and hs Hermite J accumulators
    int hs = 0;
    double *DhD = nullptr, *JH = nullptr;
    float *DhF = nullptr;
    unsigned *err = nullptr;  // device check word
    unsigned long long *cnt = nullptr;  // kCounters build counters (see above)
    int2 *big = nullptr;                // compact list of quartets sent to FP64 (mixed precision)
    unsigned *nbig = nullptr;           // [0] list length, [1] overflow count (accumulated over a build)
    unsigned cap = 0;
    int gc = 0;               // G vectors per chunk
    double *gtab = nullptr;   // [distinct p][gc]: (pi/p)^{3/2} e^{-G^2/4p} of the current G chunk
    float2 *gtab2 = nullptr;  // the same as double-floats (mixed-precision structure factors)
    size_t bytes = 0;
    // split-precision tensor-core exchange (mixed precision)
    int npad = 0, oz_slices = 0;
    std::vector<int> chunk_slices;  // slices per G chunk (mixed exchange), <= oz_slices
    __nv_bfloat16 *Ms = nullptr, *Zs = nullptr, *Ds = nullptr, *Cs = nullptr;
    int *Mex = nullptr, *Zex = nullptr, *Dex = nullptr, *Cex = nullptr;
    // low-rank form of D (pivoted LDL^T on the device, dense.cu); which form
    // a build used is known only on the device (lr.dyn)
    LowRankWs lr;
    // (slabs, slices) of every exchange chunk of the last build: with the
    // rank read back after the build they give the MMA flops it issued
    std::vector<std::pair<int, int>> chunk_log;
    // tcgen05 form: TMA descriptors of the slice buffers (K-major rows, 128-byte
    // swizzle, 64 x 128 boxes) and per-split FP64 partial sums of the exchange
    bool tc = false;
    CUtensorMap tm_Ms, tm_Ds, tm_Cs, tm_Zd, tm_Zl;
    float2 *Kpart = nullptr;  // (hi, lo) float pairs
    int kpart_splits = 0;
};

// CUDA events bracketing the phases of one build (see jk_build_times); a
// phase's events are recorded on the stream its kernels run on (`cur`).
struct PhaseTimer {
    // 0..6 as in jk_build_times, 7 tensor-core GEMMs, 8 their slicing, 9 FP64
    // list pass, 10 FP32 real-space tile kernels
    static constexpr int kPhases = 11;
    std::vector<cudaEvent_t> pool;
    std::vector<std::pair<int, std::pair<int, int>>> marks;  // phase, (start event, end event)
    int next = 0;
    int launches[kPhases] = {0};
    cudaStream_t st = nullptr, cur = nullptr;
    void begin(cudaStream_t s);
    void use(cudaStream_t s) { cur = s; }
    int start(int phase);
    void stop(int phase, int ev_start, int nlaunch);
    void destroy();
};

// D-independent reciprocal data kept between builds (jk_plan_cache): the
// structure-factor slab of every G chunk and, for mixed plans, its BF16
// exchange slices and row exponents.  Filled by the first build after it is
// switched on; later builds skip the structure factors and their slicing.
struct RecipCache {
    // m_valid: the structure factors M are filled; s_valid: so are the
    // exchange slices (mixed plans; a Coulomb-only build fills M alone)
    bool on = false, m_valid = false, s_valid = false;
    size_t bytes = 0;
    double *M = nullptr;              // [2 * ng][n][n] (FP64 plans) or [2 * ng][n (n + 1) / 2] packed upper triangles (mixed)
    __nv_bfloat16 *Ms = nullptr;      // chunk c at rows [row0[c], ...) of a (rows x npad) matrix
    int *Mex = nullptr;               // chunk c at ex0[c]
    std::vector<long long> row0, ex0;
    CUtensorMap tm_Ms;
};

struct Plan {
    int device = 0;
    jk_precision precision = JK_FP64;
    int nbf = 0, nshell = 0;
    double omega = 0, volume = 0, g_max = 0, r1_max = 0;
    jk_cutoffs cut{};
    double L[9]{}, Finv[9]{};
    // host copies
    std::vector<ShellRec> shells;
    std::vector<SpiRec> spi;
    std::vector<PpiRec> ppi;
    std::vector<SpairRec> spair;
    std::vector<int> spi_order;
    std::vector<ClassRange> classes;
    std::vector<double> r1;    // [nr1][4]
    std::vector<double> gvec;  // [ng][4]
    std::vector<double> gsize;  // [ng] bound on the exchange term of each G: (4 pi/V) e^{-G^2/4w^2}/G^2 s(G)^2
    std::vector<double> compf;
    std::vector<int> spair_class_off;  // shell pairs grouped by class: [JK_NCLASS_MAX+1]
    long long n_ord_shell_pairs = 0, n_ord_prim_pairs = 0, n_ord_local_pairs = 0;
    long long n_shell_pairs = 0, n_quartets = 0, n_quartets_schwarz = 0, n_quartets_fp64 = 0;
    double mixed_tau = 0;
    int kchunk[JK_NCLASS_MAX][JK_NCLASS_MAX];    // kets per tile (or per warp) of the real-space kernels (autotuned)
    int kvariant[JK_NCLASS_MAX][JK_NCLASS_MAX];  // kernel family: 0 lane-per-bra, 1 warp, 2 pair queue (1, 2: s and p class pairs)
    bool tuned = false;
    // device arrays
    ShellRec *d_shells = nullptr;
    SpiRec *d_spi = nullptr;
    float4 *d_kblk = nullptr;  // per 32 consecutive images: bounding-sphere centre and radius (incl. extents)
    float2 *d_kblk2 = nullptr; // per 32 consecutive images: largest S, smallest pair exponent
    PpiRec *d_ppi = nullptr;
    PpiF *d_ppf = nullptr;
    float *d_ppB = nullptr;  // |K| p^{-5/4} per primitive pair
    float *d_r1f = nullptr;
    SpairRec *d_spair = nullptr;
    int *d_spi_order = nullptr;
    double *d_boys = nullptr;
    float *d_boys_f = nullptr;
    double *d_r1 = nullptr;
    double *d_gvec = nullptr;
    double *d_g0 = nullptr;  // one G = 0 entry with unit weight (overlap)
    // structure-factor tables: distinct pair exponents, the exponent index of
    // each primitive pair, (cos, sin)(2 pi k / 1024), and (pi/p)^{3/2} (G = 0)
    std::vector<double> pvals;
    std::vector<int> ppi_pidx;
    std::vector<double2> ppi_ab;  // exponents (a, b) of each primitive pair (one-electron operators)
    double2 *d_ppi_ab = nullptr;
    double *d_pvals = nullptr, *d_gtab0 = nullptr;
    int *d_ppi_pidx = nullptr;
    double2 *d_phase = nullptr;
    // double-float structure factors (mixed precision): usable when every
    // reciprocal vector has |n_k| <= 64 in the reciprocal basis
    bool sfac_df = false;
    PpiDF *d_ppdf = nullptr;
    float4 *d_gdf = nullptr, *d_phasef = nullptr;
    double *d_compf = nullptr;
    double *d_S = nullptr;  // raw-component overlap over the pair list
    size_t device_bytes = 0;
    Workspace ws;
    RecipCache cache;
    PhaseTimer timer;
    std::mutex build_mu;
    PlanDev dev() const;
};

int build_plan(const jk_cell *cell, const jk_shell *shells, int nshell, double omega, const jk_cutoffs *cut,
               jk_precision precision, int device, Plan **out);
void destroy_plan(Plan *p);
int run_build(Plan *p, const double *D, double *J, double *K, cudaStream_t st);
int compute_overlap_raw(Plan *p, cudaStream_t st);
int build_times(Plan *p, double *ms, int *launches, int n);
int build_counts(Plan *p, long long *counts, int n);
int autotune(Plan *p, const double *D, cudaStream_t st, const char *cache_path, int *chosen);
int set_schedule(Plan *P, const int *sched, int n);
int ozaki_begin(Plan *P, cudaStream_t st);
double ozaki_mma_flops(const Plan *P, const int dyn[3]);
int ozaki_exchange_chunk(Plan *P, int chunk, const double *Mc, int m2, int S, cudaStream_t st);
int cache_reciprocal(Plan *P, size_t max_bytes);
void release_cache(Plan *P);
int ozaki_setup_tc(Plan *P);
int ozaki_finish(Plan *P, cudaStream_t st);
struct Plan;
void launch_gauss_table(const Plan *P, int g0, int gcur, double *tab, cudaStream_t st);
int one_electron(Plan *P, int natom, const double *Z, const double *xyz, double *T, double *V, cudaStream_t st);
int energy_noalloc(const Plan *P, const double *D, const double *J, const double *K, double *e_coul, double *e_exch,
                   cudaStream_t st);

// host helpers shared by plan.cu and api.cu
void boys_table(int ncol, int npts, double inv_step, std::vector<double> &out);
double ewald_point_charges_host(const double *lat, int n, const double *q, const double *xyz, double omega, double delta);

}  // namespace jk
