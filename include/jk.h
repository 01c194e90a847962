/*
 * jk.h -- C ABI of the Gamma-point periodic Coulomb (J) and exchange (K)
 * matrix build over contracted Cartesian Gaussian shells with Ewald-split
 * electron repulsion integrals (Wang, Hait, Unzueta, Zhang, Martinez,
 * "Fast and Scalable GPU-Accelerated Quantum Chemistry for Periodic Systems
 * with Gaussian Orbitals", arXiv:2410.22278).
 *
 * Units are atomic (bohr, hartree).  All entry points return a status code
 * (JK_OK = 0, negative on failure) unless stated otherwise; no C++
 * exception crosses this boundary.  jk_last_error() returns a thread-local
 * description of the most recent failure on the calling thread.
 *
 * AO order: shells in input order; inside a shell the Cartesian components
 * run lx descending, then ly descending (p: x y z; d: xx xy xz yy yz zz).
 * Matrices are nbf x nbf, row-major, FP64, symmetric.
 *
 * Threads: a plan is immutable after creation except for its one build
 * workspace.  jk_build calls on the same plan, from any host threads and on
 * any streams, are ordered one after another on the device: each call
 * enqueues, under the plan's lock, a wait for the previous build on that plan
 * before its own kernels, so two such builds never overlap on the workspace
 * (the host is not blocked).  Distinct plans build concurrently on distinct
 * streams.
 */
#ifndef JK_H
#define JK_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define JK_OK 0
#define JK_ERR_INVALID (-1)      /* bad argument: volume <= 0, exponent <= 0, nprim outside 1..16, NULL pointer */
#define JK_ERR_UNSUPPORTED (-2)  /* angular momentum above 2 (d) */
#define JK_ERR_OOM (-3)          /* device or host allocation failed, or the request exceeds a budget */
#define JK_ERR_CUDA (-4)         /* a CUDA runtime call or kernel launch failed */
#define JK_ERR_TIMEOUT (-5)      /* a wait ran out of time (jk_wait, bounded device waits) */
#define JK_ERR_DEVICE_CHECK (-6) /* a device-side bounds check tripped (an index outside its buffer) */
#define JK_ERR_BUSY (-7)         /* no free slot / server shutting down */
#define JK_ERR_NOT_FOUND (-8)    /* unknown ticket */

/* ---- problem statement (Sections 2.1, 3.6) ------------------------------ */

/* Lattice vectors as rows: lattice[0..2] = a, lattice[3..5] = b,
 * lattice[6..8] = c (bohr).  |det| must be > 0. */
typedef struct {
    double lattice[9];
} jk_cell;

/* One contracted Cartesian shell (Eq. local_contracted_basis).  exps and
 * coefs (raw contraction coefficients; normalised internally by Eq.
 * local_normalization and to unit local self-overlap) are read during
 * jk_plan_create only and may be freed afterwards.  center may lie in any
 * lattice image. */
typedef struct {
    int l;              /* 0, 1, 2 (s, p, d); larger -> JK_ERR_UNSUPPORTED */
    int nprim;          /* 1..16 */
    const double *exps; /* nprim exponents > 0 (bohr^-2) */
    const double *coefs;
    double center[3];
} jk_shell;

/* The four lattice-sum thresholds of Section 3.6 (values <= 0 select the
 * paper's default 1e-14) and the mixed-precision switch (Section 3.5):
 * an image quartet whose density-weighted size estimate is at or above
 * mixed_switch is evaluated in FP64, below it in FP32 (<= 0: 3e-3). */
typedef struct {
    double pair_R;   /* delta_pair-R, Eq. pbc_eri_pair_cutoff_implementation */
    double pair_cs;  /* delta_pair-Cauchy-Schwarz, Eq. pbc_eri_cauchy_schwarz_cutoff_implementation */
    double ewald_R;  /* delta_Ewald-R, Eq. pbc_eri_real_cutoff_implementation */
    double ewald_K;  /* delta_Ewald-K, Eq. pbc_eri_reciprocal_cutoff_implementation */
    double mixed_switch;
} jk_cutoffs;

/* JK_FP64: every step in FP64.  JK_MIXED: real-space quartets split by
 * mixed_switch (above); structure factors in double-float (pairs of FP32,
 * about 44 bits; FP64 when a reciprocal vector has an integer coordinate
 * beyond 64 in the reciprocal basis); the reciprocal exchange contraction
 * as split-precision BF16 tensor-core GEMMs, in a low-rank form when the
 * device-side factorisation of D finds a rank within 60% of nbf (a
 * closed-shell density has rank n_occ), else in the dense form;
 * accumulation, the reciprocal Coulomb contraction and the background in
 * FP64. */
typedef enum { JK_FP64 = 0, JK_MIXED = 1 } jk_precision;

typedef struct jk_plan jk_plan; /* opaque; owns its device-resident pair and G data */

/* Figures of a plan, filled by jk_plan_info. */
typedef struct {
    int nbf, nshell, n_classes;
    int n_g;                       /* half-space reciprocal vectors kept */
    long long n_shell_pairs;       /* unique shell pairs with at least one local pair */
    long long n_pair_images;       /* unique shell-pair images (I, J, R) */
    long long n_prim_pair_images;  /* local primitive pairs (Section 3.1) */
    long long n_quartets;          /* unique shell-pair-image quartets evaluated in real space */
    long long n_quartets_schwarz;  /* of those, with Schwarz product >= delta_pair-CS (the quartets/s unit) */
    long long n_quartets_fp64;     /* quartets the mixed policy sends to FP64 (all of them under JK_FP64) */
    long long n_r1_candidates;     /* lattice vectors scanned per primitive quartet */
    double omega, g_max, r1_max, volume;
    size_t device_bytes;           /* resident plan arrays */
    size_t workspace_bytes;        /* per-build scratch owned by the plan */
} jk_plan_stats;

/* ---- plan ---------------------------------------------------------------- */

/* Build the plan for one cell (Sections 3.1, 3.3, 3.4): normalise the
 * shells, build the local-pair lists over lattice images with the pair
 * cut-offs of Eqs. pbc_eri_pair_cutoff_implementation and pbc_eri_cauchy_schwarz_cutoff_implementation (minimum-image offsets, Eq.
 * lattice_image_min_norm), Schwarz estimates (Eq. pbc_eri_cauchy_schwarz_cutoff_definition) and quartet classes,
 * the reciprocal vector list, and upload everything to `device`.
 * omega <= 0 selects Eq. omega_implementation with w = 10.
 * cut == NULL means all defaults.  On success *out owns device memory until
 * jk_plan_destroy.  Errors: JK_ERR_INVALID, JK_ERR_UNSUPPORTED, JK_ERR_OOM,
 * JK_ERR_CUDA; *out is left NULL. */
int jk_plan_create(const jk_cell *cell, const jk_shell *shells, int nshell, double omega, const jk_cutoffs *cut,
                   jk_precision precision, int device, jk_plan **out);

int jk_plan_info(const jk_plan *plan, jk_plan_stats *out);

/* Host only (no device needed): the pair-list counts of Section 3.1 for a
 * cell, as jk_plan_create would build them.  counts[0] ordered shell pairs
 * with at least one local pair, counts[1] ordered primitive pairs kept,
 * counts[2] ordered local primitive pairs (lattice images included),
 * counts[3] unique shell-pair images, counts[4] half-space reciprocal
 * vectors.  Same errors as jk_plan_create's argument checks. */
int jk_pair_counts(const jk_cell *cell, const jk_shell *shells, int nshell, double omega, const jk_cutoffs *cut,
                   long long counts[5]);

/* Keep the plan's D-independent reciprocal-space data resident between
 * builds (no counterpart in the paper, which recomputes its reciprocal
 * terms per quartet): the pair structure factors of every reciprocal vector
 * (2 n_G nbf^2 FP64 for JK_FP64 plans; for JK_MIXED plans their upper
 * triangles, 2 n_G nbf (nbf + 1) / 2 FP64, which is all the Coulomb
 * contraction needs since they are symmetric in the two basis indices, and
 * their BF16 exchange slices).  The next jk_build fills the cache (a
 * Coulomb-only build fills the structure factors; the first build with K
 * adds the slices); later builds skip the structure factors and their
 * slicing, which for an SCF loop or repeated frames of one geometry are the
 * same every build.  Allocated at once if the total
 * fits max_bytes, else JK_ERR_OOM (the plan then works as before);
 * max_bytes = 0 releases it.  *bytes (may be NULL) receives the size.
 * Waits for the plan's last build.  jk_plan_info's device_bytes includes
 * the cache. */
int jk_plan_cache(jk_plan *plan, size_t max_bytes, size_t *bytes);

/* Number of basis functions of the plan (or -1 for NULL). */
int jk_plan_nbf(const jk_plan *plan);

void jk_plan_destroy(jk_plan *plan);

/* ---- build (Sections 2.5, 2.6, 3.2) --------------------------------------- */

/* J_mn = sum_ls (mn|ls) D_ls and K_mn = sum_ls (ml|sn) D_ls at the Gamma
 * point (Eqs. pbc_j_definition_k_sample and pbc_k_definition with k = 0),
 * with (mn|ls) the Ewald-split periodic ERI of Eq. pbc_eri_general_final:
 * the erfc real-space sum over R1, the reciprocal sum over K != 0 and the
 * removed K = 0 background term.
 * D, J, K: device pointers to nbf*nbf FP64, row-major, on the plan's
 * device.  D must be symmetric; J and K are overwritten and come out
 * symmetric; either may be NULL to skip it (K is the expensive one).
 * Stream-ordered on `cuda_stream` (a cudaStream_t; NULL = legacy default);
 * returns after enqueueing and never waits for the device (every decision
 * that depends on D -- the mixed-precision split, the rank of D -- is taken
 * on the device).  Caller keeps ownership of D, J, K. */
int jk_build(jk_plan *plan, const double *D, double *J, double *K, void *cuda_stream);

/* Same as jk_build with HOST buffers (row-major FP64): copies D in, builds,
 * copies J and K out, and synchronises the stream before returning. */
int jk_build_host(jk_plan *plan, const double *D_host, double *J_host, double *K_host, void *cuda_stream);

/* E_J = 1/2 sum_mn D_mn J_mn and E_K = -1/4 sum_mn D_mn K_mn (closed-shell
 * density D = 2 C C^T; the paper gives only J and K).  D, J, K device
 * pointers (J or K may be NULL, the energy is then 0).  Results are
 * written to host scalars; synchronises `cuda_stream`. */
int jk_energy(const jk_plan *plan, const double *D, const double *J, const double *K, double *e_coul, double *e_exch,
              void *cuda_stream);

/* jk_energy without any device allocation (the paper has no counterpart;
 * this is a deployment variant of the energy reduction above).  For callers
 * that must not have a library allocate device memory: a framework whose
 * pool allocator owns the device memory under a fixed budget (a foreign
 * cudaMalloc may fail there or fragment the pool), or a latency-bound loop
 * that cannot pay for an allocation or free inside the call, which may
 * synchronise the whole device.  Same arguments, results and
 * synchronisation as jk_energy; the sums are taken in a different order, so
 * the two agree to FP64 rounding, not bit for bit.
 *
 * Scratch: a fixed 64 KB device array inside the library (4096 block
 * partials and the two sums), present on every device the library is loaded
 * on until the process exits.  Nothing in it has to start at zero: every
 * value a call reads was written earlier in the same call.
 * Limit: nbf <= 16384; a larger plan returns JK_ERR_INVALID with a message
 * naming the limit (use jk_energy there).
 * First call on a device: looks up the array's device address once
 * (cudaGetSymbolAddress with the plan's device current); make that first
 * call before any stream capture begins.  The address is kept for the life
 * of the process, so the device's primary context must outlive the
 * library's use of it: after a cudaDeviceReset (or another replacement of
 * the primary context) do not call this entry point again.
 * Concurrency: all calls on one device share the array, so two calls whose
 * work overlaps on the GPU (different streams or host threads) race and may
 * return wrong sums; serialise them.
 * Errors: JK_ERR_INVALID (NULL argument, nbf above the limit), JK_ERR_CUDA. */
int jk_energy_noalloc(const jk_plan *plan, const double *D, const double *J, const double *K, double *e_coul,
                      double *e_exch, void *cuda_stream);

/* Device time of each phase of the most recent jk_build on this plan, in
 * milliseconds, from CUDA events recorded on the build's stream around the
 * phase's kernels (waits for that build to finish).  ms[0] prologue (D scaling, zeroing, density slices and
 * factorisation), ms[1] real space (fork to the last list pass), ms[2]
 * reciprocal structure factors, ms[3] reciprocal Coulomb contraction, ms[4]
 * reciprocal exchange contraction, ms[5] background and assembly, ms[6]
 * whole build, ms[7] the tensor-core GEMM launches inside ms[4] (mixed
 * precision), ms[8] their operand slicing, ms[9] the FP64 list passes inside
 * ms[1] (mixed precision), ms[10] the FP32 (mixed) or FP64 tile kernels
 * inside ms[1], ms[11] (not a time) the BF16 MMA flops the GEMMs issued;
 * launches[i] the kernel launches per phase.  n = number of slots the
 * caller provides (<= 12 used). */
int jk_build_times(jk_plan *plan, double *ms, int *launches, int n);

/* Autotuner (no counterpart in the paper): choose the tile shape of every
 * real-space class-pair kernel -- the family (0 lane-per-bra, 8 .. 128 kets
 * per tile; for class pairs of s and p shells also 1 warp-per-bra, 128 ..
 * 2048 kets per warp, and 2 pair queue, 32 .. 512 kets per tile) and its
 * tile -- by timing the candidates on two sub-ranges of bras with CUDA
 * events, on
 * `cuda_stream`, using density D (device, as in jk_build) for realistic
 * work.  If cache_path is not NULL, choices are read from and written to
 * that text file, keyed by GPU name, precision, class pair and size
 * bucket.  chosen (may be NULL) receives 42 ints: (family, kets) for each
 * of the 21 class pairs (bra class <= ket class, classes ss, ps, pp, ds,
 * dp, dd), family 0 lane-per-bra, 1 warp, 2 pair queue.  Overwrites the
 * plan's build workspace; synchronises the stream. */
int jk_autotune(jk_plan *plan, const double *D, void *cuda_stream, const char *cache_path, int *chosen);

/* Set the real-space schedule directly (what jk_autotune chooses): sched
 * holds (family, kets) for the first n class pairs in jk_autotune's order;
 * families 1 and 2 only for class pairs of s and p shells, kets in
 * 1..65535.  Results do not depend on the schedule beyond rounding.
 * Errors: JK_ERR_INVALID (nothing is changed). */
int jk_plan_set_schedule(jk_plan *plan, const int *sched, int n);

/* Work counters of the most recent jk_build (waits for it to finish):
 * counts[0] unique image quartets evaluated in real space in FP64,
 * counts[1] those evaluated in FP32 (mixed precision only), counts[2]
 * quartets that the mixed policy wanted in FP64 but that overflowed the
 * plan's FP64 list and were evaluated in FP32 (0 in a healthy build),
 * counts[3] the number of pivots of the density factorisation of a mixed
 * build with K (the numerical rank of D' when counts[6] is 1),
 * counts[4] and counts[5] the algorithmic floating-point operations of the
 * real-space evaluation in FP64 and in FP32 (the McMurchie-Davidson steps:
 * ket Hermite coefficients per bra image and ket primitive, seeds and R
 * table per lattice image inside the screening sphere, prefactor and
 * Hermite contraction per primitive quartet, digestion per image quartet;
 * a transcendental counts one, a fused multiply-add two),
 * counts[6] 1 if the reciprocal exchange took the low-rank form, else 0,
 * counts[7] and counts[8] the screening and bookkeeping operations in FP64
 * and FP32 (radii, minimum images, image search, recomputed bra
 * coefficients), counts[9] and counts[10] the lane-terms processed and the
 * lane slots offered by the FP64 primitive loops (their ratio is the lane
 * occupancy), counts[11] and counts[12] the same for FP32.  n <= 13.
 * Returns JK_ERR_TIMEOUT (and the build's J and K are NaN) if a bounded
 * device wait ran out. */
int jk_build_counts(jk_plan *plan, long long *counts, int n);

/* Gamma overlap over the plan's pair list (Eq. pbc_overlap_formula),
 * written to the device pointer S (nbf*nbf FP64); stream-ordered. */
int jk_overlap(const jk_plan *plan, double *S, void *cuda_stream);

/* One-electron operators of the cell on the plan's pair list (paper
 * Sections 2.1-2.2; the kinetic formula is in its Supporting Information):
 * T = kinetic energy, sum over images R of <mu| -1/2 nabla^2 |nu(R)>;
 * V = attraction of point charges Z (host, natom) at xyz (host, natom x 3,
 * bohr) with all their images, Ewald-split at the plan's omega as in Eq.
 * pbc_v1e_base_case_final: erfc real-space sum over charge images, the
 * reciprocal sum against rho_N(G) = sum_C Z_C e^{-iG.C} (G list and
 * structure factors of the plan), and the self term +(pi/(V w^2)) Z_tot S.
 * T and V are device pointers (nbf x nbf, row-major, FP64; either may be
 * NULL); the caller owns them.  Uses the plan's build workspace, so it is
 * ordered after earlier builds on the plan; synchronises `cuda_stream`
 * before returning.  With the electron density D, E_kin = sum D o T and
 * E_ne = sum D o V; the nuclear repulsion is jk_ewald_point_charges.
 * Errors: JK_ERR_INVALID (NULL plan, natom < 0, charges missing),
 * JK_ERR_OOM, JK_ERR_CUDA. */
int jk_one_electron(jk_plan *plan, int natom, const double *Z, const double *xyz, double *T, double *V, void *cuda_stream);

/* Ewald energy of point charges (Eq. nuclear_repulsion_energy, including the
 * removed K = 0 term -(4 pi/V)/(4 w^2) that a non-neutral set needs), on the
 * host; q[n], xyz[3n] (bohr), delta = truncation of both sums (<= 0: 1e-14).
 * A test instrument for the Ewald machinery. */
int jk_ewald_point_charges(const jk_cell *cell, int n, const double *q, const double *xyz, double omega, double delta,
                           double *energy);

/* ---- serving: continuous batching of builds (host scheduler) ------------ */

typedef struct jk_server jk_server;

/* A request server on `device` that admits builds while the sum of the
 * admitted plans' workspace stays within hbm_budget_bytes and at most
 * max_slots builds are in flight; each slot owns a stream.  Errors:
 * JK_ERR_INVALID, JK_ERR_CUDA, JK_ERR_OOM. */
int jk_server_create(int device, size_t hbm_budget_bytes, int max_slots, jk_server **out);

/* Queue one build of `plan` on device buffers D, J, K (as in jk_build);
 * returns a ticket.  The plan and buffers must stay valid until jk_wait
 * returns for that ticket.  JK_ERR_OOM if the plan alone exceeds the
 * budget; JK_ERR_BUSY after shutdown began. */
int jk_submit(jk_server *srv, jk_plan *plan, const double *D, double *J, double *K, long long *ticket);

/* Wait up to timeout_ms (< 0: forever) for a ticket.  On completion writes
 * the build's status and its latency (submit to completion, seconds).
 * JK_ERR_TIMEOUT if it has not finished; JK_ERR_NOT_FOUND for an unknown or
 * already-collected ticket. */
int jk_wait(jk_server *srv, long long ticket, int timeout_ms, int *build_status, double *latency_s);

/* Drain in-flight work, then free the server (never frees caller buffers). */
void jk_server_destroy(jk_server *srv);

/* ---- diagnostics ---------------------------------------------------------- */

/* Measurement utility (not part of a build): FMA throughput of the current
 * device in TFLOP/s (2 flops per FMA), FP64 if fp64 != 0 else FP32, from a
 * kernel of independent FMA chains timed with CUDA events.  The ALU
 * rooflines of the quartet kernels are reported against these. */
int jk_microbench_fma(int fp64, double *tflops);

const char *jk_status_string(int status);
const char *jk_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* JK_H */
