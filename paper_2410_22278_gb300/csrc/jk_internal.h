// Internal data layout shared by the host plan builder and the CUDA kernels.
//
// A plan holds, resident on the device:
//   * shells: centre, angular momentum, primitive range, first AO index;
//   * unique shell-pair images (I, J, R) -- the middle layer of the
//     three-layer pair structure of Section 3.1 -- in canonical orientation
//     (l_I >= l_J; for I == J only R >= 0 lexicographically), bucketed by
//     angular class (l_I, l_J) and sorted by descending Schwarz estimate;
//   * local primitive pairs (the bottom layer): P, P-A, P-B(R), p and the
//     prefactor K = c_a c_b exp(-ab/p |A-B-R|^2) (Eq. E_recursion_0 folded
//     into K), sorted inside each image by descending B = |K| p^{-5/4};
//   * the Boys-function Taylor table, the R1 candidate lattice vectors for
//     the real-space sums and the half-space reciprocal vectors.
#pragma once
#include <stdint.h>

#define JK_MAXL 2
#define JK_MAXLQ (4 * JK_MAXL)   // highest total angular momentum of a quartet
#define JK_NCLASS_MAX 6          // (la, lb) with la >= lb, la <= 2

// Boys table: F_m(T_k) for T_k = k / JK_BOYS_INV_STEP, k = 0 .. JK_BOYS_NPTS-1,
// m = 0 .. JK_BOYS_MCOL-1.  Above JK_BOYS_TMAX the asymptotic branch is used.
#define JK_BOYS_INV_STEP 32
#define JK_BOYS_TMAX 36.0
#define JK_BOYS_NPTS (36 * 32 + 2)
#define JK_BOYS_MCOL (JK_MAXLQ + 8)

struct ShellRec {
    double c[3];
    int l, nprim, p0, ao;
};

struct SpiRec {      // one unique shell-pair image
    int I, J;        // shells, canonical orientation
    int pp0, npp;    // local primitive pairs [pp0, pp0 + npp)
    int n[3];        // lattice image of J
    float w;         // orbit weight: 0.5 for (I, I, R = 0), else 1
    int spair;       // index of the unique shell pair (I, J)
    double Q;        // Schwarz estimate (Eq. pbc_eri_cauchy_schwarz_cutoff_definition, summed over primitives)
    float Pc[3];     // centre of the image's largest primitive pair
    float ext;       // max |P_i - Pc| over its primitive pairs
    float S;         // sum over its primitive pairs of |K| p^{-5/4} (quartet-level real-space bound)
    float pmin;      // smallest pair exponent p among them
};

struct PpiRec {      // one local primitive pair
    double P[3];
    double PA[3];    // P - A
    double PB[3];    // P - (B + R)
    double p;        // a + b
    double K;        // c_a c_b exp(-ab/p |A - B - R|^2), normalised coefficients
    double pad;      // 1/p
};

struct __align__(16) PpiF {  // single-precision copy of a local primitive pair (FP32 kernels, screening); 48 B, loaded as 3 x 16 B
    float P[3];
    float PA[3];
    float PB[3];
    float p;
    float K;
    float pad;       // 1/p
};

// One local primitive pair for the double-float structure factors: the
// fractional coordinates of P reduced mod 1 and split in three (f1 on the
// grid 2^-16, f2 on the grid 2^-33, f3 the rest), K, the index of its
// exponent among the distinct ones, and P - A, P - B and 1/2p as
// double-floats (hi, lo).
struct PpiDF {
    float4 a;  // f1x, f1y, f1z, K hi
    float4 b;  // f2x, f2y, f2z, K lo
    float4 c;  // f3x, f3y, f3z, exponent index (int bits)
    float4 d;  // (P-A)x hi, lo, (P-A)y hi, lo
    float4 e;  // (P-A)z hi, lo, (P-B)x hi, lo
    float4 f;  // (P-B)y hi, lo, (P-B)z hi, lo
    float4 g;  // 1/2p hi, lo, 0, 0
};

struct SpairRec {    // unique shell pair (I, J) with its images [spi0, spi0 + nspi)
    int I, J, spi0, nspi;
};

struct PlanDev {
    int nbf, nshell;
    int nspi, nppi, nspair;
    const ShellRec *shells;
    const SpiRec *spi;
    const float4 *kblk;          // images 32k .. 32k+31: bounding sphere (centre, radius including extents)
    const float2 *kblk2;         // the same images: largest S, smallest pair exponent
    const PpiRec *ppi;
    const SpairRec *spair;
    const int *spi_order;        // spi indices grouped by shell pair (for the reciprocal build)
    const double *boys;          // [JK_BOYS_NPTS][JK_BOYS_MCOL]
    const float *boys_f;
    const PpiF *ppf;
    const float *ppB;            // B = |K| p^{-5/4} of each primitive pair (descending inside an image)
    float mag_thr;               // B_i B_j below this: the primitive quartet is below the real-space threshold
    const double *r1;            // [nr1][4]: x, y, z, |R|, sorted by |R|
    const float *r1f;            // the same in single precision
    int nr1;
    const double *gvec;          // [ng][4]: Gx, Gy, Gz, sqrt(8 pi w(G) / V)
    int ng;
    const double *compf;         // Cartesian component factor of each AO
    const int *ppi_pidx;         // index of each primitive pair's exponent p among the distinct ones
    const double2 *phase;        // (cos, sin)(2 pi k / 1024), k = 0..1023
    const PpiDF *ppdf;           // double-float copy of the primitive pairs (mixed-precision structure factors)
    const float4 *gdf;           // [ng][3]: (n1, n2, n3, 0) with G = sum n_k b_k; (Gx, Gy) and (Gz, 0) as double-floats
    const float4 *phasef;        // (cos, sin)(2 pi k / 1024) as double-floats (cos hi, cos lo, sin hi, sin lo)
    double L[9];                 // lattice rows a, b, c
    double Finv[9];              // fractional coordinates f = Finv * r
    float Lf[9], Finvf[9];       // the same in single precision (no conversions in FP32 kernels)
    double omega, inv_omega2;
    float inv_omega2f;
    double ewald_R;              // delta_Ewald-R as given
    float log_ewald_R;           // ln of the per-term threshold used inside the real-space sums
    double volume;
    float hplane[3];             // spacing of the lattice planes of each fractional coordinate
    int orth;                    // lattice vectors mutually orthogonal: rounding f gives the minimum image
};
