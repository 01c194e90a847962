// Launch descriptors shared by the orchestration code and the per-class
// kernel instantiation units.
#pragma once
#include <cuda_runtime.h>

#include "jk_internal.h"

namespace jk {

struct RealLaunch {
    PlanDev pl;
    int b0, b1, k0, k1, same, kchunk, mode;
    double tau;
    bool fp32;
    const double *Dp, *dmax;      // FP64 kernels
    const float *Dpf, *dmaxf;     // FP32 kernels
    double *X, *Y;
    unsigned long long *cnt;
    int2 *big;           // compact list of large quartets (mixed precision)
    unsigned *nbig, *ovf;
    unsigned cap;
    bool list_pass;      // launch k_real_list over the list instead of the tile kernel
    int variant;         // 0 lane-per-bra tile kernel; for s and p class pairs also 1 warp, 2 pair-queue kernel (autotuned)
    unsigned long long *cnt64;
    // Coulomb-only builds (J-engine): Hermite densities of the primitive
    // pairs (stride hs) and their Hermite J accumulators
    const double *DhD;
    const float *DhF;
    double *JH;
    int hs;
    cudaStream_t st;
};

void launch_sfac(int cls, const PlanDev &pl, int sp0, int sp1, const double *gv, int g0, int gcur, const double *gtab, double *M,
                 cudaStream_t st);

}  // namespace jk
