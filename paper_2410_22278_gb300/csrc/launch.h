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
    const double *Dp, *dmax;
    double *X, *Y;
    unsigned long long *cnt;
    cudaStream_t st;
};

// one function per bra class cb (0..5); ck >= cb selects the ket class
void launch_real_c0(int ck, const RealLaunch &a);
void launch_real_c1(int ck, const RealLaunch &a);
void launch_real_c2(int ck, const RealLaunch &a);
void launch_real_c3(int ck, const RealLaunch &a);
void launch_real_c4(int ck, const RealLaunch &a);
void launch_real_c5(int ck, const RealLaunch &a);

void launch_sfac(int cls, const PlanDev &pl, int sp0, int sp1, const double *gv, int g0, int gcur, double *M, cudaStream_t st);

}  // namespace jk
