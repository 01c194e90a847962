// Real-space quartet kernels with bra class (2,1); generated per bra class so
// that the instantiations compile in parallel.
#include "kernels.cuh"
#include "launch.h"

namespace jk {

template <int LA, int LB, int LC, int LD>
static void go(const RealLaunch &a)
{
    const int nb = a.b1 - a.b0, nk = a.k1 - a.k0;
    if (nb <= 0 || nk <= 0) return;
    dim3 grid((nb + kRealThreads - 1) / kRealThreads, (nk + a.kchunk - 1) / a.kchunk);
    if (a.fp32)
        k_real<LA, LB, LC, LD, float><<<grid, kRealThreads, 0, a.st>>>(a.pl, a.b0, a.b1, a.k0, a.k1, a.same, a.kchunk, a.mode, a.tau, a.Dp, a.dmax, a.X, a.Y, a.cnt);
    else
        k_real<LA, LB, LC, LD, double><<<grid, kRealThreads, 0, a.st>>>(a.pl, a.b0, a.b1, a.k0, a.k1, a.same, a.kchunk, a.mode, a.tau, a.Dp, a.dmax, a.X, a.Y, a.cnt);
}

void launch_real_c4(int ck, const RealLaunch &a)
{
    switch (ck) {
    case 4: go<2, 1, 2, 1>(a); break;
    case 5: go<2, 1, 2, 2>(a); break;
    default: break;
    }
}

}  // namespace jk
