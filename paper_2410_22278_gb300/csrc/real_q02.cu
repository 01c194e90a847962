// Real-space quartet kernels for bra class (0, 0) and ket class (1, 1) (generated by gen_units.py).
#include "jeng.cuh"
#include "launch.h"
#include "real2.cuh"

namespace jk {

void launch_real_q02(const RealLaunch &a)
{
    const int nb = a.b1 - a.b0, nk = a.k1 - a.k0;
    if (nb <= 0 || nk <= 0) return;
    if (a.list_pass) {
        k_real_list_w<0, 0, 1, 1><<<152 * 8, 32 * kWarpsPerBlock, 0, a.st>>>(a.pl, a.big, a.nbig, a.cap, a.same, a.Dp, a.X, a.Y,
                                                                                  a.cnt64);
        return;
    }
    if (a.variant == 2) {
        dim3 grid((nb + kRealThreads - 1) / kRealThreads, (nk + a.kchunk - 1) / a.kchunk);
        if (a.fp32)
            k_real_q<0, 0, 1, 1, float><<<grid, kRealThreads, 0, a.st>>>(a.pl, a.b0, a.b1, a.k0, a.k1, a.same, a.kchunk,
                                                                                 a.mode, a.tau, a.Dpf, a.dmaxf, a.X, a.Y, a.cnt, a.big,
                                                                                 a.nbig, a.cap, a.ovf);
        else
            k_real_q<0, 0, 1, 1, double><<<grid, kRealThreads, 0, a.st>>>(a.pl, a.b0, a.b1, a.k0, a.k1, a.same, a.kchunk,
                                                                                  a.mode, a.tau, a.Dp, a.dmax, a.X, a.Y, a.cnt, a.big,
                                                                                  a.nbig, a.cap, a.ovf);
        return;
    }
    if (a.variant == 0) {
        dim3 grid((nb + kRealThreads - 1) / kRealThreads, (nk + a.kchunk - 1) / a.kchunk);
        if (a.fp32)
            k_real<0, 0, 1, 1, float><<<grid, kRealThreads, 0, a.st>>>(a.pl, a.b0, a.b1, a.k0, a.k1, a.same, a.kchunk, a.mode,
                                                                               a.tau, a.Dpf, a.dmaxf, a.X, a.Y, a.cnt, a.big, a.nbig,
                                                                               a.cap, a.ovf);
        else
            k_real<0, 0, 1, 1, double><<<grid, kRealThreads, 0, a.st>>>(a.pl, a.b0, a.b1, a.k0, a.k1, a.same, a.kchunk, a.mode,
                                                                                a.tau, a.Dp, a.dmax, a.X, a.Y, a.cnt, a.big, a.nbig,
                                                                                a.cap, a.ovf);
        return;
    }
    dim3 grid((nb + kWarpsPerBlock - 1) / kWarpsPerBlock, (nk + a.kchunk - 1) / a.kchunk);
    if (a.fp32)
        k_real_w<0, 0, 1, 1, float><<<grid, 32 * kWarpsPerBlock, 0, a.st>>>(a.pl, a.b0, a.b1, a.k0, a.k1, a.same, a.kchunk,
                                                                                 a.mode, a.tau, a.Dpf, a.dmaxf, a.X, a.Y, a.cnt, a.big,
                                                                                 a.nbig, a.cap, a.ovf);
    else
        k_real_w<0, 0, 1, 1, double><<<grid, 32 * kWarpsPerBlock, 0, a.st>>>(a.pl, a.b0, a.b1, a.k0, a.k1, a.same, a.kchunk,
                                                                                  a.mode, a.tau, a.Dp, a.dmax, a.X, a.Y, a.cnt, a.big,
                                                                                  a.nbig, a.cap, a.ovf);
}

void launch_jeng_q02(const RealLaunch &a)
{
    const int nb = a.b1 - a.b0, nk = a.k1 - a.k0;
    if (nb <= 0 || nk <= 0) return;
    dim3 grid((nb + kRealThreads - 1) / kRealThreads, (nk + a.kchunk - 1) / a.kchunk);
    if (a.fp32)
        k_jeng<0, 0, 1, 1, float><<<grid, kRealThreads, 0, a.st>>>(a.pl, a.b0, a.b1, a.k0, a.k1, a.same, a.kchunk, a.mode,
                                                                           a.tau, a.dmaxf, a.DhF, a.hs, a.X, a.JH, a.cnt, a.big, a.nbig,
                                                                           a.cap, a.ovf);
    else
        k_jeng<0, 0, 1, 1, double><<<grid, kRealThreads, 0, a.st>>>(a.pl, a.b0, a.b1, a.k0, a.k1, a.same, a.kchunk, a.mode,
                                                                            a.tau, a.dmax, a.DhD, a.hs, a.X, a.JH, a.cnt, a.big, a.nbig,
                                                                            a.cap, a.ovf);
}

}  // namespace jk
