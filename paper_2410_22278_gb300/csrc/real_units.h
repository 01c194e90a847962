// Declarations of the per-class-pair launchers (generated by gen_units.py).
#pragma once
#include "launch.h"

namespace jk {
void launch_real_q00(const RealLaunch &a);
void launch_jeng_q00(const RealLaunch &a);
void launch_real_q01(const RealLaunch &a);
void launch_jeng_q01(const RealLaunch &a);
void launch_real_q02(const RealLaunch &a);
void launch_jeng_q02(const RealLaunch &a);
void launch_real_q03(const RealLaunch &a);
void launch_jeng_q03(const RealLaunch &a);
void launch_real_q04(const RealLaunch &a);
void launch_jeng_q04(const RealLaunch &a);
void launch_real_q05(const RealLaunch &a);
void launch_jeng_q05(const RealLaunch &a);
void launch_real_q11(const RealLaunch &a);
void launch_jeng_q11(const RealLaunch &a);
void launch_real_q12(const RealLaunch &a);
void launch_jeng_q12(const RealLaunch &a);
void launch_real_q13(const RealLaunch &a);
void launch_jeng_q13(const RealLaunch &a);
void launch_real_q14(const RealLaunch &a);
void launch_jeng_q14(const RealLaunch &a);
void launch_real_q15(const RealLaunch &a);
void launch_jeng_q15(const RealLaunch &a);
void launch_real_q22(const RealLaunch &a);
void launch_jeng_q22(const RealLaunch &a);
void launch_real_q23(const RealLaunch &a);
void launch_jeng_q23(const RealLaunch &a);
void launch_real_q24(const RealLaunch &a);
void launch_jeng_q24(const RealLaunch &a);
void launch_real_q25(const RealLaunch &a);
void launch_jeng_q25(const RealLaunch &a);
void launch_real_q33(const RealLaunch &a);
void launch_jeng_q33(const RealLaunch &a);
void launch_real_q34(const RealLaunch &a);
void launch_jeng_q34(const RealLaunch &a);
void launch_real_q35(const RealLaunch &a);
void launch_jeng_q35(const RealLaunch &a);
void launch_real_q44(const RealLaunch &a);
void launch_jeng_q44(const RealLaunch &a);
void launch_real_q45(const RealLaunch &a);
void launch_jeng_q45(const RealLaunch &a);
void launch_real_q55(const RealLaunch &a);
void launch_jeng_q55(const RealLaunch &a);

// class pairs of s and p shells have the warp kernels of real2.cuh as a second family
inline bool real_has_warp_kernel(int cb, int ck) { return cb <= 2 && ck <= 2; }

inline void launch_real(int cb, int ck, const RealLaunch &a)
{
    switch (cb * 8 + ck) {
    case 0: launch_real_q00(a); break;
    case 1: launch_real_q01(a); break;
    case 2: launch_real_q02(a); break;
    case 3: launch_real_q03(a); break;
    case 4: launch_real_q04(a); break;
    case 5: launch_real_q05(a); break;
    case 9: launch_real_q11(a); break;
    case 10: launch_real_q12(a); break;
    case 11: launch_real_q13(a); break;
    case 12: launch_real_q14(a); break;
    case 13: launch_real_q15(a); break;
    case 18: launch_real_q22(a); break;
    case 19: launch_real_q23(a); break;
    case 20: launch_real_q24(a); break;
    case 21: launch_real_q25(a); break;
    case 27: launch_real_q33(a); break;
    case 28: launch_real_q34(a); break;
    case 29: launch_real_q35(a); break;
    case 36: launch_real_q44(a); break;
    case 37: launch_real_q45(a); break;
    case 45: launch_real_q55(a); break;
    default: break;
    }
}

// Coulomb-only builds: the J-engine kernel of a class pair (jeng.cuh)
inline void launch_jeng(int cb, int ck, const RealLaunch &a)
{
    switch (cb * 8 + ck) {
    case 0: launch_jeng_q00(a); break;
    case 1: launch_jeng_q01(a); break;
    case 2: launch_jeng_q02(a); break;
    case 3: launch_jeng_q03(a); break;
    case 4: launch_jeng_q04(a); break;
    case 5: launch_jeng_q05(a); break;
    case 9: launch_jeng_q11(a); break;
    case 10: launch_jeng_q12(a); break;
    case 11: launch_jeng_q13(a); break;
    case 12: launch_jeng_q14(a); break;
    case 13: launch_jeng_q15(a); break;
    case 18: launch_jeng_q22(a); break;
    case 19: launch_jeng_q23(a); break;
    case 20: launch_jeng_q24(a); break;
    case 21: launch_jeng_q25(a); break;
    case 27: launch_jeng_q33(a); break;
    case 28: launch_jeng_q34(a); break;
    case 29: launch_jeng_q35(a); break;
    case 36: launch_jeng_q44(a); break;
    case 37: launch_jeng_q45(a); break;
    case 45: launch_jeng_q55(a); break;
    default: break;
    }
}

}  // namespace jk
