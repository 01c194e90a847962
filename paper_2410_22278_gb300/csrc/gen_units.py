"""Generate one CUDA translation unit per angular class pair of the
real-space kernels (real_q<cb><ck>.cu), so that the 21 instantiations
compile in parallel.  Run from this directory: python gen_units.py"""
CLASSES = [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2)]

# Classes of s and p shells have three tile-kernel families, the
# lane-per-bra kernels of kernels.cuh and the warp and pair-queue kernels of
# real2.cuh, and the autotuner picks one per class pair (RealLaunch::variant); their FP64 list
# pass is the warp kernel.  Classes with a d shell keep the lane-per-bra
# kernels (their Cartesian blocks are too large for a warp-wide segmented
# reduction in registers).
UNIT_W = """// Real-space quartet kernels for bra class {lab} and ket class {lcd} (generated by gen_units.py).
#include "jeng.cuh"
#include "launch.h"
#include "real2.cuh"

namespace jk {{

void launch_real_q{cb}{ck}(const RealLaunch &a)
{{
    const int nb = a.b1 - a.b0, nk = a.k1 - a.k0;
    if (nb <= 0 || nk <= 0) return;
    if (a.list_pass) {{
        k_real_list_w<{la}, {lb}, {lc}, {ld}><<<152 * 8, 32 * kWarpsPerBlock, 0, a.st>>>(a.pl, a.big, a.nbig, a.cap, a.same, a.Dp, a.X, a.Y,
                                                                                  a.cnt64);
        return;
    }}
    if (a.variant == 2) {{
        dim3 grid((nb + kRealThreads - 1) / kRealThreads, (nk + a.kchunk - 1) / a.kchunk);
        if (a.fp32)
            k_real_q<{la}, {lb}, {lc}, {ld}, float><<<grid, kRealThreads, 0, a.st>>>(a.pl, a.b0, a.b1, a.k0, a.k1, a.same, a.kchunk,
                                                                                 a.mode, a.tau, a.Dpf, a.dmaxf, a.X, a.Y, a.cnt, a.big,
                                                                                 a.nbig, a.cap, a.ovf);
        else
            k_real_q<{la}, {lb}, {lc}, {ld}, double><<<grid, kRealThreads, 0, a.st>>>(a.pl, a.b0, a.b1, a.k0, a.k1, a.same, a.kchunk,
                                                                                  a.mode, a.tau, a.Dp, a.dmax, a.X, a.Y, a.cnt, a.big,
                                                                                  a.nbig, a.cap, a.ovf);
        return;
    }}
    if (a.variant == 0) {{
        dim3 grid((nb + kRealThreads - 1) / kRealThreads, (nk + a.kchunk - 1) / a.kchunk);
        if (a.fp32)
            k_real<{la}, {lb}, {lc}, {ld}, float><<<grid, kRealThreads, 0, a.st>>>(a.pl, a.b0, a.b1, a.k0, a.k1, a.same, a.kchunk, a.mode,
                                                                               a.tau, a.Dpf, a.dmaxf, a.X, a.Y, a.cnt, a.big, a.nbig,
                                                                               a.cap, a.ovf);
        else
            k_real<{la}, {lb}, {lc}, {ld}, double><<<grid, kRealThreads, 0, a.st>>>(a.pl, a.b0, a.b1, a.k0, a.k1, a.same, a.kchunk, a.mode,
                                                                                a.tau, a.Dp, a.dmax, a.X, a.Y, a.cnt, a.big, a.nbig,
                                                                                a.cap, a.ovf);
        return;
    }}
    dim3 grid((nb + kWarpsPerBlock - 1) / kWarpsPerBlock, (nk + a.kchunk - 1) / a.kchunk);
    if (a.fp32)
        k_real_w<{la}, {lb}, {lc}, {ld}, float><<<grid, 32 * kWarpsPerBlock, 0, a.st>>>(a.pl, a.b0, a.b1, a.k0, a.k1, a.same, a.kchunk,
                                                                                 a.mode, a.tau, a.Dpf, a.dmaxf, a.X, a.Y, a.cnt, a.big,
                                                                                 a.nbig, a.cap, a.ovf);
    else
        k_real_w<{la}, {lb}, {lc}, {ld}, double><<<grid, 32 * kWarpsPerBlock, 0, a.st>>>(a.pl, a.b0, a.b1, a.k0, a.k1, a.same, a.kchunk,
                                                                                  a.mode, a.tau, a.Dp, a.dmax, a.X, a.Y, a.cnt, a.big,
                                                                                  a.nbig, a.cap, a.ovf);
}}

void launch_jeng_q{cb}{ck}(const RealLaunch &a)
{{
    const int nb = a.b1 - a.b0, nk = a.k1 - a.k0;
    if (nb <= 0 || nk <= 0) return;
    dim3 grid((nb + kRealThreads - 1) / kRealThreads, (nk + a.kchunk - 1) / a.kchunk);
    if (a.fp32)
        k_jeng<{la}, {lb}, {lc}, {ld}, float><<<grid, kRealThreads, 0, a.st>>>(a.pl, a.b0, a.b1, a.k0, a.k1, a.same, a.kchunk, a.mode,
                                                                           a.tau, a.dmaxf, a.DhF, a.hs, a.X, a.JH, a.cnt, a.big, a.nbig,
                                                                           a.cap, a.ovf);
    else
        k_jeng<{la}, {lb}, {lc}, {ld}, double><<<grid, kRealThreads, 0, a.st>>>(a.pl, a.b0, a.b1, a.k0, a.k1, a.same, a.kchunk, a.mode,
                                                                            a.tau, a.dmax, a.DhD, a.hs, a.X, a.JH, a.cnt, a.big, a.nbig,
                                                                            a.cap, a.ovf);
}}

}}  // namespace jk
"""

UNIT = """// Real-space quartet kernels for bra class {lab} and ket class {lcd} (generated by gen_units.py).
#include "jeng.cuh"
#include "kernels.cuh"
#include "launch.h"

namespace jk {{

void launch_real_q{cb}{ck}(const RealLaunch &a)
{{
    const int nb = a.b1 - a.b0, nk = a.k1 - a.k0;
    if (nb <= 0 || nk <= 0) return;
    if (a.list_pass) {{
        k_real_list<{la}, {lb}, {lc}, {ld}><<<152 * 8, kRealThreads, 0, a.st>>>(a.pl, a.big, a.nbig, a.cap, a.same, a.Dp, a.X, a.Y, a.cnt64);
        return;
    }}
    dim3 grid((nb + kRealThreads - 1) / kRealThreads, (nk + a.kchunk - 1) / a.kchunk);
    if (a.fp32)
        k_real<{la}, {lb}, {lc}, {ld}, float><<<grid, kRealThreads, 0, a.st>>>(a.pl, a.b0, a.b1, a.k0, a.k1, a.same, a.kchunk, a.mode, a.tau,
                                                                       a.Dpf, a.dmaxf, a.X, a.Y, a.cnt, a.big, a.nbig, a.cap, a.ovf);
    else
        k_real<{la}, {lb}, {lc}, {ld}, double><<<grid, kRealThreads, 0, a.st>>>(a.pl, a.b0, a.b1, a.k0, a.k1, a.same, a.kchunk, a.mode, a.tau,
                                                                        a.Dp, a.dmax, a.X, a.Y, a.cnt, a.big, a.nbig, a.cap, a.ovf);
}}

void launch_jeng_q{cb}{ck}(const RealLaunch &a)
{{
    const int nb = a.b1 - a.b0, nk = a.k1 - a.k0;
    if (nb <= 0 || nk <= 0) return;
    dim3 grid((nb + kRealThreads - 1) / kRealThreads, (nk + a.kchunk - 1) / a.kchunk);
    if (a.fp32)
        k_jeng<{la}, {lb}, {lc}, {ld}, float><<<grid, kRealThreads, 0, a.st>>>(a.pl, a.b0, a.b1, a.k0, a.k1, a.same, a.kchunk, a.mode,
                                                                           a.tau, a.dmaxf, a.DhF, a.hs, a.X, a.JH, a.cnt, a.big, a.nbig,
                                                                           a.cap, a.ovf);
    else
        k_jeng<{la}, {lb}, {lc}, {ld}, double><<<grid, kRealThreads, 0, a.st>>>(a.pl, a.b0, a.b1, a.k0, a.k1, a.same, a.kchunk, a.mode,
                                                                            a.tau, a.dmax, a.DhD, a.hs, a.X, a.JH, a.cnt, a.big, a.nbig,
                                                                            a.cap, a.ovf);
}}

}}  // namespace jk
"""


def main():
    decls = []
    for cb, (la, lb) in enumerate(CLASSES):
        for ck in range(cb, len(CLASSES)):
            lc, ld = CLASSES[ck]
            unit = UNIT_W if max(la, lb, lc, ld) <= 1 else UNIT
            open("real_q%d%d.cu" % (cb, ck), "w").write(
                unit.format(cb=cb, ck=ck, la=la, lb=lb, lc=lc, ld=ld, lab=(la, lb), lcd=(lc, ld)))
            decls.append((cb, ck))
    with open("real_units.h", "w") as f:
        f.write("// Declarations of the per-class-pair launchers (generated by gen_units.py).\n#pragma once\n#include \"launch.h\"\n\n")
        f.write("namespace jk {\n")
        for cb, ck in decls:
            f.write("void launch_real_q%d%d(const RealLaunch &a);\n" % (cb, ck))
            f.write("void launch_jeng_q%d%d(const RealLaunch &a);\n" % (cb, ck))
        f.write("\n// class pairs of s and p shells have the warp kernels of real2.cuh as a second family\n")
        f.write("inline bool real_has_warp_kernel(int cb, int ck) { return cb <= 2 && ck <= 2; }\n")
        f.write("\ninline void launch_real(int cb, int ck, const RealLaunch &a)\n{\n    switch (cb * 8 + ck) {\n")
        for cb, ck in decls:
            f.write("    case %d: launch_real_q%d%d(a); break;\n" % (cb * 8 + ck, cb, ck))
        f.write("    default: break;\n    }\n}\n\n")
        f.write("// Coulomb-only builds: the J-engine kernel of a class pair (jeng.cuh)\n")
        f.write("inline void launch_jeng(int cb, int ck, const RealLaunch &a)\n{\n    switch (cb * 8 + ck) {\n")
        for cb, ck in decls:
            f.write("    case %d: launch_jeng_q%d%d(a); break;\n" % (cb * 8 + ck, cb, ck))
        f.write("    default: break;\n    }\n}\n\n}  // namespace jk\n")


if __name__ == "__main__":
    main()
