// Algorithmic floating-point operation counts of the real-space quartet
// evaluation, from the loop bounds of the McMurchie-Davidson formulas as the
// kernels evaluate them (Section 2.2: E recursion, R recursion, Hermite
// contraction; Eq. pbc_eri_general_final: the erfc-attenuated seeds).  An add,
// a multiply and a transcendental (exp, log, sqrt, erfc) count one each; a
// fused multiply-add counts two.  Used for the roofline of the real-space
// kernels (work per launch / launch time); the counts are per unit of work
// the kernels tally at run time.
#pragma once

namespace jk {
namespace flops {

constexpr int ncart_(int l) { return (l + 1) * (l + 2) / 2; }
constexpr int nherm_(int L) { return (L + 1) * (L + 2) * (L + 3) / 6; }
constexpr int cexp_(int l, int k, int ax)
{
    int n = 0;
    for (int lx = l; lx >= 0; --lx)
        for (int ly = l - lx; ly >= 0; --ly) {
            if (n == k) return ax == 0 ? lx : (ax == 1 ? ly : l - lx - ly);
            ++n;
        }
    return 0;
}

// one axis of E^{ij}_t for i <= LA, j <= LB
constexpr long long herm_E(int LA, int LB)
{
    long long f = 0;
    for (int i = 0; i <= LA; ++i)
        for (int j = 0; j <= LB; ++j) {
            if (i == 0 && j == 0) continue;
            for (int t = 0; t <= i + j; ++t) {
                f += 1;                          // P-A (or P-B) times E
                if (t > 0) f += 2;               // + E_{t-1} / 2p
                if (t + 1 <= i + j - 1) f += 2;  // + (t+1) E_{t+1}
            }
        }
    return f;
}

// R^0_{tuv}, t+u+v <= L, from the L+1 seeds (in-place recursion)
constexpr long long herm_R(int L)
{
    long long f = 0;
    for (int m = L - 1; m >= 0; --m)
        for (int n = L - m; n >= 1; --n)
            for (int t = n; t >= 0; --t)
                for (int u = n - t; u >= 0; --u) {
                    const int v = n - t - u;
                    const int k = t > 0 ? t : (u > 0 ? u : v);
                    f += 1 + (k > 1 ? 2 : 0);
                }
    return f;
}

// erfc-attenuated seeds (-2a)^m G_m(aX^2, c_w), m <= L (table branch)
constexpr long long seeds(int L) { return 34 + 8 * L + 2 * (L + 1); }

// one lattice image R1 of one primitive quartet: X, |X|^2, seeds, R, sum
constexpr long long per_image(int L) { return 8 + seeds(L) + herm_R(L) + nherm_(L); }

// one primitive quartet with at least one image: screening radius, minimum
// image, ket E, prefactor, Hermite contraction into the Cartesian block
constexpr long long per_prim_quartet(int LA, int LB, int LC, int LD)
{
    long long f = 31 + 45 + 8 + 3 * herm_E(LC, LD) + 6;
    const int LAB = LA + LB;
    for (int c = 0; c < ncart_(LC); ++c)
        for (int d = 0; d < ncart_(LD); ++d) {
            const long long box_cd =
                (long long)(cexp_(LC, c, 0) + cexp_(LD, d, 0) + 1) * (cexp_(LC, c, 1) + cexp_(LD, d, 1) + 1) * (cexp_(LC, c, 2) + cexp_(LD, d, 2) + 1);
            f += nherm_(LAB) * box_cd * 4;
            for (int a = 0; a < ncart_(LA); ++a)
                for (int b = 0; b < ncart_(LB); ++b) {
                    const long long box_ab = (long long)(cexp_(LA, a, 0) + cexp_(LB, b, 0) + 1) * (cexp_(LA, a, 1) + cexp_(LB, b, 1) + 1) *
                                             (cexp_(LA, a, 2) + cexp_(LB, b, 2) + 1);
                    f += box_ab * 4 + 2;
                }
        }
    return f;
}

// screening of one primitive quartet (radius test of Eq. pbc_eri_real_cutoff
// definition before the images: alpha_w, c_w, prefactor, log)
constexpr long long per_prim_screen() { return 16; }

// one bra primitive pair per quartet call (bra E coefficients)
constexpr long long per_bra_prim(int LA, int LB) { return 3 * herm_E(LA, LB) + 1; }

// one image quartet: J (both sides) and K (four index assignments) digestion
constexpr long long per_quartet(int LA, int LB, int LC, int LD)
{
    return 12LL * ncart_(LA) * ncart_(LB) * ncart_(LC) * ncart_(LD) + 4;
}

}  // namespace flops

// Event counts of one thread in a real-space kernel (32-bit, cheap to bump
// in the inner loops), turned into operation counts once per launch:
// algorithmic work (the McMurchie-Davidson steps of each lattice image,
// primitive quartet and image quartet) and screening / bookkeeping (radius
// tests, minimum images, image search, Hermite tables formed again).
struct Tally {
    unsigned screen = 0;  // primitive quartets screened
    unsigned radius = 0;  // of those, radius and minimum image formed (magnitude test passed)
    unsigned cand = 0;    // lattice-vector candidates examined
    unsigned img = 0;     // lattice images evaluated (inside the sphere)
    unsigned term = 0;    // primitive quartets with at least one image, contracted into the block
    unsigned ketp = 0;    // ket Hermite tables formed for a lane
    unsigned brap = 0;    // bra Hermite tables formed
    unsigned quart = 0;   // image quartets digested into J and K
};

template <int LA, int LB, int LC, int LD>
__host__ __device__ constexpr unsigned long long tally_alg(const Tally &t)
{
    return (unsigned long long)t.img * (flops::per_image(LA + LB + LC + LD) - 8) +
           (unsigned long long)t.term * (flops::per_prim_quartet(LA, LB, LC, LD) - 76) +
           (unsigned long long)t.quart * flops::per_quartet(LA, LB, LC, LD);
}
template <int LA, int LB, int LC, int LD>
__host__ __device__ constexpr unsigned long long tally_screen(const Tally &t)
{
    return (unsigned long long)t.screen * flops::per_prim_screen() + (unsigned long long)t.radius * 76 + (unsigned long long)t.cand * 8 +
           (unsigned long long)t.brap * flops::per_bra_prim(LA, LB) + (unsigned long long)t.ketp * 3 * flops::herm_E(LC, LD);
}

}  // namespace jk
