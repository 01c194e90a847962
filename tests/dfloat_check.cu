// Host-side check of the double-float arithmetic of the mixed-precision
// structure factors (dfloat.cuh, sfac_df_poly in kernels.cuh): the same
// __host__ __device__ functions the kernel runs, compiled for the CPU and
// compared with long double (phase) and with a plain double evaluation of
// the Hermite polynomial products.  Prints three maxima, one per line.
#include <cmath>
#include <complex>
#include <cstdio>
#include <random>

#include "../paper_2410_22278_gb300/csrc/kernels.cuh"

using namespace jk;
typedef std::complex<double> cd;

static const long double kPiL = 3.141592653589793238462643383279502884L;

// max |cos, sin error| of df_turns + df_sincos_turns over random
// fractional coordinates and reciprocal indices |n_k| <= 64
static long double phase_error(std::mt19937_64 &rng, int trials)
{
    float4 tab[1024];
    for (int k = 0; k < 1024; ++k) {
        const long double t = 2.0L * kPiL * k / 1024.0L, c = cosl(t), s = sinl(t);
        const float ch = (float)c, sh = (float)s;
        tab[k] = make_float4(ch, (float)(c - ch), sh, (float)(s - sh));
    }
    std::uniform_real_distribution<double> U(-4.0, 4.0);
    std::uniform_int_distribution<int> N(-64, 64);
    long double worst = 0;
    for (int it = 0; it < trials; ++it) {
        long double f[3];
        float f1[3], f2[3], f3[3];
        for (int k = 0; k < 3; ++k) {
            f[k] = (long double)U(rng);
            float o[3];
            frac_split3(f[k], o);
            f1[k] = o[0];
            f2[k] = o[1];
            f3[k] = o[2];
        }
        int n[3] = {N(rng), N(rng), N(rng)};
        if (it < 2) n[0] = n[1] = n[2] = it ? 64 : -64;
        dfl w, c, s;
        const int j = df_turns((float)n[0], (float)n[1], (float)n[2], f1, f2, f3, w);
        df_sincos_turns(w, tab[j & 1023], c, s);
        const long double th = 2.0L * kPiL * (n[0] * f[0] + n[1] * f[1] + n[2] * f[2]);
        worst = fmaxl(worst, fabsl((long double)c.hi + c.lo - cosl(th)));
        worst = fmaxl(worst, fabsl((long double)s.hi + s.lo - sinl(th)));
    }
    return worst;
}

static double Eref(int i, int j, int t, double PA, double PB, double oo2p)
{
    if (t < 0 || t > i + j) return 0.0;
    if (i == 0 && j == 0) return t == 0 ? 1.0 : 0.0;
    if (i > 0)
        return oo2p * Eref(i - 1, j, t - 1, PA, PB, oo2p) + PA * Eref(i - 1, j, t, PA, PB, oo2p) + (t + 1) * Eref(i - 1, j, t + 1, PA, PB, oo2p);
    return oo2p * Eref(i, j - 1, t - 1, PA, PB, oo2p) + PB * Eref(i, j - 1, t, PA, PB, oo2p) + (t + 1) * Eref(i, j - 1, t + 1, PA, PB, oo2p);
}

// max relative (to the block's largest element) error of sfac_df_poly
template <int LA, int LB>
static double poly_error(std::mt19937_64 &rng, int trials, bool twice)
{
    constexpr int NA = ncart(LA), NB = ncart(LB), L = LA + LB;
    std::uniform_real_distribution<double> U(-1, 1);
    double worst = 0;
    for (int it = 0; it < trials; ++it) {
        dfl PA[3], PB[3], Gp[3][L + 1];
        double rPA[3], rPB[3], rG[3];
        for (int k = 0; k < 3; ++k) {
            PA[k] = dfl_split(2.5 * U(rng));
            PB[k] = dfl_split(2.5 * U(rng));
            const dfl g = dfl_split(4.5 * U(rng));
            rPA[k] = dfl_value(PA[k]);
            rPB[k] = dfl_value(PB[k]);
            rG[k] = dfl_value(g);
            Gp[k][0] = dfl{1.0f, 0.0f};
            for (int t = 1; t <= L; ++t) Gp[k][t] = t == 1 ? g : df_mul(Gp[k][t - 1], g);
        }
        const dfl oo2p = dfl_split(0.5 / (0.2 + 5 * std::fabs(U(rng)))), pr = dfl_split(U(rng)), pim = dfl_split(U(rng));
        dfl re[NA * NB], im[NA * NB];
        for (int k = 0; k < NA * NB; ++k) re[k] = im[k] = dfl{0.0f, 0.0f};
        sfac_df_poly<LA, LB>(PA, PB, oo2p, Gp, pr, pim, twice, re, im);
        cd ref[NA * NB];
        for (int a = 0; a < NA; ++a)
            for (int b = 0; b < NB; ++b) {
                cd v(dfl_value(pr), dfl_value(pim));
                for (int k = 0; k < 3; ++k) {
                    const int ia = cexp(LA, a, k), jb = cexp(LB, b, k);
                    cd h = 0, pw = 1;
                    for (int t = 0; t <= ia + jb; ++t) {
                        h += Eref(ia, jb, t, rPA[k], rPB[k], dfl_value(oo2p)) * pw;
                        pw *= cd(0, -rG[k]);
                    }
                    v *= h;
                }
                ref[a * NB + b] += v;
                if (twice) ref[b * NB + a] += v;
            }
        double scale = 1e-300;
        for (int k = 0; k < NA * NB; ++k) scale = std::max(scale, std::abs(ref[k]));
        for (int k = 0; k < NA * NB; ++k)
            worst = std::max(worst, std::abs(cd(dfl_value(re[k]), dfl_value(im[k])) - ref[k]) / scale);
    }
    return worst;
}

int main()
{
    std::mt19937_64 rng(2024);
    printf("%.6Le\n", phase_error(rng, 200000));
    double pe = 0;
    pe = std::max(pe, poly_error<1, 0>(rng, 2000, false));
    pe = std::max(pe, poly_error<1, 1>(rng, 2000, true));
    pe = std::max(pe, poly_error<2, 0>(rng, 2000, false));
    pe = std::max(pe, poly_error<2, 1>(rng, 2000, false));
    pe = std::max(pe, poly_error<2, 2>(rng, 1000, true));
    printf("%.6e\n", pe);
    // error-free transformations: two_sum is exact
    std::uniform_real_distribution<double> V(-3, 3);
    long double ts = 0;
    for (int it = 0; it < 100000; ++it) {
        const float a = (float)(V(rng) * std::exp(3 * V(rng))), b = (float)(V(rng) * std::exp(3 * V(rng)));
        const dfl s = two_sum(a, b);
        ts = fmaxl(ts, fabsl(((long double)s.hi + s.lo) - ((long double)a + b)));
    }
    printf("%.6Le\n", ts);
    return 0;
}
