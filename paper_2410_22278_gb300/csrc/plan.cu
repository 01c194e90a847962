// Host plan builder: everything of Sections 3.1, 3.3 and 3.4 of
// arXiv:2410.22278 that happens once per geometry.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>
#include <set>

#include "dfloat.cuh"
#include "plan.h"

namespace jk {

static thread_local std::string g_last_error;
int fail(int status, const std::string &msg)
{
    g_last_error = msg;
    return status;
}
const char *last_error_str() { return g_last_error.c_str(); }

static const double kPi = 3.14159265358979323846;

static void inv3(const double *m, double *o)
{
    double det = m[0] * (m[4] * m[8] - m[5] * m[7]) - m[1] * (m[3] * m[8] - m[5] * m[6]) + m[2] * (m[3] * m[7] - m[4] * m[6]);
    o[0] = (m[4] * m[8] - m[5] * m[7]) / det;
    o[1] = (m[2] * m[7] - m[1] * m[8]) / det;
    o[2] = (m[1] * m[5] - m[2] * m[4]) / det;
    o[3] = (m[5] * m[6] - m[3] * m[8]) / det;
    o[4] = (m[0] * m[8] - m[2] * m[6]) / det;
    o[5] = (m[2] * m[3] - m[0] * m[5]) / det;
    o[6] = (m[3] * m[7] - m[4] * m[6]) / det;
    o[7] = (m[1] * m[6] - m[0] * m[7]) / det;
    o[8] = (m[0] * m[4] - m[1] * m[3]) / det;
}

// r = L^T n for lattice rows L
static inline void lat_point(const double *L, double n0, double n1, double n2, double *r)
{
    for (int k = 0; k < 3; ++k) r[k] = n0 * L[k] + n1 * L[3 + k] + n2 * L[6 + k];
}
static inline void frac(const double *Finv, const double *r, double *f)
{
    for (int i = 0; i < 3; ++i) f[i] = Finv[3 * i] * r[0] + Finv[3 * i + 1] * r[1] + Finv[3 * i + 2] * r[2];
}

// Section 3.3: all lattice vectors R with |R - c| < r.  The bounding cube of
// edge 2r about c is mapped to fractional indices; floor/ceil over its eight
// corners bound a parallelepiped of lattice points, each then tested
// against the sphere.
template <class F>
static void enumerate_sphere(const double *L, const double *Finv, const double *c, double r, F &&visit)
{
    int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
    for (int s = 0; s < 8; ++s) {
        double corner[3] = {c[0] + ((s & 1) ? r : -r), c[1] + ((s & 2) ? r : -r), c[2] + ((s & 4) ? r : -r)}, f[3];
        frac(Finv, corner, f);
        for (int i = 0; i < 3; ++i) {
            lo[i] = std::min(lo[i], (int)std::floor(f[i]));
            hi[i] = std::max(hi[i], (int)std::ceil(f[i]));
        }
    }
    for (int a = lo[0]; a <= hi[0]; ++a)
        for (int b = lo[1]; b <= hi[1]; ++b)
            for (int d = lo[2]; d <= hi[2]; ++d) {
                double R[3];
                lat_point(L, a, b, d, R);
                double dx = R[0] - c[0], dy = R[1] - c[1], dz = R[2] - c[2];
                if (dx * dx + dy * dy + dz * dz < r * r) visit(a, b, d, R);
            }
}

// Eq. local_normalization (radial part) times the contraction coefficients,
// rescaled to unit self-overlap of the local contracted function.
static void normalise_shell(int l, int n, const double *a, const double *c, double *out)
{
    double s = 0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double x = 2.0 * std::sqrt(a[i] * a[j]) / (a[i] + a[j]);
            s += c[i] * c[j] * std::pow(x, l + 1.5);
        }
    double inv = 1.0 / std::sqrt(s);
    for (int i = 0; i < n; ++i) out[i] = c[i] * std::pow(2.0 * a[i] / kPi, 0.75) * std::pow(8.0 * a[i], 0.5 * l) * inv;
}

static double fact_ratio(int i)  // i!/(2i)!
{
    double r = 1;
    for (int k = i + 1; k <= 2 * i; ++k) r /= k;
    return r;
}
static double comp_factor(int lx, int ly, int lz) { return std::sqrt(fact_ratio(lx) * fact_ratio(ly) * fact_ratio(lz)); }
static double comp_factor_max(int l) { return l == 0 ? 1.0 : (l == 1 ? std::sqrt(0.5) : 0.5); }

// Smaller of the radii of Eqs. pbc_eri_pair_cutoff_implementation and
// pbc_eri_cauchy_schwarz_cutoff_implementation; < 0 when either log is <= 0.
static double pair_radius(double a, double b, double cc, double amin, double dR, double dCS)
{
    double p = a + b;
    double x1 = std::sqrt(2.0) * std::pow(kPi, 1.25) * cc / (p * std::sqrt(p + 2.0 * amin) * dR);
    double x2 = std::pow(2.0, 0.25) * std::pow(kPi, 1.25) * cc / (std::pow(p, 1.25) * dCS);
    if (!(x1 > 1.0) || !(x2 > 1.0)) return -1.0;
    return std::min(std::sqrt(p / (a * b) * std::log(x1)), std::sqrt(p / (a * b) * std::log(x2)));
}

static int pair_class(int la, int lb)  // la >= lb
{
    return la * (la + 1) / 2 + lb;
}

// Cartesian exponents of component k of a shell of momentum l (lx
// descending, then ly descending)
static void cart_exps(int l, int k, int *e)
{
    int n = 0;
    for (int lx = l; lx >= 0; --lx)
        for (int ly = l - lx; ly >= 0; --ly) {
            if (n == k) {
                e[0] = lx;
                e[1] = ly;
                e[2] = l - lx - ly;
                return;
            }
            ++n;
        }
    e[0] = e[1] = e[2] = 0;
}

// Host copy of the E recursion (Eqs. E_recursion_i/j, E^{00}_0 = 1), used
// only to bound structure factors when choosing the reciprocal cut-off.
static void herm_E_host(int la, int lb, double PA, double PB, double oo2p, double E[3][3][5])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int t = 0; t < 5; ++t) E[i][j][t] = 0;
    E[0][0][0] = 1;
    for (int i = 0; i <= la; ++i)
        for (int j = 0; j <= lb; ++j) {
            if (!i && !j) continue;
            for (int t = 0; t <= i + j; ++t) {
                const double(*src)[5] = i > 0 ? &E[i - 1][j] : &E[i][j - 1];
                const double X = i > 0 ? PA : PB;
                const int top = i + j - 1;
                double v = X * (*src)[t];
                if (t > 0) v += oo2p * (*src)[t - 1];
                if (t + 1 <= top) v += (t + 1) * (*src)[t + 1];
                E[i][j][t] = v;
            }
        }
}

// Boys function F_m(T), m = 0..mmax, on the host: F_mmax by its convergent
// series e^{-T} sum_k (2T)^k / ((2m+1)(2m+3)...(2m+2k+1)) and downward
// recursion below T = 40; above, F_0 = (1/2) sqrt(pi/T) erf(sqrt T) and
// upward recursion (stable for T > mmax).
static void boys_host(int mmax, double T, double *F)
{
    const double e = std::exp(-T);
    if (T < 40.0) {
        double term = 1.0 / (2 * mmax + 1), sum = term;
        for (int k = 1; k < 600 && term > 1e-18 * sum; ++k) {
            term *= 2.0 * T / (2 * mmax + 2 * k + 1);
            sum += term;
        }
        F[mmax] = e * sum;
        for (int m = mmax - 1; m >= 0; --m) F[m] = (2.0 * T * F[m + 1] + e) / (2 * m + 1);
    } else {
        F[0] = 0.5 * std::sqrt(kPi / T) * std::erf(std::sqrt(T));
        for (int m = 0; m < mmax; ++m) F[m + 1] = ((2 * m + 1) * F[m] - e) / (2.0 * T);
    }
}

// Exact Schwarz factor of one shell-pair image: sqrt of the largest diagonal
// free-space Coulomb integral (ab|ab) over its Cartesian components (with
// their normalisation factors f_a f_b), summed over the image's primitive
// pairs by McMurchie-Davidson (Eqs. E_recursion_*, R_recursion).  Every
// term of the lattice-summed real-space ERI is a free-space integral of a
// translated pair, so |(ab|cd(R))| <= Q_ab Q_cd bounds it term by term.
static double exact_schwarz(int la, int lb, const std::vector<PpiRec> &pv, const double *fa, const double *fb)
{
    const int L = 2 * (la + lb), D = L + 1;
    const int na = (la + 1) * (la + 2) / 2, nb = (lb + 1) * (lb + 2) / 2;
    const int npp = (int)pv.size();
    std::vector<double> E((size_t)npp * 3 * 45);  // [pair][axis][i][j][t]
    for (int i = 0; i < npp; ++i)
        for (int ax = 0; ax < 3; ++ax) {
            double e[3][3][5];
            herm_E_host(la, lb, pv[i].PA[ax], pv[i].PB[ax], 0.5 / pv[i].p, e);
            std::memcpy(&E[((size_t)i * 3 + ax) * 45], e, sizeof e);
        }
    auto Eat = [&](int i, int ax, int a, int b, int t) { return E[((size_t)i * 3 + ax) * 45 + (a * 3 + b) * 5 + t]; };
    std::vector<double> diag((size_t)na * nb, 0.0);
    std::vector<double> R((size_t)D * D * D * D), F(D);
    auto Ridx = [&](int n, int t, int u, int v) -> double & { return R[(((size_t)n * D + t) * D + u) * D + v]; };
    for (int i = 0; i < npp; ++i)
        for (int j = 0; j < npp; ++j) {
            const double p = pv[i].p, q = pv[j].p, alpha = p * q / (p + q);
            const double X[3] = {pv[i].P[0] - pv[j].P[0], pv[i].P[1] - pv[j].P[1], pv[i].P[2] - pv[j].P[2]};
            boys_host(L, alpha * (X[0] * X[0] + X[1] * X[1] + X[2] * X[2]), F.data());
            // R^n_{tuv} for t+u+v <= L - n
            double f = 1.0;
            for (int n = 0; n <= L; ++n) {
                Ridx(n, 0, 0, 0) = f * F[n];
                f *= -2.0 * alpha;
            }
            for (int n = L - 1; n >= 0; --n)
                for (int s = 1; s <= L - n; ++s)
                    for (int t = 0; t <= s; ++t)
                        for (int u = 0; u <= s - t; ++u) {
                            const int v = s - t - u;
                            double r;
                            if (t > 0) r = X[0] * Ridx(n + 1, t - 1, u, v) + (t > 1 ? (t - 1) * Ridx(n + 1, t - 2, u, v) : 0.0);
                            else if (u > 0) r = X[1] * Ridx(n + 1, t, u - 1, v) + (u > 1 ? (u - 1) * Ridx(n + 1, t, u - 2, v) : 0.0);
                            else r = X[2] * Ridx(n + 1, t, u, v - 1) + (v > 1 ? (v - 1) * Ridx(n + 1, t, u, v - 2) : 0.0);
                            Ridx(n, t, u, v) = r;
                        }
            const double pref = 2.0 * std::pow(kPi, 2.5) / (p * q * std::sqrt(p + q)) * pv[i].K * pv[j].K;
            for (int a = 0; a < na; ++a)
                for (int b = 0; b < nb; ++b) {
                    int ea[3], eb[3];
                    cart_exps(la, a, ea);
                    cart_exps(lb, b, eb);
                    double v = 0;
                    for (int t0 = 0; t0 <= ea[0] + eb[0]; ++t0)
                        for (int t1 = 0; t1 <= ea[1] + eb[1]; ++t1)
                            for (int t2 = 0; t2 <= ea[2] + eb[2]; ++t2) {
                                const double et = Eat(i, 0, ea[0], eb[0], t0) * Eat(i, 1, ea[1], eb[1], t1) * Eat(i, 2, ea[2], eb[2], t2);
                                if (et == 0.0) continue;
                                for (int s0 = 0; s0 <= ea[0] + eb[0]; ++s0)
                                    for (int s1 = 0; s1 <= ea[1] + eb[1]; ++s1)
                                        for (int s2 = 0; s2 <= ea[2] + eb[2]; ++s2) {
                                            const double es = Eat(j, 0, ea[0], eb[0], s0) * Eat(j, 1, ea[1], eb[1], s1) *
                                                              Eat(j, 2, ea[2], eb[2], s2);
                                            const double sg = ((s0 + s1 + s2) & 1) ? -1.0 : 1.0;
                                            v += et * es * sg * Ridx(0, t0 + s0, t1 + s1, t2 + s2);
                                        }
                            }
                    diag[(size_t)a * nb + b] += pref * v;
                }
        }
    double m = 0;
    for (int a = 0; a < na; ++a)
        for (int b = 0; b < nb; ++b) m = std::max(m, std::fabs(diag[(size_t)a * nb + b]) * fa[a] * fa[a] * fb[b] * fb[b]);
    return std::sqrt(m);
}

// F_m(T_k) table by the convergent series at the top order and downward
// recursion, in long double.
void boys_table(int ncol, int npts, double inv_step, std::vector<double> &out)
{
    out.assign((size_t)ncol * npts, 0.0);
    for (int k = 0; k < npts; ++k) {
        long double T = (long double)k / (long double)inv_step;
        long double e = expl(-T);
        int M = ncol - 1;
        long double term = 1.0L / (2 * M + 1), sum = term;
        for (int j = 1; j < 100000; ++j) {
            term *= 2.0L * T / (2 * M + 2 * j + 1);
            sum += term;
            if (term < 1e-24L * sum) break;
        }
        long double F = e * sum;
        out[(size_t)k * ncol + M] = (double)F;
        for (int m = M - 1; m >= 0; --m) {
            F = (2.0L * T * F + e) / (2 * m + 1);
            out[(size_t)k * ncol + m] = (double)F;
        }
    }
}

// Squared real-space radius for one primitive quartet: Eq.
// pbc_eri_real_cutoff_implementation, widened for the Hermite polynomial
// growth (2 alpha_w |X|)^L that the s-type derivation leaves out.  Returns
// < 0 when the quartet has no term above delta.
static double realspace_r2(double p, double q, double KK, double omega, double delta, int L)
{
    double alpha = p * q / (p + q);
    double aw = 1.0 / (1.0 / p + 1.0 / q + 1.0 / (omega * omega));
    double cw = std::sqrt(aw / alpha);
    double C = 2.0 * std::pow(kPi, 2.5) / (p * q * std::sqrt(p + q)) * std::fabs(KK) * (1.0 - cw);
    double lg = std::log(C / delta);
    if (lg <= 0) return -1.0;
    double r = std::sqrt(lg / aw);
    for (int it = 0; it < 3; ++it) r = std::sqrt((lg + L * std::log(1.0 + 2.0 * aw * r)) / aw);
    r += L > 0 ? 0.5 + 0.25 * L : 0.0;
    return r * r;
}

PlanDev Plan::dev() const
{
    PlanDev d{};
    d.nbf = nbf;
    d.nshell = nshell;
    d.nspi = (int)spi.size();
    d.nppi = (int)ppi.size();
    d.nspair = (int)spair.size();
    d.shells = d_shells;
    d.spi = d_spi;
    d.kblk = d_kblk;
    d.kblk2 = d_kblk2;
    d.ppi = d_ppi;
    d.spair = d_spair;
    d.spi_order = d_spi_order;
    d.boys = d_boys;
    d.boys_f = d_boys_f;
    d.r1 = d_r1;
    d.ppf = d_ppf;
    d.r1f = d_r1f;
    d.nr1 = (int)(r1.size() / 4);
    d.gvec = d_gvec;
    d.ng = (int)(gvec.size() / 4);
    d.compf = d_compf;
    d.ppi_pidx = d_ppi_pidx;
    d.phase = d_phase;
    d.ppdf = d_ppdf;
    d.gdf = d_gdf;
    d.phasef = d_phasef;
    memcpy(d.L, L, sizeof L);
    memcpy(d.Finv, Finv, sizeof Finv);
    for (int i = 0; i < 9; ++i) {
        d.Lf[i] = (float)L[i];
        d.Finvf[i] = (float)Finv[i];
    }
    d.omega = omega;
    d.inv_omega2 = 1.0 / (omega * omega);
    d.inv_omega2f = (float)d.inv_omega2;
    d.ewald_R = cut.ewald_R;
    // Eq. pbc_eri_real_cutoff_definition bounds one term; a matrix element
    // sums many such terms, so the sphere is drawn at delta_Ewald-R / 10
    // (plus an angular-momentum margin in the kernels).
    d.log_ewald_R = (float)std::log(cut.ewald_R * 1e-1);
    // B_i B_j below this means 2 pi^{5/2} |K_i K_j| / (pq sqrt(p+q)) < delta/10
    d.ppB = d_ppB;
    d.mag_thr = (float)(cut.ewald_R * 1e-1 / (24.739424126 * 1.001));
    d.volume = volume;
    for (int a = 0; a < 3; ++a)
        d.hplane[a] = (float)(1.0 / std::sqrt(Finv[3 * a] * Finv[3 * a] + Finv[3 * a + 1] * Finv[3 * a + 1] + Finv[3 * a + 2] * Finv[3 * a + 2]));
    d.orth = 1;
    for (int a = 0; a < 3; ++a)
        for (int b = a + 1; b < 3; ++b) {
            const double dot = L[3 * a] * L[3 * b] + L[3 * a + 1] * L[3 * b + 1] + L[3 * a + 2] * L[3 * b + 2];
            const double na = std::sqrt(L[3 * a] * L[3 * a] + L[3 * a + 1] * L[3 * a + 1] + L[3 * a + 2] * L[3 * a + 2]);
            const double nb = std::sqrt(L[3 * b] * L[3 * b] + L[3 * b + 1] * L[3 * b + 1] + L[3 * b + 2] * L[3 * b + 2]);
            if (std::fabs(dot) > 1e-12 * na * nb) d.orth = 0;
        }
    return d;
}

template <class T>
static int upload(const std::vector<T> &h, T **d, size_t &bytes)
{
    size_t n = std::max<size_t>(h.size(), 1) * sizeof(T);
    if (cudaMalloc((void **)d, n) != cudaSuccess) return fail(JK_ERR_OOM, "cudaMalloc failed for plan array");
    if (!h.empty() && cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(JK_ERR_CUDA, "cudaMemcpy failed for plan array");
    bytes += n;
    return JK_OK;
}

static int alloc_ws(Plan *P)
{
    Workspace &w = P->ws;
    size_t n2 = (size_t)P->nbf * P->nbf;
    int ng = (int)(P->gvec.size() / 4);
    const bool mixed = P->precision == JK_MIXED;
    if (mixed) {
        w.oz_slices = 5;  // balanced 8-bit digits: about 39 significant bits per operand
        w.npad = (P->nbf + 127) / 128 * 128;
    }
    // per G: the structure-factor slab M and its GEMM partner Z (2 n^2 doubles
    // each) plus, in mixed precision, the BF16 slices of both; ~4 GB in total
    const double per_g = 32.0 * (double)n2 + (mixed ? 4.0 * 2.0 * w.oz_slices * (double)w.npad * w.npad : 0.0);
    double budget = 4.0e9;
    long long gc = (long long)(budget / per_g);
    gc = std::max<long long>(1, std::min<long long>(gc, std::max(ng, 1)));
    gc = std::min<long long>(gc, 4096);
    w.gc = (int)gc;
    if (mixed && ng > 0) {
        // Slices per G chunk.  With balanced 8-bit digits the split-precision
        // error of a chunk's exchange term scales as c 2^{-8S}, c the largest
        // G bound in the chunk (gsize; G sorted by length, so chunks are bands
        // of similar c).  Each chunk gets the fewest slices that keep its error
        // within 1/nchunk of what 5 slices everywhere give in total, so the sum
        // stays within twice that.
        const int nch = (int)((ng + gc - 1) / gc);
        std::vector<double> cch(nch, 0.0);
        for (int g = 0; g < ng; ++g) cch[g / gc] = std::max(cch[g / gc], P->gsize[g]);
        double tot = 0;
        for (double c : cch) tot += c;
        const double allow = std::ldexp(tot, -8 * w.oz_slices) / nch;
        w.chunk_slices.assign(nch, w.oz_slices);
        for (int c = 0; c < nch; ++c)
            for (int S = 1; S < w.oz_slices; ++S)
                if (std::ldexp(cch[c], -8 * S) <= allow) {
                    w.chunk_slices[c] = S;
                    break;
                }
    }
    size_t bytes = 0;
    auto al = [&](double **ptr, size_t count) -> bool {
        if (cudaMalloc((void **)ptr, std::max<size_t>(count, 1) * sizeof(double)) != cudaSuccess) return false;
        bytes += std::max<size_t>(count, 1) * sizeof(double);
        return true;
    };
    bool ok = al(&w.gtab, std::max<size_t>(1, P->pvals.size()) * (size_t)gc) && al(&w.Dp, n2) && al(&w.X, n2) && al(&w.Y, n2) && al(&w.JLR, n2) && al(&w.KLR, n2) && al(&w.T1, n2) &&
              al(&w.T2, n2) && al(&w.M, 2 * (size_t)gc * n2) && al(&w.Z, 2 * (size_t)gc * n2) && al(&w.rho, 2 * (size_t)gc) && al(&w.rho_part, 2 * (size_t)gc * kSlabSplitsMax) &&
              al(&w.dmax, (size_t)P->nshell * P->nshell) && al(&w.scal, 16) && (!mixed || al((double **)&w.Dpf, (n2 + 1) / 2)) &&
              (!mixed || al((double **)&w.dmaxf, ((size_t)P->nshell * P->nshell + 1) / 2));
    {
        // J-engine arrays: stride N_H(2 lmax)
        int lmax = 0;
        for (auto &sh : P->shells) lmax = std::max(lmax, sh.l);
        const int L2 = 2 * lmax;
        w.hs = (L2 + 1) * (L2 + 2) * (L2 + 3) / 6;
        const size_t nh = std::max<size_t>(1, P->ppi.size()) * w.hs;
        ok = ok && al(&w.DhD, nh) && al(&w.JH, nh) && al((double **)&w.DhF, (nh + 1) / 2);
    }
    if (!ok) return fail(JK_ERR_OOM, "cudaMalloc failed for build workspace");
    // the structure-factor kernels write only the entries of shell pairs with
    // images, the same ones for every G; the others must read as zero
    if (cudaMemset(w.M, 0, 2 * (size_t)gc * n2 * sizeof(double)) != cudaSuccess ||
        cudaMemset(w.Z, 0, 2 * (size_t)gc * n2 * sizeof(double)) != cudaSuccess)
        return fail(JK_ERR_CUDA, "cudaMemset failed for the structure-factor slab");
    if (mixed) {
        const size_t sl = (size_t)w.oz_slices * w.npad * w.npad;
        auto alb = [&](__nv_bfloat16 **ptr, size_t count) -> bool {
            if (cudaMalloc((void **)ptr, count * sizeof(__nv_bfloat16)) != cudaSuccess) return false;
            bytes += count * sizeof(__nv_bfloat16);
            return true;
        };
        auto ali = [&](int **ptr, size_t count) -> bool {
            if (cudaMalloc((void **)ptr, count * sizeof(int)) != cudaSuccess) return false;
            bytes += count * sizeof(int);
            return true;
        };
        if (cudaMalloc((void **)&w.gtab2, std::max<size_t>(1, P->pvals.size()) * (size_t)gc * sizeof(float2)) != cudaSuccess)
            return fail(JK_ERR_OOM, "cudaMalloc failed for the double-float Gaussian table");
        bytes += std::max<size_t>(1, P->pvals.size()) * (size_t)gc * sizeof(float2);
        if (!alb(&w.Ms, 2 * (size_t)gc * sl) || !alb(&w.Zs, 2 * (size_t)gc * sl) || !alb(&w.Ds, sl) || !alb(&w.Cs, sl) ||
            !ali(&w.Mex, 2 * (size_t)gc * w.npad) || !ali(&w.Zex, 2 * (size_t)gc * w.npad) || !ali(&w.Dex, w.npad) ||
            !ali(&w.Cex, w.npad))
            return fail(JK_ERR_OOM, "cudaMalloc failed for tensor-core exchange workspace");
        // low-rank form of D: worth it while the padded rank stays within 60%
        // of npad (closed-shell densities have rank n_occ)
        LowRankWs &lr = w.lr;
        lr.rcap = (6 * w.npad / 10) / 128 * 128;
        const size_t rc = (size_t)std::max(lr.rcap, 1);
        if (!al(&lr.Vt, (size_t)P->nbf * rc) || !al(&lr.diag, P->nbf) || !ali(&lr.done_row, P->nbf) || !al(&lr.sgn, rc) ||
            !ali(&lr.rowmap, rc) || !ali(&lr.dyn, 8) || !ali((int **)&lr.bar, 1) || !al(&lr.Ct, rc * P->nbf))
            return fail(JK_ERR_OOM, "cudaMalloc failed for the low-rank factorisation");
        cudaMemset(lr.dyn, 0, 8 * sizeof(int));
    }
    if (cudaMalloc((void **)&w.err, sizeof(unsigned)) != cudaSuccess) return fail(JK_ERR_OOM, "cudaMalloc failed");
    if (cudaMalloc((void **)&w.cnt, kCounters * sizeof(unsigned long long)) != cudaSuccess) return fail(JK_ERR_OOM, "cudaMalloc failed");
    if (P->precision == JK_MIXED) {
        // the FP64 share is a small fraction; the list holds up to 2% of all image quartets (at most 64 Mi entries)
        const long long want = std::min<long long>(std::max<long long>(P->n_quartets / 50, 1 << 20), 64ll << 20);
        w.cap = (unsigned)want;
        if (cudaMalloc((void **)&w.big, sizeof(int2) * w.cap) != cudaSuccess) return fail(JK_ERR_OOM, "cudaMalloc failed for quartet list");
        if (cudaMalloc((void **)&w.nbig, 2 * sizeof(unsigned)) != cudaSuccess) return fail(JK_ERR_OOM, "cudaMalloc failed");
        bytes += sizeof(int2) * w.cap + 2 * sizeof(unsigned);
    }
    cudaMemset(w.err, 0, sizeof(unsigned));
    w.bytes = bytes + sizeof(unsigned) + kCounters * sizeof(unsigned long long);
    if (P->precision == JK_MIXED) return ozaki_setup_tc(P);
    return JK_OK;
}

int build_plan(const jk_cell *cell, const jk_shell *shells, int nshell, double omega, const jk_cutoffs *cut,
               jk_precision precision, int device, Plan **out)
{
    if (!out) return fail(JK_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!cell || !shells || nshell <= 0) return fail(JK_ERR_INVALID, "cell or shells missing");
    if (precision != JK_FP64 && precision != JK_MIXED) return fail(JK_ERR_INVALID, "unknown precision");
    for (int i = 0; i < 9; ++i)
        if (!std::isfinite(cell->lattice[i])) return fail(JK_ERR_INVALID, "lattice not finite");
    for (int s = 0; s < nshell; ++s) {
        const jk_shell &sh = shells[s];
        if (sh.l < 0) return fail(JK_ERR_INVALID, "negative angular momentum");
        if (sh.l > JK_MAXL) return fail(JK_ERR_UNSUPPORTED, "angular momentum above d");
        if (sh.nprim < 1 || sh.nprim > 16) return fail(JK_ERR_INVALID, "nprim outside 1..16");
        if (!sh.exps || !sh.coefs) return fail(JK_ERR_INVALID, "shell arrays missing");
        for (int k = 0; k < sh.nprim; ++k)
            if (!(sh.exps[k] > 0) || !std::isfinite(sh.exps[k]) || !std::isfinite(sh.coefs[k]))
                return fail(JK_ERR_INVALID, "exponent <= 0 or non-finite coefficient");
        for (int k = 0; k < 3; ++k)
            if (!std::isfinite(sh.center[k])) return fail(JK_ERR_INVALID, "centre not finite");
    }
    Plan *P = new Plan();
    for (int i = 0; i < JK_NCLASS_MAX; ++i)
        for (int j = 0; j < JK_NCLASS_MAX; ++j) {
            // untuned: the warp kernels for s and p class pairs, 512 kets per warp
            P->kvariant[i][j] = (i <= 2 && j <= 2) ? 1 : 0;
            P->kchunk[i][j] = (i <= 2 && j <= 2) ? 512 : 32;
        }
    P->device = device;
    P->precision = precision;
    memcpy(P->L, cell->lattice, sizeof P->L);
    {
        double LT[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) LT[3 * i + j] = P->L[3 * j + i];
        double det = P->L[0] * (P->L[4] * P->L[8] - P->L[5] * P->L[7]) - P->L[1] * (P->L[3] * P->L[8] - P->L[5] * P->L[6]) +
                     P->L[2] * (P->L[3] * P->L[7] - P->L[4] * P->L[6]);
        P->volume = std::fabs(det);
        if (!(P->volume > 1e-8)) {
            delete P;
            return fail(JK_ERR_INVALID, "cell volume <= 0");
        }
        inv3(LT, P->Finv);
    }
    const double V = P->volume;
    // Eq. omega_implementation with w = 10 when the caller leaves omega to us
    P->omega = omega > 0 ? omega : std::pow(10.0 * kPi * kPi * kPi / (V * V), 1.0 / 6.0);
    jk_cutoffs c{};
    if (cut) c = *cut;
    if (!(c.pair_R > 0)) c.pair_R = 1e-14;
    if (!(c.pair_cs > 0)) c.pair_cs = 1e-14;
    if (!(c.ewald_R > 0)) c.ewald_R = 1e-14;
    if (!(c.ewald_K > 0)) c.ewald_K = 1e-14;
    // 3e-3 by default, 300 times the paper's switch-over value (Section
    // 3.5): this GPU's FP64 rate is 1/74 of its measured FP32 rate (about 1/2
    // on the paper's GPU); on the 64-water box mixed stays within 7e-9 of FP64
    // in J and K and 3e-9 Ha in E, and within 2.3e-9 of the oracle's rows
    P->mixed_tau = c.mixed_switch > 0 ? c.mixed_switch : 3e-3;
    P->cut = c;

    // ---- shells, normalised coefficients, component factors
    P->nshell = nshell;
    std::vector<double> cn, ex;
    int ao = 0, p0 = 0;
    for (int s = 0; s < nshell; ++s) {
        const jk_shell &sh = shells[s];
        ShellRec r{};
        for (int k = 0; k < 3; ++k) r.c[k] = sh.center[k];
        r.l = sh.l;
        r.nprim = sh.nprim;
        r.p0 = p0;
        r.ao = ao;
        P->shells.push_back(r);
        std::vector<double> tmp(sh.nprim);
        normalise_shell(sh.l, sh.nprim, sh.exps, sh.coefs, tmp.data());
        for (int k = 0; k < sh.nprim; ++k) {
            cn.push_back(tmp[k]);
            ex.push_back(sh.exps[k]);
        }
        for (int lx = sh.l; lx >= 0; --lx)
            for (int ly = sh.l - lx; ly >= 0; --ly) P->compf.push_back(comp_factor(lx, ly, sh.l - lx - ly));
        ao += (sh.l + 1) * (sh.l + 2) / 2;
        p0 += sh.nprim;
    }
    P->nbf = ao;
    const double amin = *std::min_element(ex.begin(), ex.end());

    // ---- unique shell pairs I <= J, their primitive pairs and images
    struct Img {
        int n[3];
        std::vector<std::pair<int, int>> pp;  // (prim of I, prim of J)
    };
    std::vector<SpiRec> spis;
    std::vector<std::vector<PpiRec>> spi_ppis;
    std::vector<std::vector<double2>> spi_ab;  // exponents (a, b) of each primitive pair, same order
    std::vector<double> spi_qx;                // exact Schwarz factor of each image (exact_schwarz)
    const double *L = P->L;
    for (int I = 0; I < nshell; ++I) {
        const ShellRec &sI = P->shells[I];
        for (int J = I; J < nshell; ++J) {
            const ShellRec &sJ = P->shells[J];
            double d[3] = {sI.c[0] - sJ.c[0], sI.c[1] - sJ.c[1], sI.c[2] - sJ.c[2]}, f[3], s[3];
            frac(P->Finv, d, f);
            double nr[3] = {std::round(f[0]), std::round(f[1]), std::round(f[2])};
            lat_point(L, nr[0], nr[1], nr[2], s);
            double dmin[3] = {d[0] - s[0], d[1] - s[1], d[2] - s[2]};  // Eq. lattice_image_min_norm
            std::map<std::array<int, 3>, std::vector<std::pair<int, int>>> imgs;
            double fac = comp_factor_max(sI.l) * comp_factor_max(sJ.l);
            for (int ia = 0; ia < sI.nprim; ++ia)
                for (int ib = 0; ib < sJ.nprim; ++ib) {
                    double a = ex[sI.p0 + ia], b = ex[sJ.p0 + ib];
                    double r = pair_radius(a, b, std::fabs(cn[sI.p0 + ia] * cn[sJ.p0 + ib]) * fac, amin, c.pair_R, c.pair_cs);
                    if (r <= 0) continue;
                    enumerate_sphere(L, P->Finv, dmin, r, [&](int n0, int n1, int n2, const double *) {
                        std::array<int, 3> key = {n0 + (int)nr[0], n1 + (int)nr[1], n2 + (int)nr[2]};
                        imgs[key].push_back({ia, ib});
                    });
                }
            if (imgs.empty()) continue;
            P->n_shell_pairs++;
            {  // ordered counts: (J, I, -R) mirrors (I, J, R) for I != J; for I == J both signs are enumerated
                std::set<std::pair<int, int>> distinct;
                long long nloc = 0;
                for (auto &kv : imgs) {
                    nloc += (long long)kv.second.size();
                    for (auto &pr : kv.second) distinct.insert(pr);
                }
                const int m = I == J ? 1 : 2;
                P->n_ord_shell_pairs += m;
                P->n_ord_prim_pairs += m * (long long)distinct.size();
                P->n_ord_local_pairs += m * nloc;
            }
            // canonical orientation: first shell has the larger l
            bool swap = sI.l < sJ.l;
            int F = swap ? J : I, S = swap ? I : J;
            for (auto &kv : imgs) {
                std::array<int, 3> n = kv.first;
                if (swap) n = {-n[0], -n[1], -n[2]};
                if (I == J) {  // keep R >= 0 lexicographically
                    bool pos = n[0] > 0 || (n[0] == 0 && (n[1] > 0 || (n[1] == 0 && n[2] >= 0)));
                    if (!pos) continue;
                }
                const ShellRec &sF = P->shells[F], &sS = P->shells[S];
                double R[3];
                lat_point(L, n[0], n[1], n[2], R);
                double A[3] = {sF.c[0], sF.c[1], sF.c[2]}, B[3] = {sS.c[0] + R[0], sS.c[1] + R[1], sS.c[2] + R[2]};
                double AB2 = (A[0] - B[0]) * (A[0] - B[0]) + (A[1] - B[1]) * (A[1] - B[1]) + (A[2] - B[2]) * (A[2] - B[2]);
                std::vector<PpiRec> pv;
                std::vector<double2> abv;
                double Q = 0;
                for (auto &pr : kv.second) {
                    int pa = swap ? pr.second : pr.first, pb = swap ? pr.first : pr.second;
                    double a = ex[sF.p0 + pa], b = ex[sS.p0 + pb], p = a + b;
                    PpiRec x{};
                    for (int k = 0; k < 3; ++k) {
                        x.P[k] = (a * A[k] + b * B[k]) / p;
                        x.PA[k] = x.P[k] - A[k];
                        x.PB[k] = x.P[k] - B[k];
                    }
                    x.p = p;
                    x.pad = 1.0 / p;
                    x.K = cn[sF.p0 + pa] * cn[sS.p0 + pb] * std::exp(-a * b / p * AB2);
                    pv.push_back(x);
                    abv.push_back(make_double2(a, b));
                    Q += std::pow(2.0, 0.25) * std::fabs(x.K) * std::pow(kPi / p, 1.25);  // Eq. pbc_eri_cauchy_schwarz_cutoff_definition per primitive
                }
                {
                    std::vector<int> ord(pv.size());
                    std::iota(ord.begin(), ord.end(), 0);
                    // descending B = |K| p^{-5/4}, the separable bound of the
                    // primitive prefactors: loops over primitives stop at the
                    // first pair below the magnitude threshold
                    auto Bof = [&](int u) { return std::fabs(pv[u].K) * std::pow(pv[u].p, -1.25); };
                    std::stable_sort(ord.begin(), ord.end(), [&](int u, int v) { return Bof(u) > Bof(v); });
                    std::vector<PpiRec> pv2;
                    std::vector<double2> ab2;
                    for (int o : ord) {
                        pv2.push_back(pv[o]);
                        ab2.push_back(abv[o]);
                    }
                    pv.swap(pv2);
                    abv.swap(ab2);
                }
                SpiRec sr{};
                sr.I = F;
                sr.J = S;
                sr.npp = (int)pv.size();
                sr.n[0] = n[0];
                sr.n[1] = n[1];
                sr.n[2] = n[2];
                sr.w = (I == J && n[0] == 0 && n[1] == 0 && n[2] == 0) ? 0.5f : 1.0f;
                sr.Q = Q;
                {
                    double fa[6], fb[6];
                    for (int k = 0; k < (sF.l + 1) * (sF.l + 2) / 2; ++k) fa[k] = P->compf[sF.ao + k];
                    for (int k = 0; k < (sS.l + 1) * (sS.l + 2) / 2; ++k) fb[k] = P->compf[sS.ao + k];
                    spi_qx.push_back(exact_schwarz(sF.l, sS.l, pv, fa, fb));
                }
                for (int k = 0; k < 3; ++k) sr.Pc[k] = (float)pv[0].P[k];
                sr.ext = 0.f;
                double Ssum = 0, pmin = 1e300;
                for (auto &x : pv) {
                    double d2 = 0;
                    for (int k = 0; k < 3; ++k) d2 += (x.P[k] - pv[0].P[k]) * (x.P[k] - pv[0].P[k]);
                    sr.ext = std::max(sr.ext, (float)std::sqrt(d2));
                    Ssum += std::fabs(x.K) * std::pow(x.p, -1.25);
                    pmin = std::min(pmin, x.p);
                }
                // rounded up and down respectively, so the float bound stays a bound
                sr.S = (float)(Ssum * (1.0 + 1e-6));
                sr.pmin = (float)(pmin * (1.0 - 1e-6));
                spis.push_back(sr);
                spi_ppis.push_back(std::move(pv));
                spi_ab.push_back(std::move(abv));
            }
        }
    }
    // ---- sort images by class, primitive count and position (Section 3.1 sorts by the Schwarz estimate)
    std::vector<int> order(spis.size());
    std::iota(order.begin(), order.end(), 0);
    auto cls_of = [&](const SpiRec &s) { return pair_class(P->shells[s.I].l, P->shells[s.J].l); };
    // class, then primitive-pair count (lanes of a warp do similar work),
    // then position: Morton order of the image centre in the cell, so that
    // the 32 bras of a warp, and consecutive kets, lie close together and the
    // quartet-level real-space bound rejects the same kets for a whole warp
    std::vector<unsigned long long> morton(spis.size());
    for (size_t i = 0; i < spis.size(); ++i) {
        unsigned long long code = 0;
        unsigned q[3];
        for (int a = 0; a < 3; ++a) {
            double f = 0;
            for (int b = 0; b < 3; ++b) f += P->Finv[3 * a + b] * spis[i].Pc[b];
            f -= std::floor(f);
            q[a] = std::min(1023u, (unsigned)(f * 1024.0));
        }
        for (int bit = 9; bit >= 0; --bit)
            for (int a = 0; a < 3; ++a) code = (code << 1) | ((q[a] >> bit) & 1u);
        morton[i] = code;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        int ca = cls_of(spis[a]), cb = cls_of(spis[b]);
        if (ca != cb) return ca < cb;
        if (spis[a].npp != spis[b].npp) return spis[a].npp > spis[b].npp;
        if (morton[a] != morton[b]) return morton[a] < morton[b];
        return spis[a].Q > spis[b].Q;
    });
    for (int idx : order) {
        SpiRec s = spis[idx];
        s.pp0 = (int)P->ppi.size();
        for (auto &x : spi_ppis[idx]) P->ppi.push_back(x);
        for (auto &e : spi_ab[idx]) P->ppi_ab.push_back(e);
        P->spi.push_back(s);
    }
    for (int cl = 0; cl < JK_NCLASS_MAX; ++cl) {
        ClassRange cr{};
        cr.la = cl == 0 ? 0 : (cl <= 2 ? 1 : 2);
        cr.lb = cl - cr.la * (cr.la + 1) / 2;
        cr.b0 = (int)P->spi.size();
        cr.b1 = 0;
        for (int i = 0; i < (int)P->spi.size(); ++i)
            if (cls_of(P->spi[i]) == cl) {
                cr.b0 = std::min(cr.b0, i);
                cr.b1 = std::max(cr.b1, i + 1);
            }
        if (cr.b1 <= cr.b0) cr.b0 = cr.b1 = 0;
        P->classes.push_back(cr);
    }
    // ---- unique shell pairs with their images (reciprocal-space build), grouped by class
    {
        std::map<std::pair<int, int>, std::vector<int>> byp;
        for (int i = 0; i < (int)P->spi.size(); ++i) byp[{P->spi[i].I, P->spi[i].J}].push_back(i);
        std::vector<std::pair<int, int>> keys;
        for (auto &kv : byp) keys.push_back(kv.first);
        std::stable_sort(keys.begin(), keys.end(), [&](const std::pair<int, int> &a, const std::pair<int, int> &b) {
            return pair_class(P->shells[a.first].l, P->shells[a.second].l) < pair_class(P->shells[b.first].l, P->shells[b.second].l);
        });
        P->spair_class_off.assign(JK_NCLASS_MAX + 1, 0);
        for (auto &k : keys) {
            SpairRec r{};
            r.I = k.first;
            r.J = k.second;
            r.spi0 = (int)P->spi_order.size();
            for (int i : byp[k]) {
                P->spi[i].spair = (int)P->spair.size();
                P->spi_order.push_back(i);
            }
            r.nspi = (int)P->spi_order.size() - r.spi0;
            P->spair_class_off[pair_class(P->shells[r.I].l, P->shells[r.J].l) + 1]++;
            P->spair.push_back(r);
        }
        for (int i = 0; i < JK_NCLASS_MAX; ++i) P->spair_class_off[i + 1] += P->spair_class_off[i];
    }
    // ---- quartet counts (unique pairs of images): Schwarz-significant ones
    // by the exact factors (the quartets/s unit), and the FP64 share the
    // mixed policy would take by the Eq. pbc_eri_cauchy_schwarz_cutoff_definition estimates
    {
        long long N = (long long)P->spi.size();
        P->n_quartets = N * (N + 1) / 2;
        auto count_pairs = [N](std::vector<double> q, double thr) {
            std::sort(q.begin(), q.end(), std::greater<double>());
            long long cnt = 0, j = N - 1;
            for (long long i = 0; i < N; ++i) {
                while (j >= i && q[i] * q[j] < thr) --j;
                if (j >= i) cnt += j - i + 1;
            }
            return cnt;
        };
        std::vector<double> q(N);
        for (long long i = 0; i < N; ++i) q[i] = P->spi[i].Q;
        P->n_quartets_schwarz = count_pairs(spi_qx, c.pair_cs);
        P->n_quartets_fp64 = precision == JK_FP64 ? P->n_quartets : count_pairs(q, P->mixed_tau);
    }
    // ---- R1 candidates for the real-space sums (Section 3.3)
    {
        std::map<double, double> kmax;  // pair exponent -> largest |K|
        int lpmax = 0;
        for (auto &s : P->spi) lpmax = std::max(lpmax, P->shells[s.I].l + P->shells[s.J].l);
        for (auto &x : P->ppi) {
            double &v = kmax[x.p];
            v = std::max(v, std::fabs(x.K));
        }
        double rmax = 0;
        for (auto &u : kmax)
            for (auto &v : kmax) {
                double r2 = realspace_r2(u.first, v.first, u.second * v.second, P->omega, c.ewald_R * 1e-1, 2 * lpmax);
                if (r2 > 0) rmax = std::max(rmax, std::sqrt(r2));
            }
        P->r1_max = rmax;
        double half = 0;
        for (int s = 0; s < 8; ++s) {
            double v[3];
            lat_point(L, (s & 1) ? 0.5 : -0.5, (s & 2) ? 0.5 : -0.5, (s & 4) ? 0.5 : -0.5, v);
            half = std::max(half, std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]));
        }
        double zero[3] = {0, 0, 0};
        std::vector<std::array<double, 4>> cand;
        enumerate_sphere(L, P->Finv, zero, rmax + half + 1e-9, [&](int, int, int, const double *R) {
            cand.push_back({R[0], R[1], R[2], std::sqrt(R[0] * R[0] + R[1] * R[1] + R[2] * R[2])});
        });
        std::sort(cand.begin(), cand.end(), [](const std::array<double, 4> &a, const std::array<double, 4> &b) { return a[3] < b[3]; });
        for (auto &v : cand)
            for (int k = 0; k < 4; ++k) P->r1.push_back(v[k]);
    }
    // ---- reciprocal vectors: half space, |G| < G_max from Eq.
    // pbc_eri_reciprocal_cutoff_definition written per pair density,
    // (4 pi/(V Kmin^2)) e^{-G^2/4w^2} s(G)^2 max(1,G)^{2Lp} > delta_K,
    // s(G) = max_pairs |K| (pi/p)^{3/2} e^{-G^2/4p}.
    {
        double B[9];
        for (int i = 0; i < 9; ++i) B[i] = 2.0 * kPi * P->Finv[i];  // rows b_i
        double kmin = 1e300;
        for (int a = -2; a <= 2; ++a)
            for (int b = -2; b <= 2; ++b)
                for (int d = -2; d <= 2; ++d) {
                    if (!a && !b && !d) continue;
                    double g[3];
                    lat_point(B, a, b, d, g);
                    kmin = std::min(kmin, std::sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]));
                }
        // per distinct pair exponent p: the largest amplitude |K| (pi/p)^{3/2}
        // and, per (i, j, t), the largest |E^{ij}_t| over its pairs and axes, so
        // that |rho_ab(G)| <= amp e^{-G^2/4p} prod_axis sum_t |E^{ij}_t| G^t
        struct PBound {
            double amp = 0;
            double E[3][3][5] = {};
            int la = 0, lb = 0;
        };
        std::map<double, PBound> pb;
        for (auto &s : P->spi) {
            const int la = P->shells[s.I].l, lb = P->shells[s.J].l;
            for (int k = s.pp0; k < s.pp0 + s.npp; ++k) {
                const PpiRec &x = P->ppi[k];
                PBound &b = pb[x.p];
                b.amp = std::max(b.amp, std::fabs(x.K) * std::pow(kPi / x.p, 1.5));
                b.la = std::max(b.la, la);
                b.lb = std::max(b.lb, lb);
                for (int ax = 0; ax < 3; ++ax) {
                    double E[3][3][5];
                    herm_E_host(la, lb, x.PA[ax], x.PB[ax], 0.5 / x.p, E);
                    for (int i = 0; i <= la; ++i)
                        for (int j = 0; j <= lb; ++j)
                            for (int t = 0; t <= i + j; ++t) b.E[i][j][t] = std::max(b.E[i][j][t], std::fabs(E[i][j][t]));
                }
            }
        }
        auto sbound = [&](double G) {
            double s = 0;
            for (auto &u : pb) {
                const PBound &b = u.second;
                double poly = 0;  // max over component pairs of the product of axis polynomials
                for (int a = 0; a < (b.la + 1) * (b.la + 2) / 2; ++a)
                    for (int c = 0; c < (b.lb + 1) * (b.lb + 2) / 2; ++c) {
                        int ea[3], eb[3];
                        cart_exps(b.la, a, ea);
                        cart_exps(b.lb, c, eb);
                        double pr = 1;
                        for (int ax = 0; ax < 3; ++ax) {
                            double q = 0, gp = 1;
                            for (int t = 0; t <= ea[ax] + eb[ax]; ++t, gp *= G) q += b.E[ea[ax]][eb[ax]][t] * gp;
                            pr *= q;
                        }
                        poly = std::max(poly, pr);
                    }
                s = std::max(s, b.amp * std::exp(-G * G / (4.0 * u.first)) * poly);
            }
            return s;
        };
        // size of the largest reciprocal term at |G|: (4 pi / V) e^{-G^2/4w^2}/G^2 s(G)^2
        double gmax = kmin;
        for (double G = kmin; G < 40.0 * P->omega + 20.0; G += 0.005 + 0.002 * G) {
            const double s = sbound(G);
            const double wgt = 4.0 * kPi / V * std::exp(-G * G / (4.0 * P->omega * P->omega)) / (G * G) * s * s;
            if (wgt > c.ewald_K * 1e-2) gmax = G;  // per-term bound; a matrix element sums many G
        }
        P->g_max = gmax;
        double zero[3] = {0, 0, 0}, BT[9], BF[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) BT[3 * i + j] = B[3 * j + i];
        inv3(BT, BF);
        std::vector<std::array<double, 4>> gl;
        enumerate_sphere(B, BF, zero, gmax, [&](int a, int b, int d, const double *g) {
            bool pos = a > 0 || (a == 0 && (b > 0 || (b == 0 && d > 0)));
            if (!pos) return;
            double g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
            double w = std::exp(-g2 / (4.0 * P->omega * P->omega)) / g2;
            gl.push_back({g[0], g[1], g[2], std::sqrt(8.0 * kPi * w / V)});
        });
        std::sort(gl.begin(), gl.end(), [](const std::array<double, 4> &a, const std::array<double, 4> &b) {
            return a[0] * a[0] + a[1] * a[1] + a[2] * a[2] < b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
        });
        for (auto &v : gl) {
            for (int k = 0; k < 4; ++k) P->gvec.push_back(v[k]);
            const double G2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2], sg = sbound(std::sqrt(G2));
            P->gsize.push_back(4.0 * kPi / V * std::exp(-G2 / (4.0 * P->omega * P->omega)) / G2 * sg * sg);
        }
    }
    *out = P;
    return JK_OK;
}

// Device side of plan creation: uploads, Boys tables, workspace, overlap.
int finish_plan_device(Plan *P)
{
    if (cudaSetDevice(P->device) != cudaSuccess) return fail(JK_ERR_CUDA, "cudaSetDevice failed");
    int rc;
    size_t &b = P->device_bytes;
    {
        // bounding spheres of blocks of 32 consecutive images (in the kernels'
        // ket order): members are moved next to the block's first image by the
        // minimum image (the lattice distance to any bra is unchanged), then
        // centre = mean, radius = max |Pc - centre| + ext
        const int nsp = (int)P->spi.size(), nblk = (nsp + 31) / 32;
        std::vector<float4> kb(std::max(nblk, 1));
        std::vector<float2> kb2(std::max(nblk, 1));
        for (int bl = 0; bl < nblk; ++bl) {
            const int i0 = 32 * bl, i1 = std::min(nsp, i0 + 32);
            std::vector<std::array<double, 3>> q;
            double c[3] = {0, 0, 0}, smax = 0, pmin = 1e300;
            for (int i = i0; i < i1; ++i) {
                double d[3], f[3];
                for (int k = 0; k < 3; ++k) d[k] = (double)P->spi[i].Pc[k] - (double)P->spi[i0].Pc[k];
                for (int a = 0; a < 3; ++a) f[a] = std::rint(P->Finv[3 * a] * d[0] + P->Finv[3 * a + 1] * d[1] + P->Finv[3 * a + 2] * d[2]);
                std::array<double, 3> x;
                for (int k = 0; k < 3; ++k) x[k] = (double)P->spi[i0].Pc[k] + d[k] - (f[0] * P->L[k] + f[1] * P->L[3 + k] + f[2] * P->L[6 + k]);
                q.push_back(x);
                for (int k = 0; k < 3; ++k) c[k] += x[k] / (i1 - i0);
                smax = std::max(smax, (double)P->spi[i].S);
                pmin = std::min(pmin, (double)P->spi[i].pmin);
            }
            double rad = 0;
            for (int i = i0; i < i1; ++i) {
                const auto &x = q[i - i0];
                const double r = std::sqrt((x[0] - c[0]) * (x[0] - c[0]) + (x[1] - c[1]) * (x[1] - c[1]) + (x[2] - c[2]) * (x[2] - c[2]));
                rad = std::max(rad, r + (double)P->spi[i].ext);
            }
            kb[bl] = make_float4((float)c[0], (float)c[1], (float)c[2], (float)(rad * (1 + 1e-6) + 1e-4));
            kb2[bl] = make_float2((float)smax, (float)pmin);
        }
        if ((rc = upload(kb, &P->d_kblk, b)) || (rc = upload(kb2, &P->d_kblk2, b))) return rc;
    }
    if ((rc = upload(P->shells, &P->d_shells, b)) || (rc = upload(P->spi, &P->d_spi, b)) || (rc = upload(P->ppi, &P->d_ppi, b)) ||
        (rc = upload(P->spair, &P->d_spair, b)) || (rc = upload(P->spi_order, &P->d_spi_order, b)) ||
        (rc = upload(P->r1, &P->d_r1, b)) || (rc = upload(P->gvec, &P->d_gvec, b)) || (rc = upload(P->compf, &P->d_compf, b)))
        return rc;
    {
        std::vector<PpiF> pf(P->ppi.size());
        for (size_t i = 0; i < P->ppi.size(); ++i) {
            const PpiRec &x = P->ppi[i];
            for (int k = 0; k < 3; ++k) {
                pf[i].P[k] = (float)x.P[k];
                pf[i].PA[k] = (float)x.PA[k];
                pf[i].PB[k] = (float)x.PB[k];
            }
            pf[i].p = (float)x.p;
            pf[i].K = (float)x.K;
            pf[i].pad = (float)(1.0 / x.p);
        }
        // B = |K| p^{-5/4} per primitive pair, rounded up so that the float
        // bound stays a bound
        std::vector<float> pB(P->ppi.size());
        for (size_t i = 0; i < P->ppi.size(); ++i)
            pB[i] = (float)(std::fabs(P->ppi[i].K) * std::pow(P->ppi[i].p, -1.25) * (1.0 + 1e-6));
        std::vector<float> r1f(P->r1.begin(), P->r1.end());
        if ((rc = upload(pf, &P->d_ppf, b)) || (rc = upload(r1f, &P->d_r1f, b)) || (rc = upload(pB, &P->d_ppB, b))) return rc;
    }
    std::vector<double> tab;
    boys_table(JK_BOYS_MCOL, JK_BOYS_NPTS, JK_BOYS_INV_STEP, tab);
    std::vector<float> tabf(tab.begin(), tab.end());
    if ((rc = upload(tab, &P->d_boys, b)) || (rc = upload(tabf, &P->d_boys_f, b))) return rc;
    std::vector<double> g0 = {0.0, 0.0, 0.0, 1.0};
    if ((rc = upload(g0, &P->d_g0, b))) return rc;
    {
        // distinct pair exponents (exact equality) and each primitive pair's index
        std::map<double, int> pid;
        for (auto &x : P->ppi) pid.emplace(x.p, 0);
        P->pvals.clear();
        for (auto &kv : pid) {
            kv.second = (int)P->pvals.size();
            P->pvals.push_back(kv.first);
        }
        P->ppi_pidx.resize(P->ppi.size());
        for (size_t i = 0; i < P->ppi.size(); ++i) P->ppi_pidx[i] = pid[P->ppi[i].p];
        std::vector<double> gt0(P->pvals.size());
        for (size_t i = 0; i < gt0.size(); ++i) gt0[i] = std::pow(kPi / P->pvals[i], 1.5);
        // phase table, rounded from extended precision
        std::vector<double2> ph(1024);
        for (int k = 0; k < 1024; ++k) {
            const long double t = 2.0L * 3.141592653589793238462643383279502884L * k / 1024.0L;
            ph[k] = make_double2((double)std::cos(t), (double)std::sin(t));
        }
        if ((rc = upload(P->ppi_ab, &P->d_ppi_ab, b))) return rc;
        if ((rc = upload(P->pvals, &P->d_pvals, b)) || (rc = upload(P->ppi_pidx, &P->d_ppi_pidx, b)) || (rc = upload(gt0, &P->d_gtab0, b)) ||
            (rc = upload(ph, &P->d_phase, b)))
            return rc;
        // double-float tables of the mixed-precision structure factors
        std::vector<float4> phf(1024);
        for (int k = 0; k < 1024; ++k) {
            const long double t = 2.0L * 3.141592653589793238462643383279502884L * k / 1024.0L;
            const long double c = std::cos(t), sn = std::sin(t);
            const float ch = (float)c, sh = (float)sn;
            phf[k] = make_float4(ch, (float)(c - ch), sh, (float)(sn - sh));
        }
        const int ng = (int)(P->gvec.size() / 4);
        std::vector<float4> gd(3 * (size_t)std::max(ng, 1));
        bool ok = true;
        for (int g = 0; g < ng; ++g) {
            const double *G = &P->gvec[4 * (size_t)g];
            float nk[3];
            for (int k = 0; k < 3; ++k) {
                // n_k = a_k . G / 2 pi (an integer for a reciprocal-lattice vector)
                const double v = (P->L[3 * k] * G[0] + P->L[3 * k + 1] * G[1] + P->L[3 * k + 2] * G[2]) / (2.0 * kPi);
                const double r = std::rint(v);
                if (std::fabs(v - r) > 1e-6 || std::fabs(r) > 64) ok = false;
                nk[k] = (float)r;
            }
            const dfl gx = dfl_split(G[0]), gy = dfl_split(G[1]), gz = dfl_split(G[2]);
            gd[3 * (size_t)g] = make_float4(nk[0], nk[1], nk[2], 0.0f);
            gd[3 * (size_t)g + 1] = make_float4(gx.hi, gx.lo, gy.hi, gy.lo);
            gd[3 * (size_t)g + 2] = make_float4(gz.hi, gz.lo, 0.0f, 0.0f);
        }
        std::vector<PpiDF> pd(std::max<size_t>(P->ppi.size(), 1));
        for (size_t i = 0; i < P->ppi.size(); ++i) {
            const PpiRec &x = P->ppi[i];
            float f[3][3];
            for (int k = 0; k < 3; ++k) {
                const long double fk = (long double)P->Finv[3 * k] * x.P[0] + (long double)P->Finv[3 * k + 1] * x.P[1] +
                                       (long double)P->Finv[3 * k + 2] * x.P[2];
                frac_split3(fk, f[k]);
            }
            const dfl K = dfl_split(x.K), oo2p = dfl_split(0.5 / x.p);
            dfl pa[3], pb[3];
            for (int k = 0; k < 3; ++k) {
                pa[k] = dfl_split(x.PA[k]);
                pb[k] = dfl_split(x.PB[k]);
            }
            int pidx = P->ppi_pidx[i];
            float pidx_bits;
            memcpy(&pidx_bits, &pidx, sizeof pidx);
            PpiDF &o = pd[i];
            o.a = make_float4(f[0][0], f[1][0], f[2][0], K.hi);
            o.b = make_float4(f[0][1], f[1][1], f[2][1], K.lo);
            o.c = make_float4(f[0][2], f[1][2], f[2][2], pidx_bits);
            o.d = make_float4(pa[0].hi, pa[0].lo, pa[1].hi, pa[1].lo);
            o.e = make_float4(pa[2].hi, pa[2].lo, pb[0].hi, pb[0].lo);
            o.f = make_float4(pb[1].hi, pb[1].lo, pb[2].hi, pb[2].lo);
            o.g = make_float4(oo2p.hi, oo2p.lo, 0.0f, 0.0f);
        }
        P->sfac_df = ok;
        if ((rc = upload(phf, &P->d_phasef, b)) || (rc = upload(gd, &P->d_gdf, b)) || (rc = upload(pd, &P->d_ppdf, b))) return rc;
    }
    std::vector<double> zeros((size_t)P->nbf * P->nbf, 0.0);
    if ((rc = upload(zeros, &P->d_S, b))) return rc;
    if ((rc = alloc_ws(P))) return rc;
    if ((rc = compute_overlap_raw(P, 0))) return rc;
    if (cudaDeviceSynchronize() != cudaSuccess) return fail(JK_ERR_CUDA, "plan setup kernels failed");
    return JK_OK;
}

void destroy_plan(Plan *P)
{
    if (!P) return;
    cudaSetDevice(P->device);
    release_cache(P);
    void *ptrs[] = {P->d_shells, P->d_spi, P->d_ppi, P->d_ppf, P->d_ppB, P->d_r1f, P->d_spair, P->d_spi_order, P->d_boys, P->d_boys_f, P->d_r1, P->d_gvec,
                    P->d_g0, P->d_compf, P->d_ppi_ab, P->d_kblk, P->d_kblk2, P->d_pvals, P->d_gtab0, P->d_ppi_pidx, P->d_phase, P->d_ppdf, P->d_gdf, P->d_phasef, P->ws.gtab, P->ws.gtab2, P->d_S, P->ws.Dp, P->ws.X, P->ws.Y, P->ws.JLR, P->ws.KLR, P->ws.T1, P->ws.T2,
                    P->ws.M, P->ws.Z, P->ws.rho, P->ws.rho_part, P->ws.DhD, P->ws.JH, P->ws.DhF, P->ws.dmax, P->ws.scal, P->ws.err, P->ws.cnt, P->ws.big, P->ws.nbig,
                    P->ws.Ms, P->ws.Zs, P->ws.Ds, P->ws.Mex, P->ws.Zex, P->ws.Dex, P->ws.Dpf, P->ws.dmaxf, P->ws.Cs, P->ws.Cex, P->ws.Kpart,
                    P->ws.lr.Vt, P->ws.lr.diag, P->ws.lr.done_row, P->ws.lr.sgn, P->ws.lr.rowmap, P->ws.lr.dyn, P->ws.lr.bar, P->ws.lr.Ct};
    for (void *p : ptrs)
        if (p) cudaFree(p);

    P->timer.destroy();
    delete P;
}

// Point-charge Ewald energy (Eq. nuclear_repulsion_energy) on the host.
double ewald_point_charges_host(const double *lat, int n, const double *q, const double *xyz, double omega, double delta)
{
    double LT[9], Finv[9], B[9], BF[9], BT[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) LT[3 * i + j] = lat[3 * j + i];
    inv3(LT, Finv);
    double V = std::fabs(lat[0] * (lat[4] * lat[8] - lat[5] * lat[7]) - lat[1] * (lat[3] * lat[8] - lat[5] * lat[6]) +
                         lat[2] * (lat[3] * lat[7] - lat[4] * lat[6]));
    for (int i = 0; i < 9; ++i) B[i] = 2.0 * kPi * Finv[i];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) BT[3 * i + j] = B[3 * j + i];
    inv3(BT, BF);
    // radii of Eqs. nuclear_repulsion_energy_real_cutoff / _reciprocal_cutoff, solved by bisection
    auto solve = [](auto f) {
        double lo = 1e-3, hi = 1.0;
        while (f(hi) > 0) hi *= 2;
        for (int it = 0; it < 200; ++it) {
            double mid = 0.5 * (lo + hi);
            (f(mid) > 0 ? lo : hi) = mid;
        }
        return hi;
    };
    double rb = solve([&](double r) { return 2.0 / std::sqrt(kPi) * std::exp(-omega * omega * r * r) / (r * r) - delta; });
    double kb = solve([&](double k) { return 4.0 * kPi / V * std::exp(-k * k / (4.0 * omega * omega)) / (k * k) - delta; });
    double E = 0;
    for (int a = 0; a < n; ++a)
        for (int bb = a; bb < n; ++bb) {
            double d[3] = {xyz[3 * a] - xyz[3 * bb], xyz[3 * a + 1] - xyz[3 * bb + 1], xyz[3 * a + 2] - xyz[3 * bb + 2]};
            double nd[3] = {-d[0], -d[1], -d[2]};
            double real = 0, recip = 0;
            enumerate_sphere(lat, Finv, nd, rb, [&](int i, int j, int k, const double *R) {
                if (a == bb && !i && !j && !k) return;
                double x = d[0] + R[0], y = d[1] + R[1], z = d[2] + R[2];
                double r = std::sqrt(x * x + y * y + z * z);
                real += std::erfc(omega * r) / r;
            });
            double zero[3] = {0, 0, 0};
            enumerate_sphere(B, BF, zero, kb, [&](int i, int j, int k, const double *G) {
                if (!i && !j && !k) return;
                double g2 = G[0] * G[0] + G[1] * G[1] + G[2] * G[2];
                recip += std::exp(-g2 / (4.0 * omega * omega)) / g2 * std::cos(G[0] * d[0] + G[1] * d[1] + G[2] * d[2]);
            });
            double term = 4.0 * kPi / V * recip - kPi / (V * omega * omega) + real;
            if (a == bb)
                E += 0.5 * q[a] * q[a] * (term - 2.0 * omega / std::sqrt(kPi));
            else
                E += q[a] * q[bb] * term;
        }
    return E;
}

}  // namespace jk
