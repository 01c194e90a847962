/*
 * Plain FP64 CPU oracle for the Gamma-point periodic J/K build with
 * Ewald-split electron repulsion integrals (Wang, Hait, Unzueta, Zhang,
 * Martinez, arXiv:2410.22278).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file; only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code with the CUDA path.
 *
 * It is deliberately slow and direct:
 *   - ordered shell pairs, no permutational symmetry, no quartet screening;
 *   - Ewald sums truncated far past the GPU's thresholds (delta 1e-18 plus a
 *     distance margin), so that the only truncation it shares with the GPU
 *     is the pair list, whose definition (Eqs. pbc_eri_pair_cutoff_implementation / pbc_eri_cauchy_schwarz_cutoff_implementation) defines the object;
 *   - the real-space (erfc) part follows Eq. pbc_eri_general_final term by
 *     term: McMurchie-Davidson E coefficients (Eqs. E_recursion_*), the
 *     attenuated Boys seeds of Eq. boys_function_split and the R recursion
 *     (Eq. R_recursion), summed over every R1 image;
 *   - the reciprocal (erf) part is the Poisson-summed Coulomb energy of the
 *     Bloch-summed AO pair densities, (4 pi / V) sum_{G != 0}
 *     exp(-G^2/4w^2)/G^2 Re[conj(rho_mn(G)) rho_ls(G)], where each pair
 *     density's Fourier transform is evaluated by binomial expansion about the
 *     Gaussian product centre and Gaussian moments with a complex shift
 *     (not through Hermite E coefficients), i.e. an independent route to the
 *     same term of Eq. pbc_eri_general_final;
 *   - the removed K = 0 (background) term is -(pi/(V w^2)) S_mn S_ls, the
 *     closed form of the last term of Eq. pbc_eri_general_final summed over
 *     images, with S the pair-list-truncated Gamma overlap (Eq.
 *     pbc_overlap_formula) from the same Fourier route at G = 0.
 *
 * Conventions: atomic units; lattice rows a, b, c; Cartesian components in
 * the order lx descending then ly descending (p: x y z; d: xx xy xz yy yz
 * zz); AO index runs over shells in input order.
 */
#include <complex.h>
#undef I /* shell indices are called I, J below; the imaginary unit is _Complex_I */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXL 2
#define ORC_MAXLT (4 * ORC_MAXL)
#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* Boys function F_m(T) = int_0^1 t^{2m} exp(-T t^2) dt  (Eq. R_recursion
 * seeds; F_0 closed form Eq. boys_function_erf_form).  For T <= 60 the
 * highest order is summed from the convergent series
 *   F_m(T) = exp(-T) sum_k (2T)^k / ((2m+1)(2m+3)...(2m+2k+1))
 * and lower orders follow by downward recursion
 *   F_m = (2T F_{m+1} + exp(-T)) / (2m+1);
 * for T > 60, F_0 from the erf form and upward recursion
 *   F_{m+1} = ((2m+1) F_m - exp(-T)) / (2T), which is stable there.    */
void orc_boys(int mmax, double T, double *F)
{
    if (T <= 0.0) {
        for (int m = 0; m <= mmax; m++) F[m] = 1.0 / (2 * m + 1);
        return;
    }
    double e = exp(-T);
    if (T > 60.0) {
        F[0] = 0.5 * sqrt(ORC_PI / T) * erf(sqrt(T));
        for (int m = 0; m < mmax; m++) F[m + 1] = ((2 * m + 1) * F[m] - e) / (2.0 * T);
        return;
    }
    double term = 1.0 / (2 * mmax + 1), sum = term;
    for (int k = 1; k < 4000; k++) {
        term *= 2.0 * T / (2 * mmax + 2 * k + 1);
        sum += term;
        if (term < 1e-18 * sum) break;
    }
    F[mmax] = e * sum;
    for (int m = mmax - 1; m >= 0; m--) F[m] = (2.0 * T * F[m + 1] + e) / (2 * m + 1);
}

/* ------------------------------------------------------------------ */
/* Basis description handed in by the Python wrapper.                  */
typedef struct {
    int nshell;
    const int *l, *nprim, *poff;
    const double *exps, *coefs, *centers; /* raw coefficients */
    double lat[9];                        /* rows a, b, c */
    double omega;                         /* 0: bare Coulomb, inf: reciprocal only */
    double pair_R, pair_cs;               /* pair-list thresholds (Eqs. pbc_eri_pair_cutoff_implementation, pbc_eri_cauchy_schwarz_cutoff_implementation) */
    double delta;                         /* Ewald truncation used by the oracle */
    double margin;                        /* extra real-space radius, bohr */
} orc_basis;

static int ncart(int l) { return (l + 1) * (l + 2) / 2; }

static void cart_comp(int l, int k, int *c)
{
    int n = 0;
    c[0] = c[1] = c[2] = 0;
    for (int lx = l; lx >= 0; lx--)
        for (int ly = l - lx; ly >= 0; ly--) {
            if (n == k) { c[0] = lx; c[1] = ly; c[2] = l - lx - ly; return; }
            n++;
        }
}

static double dfact_ratio(int i) /* i! / (2i)! */
{
    double r = 1.0;
    for (int k = i + 1; k <= 2 * i; k++) r /= k;
    return r;
}

/* Eq. local_normalization splits into a radial part (2a/pi)^{3/4}(8a)^{l/2}
 * and a component part sqrt(ix! iy! iz! / ((2ix)! (2iy)! (2iz)!)).       */
static double comp_factor(int l, int k)
{
    int c[3];
    cart_comp(l, k, c);
    return sqrt(dfact_ratio(c[0]) * dfact_ratio(c[1]) * dfact_ratio(c[2]));
}

static double comp_factor_max(int l)
{
    double m = 0;
    for (int k = 0; k < ncart(l); k++) if (comp_factor(l, k) > m) m = comp_factor(l, k);
    return m;
}

/* Contraction coefficients times the radial normalisation, rescaled so that
 * the local contracted function has unit self-overlap (the paper normalises
 * only primitives; the unit-overlap contraction is this oracle's reading).
 * For component-normalised primitives the self-overlap of the contraction
 * is sum_ij c_i c_j (2 sqrt(a_i a_j)/(a_i+a_j))^{l+3/2}.                  */
void orc_norm_coefs(int l, int n, const double *a, const double *c, double *out)
{
    double s = 0;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) s += c[i] * c[j] * pow(2.0 * sqrt(a[i] * a[j]) / (a[i] + a[j]), l + 1.5);
    for (int i = 0; i < n; i++) out[i] = c[i] * pow(2.0 * a[i] / ORC_PI, 0.75) * pow(8.0 * a[i], 0.5 * l) / sqrt(s);
}

static void mat3_inv(const double *m, double *inv)
{
    double det = m[0] * (m[4] * m[8] - m[5] * m[7]) - m[1] * (m[3] * m[8] - m[5] * m[6]) + m[2] * (m[3] * m[7] - m[4] * m[6]);
    inv[0] = (m[4] * m[8] - m[5] * m[7]) / det;
    inv[1] = (m[2] * m[7] - m[1] * m[8]) / det;
    inv[2] = (m[1] * m[5] - m[2] * m[4]) / det;
    inv[3] = (m[5] * m[6] - m[3] * m[8]) / det;
    inv[4] = (m[0] * m[8] - m[2] * m[6]) / det;
    inv[5] = (m[2] * m[3] - m[0] * m[5]) / det;
    inv[6] = (m[3] * m[7] - m[4] * m[6]) / det;
    inv[7] = (m[1] * m[6] - m[0] * m[7]) / det;
    inv[8] = (m[0] * m[4] - m[1] * m[3]) / det;
}

static double cell_volume(const double *L)
{
    return fabs(L[0] * (L[4] * L[8] - L[5] * L[7]) - L[1] * (L[3] * L[8] - L[5] * L[6]) + L[2] * (L[3] * L[7] - L[4] * L[6]));
}

/* lattice vector n1 a + n2 b + n3 c */
static void lat_vec(const double *L, double n1, double n2, double n3, double *r)
{
    for (int k = 0; k < 3; k++) r[k] = n1 * L[k] + n2 * L[3 + k] + n3 * L[6 + k];
}

/* fractional coordinates f with r = f1 a + f2 b + f3 c */
static void to_frac(const double *L, const double *r, double *f)
{
    double LT[9], inv[9];
    for (int i = 0; i < 3; i++) for (int j = 0; j < 3; j++) LT[3 * i + j] = L[3 * j + i];
    mat3_inv(LT, inv);
    for (int i = 0; i < 3; i++) f[i] = inv[3 * i] * r[0] + inv[3 * i + 1] * r[1] + inv[3 * i + 2] * r[2];
}

/* interplanar spacing of the planes spanned by two lattice vectors: V/|a_j x a_k| */
static void plane_spacings(const double *L, double *h)
{
    double V = cell_volume(L);
    for (int i = 0; i < 3; i++) {
        const double *u = L + 3 * ((i + 1) % 3), *w = L + 3 * ((i + 2) % 3);
        double c[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
        h[i] = V / sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    }
}

/* Every lattice vector R with |R - c| < r, by scanning the cube of integer
 * ranges  |n_i - f_i| <= r / h_i  (an enclosing box in fractional space).
 * Calls back with the integer triple.                                     */
typedef void (*orc_lat_cb)(const int *n, const double *R, void *ud);
static void lattice_sphere(const double *L, const double *c, double r, orc_lat_cb cb, void *ud)
{
    double f[3], h[3];
    to_frac(L, c, f);
    plane_spacings(L, h);
    int lo[3], hi[3];
    for (int i = 0; i < 3; i++) {
        lo[i] = (int)floor(f[i] - r / h[i]) - 1;
        hi[i] = (int)ceil(f[i] + r / h[i]) + 1;
    }
    for (int a = lo[0]; a <= hi[0]; a++)
        for (int b = lo[1]; b <= hi[1]; b++)
            for (int d = lo[2]; d <= hi[2]; d++) {
                double R[3];
                lat_vec(L, a, b, d, R);
                double dx = R[0] - c[0], dy = R[1] - c[1], dz = R[2] - c[2];
                if (dx * dx + dy * dy + dz * dz < r * r) {
                    int n[3] = {a, b, d};
                    cb(n, R, ud);
                }
            }
}

/* ------------------------------------------------------------------ */
/* Local primitive pairs (Section 3.1): bra mu at A (image 0), nu at B+R.  */
typedef struct {
    int I, J, ia, ib;
    int n[3];
    double a, b, p, K; /* K = c_a c_b exp(-ab/p |A-B-R|^2) */
    double A[3], B[3], P[3];
} orc_lp;

typedef struct {
    orc_lp *v;
    long n, cap;
} lp_list;

static void lp_push(lp_list *L, const orc_lp *x)
{
    if (L->n == L->cap) {
        L->cap = L->cap ? 2 * L->cap : 1024;
        L->v = (orc_lp *)realloc(L->v, L->cap * sizeof(orc_lp));
    }
    L->v[L->n++] = *x;
}

typedef struct {
    lp_list *out;
    orc_lp tmpl;
    double A[3], B[3];
    double a, b, p, cc;
} lp_ctx;

static void lp_cb(const int *n, const double *R, void *ud)
{
    lp_ctx *c = (lp_ctx *)ud;
    orc_lp x = c->tmpl;
    x.n[0] = n[0]; x.n[1] = n[1]; x.n[2] = n[2];
    double d2 = 0;
    for (int k = 0; k < 3; k++) {
        x.A[k] = c->A[k];
        x.B[k] = c->B[k] + R[k];
        x.P[k] = (c->a * x.A[k] + c->b * x.B[k]) / c->p;
        d2 += (x.A[k] - x.B[k]) * (x.A[k] - x.B[k]);
    }
    x.K = c->cc * exp(-c->a * c->b / c->p * d2);
    lp_push(c->out, &x);
}

/* Pair radius of one primitive pair: the smaller of Eq.
 * pbc_eri_pair_cutoff_implementation and Eq.
 * pbc_eri_cauchy_schwarz_cutoff_implementation.  |C_mu C_nu| is the product
 * of normalised contraction coefficients times the largest Cartesian
 * component factor of each shell.  Returns -1 if either logarithm is <= 0
 * (the primitive pair is discarded).                                      */
static double pair_radius(double a, double b, double cacb, double amin, double dR, double dCS)
{
    double p = a + b;
    double x1 = sqrt(2.0) * pow(ORC_PI, 1.25) * cacb / (p * sqrt(p + 2.0 * amin) * dR);
    double x2 = pow(2.0, 0.25) * pow(ORC_PI, 1.25) * cacb / (pow(p, 1.25) * dCS);
    if (x1 <= 1.0 || x2 <= 1.0) return -1.0;
    double r1 = sqrt(p / (a * b) * log(x1)), r2 = sqrt(p / (a * b) * log(x2));
    return r1 < r2 ? r1 : r2;
}

/* All local primitive pairs of the ordered shell pair (I, J).  The offset
 * A - B is first reduced to its minimum image by rounding its fractional
 * coordinates (Eq. lattice_image_min_norm); the sphere is then scanned.   */
static void shell_pair_lps(const orc_basis *bs, const double *cn, double amin, int I, int J, lp_list *out)
{
    const double *A = bs->centers + 3 * I, *B = bs->centers + 3 * J;
    double d[3] = {A[0] - B[0], A[1] - B[1], A[2] - B[2]}, f[3], s[3];
    to_frac(bs->lat, d, f);
    lat_vec(bs->lat, round(f[0]), round(f[1]), round(f[2]), s);
    double dmin[3] = {d[0] - s[0], d[1] - s[1], d[2] - s[2]};
    /* B + R with |A - B - R| < r  <=>  R = s + R' with |dmin - R'| < r     */
    double Bs[3] = {B[0] + s[0], B[1] + s[1], B[2] + s[2]};
    double fs[3];
    to_frac(bs->lat, s, fs);
    double fmI = comp_factor_max(bs->l[I]), fmJ = comp_factor_max(bs->l[J]);
    for (int ia = 0; ia < bs->nprim[I]; ia++)
        for (int ib = 0; ib < bs->nprim[J]; ib++) {
            double a = bs->exps[bs->poff[I] + ia], b = bs->exps[bs->poff[J] + ib];
            double ca = cn[bs->poff[I] + ia], cb = cn[bs->poff[J] + ib];
            double r = pair_radius(a, b, fabs(ca * cb) * fmI * fmJ, amin, bs->pair_R, bs->pair_cs);
            if (r <= 0) continue;
            lp_ctx ctx;
            memset(&ctx, 0, sizeof ctx);
            ctx.out = out;
            ctx.tmpl.I = I; ctx.tmpl.J = J; ctx.tmpl.ia = ia; ctx.tmpl.ib = ib;
            ctx.tmpl.a = a; ctx.tmpl.b = b; ctx.tmpl.p = a + b;
            for (int k = 0; k < 3; k++) { ctx.A[k] = A[k]; ctx.B[k] = Bs[k]; }
            ctx.a = a; ctx.b = b; ctx.p = a + b; ctx.cc = ca * cb;
            long before = out->n;
            lattice_sphere(bs->lat, dmin, r, lp_cb, &ctx);
            /* record integer image index relative to the raw centre of B   */
            for (long q = before; q < out->n; q++)
                for (int k = 0; k < 3; k++) out->v[q].n[k] += (int)lround(fs[k]);
        }
}

static double *normalised_coefs(const orc_basis *bs)
{
    int np = 0;
    for (int i = 0; i < bs->nshell; i++) np += bs->nprim[i];
    double *cn = (double *)malloc(sizeof(double) * (np > 0 ? np : 1));
    for (int i = 0; i < bs->nshell; i++)
        orc_norm_coefs(bs->l[i], bs->nprim[i], bs->exps + bs->poff[i], bs->coefs + bs->poff[i], cn + bs->poff[i]);
    return cn;
}

static double min_exponent(const orc_basis *bs)
{
    double m = INFINITY;
    for (int i = 0; i < bs->nshell; i++)
        for (int k = 0; k < bs->nprim[i]; k++) if (bs->exps[bs->poff[i] + k] < m) m = bs->exps[bs->poff[i] + k];
    return m;
}

/* Build the local pairs for ordered shell pairs (I in rows or all, J all). */
static lp_list build_lps(const orc_basis *bs, const int *rows, int nrows)
{
    lp_list out = {0, 0, 0};
    double *cn = normalised_coefs(bs);
    double amin = min_exponent(bs);
    if (rows) {
        for (int r = 0; r < nrows; r++)
            for (int J = 0; J < bs->nshell; J++) shell_pair_lps(bs, cn, amin, rows[r], J, &out);
    } else {
        for (int I = 0; I < bs->nshell; I++)
            for (int J = 0; J < bs->nshell; J++) shell_pair_lps(bs, cn, amin, I, J, &out);
    }
    free(cn);
    return out;
}

/* counts: [0] ordered shell pairs with >= 1 local pair, [1] ordered primitive
 * pairs kept, [2] ordered local primitive pairs                          */
void orc_pair_counts(const orc_basis *bs, long *counts)
{
    lp_list L = build_lps(bs, NULL, 0);
    long nsp = 0, npp = 0;
    int lastI = -1, lastJ = -1, lastia = -1, lastib = -1;
    for (long q = 0; q < L.n; q++) {
        orc_lp *x = &L.v[q];
        if (x->I != lastI || x->J != lastJ) { nsp++; lastia = lastib = -1; }
        if (x->ia != lastia || x->ib != lastib || x->I != lastI || x->J != lastJ) npp++;
        lastI = x->I; lastJ = x->J; lastia = x->ia; lastib = x->ib;
    }
    counts[0] = nsp; counts[1] = npp; counts[2] = L.n;
    free(L.v);
}

/* Export the ordered local-pair list (for tests of the definition).
 * rec layout per pair: I J ia ib n0 n1 n2 (as doubles), a b K P0 P1 P2      */
long orc_local_pairs(const orc_basis *bs, double *rec, long cap)
{
    lp_list L = build_lps(bs, NULL, 0);
    long n = L.n;
    if (rec)
        for (long q = 0; q < n && q < cap; q++) {
            orc_lp *x = &L.v[q];
            double *r = rec + 13 * q;
            r[0] = x->I; r[1] = x->J; r[2] = x->ia; r[3] = x->ib;
            r[4] = x->n[0]; r[5] = x->n[1]; r[6] = x->n[2];
            r[7] = x->a; r[8] = x->b; r[9] = x->K;
            r[10] = x->P[0]; r[11] = x->P[1]; r[12] = x->P[2];
        }
    free(L.v);
    return n;
}

/* ------------------------------------------------------------------ */
/* McMurchie-Davidson E coefficients, one axis (Eqs. E_recursion_i/j/0/out),
 * with the Gaussian factor of Eq. E_recursion_0 carried by K.            */
static void md_E(int la, int lb, double PA, double PB, double p, double E[ORC_MAXL + 1][ORC_MAXL + 1][2 * ORC_MAXL + 2])
{
    memset(E, 0, sizeof(double) * (ORC_MAXL + 1) * (ORC_MAXL + 1) * (2 * ORC_MAXL + 2));
    E[0][0][0] = 1.0;
    double h = 0.5 / p;
    for (int i = 0; i <= la; i++)
        for (int j = 0; j <= lb; j++) {
            if (i == 0 && j == 0) continue;
            for (int t = 0; t <= i + j; t++) {
                double v;
                if (i > 0) {
                    v = PA * E[i - 1][j][t];
                    if (t > 0) v += h * E[i - 1][j][t - 1];
                    if (t + 1 <= i - 1 + j) v += (t + 1) * E[i - 1][j][t + 1];
                } else {
                    v = PB * E[i][j - 1][t];
                    if (t > 0) v += h * E[i][j - 1][t - 1];
                    if (t + 1 <= i + j - 1) v += (t + 1) * E[i][j - 1][t + 1];
                }
                E[i][j][t] = v;
            }
        }
}

/* Hermite R^0_{tuv}(X) for t+u+v <= L from seeds R^m_000 = s_m (Eq.
 * R_recursion), indexed R[t][u][v].                                     */
#define RDIM (ORC_MAXLT + 1)
static void md_R(int L, const double *seed, const double *X, double R[RDIM][RDIM][RDIM])
{
    static __thread double W[RDIM][RDIM][RDIM][RDIM]; /* [m][t][u][v] */
    for (int m = 0; m <= L; m++) W[m][0][0][0] = seed[m];
    for (int n = 1; n <= L; n++)
        for (int t = n; t >= 0; t--)
            for (int u = n - t; u >= 0; u--) {
                int v = n - t - u;
                for (int m = 0; m <= L - n; m++) {
                    double r;
                    if (t > 0) {
                        r = X[0] * W[m + 1][t - 1][u][v];
                        if (t > 1) r += (t - 1) * W[m + 1][t - 2][u][v];
                    } else if (u > 0) {
                        r = X[1] * W[m + 1][t][u - 1][v];
                        if (u > 1) r += (u - 1) * W[m + 1][t][u - 2][v];
                    } else {
                        r = X[2] * W[m + 1][t][u][v - 1];
                        if (v > 1) r += (v - 1) * W[m + 1][t][u][v - 2];
                    }
                    W[m][t][u][v] = r;
                }
            }
    for (int t = 0; t <= L; t++)
        for (int u = 0; u <= L - t; u++)
            for (int v = 0; v <= L - t - u; v++) R[t][u][v] = W[0][t][u][v];
}

/* Attenuated seeds of the real-space (erfc) term (Eq. boys_function_split
 * lifted to two centres, Eq. pbc_eri_general_final):
 *   s_m = (-2 alpha)^m F_m(alpha X^2) - c_w (-2 alpha_w)^m F_m(alpha_w X^2),
 * alpha = pq/(p+q), alpha_w = 1/(1/p+1/q+1/w^2), c_w = sqrt(alpha_w/alpha).
 * omega == 0 gives the bare Coulomb seeds (c_w = 0).                      */
static void erfc_seeds(int L, double p, double q, double omega, double X2, double *s)
{
    double alpha = p * q / (p + q), F[RDIM + 1];
    orc_boys(L, alpha * X2, F);
    double f = 1.0;
    for (int m = 0; m <= L; m++) { s[m] = f * F[m]; f *= -2.0 * alpha; }
    if (omega > 0) {
        double aw = 1.0 / (1.0 / p + 1.0 / q + 1.0 / (omega * omega));
        double cw = sqrt(aw / alpha);
        orc_boys(L, aw * X2, F);
        f = 1.0;
        for (int m = 0; m <= L; m++) { s[m] -= cw * f * F[m]; f *= -2.0 * aw; }
    }
}

/* Real-space contribution of one local-pair quartet to the Cartesian ERI
 * block out[ab][cd] (component factors excluded):
 *   2 pi^{5/2}/(pq sqrt(p+q)) K_ab K_cd sum_{R1} sum_t sum_s E^ab_t E^cd_s
 *   (-1)^{|s|} R_{t+s}(P - Q - R1).                                       */
typedef struct {
    double R[RDIM][RDIM][RDIM];
    int L;
    double X0[3];
    double p, q, omega;
} rs_ctx;

static void rs_cb(const int *n, const double *R1, void *ud)
{
    (void)n;
    rs_ctx *c = (rs_ctx *)ud;
    double X[3] = {c->X0[0] - R1[0], c->X0[1] - R1[1], c->X0[2] - R1[2]};
    double s[RDIM + 1], Rt[RDIM][RDIM][RDIM];
    erfc_seeds(c->L, c->p, c->q, c->omega, X[0] * X[0] + X[1] * X[1] + X[2] * X[2], s);
    md_R(c->L, s, X, Rt);
    for (int t = 0; t <= c->L; t++)
        for (int u = 0; u <= c->L - t; u++)
            for (int v = 0; v <= c->L - t - u; v++) c->R[t][u][v] += Rt[t][u][v];
}

static void noop_sum(const int *n, const double *R1, void *ud) { rs_cb(n, R1, ud); }

/* Sum of R over the R1 images inside the real-space sphere: radius from Eq.
 * pbc_eri_real_cutoff_implementation at the oracle's delta plus a margin
 * (the equation is derived for s functions only).  A lattice-free call
 * (molecular) uses R1 = 0 alone.                                          */
static void real_space_R(const orc_basis *bs, const orc_lp *x, const orc_lp *y, int L, int periodic, rs_ctx *c)
{
    memset(c, 0, sizeof *c);
    c->L = L;
    c->p = x->p;
    c->q = y->p;
    c->omega = bs->omega;
    for (int k = 0; k < 3; k++) c->X0[k] = x->P[k] - y->P[k];
    if (!periodic) {
        double R1[3] = {0, 0, 0};
        int n[3] = {0, 0, 0};
        rs_cb(n, R1, c);
        return;
    }
    double p = x->p, q = y->p, w = bs->omega;
    double alpha = p * q / (p + q), aw = 1.0 / (1.0 / p + 1.0 / q + 1.0 / (w * w));
    double C2e = 2.0 * pow(ORC_PI, 2.5) / (p * q * sqrt(p + q)) * fabs(x->K * y->K);
    double arg = C2e * (1.0 - sqrt(aw / alpha)) / bs->delta;
    double r = (arg > 1.0 ? sqrt(log(arg) / aw) : 0.0) + bs->margin;
    lattice_sphere(bs->lat, c->X0, r, noop_sum, c);
}

static int herm_sign(int t, int u, int v) { return ((t + u + v) & 1) ? -1 : 1; }

/* Cartesian block from a summed R table: out[(ca*ncb+cb)*(ncc*ncd) + cc*ncd+cd] += pref*... */
static void contract_block(const orc_basis *bs, const orc_lp *x, const orc_lp *y, const rs_ctx *c, double *out)
{
    int la = bs->l[x->I], lb = bs->l[x->J], lc = bs->l[y->I], ld = bs->l[y->J];
    double Ex[3][ORC_MAXL + 1][ORC_MAXL + 1][2 * ORC_MAXL + 2], Ey[3][ORC_MAXL + 1][ORC_MAXL + 1][2 * ORC_MAXL + 2];
    for (int k = 0; k < 3; k++) {
        md_E(la, lb, x->P[k] - x->A[k], x->P[k] - x->B[k], x->p, Ex[k]);
        md_E(lc, ld, y->P[k] - y->A[k], y->P[k] - y->B[k], y->p, Ey[k]);
    }
    double p = x->p, q = y->p;
    double pref = 2.0 * pow(ORC_PI, 2.5) / (p * q * sqrt(p + q)) * x->K * y->K;
    int na = ncart(la), nb = ncart(lb), nc = ncart(lc), nd = ncart(ld);
    for (int ia = 0; ia < na; ia++)
        for (int ib = 0; ib < nb; ib++) {
            int a[3], b[3];
            cart_comp(la, ia, a);
            cart_comp(lb, ib, b);
            for (int ic = 0; ic < nc; ic++)
                for (int id = 0; id < nd; id++) {
                    int cc[3], dd[3];
                    cart_comp(lc, ic, cc);
                    cart_comp(ld, id, dd);
                    double sum = 0;
                    for (int t = 0; t <= a[0] + b[0]; t++)
                        for (int u = 0; u <= a[1] + b[1]; u++)
                            for (int v = 0; v <= a[2] + b[2]; v++) {
                                double eab = Ex[0][a[0]][b[0]][t] * Ex[1][a[1]][b[1]][u] * Ex[2][a[2]][b[2]][v];
                                if (eab == 0) continue;
                                for (int tt = 0; tt <= cc[0] + dd[0]; tt++)
                                    for (int uu = 0; uu <= cc[1] + dd[1]; uu++)
                                        for (int vv = 0; vv <= cc[2] + dd[2]; vv++) {
                                            double ecd = Ey[0][cc[0]][dd[0]][tt] * Ey[1][cc[1]][dd[1]][uu] * Ey[2][cc[2]][dd[2]][vv];
                                            sum += eab * ecd * herm_sign(tt, uu, vv) * c->R[t + tt][u + uu][v + vv];
                                        }
                            }
                    out[((ia * nb + ib) * nc + ic) * nd + id] += pref * sum;
                }
        }
}

/* ------------------------------------------------------------------ */
/* Fourier transform of one local primitive pair density, by the
 * Gaussian-product/binomial route:
 *   rho(r) = K prod_x (x-A)^i (x-B)^j exp(-p (x-P)^2)
 *   int rho e^{-iGr} = K prod_x e^{-i G P} sum_{k,l} C(i,k) C(j,l)
 *                      (P-A)^{i-k} (P-B)^{j-l} I_{k+l}(G)
 *   I_n(G) = int u^n e^{-p u^2 - i G u} du,
 *   I_0 = sqrt(pi/p) e^{-G^2/4p},  I_{n+1} = n/(2p) I_{n-1} - iG/(2p) I_n. */
static void ft_1d(int i, int j, double A, double B, double P, double p, double G, double complex *out)
{
    /* out[ci][cj] for ci <= i, cj <= j, computed for all lower powers too */
    double complex Im[2 * ORC_MAXL + 2];
    Im[0] = sqrt(ORC_PI / p) * exp(-G * G / (4.0 * p));
    for (int n = 0; n < i + j; n++)
        Im[n + 1] = (n > 0 ? n / (2.0 * p) * Im[n - 1] : 0.0) - _Complex_I * G / (2.0 * p) * Im[n];
    double complex ph = cexp(-_Complex_I * G * P);
    for (int ci = 0; ci <= i; ci++)
        for (int cj = 0; cj <= j; cj++) {
            double complex s = 0;
            for (int k = 0; k <= ci; k++)
                for (int l = 0; l <= cj; l++) {
                    double bk = 1, bl = 1;
                    for (int q = 0; q < k; q++) bk = bk * (ci - q) / (q + 1);
                    for (int q = 0; q < l; q++) bl = bl * (cj - q) / (q + 1);
                    s += bk * bl * pow(P - A, ci - k) * pow(P - B, cj - l) * Im[k + l];
                }
            out[ci * (ORC_MAXL + 1) + cj] = ph * s;
        }
}

/* Bloch-summed AO pair structure factors M[mu*nbf+nu] += FT of every local
 * pair of shells (I, J) in the list (component factors included).        */
static void add_pair_ft(const orc_basis *bs, const orc_lp *x, const int *ao_off, const double *G, int nbf, double complex *M)
{
    int la = bs->l[x->I], lb = bs->l[x->J];
    double complex F[3][(ORC_MAXL + 1) * (ORC_MAXL + 1)];
    for (int k = 0; k < 3; k++) ft_1d(la, lb, x->A[k], x->B[k], x->P[k], x->p, G[k], F[k]);
    for (int ia = 0; ia < ncart(la); ia++) {
        int a[3];
        cart_comp(la, ia, a);
        for (int ib = 0; ib < ncart(lb); ib++) {
            int b[3];
            cart_comp(lb, ib, b);
            double complex v = x->K * comp_factor(la, ia) * comp_factor(lb, ib);
            for (int k = 0; k < 3; k++) v *= F[k][a[k] * (ORC_MAXL + 1) + b[k]];
            M[(long)(ao_off[x->I] + ia) * nbf + ao_off[x->J] + ib] += v;
        }
    }
}

static int ao_offsets(const orc_basis *bs, int *off)
{
    int n = 0;
    for (int i = 0; i < bs->nshell; i++) { off[i] = n; n += ncart(bs->l[i]); }
    return n;
}

static void recip_basis(const double *L, double *Bm)
{
    /* rows b_i with b_i . a_j = 2 pi delta_ij: B = 2 pi (L^{-1})^T */
    double inv[9];
    mat3_inv(L, inv);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) Bm[3 * i + j] = 2.0 * ORC_PI * inv[3 * j + i];
}

/* Half-space reciprocal vectors 0 < |G| < gmax (n > 0 lexicographically). */
typedef struct { double *g; long n, cap; } g_list;
static void g_push(g_list *L, const double *g)
{
    if (L->n == L->cap) { L->cap = L->cap ? 2 * L->cap : 4096; L->g = (double *)realloc(L->g, L->cap * 3 * sizeof(double)); }
    memcpy(L->g + 3 * L->n, g, 3 * sizeof(double));
    L->n++;
}
typedef struct { g_list *out; } g_ctx;
static void g_cb(const int *n, const double *G, void *ud)
{
    g_ctx *c = (g_ctx *)ud;
    int pos = n[0] > 0 || (n[0] == 0 && (n[1] > 0 || (n[1] == 0 && n[2] > 0)));
    if (pos) g_push(c->out, G);
}
static g_list half_space_G(const double *L, double gmax)
{
    double Bm[9];
    recip_basis(L, Bm);
    g_list out = {0, 0, 0};
    g_ctx c = {&out};
    double zero[3] = {0, 0, 0};
    lattice_sphere(Bm, zero, gmax, g_cb, &c);
    return out;
}

/* Reciprocal cut-off for the oracle: the G-space weight is
 * exp(-G^2 (1/w^2 + 1/p + 1/q)/4) G^{2 Lmax - 2}; with the largest pair
 * exponents it decays slowest.  Solve (by scanning) for the radius beyond
 * which it stays below delta * 1e-3 relative to a generous prefactor.     */
static double oracle_gmax(const orc_basis *bs)
{
    double pmax = 0;
    int lmax = 0;
    for (int i = 0; i < bs->nshell; i++) {
        if (bs->l[i] > lmax) lmax = bs->l[i];
        for (int k = 0; k < bs->nprim[i]; k++) if (2 * bs->exps[bs->poff[i] + k] > pmax) pmax = 2 * bs->exps[bs->poff[i] + k];
    }
    double inv = 2.0 / pmax + (isinf(bs->omega) ? 0.0 : 1.0 / (bs->omega * bs->omega));
    double pref = 1e6 * 4.0 * ORC_PI / cell_volume(bs->lat);
    double g = 0.1;
    for (;;) {
        double w = pref * exp(-g * g * inv / 4.0) * pow(g, 4 * lmax - 2) * pow(1.0 + 1.0 / pmax, 4 * lmax);
        if (w < bs->delta * 1e-3 && g * g * inv / 4.0 > 10.0) break;
        g *= 1.02;
    }
    return g;
}

static double recip_weight(const orc_basis *bs, const double *G)
{
    double g2 = G[0] * G[0] + G[1] * G[1] + G[2] * G[2];
    double w = isinf(bs->omega) ? 1.0 : exp(-g2 / (4.0 * bs->omega * bs->omega));
    return w / g2;
}

/* Gamma overlap over the pair list (Eq. pbc_overlap_formula), as the G = 0
 * value of the pair structure factors.                                    */
void orc_overlap(const orc_basis *bs, double *S)
{
    int *off = (int *)malloc(sizeof(int) * bs->nshell);
    int nbf = ao_offsets(bs, off);
    lp_list L = build_lps(bs, NULL, 0);
    double complex *M = (double complex *)calloc((size_t)nbf * nbf, sizeof(double complex));
    double G0[3] = {0, 0, 0};
    for (long q = 0; q < L.n; q++) add_pair_ft(bs, &L.v[q], off, G0, nbf, M);
    for (long k = 0; k < (long)nbf * nbf; k++) S[k] = creal(M[k]);
    free(M);
    free(L.v);
    free(off);
}

/* Pair structure factors at one G vector (used by the tests).            */
void orc_pair_ft(const orc_basis *bs, const double *G, double *Mri)
{
    int *off = (int *)malloc(sizeof(int) * bs->nshell);
    int nbf = ao_offsets(bs, off);
    lp_list L = build_lps(bs, NULL, 0);
    double complex *M = (double complex *)calloc((size_t)nbf * nbf, sizeof(double complex));
    for (long q = 0; q < L.n; q++) add_pair_ft(bs, &L.v[q], off, G, nbf, M);
    for (long k = 0; k < (long)nbf * nbf; k++) { Mri[2 * k] = creal(M[k]); Mri[2 * k + 1] = cimag(M[k]); }
    free(M);
    free(L.v);
    free(off);
}

/* ------------------------------------------------------------------ */
/* Full periodic ERI tensor (mu nu | lambda sigma), nbf^4, for tiny cells.
 * parts: bit0 real space, bit1 reciprocal, bit2 background.               */
int orc_eri_tensor(const orc_basis *bs, int parts, double *eri)
{
    int *off = (int *)malloc(sizeof(int) * bs->nshell);
    int nbf = ao_offsets(bs, off);
    long n2 = (long)nbf * nbf;
    memset(eri, 0, sizeof(double) * n2 * n2);
    lp_list L = build_lps(bs, NULL, 0);
    double V = cell_volume(bs->lat);
    int periodic = 1;
    if (parts & 1) {
#pragma omp parallel
        {
            double *acc = (double *)calloc(n2 * n2, sizeof(double));
            double blk[6 * 6 * 6 * 6];
#pragma omp for schedule(dynamic, 4)
            for (long i = 0; i < L.n; i++) {
                const orc_lp *x = &L.v[i];
                for (long j = 0; j < L.n; j++) {
                    const orc_lp *y = &L.v[j];
                    int la = bs->l[x->I], lb = bs->l[x->J], lc = bs->l[y->I], ld = bs->l[y->J];
                    int Lt = la + lb + lc + ld;
                    rs_ctx c;
                    real_space_R(bs, x, y, Lt, periodic, &c);
                    int na = ncart(la), nb = ncart(lb), nc = ncart(lc), nd = ncart(ld);
                    memset(blk, 0, sizeof(double) * na * nb * nc * nd);
                    contract_block(bs, x, y, &c, blk);
                    for (int ia = 0; ia < na; ia++)
                        for (int ib = 0; ib < nb; ib++)
                            for (int ic = 0; ic < nc; ic++)
                                for (int id = 0; id < nd; id++) {
                                    double f = comp_factor(la, ia) * comp_factor(lb, ib) * comp_factor(lc, ic) * comp_factor(ld, id);
                                    long mu = off[x->I] + ia, nu = off[x->J] + ib, la_ = off[y->I] + ic, si = off[y->J] + id;
                                    acc[(mu * nbf + nu) * n2 + la_ * nbf + si] += f * blk[((ia * nb + ib) * nc + ic) * nd + id];
                                }
                }
            }
#pragma omp critical
            for (long k = 0; k < n2 * n2; k++) eri[k] += acc[k];
            free(acc);
        }
    }
    if (parts & 2) {
        g_list GL = half_space_G(bs->lat, oracle_gmax(bs));
#pragma omp parallel
        {
            double *acc = (double *)calloc(n2 * n2, sizeof(double));
            double complex *M = (double complex *)malloc(sizeof(double complex) * n2);
#pragma omp for schedule(dynamic, 16)
            for (long g = 0; g < GL.n; g++) {
                memset(M, 0, sizeof(double complex) * n2);
                for (long q = 0; q < L.n; q++) add_pair_ft(bs, &L.v[q], off, GL.g + 3 * g, nbf, M);
                double w = 2.0 * 4.0 * ORC_PI / V * recip_weight(bs, GL.g + 3 * g); /* +G and -G */
                for (long a = 0; a < n2; a++)
                    for (long b = 0; b < n2; b++) acc[a * n2 + b] += w * creal(conj(M[a]) * M[b]);
            }
#pragma omp critical
            for (long k = 0; k < n2 * n2; k++) eri[k] += acc[k];
            free(acc);
            free(M);
        }
        free(GL.g);
    }
    if ((parts & 4) && !isinf(bs->omega) && bs->omega > 0) {
        double *S = (double *)malloc(sizeof(double) * n2);
        orc_overlap(bs, S);
        double c = -ORC_PI / (V * bs->omega * bs->omega);
        for (long a = 0; a < n2; a++)
            for (long b = 0; b < n2; b++) eri[a * n2 + b] += c * S[a] * S[b];
        free(S);
    }
    free(L.v);
    free(off);
    return nbf;
}

/* ------------------------------------------------------------------ */
/* J and K rows for the AO functions of the listed shells, for cells too big
 * for the full tensor.  J_mn = sum_ls (mn|ls) D_ls, K_mn = sum_ls (ml|sn) D_ls
 * (Eqs. pbc_j_definition_k_sample, pbc_k_definition at the Gamma point).
 * Jrow/Krow are (nrow_ao x nbf), rows in the order of the listed shells.
 * parts as in orc_eri_tensor.                                             */
int orc_jk_rows(const orc_basis *bs, const double *D, const int *rows, int nrows, int parts, double *Jrow, double *Krow)
{
    int *off = (int *)malloc(sizeof(int) * bs->nshell);
    int nbf = ao_offsets(bs, off);
    long n2 = (long)nbf * nbf;
    int *rowoff = (int *)malloc(sizeof(int) * (nrows > 0 ? nrows : 1)), nra = 0;
    for (int r = 0; r < nrows; r++) { rowoff[r] = nra; nra += ncart(bs->l[rows[r]]); }
    memset(Jrow, 0, sizeof(double) * nra * nbf);
    memset(Krow, 0, sizeof(double) * nra * nbf);
    lp_list Lall = build_lps(bs, NULL, 0);
    double V = cell_volume(bs->lat);
    /* local row index of each AO of shell I in rows (first occurrence)    */
    int *rowpos = (int *)malloc(sizeof(int) * bs->nshell);
    for (int i = 0; i < bs->nshell; i++) rowpos[i] = -1;
    for (int r = 0; r < nrows; r++) if (rowpos[rows[r]] < 0) rowpos[rows[r]] = rowoff[r];

    if (parts & 1) {
        /* bra local pairs whose first shell is a row shell                */
        long nb = 0;
        long *bra = (long *)malloc(sizeof(long) * (Lall.n ? Lall.n : 1));
        for (long q = 0; q < Lall.n; q++) if (rowpos[Lall.v[q].I] >= 0) bra[nb++] = q;
#pragma omp parallel
        {
            double *jacc = (double *)calloc((size_t)nra * nbf, sizeof(double));
            double *kacc = (double *)calloc((size_t)nra * nbf, sizeof(double));
            double blk[6 * 6 * 6 * 6];
#pragma omp for schedule(dynamic, 1)
            for (long ii = 0; ii < nb; ii++) {
                const orc_lp *x = &Lall.v[bra[ii]];
                for (long j = 0; j < Lall.n; j++) {
                    const orc_lp *y = &Lall.v[j];
                    int la = bs->l[x->I], lb = bs->l[x->J], lc = bs->l[y->I], ld = bs->l[y->J];
                    rs_ctx c;
                    real_space_R(bs, x, y, la + lb + lc + ld, 1, &c);
                    int na = ncart(la), nbb = ncart(lb), nc = ncart(lc), nd = ncart(ld);
                    memset(blk, 0, sizeof(double) * na * nbb * nc * nd);
                    contract_block(bs, x, y, &c, blk);
                    for (int ia = 0; ia < na; ia++)
                        for (int ib = 0; ib < nbb; ib++)
                            for (int ic = 0; ic < nc; ic++)
                                for (int id = 0; id < nd; id++) {
                                    double v = blk[((ia * nbb + ib) * nc + ic) * nd + id] * comp_factor(la, ia) * comp_factor(lb, ib) *
                                               comp_factor(lc, ic) * comp_factor(ld, id);
                                    long r = rowpos[x->I] + ia, nu = off[x->J] + ib, lam = off[y->I] + ic, sig = off[y->J] + id;
                                    /* J: bra (mu nu), ket (lam sig)                     */
                                    jacc[r * nbf + nu] += v * D[lam * nbf + sig];
                                    /* K: (mu lam | sig nu) with bra (mu=r, lam=nu index), ket (sig=lam, nu=sig) */
                                    kacc[r * nbf + sig] += v * D[nu * nbf + lam];
                                }
                }
            }
#pragma omp critical
            {
                for (long k = 0; k < (long)nra * nbf; k++) { Jrow[k] += jacc[k]; Krow[k] += kacc[k]; }
            }
            free(jacc);
            free(kacc);
        }
        free(bra);
    }
    if (parts & 2) {
        g_list GL = half_space_G(bs->lat, oracle_gmax(bs));
#pragma omp parallel
        {
            double *jacc = (double *)calloc((size_t)nra * nbf, sizeof(double));
            double *kacc = (double *)calloc((size_t)nra * nbf, sizeof(double));
            double complex *M = (double complex *)malloc(sizeof(double complex) * n2);
            double complex *T = (double complex *)malloc(sizeof(double complex) * (size_t)nra * nbf);
#pragma omp for schedule(dynamic, 4)
            for (long g = 0; g < GL.n; g++) {
                memset(M, 0, sizeof(double complex) * n2);
                for (long q = 0; q < Lall.n; q++) add_pair_ft(bs, &Lall.v[q], off, GL.g + 3 * g, nbf, M);
                double w = 2.0 * 4.0 * ORC_PI / V * recip_weight(bs, GL.g + 3 * g);
                double complex rhoD = 0;
                for (long a = 0; a < n2; a++) rhoD += D[a] * M[a];
                for (int r = 0; r < nrows; r++) {
                    int I = rows[r];
                    for (int ia = 0; ia < ncart(bs->l[I]); ia++) {
                        long mu = off[I] + ia, rr = rowoff[r] + ia;
                        for (int nu = 0; nu < nbf; nu++) jacc[rr * nbf + nu] += w * creal(conj(M[mu * nbf + nu]) * rhoD);
                        /* T[rr][s] = sum_l conj(M[mu][l]) D[l][s]                 */
                        for (int s = 0; s < nbf; s++) {
                            double complex t = 0;
                            for (int l = 0; l < nbf; l++) t += conj(M[mu * nbf + l]) * D[(long)l * nbf + s];
                            T[rr * nbf + s] = t;
                        }
                        for (int nu = 0; nu < nbf; nu++) {
                            double complex k = 0;
                            for (int s = 0; s < nbf; s++) k += T[rr * nbf + s] * M[(long)s * nbf + nu];
                            kacc[rr * nbf + nu] += w * creal(k);
                        }
                    }
                }
            }
#pragma omp critical
            {
                for (long k = 0; k < (long)nra * nbf; k++) { Jrow[k] += jacc[k]; Krow[k] += kacc[k]; }
            }
            free(jacc);
            free(kacc);
            free(M);
            free(T);
        }
        free(GL.g);
    }
    if ((parts & 4) && !isinf(bs->omega) && bs->omega > 0) {
        double *S = (double *)malloc(sizeof(double) * n2);
        orc_overlap(bs, S);
        double c = -ORC_PI / (V * bs->omega * bs->omega), trDS = 0;
        for (long a = 0; a < n2; a++) trDS += D[a] * S[a];
        for (int r = 0; r < nrows; r++) {
            int I = rows[r];
            for (int ia = 0; ia < ncart(bs->l[I]); ia++) {
                long mu = off[I] + ia, rr = rowoff[r] + ia;
                for (int nu = 0; nu < nbf; nu++) {
                    Jrow[rr * nbf + nu] += c * trDS * S[mu * nbf + nu];
                    double sds = 0;
                    for (int l = 0; l < nbf; l++) {
                        double t = 0;
                        for (int s = 0; s < nbf; s++) t += D[(long)l * nbf + s] * S[(long)s * nbf + nu];
                        sds += S[mu * nbf + l] * t;
                    }
                    Krow[rr * nbf + nu] += c * sds;
                }
            }
        }
        free(S);
    }
    free(rowpos);
    free(rowoff);
    free(off);
    free(Lall.v);
    return nra;
}

/* ------------------------------------------------------------------ */
/* One primitive Cartesian quartet without a lattice (molecular), for pins
 * against closed forms and centre derivatives.  Exponents ex[4], centres
 * ctr[12], angular momenta l[4]; unit coefficients, no normalisation.
 * omega == 0: bare Coulomb; omega > 0: erfc(omega r)/r attenuated.
 * out: na*nb*nc*nd in component order.                                    */
void orc_molecular_prim_eri(const int *l, const double *ex, const double *ctr, double omega, double *out)
{
    orc_basis bs;
    memset(&bs, 0, sizeof bs);
    int ls[4] = {l[0], l[1], l[2], l[3]};
    bs.l = ls;
    bs.omega = omega;
    orc_lp x, y;
    memset(&x, 0, sizeof x);
    memset(&y, 0, sizeof y);
    x.I = 0; x.J = 1; y.I = 2; y.J = 3;
    x.a = ex[0]; x.b = ex[1]; x.p = ex[0] + ex[1];
    y.a = ex[2]; y.b = ex[3]; y.p = ex[2] + ex[3];
    double dab = 0, dcd = 0;
    for (int k = 0; k < 3; k++) {
        x.A[k] = ctr[k]; x.B[k] = ctr[3 + k]; y.A[k] = ctr[6 + k]; y.B[k] = ctr[9 + k];
        x.P[k] = (x.a * x.A[k] + x.b * x.B[k]) / x.p;
        y.P[k] = (y.a * y.A[k] + y.b * y.B[k]) / y.p;
        dab += (x.A[k] - x.B[k]) * (x.A[k] - x.B[k]);
        dcd += (y.A[k] - y.B[k]) * (y.A[k] - y.B[k]);
    }
    x.K = exp(-x.a * x.b / x.p * dab);
    y.K = exp(-y.a * y.b / y.p * dcd);
    rs_ctx c;
    real_space_R(&bs, &x, &y, l[0] + l[1] + l[2] + l[3], 0, &c);
    int n = ncart(l[0]) * ncart(l[1]) * ncart(l[2]) * ncart(l[3]);
    memset(out, 0, sizeof(double) * n);
    contract_block(&bs, &x, &y, &c, out);
}

/* ------------------------------------------------------------------ */
/* Ewald energy of point charges (Eq. nuclear_repulsion_energy), including
 * the removed-K=0 term -(4 pi / V)/(4 w^2) per pair and per charge.  Sums
 * are taken over the spheres of Eqs. nuclear_repulsion_energy_real_cutoff
 * and _reciprocal_cutoff at the given delta, found by scanning.           */
typedef struct { double acc; double d[3]; double w; int skip0; } pc_ctx;
static void pc_real_cb(const int *n, const double *R, void *ud)
{
    pc_ctx *c = (pc_ctx *)ud;
    if (c->skip0 && n[0] == 0 && n[1] == 0 && n[2] == 0) return;
    double x = c->d[0] + R[0], y = c->d[1] + R[1], z = c->d[2] + R[2];
    double r = sqrt(x * x + y * y + z * z);
    c->acc += erfc(c->w * r) / r;
}
typedef struct { double acc; double d[3]; double w; } pk_ctx;
static void pc_recip_cb(const int *n, const double *G, void *ud)
{
    pk_ctx *c = (pk_ctx *)ud;
    if (n[0] == 0 && n[1] == 0 && n[2] == 0) return;
    double g2 = G[0] * G[0] + G[1] * G[1] + G[2] * G[2];
    c->acc += exp(-g2 / (4.0 * c->w * c->w)) / g2 * cos(G[0] * c->d[0] + G[1] * c->d[1] + G[2] * c->d[2]);
}

double orc_ewald_point_charges(const double *lat, int n, const double *q, const double *xyz, double omega, double delta)
{
    double V = cell_volume(lat), Bm[9];
    recip_basis(lat, Bm);
    double rb = 1.0, kb = 1.0;
    while (2.0 / sqrt(ORC_PI) * exp(-omega * omega * rb * rb) / (rb * rb) > delta) rb *= 1.01;
    while (4.0 * ORC_PI / V * exp(-kb * kb / (4.0 * omega * omega)) / (kb * kb) > delta) kb *= 1.01;
    double E = 0;
    double zero[3] = {0, 0, 0};
    for (int A = 0; A < n; A++)
        for (int B = A; B < n; B++) {
            pc_ctx rc;
            memset(&rc, 0, sizeof rc);
            pk_ctx kc;
            memset(&kc, 0, sizeof kc);
            for (int k = 0; k < 3; k++) { rc.d[k] = xyz[3 * A + k] - xyz[3 * B + k]; kc.d[k] = rc.d[k]; }
            rc.w = omega;
            kc.w = omega;
            rc.skip0 = (A == B);
            double nd[3] = {-rc.d[0], -rc.d[1], -rc.d[2]};
            lattice_sphere(lat, A == B ? zero : nd, rb, pc_real_cb, &rc);
            lattice_sphere(Bm, zero, kb, pc_recip_cb, &kc);
            double term = 4.0 * ORC_PI / V * kc.acc - 4.0 * ORC_PI / V / (4.0 * omega * omega) + rc.acc;
            if (A == B) E += 0.5 * q[A] * q[A] * (term - 2.0 * omega / sqrt(ORC_PI));
            else E += q[A] * q[B] * term;
        }
    return E;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Timing sample for the CPU baseline: the same code paths as orc_jk_rows
 * on a bounded subset of the work of a full build.
 *   real space: every bra_stride-th ordered local pair as the bra, against
 *               every ket local pair (digested into scratch J and K);
 *   reciprocal: ng_sample half-space G vectors: all pair transforms, the
 *               Coulomb contraction and the exchange contraction of one AO
 *               row.
 * out[0] seconds of the real-space sample, out[1] bra pairs sampled,
 * out[2] ordered local pairs in total, out[3] seconds per G of the pair
 * transforms, out[4] seconds per G per AO row of the contractions,
 * out[5] half-space G vectors in the oracle's list, out[6] nbf.          */
void orc_jk_sample(const orc_basis *bs, const double *D, int bra_stride, int ng_sample, double *out)
{
    int *off = (int *)malloc(sizeof(int) * bs->nshell);
    int nbf = ao_offsets(bs, off);
    long n2 = (long)nbf * nbf;
    lp_list Lall = build_lps(bs, NULL, 0);
    double *jacc = (double *)calloc(n2, sizeof(double)), *kacc = (double *)calloc(n2, sizeof(double));
    long nb = 0;
    double t0 = omp_get_wtime();
#pragma omp parallel
    {
        double blk[6 * 6 * 6 * 6];
#pragma omp for schedule(dynamic, 1) reduction(+ : nb)
        for (long ii = 0; ii < Lall.n; ii += bra_stride) {
            nb++;
            const orc_lp *x = &Lall.v[ii];
            for (long j = 0; j < Lall.n; j++) {
                const orc_lp *y = &Lall.v[j];
                int la = bs->l[x->I], lb = bs->l[x->J], lc = bs->l[y->I], ld = bs->l[y->J];
                rs_ctx c;
                real_space_R(bs, x, y, la + lb + lc + ld, 1, &c);
                int na = ncart(la), nbb = ncart(lb), nc = ncart(lc), nd = ncart(ld);
                memset(blk, 0, sizeof(double) * na * nbb * nc * nd);
                contract_block(bs, x, y, &c, blk);
                for (int ia = 0; ia < na; ia++)
                    for (int ib = 0; ib < nbb; ib++)
                        for (int ic = 0; ic < nc; ic++)
                            for (int id = 0; id < nd; id++) {
                                double v = blk[((ia * nbb + ib) * nc + ic) * nd + id];
                                long mu = off[x->I] + ia, nu = off[x->J] + ib, lam = off[y->I] + ic, sig = off[y->J] + id;
#pragma omp atomic
                                jacc[mu * nbf + nu] += v * D[lam * nbf + sig];
#pragma omp atomic
                                kacc[mu * nbf + sig] += v * D[nu * nbf + lam];
                            }
            }
        }
    }
    out[0] = omp_get_wtime() - t0;
    out[1] = (double)nb;
    out[2] = (double)Lall.n;
    g_list GL = half_space_G(bs->lat, oracle_gmax(bs));
    double complex *M = (double complex *)malloc(sizeof(double complex) * n2);
    double complex *T = (double complex *)malloc(sizeof(double complex) * nbf);
    double tft = 0, tcon = 0;
    int ns = ng_sample < GL.n ? ng_sample : (int)GL.n;
    for (int s = 0; s < ns; s++) {
        const double *G = GL.g + 3 * (long)(s * (GL.n / (ns > 0 ? ns : 1)));
        double t1 = omp_get_wtime();
        memset(M, 0, sizeof(double complex) * n2);
        for (long q = 0; q < Lall.n; q++) add_pair_ft(bs, &Lall.v[q], off, G, nbf, M);
        double t2 = omp_get_wtime();
        double complex rhoD = 0;
        for (long a = 0; a < n2; a++) rhoD += D[a] * M[a];
        long mu = 0;
        for (int nu = 0; nu < nbf; nu++) jacc[nu] += creal(conj(M[mu * nbf + nu]) * rhoD);
        for (int s2 = 0; s2 < nbf; s2++) {
            double complex t = 0;
            for (int l = 0; l < nbf; l++) t += conj(M[mu * nbf + l]) * D[(long)l * nbf + s2];
            T[s2] = t;
        }
        for (int nu = 0; nu < nbf; nu++) {
            double complex k = 0;
            for (int s2 = 0; s2 < nbf; s2++) k += T[s2] * M[(long)s2 * nbf + nu];
            kacc[nu] += creal(k);
        }
        double t3 = omp_get_wtime();
        tft += t2 - t1;
        tcon += t3 - t2;
    }
    out[3] = ns ? tft / ns : 0;
    out[4] = ns ? tcon / ns : 0;
    out[5] = (double)GL.n;
    out[6] = (double)nbf;
    free(M);
    free(T);
    free(GL.g);
    free(jacc);
    free(kacc);
    free(Lall.v);
    free(off);
}

/* ------------------------------------------------------------------ */
/* One-electron operators of the cell: kinetic energy and nuclear
 * attraction (Sections 2.1 and 2.2 of the paper; the kinetic formula is in
 * its Supporting Information).  Like the overlap, both are sums over the
 * pair list of local integrals between mu at A and nu at B + R.          */

/* 1-D overlap of (x-A)^i e^{-a(x-A)^2} and (x-B)^j e^{-b(x-B)^2} without the
 * Gaussian factor exp(-ab/p (A-B)^2) (carried by K): binomial expansion
 * about P and the Gaussian moments int u^n e^{-p u^2} du =
 * Gamma((n+1)/2) / p^{(n+1)/2} for even n, 0 for odd n.                  */
static double ov_1d(int i, int j, double A, double B, double P, double p)
{
    double s = 0;
    for (int k = 0; k <= i; k++)
        for (int l = 0; l <= j; l++) {
            const int n = k + l;
            if (n & 1) continue;
            double bk = 1, bl = 1;
            for (int q = 0; q < k; q++) bk = bk * (i - q) / (q + 1);
            for (int q = 0; q < l; q++) bl = bl * (j - q) / (q + 1);
            s += bk * bl * pow(P - A, i - k) * pow(P - B, j - l) * tgamma(0.5 * (n + 1)) / pow(p, 0.5 * (n + 1));
        }
    return s;
}

/* 1-D kinetic element <i| -1/2 d^2/dx^2 |j> with d^2/dx^2 acting on the
 * right-hand Gaussian of exponent b:
 *   -1/2 [ j(j-1) s(i,j-2) - 2b(2j+1) s(i,j) + 4b^2 s(i,j+2) ].           */
static double kin_1d(int i, int j, double A, double B, double P, double a, double b)
{
    const double p = a + b;
    double t = -2.0 * b * (2 * j + 1) * ov_1d(i, j, A, B, P, p) + 4.0 * b * b * ov_1d(i, j + 2, A, B, P, p);
    if (j >= 2) t += j * (j - 1) * ov_1d(i, j - 2, A, B, P, p);
    return -0.5 * t;
}

/* T_mn = sum over the pair list of the local kinetic integrals (component
 * factors included), T = Tx Sy Sz + Sx Ty Sz + Sx Sy Tz per primitive pair. */
void orc_kinetic(const orc_basis *bs, double *T)
{
    int *off = (int *)malloc(sizeof(int) * bs->nshell);
    int nbf = ao_offsets(bs, off);
    memset(T, 0, sizeof(double) * nbf * nbf);
    lp_list L = build_lps(bs, NULL, 0);
    for (long q = 0; q < L.n; q++) {
        const orc_lp *x = &L.v[q];
        int la = bs->l[x->I], lb = bs->l[x->J];
        for (int ia = 0; ia < ncart(la); ia++) {
            int ca[3];
            cart_comp(la, ia, ca);
            for (int ib = 0; ib < ncart(lb); ib++) {
                int cb[3];
                cart_comp(lb, ib, cb);
                double s[3], t[3];
                for (int k = 0; k < 3; k++) {
                    s[k] = ov_1d(ca[k], cb[k], x->A[k], x->B[k], x->P[k], x->p);
                    t[k] = kin_1d(ca[k], cb[k], x->A[k], x->B[k], x->P[k], x->a, x->b);
                }
                double v = t[0] * s[1] * s[2] + s[0] * t[1] * s[2] + s[0] * s[1] * t[2];
                T[(long)(off[x->I] + ia) * nbf + off[x->J] + ib] += x->K * comp_factor(la, ia) * comp_factor(lb, ib) * v;
            }
        }
    }
    free(L.v);
    free(off);
}

/* Nuclear attraction of point charges Z_C at C with all their images,
 *   V_mn = - sum_C Z_C sum_{R_C} < mu | 1/|r - C - R_C| | nu(R) >,
 * Ewald-split as in Eq. boys_function_split / pbc_v1e_base_case_final:
 *   real part: (2 pi / p) K sum_t E^{ab}_t R_t(P - C - R_C) with seeds
 *     s_m = (-2p)^m F_m(p X^2) - c (-2 a_w)^m F_m(a_w X^2),
 *     a_w = p w^2 / (p + w^2), c = w / sqrt(p + w^2);
 *   reciprocal part: (4 pi / V) sum_{G != 0} e^{-G^2/4w^2}/G^2
 *     Re[conj(rho_mn(G)) rho_N(G)],  rho_N(G) = sum_C Z_C e^{-iG.C};
 *   self term (Eq. v1e_self_term summed over primitives and images):
 *     -(pi/(V w^2)) S_mn per unit charge.
 * Every part carries the overall -Z_C of the attraction.  parts: bit0 real,
 * bit1 reciprocal, bit2 self term, bit3 molecular (bare Coulomb of the
 * charges at C only, no images; the other bits are then ignored).         */
typedef struct {
    double R[RDIM][RDIM][RDIM];
    int L;
    double X0[3];
    double p, omega;
    int bare;
} nv_ctx;

static void nuc_seeds(int L, double p, double omega, int bare, double X2, double *s)
{
    double F[RDIM + 1];
    orc_boys(L, p * X2, F);
    double f = 1.0;
    for (int m = 0; m <= L; m++) { s[m] = f * F[m]; f *= -2.0 * p; }
    if (!bare) {
        const double aw = p * omega * omega / (p + omega * omega), c = omega / sqrt(p + omega * omega);
        orc_boys(L, aw * X2, F);
        f = 1.0;
        for (int m = 0; m <= L; m++) { s[m] -= c * f * F[m]; f *= -2.0 * aw; }
    }
}

static void nv_cb(const int *n, const double *RC, void *ud)
{
    (void)n;
    nv_ctx *c = (nv_ctx *)ud;
    double X[3] = {c->X0[0] - RC[0], c->X0[1] - RC[1], c->X0[2] - RC[2]};
    double s[RDIM + 1], Rt[RDIM][RDIM][RDIM];
    nuc_seeds(c->L, c->p, c->omega, c->bare, X[0] * X[0] + X[1] * X[1] + X[2] * X[2], s);
    md_R(c->L, s, X, Rt);
    for (int t = 0; t <= c->L; t++)
        for (int u = 0; u <= c->L - t; u++)
            for (int v = 0; v <= c->L - t - u; v++) c->R[t][u][v] += Rt[t][u][v];
}

void orc_nuclear(const orc_basis *bs, int natom, const double *Z, const double *xyz, int parts, double *Vm)
{
    int *off = (int *)malloc(sizeof(int) * bs->nshell);
    int nbf = ao_offsets(bs, off);
    long n2 = (long)nbf * nbf;
    memset(Vm, 0, sizeof(double) * n2);
    lp_list L = build_lps(bs, NULL, 0);
    const double V = cell_volume(bs->lat), w = bs->omega;
    const int molecular = (parts & 8) != 0;
    if (molecular || (parts & 1)) {
        for (long q = 0; q < L.n; q++) {
            const orc_lp *x = &L.v[q];
            int la = bs->l[x->I], lb = bs->l[x->J], Lt = la + lb;
            double E[3][ORC_MAXL + 1][ORC_MAXL + 1][2 * ORC_MAXL + 2];
            for (int k = 0; k < 3; k++) md_E(la, lb, x->P[k] - x->A[k], x->P[k] - x->B[k], x->p, E[k]);
            for (int C = 0; C < natom; C++) {
                nv_ctx c;
                memset(&c, 0, sizeof c);
                c.L = Lt;
                c.p = x->p;
                c.omega = w;
                c.bare = molecular;
                for (int k = 0; k < 3; k++) c.X0[k] = x->P[k] - xyz[3 * C + k];
                if (molecular) {
                    double R0[3] = {0, 0, 0};
                    int n0[3] = {0, 0, 0};
                    nv_cb(n0, R0, &c);
                } else {
                    const double aw = x->p * w * w / (x->p + w * w), cw = w / sqrt(x->p + w * w);
                    const double arg = 2.0 * ORC_PI / x->p * fabs(x->K) * (1.0 - cw) * fabs(Z[C]) / bs->delta;
                    const double r = (arg > 1.0 ? sqrt(log(arg) / aw) : 0.0) + bs->margin;
                    lattice_sphere(bs->lat, c.X0, r, nv_cb, &c);
                }
                const double pref = -Z[C] * 2.0 * ORC_PI / x->p * x->K;
                for (int ia = 0; ia < ncart(la); ia++) {
                    int a[3];
                    cart_comp(la, ia, a);
                    for (int ib = 0; ib < ncart(lb); ib++) {
                        int b[3];
                        cart_comp(lb, ib, b);
                        double v = 0;
                        for (int tx = 0; tx <= a[0] + b[0]; tx++)
                            for (int ty = 0; ty <= a[1] + b[1]; ty++)
                                for (int tz = 0; tz <= a[2] + b[2]; tz++)
                                    v += E[0][a[0]][b[0]][tx] * E[1][a[1]][b[1]][ty] * E[2][a[2]][b[2]][tz] * c.R[tx][ty][tz];
                        Vm[(long)(off[x->I] + ia) * nbf + off[x->J] + ib] += pref * comp_factor(la, ia) * comp_factor(lb, ib) * v;
                    }
                }
            }
        }
    }
    if (!molecular && (parts & 2)) {
        g_list GL = half_space_G(bs->lat, oracle_gmax(bs));
        double complex *M = (double complex *)malloc(sizeof(double complex) * n2);
        for (long g = 0; g < GL.n; g++) {
            const double *G = GL.g + 3 * g;
            memset(M, 0, sizeof(double complex) * n2);
            for (long q = 0; q < L.n; q++) add_pair_ft(bs, &L.v[q], off, G, nbf, M);
            double complex rn = 0;
            for (int C = 0; C < natom; C++)
                rn += Z[C] * cexp(-_Complex_I * (G[0] * xyz[3 * C] + G[1] * xyz[3 * C + 1] + G[2] * xyz[3 * C + 2]));
            const double wg = 2.0 * 4.0 * ORC_PI / V * recip_weight(bs, G); /* +G and -G */
            for (long k = 0; k < n2; k++) Vm[k] -= wg * creal(conj(M[k]) * rn);
        }
        free(M);
        free(GL.g);
    }
    if (!molecular && (parts & 4) && !isinf(w) && w > 0) {
        double *S = (double *)malloc(sizeof(double) * n2), Zt = 0;
        orc_overlap(bs, S);
        for (int C = 0; C < natom; C++) Zt += Z[C];
        const double c = ORC_PI / (V * w * w) * Zt; /* -Z times the self term -(pi/(V w^2)) S */
        for (long k = 0; k < n2; k++) Vm[k] += c * S[k];
        free(S);
    }
    free(L.v);
    free(off);
}
