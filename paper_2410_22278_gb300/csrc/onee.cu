// One-electron operators of the cell on the device: the kinetic-energy
// matrix and the nuclear attraction of point charges with their periodic
// images, Ewald-split at the plan's omega (Sections 2.1 and 2.2 of the
// paper; the kinetic formula is in its Supporting Information).  Both are
// sums over the plan's unique shell-pair images of local integrals between
// mu at A and nu at B + R, like the overlap.
//
// Nuclear attraction, per charge Z_C at C (Eq. pbc_v1e_base_case_final):
//   real part    -Z (2 pi/p) K sum_t E^{ab}_t R_t(P - C - R_C) over the images
//                R_C inside the screening sphere, seeds (-2p)^m G_m(p X^2, c),
//                c = w / sqrt(p + w^2) (the attenuated Boys difference of Eq.
//                boys_function_split written as one integral);
//   reciprocal   -(4 pi / V) sum_{G != 0} e^{-G^2/4w^2}/G^2 Re[conj(rho_ab(G))
//                rho_N(G)], rho_N(G) = sum_C Z_C e^{-iG.C}: the same
//                structure-factor slab as the Coulomb build, contracted with
//                the nuclear structure factor by one matrix-vector product;
//   self term    +(pi / (V w^2)) Z_tot S_ab (Eq. v1e_self_term).
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <vector>

#include "kernels.cuh"
#include "launch.h"
#include "plan.h"

namespace jk {
namespace {

// 1-D overlaps s[i][j] = sqrt(pi/p) E^{ij}_0, i <= LA, j <= LB + 2 (the
// Gaussian factor is in K), and the kinetic block of one primitive pair:
//   t(i, j) = -1/2 [ j(j-1) s(i,j-2) - 2b(2j+1) s(i,j) + 4b^2 s(i,j+2) ],
//   T = tx sy sz + sx ty sz + sx sy tz.
template <int LA, int LB>
__device__ __forceinline__ void kinetic_block(const PpiRec &x, double b, double *blk)
{
    constexpr int NA = ncart(LA), NB = ncart(LB), LB2 = LB + 2, NT = LA + LB2 + 1;
    double s[3][LA + 1][LB2 + 1], t[3][LA + 1][LB + 1];
    const double rp = sqrt(kPi / x.p);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double E[(LA + 1) * (LB2 + 1) * NT];
        herm_E<LA, LB2, double>(x.PA[k], x.PB[k], 0.5 / x.p, E);
#pragma unroll
        for (int i = 0; i <= LA; ++i)
#pragma unroll
            for (int j = 0; j <= LB2; ++j) s[k][i][j] = rp * E[(i * (LB2 + 1) + j) * NT];
#pragma unroll
        for (int i = 0; i <= LA; ++i)
#pragma unroll
            for (int j = 0; j <= LB; ++j) {
                double v = -2.0 * b * (2 * j + 1) * s[k][i][j] + 4.0 * b * b * s[k][i][j + 2];
                if (j >= 2) v += j * (j - 1) * s[k][i][j - 2];
                t[k][i][j] = -0.5 * v;
            }
    }
#pragma unroll
    for (int a = 0; a < NA; ++a)
#pragma unroll
        for (int c = 0; c < NB; ++c) {
            const int ax = cexp(LA, a, 0), ay = cexp(LA, a, 1), az = cexp(LA, a, 2);
            const int bx = cexp(LB, c, 0), by = cexp(LB, c, 1), bz = cexp(LB, c, 2);
            blk[a * NB + c] += x.K * (t[0][ax][bx] * s[1][ay][by] * s[2][az][bz] + s[0][ax][bx] * t[1][ay][by] * s[2][az][bz] +
                                      s[0][ax][bx] * s[1][ay][by] * t[2][az][bz]);
        }
}

// Attraction block of one primitive pair by every charge and its images:
// X0 = P - C reduced by rounding its fractional coordinates, then the
// length-sorted lattice candidates (x, y, z, |R|) until |R| - |X0| >= r.
template <int LA, int LB>
__device__ __forceinline__ void nuclear_block(const PlanDev &pl, const PpiRec &x, int natom, const double *__restrict__ Zc,
                                              const double *__restrict__ xyz, const double *__restrict__ cand, int ncand,
                                              double *blk)
{
    constexpr int NA = ncart(LA), NB = ncart(LB), L = LA + LB, NT = L + 1, D = L + 1;
    double E[3][(LA + 1) * (LB + 1) * NT];
#pragma unroll
    for (int k = 0; k < 3; ++k) herm_E<LA, LB, double>(x.PA[k], x.PB[k], 0.5 / x.p, E[k]);
    const double w2 = pl.omega * pl.omega;
    const double c = sqrt(w2 / (x.p + w2)), aw = x.p * w2 / (x.p + w2);
    double Rs[D * D * D];
#pragma unroll
    for (int k = 0; k < D * D * D; ++k) Rs[k] = 0.0;
    for (int C = 0; C < natom; ++C) {
        const double z = Zc[C];
        // screening radius of Eq. pbc_eri_real_cutoff_implementation for a
        // point charge: (2 pi/p) |K Z| (1 - c) e^{-aw r^2} above delta_R / 10
        const double lg = log(2.0 * kPi / x.p * fabs(x.K * z) * (1.0 - c)) - (double)pl.log_ewald_R;
        if (!(lg > 0.0)) continue;
        double r = sqrt(lg / aw);
        if (L > 0) {
            r = sqrt((lg + L * log(1.0 + 2.0 * aw * r)) / aw);
            r = sqrt((lg + L * log(1.0 + 2.0 * aw * r)) / aw) + 0.5 + 0.25 * L;
        }
        double X0[3] = {x.P[0] - xyz[3 * C], x.P[1] - xyz[3 * C + 1], x.P[2] - xyz[3 * C + 2]};
        double f[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) f[a] = rint(pl.Finv[3 * a] * X0[0] + pl.Finv[3 * a + 1] * X0[1] + pl.Finv[3 * a + 2] * X0[2]);
#pragma unroll
        for (int a = 0; a < 3; ++a) X0[a] -= f[0] * pl.L[a] + f[1] * pl.L[3 + a] + f[2] * pl.L[6 + a];
        const double x0n = sqrt(X0[0] * X0[0] + X0[1] * X0[1] + X0[2] * X0[2]);
        for (int q = 0; q < ncand; ++q) {
            if (cand[4 * q + 3] - x0n >= r) break;
            const double Xx = X0[0] - cand[4 * q], Xy = X0[1] - cand[4 * q + 1], Xz = X0[2] - cand[4 * q + 2];
            const double x2 = Xx * Xx + Xy * Xy + Xz * Xz;
            if (x2 >= r * r) continue;
            double G[L + 1], s[L + 1];
            boys_attenuated<L, double>(x.p * x2, c, pl.boys, G);
            double fm = -z;  // (-2p)^m times the charge of the attraction
#pragma unroll
            for (int m = 0; m <= L; ++m) {
                s[m] = fm * G[m];
                fm *= -2.0 * x.p;
            }
            double B[D * D * D];
            herm_R<L, double>(s, Xx, Xy, Xz, B);
#pragma unroll
            for (int t = 0; t <= L; ++t)
#pragma unroll
                for (int u = 0; u <= L - t; ++u)
#pragma unroll
                    for (int v = 0; v <= L - t - u; ++v) Rs[(t * D + u) * D + v] += B[(t * D + u) * D + v];
        }
    }
    const double pref = 2.0 * kPi / x.p * x.K;
#pragma unroll
    for (int a = 0; a < NA; ++a)
#pragma unroll
        for (int cc = 0; cc < NB; ++cc) {
            const int ax = cexp(LA, a, 0), ay = cexp(LA, a, 1), az = cexp(LA, a, 2);
            const int bx = cexp(LB, cc, 0), by = cexp(LB, cc, 1), bz = cexp(LB, cc, 2);
            double v = 0.0;
#pragma unroll
            for (int tx = 0; tx <= ax + bx; ++tx)
#pragma unroll
                for (int ty = 0; ty <= ay + by; ++ty)
#pragma unroll
                    for (int tz = 0; tz <= az + bz; ++tz)
                        v += E[0][(ax * (LB + 1) + bx) * NT + tx] * E[1][(ay * (LB + 1) + by) * NT + ty] *
                             E[2][(az * (LB + 1) + bz) * NT + tz] * Rs[(tx * D + ty) * D + tz];
            blk[a * NB + cc] += pref * v;
        }
}

// One thread per unique shell pair of a class: sum over its images and
// primitive pairs, then write the block and (off the diagonal) its
// transpose; the images (I, I, -R) of a diagonal pair are the transposed
// blocks of the stored (I, I, R).  op 0 kinetic, op 1 nuclear real part.
template <int LA, int LB>
__global__ void __launch_bounds__(128) k_onee(PlanDev pl, int sp0, int sp1, int op, const double2 *__restrict__ ab, int natom,
                                              const double *__restrict__ Zc, const double *__restrict__ xyz,
                                              const double *__restrict__ cand, int ncand, double *__restrict__ Out)
{
    constexpr int NA = ncart(LA), NB = ncart(LB);
    const int sp = sp0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (sp >= sp1) return;
    const SpairRec rec = pl.spair[sp];
    const bool diag = rec.I == rec.J;
    double blk[NA * NB];
#pragma unroll
    for (int k = 0; k < NA * NB; ++k) blk[k] = 0.0;
    for (int s = 0; s < rec.nspi; ++s) {
        const SpiRec si = pl.spi[pl.spi_order[rec.spi0 + s]];
        const bool rzero = si.n[0] == 0 && si.n[1] == 0 && si.n[2] == 0;
        double tmp[NA * NB];
#pragma unroll
        for (int k = 0; k < NA * NB; ++k) tmp[k] = 0.0;
        for (int q = 0; q < si.npp; ++q) {
            const PpiRec x = pl.ppi[si.pp0 + q];
            if (op == 0) kinetic_block<LA, LB>(x, ab[si.pp0 + q].y, tmp);
            else nuclear_block<LA, LB>(pl, x, natom, Zc, xyz, cand, ncand, tmp);
        }
#pragma unroll
        for (int a = 0; a < NA; ++a)
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                blk[a * NB + b] += tmp[a * NB + b];
                if (diag && !rzero) blk[b * NB + a] += tmp[a * NB + b];
            }
    }
    const int n = pl.nbf, aoI = pl.shells[rec.I].ao, aoJ = pl.shells[rec.J].ao;
#pragma unroll
    for (int a = 0; a < NA; ++a)
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            Out[(size_t)(aoI + a) * n + aoJ + b] = blk[a * NB + b];
            if (!diag) Out[(size_t)(aoJ + b) * n + aoI + a] = blk[a * NB + b];
        }
}

template <int LA, int LB>
static void onee_go(const PlanDev &pl, int sp0, int sp1, int op, const double2 *ab, int natom, const double *Z, const double *xyz,
                    const double *cand, int ncand, double *Out, cudaStream_t st)
{
    const int nt = sp1 - sp0;
    if (nt <= 0) return;
    k_onee<LA, LB><<<(nt + 127) / 128, 128, 0, st>>>(pl, sp0, sp1, op, ab, natom, Z, xyz, cand, ncand, Out);
}

static void launch_onee(int cls, const PlanDev &pl, int sp0, int sp1, int op, const double2 *ab, int natom, const double *Z,
                        const double *xyz, const double *cand, int ncand, double *Out, cudaStream_t st)
{
    switch (cls) {
    case 0: onee_go<0, 0>(pl, sp0, sp1, op, ab, natom, Z, xyz, cand, ncand, Out, st); break;
    case 1: onee_go<1, 0>(pl, sp0, sp1, op, ab, natom, Z, xyz, cand, ncand, Out, st); break;
    case 2: onee_go<1, 1>(pl, sp0, sp1, op, ab, natom, Z, xyz, cand, ncand, Out, st); break;
    case 3: onee_go<2, 0>(pl, sp0, sp1, op, ab, natom, Z, xyz, cand, ncand, Out, st); break;
    case 4: onee_go<2, 1>(pl, sp0, sp1, op, ab, natom, Z, xyz, cand, ncand, Out, st); break;
    case 5: onee_go<2, 2>(pl, sp0, sp1, op, ab, natom, Z, xyz, cand, ncand, Out, st); break;
    default: break;
    }
}

// sqrt(8 pi w(G) / V) (Re, Im) of rho_N(G) = sum_C Z_C e^{-iG.C} for the G
// of a chunk, in the column order of the structure-factor slab
__global__ void k_nuclear_sfac(int natom, const double *__restrict__ Zc, const double *__restrict__ xyz, const double *__restrict__ gv,
                               int g0, int gcur, double *__restrict__ out)
{
    const int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= gcur) return;
    const double *g = gv + 4 * (size_t)(g0 + gi);
    double re = 0, im = 0;
    for (int C = 0; C < natom; ++C) {
        double sn, cs;
        sincos(g[0] * xyz[3 * C] + g[1] * xyz[3 * C + 1] + g[2] * xyz[3 * C + 2], &sn, &cs);
        re += Zc[C] * cs;
        im -= Zc[C] * sn;
    }
    out[2 * gi] = g[3] * re;
    out[2 * gi + 1] = g[3] * im;
}

// Out = F o (A + c S_raw): component factors and the self term
__global__ void k_onee_final(int n, const double *__restrict__ f, const double *__restrict__ A, const double *__restrict__ S, double c,
                             double *__restrict__ Out)
{
    const size_t n2 = (size_t)n * n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x)
        Out[i] = f[i / n] * f[i % n] * (A[i] + c * S[i]);
}

}  // namespace

int one_electron(Plan *P, int natom, const double *Z, const double *xyz, double *T, double *V, cudaStream_t st)
{
    const int n = P->nbf;
    const size_t n2 = (size_t)n * n;
    Workspace &w = P->ws;
    const PlanDev pl = P->dev();
    auto ok = [](cudaError_t e) { return e == cudaSuccess; };
    const int grid = (int)std::min<size_t>((n2 + 255) / 256, 152 * 16);
    if (T) {
        if (!ok(cudaMemsetAsync(w.T1, 0, n2 * sizeof(double), st))) return fail(JK_ERR_CUDA, "memset failed");
        for (int c = 0; c < JK_NCLASS_MAX; ++c)
            launch_onee(c, pl, P->spair_class_off[c], P->spair_class_off[c + 1], 0, P->d_ppi_ab, 0, nullptr, nullptr, nullptr, 0, w.T1, st);
        k_onee_final<<<grid, 256, 0, st>>>(n, P->d_compf, w.T1, P->d_S, 0.0, T);
        if (!ok(cudaGetLastError())) return fail(JK_ERR_CUDA, "kinetic-energy kernels failed");
    }
    if (!V || natom <= 0) return ok(cudaStreamSynchronize(st)) ? JK_OK : fail(JK_ERR_CUDA, "one-electron kernels failed");

    // lattice candidates for the charges' images: |R| up to the largest
    // screening radius plus the cell's circumradius (the reduced X0 is at
    // most that long), sorted by length
    double zmax = 0, ztot = 0;
    for (int C = 0; C < natom; ++C) {
        zmax = std::max(zmax, std::fabs(Z[C]));
        ztot += Z[C];
    }
    const double w2 = P->omega * P->omega, lgd = std::log(P->cut.ewald_R * 1e-1);
    double rmax = 0;
    for (size_t q = 0; q < P->ppi.size(); ++q) {
        const PpiRec &x = P->ppi[q];
        const double c = std::sqrt(w2 / (x.p + w2)), aw = x.p * w2 / (x.p + w2);
        const double lg = std::log(2.0 * kPi / x.p * std::fabs(x.K) * zmax * (1.0 - c)) - lgd;
        if (lg <= 0) continue;
        double r = std::sqrt(lg / aw);
        for (int it = 0; it < 2; ++it) r = std::sqrt((lg + 4.0 * std::log(1.0 + 2.0 * aw * r)) / aw);
        rmax = std::max(rmax, r + 1.5);
    }
    double hd = 0;
    for (int s1 = -1; s1 <= 1; s1 += 2)
        for (int s2 = -1; s2 <= 1; s2 += 2)
            for (int s3 = -1; s3 <= 1; s3 += 2) {
                double v[3];
                for (int k = 0; k < 3; ++k) v[k] = 0.5 * (s1 * P->L[k] + s2 * P->L[3 + k] + s3 * P->L[6 + k]);
                hd = std::max(hd, std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]));
            }
    std::vector<std::array<double, 4>> cv;
    {
        const double R = rmax + hd;
        int nr[3];
        for (int a = 0; a < 3; ++a) {
            const double inv = std::sqrt(P->Finv[3 * a] * P->Finv[3 * a] + P->Finv[3 * a + 1] * P->Finv[3 * a + 1] +
                                         P->Finv[3 * a + 2] * P->Finv[3 * a + 2]);
            nr[a] = (int)std::ceil(R * inv) + 1;
        }
        for (int i = -nr[0]; i <= nr[0]; ++i)
            for (int j = -nr[1]; j <= nr[1]; ++j)
                for (int k = -nr[2]; k <= nr[2]; ++k) {
                    double v[3];
                    for (int a = 0; a < 3; ++a) v[a] = i * P->L[a] + j * P->L[3 + a] + k * P->L[6 + a];
                    const double len = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
                    if (len < R) cv.push_back({v[0], v[1], v[2], len});
                }
        std::sort(cv.begin(), cv.end(), [](const std::array<double, 4> &a, const std::array<double, 4> &b) { return a[3] < b[3]; });
    }
    const int ncand = (int)cv.size();
    double *dZ = nullptr, *dX = nullptr, *dC = nullptr, *dn = nullptr;
    if (!ok(cudaMallocAsync((void **)&dZ, sizeof(double) * natom, st)) || !ok(cudaMallocAsync((void **)&dX, sizeof(double) * 3 * natom, st)) ||
        !ok(cudaMallocAsync((void **)&dC, sizeof(double) * 4 * std::max(1, ncand), st)) ||
        !ok(cudaMallocAsync((void **)&dn, sizeof(double) * 2 * std::max(1, w.gc), st)))
        return fail(JK_ERR_OOM, "one-electron scratch");
    cudaMemcpyAsync(dZ, Z, sizeof(double) * natom, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(dX, xyz, sizeof(double) * 3 * natom, cudaMemcpyHostToDevice, st);
    if (ncand) cudaMemcpyAsync(dC, cv.data(), sizeof(double) * 4 * ncand, cudaMemcpyHostToDevice, st);
    if (!ok(cudaMemsetAsync(w.T2, 0, n2 * sizeof(double), st))) return fail(JK_ERR_CUDA, "memset failed");
    for (int c = 0; c < JK_NCLASS_MAX; ++c)
        launch_onee(c, pl, P->spair_class_off[c], P->spair_class_off[c + 1], 1, P->d_ppi_ab, natom, dZ, dX, dC, ncand, w.T2, st);
    // reciprocal part, chunk by chunk of G
    const int ng = (int)(P->gvec.size() / 4);
    for (int g0 = 0; g0 < ng; g0 += w.gc) {
        const int gcur = std::min(w.gc, ng - g0);
        launch_gauss_table(P, g0, gcur, w.gtab, st);
        for (int c = 0; c < JK_NCLASS_MAX; ++c)
            launch_sfac(c, pl, P->spair_class_off[c], P->spair_class_off[c + 1], P->d_gvec, g0, gcur, w.gtab, w.M, st);
        k_nuclear_sfac<<<(gcur + 127) / 128, 128, 0, st>>>(natom, dZ, dX, P->d_gvec, g0, gcur, dn);
        slab_gemv_n(w.M, (long long)n2, 2 * gcur, dn, -1.0, w.T2, st);
    }
    // self term +(pi/(V w^2)) Z_tot S and the component factors
    k_onee_final<<<grid, 256, 0, st>>>(n, P->d_compf, w.T2, P->d_S, kPi / (P->volume * w2) * ztot, V);
    cudaFreeAsync(dZ, st);
    cudaFreeAsync(dX, st);
    cudaFreeAsync(dC, st);
    cudaFreeAsync(dn, st);
    if (!ok(cudaGetLastError()) || !ok(cudaStreamSynchronize(st))) return fail(JK_ERR_CUDA, "nuclear-attraction kernels failed");
    return JK_OK;
}

}  // namespace jk
