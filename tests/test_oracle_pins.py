"""Pins of the FP64 oracle to things other than itself.

Each test checks one part of the oracle against a closed form, an
independent quadrature, a finite-difference identity, a published constant
or an invariant that the mathematics fixes (arXiv:2410.22278 prints no
worked numerical example).  A plausible mistake in each part (a dropped
term, a wrong sign or index, a transposed operand) fails one of these.
"""
import json
import math
import os

import numpy as np
import pytest

import synthcells as sc
from oracle import oracle as O

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "constants.json")))


# ---------------------------------------------------------------- Boys
def _boys_quadrature(m, T, n=30, pieces=40):
    # composite Gauss-Legendre on [0, 1] of t^{2m} exp(-T t^2): independent of the series
    x, w = np.polynomial.legendre.leggauss(n)
    edges = np.linspace(0.0, 1.0, pieces + 1)
    tot = 0.0
    for lo, hi in zip(edges[:-1], edges[1:]):
        t = lo + 0.5 * (x + 1.0) * (hi - lo)
        tot += 0.5 * (hi - lo) * np.sum(w * t ** (2 * m) * np.exp(-T * t * t))
    return tot


@pytest.mark.parametrize("T", [0.0, 1e-6, 0.03, 0.7, 3.0, 11.0, 29.5, 59.9, 60.1, 85.0, 400.0])
def test_boys_against_quadrature_and_closed_form(T):
    F = O.boys(10, T)
    for m in range(11):
        ref = _boys_quadrature(m, T) if T < 200 else None
        if ref is not None:
            assert abs(F[m] - ref) <= 2e-15 * max(1.0, abs(ref)) + 1e-17, (m, T, F[m] - ref)
    # Eq. boys_function_erf_form
    f0 = 1.0 if T == 0 else 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
    assert abs(F[0] - f0) <= 2e-16 * max(1, f0) + 1e-18


def test_boys_limits_and_recursion():
    F = O.boys(8, 0.0)
    assert np.allclose(F, [1.0 / (2 * m + 1) for m in range(9)], rtol=0, atol=1e-16)
    T = 250.0
    F = O.boys(8, T)
    for m in range(9):
        dfact = np.prod(np.arange(2 * m - 1, 0, -2)) if m > 0 else 1.0
        asym = dfact / 2 ** (m + 1) * math.sqrt(math.pi / T ** (2 * m + 1))
        assert abs(F[m] / asym - 1) < 1e-14
    for T in [0.5, 5.0, 40.0]:
        F = O.boys(9, T)
        for m in range(9):
            assert abs(F[m] - (2 * T * F[m + 1] + math.exp(-T)) / (2 * m + 1)) < 1e-15


# ---------------------------------------------------------------- normalisation
def _gauss_hermite_1d_overlap(i, a, j, b, A, B, n=80):
    # int (x-A)^i (x-B)^j exp(-a (x-A)^2 - b (x-B)^2) dx by Gauss-Hermite
    p = a + b
    P = (a * A + b * B) / p
    x, w = np.polynomial.hermite.hermgauss(n)
    xs = P + x / math.sqrt(p)
    pref = math.exp(-a * b / p * (A - B) ** 2) / math.sqrt(p)
    return pref * np.sum(w * (xs - A) ** i * (xs - B) ** j)


@pytest.mark.parametrize("l", [0, 1, 2])
def test_contracted_functions_have_unit_self_overlap(l):
    exps = np.array([13.0, 2.1, 0.31])
    coefs = np.array([0.3, 0.55, 0.9])
    cn = O.norm_coefs(l, exps, coefs)
    comps = [(lx, ly, l - lx - ly) for lx in range(l, -1, -1) for ly in range(l - lx, -1, -1)]
    for c in comps:
        fc = math.sqrt(np.prod([math.factorial(k) / math.factorial(2 * k) for k in c]))
        s = 0.0
        for i in range(3):
            for j in range(3):
                v = cn[i] * cn[j] * fc * fc
                for ax in range(3):
                    v *= _gauss_hermite_1d_overlap(c[ax], exps[i], c[ax], exps[j], 0.0, 0.0)
                s += v
        assert abs(s - 1.0) < 1e-13, (l, c, s)


# ---------------------------------------------------------------- molecular ERIs
def _ssss(ex, ctr):
    a, b, c, d = ex
    A, B, C, D = [np.asarray(x) for x in ctr]
    p, q = a + b, c + d
    P, Q = (a * A + b * B) / p, (c * C + d * D) / q
    Kab = math.exp(-a * b / p * np.sum((A - B) ** 2))
    Kcd = math.exp(-c * d / q * np.sum((C - D) ** 2))
    al = p * q / (p + q)
    T = al * np.sum((P - Q) ** 2)
    F0 = 1.0 if T == 0 else 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
    return 2 * math.pi ** 2.5 / (p * q * math.sqrt(p + q)) * Kab * Kcd * F0


EX = [1.3, 0.7, 0.9, 2.2]
CTR = [[0.1, -0.2, 0.3], [0.9, 0.4, -0.5], [-0.6, 1.1, 0.2], [0.3, 0.8, 1.4]]


def test_ssss_closed_form():
    """Eq. pbc_eri_base_case without a lattice: 2 pi^{5/2}/(pq sqrt(p+q)) F_0."""
    v = O.molecular_prim_eri([0, 0, 0, 0], EX, CTR)[0, 0, 0, 0]
    assert abs(v - _ssss(EX, CTR)) < 1e-14


def test_erfc_split_ssss_closed_form():
    """The erfc part is bare minus erf, and the erf part of (ss|ss) is
    pref sqrt(alpha_w/alpha) F_0(alpha_w R^2) (Eq. boys_function_split)."""
    w = 0.45
    a, b, c, d = EX
    p, q = a + b, c + d
    al = p * q / (p + q)
    aw = 1 / (1 / p + 1 / q + 1 / w ** 2)
    A, B, C, D = [np.asarray(x) for x in CTR]
    P, Q = (a * A + b * B) / p, (c * C + d * D) / q
    R2 = np.sum((P - Q) ** 2)
    Kab = math.exp(-a * b / p * np.sum((A - B) ** 2))
    Kcd = math.exp(-c * d / q * np.sum((C - D) ** 2))
    pref = 2 * math.pi ** 2.5 / (p * q * math.sqrt(p + q)) * Kab * Kcd
    erf_part = pref * math.sqrt(aw / al) * 0.5 * math.sqrt(math.pi / (aw * R2)) * math.erf(math.sqrt(aw * R2))
    v = O.molecular_prim_eri([0, 0, 0, 0], EX, CTR, omega=w)[0, 0, 0, 0]
    assert abs(v - (_ssss(EX, CTR) - erf_part)) < 1e-14


def _fd_eri(lmask, h=1e-4, omega=0.0):
    """(ss|ss) differentiated once per centre flagged in lmask (list of axis
    or -1), divided by 2*exponent: the unnormalised p component along that
    axis is (1/2a) d/dA of the s primitive.  Central differences."""
    import itertools

    idx = [(k, ax) for k, ax in enumerate(lmask) if ax >= 0]
    tot = 0.0
    for signs in itertools.product([1, -1], repeat=len(idx)):
        ctr = [list(c) for c in CTR]
        for (k, ax), s in zip(idx, signs):
            ctr[k][ax] += s * h
        v = O.molecular_prim_eri([0, 0, 0, 0], EX, ctr, omega=omega)[0, 0, 0, 0]
        tot += np.prod(signs) * v
    tot /= (2 * h) ** len(idx)
    for k, ax in idx:
        tot /= 2 * EX[k]
    return tot


@pytest.mark.parametrize("omega", [0.0, 0.6])
def test_p_functions_are_centre_derivatives(omega):
    """(p_x s|ss) = (1/2a) d(ss|ss)/dA_x, and likewise on every centre: pins the
    E recursion, the R recursion and the ket sign (-1)^{|s|} (reading of the
    real-space term of Eq. pbc_eri_general_final)."""
    blk = O.molecular_prim_eri([1, 1, 1, 1], EX, CTR, omega=omega)
    for combo in [(0, -1, -1, -1), (-1, 1, -1, -1), (-1, -1, 2, -1), (-1, -1, -1, 0), (0, 1, -1, -1), (-1, -1, 1, 2),
                  (2, -1, 0, -1), (0, -1, -1, 0), (1, 2, 0, 1)]:
        ls = [1 if ax >= 0 else 0 for ax in combo]
        ref = _fd_eri(list(combo), h=2e-3 if sum(ls) > 2 else 1e-4, omega=omega)
        sub = O.molecular_prim_eri(ls, EX, CTR, omega=omega)
        v = sub[tuple(ax if ax >= 0 else 0 for ax in combo)]
        # the same element inside the (pp|pp) block (s->p promoted along the axis)
        assert abs(v - ref) < (2e-6 if sum(ls) > 2 else 1e-8) * max(1.0, abs(ref)), (combo, v, ref)
    assert blk.shape == (3, 3, 3, 3)


def test_d_functions_are_second_derivatives():
    """(d_xx s|ss) = (1/4a^2) d^2/dA_x^2 (ss|ss) + (1/2a)(ss|ss);
    (d_xy s|ss) = (1/4a^2) d^2/dA_x dA_y (ss|ss)."""
    h = 1e-3
    a = EX[0]

    def f(dx, dy):
        ctr = [list(c) for c in CTR]
        ctr[0][0] += dx
        ctr[0][1] += dy
        return O.molecular_prim_eri([0, 0, 0, 0], EX, ctr)[0, 0, 0, 0]

    d2xx = (f(h, 0) - 2 * f(0, 0) + f(-h, 0)) / h ** 2
    d2xy = (f(h, h) - f(h, -h) - f(-h, h) + f(-h, -h)) / (4 * h * h)
    blk = O.molecular_prim_eri([2, 0, 0, 0], EX, CTR)[:, 0, 0, 0]
    assert abs(blk[0] - (d2xx / (4 * a * a) + f(0, 0) / (2 * a))) < 1e-6
    assert abs(blk[1] - d2xy / (4 * a * a)) < 1e-6


def test_eightfold_symmetry_molecular():
    ls = [1, 2, 0, 1]
    v = O.molecular_prim_eri(ls, EX, CTR)
    sw = O.molecular_prim_eri([ls[1], ls[0], ls[2], ls[3]], [EX[1], EX[0], EX[2], EX[3]], [CTR[1], CTR[0], CTR[2], CTR[3]])
    assert np.abs(v - sw.transpose(1, 0, 2, 3)).max() < 1e-14
    bk = O.molecular_prim_eri([ls[2], ls[3], ls[0], ls[1]], [EX[2], EX[3], EX[0], EX[1]], [CTR[2], CTR[3], CTR[0], CTR[1]])
    assert np.abs(v - bk.transpose(2, 3, 0, 1)).max() < 1e-14


# ---------------------------------------------------------------- Ewald point charges
def _nacl(r0):
    a = 2 * r0
    fcc = np.array([[0, 0, 0], [0, 0.5, 0.5], [0.5, 0, 0.5], [0.5, 0.5, 0]]) * a
    xyz = np.vstack([fcc, fcc + np.array([a / 2, 0, 0])])
    q = np.array([1.0] * 4 + [-1.0] * 4)
    return np.eye(3) * a, q, xyz


@pytest.mark.parametrize("r0,omega", [(2.0, 0.3), (2.0, 0.9), (5.3, 0.25), (5.3, 0.6)])
def test_nacl_madelung_constant(r0, omega):
    lat, q, xyz = _nacl(r0)
    E = O.ewald_point_charges(lat, q, xyz, omega)
    M = -E * r0 / 4.0
    g = GOLD["nacl_madelung"]
    assert abs(M - g["value"]) < g["tolerance"], M


def test_single_charge_background_term():
    """One unit charge per cubic cell: -xi/(2L), omega-invariant (exercises the
    -(4 pi/V)/(4 w^2) term of Eq. nuclear_repulsion_energy)."""
    for L in [3.0, 7.0]:
        vals = [O.ewald_point_charges(np.eye(3) * L, [1.0], [[0.3, 0.1, 0.2]], w / L) for w in [2.0, 3.5, 5.0]]
        assert max(vals) - min(vals) < 1e-12
        xi = -2 * L * vals[0]
        assert abs(xi - GOLD["sc_wigner_xi"]["value"]) < GOLD["sc_wigner_xi"]["tolerance"], xi


# ---------------------------------------------------------------- pair list (Section 3.1)
def test_pair_list_matches_brute_force_enumeration():
    """The oracle's local pairs equal a brute-force scan of a large cube of
    lattice vectors against Eqs. pbc_eri_pair_cutoff_implementation and
    pbc_eri_cauchy_schwarz_cutoff_implementation."""
    cell = sc.small_random_cell(3, natom=2, lmax=2, skew=True)
    lp = O.local_pairs(cell)
    got = set((int(r[0]), int(r[1]), int(r[2]), int(r[3]), int(r[4]), int(r[5]), int(r[6])) for r in lp)
    amin = min(s.exps.min() for s in cell.shells)
    dR, dCS = cell.cutoffs["pair_R"], cell.cutoffs["pair_cs"]
    cmax = {0: 1.0, 1: math.sqrt(0.5), 2: 0.5}
    n = 7
    g = np.array([(i, j, k) for i in range(-n, n + 1) for j in range(-n, n + 1) for k in range(-n, n + 1)])
    Rv = g @ cell.lattice
    want = set()
    for I, si in enumerate(cell.shells):
        ci = O.norm_coefs(si.l, si.exps, si.coefs) * cmax[si.l]
        for J, sj in enumerate(cell.shells):
            cj = O.norm_coefs(sj.l, sj.exps, sj.coefs) * cmax[sj.l]
            for ia, a in enumerate(si.exps):
                for ib, b in enumerate(sj.exps):
                    p = a + b
                    cc = abs(ci[ia] * cj[ib])
                    x1 = math.sqrt(2) * math.pi ** 1.25 * cc / (p * math.sqrt(p + 2 * amin) * dR)
                    x2 = 2 ** 0.25 * math.pi ** 1.25 * cc / (p ** 1.25 * dCS)
                    if x1 <= 1 or x2 <= 1:
                        continue
                    r = min(math.sqrt(p / (a * b) * math.log(x1)), math.sqrt(p / (a * b) * math.log(x2)))
                    d = np.linalg.norm(si.center - sj.center - Rv, axis=1)
                    for k in np.nonzero(d < r)[0]:
                        want.add((I, J, ia, ib, *[int(x) for x in g[k]]))
    assert got == want
    assert len(got) > 100


# ---------------------------------------------------------------- Fourier transform of pair densities
def test_pair_fourier_transform_against_quadrature():
    """Structure factor of one AO pair in a large cell (only the R = 0 image)
    equals a direct 1-D quadrature of int rho exp(-iG.r) per axis."""
    L = 60.0
    sh = [sc.Shell(1, np.array([1.7, 0.45]), np.array([0.6, 0.7]), np.array([1.0, 2.0, 3.0])),
          sc.Shell(2, np.array([0.8]), np.array([1.0]), np.array([1.6, 1.5, 2.4]))]
    cell = sc.Cell("ft", np.eye(3) * L, sh, 0.5, dict(pair_R=1e-14, pair_cs=1e-14, ewald_R=1e-14, ewald_K=1e-14), 1)
    G = np.array([2, -1, 3]) * (2 * math.pi / L)
    M = O.pair_ft(cell, G)
    c1 = O.norm_coefs(1, sh[0].exps, sh[0].coefs)
    c2 = O.norm_coefs(2, sh[1].exps, sh[1].coefs)
    x = np.linspace(-20, 25, 200001)
    dx = x[1] - x[0]
    comps1 = [(1, 0, 0), (0, 1, 0), (0, 0, 1)]
    comps2 = [(2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1), (0, 0, 2)]

    def fc(c):
        return math.sqrt(np.prod([math.factorial(k) / math.factorial(2 * k) for k in c]))

    for i1, c in enumerate(comps1):
        for i2, d in enumerate(comps2):
            tot = 0.0 + 0.0j
            for ia, a in enumerate(sh[0].exps):
                v = c1[ia] * c2[0] * fc(c) * fc(d)
                for ax in range(3):
                    A, B = sh[0].center[ax], sh[1].center[ax]
                    f = (x - A) ** c[ax] * (x - B) ** d[ax] * np.exp(-a * (x - A) ** 2 - sh[1].exps[0] * (x - B) ** 2)
                    v = v * np.sum(f * np.exp(-1j * G[ax] * x)) * dx
                tot += v
            assert abs(M[i1, 3 + i2] - tot) < 1e-11, (c, d, M[i1, 3 + i2], tot)


# ---------------------------------------------------------------- periodic ERIs
@pytest.fixture(scope="module")
def tiny():
    cell = sc.config(1)
    D = O.density(cell)
    return cell, D


def test_tiny_density_is_normalised(tiny):
    cell, D = tiny
    S = O.overlap(cell)
    assert abs(np.sum(D * S) - 2 * cell.n_occ) < 1e-12
    assert np.abs(S - S.T).max() < 1e-15
    assert np.linalg.eigvalsh(S).min() > 0


@pytest.mark.slow
def test_omega_invariance_and_reciprocal_only_limit(tiny):
    """Per ERI and for J, K, E: the Ewald-split result is independent of omega
    (Section 3.4) and equals the reciprocal-only sum (omega -> infinity, no
    real-space or background term)."""
    cell, D = tiny
    ref = O.eri_tensor(cell, omega=math.inf, delta=1e-16)
    Jr, Kr = O.jk_from_eri(ref, D)
    for w in [0.3, 0.5, 0.8, 1.5]:
        e = O.eri_tensor(cell, omega=w)
        assert np.abs(e - ref).max() < 1e-9, w
        J, K = O.jk_from_eri(e, D)
        assert np.abs(J - Jr).max() < 1e-9 and np.abs(K - Kr).max() < 1e-9
        EJ, EK = O.energies(D, J, K)
        EJr, EKr = O.energies(D, Jr, Kr)
        assert abs(EJ - EJr) < 1e-9 and abs(EK - EKr) < 1e-9


def test_eri_symmetry_and_positivity(tiny):
    cell, D = tiny
    e = O.eri_tensor(cell)
    n = e.shape[0]
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (1, 0, 3, 2), (3, 2, 1, 0)]:
        assert np.abs(e - e.transpose(perm)).max() < 1e-13
    # with the K = 0 component removed the Coulomb kernel is positive semidefinite
    ev = np.linalg.eigvalsh(e.reshape(n * n, n * n))
    assert ev.min() > -1e-11
    J, K = O.jk_from_eri(e, D)
    EJ, EK = O.energies(D, J, K)
    assert EJ > 0 and np.sum(D * K) > 0
    assert np.abs(J - J.T).max() < 1e-13 and np.abs(K - K.T).max() < 1e-13


def test_background_closed_form(tiny):
    """The background part of the tensor is -(pi/(V w^2)) S_mn S_ls, hence
    J_bg = -(pi/(V w^2)) Tr(DS) S and K_bg = -(pi/(V w^2)) S D S."""
    cell, D = tiny
    bg = O.eri_tensor(cell, parts=O.PART_BG)
    S = O.overlap(cell)
    c = -math.pi / (cell.volume * cell.omega ** 2)
    J, K = O.jk_from_eri(bg, D)
    assert np.abs(J - c * np.sum(D * S) * S).max() < 1e-14
    assert np.abs(K - c * S @ D @ S).max() < 1e-14


def test_rows_agree_with_tensor(tiny):
    cell, D = tiny
    e = O.eri_tensor(cell)
    J, K = O.jk_from_eri(e, D)
    rows = [1, 2]
    Jr, Kr = O.jk_rows(cell, D, rows)
    idx = O.row_indices(cell, rows)
    assert np.abs(Jr - J[idx]).max() < 1e-12
    assert np.abs(Kr - K[idx]).max() < 1e-12


def _vacuum_cell(L):
    sh = [sc.Shell(0, np.array([1.6, 0.5]), np.array([0.5, 0.6]), np.array([0.2, 0.1, -0.3])),
          sc.Shell(1, np.array([1.1]), np.array([1.0]), np.array([0.9, -0.4, 0.6]))]
    cut = dict(pair_R=1e-16, pair_cs=1e-16, ewald_R=1e-16, ewald_K=1e-16)
    return sc.Cell("vac", np.eye(3) * L, sh, 0.35, cut, 1)


def _contracted_molecular_eri(cell):
    """Bare-Coulomb contracted ERIs (no lattice) from the primitive routine."""
    off, n = O.ao_offsets(cell)
    out = np.zeros((n,) * 4)
    cn = [O.norm_coefs(s.l, s.exps, s.coefs) for s in cell.shells]

    def fcs(l):
        return [math.sqrt(np.prod([math.factorial(k) / math.factorial(2 * k) for k in c]))
                for c in [(lx, ly, l - lx - ly) for lx in range(l, -1, -1) for ly in range(l - lx, -1, -1)]]

    S = cell.shells
    for I in range(len(S)):
        for J in range(len(S)):
            for K in range(len(S)):
                for L_ in range(len(S)):
                    blk = 0
                    for a in range(S[I].nprim):
                        for b in range(S[J].nprim):
                            for c in range(S[K].nprim):
                                for d in range(S[L_].nprim):
                                    v = O.molecular_prim_eri(
                                        [S[I].l, S[J].l, S[K].l, S[L_].l],
                                        [S[I].exps[a], S[J].exps[b], S[K].exps[c], S[L_].exps[d]],
                                        [S[I].center, S[J].center, S[K].center, S[L_].center])
                                    blk = blk + v * cn[I][a] * cn[J][b] * cn[K][c] * cn[L_][d]
                    f = np.einsum("i,j,k,l->ijkl", fcs(S[I].l), fcs(S[J].l), fcs(S[K].l), fcs(S[L_].l))
                    out[off[I]:off[I] + blk.shape[0], off[J]:off[J] + blk.shape[1], off[K]:off[K] + blk.shape[2],
                        off[L_]:off[L_] + blk.shape[3]] = blk * f
    return out


def _pair_moments(cell, n=60):
    """Charge S, dipole d and second moment M2 of every AO pair density, by
    Gauss-Hermite quadrature (no lattice images; the cell is large)."""
    off, nbf = O.ao_offsets(cell)
    cn = [O.norm_coefs(s.l, s.exps, s.coefs) for s in cell.shells]
    comps = {0: [(0, 0, 0)], 1: [(1, 0, 0), (0, 1, 0), (0, 0, 1)]}
    S = np.zeros((nbf, nbf))
    d = np.zeros((nbf, nbf, 3))
    M2 = np.zeros((nbf, nbf))
    x, w = np.polynomial.hermite.hermgauss(n)
    for I, si in enumerate(cell.shells):
        for J, sj in enumerate(cell.shells):
            for ia, a in enumerate(si.exps):
                for ib, b in enumerate(sj.exps):
                    p = a + b
                    for ci, c1 in enumerate(comps[si.l]):
                        for cj, c2 in enumerate(comps[sj.l]):
                            m = np.zeros((3, 3))  # axis, power 0..2
                            for ax in range(3):
                                A, B = si.center[ax], sj.center[ax]
                                P = (a * A + b * B) / p
                                xs = P + x / math.sqrt(p)
                                pref = math.exp(-a * b / p * (A - B) ** 2) / math.sqrt(p)
                                base = (xs - A) ** c1[ax] * (xs - B) ** c2[ax]
                                for k in range(3):
                                    m[ax, k] = pref * np.sum(w * base * xs ** k)
                            coef = cn[I][ia] * cn[J][ib]
                            s0 = coef * m[0, 0] * m[1, 0] * m[2, 0]
                            dd = coef * np.array([m[0, 1] * m[1, 0] * m[2, 0], m[0, 0] * m[1, 1] * m[2, 0], m[0, 0] * m[1, 0] * m[2, 1]])
                            mm = coef * (m[0, 2] * m[1, 0] * m[2, 0] + m[0, 0] * m[1, 2] * m[2, 0] + m[0, 0] * m[1, 0] * m[2, 2])
                            fc = 1.0 if si.l == 0 else math.sqrt(0.5)
                            fc *= 1.0 if sj.l == 0 else math.sqrt(0.5)
                            S[off[I] + ci, off[J] + cj] += fc * s0
                            d[off[I] + ci, off[J] + cj] += fc * dd
                            M2[off[I] + ci, off[J] + cj] += fc * mm
    return S, d, M2


@pytest.mark.slow
def test_large_vacuum_cell_multipole_asymptotics():
    """(ab|cd)_periodic - (ab|cd)_molecular = -(xi/L) S_ab S_cd
    + (2 pi/(3 L^3)) [S_ab M2_cd + S_cd M2_ab - 2 d_ab.d_cd] + O(L^-5) for
    compact distributions in a cubic cell of side L (the periodic Coulomb
    kernel with its K = 0 component removed is 1/r - xi/L + (2 pi/3V) r^2 +
    ...).  Pins the normalisation of the reciprocal and background terms."""
    xi = GOLD["sc_wigner_xi"]["value"]
    res = []
    for L in [30.0, 45.0, 60.0]:
        cell = _vacuum_cell(L)
        per = O.eri_tensor(cell, delta=1e-17)
        mol = _contracted_molecular_eri(cell)
        S, d, M2 = _pair_moments(cell)
        corr = -(xi / L) * np.einsum("ab,cd->abcd", S, S) + (2 * math.pi / (3 * L ** 3)) * (
            np.einsum("ab,cd->abcd", S, M2) + np.einsum("ab,cd->abcd", M2, S) - 2 * np.einsum("abx,cdx->abcd", d, d))
        diff = per - mol
        r = np.abs(diff - corr).max()
        res.append(r)
        assert np.abs(diff).max() > 1e3 * r  # the correction explains the difference
    # residual falls at least like L^-4 (expected L^-5)
    assert res[2] < res[0] * (30.0 / 60.0) ** 4 * 1.5
