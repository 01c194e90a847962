"""Pins of the oracle's one-electron operators of the cell (Sections 2.1 and
2.2 of the paper: kinetic energy and nuclear attraction of point charges
with their images, Ewald-split) against things fixed independently of it:
closed forms, finite differences of the pinned overlap and of the closed
form, omega invariance, and the multipole expansion of the periodic Coulomb
kernel in a large cell."""
import math

import numpy as np
import pytest

import synthcells as sc
from oracle import oracle as O
from test_oracle_pins import GOLD, _pair_moments, _vacuum_cell

TIGHT = dict(pair_R=1e-16, pair_cs=1e-16, ewald_R=1e-16, ewald_K=1e-16)


def _cell(shells, L=40.0, omega=0.4, lat=None):
    lattice = np.eye(3) * L if lat is None else lat
    pos = np.array([s.center for s in shells])
    return sc.Cell("pin", lattice, shells, omega, dict(TIGHT), 1, ["X"] * len(shells), pos)


def _fcs(l):
    return [math.sqrt(np.prod([math.factorial(k) / math.factorial(2 * k) for k in c]))
            for c in [(lx, ly, l - lx - ly) for lx in range(l, -1, -1) for ly in range(l - lx, -1, -1)]]


# ---------------------------------------------------------------- kinetic energy
def test_kinetic_ss_closed_form():
    """s primitives: T_ab = mu (3 - 2 mu |A-B|^2) S_ab with mu = ab/(a+b);
    T_aa = 3a/2 for a normalised s function."""
    a, b = 1.3, 0.7
    A, B = np.array([0.1, -0.2, 0.3]), np.array([0.9, 0.4, -0.5])
    cell = _cell([sc.Shell(0, np.array([a]), np.array([1.0]), A), sc.Shell(0, np.array([b]), np.array([1.0]), B)])
    T, S = O.kinetic(cell), O.overlap(cell)
    mu = a * b / (a + b)
    R2 = float(np.sum((A - B) ** 2))
    assert abs(T[0, 1] - mu * (3 - 2 * mu * R2) * S[0, 1]) < 1e-14
    assert abs(T[0, 0] - 1.5 * a) < 1e-13 and abs(T[1, 1] - 1.5 * b) < 1e-13
    assert np.abs(T - T.T).max() < 1e-15


@pytest.mark.parametrize("la,lb", [(0, 1), (1, 1), (2, 0), (1, 2), (2, 2)])
def test_kinetic_is_laplacian_of_overlap(la, lb):
    """-1/2 nabla^2 acting on nu(r - B) equals -1/2 nabla_B^2 of nu, so T_ab =
    -1/2 sum_axis d^2 S_ab / dB_axis^2: the kinetic matrix against second
    differences (Richardson-extrapolated) of the pinned overlap."""
    A, B = np.array([0.3, -0.1, 0.2]), np.array([1.1, 0.5, -0.4])
    ea, eb = np.array([1.7, 0.45]), np.array([0.9, 0.3])
    ca, cb = np.array([0.6, 0.7]), np.array([0.5, 0.8])

    def S_at(Bv):
        c = _cell([sc.Shell(la, ea, ca, A), sc.Shell(lb, eb, cb, Bv)])
        return O.overlap(c)

    na = (la + 1) * (la + 2) // 2
    T = O.kinetic(_cell([sc.Shell(la, ea, ca, A), sc.Shell(lb, eb, cb, B)]))[:na, na:]

    def lap(h):
        out = 0
        for ax in range(3):
            e = np.zeros(3)
            e[ax] = h
            out = out + (S_at(B + e) - 2 * S_at(B) + S_at(B - e)) / h ** 2
        return out[:na, na:]

    h = 4e-3
    fd = (4 * lap(h / 2) - lap(h)) / 3
    assert np.abs(T - (-0.5) * fd).max() < 2e-8 * max(1.0, np.abs(T).max()), np.abs(T + 0.5 * fd).max()


# ---------------------------------------------------------------- nuclear attraction
def test_nuclear_molecular_ss_closed_form():
    """Bare attraction of point charges by an s-s product: -Z (2 pi/p)
    N_a N_b e^{-mu |A-B|^2} F_0(p |P - C|^2), F_0(T) = (1/2) sqrt(pi/T) erf(sqrt T)
    (Eqs. pbc_v1e_base_case and boys_function_erf_form, one image)."""
    a, b = 1.3, 0.7
    A, B = np.array([0.1, -0.2, 0.3]), np.array([0.9, 0.4, -0.5])
    cell = _cell([sc.Shell(0, np.array([a]), np.array([1.0]), A), sc.Shell(0, np.array([b]), np.array([1.0]), B)])
    Z = np.array([1.5, 0.7])
    C = np.array([[0.4, 0.0, 0.1], [-0.7, 1.2, 0.8]])
    V = O.nuclear(cell, Z, C, parts=O.PART_MOLECULAR)
    p, mu = a + b, a * b / (a + b)
    P = (a * A + b * B) / p
    Na, Nb = (2 * a / math.pi) ** 0.75, (2 * b / math.pi) ** 0.75
    ref = 0.0
    for z, c in zip(Z, C):
        T = p * float(np.sum((P - c) ** 2))
        F0 = 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
        ref -= z * 2 * math.pi / p * Na * Nb * math.exp(-mu * float(np.sum((A - B) ** 2))) * F0
    assert abs(V[0, 1] - ref) < 1e-14 * abs(ref), (V[0, 1], ref)


def _raw_v(la, Acen, a=1.3, b=0.7, B=(0.9, 0.4, -0.5), Z=(1.5,), C=((0.4, 0.0, 0.1),)):
    """Molecular attraction block of single primitives with the normalised
    contraction coefficients and component factors divided out."""
    cell = _cell([sc.Shell(la, np.array([a]), np.array([1.0]), np.asarray(Acen, dtype=float)),
                  sc.Shell(0, np.array([b]), np.array([1.0]), np.asarray(B, dtype=float))])
    V = O.nuclear(cell, np.array(Z), np.array(C), parts=O.PART_MOLECULAR)
    na = (la + 1) * (la + 2) // 2
    ca = O.norm_coefs(la, [a], [1.0])[0] * np.array(_fcs(la))
    cb = O.norm_coefs(0, [b], [1.0])[0]
    return V[:na, na] / (ca * cb)


def test_nuclear_p_d_from_centre_derivatives():
    """The unnormalised p_x primitive is (1/2a) d/dA_x of the s primitive and
    d_xx = (1/4a^2) d^2/dA_x^2 + (1/2a), d_xy = (1/4a^2) d^2/dA_x dA_y: pins
    the E coefficients and R recursion of the oracle's attraction."""
    a = 1.3
    A0 = np.array([0.1, -0.2, 0.3])
    ss = lambda A: _raw_v(0, A)[0]
    p = _raw_v(1, A0)
    h = 1e-4
    for ax in range(3):
        e = np.zeros(3)
        e[ax] = h
        ref = (ss(A0 + e) - ss(A0 - e)) / (2 * h) / (2 * a)
        assert abs(p[ax] - ref) < 1e-8 * max(1.0, abs(ref)), (ax, p[ax], ref)
    d = _raw_v(2, A0)  # xx xy xz yy yz zz
    h = 2e-3
    ex, ey = np.array([h, 0, 0]), np.array([0, h, 0])
    dxx = (ss(A0 + ex) - 2 * ss(A0) + ss(A0 - ex)) / h ** 2 / (4 * a * a) + ss(A0) / (2 * a)
    dxy = (ss(A0 + ex + ey) - ss(A0 + ex - ey) - ss(A0 - ex + ey) + ss(A0 - ex - ey)) / (4 * h * h) / (4 * a * a)
    assert abs(d[0] - dxx) < 2e-6 * max(1.0, abs(dxx)), (d[0], dxx)
    assert abs(d[1] - dxy) < 2e-6 * max(1.0, abs(dxy)), (d[1], dxy)


@pytest.mark.parametrize("which", ["tiny", "skewed"])
def test_nuclear_omega_invariance(which):
    """Real-space, reciprocal and self terms move with omega but their sum
    does not (Eq. pbc_v1e_base_case_final)."""
    cell = sc.config(1) if which == "tiny" else sc.small_random_cell(2, 2, 1, True)
    Vs = [O.nuclear(cell, omega=w) for w in (0.35, 0.6, 1.1)]
    scale = np.abs(Vs[0]).max()
    for V in Vs[1:]:
        assert np.abs(V - Vs[0]).max() < 1e-11 * max(1.0, scale), np.abs(V - Vs[0]).max()
    parts = [O.nuclear(cell, omega=0.6, parts=k) for k in (1, 2, 4)]
    assert min(np.abs(x).max() for x in parts) > 1e-6  # every part contributes


@pytest.mark.slow
def test_nuclear_large_cell_multipoles():
    """V_periodic - V_molecular = -sum_C Z_C [-(xi/L) S_ab + (2 pi/(3 L^3))
    <a| |r - C|^2 |b>] + O(L^-5) in a cubic cell of side L (the periodic
    kernel with its K = 0 part removed is 1/r - xi/L + (2 pi / 3V) r^2 + ...):
    pins the normalisation of the reciprocal and self terms."""
    xi = GOLD["sc_wigner_xi"]["value"]
    Z = np.array([1.0, 2.0])
    C = np.array([[0.5, 0.2, -0.1], [-0.3, 0.4, 0.6]])
    res = []
    for L in [30.0, 45.0, 60.0]:
        cell = _vacuum_cell(L)
        per = O.nuclear(cell, Z, C, delta=1e-17)
        mol = O.nuclear(cell, Z, C, parts=O.PART_MOLECULAR)
        S, d, M2 = _pair_moments(cell)
        corr = 0
        for z, c in zip(Z, C):
            m2c = M2 - 2 * np.einsum("abx,x->ab", d, c) + float(c @ c) * S
            corr = corr - z * (-(xi / L) * S + (2 * math.pi / (3 * L ** 3)) * m2c)
        diff = per - mol
        r = np.abs(diff - corr).max()
        res.append(r)
        assert np.abs(diff).max() > 1e3 * r
    assert res[2] < res[0] * (30.0 / 60.0) ** 4 * 1.5
