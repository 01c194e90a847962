"""Seeded synthetic cells, bases and orbital matrices.

Stand-ins for the paper's workloads (ice XI, Si, ZnO, ... with def2-SVP,
Section 4), which are not available: a two-atom tiny cell, a water-like box
(molecular crystal), diamond-like supercells (dense covalent solid) and a
stream of serving requests.  Everything is in bohr.  Shell exponents are
log-uniform over a split-valence-like range, sorted descending; contraction
coefficients are raw draws in (0.1, 1) that each implementation normalises
itself.

This module holds none of the J/K method's arithmetic: it draws positions,
exponents, coefficients and Gaussian matrices.  ``density_from_overlap`` is
plain linear algebra on an overlap matrix that the caller computes.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .rng import Stream, stream

BOHR_PER_ANGSTROM = 1.0 / 0.529177210903  # CODATA 2018 Bohr radius


def ncart(l: int) -> int:
    return (l + 1) * (l + 2) // 2


@dataclass
class Shell:
    l: int
    exps: np.ndarray
    coefs: np.ndarray  # raw contraction coefficients, not normalised
    center: np.ndarray  # bohr

    @property
    def nprim(self) -> int:
        return len(self.exps)


@dataclass
class Cell:
    name: str
    lattice: np.ndarray  # 3x3, rows are the lattice vectors a, b, c (bohr)
    shells: list
    omega: float
    cutoffs: dict  # pair_R, pair_cs, ewald_R, ewald_K
    n_occ: int
    symbols: list = field(default_factory=list)
    positions: np.ndarray = None  # (natom, 3) bohr
    orbital_key: int = 0

    @property
    def nbf(self) -> int:
        return sum(ncart(s.l) for s in self.shells)

    @property
    def volume(self) -> float:
        return abs(float(np.linalg.det(self.lattice)))

    def orbital_guess(self) -> np.ndarray:
        """Seeded Gaussian matrix X (nbf x n_occ) from which the occupied
        orbitals are made by orthonormalising in the overlap metric."""
        st = Stream(self.orbital_key)
        return st.normal(self.nbf * self.n_occ).reshape(self.nbf, self.n_occ)


def density_from_overlap(X: np.ndarray, S: np.ndarray) -> np.ndarray:
    """D = 2 C C^T with C = X L^{-T}, L L^T = X^T S X, so that C^T S C = 1."""
    M = X.T @ S @ X
    M = 0.5 * (M + M.T)
    L = np.linalg.cholesky(M)
    C = np.linalg.solve(L, X.T).T  # X L^{-T}
    D = 2.0 * C @ C.T
    return 0.5 * (D + D.T)


def _draw_shell_params(st: Stream, l: int, nprim: int, lo: float, hi: float):
    exps = np.sort(st.loguniform(nprim, lo, hi))[::-1].copy()
    coefs = st.uniform(nprim, 0.1, 1.0)
    return exps, coefs


def _basis_for(st: Stream, spec, lo, hi):
    """spec: list of (l, nprim).  Returns list of (l, exps, coefs)."""
    return [(l, *_draw_shell_params(st, l, n, lo, hi)) for (l, n) in spec]


def _attach(basis, center):
    return [Shell(l, e.copy(), c.copy(), np.array(center, dtype=np.float64)) for (l, e, c) in basis]


DEFAULT_CUTOFFS = dict(pair_R=1e-14, pair_cs=1e-14, ewald_R=1e-14, ewald_K=1e-14)


def tiny_cell() -> Cell:
    """Cubic a = 4.0 A, atoms at 0 and (1/2,1/2,1/2)a, s(3)+p(2) on each atom,
    exponents log-uniform in [0.2, 20], 8 basis functions, omega = 0.5."""
    a = 4.0 * BOHR_PER_ANGSTROM
    lat = np.eye(3) * a
    st = stream(1, 1)
    basis = _basis_for(st, [(0, 3), (1, 2)], 0.2, 20.0)
    pos = np.array([[0.0, 0.0, 0.0], [0.5 * a, 0.5 * a, 0.5 * a]])
    shells = _attach(basis, pos[0]) + _attach(basis, pos[1])
    cut = dict(pair_R=1e-12, pair_cs=1e-12, ewald_R=1e-12, ewald_K=1e-12)
    return Cell("tiny", lat, shells, 0.5, cut, 2, ["X", "X"], pos, orbital_key=(stream(1, 9).key.item()))


def _rotation_from_quaternion(q):
    w, x, y, z = q
    return np.array(
        [
            [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
            [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
            [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
        ]
    )


def _random_quaternion(st: Stream):
    u1, u2, u3 = st.uniform(3)
    return np.array(
        [
            np.sqrt(1 - u1) * np.sin(2 * np.pi * u2),
            np.sqrt(1 - u1) * np.cos(2 * np.pi * u2),
            np.sqrt(u1) * np.sin(2 * np.pi * u3),
            np.sqrt(u1) * np.cos(2 * np.pi * u3),
        ]
    )


def _min_image_dist(lat, d):
    f = np.linalg.solve(lat.T, d.T).T
    f -= np.round(f)
    return np.linalg.norm(f @ lat, axis=-1)


WATER_SPEC_O = [(0, 6), (0, 3), (0, 1), (1, 3), (1, 1)]
WATER_SPEC_H = [(0, 3), (0, 1)]


def water_basis():
    st = stream(2, 1)
    return _basis_for(st, WATER_SPEC_O, 0.1, 5000.0), _basis_for(st, WATER_SPEC_H, 0.1, 5000.0)


def _water_box(key_geo: Stream, nmol: int, edge_bohr: float):
    lat = np.eye(3) * edge_bohr
    roh = 0.957 * BOHR_PER_ANGSTROM
    th = np.deg2rad(104.5)
    local = np.array(
        [[0.0, 0.0, 0.0], [roh * np.sin(th / 2), 0.0, roh * np.cos(th / 2)], [-roh * np.sin(th / 2), 0.0, roh * np.cos(th / 2)]]
    )
    dmin = 2.6 * BOHR_PER_ANGSTROM
    oxy = []
    tries = 0
    while len(oxy) < nmol:
        tries += 1
        if tries > 2_000_000:
            raise RuntimeError("water packing failed")
        p = key_geo.uniform(3) @ lat
        if oxy and np.min(_min_image_dist(lat, np.array(oxy) - p)) < dmin:
            continue
        oxy.append(p)
    syms, pos = [], []
    for o in oxy:
        R = _rotation_from_quaternion(_random_quaternion(key_geo))
        for s, r in zip(["O", "H", "H"], local @ R.T + o):
            syms.append(s)
            pos.append(r)
    return lat, syms, np.array(pos)


def water_cell(nmol: int = 64, edge_angstrom: float = 12.42, omega: float = 0.4, cutoffs=None, n_occ: int = 256,
               config_index: int = 2, geo_purpose: int = 2) -> Cell:
    """64 rigid H2O in a cubic box a = 12.42 A, random orientations, minimum
    O-O distance 2.6 A; O: 1s(6) 2s(3) 2s(1) 2p(3) 2p(1), H: s(3) s(1)."""
    bo, bh = water_basis()
    lat, syms, pos = _water_box(stream(config_index, geo_purpose), nmol, edge_angstrom * BOHR_PER_ANGSTROM)
    shells = []
    for s, r in zip(syms, pos):
        shells += _attach(bo if s == "O" else bh, r)
    cut = dict(DEFAULT_CUTOFFS if cutoffs is None else cutoffs)
    return Cell("water%d" % nmol, lat, shells, omega, cut, n_occ, syms, pos,
                orbital_key=stream(config_index, 9 + geo_purpose).key.item())


DIAMOND_FRAC = np.array(
    [[0, 0, 0], [0, 0.5, 0.5], [0.5, 0, 0.5], [0.5, 0.5, 0], [0.25, 0.25, 0.25], [0.25, 0.75, 0.75], [0.75, 0.25, 0.75],
     [0.75, 0.75, 0.25]]
)
DIAMOND_SPEC = [(0, 6), (0, 3), (1, 1), (2, 1)]
DIAMOND_LARGE_SPEC = [(0, 6), (0, 4), (1, 1)]


def diamond_basis(large: bool = False):
    if large:
        return _basis_for(stream(5, 1), DIAMOND_LARGE_SPEC, 0.15, 3000.0)
    return _basis_for(stream(3, 1), DIAMOND_SPEC, 0.15, 3000.0)


def _diamond_positions(st: Stream, n: int, a_conv_bohr: float, jitter_bohr: float):
    pos = []
    for i in range(n):
        for j in range(n):
            for k in range(n):
                for f in DIAMOND_FRAC:
                    pos.append((np.array([i, j, k]) + f) * a_conv_bohr)
    pos = np.array(pos)
    pos += jitter_bohr * st.normal(pos.size).reshape(pos.shape)
    return pos


def diamond_cell(n: int = 3, omega: float = 0.5, cutoffs=None, n_occ=None, large: bool = False,
                 config_index: int = 3, geo_purpose: int = 2) -> Cell:
    """n x n x n conventional diamond supercell, a = 3.5667 A per cell, with a
    seeded 0.05 A Gaussian jitter; basis s(6) s(3) p(1) d(1) (or s(6) s(4) p(1)
    for the large cell), exponents log-uniform in [0.15, 3000]."""
    a_conv = 3.5667 * BOHR_PER_ANGSTROM
    pos = _diamond_positions(stream(config_index, geo_purpose), n, a_conv, 0.05 * BOHR_PER_ANGSTROM)
    basis = diamond_basis(large)
    shells = []
    for r in pos:
        shells += _attach(basis, r)
    lat = np.eye(3) * (n * a_conv)
    cut = dict(DEFAULT_CUTOFFS if cutoffs is None else cutoffs)
    natom = len(pos)
    if n_occ is None:
        n_occ = 3 * natom
    return Cell("diamond%d" % n + ("L" if large else ""), lat, shells, omega, cut, n_occ, ["C"] * natom, pos,
                orbital_key=stream(config_index, 9 + geo_purpose).key.item())


def large_cell() -> Cell:
    """6x6x6 diamond, 1728 atoms, s(6) s(4) p(1), omega = 0.4, Schwarz 1e-11."""
    cut = dict(DEFAULT_CUTOFFS)
    cut["pair_cs"] = 1e-11
    return diamond_cell(6, omega=0.4, cutoffs=cut, n_occ=3456, large=True, config_index=5)


def small_random_cell(seed: int, natom: int = 2, lmax: int = 2, skew: bool = True, omega: float = 0.6,
                      edge_bohr: float = 6.0, cut: float = 1e-11) -> Cell:
    """A small, possibly non-orthogonal cell with 1-4 atoms and s/p/d shells,
    for parity tests across every angular-momentum class."""
    st = Stream((MASTER_SEED_SMALL << 16) ^ seed)
    lat = np.eye(3) * edge_bohr
    if skew:
        lat = lat + st.uniform(9, -0.25, 0.25).reshape(3, 3) * edge_bohr
    pos = st.uniform(3 * natom).reshape(natom, 3) @ lat
    shells = []
    for r in pos:
        for l in range(lmax + 1):
            nprim = int(st.integers(1, 1, 3)[0])
            e, c = _draw_shell_params(st, l, nprim, 0.3, 12.0)
            shells.append(Shell(l, e, c, r.copy()))
    cuts = dict(pair_R=cut, pair_cs=cut, ewald_R=cut, ewald_K=cut)
    nbf = sum(ncart(s.l) for s in shells)
    return Cell("small%d" % seed, lat, shells, omega, cuts, max(1, min(nbf // 3, 4)), ["X"] * natom, pos,
                orbital_key=(MASTER_SEED_SMALL << 20) ^ (seed * 7919 + 1))


MASTER_SEED_SMALL = 2410022278 + 100


# nuclear charges of the cells' atoms (the synthetic "X" atoms of the tiny
# and small cells carry 2, so that the tiny cell with 2 occupied orbitals is
# neutral)
NUCLEAR_CHARGE = {"H": 1.0, "C": 6.0, "O": 8.0, "X": 2.0}


def nuclear_charges(cell: Cell) -> np.ndarray:
    return np.array([NUCLEAR_CHARGE[s] for s in cell.symbols], dtype=np.float64)


def config(index: int, **kw) -> Cell:
    """The synthetic stand-in for workload ``index`` (1 tiny, 2 water,
    3 diamond 3x3x3, 5 diamond 6x6x6)."""
    if index == 1:
        return tiny_cell()
    if index == 2:
        return water_cell(**kw)
    if index == 3:
        return diamond_cell(3, **kw)
    if index == 5:
        return large_cell()
    raise ValueError(index)


@dataclass
class Request:
    rid: int
    arrival_s: float
    kind: str
    natom_target: int
    n_iter: int
    cell: Cell


def serving_requests(n_requests: int = 256, rate_per_s: float = 50.0, lo_atoms: int = 8, hi_atoms: int = 512):
    """Poisson arrivals (seeded exponential gaps), log-uniform size in
    [8, 512] atoms, diamond-like or water-like 50/50, 3-20 SCF iterations."""
    st = stream(4, 1)
    t = 0.0
    reqs = []
    for rid in range(n_requests):
        t += -np.log(max(st.uniform(1)[0], 1e-300)) / rate_per_s
        natom = float(st.loguniform(1, lo_atoms, hi_atoms)[0])
        kind = "diamond" if st.uniform(1)[0] < 0.5 else "water"
        n_iter = int(st.integers(1, 3, 20)[0])
        if kind == "diamond":
            k = max(1, int(round((natom / 8.0) ** (1.0 / 3.0))))
            cell = diamond_cell(k, omega=0.5, n_occ=None, config_index=4, geo_purpose=16 + rid)
        else:
            nmol = max(1, int(round(natom / 3.0)))
            edge = (29.94 * nmol) ** (1.0 / 3.0)
            cell = water_cell(nmol, edge, omega=0.4, n_occ=max(1, 4 * nmol), config_index=4, geo_purpose=16 + rid)
        reqs.append(Request(rid, t, kind, int(round(natom)), n_iter, cell))
    return reqs


def density_perturbation(key: int, nbf: int, frob: float = 1e-3) -> np.ndarray:
    """A symmetric Gaussian matrix with Frobenius norm ``frob``."""
    st = Stream(key)
    E = st.normal(nbf * nbf).reshape(nbf, nbf)
    E = 0.5 * (E + E.T)
    return E * (frob / np.linalg.norm(E))
