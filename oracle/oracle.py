"""Python face of the FP64 CPU oracle (``jk_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product package
never imports this module, and this module never imports the product.

Each function names the passage of arXiv:2410.22278 it follows; the C file
holds the arithmetic.  Inputs come from ``synthcells`` (seeded geometry and
basis draws) and, for the density, from ``density_from_overlap`` applied to
this oracle's own overlap matrix.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liboracle.so")
SRC = os.path.join(HERE, "jk_oracle.c")

ORACLE_DELTA = 1e-18  # Ewald truncation used by the oracle (far past the GPU's)
ORACLE_MARGIN = 4.0  # bohr added to every real-space sphere radius

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, OpenMP)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < os.path.getmtime(SRC):
        tmp = LIB_PATH + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


class _Basis(ctypes.Structure):
    _fields_ = [
        ("nshell", ctypes.c_int),
        ("l", ctypes.POINTER(ctypes.c_int)),
        ("nprim", ctypes.POINTER(ctypes.c_int)),
        ("poff", ctypes.POINTER(ctypes.c_int)),
        ("exps", ctypes.POINTER(ctypes.c_double)),
        ("coefs", ctypes.POINTER(ctypes.c_double)),
        ("centers", ctypes.POINTER(ctypes.c_double)),
        ("lat", ctypes.c_double * 9),
        ("omega", ctypes.c_double),
        ("pair_R", ctypes.c_double),
        ("pair_cs", ctypes.c_double),
        ("delta", ctypes.c_double),
        ("margin", ctypes.c_double),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            B = ctypes.POINTER(_Basis)
            _lib.orc_boys.argtypes = [ctypes.c_int, ctypes.c_double, dp]
            _lib.orc_norm_coefs.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp]
            _lib.orc_pair_counts.argtypes = [B, ctypes.POINTER(ctypes.c_long)]
            _lib.orc_local_pairs.argtypes = [B, dp, ctypes.c_long]
            _lib.orc_local_pairs.restype = ctypes.c_long
            _lib.orc_overlap.argtypes = [B, dp]
            _lib.orc_pair_ft.argtypes = [B, dp, dp]
            _lib.orc_eri_tensor.argtypes = [B, ctypes.c_int, dp]
            _lib.orc_eri_tensor.restype = ctypes.c_int
            _lib.orc_jk_rows.argtypes = [B, dp, ip, ctypes.c_int, ctypes.c_int, dp, dp]
            _lib.orc_jk_rows.restype = ctypes.c_int
            _lib.orc_molecular_prim_eri.argtypes = [ip, dp, dp, ctypes.c_double, dp]
            _lib.orc_ewald_point_charges.argtypes = [dp, ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_double]
            _lib.orc_ewald_point_charges.restype = ctypes.c_double
            _lib.orc_num_threads.restype = ctypes.c_int
            _lib.orc_jk_sample.argtypes = [B, dp, ctypes.c_int, ctypes.c_int, dp]
            _lib.orc_kinetic.argtypes = [B, dp]
            _lib.orc_nuclear.argtypes = [B, ctypes.c_int, dp, dp, ctypes.c_int, dp]
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


class Basis:
    """Flat arrays of a synthcells.Cell, kept alive for the C side."""

    def __init__(self, cell, omega=None, delta=ORACLE_DELTA, margin=ORACLE_MARGIN):
        sh = cell.shells
        self.l = np.array([s.l for s in sh], dtype=np.int32)
        self.nprim = np.array([s.nprim for s in sh], dtype=np.int32)
        self.poff = np.concatenate([[0], np.cumsum(self.nprim)[:-1]]).astype(np.int32)
        self.exps = np.ascontiguousarray(np.concatenate([s.exps for s in sh]), dtype=np.float64)
        self.coefs = np.ascontiguousarray(np.concatenate([s.coefs for s in sh]), dtype=np.float64)
        self.centers = np.ascontiguousarray(np.array([s.center for s in sh]).reshape(-1), dtype=np.float64)
        self.nbf = int(sum((l + 1) * (l + 2) // 2 for l in self.l))
        b = _Basis()
        b.nshell = len(sh)
        b.l, b.nprim, b.poff = _ip(self.l), _ip(self.nprim), _ip(self.poff)
        b.exps, b.coefs, b.centers = _dp(self.exps), _dp(self.coefs), _dp(self.centers)
        for k, v in enumerate(np.asarray(cell.lattice, dtype=np.float64).reshape(-1)):
            b.lat[k] = v
        b.omega = float(cell.omega if omega is None else omega)
        b.pair_R = float(cell.cutoffs["pair_R"])
        b.pair_cs = float(cell.cutoffs["pair_cs"])
        b.delta = float(delta)
        b.margin = float(margin)
        self.c = b

    def ref(self):
        return ctypes.byref(self.c)


# --------------------------------------------------------------------------
def boys(mmax: int, T: float) -> np.ndarray:
    """F_0..F_mmax at T (Eqs. boys_function_erf_form and R_recursion seeds)."""
    out = np.zeros(mmax + 1)
    lib().orc_boys(mmax, float(T), _dp(out))
    return out


def norm_coefs(l, exps, coefs) -> np.ndarray:
    """Contraction x radial normalisation (Eq. local_normalization), unit
    self-overlap of the contracted local function."""
    exps = np.ascontiguousarray(exps, dtype=np.float64)
    coefs = np.ascontiguousarray(coefs, dtype=np.float64)
    out = np.zeros_like(exps)
    lib().orc_norm_coefs(int(l), len(exps), _dp(exps), _dp(coefs), _dp(out))
    return out


def pair_counts(cell):
    """(ordered shell pairs, ordered primitive pairs, ordered local pairs)
    after the pair cut-offs of Eqs. pbc_eri_pair_cutoff_implementation and pbc_eri_cauchy_schwarz_cutoff_implementation (Section 3.1)."""
    b = Basis(cell)
    c = (ctypes.c_long * 3)()
    lib().orc_pair_counts(b.ref(), c)
    return tuple(int(x) for x in c)


def local_pairs(cell) -> np.ndarray:
    """Ordered local primitive pairs: columns I J ia ib n0 n1 n2 a b K P0 P1 P2."""
    b = Basis(cell)
    n = lib().orc_local_pairs(b.ref(), None, 0)
    out = np.zeros((n, 13))
    lib().orc_local_pairs(b.ref(), _dp(out), n)
    return out


def overlap(cell) -> np.ndarray:
    """Gamma overlap over the pair list (Eq. pbc_overlap_formula)."""
    b = Basis(cell)
    S = np.zeros((b.nbf, b.nbf))
    lib().orc_overlap(b.ref(), _dp(S))
    return S


def pair_ft(cell, G) -> np.ndarray:
    """Bloch-summed AO pair density Fourier transforms at one G (complex nbf x nbf)."""
    b = Basis(cell)
    G = np.ascontiguousarray(G, dtype=np.float64)
    out = np.zeros((b.nbf, b.nbf, 2))
    lib().orc_pair_ft(b.ref(), _dp(G), _dp(out))
    return out[..., 0] + 1j * out[..., 1]


PART_REAL, PART_RECIP, PART_BG = 1, 2, 4


def eri_tensor(cell, omega=None, parts=7, delta=ORACLE_DELTA, margin=ORACLE_MARGIN) -> np.ndarray:
    """The periodic ERI tensor (mu nu|lambda sigma) of Eq. pbc_eri_general_final
    at the Gamma point, all nbf^4 elements, every ordered pair (tiny cells).
    omega = inf gives the reciprocal-only evaluation (no real-space or
    background term)."""
    b = Basis(cell, omega=omega, delta=delta, margin=margin)
    if math.isinf(b.c.omega):
        parts &= PART_RECIP
    n = b.nbf
    eri = np.zeros((n, n, n, n))
    lib().orc_eri_tensor(b.ref(), int(parts), _dp(eri))
    return eri


def kinetic(cell) -> np.ndarray:
    """Gamma kinetic-energy matrix over the pair list (local integrals of
    -1/2 nabla^2 from 1-D overlaps; Section 2.1 and its Supporting
    Information)."""
    b = Basis(cell)
    T = np.zeros((b.nbf, b.nbf))
    lib().orc_kinetic(b.ref(), _dp(T))
    return T


PART_MOLECULAR = 8


def nuclear(cell, Z=None, xyz=None, omega=None, parts=7, delta=ORACLE_DELTA, margin=ORACLE_MARGIN) -> np.ndarray:
    """Nuclear attraction of point charges Z at xyz (default: the cell's
    atoms) with their images, Ewald-split at omega (Section 2.2, Eq.
    pbc_v1e_base_case_final): parts bit0 real, bit1 reciprocal, bit2 self
    term; PART_MOLECULAR alone gives the bare molecular attraction."""
    import synthcells as sc

    Z = np.ascontiguousarray(sc.nuclear_charges(cell) if Z is None else Z, dtype=np.float64)
    xyz = np.ascontiguousarray(cell.positions if xyz is None else xyz, dtype=np.float64).reshape(-1)
    b = Basis(cell, omega=omega, delta=delta, margin=margin)
    V = np.zeros((b.nbf, b.nbf))
    lib().orc_nuclear(b.ref(), len(Z), _dp(Z), _dp(xyz), int(parts), _dp(V))
    return V


def jk_from_eri(eri, D):
    """J_mn = sum (mn|ls) D_ls, K_mn = sum (ml|sn) D_ls (Eqs.
    pbc_j_definition_k_sample and pbc_k_definition, Gamma point, w = 1)."""
    J = np.einsum("mnls,ls->mn", eri, D)
    K = np.einsum("mlsn,ls->mn", eri, D)
    return J, K


def jk_rows(cell, D, shells, omega=None, parts=7, delta=ORACLE_DELTA, margin=ORACLE_MARGIN):
    """Rows of J and K for the AOs of the listed shells (in listed order)."""
    b = Basis(cell, omega=omega, delta=delta, margin=margin)
    rows = np.ascontiguousarray(shells, dtype=np.int32)
    nra = int(sum((cell.shells[i].l + 1) * (cell.shells[i].l + 2) // 2 for i in rows))
    D = np.ascontiguousarray(D, dtype=np.float64)
    J = np.zeros((nra, b.nbf))
    K = np.zeros((nra, b.nbf))
    lib().orc_jk_rows(b.ref(), _dp(D), _ip(rows), len(rows), int(parts), _dp(J), _dp(K))
    return J, K


def ao_offsets(cell):
    off, n = [], 0
    for s in cell.shells:
        off.append(n)
        n += (s.l + 1) * (s.l + 2) // 2
    return np.array(off), n


def row_indices(cell, shells):
    off, _ = ao_offsets(cell)
    return np.concatenate([off[i] + np.arange((cell.shells[i].l + 1) * (cell.shells[i].l + 2) // 2) for i in shells])


def energies(D, J, K):
    """E_J = 1/2 sum D.J, E_K = -1/4 sum D.K (closed-shell reading, D = 2CC^T)."""
    return 0.5 * float(np.sum(D * J)), -0.25 * float(np.sum(D * K))


def molecular_prim_eri(l, exps, centers, omega=0.0) -> np.ndarray:
    """One primitive Cartesian quartet without a lattice: bare Coulomb
    (omega = 0, Eq. pbc_eri_base_case's molecular limit) or erfc-attenuated."""
    l = np.ascontiguousarray(l, dtype=np.int32)
    exps = np.ascontiguousarray(exps, dtype=np.float64)
    centers = np.ascontiguousarray(np.asarray(centers).reshape(-1), dtype=np.float64)
    shape = tuple((x + 1) * (x + 2) // 2 for x in l)
    out = np.zeros(int(np.prod(shape)))
    lib().orc_molecular_prim_eri(_ip(l), _dp(exps), _dp(centers), float(omega), _dp(out))
    return out.reshape(shape)


def ewald_point_charges(lattice, q, xyz, omega, delta=1e-17) -> float:
    """Ewald energy of point charges in a periodic cell (Eq.
    nuclear_repulsion_energy), with the removed K = 0 term."""
    lat = np.ascontiguousarray(lattice, dtype=np.float64).reshape(-1)
    q = np.ascontiguousarray(q, dtype=np.float64)
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1)
    return float(lib().orc_ewald_point_charges(_dp(lat), len(q), _dp(q), _dp(xyz), float(omega), float(delta)))


def density(cell) -> np.ndarray:
    """D = 2 C C^T from the cell's seeded orbital guess, orthonormalised in
    this oracle's overlap metric."""
    from synthcells import density_from_overlap

    return density_from_overlap(cell.orbital_guess(), overlap(cell))


def jk_sample_seconds(cell, D, bra_stride, ng_sample=1, delta=ORACLE_DELTA, margin=ORACLE_MARGIN):
    """Time a bounded sample of a full J+K build with the oracle's own code
    paths and extrapolate: (estimated seconds of a full build, detail dict).
    Real space: every bra_stride-th ordered local pair against all; reciprocal:
    ng_sample G vectors (pair transforms, Coulomb and one exchange row)."""
    b = Basis(cell, delta=delta, margin=margin)
    D = np.ascontiguousarray(D, dtype=np.float64)
    out = np.zeros(7)
    lib().orc_jk_sample(b.ref(), _dp(D), int(bra_stride), int(ng_sample), _dp(out))
    t_real, nb, nlp, t_ft, t_row, ng, nbf = out
    full = t_real * nlp / max(nb, 1) + ng * (t_ft + t_row * nbf)
    detail = dict(real_s=t_real, bra_sampled=int(nb), local_pairs=int(nlp), ft_s_per_G=t_ft, row_s_per_G=t_row,
                  n_g=int(ng), nbf=int(nbf), sample_s=t_real + ng_sample * (t_ft + t_row))
    return full, detail


def num_threads() -> int:
    return int(lib().orc_num_threads())
