"""ctypes binding of the C ABI in include/jk.h (argument marshalling only).

Every step of the J/K build runs in libjk.so's CUDA kernels; this module
only converts Python objects to the ABI's plain pointers and sizes.  It
fails loudly when the library is missing: there is no CPU fallback.
Device buffers are passed as integer device addresses (e.g. the
``data_ptr()`` of a CUDA torch tensor); streams as raw ``cudaStream_t``
handles (``torch.cuda.Stream.cuda_stream``) or 0.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libjk.so")

JK_OK = 0
JK_ERR_INVALID = -1
JK_ERR_UNSUPPORTED = -2
JK_ERR_OOM = -3
JK_ERR_CUDA = -4
JK_ERR_TIMEOUT = -5
JK_ERR_DEVICE_CHECK = -6
JK_ERR_BUSY = -7
JK_ERR_NOT_FOUND = -8
JK_FP64 = 0
JK_MIXED = 1

# every symbol declared in include/jk.h
EXPORTS = [
    "jk_plan_create", "jk_plan_info", "jk_pair_counts", "jk_plan_nbf", "jk_plan_destroy", "jk_build", "jk_build_host", "jk_build_times", "jk_build_counts", "jk_autotune", "jk_energy",
    "jk_energy_noalloc", "jk_one_electron",
    "jk_overlap", "jk_ewald_point_charges", "jk_server_create", "jk_submit", "jk_wait", "jk_server_destroy",
    "jk_status_string", "jk_last_error", "jk_microbench_fma", "jk_plan_cache", "jk_plan_set_schedule",
]


class JkError(RuntimeError):
    def __init__(self, status, where):
        msg = "%s failed: %s (%d): %s" % (where, status_string(status), status, last_error())
        super().__init__(msg)
        self.status = status


class jk_cell(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_double * 9)]


class jk_shell(ctypes.Structure):
    _fields_ = [("l", ctypes.c_int), ("nprim", ctypes.c_int), ("exps", ctypes.POINTER(ctypes.c_double)),
                ("coefs", ctypes.POINTER(ctypes.c_double)), ("center", ctypes.c_double * 3)]


class jk_cutoffs(ctypes.Structure):
    _fields_ = [("pair_R", ctypes.c_double), ("pair_cs", ctypes.c_double), ("ewald_R", ctypes.c_double),
                ("ewald_K", ctypes.c_double), ("mixed_switch", ctypes.c_double)]


class jk_plan_stats(ctypes.Structure):
    _fields_ = [("nbf", ctypes.c_int), ("nshell", ctypes.c_int), ("n_classes", ctypes.c_int), ("n_g", ctypes.c_int),
                ("n_shell_pairs", ctypes.c_longlong), ("n_pair_images", ctypes.c_longlong),
                ("n_prim_pair_images", ctypes.c_longlong), ("n_quartets", ctypes.c_longlong),
                ("n_quartets_schwarz", ctypes.c_longlong), ("n_quartets_fp64", ctypes.c_longlong),
                ("n_r1_candidates", ctypes.c_longlong), ("omega", ctypes.c_double), ("g_max", ctypes.c_double),
                ("r1_max", ctypes.c_double), ("volume", ctypes.c_double), ("device_bytes", ctypes.c_size_t),
                ("workspace_bytes", ctypes.c_size_t)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    """Load libjk.so (built by paper_2410_22278_gb300.build); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libjk.so is not built (%s); run paper_2410_22278_gb300.build.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        vp, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
        L.jk_plan_create.argtypes = [ctypes.POINTER(jk_cell), ctypes.POINTER(jk_shell), ctypes.c_int, ctypes.c_double,
                                     ctypes.POINTER(jk_cutoffs), ctypes.c_int, ctypes.c_int, ctypes.POINTER(vp)]
        L.jk_plan_info.argtypes = [vp, ctypes.POINTER(jk_plan_stats)]
        L.jk_plan_nbf.argtypes = [vp]
        L.jk_pair_counts.argtypes = [ctypes.POINTER(jk_cell), ctypes.POINTER(jk_shell), ctypes.c_int, ctypes.c_double,
                                     ctypes.POINTER(jk_cutoffs), ctypes.POINTER(ctypes.c_longlong)]
        L.jk_plan_destroy.argtypes = [vp]
        L.jk_plan_destroy.restype = None
        L.jk_build.argtypes = [vp, vp, vp, vp, vp]
        L.jk_plan_cache.argtypes = [vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
        L.jk_build_host.argtypes = [vp, dp, dp, dp, vp]
        L.jk_build_times.argtypes = [vp, dp, ctypes.POINTER(ctypes.c_int), ctypes.c_int]
        L.jk_build_counts.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.c_int]
        L.jk_plan_set_schedule.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.c_int]
        L.jk_autotune.argtypes = [vp, vp, vp, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int)]
        L.jk_energy.argtypes = [vp, vp, vp, vp, dp, dp, vp]
        L.jk_energy_noalloc.argtypes = [vp, vp, vp, vp, dp, dp, vp]
        L.jk_one_electron.argtypes = [vp, ctypes.c_int, dp, dp, vp, vp, vp]
        L.jk_overlap.argtypes = [vp, vp, vp]
        L.jk_ewald_point_charges.argtypes = [ctypes.POINTER(jk_cell), ctypes.c_int, dp, dp, ctypes.c_double,
                                             ctypes.c_double, dp]
        L.jk_server_create.argtypes = [ctypes.c_int, ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(vp)]
        L.jk_submit.argtypes = [vp, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_longlong)]
        L.jk_wait.argtypes = [vp, ctypes.c_longlong, ctypes.c_int, ctypes.POINTER(ctypes.c_int), dp]
        L.jk_server_destroy.argtypes = [vp]
        L.jk_server_destroy.restype = None
        L.jk_status_string.argtypes = [ctypes.c_int]
        L.jk_status_string.restype = ctypes.c_char_p
        L.jk_last_error.argtypes = []
        L.jk_last_error.restype = ctypes.c_char_p
        L.jk_microbench_fma.argtypes = [ctypes.c_int, dp]
        _lib = L
    return _lib


def status_string(s: int) -> str:
    return lib().jk_status_string(int(s)).decode()


def last_error() -> str:
    return lib().jk_last_error().decode()


def _check(rc, where):
    if rc != JK_OK:
        raise JkError(rc, where)


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class _Keep:
    arrays: list


def make_cell(lattice) -> jk_cell:
    c = jk_cell()
    for k, v in enumerate(np.asarray(lattice, dtype=np.float64).reshape(-1)):
        c.lattice[k] = float(v)
    return c


def make_shells(shells):
    """shells: objects with l, exps, coefs, center (synthcells.Shell)."""
    arr = (jk_shell * len(shells))()
    keep = []
    for i, s in enumerate(shells):
        e = np.ascontiguousarray(s.exps, dtype=np.float64)
        c = np.ascontiguousarray(s.coefs, dtype=np.float64)
        keep += [e, c]
        arr[i].l = int(s.l)
        arr[i].nprim = len(e)
        arr[i].exps = _dp(e)
        arr[i].coefs = _dp(c)
        for k in range(3):
            arr[i].center[k] = float(s.center[k])
    return arr, _Keep(keep)


def make_cutoffs(pair_R=0.0, pair_cs=0.0, ewald_R=0.0, ewald_K=0.0, mixed_switch=0.0) -> jk_cutoffs:
    return jk_cutoffs(float(pair_R), float(pair_cs), float(ewald_R), float(ewald_K), float(mixed_switch))


class Plan:
    """Owns one jk_plan (jk_plan_create / jk_plan_destroy)."""

    def __init__(self, lattice, shells, omega=0.0, cutoffs=None, precision=JK_FP64, device=0):
        self._h = None
        cell = make_cell(lattice)
        arr, keep = make_shells(shells)
        cut = cutoffs if isinstance(cutoffs, jk_cutoffs) else make_cutoffs(**(cutoffs or {}))
        h = ctypes.c_void_p()
        _check(lib().jk_plan_create(ctypes.byref(cell), arr, len(shells), float(omega), ctypes.byref(cut),
                                    int(precision), int(device), ctypes.byref(h)), "jk_plan_create")
        del keep
        self._h = h

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        s = jk_plan_stats()
        _check(lib().jk_plan_info(self._h, ctypes.byref(s)), "jk_plan_info")
        return s.as_dict()

    @property
    def nbf(self) -> int:
        return int(lib().jk_plan_nbf(self._h))

    def cache(self, max_bytes: int) -> int:
        """Keep the D-independent reciprocal data resident (jk_plan_cache);
        returns its size in bytes (0 releases it)."""
        b = ctypes.c_size_t()
        _check(lib().jk_plan_cache(self._h, ctypes.c_size_t(int(max_bytes)), ctypes.byref(b)), "jk_plan_cache")
        return int(b.value)

    def build(self, D_ptr: int, J_ptr: int, K_ptr: int, stream: int = 0):
        _check(lib().jk_build(self._h, D_ptr or None, J_ptr or None, K_ptr or None, stream or None), "jk_build")

    def build_host(self, D: np.ndarray, want_J=True, want_K=True, stream: int = 0):
        n = self.nbf
        D = np.ascontiguousarray(D, dtype=np.float64)
        assert D.shape == (n, n)
        J = np.zeros((n, n)) if want_J else None
        K = np.zeros((n, n)) if want_K else None
        _check(lib().jk_build_host(self._h, _dp(D), _dp(J) if J is not None else None, _dp(K) if K is not None else None,
                                   stream or None), "jk_build_host")
        return J, K

    def build_host_into(self, D: np.ndarray, J: np.ndarray, K: np.ndarray, stream: int = 0):
        """Host buffers owned by the caller (pinned or pageable)."""
        _check(lib().jk_build_host(self._h, _dp(D), _dp(J) if J is not None else None, _dp(K) if K is not None else None,
                                   stream or None), "jk_build_host")

    PHASES = ["prologue", "real_space", "recip_sfac", "recip_j", "recip_k", "epilogue", "total", "tensor_gemm", "tensor_slice",
              "real_fp64_list", "real_tiles"]

    def build_times(self):
        """{phase: (ms, launches)} of the most recent build (device events),
        plus "mma_flops": BF16 MMA flops issued by the tensor-core GEMMs."""
        ms = (ctypes.c_double * 12)()
        nl = (ctypes.c_int * 12)()
        _check(lib().jk_build_times(self._h, ms, nl, 12), "jk_build_times")
        out = {p: (ms[i], nl[i]) for i, p in enumerate(self.PHASES)}
        out["mma_flops"] = (ms[11], 0)
        return out

    def autotune(self, D_ptr: int, stream: int = 0, cache_path: str = None):
        """Real-space schedule chosen by timing (jk_autotune): a list of 21
        (family, kets) pairs, family 0 lane-per-bra, 1 warp."""
        chosen = (ctypes.c_int * 42)()
        _check(lib().jk_autotune(self._h, D_ptr, stream or None, cache_path.encode() if cache_path else None, chosen),
               "jk_autotune")
        return [(chosen[2 * k], chosen[2 * k + 1]) for k in range(21)]

    def set_schedule(self, sched):
        """Set (family, kets) per class pair (jk_plan_set_schedule)."""
        flat = (ctypes.c_int * (2 * len(sched)))(*[int(v) for pair in sched for v in pair])
        _check(lib().jk_plan_set_schedule(self._h, flat, len(sched)), "jk_plan_set_schedule")

    COUNTS = ["quartets_fp64", "quartets_fp32", "list_overflow", "density_rank", "flops_fp64", "flops_fp32", "lowrank",
              "screen_fp64", "screen_fp32", "lane_terms_fp64", "lane_slots_fp64", "lane_terms_fp32", "lane_slots_fp32"]

    def build_counts(self):
        """(FP64 image quartets, FP32 image quartets) of the most recent build."""
        c = self.counters()
        return c["quartets_fp64"], c["quartets_fp32"]

    def counters(self) -> dict:
        """Every work counter of the most recent build (jk_build_counts)."""
        c = (ctypes.c_longlong * 13)()
        _check(lib().jk_build_counts(self._h, c, 13), "jk_build_counts")
        return {k: int(c[i]) for i, k in enumerate(self.COUNTS)}

    def real_space_flops(self):
        """(FP64, FP32) algorithmic flops of the real-space evaluation in the most recent build."""
        c = self.counters()
        return c["flops_fp64"], c["flops_fp32"]

    def energy(self, D_ptr: int, J_ptr: int, K_ptr: int, stream: int = 0):
        ej, ek = ctypes.c_double(), ctypes.c_double()
        _check(lib().jk_energy(self._h, D_ptr, J_ptr or None, K_ptr or None, ctypes.byref(ej), ctypes.byref(ek),
                               stream or None), "jk_energy")
        return ej.value, ek.value

    def energy_noalloc(self, D_ptr: int, J_ptr: int, K_ptr: int, stream: int = 0):
        """jk_energy with the library's fixed device scratch: allocates nothing."""
        ej, ek = ctypes.c_double(), ctypes.c_double()
        _check(lib().jk_energy_noalloc(self._h, D_ptr, J_ptr or None, K_ptr or None, ctypes.byref(ej), ctypes.byref(ek),
                                       stream or None), "jk_energy_noalloc")
        return ej.value, ek.value

    def one_electron(self, Z, xyz, T_ptr: int, V_ptr: int, stream: int = 0):
        """Kinetic-energy and nuclear-attraction matrices (jk_one_electron)
        into device buffers; Z (natom) and xyz (natom x 3, bohr) on the host."""
        Z = np.ascontiguousarray(Z, dtype=np.float64)
        xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1)
        _check(lib().jk_one_electron(self._h, len(Z), _dp(Z), _dp(xyz), T_ptr or None, V_ptr or None, stream or None),
               "jk_one_electron")

    def overlap(self, S_ptr: int, stream: int = 0):
        _check(lib().jk_overlap(self._h, S_ptr, stream or None), "jk_overlap")

    def close(self):
        if self._h is not None and self._h.value:
            lib().jk_plan_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plan_from_cell(cell, precision=JK_FP64, device=0, omega=None, mixed_switch=0.0):
    """A Plan for a synthcells.Cell with its omega and thresholds."""
    cut = dict(cell.cutoffs)
    cut["mixed_switch"] = mixed_switch
    return Plan(cell.lattice, cell.shells, cell.omega if omega is None else omega, cut, precision, device)


def pair_counts(lattice, shells, omega=0.0, cutoffs=None):
    """Host-only pair-list counts: (ordered shell pairs, ordered primitive
    pairs, ordered local pairs, unique shell-pair images, half-space G)."""
    cell = make_cell(lattice)
    arr, keep = make_shells(shells)
    cut = cutoffs if isinstance(cutoffs, jk_cutoffs) else make_cutoffs(**(cutoffs or {}))
    out = (ctypes.c_longlong * 5)()
    _check(lib().jk_pair_counts(ctypes.byref(cell), arr, len(shells), float(omega), ctypes.byref(cut), out), "jk_pair_counts")
    del keep
    return tuple(int(x) for x in out)


def ewald_point_charges(lattice, q, xyz, omega, delta=0.0) -> float:
    cell = make_cell(lattice)
    q = np.ascontiguousarray(q, dtype=np.float64)
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1)
    e = ctypes.c_double()
    _check(lib().jk_ewald_point_charges(ctypes.byref(cell), len(q), _dp(q), _dp(xyz), float(omega), float(delta),
                                        ctypes.byref(e)), "jk_ewald_point_charges")
    return e.value


def microbench_fma(fp64: bool) -> float:
    """FMA throughput of the current device in TFLOP/s (measurement utility)."""
    t = ctypes.c_double()
    _check(lib().jk_microbench_fma(1 if fp64 else 0, ctypes.byref(t)), "jk_microbench_fma")
    return t.value


class Server:
    """Owns one jk_server (continuous batching of builds)."""

    def __init__(self, device=0, hbm_budget_bytes=64 << 30, max_slots=4):
        h = ctypes.c_void_p()
        _check(lib().jk_server_create(int(device), int(hbm_budget_bytes), int(max_slots), ctypes.byref(h)),
               "jk_server_create")
        self._h = h

    def submit(self, plan: Plan, D_ptr: int, J_ptr: int, K_ptr: int) -> int:
        t = ctypes.c_longlong()
        _check(lib().jk_submit(self._h, plan.handle, D_ptr, J_ptr or None, K_ptr or None, ctypes.byref(t)), "jk_submit")
        return t.value

    def wait(self, ticket: int, timeout_ms: int = -1):
        st, lat = ctypes.c_int(), ctypes.c_double()
        rc = lib().jk_wait(self._h, int(ticket), int(timeout_ms), ctypes.byref(st), ctypes.byref(lat))
        if rc != JK_OK:
            raise JkError(rc, "jk_wait")
        return st.value, lat.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().jk_server_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
