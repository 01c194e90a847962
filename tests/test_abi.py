"""The C ABI library without a GPU: it loads, exports every symbol that
include/jk.h declares, and its host-only entry points (pair-list counts,
point-charge Ewald sum, argument checks) behave as specified."""
import json
import math
import os
import re

import numpy as np
import pytest

import synthcells as sc
from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLD = json.load(open(os.path.join(ROOT, "tests", "golden", "constants.json")))


@pytest.fixture(scope="module")
def jk():
    from paper_2410_22278_gb300 import build, jk

    build.build()
    jk.lib()
    return jk


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "jk.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(jk_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(jk):
    decl = _declared_functions()
    assert len(decl) >= 15
    for name in decl:
        assert hasattr(jk.lib(), name), name
    assert sorted(jk.EXPORTS) == decl


def test_status_strings(jk):
    for code in range(0, -9, -1):
        assert jk.status_string(code)
    assert jk.status_string(-5) == "timed out"


@pytest.mark.parametrize("which", ["tiny", "small3", "small4", "small7"])
def test_pair_counts_match_oracle(jk, which):
    cell = {"tiny": lambda: sc.config(1), "small3": lambda: sc.small_random_cell(3, natom=2, lmax=2),
            "small4": lambda: sc.small_random_cell(4, natom=3, lmax=1),
            "small7": lambda: sc.small_random_cell(7, natom=4, lmax=2, cut=1e-13)}[which]()
    mine = jk.pair_counts(cell.lattice, cell.shells, cell.omega, cell.cutoffs)
    assert mine[:3] == O.pair_counts(cell)


@pytest.mark.slow
def test_pair_counts_match_oracle_water_box(jk):
    cell = sc.config(2)
    mine = jk.pair_counts(cell.lattice, cell.shells, cell.omega, cell.cutoffs)
    assert mine[:3] == O.pair_counts(cell)


def test_point_charge_ewald(jk):
    r0 = 2.7
    a = 2 * r0
    fcc = np.array([[0, 0, 0], [0, 0.5, 0.5], [0.5, 0, 0.5], [0.5, 0.5, 0]]) * a
    xyz = np.vstack([fcc, fcc + np.array([a / 2, 0, 0])])
    q = np.array([1.0] * 4 + [-1.0] * 4)
    for w in [0.3, 0.7]:
        E = jk.ewald_point_charges(np.eye(3) * a, q, xyz, w, 1e-16)
        assert abs(-E * r0 / 4 - GOLD["nacl_madelung"]["value"]) < GOLD["nacl_madelung"]["tolerance"]
    L = 5.0
    E1 = jk.ewald_point_charges(np.eye(3) * L, [1.0], [[0.1, 0.2, 0.3]], 0.9, 1e-16)
    assert abs(-2 * L * E1 - GOLD["sc_wigner_xi"]["value"]) < GOLD["sc_wigner_xi"]["tolerance"]


def test_argument_checks(jk):
    cell = sc.config(1)
    bad = [sc.Shell(3, np.array([1.0]), np.array([1.0]), np.zeros(3))]
    with pytest.raises(jk.JkError) as e:
        jk.pair_counts(cell.lattice, bad)
    assert e.value.status == jk.JK_ERR_UNSUPPORTED
    bad = [sc.Shell(0, np.array([-1.0]), np.array([1.0]), np.zeros(3))]
    with pytest.raises(jk.JkError) as e:
        jk.pair_counts(cell.lattice, bad)
    assert e.value.status == jk.JK_ERR_INVALID
    with pytest.raises(jk.JkError) as e:
        jk.pair_counts(np.zeros((3, 3)), cell.shells)
    assert e.value.status == jk.JK_ERR_INVALID
    with pytest.raises(jk.JkError) as e:
        jk.ewald_point_charges(np.eye(3), [1.0], [[0, 0, 0]], -1.0)
    assert e.value.status == jk.JK_ERR_INVALID


def test_plan_create_without_device_fails_cleanly(jk):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    cell = sc.config(1)
    with pytest.raises(jk.JkError) as e:
        jk.plan_from_cell(cell)
    assert e.value.status == jk.JK_ERR_CUDA


def test_null_plan_is_rejected_before_any_device_call(jk):
    """Every entry point that takes a plan answers a NULL plan (or NULL
    outputs) with JK_ERR_INVALID and touches no device."""
    import ctypes

    L = jk.lib()
    e1, e2 = ctypes.c_double(), ctypes.c_double()
    cnt = (ctypes.c_longlong * 6)()
    ms = (ctypes.c_double * 11)()
    nl = ctypes.c_int()
    tk = ctypes.c_longlong()
    calls = {
        "jk_build": lambda: L.jk_build(None, None, None, None, None),
        "jk_build_host": lambda: L.jk_build_host(None, None, None, None, None),
        "jk_build_times": lambda: L.jk_build_times(None, ms, ctypes.byref(nl), 11),
        "jk_build_counts": lambda: L.jk_build_counts(None, cnt, 6),
        "jk_autotune": lambda: L.jk_autotune(None, None, None, None, None),
        "jk_energy": lambda: L.jk_energy(None, None, None, None, ctypes.byref(e1), ctypes.byref(e2), None),
        "jk_energy_noalloc": lambda: L.jk_energy_noalloc(None, None, None, None, ctypes.byref(e1), ctypes.byref(e2), None),
        "jk_overlap": lambda: L.jk_overlap(None, None, None),
        "jk_one_electron": lambda: L.jk_one_electron(None, 0, None, None, None, None, None),
        "jk_plan_info": lambda: L.jk_plan_info(None, None),
        "jk_submit": lambda: L.jk_submit(None, None, None, None, None, ctypes.byref(tk)),
        "jk_wait": lambda: L.jk_wait(None, 0, 0, None, None),
    }
    for name, call in calls.items():
        assert call() == jk.JK_ERR_INVALID, name
    assert L.jk_plan_nbf(None) == -1
    srv = ctypes.c_void_p()
    assert L.jk_server_create(0, 1 << 30, 0, ctypes.byref(srv)) == jk.JK_ERR_INVALID
    assert L.jk_server_create(0, 0, 4, ctypes.byref(srv)) == jk.JK_ERR_INVALID
    L.jk_plan_destroy(None)
    L.jk_server_destroy(None)
