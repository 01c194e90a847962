"""GPU path (through the C ABI) against the FP64 oracle, element by element.

FP64 path: max |dJ|, |dK| <= 1e-10 (the parity bound for the FP64 path);
mixed path: <= 1e-7 and |dE| <= 1e-6 Ha per cell.  The oracle sums the
Ewald series to 1e-18 with a margin, so the tolerance covers the GPU's
truncation at the cell's thresholds plus rounding.
"""
import math

import numpy as np
import pytest

import synthcells as sc
from oracle import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOLMIX = 1e-7


@pytest.fixture(scope="module")
def jk():
    from paper_2410_22278_gb300 import build, jk

    build.build()
    assert torch.cuda.is_available()
    return jk


_cache = {}


def oracle_jk(cell, omega=None):
    key = (cell.name, omega)
    if key not in _cache:
        D = O.density(cell)
        e = O.eri_tensor(cell, omega=omega)
        J, K = O.jk_from_eri(e, D)
        _cache[key] = (D, J, K)
    return _cache[key]


def gpu_jk(jk, cell, D, precision=0, omega=None, mixed_switch=0.0, want_J=True, want_K=True):
    plan = jk.plan_from_cell(cell, precision=precision, omega=omega, mixed_switch=mixed_switch)
    dev = torch.device("cuda:0")
    Dt = torch.from_numpy(np.ascontiguousarray(D)).to(dev)
    Jt = torch.full_like(Dt, float("nan"))
    Kt = torch.full_like(Dt, float("nan"))
    st = torch.cuda.current_stream().cuda_stream
    plan.build(Dt.data_ptr(), Jt.data_ptr() if want_J else 0, Kt.data_ptr() if want_K else 0, st)
    torch.cuda.synchronize()
    E = plan.energy(Dt.data_ptr(), Jt.data_ptr() if want_J else 0, Kt.data_ptr() if want_K else 0, st)
    out = (Jt.cpu().numpy(), Kt.cpu().numpy(), E, plan.info())
    plan.close()
    return out


def test_tiny_fp64(jk):
    cell = sc.config(1)
    D, Jo, Ko = oracle_jk(cell)
    J, K, (ej, ek), info = gpu_jk(jk, cell, D)
    assert np.abs(J - Jo).max() < TOL64, np.abs(J - Jo).max()
    assert np.abs(K - Ko).max() < TOL64, np.abs(K - Ko).max()
    eoj, oek = O.energies(D, Jo, Ko)
    assert abs(ej - eoj) < TOL64 and abs(ek - oek) < TOL64
    assert np.abs(J - J.T).max() < 1e-13 and np.abs(K - K.T).max() < 1e-13


SMALL = [(1, 1, 2, True), (2, 2, 1, False), (3, 2, 2, True), (4, 3, 1, True), (5, 2, 2, False), (6, 1, 1, True)]


@pytest.mark.parametrize("seed,natom,lmax,skew", SMALL)
def test_small_cells_fp64(jk, seed, natom, lmax, skew):
    cell = sc.small_random_cell(seed, natom=natom, lmax=lmax, skew=skew)
    D, Jo, Ko = oracle_jk(cell)
    J, K, _, info = gpu_jk(jk, cell, D)
    scale = max(1.0, np.abs(Jo).max())
    assert np.abs(J - Jo).max() < TOL64 * scale, np.abs(J - Jo).max()
    assert np.abs(K - Ko).max() < TOL64 * scale, np.abs(K - Ko).max()


def test_overlap_matches_oracle(jk):
    for cell in [sc.config(1), sc.small_random_cell(3, natom=2, lmax=2)]:
        plan = jk.plan_from_cell(cell)
        S = torch.empty((cell.nbf, cell.nbf), dtype=torch.float64, device="cuda:0")
        plan.overlap(S.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert np.abs(S.cpu().numpy() - O.overlap(cell)).max() < 1e-14
        plan.close()


def test_only_J_or_only_K(jk):
    cell = sc.small_random_cell(3, natom=2, lmax=2)
    D, Jo, Ko = oracle_jk(cell)
    J, _, _, _ = gpu_jk(jk, cell, D, want_K=False)
    assert np.abs(J - Jo).max() < TOL64 * 10
    _, K, _, _ = gpu_jk(jk, cell, D, want_J=False)
    assert np.abs(K - Ko).max() < TOL64 * 10


def test_host_buffers_match_device(jk):
    cell = sc.config(1)
    D, Jo, Ko = oracle_jk(cell)
    plan = jk.plan_from_cell(cell)
    J, K = plan.build_host(D)
    assert np.abs(J - Jo).max() < TOL64 and np.abs(K - Ko).max() < TOL64
    plan.close()


@pytest.mark.parametrize("which", ["tiny", "small3"])
def test_mixed_precision_tolerance(jk, which):
    cell = sc.config(1) if which == "tiny" else sc.small_random_cell(3, natom=2, lmax=2)
    D, Jo, Ko = oracle_jk(cell)
    J, K, (ej, ek), info = gpu_jk(jk, cell, D, precision=1)
    assert np.abs(J - Jo).max() < TOLMIX, np.abs(J - Jo).max()
    assert np.abs(K - Ko).max() < TOLMIX, np.abs(K - Ko).max()
    eoj, oek = O.energies(D, Jo, Ko)
    assert abs(ej + ek - eoj - oek) < 1e-6


def test_omega_invariance_on_gpu(jk):
    """Results do not depend on the Ewald split (Section 3.4)."""
    cell = sc.config(1)
    D, Jo, Ko = oracle_jk(cell)
    for w in [0.3, 0.8, 1.2]:
        J, K, _, _ = gpu_jk(jk, cell, D, omega=w)
        assert np.abs(J - Jo).max() < 1e-9 and np.abs(K - Ko).max() < 1e-9, w
