"""jk_energy_noalloc (fixed device scratch, no allocation) against jk_energy.

Two calls in a row on the same plan, each with its own inputs, must give
what jk_energy gives on those inputs; the second call also shows that
nothing left in the fixed scratch by the first reaches its result.  This
file is collected last so that it runs after every other GPU test, and it
also passes alone in a fresh process.
"""
import numpy as np
import pytest

import synthcells as sc

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def jk():
    from paper_2410_22278_gb300 import build, jk

    build.build()
    assert torch.cuda.is_available()
    return jk


def _close(a, b, scale):
    # both are FP64 sums of the same n^2 products in different orders
    assert abs(a - b) <= 1e-13 * scale + 1e-300, (a, b, scale)


def test_noalloc_rejects_null_plan():
    """Argument check on the host (no device needed)."""
    import ctypes

    from paper_2410_22278_gb300 import jk

    ej, ek = ctypes.c_double(), ctypes.c_double()
    rc = jk.lib().jk_energy_noalloc(None, None, None, None, ctypes.byref(ej), ctypes.byref(ek), None)
    assert rc == -1  # JK_ERR_INVALID


@pytest.mark.gpu
def test_noalloc_after_build(jk):
    """Energies of a real J/K build (tiny cell), two calls in a row."""
    cell = sc.config(1)
    plan = jk.plan_from_cell(cell)
    dev = torch.device("cuda:0")
    st = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(7)
    for call in range(2):
        X = rng.standard_normal((cell.nbf, cell.nbf))
        D = torch.from_numpy(X + X.T).to(dev)
        J = torch.empty_like(D)
        K = torch.empty_like(D)
        plan.build(D.data_ptr(), J.data_ptr(), K.data_ptr(), st)
        ej, ek = plan.energy(D.data_ptr(), J.data_ptr(), K.data_ptr(), st)
        nj, nk = plan.energy_noalloc(D.data_ptr(), J.data_ptr(), K.data_ptr(), st)
        sj = float((D * J).abs().sum()) * 0.5
        sk = float((D * K).abs().sum()) * 0.25
        _close(nj, ej, sj)
        _close(nk, ek, sk)
    plan.close()


@pytest.mark.gpu
def test_noalloc_many_blocks(jk):
    """A 208-function plan (several first-pass blocks), two calls in a row
    with different matrices, and a call with K omitted."""
    cell = sc.water_cell(16, 12.42 / 4 ** (1.0 / 3.0), omega=0.4, n_occ=64, geo_purpose=3)
    plan = jk.plan_from_cell(cell, precision=jk.JK_MIXED)
    n = cell.nbf
    dev = torch.device("cuda:0")
    st = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(11)
    for call in range(2):
        D, J, K = (torch.from_numpy(rng.standard_normal((n, n)) * (call + 1)).to(dev) for _ in range(3))
        ej, ek = plan.energy(D.data_ptr(), J.data_ptr(), K.data_ptr(), st)
        nj, nk = plan.energy_noalloc(D.data_ptr(), J.data_ptr(), K.data_ptr(), st)
        _close(nj, ej, 0.5 * float((D * J).abs().sum()))
        _close(nk, ek, 0.25 * float((D * K).abs().sum()))
    nj, nk = plan.energy_noalloc(D.data_ptr(), J.data_ptr(), 0, st)
    ej, _ = plan.energy(D.data_ptr(), J.data_ptr(), 0, st)
    _close(nj, ej, 0.5 * float((D * J).abs().sum()))
    assert nk == 0.0
    plan.close()
