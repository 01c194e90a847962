"""Full-size parity on the water box (the benchmark workload, 832 basis
functions), in the benchmark's launch configuration, on sampled outputs:
the J and K rows of a few shells, computed one by one by the oracle and
stored in tests/golden/water_rows_*.npz by tests/golden/make_rows.py.
Also checks properties that hold at any size: symmetry, Tr(DS) = 2 n_occ,
and that the mixed path stays within its tolerance of the FP64 path."""
import glob
import os

import numpy as np
import pytest

import synthcells as sc
from oracle import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLD = sorted(glob.glob(os.path.join(os.path.dirname(__file__), "golden", "water_rows_*.npz")))


@pytest.fixture(scope="module")
def water_results():
    from paper_2410_22278_gb300 import build, jk

    build.build()
    cell = sc.config(2)
    D = O.density(cell)
    dev = torch.device("cuda:0")
    Dt = torch.from_numpy(D).to(dev)
    out = {}
    for prec in (jk.JK_FP64, jk.JK_MIXED):
        plan = jk.plan_from_cell(cell, precision=prec)
        J = torch.empty_like(Dt)
        K = torch.empty_like(Dt)
        plan.build(Dt.data_ptr(), J.data_ptr(), K.data_ptr(), 0)
        torch.cuda.synchronize()
        E = plan.energy(Dt.data_ptr(), J.data_ptr(), K.data_ptr(), 0)
        S = torch.empty_like(Dt)
        plan.overlap(S.data_ptr(), 0)
        torch.cuda.synchronize()
        out[prec] = (J.cpu().numpy(), K.cpu().numpy(), E, S.cpu().numpy())
        plan.close()
    return cell, D, out


@pytest.mark.skipif(not GOLD, reason="no golden rows")
@pytest.mark.parametrize("path", GOLD)
def test_fp64_rows_match_oracle(water_results, path):
    cell, D, out = water_results
    g = np.load(path)
    J, K, _, _ = out[0]
    rows = g["rows"]
    assert np.abs(J[rows] - g["J"]).max() < 1e-10, np.abs(J[rows] - g["J"]).max()
    assert np.abs(K[rows] - g["K"]).max() < 1e-10, np.abs(K[rows] - g["K"]).max()


@pytest.mark.skipif(not GOLD, reason="no golden rows")
@pytest.mark.parametrize("path", GOLD)
def test_mixed_rows_match_oracle(water_results, path):
    cell, D, out = water_results
    g = np.load(path)
    J, K, _, _ = out[1]
    rows = g["rows"]
    assert np.abs(J[rows] - g["J"]).max() < 1e-7
    assert np.abs(K[rows] - g["K"]).max() < 1e-7


def test_properties_at_full_size(water_results):
    cell, D, out = water_results
    J64, K64, (ej64, ek64), S = out[0]
    Jm, Km, (ejm, ekm), _ = out[1]
    assert abs(np.sum(D * S) - 2 * cell.n_occ) < 1e-9
    assert np.abs(S - O.overlap(cell)).max() < 1e-13
    for A in (J64, K64, Jm, Km):
        assert np.abs(A - A.T).max() < 1e-12
    assert ej64 > 0 and np.sum(D * K64) > 0
    assert np.abs(Jm - J64).max() < 1e-7 and np.abs(Km - K64).max() < 1e-7
    assert abs((ejm + ekm) - (ej64 + ek64)) < 1e-6
