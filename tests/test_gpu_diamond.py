"""Full-size check of the diamond-like 3x3x3 supercell (216 atoms, s s p d
shells, 2376 basis functions) in the mixed path, through properties that
hold at any size: the Ewald split parameter omega only moves work between
the real-space and reciprocal sums, so J, K and the energies at omega =
0.3, 0.5 and 0.8 must agree (to the mixed tolerance 1e-7 in J and K, 1e-6
Ha in E); J and K are symmetric; Tr(D S) = 2 n_occ for the density the
oracle's construction gives in the library's overlap metric."""
import numpy as np
import pytest

import synthcells as sc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OMEGAS = (0.3, 0.5, 0.8)
TOL_JK = 1e-7
TOL_E = 1e-6


@pytest.fixture(scope="module")
def diamond():
    from paper_2410_22278_gb300 import build, jk

    build.build()
    dev = torch.device("cuda:0")
    out, D, S0 = {}, None, None
    for om in OMEGAS:
        cell = sc.config(3, omega=om)
        plan = jk.plan_from_cell(cell, precision=jk.JK_MIXED)
        n = cell.nbf
        if D is None:
            S = torch.empty((n, n), dtype=torch.float64, device=dev)
            plan.overlap(S.data_ptr(), 0)
            torch.cuda.synchronize()
            S0 = S.cpu().numpy()
            D = torch.from_numpy(sc.density_from_overlap(cell.orbital_guess(), S0)).to(dev)
        J = torch.empty_like(D)
        K = torch.empty_like(D)
        plan.build(D.data_ptr(), J.data_ptr(), K.data_ptr(), 0)
        torch.cuda.synchronize()
        E = plan.energy(D.data_ptr(), J.data_ptr(), K.data_ptr(), 0)
        out[om] = (J.cpu().numpy(), K.cpu().numpy(), E)
        plan.close()
    return cell, D.cpu().numpy(), S0, out


def test_diamond_size_and_trace(diamond):
    cell, D, S, _ = diamond
    assert cell.nbf == 2376
    assert abs(np.sum(D * S) - 2 * cell.n_occ) < 1e-8 * cell.n_occ


@pytest.mark.parametrize("om", OMEGAS)
def test_diamond_symmetric_finite(diamond, om):
    _, _, _, out = diamond
    J, K, E = out[om]
    assert np.isfinite(J).all() and np.isfinite(K).all()
    assert np.abs(J - J.T).max() < 1e-10 * max(1.0, np.abs(J).max())
    assert np.abs(K - K.T).max() < 1e-10 * max(1.0, np.abs(K).max())
    assert E[0] > 0 and E[1] < 0


@pytest.mark.parametrize("pair", [(0.3, 0.5), (0.5, 0.8), (0.3, 0.8)])
def test_diamond_omega_invariance(diamond, pair):
    _, _, _, out = diamond
    a, b = out[pair[0]], out[pair[1]]
    dJ = np.abs(a[0] - b[0]).max()
    dK = np.abs(a[1] - b[1]).max()
    dE = abs((a[2][0] + a[2][1]) - (b[2][0] + b[2][1]))
    assert dJ < TOL_JK, dJ
    assert dK < TOL_JK, dK
    assert dE < TOL_E, dE
