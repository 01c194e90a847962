"""One-electron operators through the C ABI (jk_one_electron) against the
FP64 oracle, element by element (tolerance 1e-10, the FP64 parity bound):
kinetic energy and nuclear attraction on the tiny cell and on small s/p/d
cells, including skewed ones; at full size (the 64-water box) the
attraction's omega invariance and symmetry, and the total energy per cell
being omega-invariant."""
import numpy as np
import pytest

import synthcells as sc
from oracle import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def jk():
    from paper_2410_22278_gb300 import build, jk

    build.build()
    assert torch.cuda.is_available()
    return jk


def gpu_onee(jk, cell, omega=None):
    plan = jk.plan_from_cell(cell, omega=omega)
    n = cell.nbf
    dev = torch.device("cuda:0")
    T = torch.full((n, n), float("nan"), dtype=torch.float64, device=dev)
    V = torch.full_like(T, float("nan"))
    plan.one_electron(sc.nuclear_charges(cell), cell.positions, T.data_ptr(), V.data_ptr(), 0)
    out = (T.cpu().numpy(), V.cpu().numpy())
    plan.close()
    return out


CELLS = [("tiny", lambda: sc.config(1))] + [
    ("small%d" % s, (lambda s=s, na=na, lm=lm, sk=sk: sc.small_random_cell(s, na, lm, sk)))
    for s, na, lm, sk in [(1, 2, 1, False), (2, 2, 2, True), (3, 3, 2, True), (4, 1, 2, False)]]


@pytest.mark.parametrize("name,make", CELLS)
def test_kinetic_and_attraction_match_oracle(jk, name, make):
    cell = make()
    T, V = gpu_onee(jk, cell)
    To, Vo = O.kinetic(cell), O.nuclear(cell)
    assert np.abs(T - To).max() < TOL, (name, np.abs(T - To).max())
    assert np.abs(V - Vo).max() < TOL, (name, np.abs(V - Vo).max())


def test_attraction_omega_invariance_on_gpu(jk):
    cell = sc.small_random_cell(2, 2, 2, True)
    _, V1 = gpu_onee(jk, cell, omega=0.45)
    _, V2 = gpu_onee(jk, cell, omega=0.9)
    assert np.abs(V1 - V2).max() < TOL, np.abs(V1 - V2).max()


def test_full_size_water_one_electron(jk):
    """64-water box: the attraction at omega 0.4 and 0.6 agrees, both
    operators are symmetric, and E_kin + E_ne + E_J + E_K + E_nn per cell is
    the same at both omega to 1e-10 of the size of its terms (traces over
    n^2 = 692,224 elements, each within 1e-10, and mixed-precision J/K)."""
    cell = sc.config(2)
    dev = torch.device("cuda:0")
    Z, X = sc.nuclear_charges(cell), cell.positions
    E, Vs = {}, {}
    D = None
    for om in (0.4, 0.6):
        plan = jk.plan_from_cell(cell, precision=jk.JK_MIXED, omega=om)
        n = cell.nbf
        if D is None:
            S = torch.empty((n, n), dtype=torch.float64, device=dev)
            plan.overlap(S.data_ptr(), 0)
            torch.cuda.synchronize()
            D = torch.from_numpy(sc.density_from_overlap(cell.orbital_guess(), S.cpu().numpy())).to(dev)
        T = torch.empty_like(D)
        V = torch.empty_like(D)
        J = torch.empty_like(D)
        K = torch.empty_like(D)
        plan.one_electron(Z, X, T.data_ptr(), V.data_ptr(), 0)
        plan.build(D.data_ptr(), J.data_ptr(), K.data_ptr(), 0)
        torch.cuda.synchronize()
        ej, ek = plan.energy(D.data_ptr(), J.data_ptr(), K.data_ptr(), 0)
        enn = jk.ewald_point_charges(cell.lattice, Z, X, om)
        Tn, Vn = T.cpu().numpy(), V.cpu().numpy()
        assert np.abs(Tn - Tn.T).max() < 1e-12 * np.abs(Tn).max()
        assert np.abs(Vn - Vn.T).max() < 1e-12 * np.abs(Vn).max()
        Dn = D.cpu().numpy()
        terms = [float(np.sum(Dn * Tn)), float(np.sum(Dn * Vn)), ej, ek, enn]
        E[om] = sum(terms)
        E["scale"] = max(E.get("scale", 0.0), sum(abs(t) for t in terms))
        Vs[om] = Vn
        plan.close()
    assert np.abs(Vs[0.4] - Vs[0.6]).max() < TOL, np.abs(Vs[0.4] - Vs[0.6]).max()
    assert abs(E[0.4] - E[0.6]) < 1e-10 * E["scale"], E
