"""Request server (continuous batching) through the C ABI: every result is
the same alone and in the mix, admission respects the HBM budget, unknown
tickets are reported."""
import numpy as np
import pytest

import synthcells as sc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def jk():
    from paper_2410_22278_gb300 import build, jk

    build.build()
    return jk


def _cells():
    return [sc.config(1), sc.small_random_cell(3, natom=2, lmax=2), sc.small_random_cell(4, natom=3, lmax=1)]


def _density(cell, k):
    rng = np.random.default_rng(100 + k)
    X = rng.standard_normal((cell.nbf, cell.nbf))
    return 0.05 * (X + X.T) + np.eye(cell.nbf)


def test_results_alone_equal_results_in_the_mix(jk):
    dev = torch.device("cuda:0")
    cells = _cells()
    plans = [jk.plan_from_cell(c) for c in cells]
    alone = []
    Ds = []
    for k, (c, p) in enumerate(zip(cells, plans)):
        D = torch.from_numpy(_density(c, k)).to(dev)
        J = torch.empty_like(D)
        K = torch.empty_like(D)
        p.build(D.data_ptr(), J.data_ptr(), K.data_ptr(), 0)
        torch.cuda.synchronize()
        alone.append((J.cpu().numpy(), K.cpu().numpy()))
        Ds.append(D)
    srv = jk.Server(device=0, hbm_budget_bytes=8 << 30, max_slots=2)
    outs, tickets = [], []
    for rep in range(3):
        for k, p in enumerate(plans):
            J = torch.empty_like(Ds[k])
            K = torch.empty_like(Ds[k])
            outs.append((k, J, K))
            tickets.append(srv.submit(p, Ds[k].data_ptr(), J.data_ptr(), K.data_ptr()))
    lat = []
    for t in tickets:
        st, l = srv.wait(t, timeout_ms=60000)
        assert st == 0
        lat.append(l)
    for k, J, K in outs:
        assert np.abs(J.cpu().numpy() - alone[k][0]).max() < 1e-12
        assert np.abs(K.cpu().numpy() - alone[k][1]).max() < 1e-12
    assert all(l > 0 for l in lat)
    with pytest.raises(jk.JkError) as e:
        srv.wait(tickets[0], timeout_ms=10)
    assert e.value.status == jk.JK_ERR_NOT_FOUND
    srv.close()
    for p in plans:
        p.close()


def test_budget_refusal(jk):
    cell = sc.config(1)
    p = jk.plan_from_cell(cell)
    srv = jk.Server(device=0, hbm_budget_bytes=1024, max_slots=1)
    D = torch.eye(cell.nbf, dtype=torch.float64, device="cuda:0")
    J = torch.empty_like(D)
    with pytest.raises(jk.JkError) as e:
        srv.submit(p, D.data_ptr(), J.data_ptr(), 0)
    assert e.value.status == jk.JK_ERR_OOM
    srv.close()
    p.close()


def test_mixed_plans_alone_equal_in_the_mix_and_match_oracle(jk):
    """Mixed-precision plans served with the serving stream's iteration
    densities D_k = D_0 + E_k (E_k symmetric, Frobenius norm 1e-3: full rank,
    so the exchange contraction takes its dense split-precision form).  Each
    result is the same alone and in the mix, and one cell's result matches
    the FP64 oracle within the mixed tolerance."""
    from oracle import oracle as O

    dev = torch.device("cuda:0")
    cells = _cells()
    plans = [jk.plan_from_cell(c, precision=jk.JK_MIXED) for c in cells]
    Ds, alone = [], []
    for k, (c, p) in enumerate(zip(cells, plans)):
        D = O.density(c) + sc.density_perturbation(7000 + k, c.nbf)
        Dt = torch.from_numpy(D).to(dev)
        J = torch.empty_like(Dt)
        K = torch.empty_like(Dt)
        p.build(Dt.data_ptr(), J.data_ptr(), K.data_ptr(), 0)
        torch.cuda.synchronize()
        alone.append((J.cpu().numpy(), K.cpu().numpy()))
        Ds.append((D, Dt))
    srv = jk.Server(device=0, hbm_budget_bytes=16 << 30, max_slots=3)
    outs, tickets = [], []
    for rep in range(3):
        for k, p in enumerate(plans):
            J = torch.empty_like(Ds[k][1])
            K = torch.empty_like(Ds[k][1])
            outs.append((k, J, K))
            tickets.append(srv.submit(p, Ds[k][1].data_ptr(), J.data_ptr(), K.data_ptr()))
    for t in tickets:
        st, lat = srv.wait(t, timeout_ms=120000)
        assert st == 0 and lat > 0
    for k, J, K in outs:
        assert np.abs(J.cpu().numpy() - alone[k][0]).max() < 1e-12
        assert np.abs(K.cpu().numpy() - alone[k][1]).max() < 1e-12
    srv.close()
    # the first cell against the oracle with its perturbed density
    D0 = Ds[0][0]
    Jo, Ko = O.jk_from_eri(O.eri_tensor(cells[0]), D0)
    assert np.abs(alone[0][0] - Jo).max() < 1e-7
    assert np.abs(alone[0][1] - Ko).max() < 1e-7
    for p in plans:
        p.close()
