"""Mixed-precision path against the FP64 oracle, with the share of the work
that the FP32 real-space kernels did stated and checked.

* Forced FP32: mixed_switch is raised so far that no quartet's size estimate
  reaches it, so every image quartet outside the short-interval rule goes to
  the FP32 tile kernels; the counters of jk_build_counts show that they did
  (more than 90% of the image quartets), and the result is compared with the
  oracle element by element.  With every quartet in FP32 -- the largest
  ones included, which the mixed policy keeps in FP64 -- the bound is FP32
  rounding: 16 u (u = 2^-24, so about 1e-6) relative to the largest element,
  for every class pair of s, p and d shells.
* Default switch: the same cells within the mixed tolerance 1e-7, with the
  FP32 share of the image quartets stated.
* Default switch on the diamond-basis cell (config-3 basis: s(6) s(3) p(1)
  d(1), exponents up to 3000, one conventional 8-atom cell, 88 basis
  functions): the whole J and K against the oracle's (tests/golden, written
  by make_rows.py), FP64 within 1e-10 and mixed within 1e-7.
* Concurrency: two host threads build one plan on two streams; each result
  equals the lone build.
"""
import os
import threading

import numpy as np
import pytest

import synthcells as sc
from oracle import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOLMIX = 1e-7
GOLD_D1 = os.path.join(os.path.dirname(__file__), "golden", "diamond1_rows_all.npz")


@pytest.fixture(scope="module")
def jk():
    from paper_2410_22278_gb300 import build, jk

    build.build()
    assert torch.cuda.is_available()
    return jk


_cache = {}


def oracle_jk(cell):
    if cell.name not in _cache:
        D = O.density(cell)
        e = O.eri_tensor(cell)
        J, K = O.jk_from_eri(e, D)
        _cache[cell.name] = (D, J, K, e)
    return _cache[cell.name]


def run(jk, cell, D, precision, mixed_switch=0.0):
    plan = jk.plan_from_cell(cell, precision=precision, mixed_switch=mixed_switch)
    dev = torch.device("cuda:0")
    Dt = torch.from_numpy(np.ascontiguousarray(D)).to(dev)
    Jt = torch.full_like(Dt, float("nan"))
    Kt = torch.full_like(Dt, float("nan"))
    plan.build(Dt.data_ptr(), Jt.data_ptr(), Kt.data_ptr(), 0)
    torch.cuda.synchronize()
    counts = plan.build_counts()
    E = plan.energy(Dt.data_ptr(), Jt.data_ptr(), Kt.data_ptr(), 0)
    out = (Jt.cpu().numpy(), Kt.cpu().numpy(), E, counts)
    plan.close()
    return out


FORCED = [("tiny", None), ("small1", (1, 1, 2, True)), ("small3", (3, 2, 2, True)), ("small5", (5, 2, 2, False))]


def _cell(which, spec):
    if which == "tiny":
        return sc.config(1)
    seed, natom, lmax, skew = spec
    return sc.small_random_cell(seed, natom=natom, lmax=lmax, skew=skew)


TOL_FP32_REL = 16 * 2.0 ** -24


@pytest.mark.parametrize("which,spec", FORCED)
def test_forced_fp32_against_oracle(jk, which, spec):
    cell = _cell(which, spec)
    D, Jo, Ko, _ = oracle_jk(cell)
    J, K, (ej, ek), (n64, n32) = run(jk, cell, D, jk.JK_MIXED, mixed_switch=1e30)
    share = n32 / max(1, n32 + n64)
    dJ, dK = np.abs(J - Jo).max(), np.abs(K - Ko).max()
    eoj, oek = O.energies(D, Jo, Ko)
    print("%s forced FP32: share %.4f (%d of %d image quartets), max|dJ| %.2e max|dK| %.2e dE %.2e"
          % (which, share, n32, n32 + n64, dJ, dK, ej + ek - eoj - oek))
    assert share > 0.9, share
    assert dJ < TOL_FP32_REL * max(1.0, np.abs(Jo).max()), dJ
    assert dK < TOL_FP32_REL * max(1.0, np.abs(Ko).max()), dK


@pytest.mark.parametrize("which,spec", FORCED)
def test_default_switch_against_oracle(jk, which, spec):
    cell = _cell(which, spec)
    D, Jo, Ko, _ = oracle_jk(cell)
    J, K, (ej, ek), (n64, n32) = run(jk, cell, D, jk.JK_MIXED)
    share = n32 / max(1, n32 + n64)
    dJ, dK = np.abs(J - Jo).max(), np.abs(K - Ko).max()
    eoj, oek = O.energies(D, Jo, Ko)
    print("%s default switch: FP32 share %.4f (%d of %d image quartets), max|dJ| %.2e max|dK| %.2e dE %.2e"
          % (which, share, n32, n32 + n64, dJ, dK, ej + ek - eoj - oek))
    assert dJ < TOLMIX and dK < TOLMIX, (dJ, dK)
    assert abs(ej + ek - eoj - oek) < 1e-6


@pytest.mark.skipif(not os.path.exists(GOLD_D1), reason="no diamond-basis oracle matrices")
@pytest.mark.parametrize("precision", [0, 1])
def test_diamond_basis_cell_against_oracle(jk, precision):
    cell = sc.diamond_cell(1)
    g = np.load(GOLD_D1)
    assert list(g["rows"]) == list(range(cell.nbf))
    D = O.density(cell)
    J, K, _, (n64, n32) = run(jk, cell, D, precision)
    dJ, dK = np.abs(J - g["J"]).max(), np.abs(K - g["K"]).max()
    print("diamond1 precision %d: max|dJ| %.2e max|dK| %.2e (FP64 %d, FP32 %d image quartets)" % (precision, dJ, dK, n64, n32))
    tol = TOL64 if precision == 0 else TOLMIX
    assert dJ < tol and dK < tol, (dJ, dK)
    if precision == 1:
        assert n32 > 0.9 * (n32 + n64)  # the FP32 kernels did most of the quartets


@pytest.mark.skipif(not os.path.exists(GOLD_D1), reason="no diamond-basis oracle matrices")
def test_diamond_basis_cell_forced_fp32(jk):
    cell = sc.diamond_cell(1)
    g = np.load(GOLD_D1)
    D = O.density(cell)
    J, K, _, (n64, n32) = run(jk, cell, D, 1, mixed_switch=1e30)
    dJ, dK = np.abs(J - g["J"]).max(), np.abs(K - g["K"]).max()
    share = n32 / max(1, n32 + n64)
    print("diamond1 forced FP32: share %.4f max|dJ| %.2e max|dK| %.2e" % (share, dJ, dK))
    assert share > 0.9
    # every d-shell class pair ran in FP32 here; the bound is the FP32
    # rounding of the largest quartets, not the mixed policy's 1e-7
    assert dJ < TOL_FP32_REL * max(1.0, np.abs(g["J"]).max()), dJ
    assert dK < TOL_FP32_REL * max(1.0, np.abs(g["K"]).max()), dK


def test_two_threads_one_plan(jk):
    """jk_build on one plan from two host threads and two streams: the
    builds are ordered one after the other on the plan's workspace and each
    result equals the lone build."""
    cell = sc.small_random_cell(3, natom=2, lmax=2)
    D, Jo, Ko, _ = oracle_jk(cell)
    for prec in (jk.JK_FP64, jk.JK_MIXED):
        plan = jk.plan_from_cell(cell, precision=prec)
        dev = torch.device("cuda:0")
        Dt = torch.from_numpy(D).to(dev)
        J0 = torch.empty_like(Dt)
        K0 = torch.empty_like(Dt)
        plan.build(Dt.data_ptr(), J0.data_ptr(), K0.data_ptr(), 0)
        torch.cuda.synchronize()
        streams = [torch.cuda.Stream(), torch.cuda.Stream()]
        outs = [[(torch.empty_like(Dt), torch.empty_like(Dt)) for _ in range(4)] for _ in streams]
        errs = []

        def worker(i):
            try:
                for J, K in outs[i]:
                    plan.build(Dt.data_ptr(), J.data_ptr(), K.data_ptr(), streams[i].cuda_stream)
            except Exception as e:  # pragma: no cover - reported below
                errs.append(e)

        th = [threading.Thread(target=worker, args=(i,)) for i in range(2)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        torch.cuda.synchronize()
        assert not errs, errs
        for o in outs:
            for J, K in o:
                assert (J - J0).abs().max().item() < 1e-12
                assert (K - K0).abs().max().item() < 1e-12
        # the FP64 parity bound scaled by the largest element, as for the other small cells
        tol = (TOL64 if prec == jk.JK_FP64 else TOLMIX) * max(1.0, np.abs(Jo).max())
        assert np.abs(J0.cpu().numpy() - Jo).max() < tol and np.abs(K0.cpu().numpy() - Ko).max() < tol
        plan.close()


@pytest.mark.parametrize("family", [0, 1, 2])
@pytest.mark.parametrize("precision", [0, 1, "fp32"])
def test_every_kernel_family_matches_oracle(jk, family, precision):
    """The s and p class pairs have three real-space kernel families (lane
    per bra, warp per bra, pair queue); each, forced through
    jk_plan_set_schedule for every such class pair, matches the oracle on a
    skewed s/p/d cell, in FP64, in the mixed form and with every quartet
    forced to FP32 (the FP32 rounding bound)."""
    cell = sc.small_random_cell(3, natom=2, lmax=2)
    D, Jo, Ko, _ = oracle_jk(cell)
    forced = precision == "fp32"
    plan = jk.plan_from_cell(cell, precision=jk.JK_MIXED if forced else precision, mixed_switch=1e30 if forced else 0.0)
    classes = [(a, b) for a in range(6) for b in range(a, 6)]
    plan.set_schedule([(family if (a <= 2 and b <= 2) else 0, 512 if (family == 1 and a <= 2 and b <= 2) else 16)
                       for a, b in classes])
    dev = torch.device("cuda:0")
    Dt = torch.from_numpy(D).to(dev)
    J = torch.empty_like(Dt)
    K = torch.empty_like(Dt)
    plan.build(Dt.data_ptr(), J.data_ptr(), K.data_ptr(), 0)
    torch.cuda.synchronize()
    n64, n32 = plan.build_counts()[:2]
    plan.close()
    if forced:
        assert n32 > 0.9 * (n32 + n64), (n32, n64)
        assert np.abs(J.cpu().numpy() - Jo).max() < TOL_FP32_REL * max(1.0, np.abs(Jo).max())
        assert np.abs(K.cpu().numpy() - Ko).max() < TOL_FP32_REL * max(1.0, np.abs(Ko).max())
        return
    tol = (TOL64 * max(1.0, np.abs(Jo).max())) if precision == 0 else TOLMIX
    assert np.abs(J.cpu().numpy() - Jo).max() < tol
    assert np.abs(K.cpu().numpy() - Ko).max() < tol
    with pytest.raises(jk.JkError):
        jk.plan_from_cell(cell).set_schedule([(1, 16)] * 21)  # no warp kernels for d classes


@pytest.mark.parametrize("precision", [0, 1])
def test_reciprocal_cache(jk, precision):
    """jk_plan_cache: the build that fills the cache and the builds that read
    it give the uncached result (the cached data are D-independent), also
    for a different density and after Coulomb-only builds; 0 releases the
    cache."""
    cell = sc.small_random_cell(4, natom=3, lmax=1)
    dev = torch.device("cuda:0")
    D1 = torch.from_numpy(O.density(cell)).to(dev)
    D2 = torch.from_numpy(O.density(cell) + sc.density_perturbation(99, cell.nbf)).to(dev)

    def build(plan, D):
        J = torch.empty_like(D)
        K = torch.empty_like(D)
        plan.build(D.data_ptr(), J.data_ptr(), K.data_ptr(), 0)
        torch.cuda.synchronize()
        return J.cpu().numpy(), K.cpu().numpy()

    plain = jk.plan_from_cell(cell, precision=precision)
    ref1, ref2 = build(plain, D1), build(plain, D2)
    plain.close()
    plan = jk.plan_from_cell(cell, precision=precision)
    nbytes = plan.cache(1 << 30)
    assert nbytes > 0 and plan.info()["device_bytes"] >= nbytes
    for D, ref in [(D1, ref1), (D1, ref1), (D2, ref2)]:
        J, K = build(plan, D)
        assert np.abs(J - ref[0]).max() < 1e-12 and np.abs(K - ref[1]).max() < 1e-12
    assert plan.cache(0) == 0
    with pytest.raises(jk.JkError) as e:
        plan.cache(16)  # far too small: refused, the plan works as before
    assert e.value.status == jk.JK_ERR_OOM
    J, K = build(plan, D2)
    assert np.abs(J - ref2[0]).max() < 1e-12
    # a Coulomb-only build fills the structure factors alone; the next J+K
    # build forms the exchange slices from them, and later ones reuse both
    assert plan.cache(1 << 30) > 0
    for D, ref, with_k in [(D1, ref1, False), (D2, ref2, False), (D2, ref2, True), (D1, ref1, True)]:
        J = torch.empty_like(D)
        K = torch.empty_like(D) if with_k else None
        plan.build(D.data_ptr(), J.data_ptr(), K.data_ptr() if with_k else 0, 0)
        torch.cuda.synchronize()
        assert np.abs(J.cpu().numpy() - ref[0]).max() < 1e-12
        if with_k:
            assert np.abs(K.cpu().numpy() - ref[1]).max() < 1e-12
    plan.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_coulomb_only_builds_match_oracle(jk, precision):
    """A build that asks for J alone (K = NULL) skips the exchange and runs
    the Hermite J-engine (Hermite ket densities, J in the Hermite basis, back
    to Cartesian) for the class pairs with a d shell on both sides.  Its J
    matches the oracle on s/p/d cells (the diamond-basis cell covers every
    class pair up to (dd|dd)) and the J of a J+K build."""
    cells = [sc.config(1), sc.small_random_cell(3, natom=2, lmax=2)]
    refs = [oracle_jk(c)[:2] for c in cells]
    if os.path.exists(GOLD_D1):
        c1 = sc.diamond_cell(1)
        cells.append(c1)
        refs.append((O.density(c1), np.load(GOLD_D1)["J"]))
    dev = torch.device("cuda:0")
    for cell, (D, Jo) in zip(cells, refs):
        plan = jk.plan_from_cell(cell, precision=precision)
        Dt = torch.from_numpy(np.ascontiguousarray(D)).to(dev)
        J1 = torch.full_like(Dt, float("nan"))
        plan.build(Dt.data_ptr(), J1.data_ptr(), 0, 0)
        J2 = torch.full_like(Dt, float("nan"))
        K2 = torch.full_like(Dt, float("nan"))
        plan.build(Dt.data_ptr(), J2.data_ptr(), K2.data_ptr(), 0)
        torch.cuda.synchronize()
        plan.close()
        J1, J2 = J1.cpu().numpy(), J2.cpu().numpy()
        tol = TOL64 * max(1.0, np.abs(Jo).max()) if precision == 0 else TOLMIX
        print("%s precision %d J-engine: max|dJ| %.2e vs oracle, %.2e vs the J+K build"
              % (cell.name, precision, np.abs(J1 - Jo).max(), np.abs(J1 - J2).max()))
        assert np.abs(J1 - Jo).max() < tol
        assert np.abs(J1 - J2).max() < tol
        assert np.abs(J1 - J1.T).max() < 1e-12
