"""Coordinate-selection strategies of Section 3 / Section 5.1 on one worker.

* RCD (csc_rcd_solve) consumes the same random order as the oracle's
  coordinate descent: objective within 1e-5 relative, Z close.
* Cyclic order repeated until the KKT test holds reaches the oracle's LGCD
  objective.
* Greedy CD (one sub-domain covering the domain) and cyclic CD (sub-domains
  of one position) through csc_lgcd_solve with one worker match the oracle
  run with the same sub-domains.
* An index outside K x Omega is reported, not read."""
import numpy as np
import pytest

from synthetic import Workload, make_problem
from tests._gpu import dev, host

pytestmark = pytest.mark.gpu

W1D = Workload("sel1d", P=2, K=3, T=(400,), L=(8,), density=0.02, sigma=0.1)
W2D = Workload("sel2d", P=1, K=4, T=(40, 40), L=(6, 6), density=0.01, sigma=0.1)
TOL = 1e-4


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1901_09235_gb300 as p
    from paper_1901_09235_gb300 import build
    build.build()
    p.load()
    return p


def _setup(pkg, w, seed):
    import torch
    X, D, _ = make_problem(w, seed)
    Xd, Dd = dev(X), dev(D)
    beta, dtd, lm = pkg.csc_init_beta(Xd, Dd)
    lam = float(np.float32(0.1 * lm))
    Z = torch.zeros_like(beta)
    return X, D, Xd, Dd, beta, dtd, Z, lam


@pytest.mark.parametrize("w", [W1D, W2D], ids=["1d", "2d"])
def test_rcd_matches_oracle_on_the_same_order(pkg, orc, w):
    import torch
    X, D, Xd, Dd, beta, dtd, Z, lam = _setup(pkg, w, 31)
    n_coord = int(np.prod(beta.shape))
    coords = np.random.default_rng(8).integers(0, n_coord, 6000).astype(np.int32)
    changed = pkg.csc_rcd_solve(X.shape, Dd, dtd, beta, Z, lam, torch.from_numpy(coords).cuda())
    Zr, _, changed_ref = orc.rcd(X, D, lam, coords.astype(np.uint32))
    Zg = host(Z).astype(np.float64)
    f_g, f_r = orc.objective(X, D, Zg, lam), orc.objective(X, D, Zr, lam)
    assert abs(f_g - f_r) <= 1e-5 * abs(f_r), (f_g, f_r)
    assert abs(changed - changed_ref) <= max(3, changed_ref // 100)
    assert np.abs(Zg - Zr).max() <= 1e-3 * max(1.0, np.abs(Zr).max())


def test_rcd_cyclic_order_reaches_the_lgcd_solution(pkg, orc):
    import torch
    X, D, Xd, Dd, beta, dtd, Z, lam = _setup(pkg, W1D, 32)
    order = torch.arange(int(np.prod(beta.shape)), dtype=torch.int32, device="cuda")
    ws = pkg.workspace(pkg.make_shape(X.shape, D.shape))
    for _ in range(200):
        pkg.csc_rcd_solve(X.shape, Dd, dtd, beta, Z, lam, order, ws=ws)
        _, mdz, obj = pkg.csc_refresh_beta(Xd, Dd, Z, lam, beta=beta, ws=ws)
        if mdz < TOL:
            break
    assert mdz < TOL
    ref = orc.lgcd(X, D, lam, TOL)
    f_ref = orc.objective(X, D, ref["Z"], lam)
    assert abs(obj - f_ref) <= 1e-5 * abs(f_ref)


@pytest.mark.parametrize("rule", ["greedy", "cyclic"])
@pytest.mark.parametrize("w", [W1D, W2D], ids=["1d", "2d"])
def test_greedy_and_cyclic_cd_match_the_oracle(pkg, orc, w, rule):
    X, D, Xd, Dd, beta, dtd, Z, lam = _setup(pkg, w, 33)
    zs = beta.shape[1:]
    if len(w.T) == 1:
        sub = [zs[-1]] if rule == "greedy" else [1]
    else:
        sub = list(zs) if rule == "greedy" else [1, 1]
    o = pkg.default_opts(max_workers=1, sub=sub)
    Zg, st = pkg.csc_lgcd_solve(Xd, Dd, dtd, beta, lam, TOL, opts=o)
    assert st["status"] == 0 and st["workers"] == 1
    ref = orc.lgcd(X, D, lam, TOL, sub=tuple(sub))
    f_g = orc.objective(X, D, host(Zg), lam)
    f_r = orc.objective(X, D, ref["Z"], lam)
    assert abs(f_g - f_r) <= 1e-5 * abs(f_r)
    assert orc.kkt(X, D, host(Zg), lam) < TOL


def test_rcd_reports_an_index_outside_the_domain(pkg):
    import torch
    X, D, Xd, Dd, beta, dtd, Z, lam = _setup(pkg, W1D, 34)
    bad = torch.tensor([0, 5, int(np.prod(beta.shape))], dtype=torch.int32, device="cuda")
    with pytest.raises(pkg.CscError) as e:
        pkg.csc_rcd_solve(X.shape, Dd, dtd, beta, Z, lam, bad)
    assert e.value.status == pkg.CSC_ERR_INVALID
