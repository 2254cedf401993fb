"""Parity at the full sizes of the benchmark workloads, in the launch
configuration bench.py times (default options).

* 1-D, P = 5, T = 200,000, K = 10, L = 64: the oracle finishes the whole
  problem in seconds, so everything is compared in full.
* 2-D 4096 x 4096, K = 25 atoms of 32 x 32: too large for the full oracle
  solve; outputs the oracle computes one by one (beta-init and beta recomputed
  from Z at sampled coordinates, every nonzero of Z included), properties that
  hold at any size (objective from the nonzeros, KKT at the samples) and the
  dictionary statistics phi / psi from the nonzeros of the GPU's Z are checked.
* 2-D 1024 x 1024 image of the same family (same generator, 25 atoms of
  32 x 32, density, noise): the full oracle solve, against the same
  global-tile path."""
import numpy as np
import pytest

from synthetic import IMAGE_4096, SIGNAL_200K, make_problem, scaled
from tests._gpu import dev, gamma, host, kkt_fp64_within_bound, support_mismatch

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
    assert st["max_dz_final"] < w.tol
    # FP64 KKT within the FP32 recomputation's rounding bound (tests/_gpu.py)
    assert kkt_fp64_within_bound(orc, X, D, Zh, lam, w.tol)[0]
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
    # KKT on beta recomputed from Z by the oracle, at nonzeros (up to 200) and
    # at random coordinates, within the FP32 recomputation's rounding bound
    nzk, nzs = np.nonzero(Zh.reshape(w.K, -1))
    pick = rng.permutation(len(nzk))[:200]
    ks2 = np.concatenate([nzk[pick], rng.integers(0, w.K, 200)])
    ss2 = np.concatenate([nzs[pick], rng.integers(0, n, 200)])
    ok, dzmax, bmax = kkt_fp64_within_bound(orc, X, D, Zh, float(np.float32(lam)), w.tol, ks2, ss2)
    assert ok, (dzmax, bmax)
    # phi and psi of the GPU's Z against the oracle's, from the nonzeros
    phi, psi = pkg.cdl_dict_stats(Z, Xd, D.shape, prob.phi, prob.psi, prob.ws)
    zi, zj = nzs // Tz[1], nzs % Tz[1]
    zv = Zh.reshape(w.K, -1)[nzk, nzs]
    pr, sr = orc.phi_psi_nz(X, w.L, w.K, nzk, zi, zj, zv)
    pa, sa = orc.phi_psi_nz(np.abs(X), w.L, w.K, nzk, zi, zj, np.abs(zv))
    # phi: FP64 products and sums, rounded once to FP32
    assert np.all(np.abs(host(phi) - pr) <= 2.0 ** -24 * np.abs(pr) + 1e-12 * pa)
    # psi: FP32 sums over chunks of at most 64 nonzeros, FP64 across chunks,
    # rounded once to FP32
    assert np.all(np.abs(host(psi) - sr) <= gamma(65) * sa + 1e-12 * np.abs(sr).max())


def test_image_1024_of_the_4096_family_against_the_oracle_solve(pkg, orc):
    """The full oracle solve (Alg. 1, FP64) of a 1024 x 1024 image drawn like
    the 4096 x 4096 workload, against the GPU's global-tile path with the
    default options: objective within 1e-5 relative, support within the
    stated count, KKT on the GPU and on the oracle's FP64 beta."""
    w = scaled(IMAGE_4096, (1024, 1024))
    X, D, _ = make_problem(w, 3)
    lam = w.reg * orc.lambda_max(X, D)
    ref = orc.lgcd(X, D, lam, w.tol)
    assert ref["status"] == 0
    Xd, Dd = dev(X), dev(D)
    prob = pkg.Problem.create(Xd, Dd)
    beta, dtd, _ = pkg.csc_init_beta(Xd, Dd, prob.beta, prob.dtd, prob.ws)
    Z, st = pkg.csc_lgcd_solve(Xd, Dd, dtd, beta, lam, w.tol, Z=prob.Z, ws=prob.ws)
    assert st["status"] == 0 and st["placement"] == 2 and st["workers"] > 1, st
    assert st["max_dz_final"] < w.tol
    Zh = host(Z)
    f_ref = orc.objective(X, D, ref["Z"], lam)
    f_gpu = orc.objective(X, D, Zh, lam)
    assert abs(f_gpu - f_ref) <= 1e-5 * abs(f_ref), (f_gpu, f_ref)
    assert abs(st["objective"] - f_gpu) <= 1e-6 * abs(f_gpu)
    ok, dzmax, bmax = kkt_fp64_within_bound(orc, X, D, Zh, float(np.float32(lam)), w.tol)
    assert ok, (dzmax, bmax)
    nnz = int((ref["Z"] != 0).sum())
    cnt, worst = support_mismatch(Zh, ref["Z"], w.tol)
    assert cnt <= max(10, 0.01 * nnz) and worst <= 100 * w.tol, (cnt, nnz, worst)
