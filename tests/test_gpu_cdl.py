"""The outer dictionary-learning loop (Alg. 2) through cdl_fit.

* A small image (the 8192^2 family at 96 x 96): the cost after every CSC step
  and after every dictionary step matches the oracle's loop.
* The 8192 x 8192 workload (25 atoms of 32 x 32): self-checks that hold at any
  size -- the cost never increases, the final cost equals the oracle's
  objective from the nonzeros of the final Z, and every atom stays in the
  unit ball."""
import numpy as np
import pytest

from synthetic import IMAGE_8192, Workload, make_problem
from tests._gpu import dev, host

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


def _monotone(trace, rel=1e-5):
    prev = np.inf
    for c_csc, c_dict in trace:
        assert c_csc <= prev * (1 + rel)
        assert c_dict <= c_csc * (1 + rel)
        prev = c_dict


def test_cdl_small_matches_oracle(pkg, orc):
    w = Workload("cdl96", P=1, K=4, T=(96, 96), L=(8, 8), density=5e-3, sigma=0.05, nonneg=True)
    X, D0, _ = make_problem(w, 41)
    rng = np.random.default_rng(5)
    D0 = D0 + 0.3 * rng.standard_normal(D0.shape).astype(np.float32)
    D0 /= np.sqrt((D0.reshape(w.K, -1) ** 2).sum(1)).reshape(-1, 1, 1, 1)
    _, _, tr_ref = orc.cdl(X, D0, 0.1, 1e-4, 3, pgd_max_iter=20)
    Dd = dev(D0)
    Z, tr, rc = pkg.cdl_fit(dev(X), Dd, reg=0.1, tol=1e-4, max_outer=3, pgd_max_iter=20)
    assert rc == 0 and len(tr) == 3
    for (a, b), (ra, rb) in zip(tr, tr_ref):
        assert abs(a - ra) <= 1e-4 * abs(ra)
        assert abs(b - rb) <= 1e-4 * abs(rb)
    _monotone(tr)


def test_cdl_small_mixed_precision_matches_oracle(pkg, orc):
    """The same loop with the beta-init of every iteration after the first on
    the tensor cores (split bf16): each solve still ends on a beta recomputed
    in FP32, so the costs match the oracle's loop as closely as in FP32."""
    w = Workload("cdl96", P=1, K=4, T=(96, 96), L=(8, 8), density=5e-3, sigma=0.05, nonneg=True)
    X, D0, _ = make_problem(w, 41)
    rng = np.random.default_rng(5)
    D0 = D0 + 0.3 * rng.standard_normal(D0.shape).astype(np.float32)
    D0 /= np.sqrt((D0.reshape(w.K, -1) ** 2).sum(1)).reshape(-1, 1, 1, 1)
    _, _, tr_ref = orc.cdl(X, D0, 0.1, 1e-4, 3, pgd_max_iter=20)
    opts = pkg.default_opts(beta_init=1)
    Z, tr, rc = pkg.cdl_fit(dev(X), dev(D0), reg=0.1, tol=1e-4, max_outer=3, pgd_max_iter=20, opts=opts)
    assert rc == 0 and len(tr) == 3
    for (a, b), (ra, rb) in zip(tr, tr_ref):
        assert abs(a - ra) <= 1e-4 * abs(ra)
        assert abs(b - rb) <= 1e-4 * abs(rb)
    _monotone(tr)


def test_cdl_small_repeated_solves_terminate(pkg):
    """Exact ties between border candidates of neighbouring tiles are common
    late in a solve on this problem (|dZ| values near tol are coarsely
    quantised in FP32); the soft-lock test must let one side win every time.
    36 asynchronous solves, each bounded by a 5 s device limit."""
    w = Workload("cdl96", P=1, K=4, T=(96, 96), L=(8, 8), density=5e-3, sigma=0.05, nonneg=True)
    X, D0, _ = make_problem(w, 41)
    rng = np.random.default_rng(5)
    D0 = D0 + 0.3 * rng.standard_normal(D0.shape).astype(np.float32)
    D0 /= np.sqrt((D0.reshape(w.K, -1) ** 2).sum(1)).reshape(-1, 1, 1, 1)
    Xd = dev(X)
    opts = pkg.default_opts(timeout_s=5.0)
    prob = pkg.Problem.create(Xd, dev(D0))
    for rep in range(12):
        Dd = dev(D0)
        prob.D = Dd
        _, tr, rc = pkg.cdl_fit(Xd, Dd, reg=0.1, tol=1e-4, max_outer=3, pgd_max_iter=20, opts=opts,
                                prob=prob)
        assert rc == 0 and len(tr) == 3, rep
        _monotone(tr)


def test_cdl_image_8192_selfchecks(pkg, orc):
    import torch
    w = IMAGE_8192
    X, D0, _ = make_problem(w, 0)
    Xd, Dd = dev(X), dev(D0)
    Z, tr, rc = pkg.cdl_fit(Xd, Dd, reg=w.reg, tol=w.tol, max_outer=3)
    assert rc == 0 and len(tr) == 3
    _monotone(tr)
    # the last cost equals the oracle's objective from the nonzeros of the
    # final Z with the final D and the same (fp32) lambda
    _, _, lmax0 = pkg.csc_init_beta(Xd, dev(D0))
    lam = float(np.float32(w.reg * lmax0))
    nz = torch.nonzero(Z).cpu().numpy()
    vals = host(Z[tuple(torch.from_numpy(nz.T.copy()).to(Z.device))])
    f_ref = orc.objective_nz(X, host(Dd), nz[:, 0], nz[:, 1], nz[:, 2], vals, lam)
    assert abs(tr[-1][1] - f_ref) <= 1e-9 * abs(f_ref)
    nr = np.sqrt((host(Dd).reshape(w.K, -1).astype(np.float64) ** 2).sum(1))
    assert np.all(nr <= 1 + 1e-6)


@pytest.mark.parametrize("w", [
    Workload("step1d", P=5, K=10, T=(3001,), L=(64,), density=0.005, sigma=0.1),
    Workload("step2d", P=2, K=5, T=(70, 150), L=(8, 12), density=0.01, sigma=0.1),
], ids=["1d", "2d"])
def test_cdl_step_matches_the_separate_calls(pkg, orc, w):
    """cdl_step (one pass of the loop body in one call, the nonzero count read
    back only at the end) gives what the four calls give: the same lambda, a
    solve within 1e-5 of the oracle's objective, phi / psi equal to
    cdl_dict_stats on its Z, and D, F and the iteration count of
    cdl_dict_update on its phi / psi, bit for bit."""
    import torch
    X, D0, _ = make_problem(w, 43)
    Xd = dev(X)
    xs = float(np.sum(X.astype(np.float64) ** 2))
    D = dev(D0)
    prob = pkg.Problem.create(Xd, D)
    Z, st = pkg.cdl_step(Xd, D, prob, reg=0.1, tol=1e-4, x_sqnorm=xs, pgd_max_iter=50, pgd_tol=1e-8)
    assert st["status"] == 0
    _, _, lm = pkg.csc_init_beta(Xd, dev(D0))
    assert st["lambda"] == float(np.float32(0.1 * lm))
    lam = st["lambda"]
    f_ref = orc.objective(X, D0, orc.lgcd(X, D0, lam, 1e-4)["Z"], lam)
    f_gpu = orc.objective(X, D0, host(Z).astype(np.float64), lam)
    assert abs(f_gpu - f_ref) <= 1e-5 * abs(f_ref)
    phi2, psi2 = pkg.cdl_dict_stats(Z, Xd, tuple(D0.shape))
    assert torch.allclose(prob.phi, phi2, rtol=1e-6, atol=0)
    assert torch.allclose(prob.psi, psi2, rtol=1e-6, atol=0)
    D2 = dev(D0)
    F2, it2 = pkg.cdl_dict_update(prob.phi, prob.psi, xs, D2, tuple(X.shape), max_iter=50, tol=1e-8)
    assert torch.equal(D2, D)
    assert F2 == st["dict_F"] and it2 == st["dict_iters"]


def test_chained_cdl_steps_with_a_fixed_lambda_follow_cdl_fit(pkg, orc):
    """Two cdl_step calls, the second with the first one's lambda, solve the
    fixed problem of Alg. 2 as cdl_fit's first two iterations do: the costs
    after each CSC step agree and so do the dictionaries.  The solves are
    asynchronous: each stops somewhere in the set where max |dZ| < tol (Alg. 1
    stops there, not at the optimum), and two runs of the same solve spread
    by about 1.1e-5 relative on this image, so costs are compared at 5e-5.  ||X||^2 is
    summed on the device; beta-init in FP32 and, for the second call, on the
    tensor cores."""
    w = Workload("chain96", P=1, K=4, T=(96, 96), L=(8, 8), density=5e-3, sigma=0.05, nonneg=True)
    X, D0, _ = make_problem(w, 41)
    rng = np.random.default_rng(5)
    D0 = D0 + 0.3 * rng.standard_normal(D0.shape).astype(np.float32)
    D0 /= np.sqrt((D0.reshape(w.K, -1) ** 2).sum(1)).reshape(-1, 1, 1, 1)
    Xd = dev(X)
    Dfit = dev(D0)
    _, tr, rc = pkg.cdl_fit(Xd, Dfit, reg=0.1, tol=1e-4, max_outer=2, nu=0.0, pgd_max_iter=20)
    assert rc == 0 and len(tr) == 2
    for beta_init in (0, 1):
        D = dev(D0)
        prob = pkg.Problem.create(Xd, D)
        _, s1 = pkg.cdl_step(Xd, D, prob, reg=0.1, tol=1e-4, pgd_max_iter=20)
        lam = s1["lambda"]
        _, s2 = pkg.cdl_step(Xd, D, prob, reg=0.0, lam=lam, tol=1e-4, pgd_max_iter=20,
                             opts=pkg.default_opts(beta_init=beta_init))
        assert s1["status"] == 0 and s2["status"] == 0 and s2["lambda"] == lam
        for st, (c_csc, _) in zip((s1, s2), tr):
            assert abs(st["objective"] - c_csc) <= 5e-5 * abs(c_csc), (st["objective"], c_csc)
        assert np.allclose(host(D), host(Dfit), rtol=0, atol=1e-3)
        # the same cost on the oracle's side: its loop with the same fixed lambda
        _, _, tr_ref = orc.cdl(X, D0, 0.1, 1e-4, 2, pgd_max_iter=20)
        assert abs(s2["objective"] - tr_ref[1][0]) <= 1e-4 * abs(tr_ref[1][0])


def test_cdl_step_reports_a_nonzero_list_overflow(pkg):
    """A Z with more nonzeros than the workspace's list holds: cdl_step, which
    reads the count back only at the end, still answers CSC_ERR_WORKSPACE
    (the statistics kernels skip the unwritten list).  The dense Z comes from
    a warm start that the solve leaves after one update (max_updates = 1)."""
    import torch
    w = Workload("dense1d", P=1, K=4, T=(400_000,), L=(16,), density=0.005, sigma=0.1)
    X, D0, _ = make_problem(w, 47)
    Xd, D = dev(X), dev(D0)
    prob = pkg.Problem.create(Xd, D)
    gen = torch.Generator(device="cuda").manual_seed(3)
    prob.Z.copy_(0.01 * (torch.rand(prob.Z.shape, generator=gen, device="cuda") + 0.5))
    opts = pkg.default_opts(warm_start=1, max_updates=1)
    D_before = D.clone()
    with pytest.raises(pkg.CscError) as e:
        pkg.cdl_step(Xd, D, prob, reg=0.1, tol=1e-4, opts=opts)
    assert e.value.status == pkg.CSC_ERR_WORKSPACE
    # the dictionary step did not run on the statistics that were not computed
    assert torch.equal(D, D_before)
    # the separate statistics call reports the same overflow
    with pytest.raises(pkg.CscError) as e2:
        pkg.cdl_dict_stats(prob.Z, Xd, tuple(D0.shape), prob.phi, prob.psi, prob.ws)
    assert e2.value.status == pkg.CSC_ERR_WORKSPACE


_CROP = {}


def _crop_8192_family_oracle(orc):
    """A 1024 x 1024 image of the 8192^2 workload's family (same generator,
    25 atoms of 32 x 32, density 5e-5, noise 0.05) and the oracle's loop on it
    (Alg. 2 from the generating atoms, three outer iterations, five PGD
    iterations each), computed once for both precisions."""
    if not _CROP:
        from synthetic import scaled
        w = scaled(IMAGE_8192, (1024, 1024))
        X, D0, _ = make_problem(w, 5)
        _, _, tr = orc.cdl(X, D0, w.reg, w.tol, 3, pgd_max_iter=5)
        _CROP.update(w=w, X=X, D0=D0, trace=tr)
    return _CROP


@pytest.mark.parametrize("beta_init", [0, 1], ids=["fp32", "bf16x3"])
def test_cdl_1024_crop_of_the_8192_family_against_the_oracle_loop(pkg, orc, beta_init):
    """cdl_fit on the crop in the bench's precisions (FP32 beta-init, or split
    bf16 after the first iteration) against the oracle's loop: the cost after
    every CSC step and after every dictionary step within 1e-4 relative."""
    c = _crop_8192_family_oracle(orc)
    w = c["w"]
    Dd = dev(c["D0"])
    _, tr, rc = pkg.cdl_fit(dev(c["X"]), Dd, reg=w.reg, tol=w.tol, max_outer=3, nu=0.0, pgd_max_iter=5,
                            opts=pkg.default_opts(beta_init=beta_init))
    assert rc == 0 and len(tr) == 3
    for (a, b), (ra, rb) in zip(tr, c["trace"]):
        assert abs(a - ra) <= 1e-4 * abs(ra), (a, ra)
        assert abs(b - rb) <= 1e-4 * abs(rb), (b, rb)
    _monotone(tr)
