"""Failure statuses of the solve and the soft-lock, on the GPU, in the forms
that leave the device usable: every device-side wait and loop of the LGCD
kernels is bounded by the solve's deadline and stop word, so a run that
cannot finish returns a status instead of hanging.

* CSC_ERR_TIMEOUT: a deadline far shorter than the solve; the call returns
  the status and the next solve on the same buffers is correct.
* CSC_NOT_CONVERGED: a cap on the number of coordinate updates.
* CSC_ERR_DIVERGED: the guard of Section 5.1 (|Z| above min_k 50 / max|D_k|)
  on an observation scaled so that the exact solution itself passes the
  bound.
* Soft-locks (Eq. soft_lock): with small tiles the asynchronous solve rejects
  border candidates and still reaches the oracle's objective; the no-lock
  ablation on the same input ends with a valid status (the interference of
  Prop. A.2 it may suffer is shown deterministically by the CPU protocol
  simulation in tests/test_protocol_sim.py)."""
import numpy as np
import pytest

from synthetic import Workload, make_problem
from tests._gpu import dev, host, kkt_fp64_within_bound

pytestmark = pytest.mark.gpu

W1 = Workload("fail1d", P=3, K=4, T=(6000,), L=(32,), density=0.01, sigma=0.1)
W2 = Workload("fail2d", P=1, K=25, T=(512, 512), L=(32, 32), density=1e-4, sigma=0.05, nonneg=True)
CASES = [(W1, 1), (W2, 2)]  # (workload, expected placement)


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


def _setup(pkg, w, seed, scale=1.0):
    X, D, _ = make_problem(w, seed)
    X = (X * np.float32(scale)).astype(np.float32)
    Xd, Dd = dev(X), dev(D)
    prob = pkg.Problem.create(Xd, Dd)
    beta, dtd, lmax = pkg.csc_init_beta(Xd, Dd, prob.beta, prob.dtd, prob.ws)
    return X, D, Xd, Dd, prob, lmax


@pytest.mark.parametrize("w,placement", CASES, ids=["smem_tiles", "global_tiles"])
def test_deadline_returns_timeout_and_the_next_solve_is_correct(pkg, orc, w, placement):
    X, D, Xd, Dd, prob, lmax = _setup(pkg, w, 41)
    lam = 0.1 * lmax
    beta0 = prob.beta.clone()
    with pytest.raises(pkg.CscError) as e:
        pkg.csc_lgcd_solve(Xd, Dd, prob.dtd, prob.beta, lam, 1e-4, Z=prob.Z, ws=prob.ws,
                           opts=pkg.default_opts(timeout_s=2e-6))
    assert e.value.status == pkg.CSC_ERR_TIMEOUT
    assert e.value.stats["status"] == pkg.CSC_ERR_TIMEOUT
    # the same buffers, a normal solve: the context and the workspace are fine
    prob.beta.copy_(beta0)
    Z, st = pkg.csc_lgcd_solve(Xd, Dd, prob.dtd, prob.beta, lam, 1e-4, Z=prob.Z, ws=prob.ws)
    assert st["status"] == pkg.CSC_OK and st["placement"] == placement, st
    assert st["max_dz_final"] < 1e-4
    Zh = host(Z)
    assert abs(st["objective"] - orc.objective_sparse(X, D, Zh, float(np.float32(lam)))) <= 1e-9 * st["objective"]


@pytest.mark.parametrize("w,placement", CASES, ids=["smem_tiles", "global_tiles"])
def test_update_cap_returns_not_converged(pkg, orc, w, placement):
    X, D, Xd, Dd, prob, lmax = _setup(pkg, w, 42)
    lam = 0.1 * lmax
    cap = 40
    Z, st = pkg.csc_lgcd_solve(Xd, Dd, prob.dtd, prob.beta, lam, 1e-4, Z=prob.Z, ws=prob.ws,
                               opts=pkg.default_opts(max_updates=cap))
    assert st["status"] == pkg.CSC_NOT_CONVERGED and st["placement"] == placement, st
    # the cap stops every worker; those already past their check finish their update
    assert cap <= st["updates"] <= cap + st["workers"]
    Zh = host(Z)
    assert 0 < int((Zh != 0).sum()) <= st["updates"]
    # every accepted update lowered the cost (Prop. A.1, soft-locks on)
    f0 = 0.5 * float(np.sum(X.astype(np.float64) ** 2))
    assert orc.objective_sparse(X, D, Zh, float(np.float32(lam))) < f0


@pytest.mark.parametrize("w,placement", CASES, ids=["smem_tiles", "global_tiles"])
def test_divergence_guard(pkg, orc, w, placement):
    """An observation scaled by 1e4: the solution's activations exceed the
    guard's bound min_k 50 / max|D_k|, so with the guard on the solve stops
    with CSC_ERR_DIVERGED; with it off the same solve converges."""
    X, D, Xd, Dd, prob, lmax = _setup(pkg, w, 43, scale=1e4)
    lam = 0.1 * lmax
    bound = min(50.0 / np.abs(D[k]).max() for k in range(w.K))
    beta0 = prob.beta.clone()
    Z, st = pkg.csc_lgcd_solve(Xd, Dd, prob.dtd, prob.beta, lam, 1e-4 * 1e4, Z=prob.Z, ws=prob.ws,
                               opts=pkg.default_opts(divergence_guard=1))
    assert st["status"] == pkg.CSC_ERR_DIVERGED and st["placement"] == placement, st
    assert np.abs(host(Z)).max() > bound
    prob.beta.copy_(beta0)
    Z, st = pkg.csc_lgcd_solve(Xd, Dd, prob.dtd, prob.beta, lam, 1e-4 * 1e4, Z=prob.Z, ws=prob.ws,
                               opts=pkg.default_opts(divergence_guard=0))
    assert st["status"] == pkg.CSC_OK, st
    assert np.abs(host(Z)).max() > bound


# small tiles (2 L) and dense activations: many border candidates compete
W_LOCK = Workload("lock1d", P=2, K=3, T=(8000,), L=(32,), density=0.03, sigma=0.1)


def test_softlock_rejects_border_candidates_and_keeps_parity(pkg, orc):
    X, D, Xd, Dd, prob, lmax = _setup(pkg, W_LOCK, 44)
    lam = 0.1 * orc.lambda_max(X, D)
    tol = 1e-4
    beta0 = prob.beta.clone()
    opts = pkg.default_opts(tile=(64,))
    Z, st = pkg.csc_lgcd_solve(Xd, Dd, prob.dtd, prob.beta, lam, tol, Z=prob.Z, ws=prob.ws, opts=opts)
    assert st["status"] == pkg.CSC_OK and st["workers"] > 100, st
    assert st["rejected_softlock"] > 0, st
    ref = orc.lgcd(X, D, lam, tol)
    Zh = host(Z)
    f_ref = orc.objective(X, D, ref["Z"], lam)
    assert abs(orc.objective(X, D, Zh, lam) - f_ref) <= 1e-5 * abs(f_ref)
    assert kkt_fp64_within_bound(orc, X, D, Zh, lam, tol)[0]
    # the no-lock ablation on the same input: accepted border updates are not
    # checked against the neighbours, no candidate is rejected, and the solve
    # ends with a status (converged, capped or stopped by the guard)
    prob.beta.copy_(beta0)
    nl = pkg.default_opts(tile=(64,), mode=pkg.MODE_NOLOCK, divergence_guard=1, max_updates=200000, timeout_s=5.0)
    Zn, sn = pkg.csc_lgcd_solve(Xd, Dd, prob.dtd, prob.beta, lam, tol, Z=prob.Z, ws=prob.ws, opts=nl)
    assert sn["status"] in (pkg.CSC_OK, pkg.CSC_NOT_CONVERGED, pkg.CSC_ERR_DIVERGED), sn
    assert sn["rejected_softlock"] == 0
    if sn["status"] == pkg.CSC_OK:
        assert sn["max_dz_final"] < tol
