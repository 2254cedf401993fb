"""CUDA path against the FP64 oracle, element by element, through the C ABI.

Sizes are small enough for the oracle to finish in seconds yet span several
CTA tiles / worker tiles with ragged tails."""
import numpy as np
import pytest

from synthetic import Workload, make_problem
from tests._gpu import dev, gamma, host, kkt_fp64_within_bound, support_mismatch

pytestmark = pytest.mark.gpu

W_1D = Workload("t1d", P=5, K=10, T=(3001,), L=(64,), density=0.005, sigma=0.1)
W_2D = Workload("t2d", P=2, K=5, T=(70, 150), L=(8, 12), density=0.01, sigma=0.1)
W_IMG = Workload("img64", P=1, K=5, T=(64, 64), L=(8, 8), density=0.01, sigma=0.1)
W_DEG = Workload("deg", P=3, K=1, T=(37, 41), L=(1, 1), density=0.05, sigma=0.1)
W_ONE = Workload("one", P=2, K=4, T=(9, 7), L=(9, 7), density=1.0, sigma=0.1)
# 25 atoms: the dictionary step's cluster holds 2 atoms per CTA and the last CTA one
W_RAG = Workload("rag", P=1, K=25, T=(40, 40), L=(4, 4), density=0.02, sigma=0.1)
# 9 channels: the dictionary step's convolution takes them in chunks of 8
W_P9 = Workload("p9", P=9, K=3, T=(400,), L=(16,), density=0.01, sigma=0.1)
SHAPES = [W_1D, W_2D, W_IMG, W_DEG, W_ONE]


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


@pytest.mark.parametrize("w", SHAPES, ids=[w.name for w in SHAPES])
def test_init_beta_and_dtd_fp32(pkg, orc, w):
    """beta = D~ * X, the D^T D table and lambda_max within the gamma_n bound
    of an n = P|Theta| term fp32 dot product."""
    import torch
    X, D, _ = make_problem(w, 21)
    beta, dtd, lmax = pkg.csc_init_beta(dev(X), dev(D))
    torch.cuda.synchronize()
    ref = orc.beta_init(X, D)
    n = w.P * int(np.prod(w.L))
    bound = gamma(n) * orc.beta_init(np.abs(X), np.abs(D)) + 1e-30
    assert np.all(np.abs(host(beta) - ref) <= bound)
    d = len(w.L)
    tref = orc.dtd(D, d)
    tbound = gamma(n) * orc.dtd(np.abs(D), d) + 1e-30
    assert np.all(np.abs(host(dtd) - tref) <= tbound)
    assert abs(lmax - np.abs(ref).max()) <= bound.max()


@pytest.mark.parametrize("w", [W_1D, W_2D], ids=["1d", "2d"])
def test_init_beta_fp64(pkg, orc, w):
    import torch
    X, D, _ = make_problem(w, 22)
    beta, dtd, lmax = pkg.csc_init_beta(dev(X, torch.float64), dev(D, torch.float64))
    n = w.P * int(np.prod(w.L))
    bound = gamma(n, 2.0 ** -53) * orc.beta_init(np.abs(X), np.abs(D)) * 2 + 1e-300
    assert np.all(np.abs(host(beta) - orc.beta_init(X, D)) <= bound)
    assert abs(lmax - orc.lambda_max(X, D)) <= bound.max()


PHASED = [
    (Workload("p1d", P=2, K=3, T=(600,), L=(16,), density=0.01, sigma=0.1), (64,)),
    (Workload("p1d_b", P=1, K=2, T=(500,), L=(9,), density=0.02, sigma=0.1), (40,)),
    (Workload("p2d", P=1, K=3, T=(60, 70), L=(6, 5), density=0.01, sigma=0.1), (14, 12)),
    (Workload("p2d_b", P=2, K=2, T=(45, 33), L=(4, 4), density=0.02, sigma=0.1), (8, 9)),
]


@pytest.mark.parametrize("w,tile", PHASED, ids=[p[0].name for p in PHASED])
def test_phased_fp64_equals_oracle_schedule(pkg, orc, w, tile):
    """The deterministic checkerboard mode in FP64 makes the same choices as
    the oracle's tiled schedule: same number of updates, same Z to 1e-12."""
    import torch
    X, D, _ = make_problem(w, 23)
    lam = 0.1 * orc.lambda_max(X, D)
    tol = 1e-6
    ref = orc.lgcd(X, D, lam, tol, tile=tile)
    assert ref["status"] == 0
    Xd, Dd = dev(X, torch.float64), dev(D, torch.float64)
    beta, dtd, _ = pkg.csc_init_beta(Xd, Dd)
    opts = pkg.default_opts(mode=pkg.MODE_PHASED, tile=tile, beta_refresh=0)
    Z, st = pkg.csc_lgcd_solve(Xd, Dd, dtd, beta, lam, tol, opts=opts)
    assert st["status"] == 0, st
    assert st["updates"] == ref["n_updates"]
    np.testing.assert_allclose(host(Z), ref["Z"], rtol=0, atol=1e-12)
    assert st["max_dz_final"] < tol


@pytest.mark.parametrize("w,tile", PHASED, ids=[p[0].name for p in PHASED])
def test_phased_fp32_objective(pkg, orc, w, tile):
    X, D, _ = make_problem(w, 24)
    lam = 0.1 * orc.lambda_max(X, D)
    tol = 1e-4
    ref = orc.lgcd(X, D, lam, tol, tile=tile)
    Xd, Dd = dev(X), dev(D)
    beta, dtd, _ = pkg.csc_init_beta(Xd, Dd)
    opts = pkg.default_opts(mode=pkg.MODE_PHASED, tile=tile)
    Z, st = pkg.csc_lgcd_solve(Xd, Dd, dtd, beta, lam, tol, opts=opts)
    assert st["status"] == 0, st
    f_ref = orc.objective(X, D, ref["Z"], lam)
    f_gpu = orc.objective(X, D, host(Z), lam)
    assert abs(f_gpu - f_ref) <= 1e-5 * abs(f_ref)
    # FP64 KKT within the FP32 recomputation's rounding bound (tests/_gpu.py)
    assert kkt_fp64_within_bound(orc, X, D, host(Z), lam, tol)[0]


ASYNC = [
    Workload("a1d", P=5, K=10, T=(20000,), L=(64,), density=0.005, sigma=0.1),
    Workload("a1d_small_tiles", P=2, K=4, T=(5000,), L=(16,), density=0.01, sigma=0.1),
    W_IMG,
    Workload("a2d", P=1, K=5, T=(200, 230), L=(8, 8), density=0.01, sigma=0.1),
    Workload("a2d_rgb", P=3, K=6, T=(120, 90), L=(12, 12), density=0.002, sigma=0.1),
]


@pytest.mark.parametrize("w", ASYNC, ids=[w.name for w in ASYNC])
def test_async_softlock_matches_oracle(pkg, orc, w):
    """Asynchronous tiles with soft-locks reach the oracle's objective within
    1e-5 relative, satisfy max|dZ| < tol on a beta recomputed in FP64, and
    differ from the oracle's support only on small coordinates."""
    X, D, _ = make_problem(w, 25)
    lam = 0.1 * orc.lambda_max(X, D)
    tol = 1e-4
    ref = orc.lgcd(X, D, lam, tol)
    Xd, Dd = dev(X), dev(D)
    beta, dtd, _ = pkg.csc_init_beta(Xd, Dd)
    Z, st = pkg.csc_lgcd_solve(Xd, Dd, dtd, beta, lam, tol)
    assert st["status"] == 0, st
    assert st["workers"] > 1
    Zh = host(Z)
    f_ref = orc.objective(X, D, ref["Z"], lam)
    f_gpu = orc.objective(X, D, Zh, lam)
    assert abs(f_gpu - f_ref) <= 1e-5 * abs(f_ref)
    assert abs(st["objective"] - f_gpu) <= 1e-6 * abs(f_gpu)
    # FP64 KKT within the FP32 recomputation's rounding bound (tests/_gpu.py)
    assert kkt_fp64_within_bound(orc, X, D, Zh, lam, tol)[0]
    nnz = int((ref["Z"] != 0).sum())
    cnt, worst = support_mismatch(Zh, ref["Z"], tol)
    assert cnt <= max(10, 0.01 * nnz), (cnt, nnz)
    assert worst <= 100 * tol


def test_lambda_max_gives_zero(pkg, orc):
    """lambda >= lambda_max: Z = 0 exactly and no update (Section 2)."""
    X, D, _ = make_problem(W_2D, 26)
    Xd, Dd = dev(X), dev(D)
    beta, dtd, lmax = pkg.csc_init_beta(Xd, Dd)
    Z, st = pkg.csc_lgcd_solve(Xd, Dd, dtd, beta, lmax * 1.0001, 1e-4)
    assert st["status"] == 0 and st["updates"] == 0
    assert not host(Z).any()


def test_objective_call(pkg, orc):
    rng = np.random.default_rng(0)
    X, D, Z = make_problem(W_2D, 27)
    Zp = (Z + 0.01 * rng.standard_normal(Z.shape) * (rng.random(Z.shape) < 0.01)).astype(np.float32)
    lam = 0.37
    got = pkg.csc_objective(dev(X), dev(D), dev(Zp), lam)
    ref = orc.objective(X, D, Zp, lam)
    assert abs(got - ref) <= 1e-12 * abs(ref) + 1e-12


@pytest.mark.parametrize("w", [W_1D, W_2D, W_IMG], ids=["1d", "2d", "img"])
def test_dict_stats(pkg, orc, w):
    """phi and psi from the nonzeros of Z (Section 4.2) against their
    definitions; psi partial sums run in fp32 over chunks of 64 nonzeros."""
    X, D, Z = make_problem(w, 28)
    phi, psi = pkg.cdl_dict_stats(dev(Z), dev(X), D.shape)
    pref, sref = orc.phi_psi(Z, X, w.L)
    np.testing.assert_allclose(host(phi), pref, rtol=1e-6, atol=1e-6 * np.abs(pref).max())
    sb = gamma(64) * orc.phi_psi(np.abs(Z), np.abs(X), w.L)[1] * 2 + 1e-7 * np.abs(sref).max()
    assert np.all(np.abs(host(psi) - sref) <= sb)


def check_dict_step(orc, phi32, psi32, xs, D0, Dg, f_gpu, f_ref, L):
    """The GPU dictionary (evaluated in FP64) reaches at least 99.99 % of the
    oracle's decrease and stays in the unit ball; the cost the GPU reports
    agrees with the FP64 value within the FP32 accumulation bound of
    F = xs/2 - <D, psi> + <D, phi * D>/2 (phi * D summed over K prod(2L - 1)
    terms, products with psi rounded once)."""
    K = D0.shape[0]
    f0 = orc.dict_objective(phi32, psi32, xs, D0)
    f_d = orc.dict_objective(phi32, psi32, xs, Dg)
    assert f_d <= f0
    assert f_d - f_ref <= 1e-4 * (f0 - f_ref) + 1e-12 * abs(f_ref)
    quad = orc.dict_objective(np.abs(phi32), np.zeros_like(psi32), 0.0, np.abs(Dg))
    lin = -orc.dict_objective(np.zeros_like(phi32), np.abs(psi32), 0.0, np.abs(Dg))
    n = K * int(np.prod([2 * l - 1 for l in L])) + 1
    assert abs(f_gpu - f_d) <= gamma(n) * quad + gamma(1) * lin
    nr = np.sqrt((Dg.reshape(K, -1).astype(np.float64) ** 2).sum(1))
    assert np.all(nr <= 1 + 1e-6)


@pytest.mark.parametrize("w", [W_1D, W_2D, W_IMG, W_RAG, W_P9], ids=["1d", "2d", "img", "ragged", "p9"])
def test_dict_update(pkg, orc, w):
    """PGD + Armijo on the same (phi, psi) as the oracle's (Alg. 2)."""
    X, D, Z = make_problem(w, 29)
    rng = np.random.default_rng(3)
    D0 = (D + 0.3 * rng.standard_normal(D.shape)).astype(np.float32)
    phi, psi = orc.phi_psi(Z, X, w.L)
    phi32, psi32 = phi.astype(np.float32), psi.astype(np.float32)
    xs = float(np.sum(X.astype(np.float64) ** 2))
    Dd = dev(D0)
    f_gpu, it = pkg.cdl_dict_update(dev(phi32), dev(psi32), xs, Dd, X.shape, max_iter=50, tol=1e-8)
    D_ref, f_ref, it_ref = orc.pgd_armijo(phi32, psi32, xs, D0, max_iter=50, tol=1e-8)
    check_dict_step(orc, phi32, psi32, xs, D0, host(Dd), f_gpu, f_ref, w.L)
    # the reported iteration count: a perturbed D needs steps, never more than the cap
    assert 1 <= it <= 50 and 1 <= it_ref <= 50


@pytest.mark.parametrize("w", [W_1D, W_2D], ids=["1d", "2d"])
def test_dict_update_from_the_generating_atoms(pkg, orc, w):
    """Started from the unit-norm atoms that generated X (norm constraints
    active near the solution, as in the CDL loop), the FP32 step stops by its
    own tests before the iteration cap and its cost is within 10^-6
    (relative) of the FP64 oracle's."""
    X, D, Z = make_problem(w, 31)
    phi, psi = orc.phi_psi(Z, X, w.L)
    phi32, psi32 = phi.astype(np.float32), psi.astype(np.float32)
    xs = float(np.sum(X.astype(np.float64) ** 2))
    Dd = dev(D)
    _, it = pkg.cdl_dict_update(dev(phi32), dev(psi32), xs, Dd, X.shape, max_iter=50, tol=1e-8)
    _, f_ref, it_ref = orc.pgd_armijo(phi32, psi32, xs, D, max_iter=50, tol=1e-8)
    f_d = orc.dict_objective(phi32, psi32, xs, host(Dd))
    assert it < 50, (it, it_ref)
    assert f_d - f_ref <= 1e-6 * abs(f_ref), (f_d, f_ref, it, it_ref)


@pytest.mark.parametrize("w", ASYNC, ids=[w.name for w in ASYNC])
def test_async_global_tiles_match_oracle(pkg, orc, w):
    """The global-memory variant (beta, Z in HBM, atomic window updates,
    neighbour flags) forced on the same cases reaches the same bar."""
    X, D, _ = make_problem(w, 35)
    lam = 0.1 * orc.lambda_max(X, D)
    tol = 1e-4
    ref = orc.lgcd(X, D, lam, tol)
    Xd, Dd = dev(X), dev(D)
    beta, dtd, _ = pkg.csc_init_beta(Xd, Dd)
    Z, st = pkg.csc_lgcd_solve(Xd, Dd, dtd, beta, lam, tol, opts=pkg.default_opts(placement=2))
    assert st["status"] == 0, st
    assert st["placement"] == 2 and st["workers"] > 1
    Zh = host(Z)
    f_ref = orc.objective(X, D, ref["Z"], lam)
    f_gpu = orc.objective(X, D, Zh, lam)
    assert abs(f_gpu - f_ref) <= 1e-5 * abs(f_ref)
    # FP64 KKT within the FP32 recomputation's rounding bound (tests/_gpu.py)
    assert kkt_fp64_within_bound(orc, X, D, Zh, lam, tol)[0]
    cnt, worst = support_mismatch(Zh, ref["Z"], tol)
    assert cnt <= max(10, 0.01 * int((ref["Z"] != 0).sum()))
    assert worst <= 100 * tol


def test_global_tiles_refuse_beta_or_z_off_a_16_byte_boundary(pkg, orc):
    """The FP32 global-tile worker reads and reduces beta and Z in aligned
    groups of four: arrays that do not start on a 16-byte boundary are refused
    on the host before any launch."""
    import torch
    w = ASYNC[3]
    X, D, _ = make_problem(w, 36)
    Xd, Dd = dev(X), dev(D)
    beta, dtd, lm = pkg.csc_init_beta(Xd, Dd)
    buf = torch.zeros(beta.numel() + 1, dtype=torch.float32, device=beta.device)
    Zoff = buf[1:].view(beta.shape)
    with pytest.raises(pkg.CscError) as e:
        pkg.csc_lgcd_solve(Xd, Dd, dtd, beta, 0.1 * lm, 1e-4, Z=Zoff, opts=pkg.default_opts(placement=2))
    assert e.value.status == pkg.CSC_ERR_INVALID


def test_global_tiles_with_more_than_64_subdomains_per_tile(pkg, orc):
    """Tiles of more than 64 sub-domains keep no dirty mask: they scan
    cyclically, pause after a quiet sweep and wake on any neighbour's
    notification.  Same bar as the other global-tile cases."""
    w = ASYNC[3]
    X, D, _ = make_problem(w, 37)
    lam = 0.1 * orc.lambda_max(X, D)
    tol = 1e-4
    ref = orc.lgcd(X, D, lam, tol)
    Xd, Dd = dev(X), dev(D)
    beta, dtd, _ = pkg.csc_init_beta(Xd, Dd)
    opts = pkg.default_opts(placement=2, sub=(2, 2), tile=(40, 46))
    Z, st = pkg.csc_lgcd_solve(Xd, Dd, dtd, beta, lam, tol, opts=opts)
    assert st["status"] == 0 and st["placement"] == 2 and st["workers"] > 4, st
    Zh = host(Z)
    f_ref = orc.objective(X, D, ref["Z"], lam)
    assert abs(orc.objective(X, D, Zh, lam) - f_ref) <= 1e-5 * abs(f_ref)
    assert kkt_fp64_within_bound(orc, X, D, Zh, lam, tol)[0]


def test_global_tiles_narrower_than_a_window_are_refused(pkg):
    """The soft-lock of a global-memory tile tests one strip of V(s0) per
    dimension, so asynchronous global tiles must be at least 2 L_i - 1 wide;
    a narrower tile is refused before any launch (the no-lock and automatic
    plans are unaffected)."""
    w = ASYNC[3]  # L = 8 x 8
    X, D, _ = make_problem(w, 38)
    Xd, Dd = dev(X), dev(D)
    beta, dtd, lmax = pkg.csc_init_beta(Xd, Dd)
    with pytest.raises(pkg.CscError) as e:
        pkg.csc_lgcd_solve(Xd, Dd, dtd, beta, 0.1 * lmax, 1e-4,
                           opts=pkg.default_opts(placement=2, tile=(14, 46)))
    assert e.value.status == pkg.CSC_ERR_INVALID
    Z, st = pkg.csc_lgcd_solve(Xd, Dd, dtd, beta, 0.1 * lmax, 1e-4,
                               opts=pkg.default_opts(placement=2, tile=(15, 46)))
    assert st["status"] == pkg.CSC_OK and st["placement"] == 2
