"""Pins for the FP64 oracle: facts fixed by the paper and by the mathematics,
checked through routes that do not share the oracle's code (explicit design
matrices built from library convolutions, FISTA, closed forms, finite
differences, hand-derived worked examples)."""
import json
import os

import numpy as np
import pytest
from scipy.optimize import minimize_scalar
from scipy.signal import convolve

from synthetic import Workload, make_problem
from tests._explicit import beta_explicit, cd_explicit, design_matrix, fista, lasso_objective

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

W1D = Workload("tiny1d", P=2, K=3, T=(40,), L=(5,), density=0.05, sigma=0.1)
W2D = Workload("tiny2d", P=2, K=2, T=(12, 11), L=(3, 4), density=0.06, sigma=0.1)


def _problem(w, seed):
    X, D, Z = make_problem(w, seed)
    return X.astype(np.float64), D.astype(np.float64), Z


@pytest.mark.parametrize("w", [W1D, W2D], ids=["1d", "2d"])
def test_beta_init_is_adjoint_of_model(orc, w):
    """beta_init = D~ * X equals A^T x for the explicit model matrix (Alg. 1 init)."""
    X, D, _ = _problem(w, 1)
    A = design_matrix(D, w.T)
    ref = (A.T @ X.ravel()).reshape((w.K,) + tuple(t - l + 1 for t, l in zip(w.T, w.L)))
    np.testing.assert_allclose(orc.beta_init(X, D), ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("w", [W1D, W2D], ids=["1d", "2d"])
def test_dtd_is_gram_of_model(orc, w):
    """<A_(k,s), A_(k2,s2)> = C[k][k2][s - s2] inside the window, 0 outside
    (the table of Eq. beta_update); C_kk[0] = ||D_k||^2; C symmetric."""
    X, D, _ = _problem(w, 2)
    A = design_matrix(D, w.T)
    G = A.T @ A
    Cm = orc.dtd(D, len(w.T))
    Tz = tuple(t - l + 1 for t, l in zip(w.T, w.L))
    pos = list(np.ndindex(*Tz))
    n = len(pos)
    L = w.L
    for a in range(0, w.K * n, 7):
        k, s = divmod(a, n)
        for b in range(w.K * n):
            k2, s2 = divmod(b, n)
            dlt = tuple(pos[s][i] - pos[s2][i] for i in range(len(L)))
            if all(abs(dlt[i]) < L[i] for i in range(len(L))):
                idx = tuple(dlt[i] + L[i] - 1 for i in range(len(L)))
                assert abs(G[a, b] - Cm[(k, k2) + idx]) < 1e-12
            else:
                assert abs(G[a, b]) < 1e-12
    nrm = orc.atom_sqnorms(D)
    center = tuple(l - 1 for l in L)
    for k in range(w.K):
        assert abs(Cm[(k, k) + center] - nrm[k]) < 1e-12
    flip = Cm[(slice(None), slice(None)) + (slice(None, None, -1),) * len(L)]
    np.testing.assert_allclose(Cm, flip.transpose((1, 0) + tuple(range(2, 2 + len(L)))),
                               atol=1e-12)


def test_single_coordinate_update_minimises(orc):
    """With one coordinate (T = L, K = 1) LGCD makes exactly the update
    Z' = ST(beta, lambda) / ||D||^2 (Eq. pb_coord, Prop. A.1), which must be
    the minimiser of 1/2||X - z D||^2 + lambda |z| found by a scalar search."""
    rng = np.random.default_rng(3)
    for trial in range(20):
        D = rng.standard_normal((1, 2, 6)) * rng.uniform(0.3, 2.0)
        X = rng.standard_normal((2, 6)) * 3
        lam = float(rng.uniform(0.0, 4.0))
        out = orc.lgcd(X, D, lam, 1e-14)
        z = out["Z"].ravel()[0]
        f = lambda u: 0.5 * np.sum((X - u * D[0]) ** 2) + lam * abs(u)
        res = minimize_scalar(f, bracket=(-50, 50), tol=1e-14)
        assert f(z) <= f(res.x) + 1e-10
        assert abs(z - res.x) < 1e-6
        grid = np.linspace(z - 1, z + 1, 4001)
        assert f(z) <= min(f(u) for u in grid) + 1e-12


@pytest.mark.parametrize("w", [W1D, W2D], ids=["1d", "2d"])
def test_zero_solution_at_lambda_max(orc, w):
    """Z = 0 is optimal iff lambda >= lambda_max = ||X * D~||_inf (Section 2)."""
    X, D, _ = _problem(w, 4)
    lmax = orc.lambda_max(X, D)
    A = design_matrix(D, w.T)
    assert abs(lmax - np.max(np.abs(A.T @ X.ravel()))) < 1e-12
    out = orc.lgcd(X, D, lmax, 1e-12)
    assert out["n_updates"] == 0 and np.all(out["Z"] == 0)
    out = orc.lgcd(X, D, lmax * (1 - 1e-6), 1e-12)
    assert out["n_updates"] >= 1 and np.count_nonzero(out["Z"]) >= 1


@pytest.mark.parametrize("w", [W1D, W2D], ids=["1d", "2d"])
@pytest.mark.parametrize("reg", [0.1, 0.5])
def test_lgcd_reaches_fista_optimum(orc, w, reg):
    """LGCD run to a tight tolerance reaches the LASSO optimum that FISTA on the
    explicit matrix finds (Eq. csc is a LASSO with a Toeplitz design)."""
    X, D, _ = _problem(w, 5)
    lam = reg * orc.lambda_max(X, D)
    A = design_matrix(D, w.T)
    x = X.ravel()
    z_f = fista(A, x, lam)
    out = orc.lgcd(X, D, lam, 1e-11)
    assert out["status"] == 0
    f_l = lasso_objective(A, x, out["Z"].ravel(), lam)
    f_f = lasso_objective(A, x, z_f, lam)
    assert abs(f_l - f_f) <= 1e-9 * abs(f_f)
    assert abs(orc.objective(X, D, out["Z"], lam) - f_l) <= 1e-10 * abs(f_l)


@pytest.mark.parametrize("w", [W1D, W2D], ids=["1d", "2d"])
def test_incremental_beta_matches_definition(orc, w):
    """The beta maintained by Eq. beta_update equals the definition of beta
    recomputed from scratch (Section 3); so does orc.beta_from_Z."""
    X, D, _ = _problem(w, 6)
    lam = 0.1 * orc.lambda_max(X, D)
    out = orc.lgcd(X, D, lam, 1e-6)
    A = design_matrix(D, w.T)
    ref = beta_explicit(A, X.ravel(), out["Z"].ravel()).reshape(out["beta"].shape)
    np.testing.assert_allclose(out["beta"], ref, rtol=0, atol=1e-11)
    np.testing.assert_allclose(orc.beta_from_Z(X, D, out["Z"]), ref, rtol=0, atol=1e-11)


@pytest.mark.parametrize("w", [W1D, W2D], ids=["1d", "2d"])
def test_cost_decrease_is_prop_a1(orc, w):
    """Every LGCD update lowers the cost by exactly the Delta E of Prop. A.1,
    and the recorded beta is the definition of beta at that state."""
    X, D, _ = _problem(w, 7)
    lam = 0.1 * orc.lambda_max(X, D)
    out = orc.lgcd(X, D, lam, 1e-8, trace_cap=400)
    tr = out["trace"]
    A = design_matrix(D, w.T)
    x = X.ravel()
    nrm = orc.atom_sqnorms(D)
    nz = int(np.prod(out["Z"].shape[1:]))
    z = np.zeros(A.shape[1])
    f = lasso_objective(A, x, z, lam)
    assert len(tr["k0"]) >= 20
    for k0, s0, zo, zn, b in zip(tr["k0"], tr["s0"], tr["z_old"], tr["z_new"], tr["beta"]):
        c = int(k0) * nz + int(s0)
        assert z[c] == zo
        assert abs(beta_explicit(A, x, z)[c] - b) < 1e-10
        dE = nrm[k0] / 2 * (zo ** 2 - zn ** 2) - b * (zo - zn) + lam * (abs(zo) - abs(zn))
        z[c] = zn
        f_new = lasso_objective(A, x, z, lam)
        assert abs((f - f_new) - dE) <= 1e-10 * max(1.0, abs(f))
        # the exact coordinate minimiser lowers the cost by at least ||D||^2/2 dZ^2
        assert dE >= 0.5 * nrm[k0] * (zn - zo) ** 2 - 1e-13
        f = f_new


@pytest.mark.parametrize("w", [W1D, W2D], ids=["1d", "2d"])
def test_final_kkt_below_tolerance(orc, w):
    """At the end of Alg. 1 max |dZ| < eps with beta recomputed from scratch."""
    X, D, _ = _problem(w, 8)
    lam = 0.1 * orc.lambda_max(X, D)
    eps = 1e-4
    out = orc.lgcd(X, D, lam, eps)
    A = design_matrix(D, w.T)
    b = beta_explicit(A, X.ravel(), out["Z"].ravel())
    nrm = (A * A).sum(axis=0)
    kkt = np.max(np.abs(np.sign(b) * np.maximum(np.abs(b) - lam, 0) / nrm - out["Z"].ravel()))
    assert kkt < eps
    assert orc.kkt(X, D, out["Z"], lam) < eps


def test_L1_K1_closed_form(orc):
    """With |Theta| = 1 and K = 1 the problem separates per position:
    Z[s] = ST(sum_p D_p X_p[s], lambda) / ||D||^2."""
    rng = np.random.default_rng(9)
    X = rng.standard_normal((3, 7, 9))
    D = rng.standard_normal((1, 3, 1, 1))
    lam = 0.7
    out = orc.lgcd(X, D, lam, 1e-14)
    b = np.einsum("p,pij->ij", D[0, :, 0, 0], X)
    ref = np.sign(b) * np.maximum(np.abs(b) - lam, 0) / np.sum(D ** 2)
    np.testing.assert_allclose(out["Z"][0], ref, rtol=0, atol=1e-13)


def _blocks(K, Tz, sub):
    """Column blocks of the explicit matrix for box sub-domains of side ``sub``,
    row-major, columns ordered by (position, k)."""
    n = int(np.prod(Tz))
    grid = [range(0, t, s) for t, s in zip(Tz, sub)]
    blocks = []
    for origin in np.ndindex(*[len(g) for g in grid]):
        lo = [grid[i][origin[i]] for i in range(len(Tz))]
        hi = [min(lo[i] + sub[i], Tz[i]) for i in range(len(Tz))]
        cols = []
        for pos in np.ndindex(*[hi[i] - lo[i] for i in range(len(Tz))]):
            s = int(np.ravel_multi_index(tuple(lo[i] + pos[i] for i in range(len(Tz))), Tz))
            cols += [k * n + s for k in range(K)]
        blocks.append(np.array(cols))
    return blocks


@pytest.mark.parametrize("w", [W1D, W2D], ids=["1d", "2d"])
@pytest.mark.parametrize("kind", ["cyclic", "greedy", "lgcd"])
def test_selection_reductions(orc, w, kind):
    """|C_m| = 1 gives cyclic CD, M = 1 gives greedy CD, and the default
    sub-domains of side 2L give LGCD (Section 3), replayed on the explicit matrix."""
    X, D, _ = _problem(w, 10)
    lam = 0.2 * orc.lambda_max(X, D)
    Tz = tuple(t - l + 1 for t, l in zip(w.T, w.L))
    sub = {"cyclic": (1,) * len(Tz), "greedy": Tz,
           "lgcd": tuple(2 * l for l in w.L)}[kind]
    out = orc.lgcd(X, D, lam, 1e-7, sub=sub)
    A = design_matrix(D, w.T)
    z, nupd = cd_explicit(A, X.ravel(), lam, 1e-7, _blocks(w.K, Tz, sub))
    assert nupd == out["n_updates"]
    np.testing.assert_allclose(out["Z"].ravel(), z, rtol=0, atol=1e-11)


@pytest.mark.parametrize("w", [W1D, W2D], ids=["1d", "2d"])
def test_interference_prop_a2(orc, w):
    """Simultaneous updates change the cost by sum Delta E_w minus the pairwise
    interference C[k_w][k_w'][s_w - s_w'] dZ_w dZ_w' (Prop. A.2, each pair once)."""
    X, D, _ = _problem(w, 11)
    A = design_matrix(D, w.T)
    x = X.ravel()
    Cm = orc.dtd(D, len(w.T))
    Tz = tuple(t - l + 1 for t, l in zip(w.T, w.L))
    n = int(np.prod(Tz))
    rng = np.random.default_rng(0)
    lam = 0.3
    for trial in range(30):
        z = np.where(rng.random(A.shape[1]) < 0.1, rng.standard_normal(A.shape[1]), 0.0)
        W = int(rng.integers(2, 4))
        center = np.array([rng.integers(0, t) for t in Tz])
        picks = []
        while len(picks) < W:
            s = tuple(int(np.clip(center[i] + rng.integers(-w.L[i] + 1, w.L[i]), 0, Tz[i] - 1))
                      for i in range(len(Tz)))
            k = int(rng.integers(0, w.K))
            c = k * n + int(np.ravel_multi_index(s, Tz))
            if c not in [p[2] for p in picks]:
                picks.append((k, s, c, float(rng.standard_normal())))
        f0 = lasso_objective(A, x, z, lam)
        single = 0.0
        for k, s, c, dz in picks:
            z1 = z.copy()
            z1[c] += dz
            single += f0 - lasso_objective(A, x, z1, lam)
        zall = z.copy()
        for k, s, c, dz in picks:
            zall[c] += dz
        total = f0 - lasso_objective(A, x, zall, lam)
        inter = 0.0
        for a in range(W):
            for b in range(a + 1, W):
                ka, sa, _, da = picks[a]
                kb, sb, _, db = picks[b]
                dl = tuple(sa[i] - sb[i] for i in range(len(Tz)))
                if all(abs(dl[i]) < w.L[i] for i in range(len(Tz))):
                    inter += Cm[(ka, kb) + tuple(dl[i] + w.L[i] - 1 for i in range(len(Tz)))] * da * db
        assert abs(total - (single - inter)) < 1e-10 * max(1.0, abs(f0))


@pytest.mark.parametrize("w", [W1D, W2D], ids=["1d", "2d"])
def test_phased_single_tile_is_alg1(orc, w):
    """The tiled checkerboard schedule with one tile is exactly Alg. 1."""
    X, D, _ = _problem(w, 12)
    lam = 0.1 * orc.lambda_max(X, D)
    a = orc.lgcd(X, D, lam, 1e-6)
    Tz = tuple(t - l + 1 for t, l in zip(w.T, w.L))
    b = orc.lgcd(X, D, lam, 1e-6, tile=Tz)
    assert a["n_updates"] == b["n_updates"]
    assert np.array_equal(a["Z"], b["Z"])


@pytest.mark.parametrize("tile", [(8,), (12,), (17,)])
def test_phased_tiles_reach_optimum_1d(orc, tile):
    """The tiled schedule (workers S_w of Alg. 3) converges to the same LASSO
    optimum and ends with max |dZ| < eps on a fresh beta."""
    w = Workload("tiny1d_long", P=2, K=3, T=(70,), L=(4,), density=0.05, sigma=0.1)
    X, D, _ = _problem(w, 13)
    lam = 0.1 * orc.lambda_max(X, D)
    out = orc.lgcd(X, D, lam, 1e-11, tile=tile)
    A = design_matrix(D, w.T)
    f_f = lasso_objective(A, X.ravel(), fista(A, X.ravel(), lam), lam)
    assert abs(lasso_objective(A, X.ravel(), out["Z"].ravel(), lam) - f_f) <= 1e-9 * f_f
    assert orc.kkt(X, D, out["Z"], lam) < 1e-11


@pytest.mark.parametrize("tile", [(4, 4), (5, 6), (7, 3)])
def test_phased_tiles_reach_optimum_2d(orc, tile):
    X, D, _ = _problem(W2D, 14)
    lam = 0.1 * orc.lambda_max(X, D)
    out = orc.lgcd(X, D, lam, 1e-11, tile=tile)
    A = design_matrix(D, W2D.T)
    f_f = lasso_objective(A, X.ravel(), fista(A, X.ravel(), lam), lam)
    assert abs(lasso_objective(A, X.ravel(), out["Z"].ravel(), lam) - f_f) <= 1e-9 * f_f


def test_max_updates_reports_not_converged(orc):
    X, D, _ = _problem(W1D, 15)
    lam = 0.05 * orc.lambda_max(X, D)
    out = orc.lgcd(X, D, lam, 1e-12, max_updates=3)
    assert out["status"] == 1 and out["n_updates"] == 3


# ----------------------------------------------------------------- dictionary

def _direct_F(X, D, Z):
    """1/2 ||X - Z * D||^2 with library convolutions (Eq. dict_update)."""
    K, P = D.shape[:2]
    rec = np.zeros_like(X)
    for k in range(K):
        for p in range(P):
            rec[p] += convolve(Z[k], D[k, p], mode="full")
    return 0.5 * float(np.sum((X - rec) ** 2))


@pytest.mark.parametrize("w", [W1D, W2D], ids=["1d", "2d"])
def test_stats_give_objective_and_gradient(orc, w):
    """F(D) from (phi, psi, ||X||^2) equals the direct objective, its gradient
    phi * D - psi matches central finite differences, and phi is symmetric
    phi_{k,k2}[d] = phi_{k2,k}[-d] (Section 4.2, Eq. phi)."""
    X, D, Z = _problem(w, 16)
    Z = Z.astype(np.float64)
    phi, psi = orc.phi_psi(Z, X, w.L)
    xs = float(np.sum(X ** 2))
    rng = np.random.default_rng(1)
    for _ in range(3):
        Dt = D + 0.3 * rng.standard_normal(D.shape)
        f = orc.dict_objective(phi, psi, xs, Dt)
        assert abs(f - _direct_F(X, Dt, Z)) <= 1e-10 * max(1.0, abs(f))
    g = orc.dict_grad(phi, psi, D)
    h = 1e-5
    for idx in list(np.ndindex(*D.shape))[::5]:
        Dp, Dm = D.copy(), D.copy()
        Dp[idx] += h
        Dm[idx] -= h
        fd = (_direct_F(X, Dp, Z) - _direct_F(X, Dm, Z)) / (2 * h)
        assert abs(fd - g[idx]) < 1e-5 * max(1.0, abs(g[idx]))
    nd = len(w.L)
    flip = phi[(slice(None), slice(None)) + (slice(None, None, -1),) * nd]
    np.testing.assert_allclose(phi, flip.transpose((1, 0) + tuple(range(2, 2 + nd))), atol=1e-12)


@pytest.mark.parametrize("w", [W1D, W2D], ids=["1d", "2d"])
def test_pgd_armijo_monotone_feasible_optimal(orc, w):
    """PGD with Armijo (Alg. 2): F decreases, every atom stays in the unit ball,
    and at convergence the projected-gradient KKT conditions of Eq.
    dict_update hold: per atom either ||D_k|| < 1 and grad_k = 0, or
    ||D_k|| = 1 and grad_k = -mu_k D_k with mu_k >= 0."""
    X, D0, Z = _problem(w, 17)
    rng = np.random.default_rng(2)
    D0 = D0 + 0.5 * rng.standard_normal(D0.shape)
    phi, psi = orc.phi_psi(Z, X, w.L)
    xs = float(np.sum(X ** 2))
    prev = orc.dict_objective(phi, psi, xs, D0)
    for it in range(1, 6):
        D, f, n = orc.pgd_armijo(phi, psi, xs, D0, max_iter=it, tol=0.0)
        assert f <= prev + 1e-9 * abs(prev)
        prev = f
        nr = np.sqrt((D.reshape(w.K, -1) ** 2).sum(1))
        assert np.all(nr <= 1 + 1e-12)
    D, f, n = orc.pgd_armijo(phi, psi, xs, D0, max_iter=20000, tol=1e-13)
    g = orc.dict_grad(phi, psi, D).reshape(w.K, -1)
    Df = D.reshape(w.K, -1)
    for k in range(w.K):
        nr = np.linalg.norm(Df[k])
        gn = np.linalg.norm(g[k])
        if nr < 1 - 1e-6:
            assert gn < 1e-6 * max(1.0, np.abs(psi).max())
        else:
            mu = -float(g[k] @ Df[k])
            assert mu >= -1e-8
            assert np.linalg.norm(g[k] + mu * Df[k]) < 1e-6 * max(1.0, gn)


# ------------------------------------------------------- hand-derived examples

def test_golden_worked_examples(orc):
    """Small examples worked by hand from Eq. pb_coord / Eq. beta_update."""
    with open(os.path.join(GOLDEN, "worked_examples.json")) as fh:
        cases = json.load(fh)["cases"]
    for c in cases:
        X = np.array(c["X"], dtype=np.float64)
        D = np.array(c["D"], dtype=np.float64)
        out = orc.lgcd(X, D, c["lambda"], c["eps"])
        np.testing.assert_allclose(out["Z"], np.array(c["Z"]), rtol=0, atol=1e-12)
        np.testing.assert_allclose(out["beta"], np.array(c["beta_final"]), rtol=0, atol=1e-12)
        assert out["n_updates"] == c["n_updates"]
        assert abs(orc.objective(X, D, out["Z"], c["lambda"]) - c["objective"]) < 1e-12
        assert abs(orc.lambda_max(X, D) - c["lambda_max"]) < 1e-12


@pytest.mark.parametrize("w", [W1D, W2D], ids=["1d", "2d"])
def test_sampled_routines_match_explicit_model(orc, w):
    """beta at listed coordinates, beta from Z at listed coordinates and the
    zero-skipping objective agree with the explicit design matrix."""
    X, D, Z = _problem(w, 18)
    Z = Z.astype(np.float64)
    A = design_matrix(D, w.T)
    Tz = tuple(t - l + 1 for t, l in zip(w.T, w.L))
    n = int(np.prod(Tz))
    rng = np.random.default_rng(4)
    ks = rng.integers(0, w.K, 40)
    ss = rng.integers(0, n, 40)
    cols = ks * n + ss
    np.testing.assert_allclose(orc.beta_at(X, D, ks, ss), (A.T @ X.ravel())[cols], rtol=0, atol=1e-12)
    bz = beta_explicit(A, X.ravel(), Z.ravel())
    np.testing.assert_allclose(orc.beta_from_Z_at(X, D, Z, ks, ss), bz[cols], rtol=0, atol=1e-11)
    lam = 0.3
    f = lasso_objective(A, X.ravel(), Z.ravel(), lam)
    assert abs(orc.objective_sparse(X, D, Z, lam) - f) <= 1e-12 * f
    # the same objective from the list of nonzeros
    nz = np.nonzero(Z)
    k, i, j = (nz[0], np.zeros_like(nz[1]), nz[1]) if Z.ndim == 2 else nz
    assert abs(orc.objective_nz(X, D, k, i, j, Z[nz], lam) - f) <= 1e-12 * f


@pytest.mark.parametrize("w", [W1D, W2D], ids=["1d", "2d"])
def test_phi_psi_from_nonzeros_match_correlations(orc, w):
    """phi and psi from a list of nonzeros (the routine used on activation
    maps too large for the dense one) equal the correlations of their
    definitions (Eq. phi), computed here with scipy's correlate, and the dense
    routine, whatever the order of the list."""
    from scipy.signal import correlate
    X, D, Z = _problem(w, 23)
    Z = Z.astype(np.float64)
    if not Z.any():
        Z.reshape(-1)[::7] = 0.5
    L = w.L
    K, P = w.K, w.P
    Zs = Z if Z.ndim == 3 else Z[:, None, :]
    Xs = X if X.ndim == 3 else X[:, None, :]
    L0, L1 = (1, L[0]) if len(L) == 1 else L
    N0, N1 = Zs.shape[1:]
    phi_ref = np.zeros((K, K, 2 * L0 - 1, 2 * L1 - 1))
    for k in range(K):
        for k2 in range(K):
            c = correlate(Zs[k2], Zs[k], mode="full")  # c[lag + N - 1] = sum_s Z_k[s] Z_k2[s + lag]
            phi_ref[k, k2] = c[N0 - 1 - (L0 - 1):N0 - 1 + L0, N1 - 1 - (L1 - 1):N1 - 1 + L1]
    psi_ref = np.zeros((K, P, L0, L1))
    for k in range(K):
        for p in range(P):
            psi_ref[k, p] = correlate(Xs[p], Zs[k], mode="valid")  # sum_s Z_k[s] X_p[s + tau]
    nz = np.nonzero(Zs)
    perm = np.random.default_rng(3).permutation(len(nz[0]))
    k, i, j = (a[perm] for a in nz)
    phi, psi = orc.phi_psi_nz(X, L, K, k, i, j, Zs[nz][perm])
    if len(L) == 1:
        phi_ref, psi_ref = phi_ref[:, :, 0, :], psi_ref[:, :, 0, :]
    np.testing.assert_allclose(phi, phi_ref, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(psi, psi_ref, rtol=1e-12, atol=1e-12)
    pd, sd = orc.phi_psi(Z, X, L)
    np.testing.assert_allclose(phi, pd, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(psi, sd, rtol=1e-12, atol=1e-13)
    with pytest.raises(ValueError):
        orc.phi_psi_nz(X, L, K, [0], [0], [N1], [1.0])


@pytest.mark.parametrize("d0", [0.4, 1.0])
@pytest.mark.parametrize("dims", [1, 2], ids=["1d", "2d"])
def test_cdl_loop_one_tap_closed_form(orc, dims, d0):
    """Alg. 2 with one atom of a single tap (L = 1): the CSC step has the
    closed form Z = ST(d X, lambda) / d^2 (coordinates decouple) and the
    dictionary step minimises 1/2 ||X - d Z||^2 over |d| <= 1, so
    d' = clip(<X, Z> / ||Z||^2, -1, 1).  Two outer iterations; from d = 1 the
    unconstrained minimiser lies outside the unit ball (projection active)."""
    rng = np.random.default_rng(21)
    shape = (1, 300) if dims == 1 else (1, 17, 19)
    X = rng.standard_normal(shape)
    D0 = np.full((1, 1) + (1,) * dims, d0)
    reg = 0.3
    D, Z, trace = orc.cdl(X, D0, reg, 1e-10, 2, pgd_max_iter=200, pgd_tol=1e-14)
    x = X.reshape(-1)
    d = d0
    lam = reg * abs(d) * np.abs(x).max()
    costs = []
    for _ in range(2):
        z = np.sign(d * x) * np.maximum(np.abs(d * x) - lam, 0.0) / d ** 2
        c_csc = 0.5 * ((x - d * z) ** 2).sum() + lam * np.abs(z).sum()
        d = float(np.clip(x @ z / (z @ z), -1.0, 1.0))
        c_dict = 0.5 * ((x - d * z) ** 2).sum() + lam * np.abs(z).sum()
        costs.append((c_csc, c_dict))
    assert abs(float(D.reshape(-1)[0]) - d) <= 1e-9
    np.testing.assert_allclose(Z.reshape(-1), z, rtol=0, atol=1e-9)
    np.testing.assert_allclose(np.asarray(trace), np.asarray(costs), rtol=1e-10, atol=0)


# ---------------------------------------------------------------- RCD
def _rcd_problem():
    from synthetic import Workload, make_problem
    w = Workload("rcd_pin", P=2, K=3, T=(120,), L=(8,), density=0.03, sigma=0.1)
    X, D, _ = make_problem(w, 17)
    return X, D


def test_rcd_step_is_the_coordinate_minimiser(orc):
    """One step of orc.rcd lands at the minimum of the objective along that
    coordinate, found by a dense grid search of the objective itself."""
    X, D = _rcd_problem()
    lam = 0.1 * orc.lambda_max(X, D)
    rng = np.random.default_rng(3)
    Z = np.zeros((3, 113))
    Z[rng.integers(0, 3, 6), rng.integers(0, 113, 6)] = rng.standard_normal(6)
    beta = orc.beta_from_Z(X, D, Z)
    for c in (5, 120, 300):
        k, s = divmod(c, 113)
        Z1, _, _ = orc.rcd(X, D, lam, [c], Z=Z, beta=beta)
        z_star = Z1[k, s]
        grid = z_star + np.linspace(-0.05, 0.05, 201)
        vals = []
        for zg in grid:
            Zg = Z.copy()
            Zg[k, s] = zg
            vals.append(orc.objective(X, D, Zg, lam))
        assert abs(grid[int(np.argmin(vals))] - z_star) <= 0.0005 + 1e-12
        assert orc.objective(X, D, Z1, lam) <= min(vals) + 1e-12


def test_rcd_objective_never_increases_and_beta_stays_consistent(orc):
    X, D = _rcd_problem()
    lam = 0.1 * orc.lambda_max(X, D)
    coords = np.random.default_rng(5).integers(0, 3 * 113, 2000).astype(np.uint32)
    Z, beta = None, None
    prev = np.inf
    for chunk in np.array_split(coords, 20):
        Z, beta, _ = orc.rcd(X, D, lam, chunk, Z=Z, beta=beta)
        f = orc.objective(X, D, Z, lam)
        assert f <= prev * (1 + 1e-12)
        prev = f
    assert np.abs(beta - orc.beta_from_Z(X, D, Z)).max() < 1e-9


def test_rcd_cyclic_order_reaches_the_greedy_solution(orc):
    """The LASSO minimiser is unique: cyclic CD (RCD with the sequential
    order) and greedy CD (LGCD with one sub-domain) reach the same objective,
    and both pass the KKT test."""
    X, D = _rcd_problem()
    lam = 0.1 * orc.lambda_max(X, D)
    order = np.arange(3 * 113, dtype=np.uint32)
    Z, beta = None, None
    for _ in range(400):
        Z, beta, changed = orc.rcd(X, D, lam, order, Z=Z, beta=beta)
        if orc.kkt(X, D, Z, lam) < 1e-10:
            break
    g = orc.lgcd(X, D, lam, 1e-10, sub=(113,))
    f_c, f_g = orc.objective(X, D, Z, lam), orc.objective(X, D, g["Z"], lam)
    assert abs(f_c - f_g) <= 1e-9 * abs(f_g)
    assert orc.kkt(X, D, Z, lam) < 1e-8 and orc.kkt(X, D, g["Z"], lam) < 1e-8


def test_rcd_rejects_indices_outside_the_domain(orc):
    X, D = _rcd_problem()
    with pytest.raises(ValueError):
        orc.rcd(X, D, 0.1, [3 * 113])
