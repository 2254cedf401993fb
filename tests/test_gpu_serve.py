"""The continuous-batching server (paper_1901_09235_gb300.serve).

Requests of the served family (3 channels, 16 resident atoms of 12 x 12,
lambda = 0.1 lambda_max each, image sides log-uniform) arrive as a Poisson
stream while earlier ones are on the GPU.

* Each result is the same served alone, served in the mix, and from the plain
  single-solve call: objective within 1e-5 relative, KKT below tol on a beta
  recomputed from scratch.
* Admission keeps the device footprint of the admitted requests within the
  HBM budget; requests that do not fit wait and are admitted when memory
  frees up.
* The split-bf16 beta-init on the tensor cores gives the same results."""
import numpy as np
import pytest

from synthetic import SERVED_ATOMS, Workload, make_dictionary, make_problem, poisson_arrivals, served_sizes
from tests._gpu import dev

pytestmark = pytest.mark.gpu

P, K, L = SERVED_ATOMS["P"], SERVED_ATOMS["K"], SERVED_ATOMS["L"]
TOL = 1e-4
REL = 1e-5


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


@pytest.fixture(scope="module")
def served():
    import torch
    D = make_dictionary(np.random.default_rng(21), K, P, L)
    sides = served_sizes(16, seed=5, lo=64, hi=384)
    rng = np.random.default_rng(6)
    imgs = []
    for i, s in enumerate(sides):
        s1 = max(48, int(s * rng.uniform(0.7, 1.3)))
        w = Workload(f"served{s}x{s1}", P, K, (int(s), s1), L, SERVED_ATOMS["density"], SERVED_ATOMS["sigma"])
        imgs.append(torch.from_numpy(make_problem(w, 200 + i, D=D)[0]).pin_memory())
    return D, imgs


def _requests(serve_mod, imgs, arrivals):
    return [serve_mod.Request(X=x, arrival=float(a)) for x, a in zip(imgs, arrivals)]


def _check_done(reqs):
    for r in reqs:
        assert r.status == 0, (r.status, tuple(r.X.shape))
        assert r.max_dz < TOL


def test_served_same_alone_and_in_the_mix(pkg, served):
    from paper_1901_09235_gb300 import serve
    D, imgs = served
    Dd = dev(D)
    arr = poisson_arrivals(len(imgs), rate_hz=400.0, seed=8)
    with serve.Server(Dd, hbm_budget=1 << 30, max_side=(512, 512), run_seconds=120.0) as srv:
        mix = srv.serve(_requests(serve, imgs, arr))
        alone = [srv.serve(_requests(serve, [x], [0.0]))[0] for x in imgs]
    _check_done(mix)
    _check_done(alone)
    # the mix overlapped: some request was admitted while others were in flight
    spans = sorted((r.t_admit, r.t_done) for r in mix)
    assert any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))
    for i, (a, m) in enumerate(zip(alone, mix)):
        assert abs(m.objective - a.objective) <= REL * abs(a.objective), (i, m.objective, a.objective)
        # the plain single-solve path on the same image
        X = dev(imgs[i].numpy())
        beta, dtd, lm = pkg.csc_init_beta(X, Dd)
        assert abs(0.1 * lm - a.lam) <= 1e-12 * a.lam
        Z, st = pkg.csc_lgcd_solve(X, Dd, dtd, beta, a.lam, TOL)
        assert st["status"] == 0
        obj = pkg.csc_objective(X, Dd, Z, float(np.float32(a.lam)))
        assert abs(a.objective - obj) <= REL * abs(obj), (i, a.objective, obj)


def test_admission_keeps_within_hbm_budget(pkg, served):
    from paper_1901_09235_gb300 import serve
    D, imgs = served
    Dd = dev(D)
    fps = [serve.footprint(tuple(D.shape), tuple(x.shape)) for x in imgs]
    budget = 2 * max(fps)
    with serve.Server(Dd, hbm_budget=budget, max_side=(512, 512), run_seconds=120.0) as srv:
        reqs = srv.serve(_requests(serve, imgs, np.zeros(len(imgs))))
        peak = srv.arena.peak
        assert srv.arena.used == 0
    _check_done(reqs)
    assert peak <= budget
    # everything arrived at once and could not all fit: the later ones waited
    # for earlier ones to finish
    assert sum(fps) > budget
    waited = [r for r in reqs if r.t_admit > min(q.t_done for q in reqs)]
    assert waited


def test_served_bf16x3_same_results(pkg, served):
    from paper_1901_09235_gb300 import serve
    D, imgs = served
    Dd = dev(D)
    arr = poisson_arrivals(len(imgs), rate_hz=400.0, seed=9)
    with serve.Server(Dd, hbm_budget=1 << 30, max_side=(512, 512), run_seconds=120.0) as srv:
        ref = srv.serve(_requests(serve, imgs, arr))
    with serve.Server(Dd, hbm_budget=1 << 30, max_side=(512, 512), precision="bf16x3",
                      run_seconds=120.0) as srv:
        mp = srv.serve(_requests(serve, imgs, arr))
    _check_done(ref)
    _check_done(mp)
    for a, b in zip(ref, mp):
        assert abs(a.objective - b.objective) <= REL * abs(a.objective)


def test_autotuned_options_same_results(pkg, served):
    """The autotuner picks a sub-domain side and stop margin per size class
    (here the two smallest classes); serving with its table changes the
    schedule, not the results."""
    from paper_1901_09235_gb300 import autotune, serve
    from synthetic import make_image_device
    D, imgs = served
    Dd = dev(D)

    def make_image(side, seed):
        w = Workload("tune", P, K, (side, side), L, SERVED_ATOMS["density"], SERVED_ATOMS["sigma"])
        return make_image_device(w, 900 + seed, D)

    table = autotune.tune(Dd, make_image, classes=[0, 1], reps=1)
    assert set(table) == {"0", "1"}
    for e in table.values():
        assert e["sub"] in autotune.sub_candidates(L[0]) and 0 < e["stop_margin"] <= 1
        assert e["ms"] == min(e["tried"].values())
    small = [x for x in imgs if max(x.shape[1:]) <= 192]
    arr = np.zeros(len(small))
    with serve.Server(Dd, hbm_budget=1 << 30, max_side=(512, 512), run_seconds=120.0) as srv:
        ref = srv.serve(_requests(serve, small, arr))
    with serve.Server(Dd, hbm_budget=1 << 30, max_side=(512, 512), run_seconds=120.0, tuning=table) as srv:
        tuned = srv.serve(_requests(serve, small, arr))
    _check_done(ref)
    _check_done(tuned)
    for a, b in zip(ref, tuned):
        assert abs(a.objective - b.objective) <= REL * abs(a.objective)


def test_served_result_copied_out_and_budget_enforced(pkg, served):
    """Z_out receives the solution whose objective the server reports; a
    request that cannot fit the HBM budget is refused before serving."""
    import torch
    from paper_1901_09235_gb300 import serve
    D, imgs = served
    Dd = dev(D)
    x = imgs[0]
    zs = (K, x.shape[1] - L[0] + 1, x.shape[2] - L[1] + 1)
    z_out = torch.empty(zs, dtype=torch.float32, pin_memory=True)
    with serve.Server(Dd, hbm_budget=1 << 28, max_side=(512, 512), run_seconds=60.0) as srv:
        (r,) = srv.serve([serve.Request(X=x, Z_out=z_out)])
    assert r.status == 0
    obj = pkg.csc_objective(dev(x.numpy()), Dd, z_out.cuda(), float(np.float32(r.lam)))
    assert abs(obj - r.objective) <= 1e-12 * abs(obj) + 1e-12
    small = serve.footprint(tuple(D.shape), tuple(x.shape))
    with serve.Server(Dd, hbm_budget=small - 256, max_side=(512, 512), run_seconds=60.0) as srv:
        with pytest.raises(ValueError):
            srv.serve([serve.Request(X=x)])
