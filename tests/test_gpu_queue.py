"""Many solves of uneven size in one persistent launch (the csc_queue_* calls).

* Small images of the served family (3 channels, 16 atoms of 12 x 12) solved
  through the queue match the oracle's LGCD objective and satisfy the KKT test
  on a beta recomputed from scratch.
* A mix of image sizes: each image's result is the same when it is the only
  job in flight, when it runs beside all the others, and from the plain
  single-solve call (objective within 1e-5 relative, KKT below tol).
* Jobs submitted while a large job runs start on the CTAs it leaves free and
  complete before it.
* Host-side limits (job table, control slots) answer with an error code."""
import numpy as np
import pytest

from synthetic import SERVED_ATOMS, Workload, make_dictionary, make_problem, served_sizes
from tests._gpu import dev, host

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


def _atoms(seed=7):
    return make_dictionary(np.random.default_rng(seed), K, P, L)


def _image(side0, side1, seed, D):
    w = Workload(f"served{side0}x{side1}", P, K, (int(side0), int(side1)), L,
                 SERVED_ATOMS["density"], SERVED_ATOMS["sigma"])
    X, _, _ = make_problem(w, seed, D=D)
    return X


class _Req:
    """One image and its device state."""

    def __init__(self, pkg, X, Dd):
        import torch
        self.X = dev(X)
        self.beta, self.dtd, lm = pkg.csc_init_beta(self.X, Dd)
        self.lam = 0.1 * lm
        self.Z = torch.empty_like(self.beta)
        self.ws = pkg.workspace(pkg.make_shape(tuple(self.X.shape), tuple(Dd.shape)))


def _finish(pkg, q, r, Dd, job, max_rounds=4):
    """Wait for a job; refresh beta; resubmit warm until the KKT test holds."""
    st = q.wait(job)
    for _ in range(max_rounds):
        assert st["status"] == 0, st
        _, mdz, obj = pkg.csc_refresh_beta(r.X, Dd, r.Z, r.lam, beta=r.beta, ws=r.ws)
        if mdz < TOL:
            return obj, mdz
        st = q.wait(q.submit(r.beta, r.Z, r.lam, TOL, warm_start=True))
    raise AssertionError(f"KKT {mdz} >= {TOL} after {max_rounds} refresh rounds")


def test_queue_small_images_match_oracle(pkg, orc):
    D = _atoms()
    Dd = dev(D)
    imgs = [_image(40, 40, 1, D), _image(35, 58, 2, D), _image(64, 47, 3, D)]
    reqs = [_Req(pkg, X, Dd) for X in imgs]
    with pkg.Queue(Dd, reqs[0].dtd, max_jobs=64, ctl_slots=16, run_seconds=60.0) as q:
        jobs = [q.submit(r.beta, r.Z, r.lam, TOL) for r in reqs]
        res = [_finish(pkg, q, r, Dd, j) for r, j in zip(reqs, jobs)]
    for X, r, (obj, mdz) in zip(imgs, reqs, res):
        ref = orc.lgcd(X, D, r.lam, TOL)
        obj_ref = orc.objective(X, D, ref["Z"], r.lam)
        obj_gpu = orc.objective(X, D, host(r.Z), r.lam)
        assert abs(obj_gpu - obj_ref) <= REL * abs(obj_ref), (obj_gpu, obj_ref)
        # the refresh's objective: FP64 sums, lambda as passed (FP32)
        obj_l32 = orc.objective(X, D, host(r.Z), float(np.float32(r.lam)))
        assert abs(obj - obj_l32) <= 1e-12 * abs(obj_l32) + 1e-12
        assert orc.kkt(X, D, host(r.Z), r.lam) < TOL


def test_queue_same_alone_and_in_the_mix(pkg):
    import torch
    D = _atoms(11)
    Dd = dev(D)
    sides = served_sizes(10, seed=3, lo=64, hi=512)
    rng = np.random.default_rng(4)
    imgs = [_image(s, max(48, int(s * rng.uniform(0.6, 1.4))), 100 + i, D) for i, s in enumerate(sides)]
    alone, mixed = [_Req(pkg, X, Dd) for X in imgs], [_Req(pkg, X, Dd) for X in imgs]
    with pkg.Queue(Dd, alone[0].dtd, max_jobs=128, ctl_slots=32, run_seconds=120.0) as q:
        # alone: one job in flight at a time
        obj_alone = [_finish(pkg, q, r, Dd, q.submit(r.beta, r.Z, r.lam, TOL))[0] for r in alone]
        # in the mix: every job submitted before the first completes
        jobs = [q.submit(r.beta, r.Z, r.lam, TOL) for r in mixed]
        obj_mix = [_finish(pkg, q, r, Dd, j)[0] for r, j in zip(mixed, jobs)]
    for i, X in enumerate(imgs):
        r = alone[i]
        beta = pkg.csc_init_beta(r.X, Dd)[0]
        Z, st = pkg.csc_lgcd_solve(r.X, Dd, r.dtd, beta, r.lam, TOL)
        assert st["status"] == 0
        obj_single = pkg.csc_objective(r.X, Dd, Z, r.lam)
        assert abs(obj_alone[i] - obj_single) <= REL * abs(obj_single), (i, obj_alone[i], obj_single)
        assert abs(obj_mix[i] - obj_single) <= REL * abs(obj_single), (i, obj_mix[i], obj_single)
        assert abs(obj_mix[i] - obj_alone[i]) <= REL * abs(obj_alone[i])
    torch.cuda.synchronize()


def test_queue_admits_jobs_while_a_large_one_runs(pkg):
    D = _atoms(13)
    Dd = dev(D)
    big = _Req(pkg, _image(2048, 2048, 50, D), Dd)
    small = [_Req(pkg, _image(96, 96, 60 + i, D), Dd) for i in range(6)]
    with pkg.Queue(Dd, big.dtd, max_jobs=64, ctl_slots=16, run_seconds=120.0) as q:
        jb = q.submit(big.beta, big.Z, big.lam, TOL)
        js = [q.submit(r.beta, r.Z, r.lam, TOL) for r in small]
        done_small = [q.wait(j) for j in js]
        big_running = q.poll(jb) is None
        for r, j in zip(small, js):
            _finish(pkg, q, r, Dd, j)
        _finish(pkg, q, big, Dd, jb)
    assert all(s["status"] == 0 for s in done_small)
    # the big image takes at most 7/8 of the CTAs; the small ones run beside it
    assert big_running


def test_queue_limits(pkg):
    D = _atoms(17)
    Dd = dev(D)
    r = _Req(pkg, _image(48, 48, 70, D), Dd)
    import torch
    extra = [(torch.empty_like(r.beta), torch.empty_like(r.Z)) for _ in range(3)]
    for b, _ in extra:
        b.copy_(r.beta)
    with pkg.Queue(Dd, r.dtd, max_jobs=3, ctl_slots=2, run_seconds=60.0) as q:
        j0 = q.submit(r.beta, r.Z, r.lam, TOL)
        j1 = q.submit(extra[0][0], extra[0][1], r.lam, TOL)
        # both control slots are held until the jobs are polled
        with pytest.raises(pkg.CscError) as e:
            q.submit(extra[1][0], extra[1][1], r.lam, TOL)
        assert e.value.status == pkg.CSC_ERR_WORKSPACE
        q.wait(j0)
        q.wait(j1)
        q.wait(q.submit(extra[1][0], extra[1][1], r.lam, TOL))
        # the job table holds 3 jobs in total
        with pytest.raises(pkg.CscError) as e:
            q.submit(extra[2][0], extra[2][1], r.lam, TOL)
        assert e.value.status == pkg.CSC_ERR_WORKSPACE


def test_queue_degenerate_and_thin_images(pkg):
    """A 1 x 1 activation map (image = atom size), thin strips in both
    orientations and a small square, mixed in one queue: each matches the
    plain single solve."""
    D = _atoms(19)
    Dd = dev(D)
    shapes = [(12, 12), (13, 300), (400, 14), (30, 30), (12, 700)]
    reqs = [_Req(pkg, _image(s0, s1, 80 + i, D), Dd) for i, (s0, s1) in enumerate(shapes)]
    with pkg.Queue(Dd, reqs[0].dtd, max_jobs=64, ctl_slots=16, run_seconds=60.0) as q:
        jobs = [q.submit(r.beta, r.Z, r.lam, TOL) for r in reqs]
        objs = [_finish(pkg, q, r, Dd, j)[0] for r, j in zip(reqs, jobs)]
    for r, obj in zip(reqs, objs):
        beta, _, _ = pkg.csc_init_beta(r.X, Dd)
        Z, st = pkg.csc_lgcd_solve(r.X, Dd, r.dtd, beta, r.lam, TOL)
        assert st["status"] == 0
        ref = pkg.csc_objective(r.X, Dd, Z, float(np.float32(r.lam)))
        assert abs(obj - ref) <= REL * abs(ref) + 1e-9, (tuple(r.X.shape), obj, ref)


def test_queue_three_ctas_per_sm(pkg):
    """The denser grid (three CTAs per SM) with the FP32 beta-init and refresh
    beside it gives the same results as single solves; densities other than 2
    or 3 are refused."""
    D = _atoms(23)
    Dd = dev(D)
    reqs = [_Req(pkg, _image(s0, s1, 90 + i, D), Dd) for i, (s0, s1) in enumerate([(300, 260), (96, 128), (700, 650)])]
    with pkg.Queue(Dd, reqs[0].dtd, max_jobs=64, ctl_slots=16, run_seconds=60.0, ctas_per_sm=3) as q:
        jobs = [q.submit(r.beta, r.Z, r.lam, TOL) for r in reqs]
        # an FP32 beta-init beside the running queue (the refreshes below too)
        extra = _Req(pkg, _image(200, 200, 99, D), Dd)
        objs = [_finish(pkg, q, r, Dd, j)[0] for r, j in zip(reqs, jobs)]
        obj_x = _finish(pkg, q, extra, Dd, q.submit(extra.beta, extra.Z, extra.lam, TOL))[0]
    for r, obj in zip(reqs + [extra], objs + [obj_x]):
        beta, _, _ = pkg.csc_init_beta(r.X, Dd)
        Z, st = pkg.csc_lgcd_solve(r.X, Dd, r.dtd, beta, r.lam, TOL)
        ref = pkg.csc_objective(r.X, Dd, Z, float(np.float32(r.lam)))
        assert abs(obj - ref) <= REL * abs(ref)
    with pytest.raises(pkg.CscError) as e:
        pkg.Queue(Dd, reqs[0].dtd, max_jobs=4, ctl_slots=2, ctas_per_sm=5)
    assert e.value.status == pkg.CSC_ERR_INVALID


def test_dropped_queue_stops_its_kernel(pkg):
    """A queue that goes out of scope without close() ends its persistent
    kernel at once, not after run_seconds."""
    import gc
    import time
    D = _atoms()
    Dd = dev(D)
    r = _Req(pkg, _image(40, 40, 11, D), Dd)
    q = pkg.Queue(Dd, r.dtd, max_jobs=8, ctl_slots=4, run_seconds=30.0)
    st = q.wait(q.submit(r.beta, r.Z, r.lam, TOL))
    assert st["status"] == 0
    ks = q.kernel_stream
    del q
    gc.collect()
    t0 = time.monotonic()
    ks.synchronize()  # returns by run_seconds at the latest
    assert time.monotonic() - t0 < 5.0


def test_deferred_queue_drains_jobs_published_before_its_start(pkg, orc):
    """Jobs submitted to a queue made with start=False are all published
    before its kernel runs; start(drain=True) lets the kernel end by itself
    once they are done, so no host copy overlaps the kernel.  Results match
    the oracle; a submit after a draining start is refused."""
    import torch
    D = _atoms(9)
    Dd = dev(D)
    imgs = [_image(48, 40, 21, D), _image(33, 61, 22, D), _image(70, 70, 23, D)]
    reqs = [_Req(pkg, X, Dd) for X in imgs]
    rounds = [0] * len(reqs)
    pending = list(range(len(reqs)))
    warm = False
    while pending:
        q = pkg.Queue(Dd, reqs[0].dtd, max_jobs=16, ctl_slots=8, run_seconds=60.0, start=False)
        jobs = {i: q.submit(reqs[i].beta, reqs[i].Z, reqs[i].lam, TOL, warm_start=warm) for i in pending}
        q.start(drain=True)
        with pytest.raises(pkg.CscError) as e:
            q.submit(reqs[0].beta, reqs[0].Z, reqs[0].lam, TOL)
        assert e.value.status == pkg.CSC_ERR_INVALID
        stats = {i: q.wait(j) for i, j in jobs.items()}
        q.close()
        nxt = []
        for i in pending:
            assert stats[i]["status"] == 0, stats[i]
            r = reqs[i]
            _, mdz, _ = pkg.csc_refresh_beta(r.X, Dd, r.Z, r.lam, beta=r.beta, ws=r.ws)
            rounds[i] += 1
            if mdz >= TOL:
                assert rounds[i] < 4, (i, mdz)
                nxt.append(i)
        pending, warm = nxt, True
    torch.cuda.synchronize()
    for X, r in zip(imgs, reqs):
        ref = orc.lgcd(X, D, r.lam, TOL)
        f_ref = orc.objective(X, D, ref["Z"], r.lam)
        f = orc.objective(X, D, host(r.Z), r.lam)
        assert abs(f - f_ref) <= REL * abs(f_ref), (f, f_ref)


def test_deferred_queue_closed_without_start(pkg):
    D = _atoms(9)
    Dd = dev(D)
    r = _Req(pkg, _image(40, 40, 24, D), Dd)
    q = pkg.Queue(Dd, r.dtd, max_jobs=4, ctl_slots=2, run_seconds=10.0, start=False)
    q.submit(r.beta, r.Z, r.lam, TOL)
    q.close()  # the kernel never ran; the handle is released
    with pytest.raises(RuntimeError):
        q.submit(r.beta, r.Z, r.lam, TOL)
