"""The worker protocol of the global-memory LGCD tiles (Alg. 3: soft-locks,
notifications, the `pending` termination count), run on the CPU model of
tests/_protocol_sim.py under schedules the GPU never promises: seeded
random interleavings of every worker step (a neighbour can see half of a
window update), notifications delayed by up to 200 steps, lock-step rounds
in which every worker scans before any applies.

* With soft-locks every run terminates with nothing pending and nothing in
  flight, at max |dZ| < eps on a beta recomputed from scratch, at the FP64
  oracle's objective (Alg. 1 on one worker) within 1e-9 relative.
* Without them (the ablation of Section 5.1), four workers updating around
  each tile corner at once interfere (Prop. A.2) and the activations grow
  until the divergence guard stops the run, while the soft-locks on the same
  lock-step schedule converge to the oracle's optimum."""
import numpy as np
import pytest

from synthetic import Workload, make_problem
from tests._protocol_sim import Problem, Sim

W1 = Workload("sim1d", P=2, K=3, T=(300,), L=(8,), density=0.05, sigma=0.1)
W2 = Workload("sim2d", P=1, K=2, T=(40, 44), L=(4, 4), density=0.04, sigma=0.1)
EPS = 1e-6

CASES = [
    (W1, (16,), "random", 0, 20), (W1, (8,), "random", 1, 200), (W1, (8,), "lockstep", 0, 1),
    (W2, (8, 8), "random", 2, 20), (W2, (4, 5), "random", 3, 200), (W2, (4, 5), "lockstep", 0, 1),
]


@pytest.mark.parametrize("w,tile,schedule,seed,delay", CASES,
                         ids=[f"{c[0].name}-{'x'.join(map(str, c[1]))}-{c[2]}{c[3]}" for c in CASES])
def test_soft_locks_terminate_at_the_oracle_optimum(orc, w, tile, schedule, seed, delay):
    X, D, _ = make_problem(w, 1)
    lam = 0.1 * orc.lambda_max(X, D)
    pb = Problem(X, D, lam, EPS)
    sim = Sim(pb, tile=tile, sub=tuple(2 * l for l in w.L), lock=True, schedule=schedule, seed=seed,
              max_delay=delay)
    sim.run()
    assert sim.stop is None
    assert sim.pending == 0 and not sim.in_flight and sim.G > 4
    # border candidates met competition and the lock decided
    assert sim.lock_checks > 0 and sim.rejected > 0 and sim.accept_log
    assert all(d0 > lo and d0 >= hi for d0, lo, hi in sim.accept_log)
    assert pb.kkt(sim.Z) < EPS * (1 + 1e-9)
    ref = orc.lgcd(X, D, lam, EPS)
    f_ref = orc.objective(X, D, ref["Z"], lam)
    assert abs(pb.objective(sim.Z) - f_ref) <= 1e-9 * f_ref


SUB_CASES = [(W2, (16, 16), (4, 4), "random", 4, 50), (W2, (12, 20), (4, 4), "lockstep", 0, 1),
             (W1, (32,), (8,), "random", 5, 50)]


@pytest.mark.parametrize("w,tile,sub,schedule,seed,delay", SUB_CASES,
                         ids=[f"{c[0].name}-{'x'.join(map(str, c[1]))}-sub{'x'.join(map(str, c[2]))}-{c[3]}{c[4]}"
                              for c in SUB_CASES])
def test_direction_marking_with_many_sub_domains(orc, w, tile, sub, schedule, seed, delay):
    """Sub-domains of side L inside tiles of several of them, as the GPU
    runs (4096^2 image: 32 x 32 sub-domains of 255 x 214 tiles): a bump from
    a neighbour marks only the receiver's sub-domains facing it, and the run
    still ends at the oracle's optimum with max |dZ| < eps."""
    X, D, _ = make_problem(w, 2)
    lam = 0.1 * orc.lambda_max(X, D)
    pb = Problem(X, D, lam, EPS)
    sim = Sim(pb, tile=tile, sub=sub, lock=True, schedule=schedule, seed=seed, max_delay=delay)
    sim.run()
    assert sim.stop is None
    assert sim.pending == 0 and not sim.in_flight and sim.G >= 4
    assert sim.accepted > 0
    assert pb.kkt(sim.Z) < EPS * (1 + 1e-9)
    ref = orc.lgcd(X, D, lam, EPS)
    f_ref = orc.objective(X, D, ref["Z"], lam)
    assert abs(pb.objective(sim.Z) - f_ref) <= 1e-9 * f_ref


DYN_CASES = [(W2, (8, 8), (4, 4), 4, "random", 6, 50), (W2, (8, 11), (4, 4), 3, "lockstep", 0, 1),
             (W1, (16,), (8,), 5, "random", 7, 100)]


@pytest.mark.parametrize("w,tile,sub,workers,schedule,seed,delay", DYN_CASES,
                         ids=[f"{c[0].name}-{'x'.join(map(str, c[1]))}-{c[3]}workers-{c[4]}{c[5]}"
                              for c in DYN_CASES])
def test_dynamic_tile_scheduling_terminates_at_the_optimum(orc, w, tile, sub, workers, schedule, seed, delay):
    """More tiles than workers: a worker runs a tile until it would pause,
    leaves it idle with its state (dirty set, seen counters) and takes the
    next ready one; a notification to an idle tile queues it again.  The
    termination count (tiles queued or running plus unobserved notifications)
    still ends the run only at a point where no coordinate can move by eps,
    and that point is the oracle's optimum."""
    X, D, _ = make_problem(w, 3)
    lam = 0.1 * orc.lambda_max(X, D)
    pb = Problem(X, D, lam, EPS)
    sim = Sim(pb, tile=tile, sub=sub, lock=True, schedule=schedule, seed=seed, max_delay=delay, workers=workers)
    assert sim.workers < sim.G
    sim.run()
    assert sim.stop is None
    assert sim.pending == 0 and not sim.in_flight and not sim.ready
    assert all(st == "idle" for st in sim.status)
    assert sim.activations > sim.G  # tiles were taken up again after pausing
    assert pb.kkt(sim.Z) < EPS * (1 + 1e-9)
    ref = orc.lgcd(X, D, lam, EPS)
    f_ref = orc.objective(X, D, ref["Z"], lam)
    assert abs(pb.objective(sim.Z) - f_ref) <= 1e-9 * f_ref


@pytest.mark.parametrize("workers", [None, 5], ids=["resident", "dynamic"])
def test_dropped_and_retried_notifications(orc, workers):
    """A third of the notification deliveries fail and are sent again after a
    fresh delay: the counts they hold keep the run alive until they land, and
    it ends at the oracle's optimum."""
    X, D, _ = make_problem(W2, 4)
    lam = 0.1 * orc.lambda_max(X, D)
    pb = Problem(X, D, lam, EPS)
    sim = Sim(pb, tile=(8, 8), sub=(4, 4), lock=True, schedule="random", seed=8, max_delay=30, workers=workers,
              drop=0.33)
    sim.run()
    assert sim.stop is None and sim.dropped > 0
    assert sim.pending == 0 and not sim.in_flight
    assert pb.kkt(sim.Z) < EPS * (1 + 1e-9)
    ref = orc.lgcd(X, D, lam, EPS)
    assert abs(pb.objective(sim.Z) - orc.objective(X, D, ref["Z"], lam)) <= 1e-9 * pb.objective(sim.Z)


def _corner_problem():
    """One 4 x 4 box atom; activations of 5 at every tile corner of a 4 x 4
    tile grid, so the four tiles around a corner all find their best
    candidate next to it."""
    from scipy.signal import convolve
    L, T = 4, 36
    D = np.ones((1, 1, L, L)) / L
    Zt = np.zeros((T - L + 1, T - L + 1))
    for ci in range(4, 33, 4):
        for cj in range(4, 33, 4):
            Zt[ci - 2, cj - 2] = 5.0
    X = convolve(Zt, D[0, 0], mode="full")[None] + 0.01 * np.random.default_rng(0).standard_normal((1, T, T))
    return X, D, L


def test_without_soft_locks_corner_updates_diverge(orc):
    X, D, L = _corner_problem()
    lam = 0.01 * orc.lambda_max(X, D)
    pb = Problem(X, D, lam, EPS)
    guard = 50.0 / np.abs(D).max()  # the bound of Section 5.1
    nolock = Sim(pb, tile=(L, L), sub=(2 * L, 2 * L), lock=False, schedule="lockstep", guard=guard)
    nolock.run(max_ticks=40000)
    assert nolock.stop == "diverged"
    assert np.abs(nolock.Z).max() > guard
    assert pb.objective(nolock.Z) > pb.objective(np.zeros_like(nolock.Z))
    locked = Sim(pb, tile=(L, L), sub=(2 * L, 2 * L), lock=True, schedule="lockstep", guard=guard)
    locked.run(max_ticks=200000)
    assert locked.stop is None and locked.pending == 0
    assert pb.kkt(locked.Z) < EPS * (1 + 1e-9)
    ref = orc.lgcd(X, D, lam, EPS)
    f_ref = orc.objective(X, D, ref["Z"], lam)
    assert abs(pb.objective(locked.Z) - f_ref) <= 1e-9 * f_ref
