"""A CPU model of the worker protocol the GPU's global-memory LGCD tiles run
(Alg. 3 of the paper: one locally greedy worker per tile, soft-locks on
border updates, neighbour notifications, global convergence), used to check
the protocol itself under schedules the GPU never promises: seeded random
interleavings, delayed notifications, lock-step rounds.

Everything is FP64, on a 1-D (T0 = L0 = 1) or 2-D problem: X (P, T0, T1),
D (K, P, L0, L1).  Shared state is what the GPU keeps in global memory: beta
and Z over the whole activation domain, one notification counter per tile
and neighbour direction, and the `pending` count of active workers plus
notifications not yet observed.  A worker is a generator that yields at every point where another
worker may run: after reading its counters, after the scan, after the soft-lock
test, after writing Z and after each chunk of rows of its window update (so
neighbours see a half-applied window).  Notifications (counter increments)
reach their tile after a delay the scheduler draws, out of order, and with
`drop` > 0 some deliveries fail and are retried after a fresh delay.

The worker's steps mirror the kernel (paper_1901_09235_gb300/csrc/
lgcd_global.cuh): scan the dirty sub-domain C_m for the largest
|Z' - Z|, Z' = ST(beta, lambda) / ||D_k||^2 (Eq. pb_coord); skip it when
below eps; a candidate whose window V(s0) leaves the tile is accepted only if
its |dZ| is above every |dZ| in V(s0) held by a lower-index tile and not below
any held by a higher-index one (Eq. soft_lock, ties to the lower row-major
tile index); an accepted update writes Z, subtracts C[k][k0][s - s0] dZ from
beta over V(s0) (Eq. beta_update) and notifies the tiles V(s0) reaches,
each on its counter for the direction the sender lies in; a bump marks dirty
the sub-domains of the receiver within L - 1 of the edge or corner it shares
with the sender; a worker whose sub-domains are all clean pauses
(pending - 1) until a notification arrives (pending + 1) or pending
reaches 0.

With `workers` below the number of tiles the model also runs a dynamic
schedule that the GPU does not (yet): workers take ready tiles from a queue,
a tile that would pause goes idle, and a notification queues an idle tile.

This module is test infrastructure: it shares nothing with the CUDA library."""
from __future__ import annotations

import numpy as np
from scipy.signal import correlate


class Problem:
    """X (P, T0, T1), D (K, P, L0, L1) (1-D: T0 = L0 = 1), lambda, eps."""

    def __init__(self, X, D, lam, eps):
        X = np.asarray(X, np.float64)
        D = np.asarray(D, np.float64)
        if X.ndim == 2:
            X, D = X[:, None, :], D[:, :, None, :]
        self.X, self.D = X, D
        self.P, self.T0, self.T1 = X.shape
        self.K, _, self.L0, self.L1 = D.shape
        self.N0, self.N1 = self.T0 - self.L0 + 1, self.T1 - self.L1 + 1
        self.lam, self.eps = float(lam), float(eps)
        K = self.K
        # C[k][k2][d + L - 1] = sum_p sum_tau D_kp[tau] D_k2p[tau + d]
        self.C = np.zeros((K, K, 2 * self.L0 - 1, 2 * self.L1 - 1))
        for k in range(K):
            for k2 in range(K):
                for p in range(self.P):
                    self.C[k, k2] += correlate(D[k2, p], D[k, p], mode="full")
        self.nrm = np.array([self.C[k, k, self.L0 - 1, self.L1 - 1] for k in range(K)])

    def correlate_X(self, R):
        b = np.zeros((self.K, self.N0, self.N1))
        for k in range(self.K):
            for p in range(self.P):
                b[k] += correlate(R[p], self.D[k, p], mode="valid")
        return b

    def residual(self, Z):
        from scipy.signal import convolve
        R = self.X.copy()
        for k in range(self.K):
            for p in range(self.P):
                R[p] -= convolve(Z[k], self.D[k, p], mode="full")
        return R

    def beta_init(self):
        return self.correlate_X(self.X)

    def beta_of(self, Z):
        """beta from its definition for Z (Section 3)."""
        return self.correlate_X(self.residual(Z)) + self.nrm[:, None, None] * Z

    def objective(self, Z):
        R = self.residual(Z)
        return 0.5 * float(np.sum(R * R)) + self.lam * float(np.abs(Z).sum())

    def kkt(self, Z):
        b = self.beta_of(Z)
        zn = np.sign(b) * np.maximum(np.abs(b) - self.lam, 0.0) / self.nrm[:, None, None]
        return float(np.abs(zn - Z).max())

    def zprime(self, beta, k):
        return np.sign(beta) * max(abs(beta) - self.lam, 0.0) / self.nrm[k]


class Sim:
    """Tiles of t0 x t1 positions, sub-domains of sub0 x sub1; `lock` False
    is the no-lock ablation.  `schedule` is "random" (one seeded worker step
    per tick, notification delays drawn up to `max_delay` ticks) or
    "lockstep" (every live worker advances one step per tick, notifications
    arrive the next tick)."""

    def __init__(self, pb: Problem, tile, sub, lock=True, schedule="random", seed=0, max_delay=20,
                 chunks=4, guard=None, workers=None, drop=0.0):
        self.pb = pb
        self.t0, self.t1 = (1, tile[0]) if len(tile) == 1 else tile
        self.s0, self.s1 = (1, sub[0]) if len(sub) == 1 else sub
        self.G0, self.G1 = -(-pb.N0 // self.t0), -(-pb.N1 // self.t1)
        self.G = self.G0 * self.G1
        self.lock, self.schedule, self.max_delay, self.chunks = lock, schedule, max_delay, chunks
        # a delivery attempt fails with this probability and the sender tries
        # again after a fresh delay (the count it added stays in `pending`)
        self.drop, self.dropped = float(drop), 0
        self.rng = np.random.default_rng(seed)
        self.guard = guard
        self.beta = pb.beta_init()
        self.Z = np.zeros_like(self.beta)
        # flag[w][(dr, dc)]: bumps tile w received from its neighbour at
        # tile-grid offset (dr, dc)
        self.flag = [dict() for _ in range(self.G)]
        self.pending = self.G
        self.in_flight = []  # [deliver at tick, tile]
        self.tick = 0
        self.stop = None     # None, "timeout" or "diverged"
        self.accepted = self.rejected = self.lock_checks = 0
        # workers < tiles: tiles are scheduled dynamically (see run_dynamic)
        self.workers = self.G if workers is None else min(int(workers), self.G)
        self.status = ["queued"] * self.G   # queued / running / idle (dynamic mode)
        self.ready = list(range(self.G))    # tiles waiting for a worker, in order
        self.tstate = {}                    # a tile's dirty set, seen counters, m
        self.activations = 0
        # every accepted border update: |dZ| and the largest competing |dZ|
        # in V(s0) of lower / higher tiles at the time of the test
        self.accept_log = []

    def tile_of(self, i, j):
        return (i // self.t0) * self.G1 + j // self.t1

    def activate(self, w):
        """An idle tile with news joins the ready queue (dynamic mode)."""
        if self.status[w] == "idle":
            self.status[w] = "queued"
            self.pending += 1
            self.ready.append(w)

    def worker(self, w, dynamic=False):
        """Tile w's worker.  Resident (dynamic False): runs until the solve
        ends, pausing in place.  Dynamic: returns when the tile would pause,
        leaving it idle (pending - 1) with its state kept for the next
        worker that takes it -- a notification that reached it meanwhile
        queues it again -- and also when its candidate is soft-locked, the
        tile then queued again at once: a worker that kept retrying could
        wait forever on a blocker whose tile has no worker."""
        pb = self.pb
        ta, tb = divmod(w, self.G1)
        r0, c0 = ta * self.t0, tb * self.t1
        h, wd = min(self.t0, pb.N0 - r0), min(self.t1, pb.N1 - c0)
        L0, L1 = pb.L0, pb.L1
        ns0, ns1 = -(-h // self.s0), -(-wd // self.s1)
        M = ns0 * ns1

        def box(q):
            qr, qc = divmod(q, ns1)
            return (r0 + qr * self.s0, min(r0 + h, r0 + (qr + 1) * self.s0),
                    c0 + qc * self.s1, min(c0 + wd, c0 + (qc + 1) * self.s1))

        def in_band(i, j):
            return (i - r0 < L0 - 1 or i - r0 >= h - (L0 - 1) or j - c0 < L1 - 1 or j - c0 >= wd - (L1 - 1))

        def facing(d):
            """Sub-domains within L - 1 of the edge or corner shared with the
            neighbour at offset d."""
            dr, dc = d
            ra, rb = (h - (L0 - 1) if dr > 0 else 0), (L0 - 1 if dr < 0 else h)
            ca, cb = (wd - (L1 - 1) if dc > 0 else 0), (L1 - 1 if dc < 0 else wd)
            out = set()
            for q in range(M):
                a0, a1, b0, b1 = box(q)
                if a0 - r0 < rb and a1 - r0 > ra and b0 - c0 < cb and b1 - c0 > ca:
                    out.add(q)
            return out

        st = self.tstate.setdefault(w, {"dirty": set(range(M)), "seen": {}, "m": 0})
        dirty, seen, m = st["dirty"], st["seen"], st["m"]
        while True:
            f_now = dict(self.flag[w])
            yield
            if self.stop:
                return
            new = {d: n - seen.get(d, 0) for d, n in f_now.items() if n != seen.get(d, 0)}
            got = sum(new.values())
            if got:
                self.pending -= got
                seen.update({d: f_now[d] for d in new})
            # scan C_m
            a0, a1, b0, b1 = box(m)
            best = None
            for i in range(a0, a1):
                for j in range(b0, b1):
                    for k in range(pb.K):
                        zn = pb.zprime(self.beta[k, i, j], k)
                        d = abs(zn - self.Z[k, i, j])
                        key = ((i - r0) * self.t1 + (j - c0)) * pb.K + k
                        if best is None or d > best[0] or (d == best[0] and key < best[1]):
                            best = (d, key, k, i, j, zn)
            yield
            accepted = False
            active = best[0] >= pb.eps
            if active:
                d0, _, k0, i0, j0, zn = best
                v = (max(0, i0 - L0 + 1), min(pb.N0, i0 + L0), max(0, j0 - L1 + 1), min(pb.N1, j0 + L1))
                ok = True
                if self.lock and in_band(i0, j0):
                    self.lock_checks += 1
                    lo_max = hi_max = -1.0
                    for i in range(v[0], v[1]):
                        for j in range(v[2], v[3]):
                            ws = self.tile_of(i, j)
                            if ws == w:
                                continue
                            for k in range(pb.K):
                                d = abs(pb.zprime(self.beta[k, i, j], k) - self.Z[k, i, j])
                                if ws < w:
                                    lo_max = max(lo_max, d)
                                else:
                                    hi_max = max(hi_max, d)
                    ok = d0 > lo_max and d0 >= hi_max
                    if ok:
                        self.accept_log.append((d0, lo_max, hi_max))
                    yield
                if ok:
                    accepted = True
                    self.accepted += 1
                    dz = zn - self.Z[k0, i0, j0]
                    self.Z[k0, i0, j0] = zn
                    if self.guard is not None and abs(zn) > self.guard:
                        self.stop = "diverged"
                    yield
                    # window update by chunks of rows; neighbours may run in between
                    rows = np.arange(v[0], v[1])
                    for part in np.array_split(rows, min(self.chunks, len(rows))):
                        for i in part:
                            for j in range(v[2], v[3]):
                                for k in range(pb.K):
                                    if k == k0 and i == i0 and j == j0:
                                        continue
                                    self.beta[k, i, j] -= pb.C[k, k0, i - i0 + L0 - 1, j - j0 + L1 - 1] * dz
                        yield
                    targets = {self.tile_of(i, j) for i in (v[0], v[1] - 1) for j in (v[2], v[3] - 1)}
                    targets |= {self.tile_of(i, j0) for i in (v[0], v[1] - 1)} | {self.tile_of(i0, j) for j in (v[2], v[3] - 1)}
                    targets.discard(w)
                    if targets:
                        self.pending += len(targets)
                        for tw in sorted(targets):
                            delay = 1 if self.schedule == "lockstep" else int(self.rng.integers(0, self.max_delay + 1))
                            # the receiver sees this tile at the opposite offset
                            d = (ta - tw // self.G1, tb - tw % self.G1)
                            self.in_flight.append([self.tick + delay, tw, d])
                    for q in range(M):
                        q0, q1, p0, p1 = box(q)
                        if q0 < v[1] and q1 > v[0] and p0 < v[3] and p1 > v[2]:
                            dirty.add(q)
                else:
                    self.rejected += 1
                    if dynamic:
                        # the blocker may sit in a tile that waits for a
                        # worker: give this one up and queue the tile again
                        # (it stays active), so that every tile gets to run
                        for d in new:
                            dirty |= facing(d)
                        nxt = sorted(q for q in dirty if q > m) or sorted(dirty)
                        st["m"] = nxt[0]
                        self.status[w] = "queued"
                        self.ready.append(w)
                        return
            else:
                dirty.discard(m)
            for d in new:
                dirty |= facing(d)
            if not dirty and dynamic:
                st["m"] = m
                self.status[w] = "idle"
                self.pending -= 1
                if any(n != seen.get(d, 0) for d, n in self.flag[w].items()):
                    self.activate(w)  # a bump it has not seen yet
                return
            if not dirty:
                self.pending -= 1
                while True:
                    woke = [d for d, n in self.flag[w].items() if n != seen.get(d, 0)]
                    if woke:
                        # the bumps themselves are accounted for by the next
                        # iteration's read of the counters
                        self.pending += 1
                        for d in woke:
                            dirty |= facing(d)
                        dirty = dirty or set(range(M))
                        break
                    if self.pending == 0 or self.stop:
                        return
                    yield
            nxt = sorted(q for q in dirty if q > m) or sorted(dirty)
            m = nxt[0]
            st["m"] = m

    def deliver(self):
        keep = []
        for at, tw, d in self.in_flight:
            if at <= self.tick and self.drop > 0 and self.rng.random() < self.drop:
                self.dropped += 1
                keep.append([self.tick + 1 + int(self.rng.integers(0, self.max_delay + 1)), tw, d])
            elif at <= self.tick:
                self.flag[tw][d] = self.flag[tw].get(d, 0) + 1
                if self.workers < self.G:
                    self.activate(tw)  # the sender queues an idle receiver
            else:
                keep.append([at, tw, d])
        self.in_flight = keep

    def slot(self):
        """One worker of the dynamic mode: takes the first ready tile, runs
        it until it would pause, takes the next; ends when no tile is active
        and no notification is in flight (pending = 0)."""
        while True:
            while not self.ready:
                if self.pending == 0 or self.stop:
                    return
                yield
            w = self.ready.pop(0)
            self.status[w] = "running"
            self.activations += 1
            yield from self.worker(w, dynamic=True)
            if self.stop:
                return

    def run(self, max_ticks=2_000_000):
        """Runs until every worker has returned.  Returns the tick count; a
        run that reaches max_ticks is stopped ("timeout") like the GPU's
        deadline stops a kernel."""
        if self.workers < self.G:
            live = {q: self.slot() for q in range(self.workers)}
        else:
            live = {w: self.worker(w) for w in range(self.G)}
        while live:
            if self.tick >= max_ticks and not self.stop:
                self.stop = "timeout"
            self.deliver()
            order = list(live) if self.schedule == "lockstep" else [list(live)[int(self.rng.integers(0, len(live)))]]
            if self.stop:
                order = list(live)  # let every worker see the stop word and return
            for w in order:
                try:
                    next(live[w])
                except StopIteration:
                    del live[w]
            self.tick += 1
        return self.tick
