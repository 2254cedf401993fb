"""Continuous-batching CSC server over the persistent LGCD queue.

Requests are 2-D images (P, T0, T1) in pinned host memory, all coded against
one resident dictionary D (K, P, L0, L1).  The server

* admits a request when its device footprint (X, beta, Z) fits in the HBM
  budget that is still free and the queue has a control slot, in arrival
  order (the head of the line waits for room; nothing overtakes it);
* copies X to the device, initialises beta = D~ * X and lambda_max (FP32 or
  split-bf16 on the tensor cores), and submits the LGCD job (Alg. 3 over the
  image's tiles) to the persistent kernel, which is already solving the
  requests admitted before it;
* when a job completes, recomputes beta from Z and checks max |dZ| < tol
  (the stopping rule of Alg. 1 on a beta free of rounding drift); a request
  that fails the check is resubmitted warm, one that passes is finished, its
  result copied out if asked, and its memory released for the next admission.

Every step runs in the CUDA library (queue kernel, beta-init, refresh);
this module is host-side bookkeeping.  All device memory comes from one
arena allocated before the queue starts, so that no allocation runs beside
the persistent kernel.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import (Queue, csc_init_beta, csc_init_beta_bf16x3, csc_refresh_beta, make_shape,
               workspace_size, z_shape)

ALIGN = 256


class Arena:
    """First-fit allocator over one device buffer (byte offsets, ALIGN-aligned)."""

    def __init__(self, nbytes: int, device):
        import torch
        self.size = int(nbytes)
        self.buf = torch.empty(self.size, dtype=torch.uint8, device=device)
        self.free = [(0, self.size)]  # sorted, coalesced (offset, size)
        self.used = 0
        self.peak = 0

    @staticmethod
    def rounded(nbytes: int) -> int:
        return (int(nbytes) + ALIGN - 1) // ALIGN * ALIGN

    def alloc(self, nbytes: int):
        n = self.rounded(nbytes)
        for i, (off, sz) in enumerate(self.free):
            if sz >= n:
                if sz == n:
                    self.free.pop(i)
                else:
                    self.free[i] = (off + n, sz - n)
                self.used += n
                self.peak = max(self.peak, self.used)
                return off
        return None

    def release(self, off: int, nbytes: int):
        n = self.rounded(nbytes)
        self.used -= n
        fr = self.free
        i = 0
        while i < len(fr) and fr[i][0] < off:
            i += 1
        fr.insert(i, (off, n))
        if i + 1 < len(fr) and fr[i][0] + fr[i][1] == fr[i + 1][0]:
            fr[i] = (fr[i][0], fr[i][1] + fr[i + 1][1])
            fr.pop(i + 1)
        if i > 0 and fr[i - 1][0] + fr[i - 1][1] == fr[i][0]:
            fr[i - 1] = (fr[i - 1][0], fr[i - 1][1] + fr[i][1])
            fr.pop(i)

    def view(self, off: int, shape, dtype):
        import torch
        n = int(np.prod(shape)) * torch.empty((), dtype=dtype).element_size()
        return self.buf[off:off + n].view(dtype).view(tuple(shape))


def footprint(D_shape, X_shape) -> int:
    """Device bytes one request holds while admitted: X, beta and Z (FP32)."""
    P, T0, T1 = X_shape
    K, _, L0, L1 = D_shape
    nz = K * (T0 - L0 + 1) * (T1 - L1 + 1)
    return Arena.rounded(P * T0 * T1 * 4) + 2 * Arena.rounded(nz * 4)


@dataclass
class Request:
    """One CSC request: X in pinned host memory; arrival in seconds from the
    start of serve().  Z_out (pinned host, shape of Z) receives the result
    when given."""
    X: object
    arrival: float = 0.0
    Z_out: object = None
    # filled in by the server
    t_admit: float = float("nan")
    t_done: float = float("nan")
    lam: float = float("nan")
    objective: float = float("nan")
    max_dz: float = float("nan")
    updates: int = 0
    rounds: int = 0
    status: int = -1
    job_ms: float = 0.0
    _alloc: list = field(default_factory=list, repr=False)
    _dev: tuple = field(default=None, repr=False)

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival


class Server:
    """Continuous batching of CSC solves against a resident dictionary D."""

    def __init__(self, D, hbm_budget: int, max_side=(2048, 2048), reg: float = 0.1, tol: float = 1e-4,
                 precision: str = "fp32", max_jobs: int = 8192, ctl_slots: int = 256,
                 run_seconds: float = 600.0, max_rounds: int = 4, tuning: dict | None = None,
                 ctas_per_sm: int | None = None):
        import torch
        if precision not in ("fp32", "bf16x3"):
            raise ValueError("precision must be 'fp32' or 'bf16x3'")
        if D.dim() != 4:
            raise ValueError("D must be (K, P, L0, L1)")
        self.D, self.reg, self.tol, self.max_rounds = D, float(reg), float(tol), int(max_rounds)
        self.precision = precision
        self.tuning = tuning  # size class -> sub-domain side and stop margin (autotune.tune)
        self.device = D.device
        K, P, L0, L1 = D.shape
        self.stream = torch.cuda.Stream(device=self.device)  # copies, beta-init, refresh
        cur = torch.cuda.current_stream(self.device)
        self.stream.wait_stream(cur)
        big = make_shape((P,) + tuple(max_side), tuple(D.shape))
        self.max_side = tuple(max_side)
        # one refresh / init workspace, shared: those calls are serialised on self.stream
        self.ws = torch.empty(workspace_size(big), dtype=torch.uint8, device=self.device)
        self.arena = Arena(hbm_budget, self.device)
        with torch.cuda.stream(self.stream):
            x0 = torch.zeros((P, L0, L1), dtype=torch.float32, device=self.device)
            _, self.dtd, _ = csc_init_beta(x0, D, ws=self.ws, stream=self.stream)
            self.dtd_scratch = torch.empty_like(self.dtd)
        self.stream.synchronize()
        # three queue CTAs per SM when only FP32 kernels run beside it, two
        # when the tensor-core beta-init must fit too
        if ctas_per_sm is None:
            ctas_per_sm = 3 if precision == "fp32" else 2
        if precision == "bf16x3" and ctas_per_sm == 3:
            raise ValueError("the tensor-core beta-init does not fit beside a queue of three CTAs per SM")
        self.ctas_per_sm = ctas_per_sm
        self.q = Queue(D, self.dtd, max_jobs=max_jobs, ctl_slots=ctl_slots, run_seconds=run_seconds,
                       ctas_per_sm=ctas_per_sm)
        self.active = {}
        self.n_free_ctl = ctl_slots

    def footprint(self, X_shape) -> int:
        return footprint(tuple(self.D.shape), X_shape)

    # ------------------------------------------------------------- lifecycle
    def _admit(self, r: Request, now: float) -> bool:
        import torch
        P, T0, T1 = r.X.shape
        if T0 > self.max_side[0] or T1 > self.max_side[1]:
            raise ValueError(f"request {tuple(r.X.shape)} above max_side {self.max_side}")
        if self.n_free_ctl <= 0:
            return False
        s = make_shape(tuple(r.X.shape), tuple(self.D.shape))
        zs = z_shape(s)
        sizes = [P * T0 * T1 * 4, int(np.prod(zs)) * 4, int(np.prod(zs)) * 4]
        offs = []
        for n in sizes:
            o = self.arena.alloc(n)
            if o is None:
                for oo, nn in zip(offs, sizes):
                    self.arena.release(oo, nn)
                return False
            offs.append(o)
        r._alloc = list(zip(offs, sizes))
        X = self.arena.view(offs[0], (P, T0, T1), torch.float32)
        beta = self.arena.view(offs[1], zs, torch.float32)
        Z = self.arena.view(offs[2], zs, torch.float32)
        r._dev = (X, beta, Z)
        r.t_admit = now
        try:
            with torch.cuda.stream(self.stream):
                X.copy_(r.X, non_blocking=True)
                init = csc_init_beta_bf16x3 if self.precision == "bf16x3" else csc_init_beta
                _, _, lmax = init(X, self.D, beta=beta, dtd=self.dtd_scratch, ws=self.ws, stream=self.stream)
            r.lam = self.reg * lmax
            self._submit(r, warm=False)
        except Exception:
            self._release(r)
            raise
        return True

    def _release(self, r: Request):
        for o, n in r._alloc:
            self.arena.release(o, n)
        r._alloc, r._dev = [], None

    def _submit(self, r: Request, warm: bool):
        _, beta, Z = r._dev
        opts = None
        if self.tuning:
            from .autotune import opts_for
            opts = opts_for(self.tuning, max(int(r.X.shape[1]), int(r.X.shape[2])))
        j = self.q.submit(beta, Z, r.lam, self.tol, warm_start=warm, stream=self.stream, opts=opts)
        self.active[j] = r
        self.n_free_ctl -= 1

    def _complete(self, r: Request, st: dict, now_fn):
        import torch
        self.n_free_ctl += 1
        r.updates += st["updates"]
        r.rounds += 1
        r.job_ms += st["kernel_ms"]
        X, beta, Z = r._dev
        if st["status"] == 0:
            _, r.max_dz, r.objective = csc_refresh_beta(X, self.D, Z, r.lam, beta=beta, ws=self.ws,
                                                        stream=self.stream)
            if r.max_dz >= self.tol and r.rounds < self.max_rounds:
                self._submit(r, warm=True)
                return False
            r.status = 0 if r.max_dz < self.tol else 3
        else:
            r.status = st["status"]
        if r.Z_out is not None:
            with torch.cuda.stream(self.stream):
                r.Z_out.copy_(Z, non_blocking=True)
            self.stream.synchronize()
        self._release(r)
        r.t_done = now_fn()
        return True

    def serve(self, requests, poll_sleep: float = 0.0, stall_s: float = 90.0):
        """Serve `requests` (list of Request, arrival times in seconds from
        now); returns them with their results and timings filled in.  Raises
        if no job completes for stall_s seconds while jobs are in flight."""
        t0 = time.perf_counter()
        last = t0
        now = lambda: time.perf_counter() - t0  # noqa: E731
        for r in requests:
            if self.footprint(tuple(r.X.shape)) > self.arena.size:
                raise ValueError(f"request {tuple(r.X.shape)} does not fit the HBM budget")
        future = deque(sorted(requests, key=lambda r: r.arrival))
        line = deque()
        n_done = 0
        while n_done < len(requests):
            t = now()
            while future and future[0].arrival <= t:
                line.append(future.popleft())
            progressed = False
            while line and self._admit(line[0], now()):
                line.popleft()
                progressed = True
            for j in list(self.active):
                st = self.q.poll(j)
                if st is not None:
                    r = self.active.pop(j)
                    if self._complete(r, st, now):
                        n_done += 1
                    progressed = True
            if progressed:
                last = time.perf_counter()
            elif self.active and time.perf_counter() - last > stall_s:
                state = {j: self.q.inspect(j) for j in list(self.active)[:8]}
                raise RuntimeError(f"queue stalled for {stall_s} s; in flight: {state}")
            if not progressed:
                if not self.active and not line and future:
                    time.sleep(max(0.0, min(future[0].arrival - now(), 1e-3)))
                elif poll_sleep > 0:
                    time.sleep(poll_sleep)
        return requests

    def close(self):
        self.q.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def latency_summary(requests) -> dict:
    lat = np.array([r.latency for r in requests]) * 1e3
    return dict(p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
                mean_ms=float(lat.mean()), max_ms=float(lat.max()))
