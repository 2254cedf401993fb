"""Benchmark of the CSC hot path on GB300.

Default workload (``--workload image4096``): the plain large-image CSC solve,
a 4096 x 4096 image (P = 1) with K = 25 atoms of 32 x 32, Z drawn
Bernoulli(1e-4) x |N(0,1)|, noise sigma = 0.05, lambda = 0.1 lambda_max,
tol 1e-4.  One step = one solve:
  csc_init_beta  (beta = D~ * X, the D^T D table, lambda_max; FP32)
  csc_lgcd_solve (LGCD over a 2-D grid of global-memory tiles with soft-locks
                  to max |dZ| < tol, then beta recomputed from Z, the KKT test
                  max |dZ| < tol on it and the FP64 objective)
Every step starts from the same X and D.  The metric is solves/s with p50/p99
step latency and coordinate updates/s.

``--workload signal``: the 1-D multichannel workload (P = 5, T = 200,000,
K = 10, L = 64), one step = csc_init_beta + csc_lgcd_solve + cdl_dict_stats +
cdl_dict_update issued as one cdl_step call (``--api calls``: four calls).
Other workloads (served trace, single served-family images, the coordinate
selection and lambda sweeps) are listed under ``--workload``.

Timing: W warm-up steps, then K steps, each bracketed by CUDA events on the
launching stream; L2 is flushed (256 MiB write) between steps outside the
events.  `e2e` repeats the measurement through host buffers (pinned inputs
copied in, the step's result copied out, every step).

``--impl reference`` times the FP64 CPU oracle instead.  Under torchrun
(N > 1) every rank solves its own problem (independent replicas, no
collective on the data path); value = all solves / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CSC coordinate updates/s and solves/s to tol 1e-4 (p50/p99 latency), 1 GB300 vs plain"
UNIT = "solves/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 200 for the GPU arm of the 1-D workload, 30 for the "
                         "4096^2 image, 20 otherwise)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--workload", default="image4096",
                    choices=["image4096", "signal", "cdl", "betainit", "served", "image", "selection", "lambda"],
                    help="image4096: the plain 4096^2 CSC solve, 25 atoms of 32 x 32 (default); "
                         "signal: the 1-D multichannel solve + dictionary step; "
                         "cdl: 10 outer iterations of Alg. 2 on an 8192^2 image, split-bf16 beta-init "
                         "against plain FP32; betainit: beta-init alone (FP32 CUDA cores and split bf16 on the "
                         "tensor cores) on the 4096^2 family (--side); "
                         "served: the request trace through the continuous-batching server; "
                         "image: single solves of one served-family image (--side); "
                         "selection: LGCD / greedy / randomized / cyclic CD on one worker (Section 5.1); "
                         "lambda: 2-D solves over lambda x workers x {greedy, LGCD}")
    ap.add_argument("--cap", type=float, default=60.0, help="selection / lambda: seconds per solve")
    ap.add_argument("--side", type=int, default=1024,
                    help="image: side of the square image; image4096: another side for the same family "
                         "(profiling cases; default 4096)")
    ap.add_argument("--sub", type=int, default=0,
                    help="image4096 / cdl: sub-domain side (0: chosen by the autotuner, or 2 L with --no-tune)")
    ap.add_argument("--crop", type=int, default=512,
                    help="image4096: side of the crop of the same family that the oracle arms solve")
    ap.add_argument("--requests", type=int, default=512, help="served: requests in the trace")
    ap.add_argument("--rate", type=float, default=1000.0, help="served: Poisson arrival rate (1/s)")
    ap.add_argument("--budget-gb", type=float, default=32.0, help="served: HBM admission budget")
    ap.add_argument("--precision", default="bf16x3", choices=["bf16x3", "fp32"],
                    help="served: beta-init precision of the served arm")
    ap.add_argument("--api", default="step", choices=["step", "calls"],
                    help="signal: one cdl_step call per step (default) or the four separate calls")
    ap.add_argument("--no-tune", action="store_true",
                    help="served / image4096: skip the sub-domain (and stop-margin) autotuner (library defaults)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload():
    from synthetic import SIGNAL_200K
    return SIGNAL_200K


def config_dict(w, extra=None):
    d = {"workload": w.name, "P": w.P, "K": w.K, "T": list(w.T), "L": list(w.L),
         "density": w.density, "sigma": w.sigma, "lambda": f"{w.reg} * lambda_max", "tol": w.tol,
         "step": "init_beta + lgcd_solve + dict_stats + dict_update",
         "l2": "flushed between steps (256 MiB write), inputs 4 MB < L2"}
    if extra:
        d.update(extra)
    return d


# ----------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.proc = None
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------- GPU arm
class GpuStep:
    """Device-resident buffers and one hot-path step through the C ABI."""

    def __init__(self, X, D0, w, device, api="step"):
        import torch
        import paper_1901_09235_gb300 as pkg
        self.pkg, self.w, self.api = pkg, w, api
        self.X = torch.from_numpy(X).to(device)
        self.D0 = torch.from_numpy(D0).to(device)
        self.D = self.D0.clone()
        self.prob = pkg.Problem.create(self.X, self.D)
        self.xs = float((X.astype(np.float64) ** 2).sum())
        self.opts = pkg.default_opts()
        self.last = {}

    def run(self, X=None, D=None):
        pkg, p = self.pkg, self.prob
        Xd = self.X if X is None else X
        if D is None:
            self.D.copy_(self.D0, non_blocking=True)
            D = self.D
        if self.api == "step":
            _, st = pkg.cdl_step(Xd, D, p, reg=self.w.reg, tol=self.w.tol, x_sqnorm=self.xs, pgd_max_iter=50,
                                 pgd_tol=1e-8, opts=self.opts)
            if st["status"] != pkg.CSC_OK:
                raise RuntimeError(f"solve status {st['status']}: {pkg.status_string(st['status'])}")
            self.last = st
            return st
        _, _, lmax = pkg.csc_init_beta(Xd, D, p.beta, p.dtd, p.ws)
        lam = self.w.reg * lmax
        Z, st = pkg.csc_lgcd_solve(Xd, D, p.dtd, p.beta, lam, self.w.tol, Z=p.Z, opts=self.opts,
                                   ws=p.ws)
        if st["status"] != pkg.CSC_OK:
            raise RuntimeError(f"solve status {st['status']}: {pkg.status_string(st['status'])}")
        pkg.cdl_dict_stats(Z, Xd, tuple(D.shape), p.phi, p.psi, p.ws)
        F, it = pkg.cdl_dict_update(p.phi, p.psi, self.xs, D, tuple(Xd.shape), max_iter=50, tol=1e-8,
                                    ws=p.ws)
        st["dict_F"], st["dict_iters"], st["lambda"] = F, it, lam
        self.last = st
        return st


def launches_per_step(st):
    # init_beta: corr + dtd; solve: atom norms + per round (header reset, LGCD,
    # 7 refresh kernels); dict_stats: 7; dict_update: 1
    return 2 + 1 + 9 * int(st["refresh_rounds"]) + 7 + 1


def lgcd_algorithmic_bytes(st, w):
    """Bytes one LGCD launch must move by its definition: every iteration
    reads beta and Z over K x |C_m| (8 B per candidate; the kernel counts the
    candidates, sub-domains clipped at tile edges included); every accepted
    update reads and writes beta and reads the D^T D table over K x |window|
    (12 B per entry) and writes one Z (4 B)."""
    win = int(np.prod([2 * l - 1 for l in w.L]))
    return 8 * st["candidates"] + st["updates"] * (12 * w.K * win + 4)


def source_digest(paths):
    """SHA-256 of kernel sources with comments and blank lines taken out, so
    that a committed ncu summary stays tied to the code it measured and not
    to the wording of its comments."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in paths:
        text = open(f).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        lines = [ln.rstrip() for ln in text.splitlines() if ln.strip()]
        h.update("\n".join(lines).encode())
    return h.hexdigest()


def lgcd_traffic_per_launch():
    """DRAM bytes per LGCD launch from the committed ncu summary, or None when
    the kernel sources changed since those counters were taken."""
    prof = os.path.join(ROOT, "profiles", "lgcd_async_kernel_csc1d_T200000_P5_K10_L64.md")
    src = [os.path.join(ROOT, "paper_1901_09235_gb300", "csrc", f)
           for f in ("lgcd_async.cu", "lgcd_common.cuh", "common.cuh")]
    try:
        text = open(prof).read()
        h = source_digest(src)
    except OSError:
        return None
    vals = dict(line.split(" = ", 1) for line in text.splitlines() if " = " in line)
    if vals.get("source_sha256", "").strip() != h:
        return None
    return int(vals["dram_bytes_per_launch"])


def smem_peak_gbs(sm_mhz=2070.0, sms=152):
    """Shared-memory bandwidth: 128 B per clock per SM (32 banks x 4 B)."""
    return sms * 128 * sm_mhz * 1e6 / 1e9


def max_over_ranks(values, device=None):
    """Element-wise maximum of per-rank timings over all ranks (the slowest
    rank sets the whole-job time); the values themselves on one rank."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def l2_copy_gbs(device, mib=32, iters=50):
    """L2 bandwidth probe: a device copy of a buffer that fits L2 twice over
    (read + write bytes per second, CUDA events, best of three runs).  The
    measured-peaks file holds HBM and tensor peaks only."""
    import torch
    a = torch.ones(mib * (1 << 20) // 4, dtype=torch.float32, device=device)
    b = torch.empty_like(a)
    best = 0.0
    for _ in range(3):
        for _ in range(5):
            b.copy_(a)
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        for _ in range(iters):
            b.copy_(a)
        e.record()
        torch.cuda.synchronize()
        best = max(best, 2 * a.numel() * 4 * iters / (s.elapsed_time(e) / 1e3) / 1e9)
    return best


def flush_l2(buf):
    buf.add_(1.0)


def time_gpu(step, steps, warmup, flush, stream, e2e=None):
    import torch
    for _ in range(warmup):
        step.run() if e2e is None else e2e()
    torch.cuda.synchronize()
    times, stats = [], []
    for _ in range(steps):
        flush_l2(flush)
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        s.record(stream)
        st = step.run() if e2e is None else e2e()
        e.record(stream)
        torch.cuda.synchronize()
        times.append(s.elapsed_time(e) / 1e3)
        stats.append(dict(st))
    return times, stats


def cpu_oracle_step(X, D0, w):
    import oracle
    t0 = time.perf_counter()
    lm = oracle.lambda_max(X, D0)
    lam = w.reg * lm
    out = oracle.lgcd(X, D0, lam, w.tol)
    Z = out["Z"]
    obj = oracle.objective(X, D0, Z, lam)
    phi, psi = oracle.phi_psi(Z, X, w.L)
    xs = float((X.astype(np.float64) ** 2).sum())
    oracle.pgd_armijo(phi, psi, xs, D0, max_iter=50, tol=1e-8)
    return time.perf_counter() - t0, out["n_updates"], obj


def cpu_baseline(X, D0, w, seconds):
    import oracle
    oracle.build()
    done, total, upd, obj = 0, 0.0, 0, None
    while total < seconds and done < 20:
        dt, u, obj = cpu_oracle_step(X, D0, w)
        total += dt
        upd += u
        done += 1
    return {"value": done / total, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{done} full oracle steps of the same workload (lambda_max, LGCD, objective, "
                      f"phi/psi, PGD) on one core, {total:.1f} s",
            "updates_per_s": upd / total, "objective": obj}


# ------------------------------------------------------------ served trace
def served_trace(n, seed):
    """The request trace: resident atoms, square sides log-uniform in
    [64, 2048], Poisson arrival order (times are scaled by --rate)."""
    from synthetic import SERVED_ATOMS, Workload, make_dictionary, served_sizes
    P, K, L = SERVED_ATOMS["P"], SERVED_ATOMS["K"], SERVED_ATOMS["L"]
    D = make_dictionary(np.random.default_rng(seed), K, P, L)
    sides = served_sizes(n, seed + 1)
    ws = [Workload(f"served{s}", P, K, (int(s), int(s)), L, SERVED_ATOMS["density"], SERVED_ATOMS["sigma"])
          for s in sides]
    return D, ws


def served_name(n):
    return f"served_{n}req_sides64-2048_P3_K16_L12"


def served_main(args):
    rank, world, local = dist_env()
    from synthetic import make_problem, poisson_arrivals
    D, ws = served_trace(args.requests, args.seed)
    arrivals = poisson_arrivals(args.requests, args.rate, args.seed + 2)
    base_cfg = {"workload": served_name(args.requests), "requests": args.requests, "P": 3, "K": 16,
                "L": [12, 12], "sides": "log-uniform 64..2048 (square)", "density": 0.002,
                "lambda": "0.1 * lambda_max each", "tol": 1e-4, "arrivals": f"Poisson {args.rate:g}/s",
                "hbm_budget_gb": args.budget_gb}
    if args.impl == "reference":
        if rank != 0:
            return 0
        import oracle
        oracle.build()
        # a bounded sample: the smallest requests of the trace, whole solves
        order = np.argsort([w.T[0] for w in ws])
        times, done = [], 0
        for i in order:
            X, _, _ = make_problem(ws[i], args.seed + 100 + int(i), D=D)
            t0 = time.perf_counter()
            lam = 0.1 * oracle.lambda_max(X, D)
            out = oracle.lgcd(X, D, lam, 1e-4)
            oracle.objective(X, D, out["Z"], lam)
            times.append(time.perf_counter() - t0)
            done += 1
            if sum(times) > args.cpu_seconds or done >= args.steps + args.warmup:
                break
        t = times[min(args.warmup, len(times) - 1):] if len(times) > args.warmup else times
        val = len(t) / sum(t)
        sample = f"{len(t)} of the smallest requests of the trace (sides {ws[order[0]].T[0]}..{ws[order[len(times) - 1]].T[0]}), one core"
        line = {"metric": METRIC, "value": val, "unit": UNIT, "impl": "reference", "n_gpus": world,
                "steps": len(t), "warmup": len(times) - len(t), "ms_per_step": 1e3 * sum(t) / len(t),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": dict(base_cfg, arm="FP64 CPU oracle, single thread"),
                "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
                "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    import torch
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_1901_09235_gb300 as pkg
    from paper_1901_09235_gb300 import serve
    from synthetic import make_image_device
    Dd = torch.from_numpy(D).to(device)
    # inputs: built on the device, kept in pinned host memory (requests arrive from the host)
    Xs = []
    for i, w in enumerate(ws):
        Xd = make_image_device(w, args.seed + 100 + i, D, device)
        Xh = torch.empty(Xd.shape, dtype=torch.float32, pin_memory=True)
        Xh.copy_(Xd)
        Xs.append(Xh)
    del Xd
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    n_px = sum(int(w.T[0]) * int(w.T[1]) for w in ws)
    h2d = sum(x.numel() * 4 for x in Xs)

    # ---- autotuner (before the timed region; its own images, other seeds)
    tuning, tune_s = None, 0.0
    if not args.no_tune:
        from paper_1901_09235_gb300 import autotune
        from synthetic import SERVED_ATOMS, Workload
        t0 = time.perf_counter()

        def make_image(side, seed):
            wt = Workload("tune", 3, 16, (side, side), (12, 12), SERVED_ATOMS["density"], SERVED_ATOMS["sigma"])
            return make_image_device(wt, 7_000_000 + seed, D, device)

        tuning = autotune.tune(Dd, make_image, ctas_per_sm=3 if args.precision == "fp32" else 2)
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        tune_s = time.perf_counter() - t0

    # ---- served arm
    budget = int(args.budget_gb * (1 << 30))
    with serve.Server(Dd, budget, max_side=(2048, 2048), precision=args.precision,
                      run_seconds=900.0, tuning=tuning) as srv:
        order = np.argsort([x.shape[1] for x in Xs])
        warm = [serve.Request(X=Xs[i], arrival=0.0) for i in order[:max(3, args.warmup)]]
        srv.serve(warm)
        reqs = [serve.Request(X=x, arrival=float(a)) for x, a in zip(Xs, arrivals)]
        with ClockSampler(local) as clk:
            t0 = time.perf_counter()
            srv.serve(reqs)
            makespan = time.perf_counter() - t0
        clocks = clk.summary()
        peak_bytes = srv.arena.peak
    bad = [i for i, r in enumerate(reqs) if r.status != 0 or not r.max_dz < 1e-4]
    lat = serve.latency_summary(reqs)
    served_val = len(reqs) / makespan

    # ---- plain arm: FP32 single solves one after another, X copied in each time
    opts = pkg.default_opts()
    plain_obj = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for x in Xs:
        Xd = x.to(device, non_blocking=True)
        beta, dtd, lm = pkg.csc_init_beta(Xd, Dd)
        Z, st = pkg.csc_lgcd_solve(Xd, Dd, dtd, beta, 0.1 * lm, 1e-4, opts=opts)
        plain_obj.append((st["objective"], st["status"]))
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - t0
    rel = [abs(r.objective - o) / abs(o) for r, (o, stt) in zip(reqs, plain_obj) if stt == 0]
    line = {
        "metric": METRIC, "value": served_val, "unit": UNIT, "n_gpus": 1, "steps": len(reqs),
        "warmup": len(warm), "ms_per_step": 1e3 * makespan / len(reqs), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (device-built images copied to pinned host memory)",
        "config": dict(base_cfg, arm=f"served: persistent queue ({3 if args.precision == 'fp32' else 2} CTAs "
                       f"per SM), {args.precision} beta-init"
                       + (", autotuned sub-domains" if tuning else ", default sub-domains"),
                       pixels=n_px, timing="host wall clock from the first arrival to the last "
                       "result; every request's X copied in from pinned host memory"),
        "tuning": ({c: {"sub": e["sub"], "stop_margin": e["stop_margin"], "side": e["side"]}
                    for c, e in tuning.items()} if tuning else None),
        "tuning_seconds": tune_s,
        "p50_ms": lat["p50_ms"], "p99_ms": lat["p99_ms"], "mean_latency_ms": lat["mean_ms"],
        "updates_per_s": sum(r.updates for r in reqs) / makespan,
        "failed": len(bad), "hbm_peak_gb": peak_bytes / (1 << 30),
        "refresh_rounds_max": max(r.rounds for r in reqs),
        "plain_fp32_single_solve": {"value": len(Xs) / plain_s, "unit": UNIT, "seconds": plain_s,
                                    "failed": sum(1 for _, stt in plain_obj if stt != 0)},
        "objective_rel_diff_vs_plain_max": max(rel) if rel else None,
        "e2e": {"value": served_val, "unit": UNIT, "h2d_bytes_per_step": int(h2d / len(Xs)),
                "d2h_bytes_per_step": 16},
        "gpu_launches": 1 + sum(3 + 7 * r.rounds for r in reqs),
        "clocks": clocks,
    }
    print(json.dumps(line))
    return 0


def image_main(args):
    """Single solves (beta-init + LGCD with its fresh-beta check) of one
    served-family image: the global-tile worker on its own."""
    import torch
    rank, world, local = dist_env()
    from synthetic import SERVED_ATOMS, Workload, make_dictionary, make_image_device
    P, K, L = SERVED_ATOMS["P"], SERVED_ATOMS["K"], SERVED_ATOMS["L"]
    side = args.side
    w = Workload(f"served_image_{side}x{side}_P3_K16_L12", P, K, (side, side), L, SERVED_ATOMS["density"],
                 SERVED_ATOMS["sigma"])
    cfg = {"workload": w.name, "P": P, "K": K, "T": [side, side], "L": list(L), "density": w.density,
           "lambda": "0.1 * lambda_max", "tol": 1e-4, "step": "init_beta + lgcd_solve (global tiles)",
           "l2": "flushed between steps (256 MiB write)"}
    if args.impl == "reference":
        if rank != 0:
            return 0
        print(json.dumps({"impl": "reference", "unavailable": "image workload: the oracle arm is timed "
                          "by --workload signal and --workload served"}))
        return 0
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_1901_09235_gb300 as pkg
    D = make_dictionary(np.random.default_rng(args.seed), K, P, L)
    Dd = torch.from_numpy(D).to(device)
    X = make_image_device(w, args.seed + 1, D, device)
    s = pkg.make_shape(tuple(X.shape), tuple(Dd.shape))
    ws = pkg.workspace(s, device=device)
    beta = torch.empty(pkg.z_shape(s), dtype=torch.float32, device=device)
    Z = torch.empty_like(beta)
    dtd = torch.empty(pkg.tab_shape(s), dtype=torch.float32, device=device)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=device)
    stream = torch.cuda.current_stream()

    class Step:
        def run(self):
            _, _, lm = pkg.csc_init_beta(X, Dd, beta, dtd, ws)
            _, st = pkg.csc_lgcd_solve(X, Dd, dtd, beta, 0.1 * lm, 1e-4, Z=Z, ws=ws)
            if st["status"] != pkg.CSC_OK:
                raise RuntimeError(f"solve status {st['status']}")
            return st

    with ClockSampler(local) as clk:
        times, stats = time_gpu(Step(), args.steps, max(3, args.warmup), flush, stream)
    clocks = clk.summary()
    tot = max_over_ranks([sum(times)], device)[0]
    if rank != 0:
        return 0
    kms = sum(st["kernel_ms"] for st in stats) / 1e3
    nz = K * (side - L[0] + 1) * (side - L[1] + 1)
    # 8 B per scanned candidate (beta, Z); per update 12 B per window entry
    # (beta read + write, table) + 4 B for Z
    abytes = sum(lgcd_algorithmic_bytes(st, w) for st in stats)
    achieved = abytes / kms / 1e9
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    last = stats[-1]
    line = {"metric": METRIC, "value": world * args.steps / tot, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": cfg,
            "p50_ms": 1e3 * float(np.percentile(times, 50)), "p99_ms": 1e3 * float(np.percentile(times, 99)),
            "lgcd_kernel_ms_per_step": 1e3 * kms / args.steps,
            "updates_per_solve": sum(st["updates"] for st in stats) / args.steps,
            "solve_stats": {k: last[k] for k in ("workers", "tile_size", "iterations", "rejected_softlock",
                                                  "skipped_subtol", "max_worker_iterations", "refresh_rounds",
                                                  "phase_cycles")},
            "roofline": {"bound": "hbm", "kernel": "lgcd_global_kernel", "achieved": achieved, "peak": hbm,
                         "unit": "GB/s", "frac": achieved / hbm, "traffic": None,
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                         "algorithmic_bytes_per_launch": abytes / len(stats), "Z_entries": nz},
            "e2e": None, "gpu_launches": None, "clocks": clocks}
    l2 = l2_copy_gbs(device)
    line["roofline_l2"] = {"bound": "l2", "kernel": "lgcd_global_kernel", "achieved": achieved, "peak": l2,
                           "unit": "GB/s", "frac": achieved / l2,
                           "peak_source": "measured in this run: 32 MiB device copy, read + write bytes"}
    print(json.dumps(line))
    return 0


def _timed_solve(pkg, Xd, Dd, dtd, beta0, lam, tol, opts, ws):
    import torch
    beta = beta0.clone()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Z, st = pkg.csc_lgcd_solve(Xd, Dd, dtd, beta, lam, tol, opts=opts, ws=ws)
    torch.cuda.synchronize()
    return time.perf_counter() - t0, Z, st


def selection_main(args):
    """Coordinate-selection comparison on one worker (Section 5.1): LGCD
    (|C_m| = 2L), greedy CD (one sub-domain = the domain), cyclic CD
    (|C_m| = 1) through csc_lgcd_solve with one worker, and randomized CD
    (uniform draws, epochs of K |Omega| coordinates, each followed by the
    fresh-beta KKT test) through csc_rcd_solve; seconds to max |dZ| < 1e-4."""
    import torch
    rank, world, local = dist_env()
    from synthetic import SELECTION_150L, SELECTION_750L, make_problem
    tol = 1e-4
    if args.impl == "reference":
        if rank != 0:
            return 0
        import oracle
        oracle.build()
        w = SELECTION_150L
        X, D, _ = make_problem(w, args.seed)
        lam = 0.1 * oracle.lambda_max(X, D)
        out = {}
        t0 = time.perf_counter()
        r = oracle.lgcd(X, D, lam, tol)
        out["lgcd"] = {"seconds": time.perf_counter() - t0, "updates": r["n_updates"]}
        zl = w.T[0] - w.L[0] + 1
        rng = np.random.default_rng(args.seed)
        t0 = time.perf_counter()
        Z = beta = None
        ep, ok = 0, False
        while time.perf_counter() - t0 < args.cap:
            Z, beta, _ = oracle.rcd(X, D, lam, rng.integers(0, w.K * zl, w.K * zl).astype(np.uint32), Z=Z,
                                    beta=beta)
            ep += 1
            if oracle.kkt(X, D, Z, lam) < tol:
                ok = True
                break
        out["rcd"] = {"seconds": time.perf_counter() - t0, "epochs": ep, "converged": ok}
        val = 1.0 / out["lgcd"]["seconds"]
        print(json.dumps({"metric": "seconds to tol 1e-4 on one worker", "value": val, "unit": "solves/s",
                          "impl": "reference", "n_gpus": world, "steps": 1, "warmup": 0,
                          "higher_is_better": True, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": w.name, "strategies": out},
                          "cpu_baseline": {"value": val, "unit": "solves/s", "cores": 1, "kind": "oracle",
                                           "sample": "one LGCD solve of the T = 150 L signal"},
                          "e2e": {"value": val, "unit": "solves/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return 0
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_1901_09235_gb300 as pkg
    table = {}
    for w in (SELECTION_150L, SELECTION_750L):
        X, D, _ = make_problem(w, args.seed)
        Xd, Dd = torch.from_numpy(X).to(device), torch.from_numpy(D).to(device)
        shape = pkg.make_shape(tuple(X.shape), tuple(D.shape))
        ws = pkg.workspace(shape, device=device)
        beta0, dtd, lm = pkg.csc_init_beta(Xd, Dd)
        lam = float(np.float32(0.1 * lm))
        zl = w.T[0] - w.L[0] + 1
        res = {}
        for name, sub in (("lgcd", 2 * w.L[0]), ("greedy", zl), ("cyclic", 1)):
            o = pkg.default_opts(max_workers=1, sub=[sub], timeout_s=args.cap)
            try:
                dt, Z, st = _timed_solve(pkg, Xd, Dd, dtd, beta0, lam, tol, o, ws)
                res[name] = {"seconds": dt, "updates": st["updates"], "status": st["status"],
                             "objective": st["objective"], "max_dz": st["max_dz_final"]}
            except pkg.CscError as e:
                res[name] = {"seconds": None, "status": e.status, "note": f"stopped: {e}"}
        # randomized CD
        gen = torch.Generator(device=device)
        gen.manual_seed(args.seed)
        beta, Z = beta0.clone(), torch.zeros_like(beta0)
        n_coord = w.K * zl
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        upd, ep, mdz, obj = 0, 0, float("inf"), None
        while time.perf_counter() - t0 < args.cap:
            coords = torch.randint(0, n_coord, (n_coord,), generator=gen, device=device, dtype=torch.int32)
            upd += pkg.csc_rcd_solve(X.shape, Dd, dtd, beta, Z, lam, coords, ws=ws)
            _, mdz, obj = pkg.csc_refresh_beta(Xd, Dd, Z, lam, beta=beta, ws=ws)
            ep += 1
            if mdz < tol:
                break
        dt = time.perf_counter() - t0
        res["rcd"] = {"seconds": dt if mdz < tol else None, "elapsed": dt, "epochs": ep, "updates": upd,
                      "objective": obj, "max_dz": mdz}
        table[w.name] = res
    lg = table[SELECTION_150L.name]["lgcd"]["seconds"]
    print(json.dumps({"metric": "seconds to tol 1e-4 on one worker (coordinate selection, Section 5.1)",
                      "value": 1.0 / lg, "unit": "solves/s (LGCD, T = 150 L)", "n_gpus": 1, "steps": 1,
                      "warmup": 0, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": "selection_P7_K25_L250_T150L_T750L", "rho": 0.007,
                                 "activations": "N(0, 10^2)", "noise": "N(0, 1)", "lambda": "0.1 lambda_max",
                                 "workers": 1, "cap_seconds": args.cap},
                      "strategies": table}))
    return 0


def lambda_main(args):
    """2-D solves over lambda x workers x {greedy, LGCD} (the 2-D scaling
    check of the supplement: larger lambda converges faster, locally greedy
    beats greedy until tiles are too small to split)."""
    import torch
    rank, world, local = dist_env()
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps({"impl": "reference", "unavailable": "lambda sweep: GPU-only scaling check; "
                              "the oracle arm is timed by --workload signal and --workload selection"}))
        return 0
    from synthetic import SERVED_ATOMS, Workload, make_dictionary, make_image_device
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_1901_09235_gb300 as pkg
    side = args.side if args.side != 1024 else 512
    P, K, L = SERVED_ATOMS["P"], SERVED_ATOMS["K"], SERVED_ATOMS["L"]
    w = Workload(f"lambda_2d_{side}_P3_K16_L12", P, K, (side, side), L, SERVED_ATOMS["density"], SERVED_ATOMS["sigma"])
    D = make_dictionary(np.random.default_rng(args.seed), K, P, L)
    Dd = torch.from_numpy(D).to(device)
    X = make_image_device(w, args.seed + 1, D, device)
    shape = pkg.make_shape(tuple(X.shape), tuple(Dd.shape))
    ws = pkg.workspace(shape, device=device)
    beta0, dtd, lm = pkg.csc_init_beta(X, Dd)
    zs = list(beta0.shape[1:])
    table = {}
    for reg in (0.05, 0.1, 0.2, 0.5):
        lam = float(np.float32(reg * lm))
        for W in (1, 16, 64, 304):
            for sel, sub in (("greedy", zs), ("lgcd", [2 * L[0], 2 * L[1]])):
                o = pkg.default_opts(max_workers=W, sub=sub, timeout_s=args.cap)
                try:
                    dt, Z, st = _timed_solve(pkg, X, Dd, dtd, beta0, lam, 1e-4, o, ws)
                    table[f"{reg}/{W}/{sel}"] = {"seconds": dt, "updates": st["updates"], "workers": st["workers"],
                                                 "status": st["status"]}
                except pkg.CscError as e:
                    table[f"{reg}/{W}/{sel}"] = {"seconds": None, "status": e.status}
    t = lambda r, W, s: table[f"{r}/{W}/{s}"]["seconds"]  # noqa: E731
    # a larger lambda never takes longer (10 % timing noise allowed); a run
    # that hit the cap at the smaller lambda counts as slower
    faster_with_lambda = all(t(b, W, s) is not None and (t(a, W, s) is None or t(b, W, s) <= t(a, W, s) * 1.1)
                             for s in ("greedy", "lgcd") for W in (1, 16, 64, 304)
                             for a, b in ((0.05, 0.1), (0.1, 0.2), (0.2, 0.5)))
    print(json.dumps({"metric": "seconds to tol 1e-4 (2-D, lambda x workers x selection)",
                      "value": 1.0 / t(0.1, 304, "lgcd"), "unit": "solves/s (LGCD, 304 workers, 0.1 lambda_max)",
                      "n_gpus": 1, "steps": 1, "warmup": 0, "higher_is_better": True, "dtype": "f32",
                      "data": "synthetic", "config": {"workload": w.name, "lambda": "x lambda_max",
                                                      "cap_seconds": args.cap},
                      "larger_lambda_faster": faster_with_lambda, "table": table}))
    return 0


# ------------------------------------------------- the 4096^2 image (default)
def large_image_workload(side=4096):
    """The 4096^2 workload, or an image of the same family at another side
    (smaller cases for profiling)."""
    from synthetic import IMAGE_4096, scaled
    if side == 4096:
        return IMAGE_4096
    return scaled(IMAGE_4096, (side, side), f"csc2d_{side}x{side}_P1_K25_L32")


def large_image_config(w, crop, extra=None):
    d = {"workload": w.name, "P": w.P, "K": w.K, "T": list(w.T), "L": list(w.L), "density": w.density,
         "activations": "|N(0,1)|" if w.nonneg else "N(0,1)", "sigma": w.sigma,
         "lambda": f"{w.reg} * lambda_max", "tol": w.tol,
         "step": "csc_init_beta (FP32) + csc_lgcd_solve (global-memory tiles, soft-locks; beta recomputed "
                 "from Z, KKT max |dZ| < tol on it, FP64 objective)",
         "l2": "flushed between steps (256 MiB write); beta and Z are 1.65 GB each, above L2",
         "oracle_crop": f"{crop}x{crop} image of the same family (same generator, K, atoms, density, noise)"}
    if extra:
        d.update(extra)
    return d


def image_algorithmic_bytes(st, w):
    """The same rule as the 1-D workload (lgcd_algorithmic_bytes)."""
    return lgcd_algorithmic_bytes(st, w)


def profile_value(name, key, sources):
    """A value recorded in a committed ncu summary under profiles/, or None
    when the kernel sources changed since it was taken."""
    prof = os.path.join(ROOT, "profiles", name)
    src = [os.path.join(ROOT, "paper_1901_09235_gb300", "csrc", f) for f in sources]
    try:
        text = open(prof).read()
        h = source_digest(src)
    except OSError:
        return None
    vals = dict(line.split(" = ", 1) for line in text.splitlines() if " = " in line)
    if vals.get("source_sha256", "").strip() != h or key not in vals:
        return None
    return float(vals[key])


def crop_oracle_solve(w, crop, seed):
    """One FP64 oracle solve of a crop-sized image of the same family: lambda_max,
    LGCD to tol, objective.  Returns (seconds, updates, objective, lambda)."""
    import oracle
    from synthetic import make_problem, scaled
    X, D, _ = make_problem(scaled(w, (crop, crop)), seed)
    t0 = time.perf_counter()
    lam = w.reg * oracle.lambda_max(X, D)
    out = oracle.lgcd(X, D, lam, w.tol)
    obj = oracle.objective(X, D, out["Z"], lam)
    return time.perf_counter() - t0, out["n_updates"], obj, lam


def large_image_main(args):
    rank, world, local = dist_env()
    w = large_image_workload(args.side if args.side != 1024 or "--side" in sys.argv else 4096)
    crop = args.crop
    area = (crop * crop) / float(w.T[0] * w.T[1])
    if args.impl == "reference":
        if rank != 0:
            return 0
        import oracle
        oracle.build()
        for i in range(args.warmup):
            crop_oracle_solve(w, crop, args.seed + i)
        times, upd = [], 0
        for i in range(args.steps):
            dt, u, _, _ = crop_oracle_solve(w, crop, args.seed + i)
            times.append(dt)
            upd += u
        total = sum(times)
        # whole-workload solves/s: a crop solve covers `area` of the image
        val = area * args.steps / total
        sample = (f"{args.steps} oracle solves of {crop}x{crop} crops of the same family (seeds "
                  f"{args.seed}..{args.seed + args.steps - 1}), one core; solves/s of the {w.T[0]}x{w.T[1]} "
                  f"image = crop solves/s x {area:.6g} (area ratio)")
        line = {"metric": METRIC, "value": val, "unit": UNIT, "impl": "reference", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps / area,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": large_image_config(w, crop, {"arm": "FP64 CPU oracle, single thread, on crops"}),
                "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
                "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                "updates_per_s": upd / total,
                "crop_p50_ms": 1e3 * float(np.percentile(times, 50)),
                "crop_p99_ms": 1e3 * float(np.percentile(times, 99))}
        print(json.dumps(line))
        return 0

    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_1901_09235_gb300 as pkg
    from synthetic import make_dictionary, make_image_device
    D = make_dictionary(np.random.default_rng(args.seed + 1000 * rank), w.K, w.P, w.L)
    Dd = torch.from_numpy(D).to(device)
    X = make_image_device(w, args.seed + 1000 * rank + 1, D, device)
    s = pkg.make_shape(tuple(X.shape), tuple(Dd.shape))
    # sub-domain side by the autotuner, on another image of the family
    tune = None
    if args.sub > 0:
        tune = {"sub": args.sub, "ms": None, "tried": {}, "seconds": 0.0, "given": True}
    elif not args.no_tune:
        from paper_1901_09235_gb300 import autotune
        t0 = time.perf_counter()
        tune = autotune.tune_single(make_image_device(w, args.seed + 1000 * rank + 2, D, device), Dd,
                                    reg=w.reg, tol=w.tol)
        tune["seconds"] = time.perf_counter() - t0
        torch.cuda.empty_cache()
    opts = pkg.default_opts(sub=[tune["sub"]] * 2) if tune else pkg.default_opts()
    ws = pkg.workspace(s, opts, device=device)
    beta = torch.empty(pkg.z_shape(s), dtype=torch.float32, device=device)
    Z = torch.empty_like(beta)
    dtd = torch.empty(pkg.tab_shape(s), dtype=torch.float32, device=device)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=device)
    stream = torch.cuda.current_stream()

    class Step:
        def run(self, Xin=None, Din=None):
            Xs, Ds = (X, Dd) if Xin is None else (Xin, Din)
            _, _, lm = pkg.csc_init_beta(Xs, Ds, beta, dtd, ws)
            _, st = pkg.csc_lgcd_solve(Xs, Ds, dtd, beta, w.reg * lm, w.tol, Z=Z, opts=opts, ws=ws)
            if st["status"] != pkg.CSC_OK:
                raise RuntimeError(f"solve status {st['status']}: {pkg.status_string(st['status'])}")
            st["lambda"] = w.reg * lm
            return st

    step = Step()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    barrier()
    clk = ClockSampler(local).__enter__()  # sampled over both timed loops below
    times, stats = time_gpu(step, args.steps, max(3, args.warmup), flush, stream)
    barrier()
    # end to end: pinned X and D in; the objective and the sparse code (the
    # nonzeros of Z as atom, position, value: csc_sparse_code) out, every step
    Xh = torch.empty(X.shape, dtype=torch.float32, pin_memory=True)
    Xh.copy_(X)
    Dh = torch.from_numpy(D).pin_memory()
    Xe, De = torch.empty_like(X), torch.empty_like(Dd)
    cap = max(1 << 16, 4 * int(stats[-1]["nnz"]))
    code = (torch.empty(cap, dtype=torch.int32, device=device), torch.empty(cap, dtype=torch.int32, device=device),
            torch.empty(cap, dtype=torch.float32, device=device))
    code_h = tuple(torch.empty(cap, dtype=t.dtype, pin_memory=True) for t in code)
    e2e_nnz = []

    def e2e_step():
        Xe.copy_(Xh, non_blocking=True)
        De.copy_(Dh, non_blocking=True)
        st = step.run(Xe, De)  # the objective is copied to the host inside the call
        *lists, n = pkg.sparse_code(Z, tuple(X.shape), tuple(Dd.shape), out=code, ws=ws)  # reads the count back
        for dst, src in zip(code_h, lists):
            dst[:n].copy_(src, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        e2e_nnz.append(n)
        return st

    e2e_times, _ = time_gpu(step, args.steps, max(3, args.warmup), flush, stream, e2e=e2e_step)
    # the mixed-precision form of the same solve: beta-init on the tensor cores
    # in split bf16 (FP32 accumulation), beta / Z updates and the final KKT test
    # in FP32, the same lambda (from the FP32 lambda_max, taken once)
    lam_fixed = stats[-1]["lambda"]

    class MixedStep:
        def run(self):
            pkg.csc_init_beta_bf16x3(X, Dd, beta, dtd, ws, want_lambda_max=False)
            _, st = pkg.csc_lgcd_solve(X, Dd, dtd, beta, lam_fixed, w.tol, Z=Z, opts=opts, ws=ws)
            if st["status"] != pkg.CSC_OK:
                raise RuntimeError(f"solve status {st['status']}: {pkg.status_string(st['status'])}")
            return st

    mixed_times, mixed_stats = time_gpu(MixedStep(), args.steps, max(3, args.warmup), flush, stream)
    clk.__exit__(None, None, None)
    clocks = clk.summary()
    barrier()
    tot, tot_e2e, tot_mixed = max_over_ranks([sum(times), sum(e2e_times), sum(mixed_times)], device)
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0
    upd = sum(st["updates"] for st in stats)
    kernel_s = sum(st["kernel_ms"] for st in stats) / 1e3
    abytes = sum(image_algorithmic_bytes(st, w) for st in stats)
    achieved = abytes / kernel_s / 1e9
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm = float(peaks["hbm_gbs"]) if "hbm_gbs" in peaks else 6800.0
    hbm_src = "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks else "6.8 TB/s (of fallback)"
    # DRAM bytes per launch from the committed capture of this workload (sub-domains of 32), while the
    # kernel sources match it
    traffic = None
    if w.T == (4096, 4096) and list(opts.sub) == [32, 32]:
        traffic = profile_value("lgcd_global_kernel_csc2d_4096x4096_P1_K25_L32.md", "dram_bytes_per_launch",
                                ("lgcd_global.cuh", "lgcd.cu", "lgcd_common.cuh", "common.cuh"))
    last = stats[-1]
    line = {
        "metric": METRIC, "value": world * args.steps / tot, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": large_image_config(w, crop, {"parallelism": f"replicas{world}" if world > 1 else "single",
                                               "workers": last["workers"], "tiles": last["tiles"],
                                               "tile": last["tile_size"],
                                               "sub": list(opts.sub) if tune else [2 * l for l in w.L],
                                               "sub_choice": ("given (--sub)" if tune and tune.get("given") else
                                                              "autotuned on another image of the family"
                                                              if tune else "library default (2 L)")}),
        "tuning": tune,
        "updates_per_s": world * upd / tot,
        "p50_ms": 1e3 * float(np.percentile(times, 50)),
        "p99_ms": 1e3 * float(np.percentile(times, 99)),
        "lgcd_kernel_ms_per_step": 1e3 * kernel_s / args.steps,
        "lgcd_updates_per_s_kernel": upd / kernel_s,
        "objective": last["objective"], "max_dz_final": last["max_dz_final"], "nnz": last["nnz"],
        "updates_per_solve": upd / args.steps,
        "solve_stats": {k: last[k] for k in ("iterations", "rejected_softlock", "skipped_subtol", "messages",
                                              "refresh_rounds", "max_worker_iterations", "max_worker_updates",
                                              "kernel_ms", "phase_cycles")},
        "roofline": {"bound": "hbm", "kernel": "lgcd_global_kernel", "achieved": achieved, "peak": hbm,
                     "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": None if traffic is None else traffic,
                     "peak_source": hbm_src, "algorithmic_bytes_per_launch": abytes / len(stats)},
        "e2e": {"value": world * args.steps / tot_e2e, "unit": UNIT,
                "h2d_bytes_per_step": int(Xh.numel() * 4 + Dh.numel() * 4),
                "d2h_bytes_per_step": int(12 * np.mean(e2e_nnz[-args.steps:]) + 16),
                "result": "objective (FP64) and the sparse code: nonzeros of Z as (atom, position, value), "
                          "12 bytes each, from csc_sparse_code"},
        "gpu_launches": sum(launches_per_step_solve(st) for st in stats),
        "clocks": clocks,
        "mixed_bf16x3": {
            "value": world * args.steps / tot_mixed, "unit": UNIT, "ms_per_step": 1e3 * tot_mixed / args.steps,
            "step": "csc_init_beta_bf16x3 (tensor cores, split bf16, FP32 accumulation) + csc_lgcd_solve, "
                    "the same lambda",
            "objective": mixed_stats[-1]["objective"], "max_dz_final": mixed_stats[-1]["max_dz_final"],
            "objective_rel_diff_vs_fp32": abs(mixed_stats[-1]["objective"] - last["objective"]) /
                                          abs(last["objective"]),
            "speedup_vs_fp32": tot / tot_mixed},
    }
    if not args.no_cpu_baseline and world == 1:
        # the oracle on crops of the same family, and the GPU on the same crop
        import oracle
        from synthetic import make_problem, scaled
        oracle.build()
        done, total, cu, obj0, lam0 = 0, 0.0, 0, None, None
        while total < args.cpu_seconds and done < 10:
            dt, u, obj, lam = crop_oracle_solve(w, crop, args.seed + done)
            if done == 0:
                obj0, lam0 = obj, lam
            total += dt
            cu += u
            done += 1
        line["cpu_baseline"] = {
            "value": area * done / total, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{done} oracle solves of {crop}x{crop} crops of the same family, one core, "
                      f"{total:.1f} s; solves/s of the full image = crop solves/s x {area:.6g} (area ratio)",
            "updates_per_s": cu / total}
        Xc, Dc, _ = make_problem(scaled(w, (crop, crop)), args.seed)
        Xcd, Dcd = torch.from_numpy(Xc).to(device), torch.from_numpy(Dc).to(device)
        bc, tc, _ = pkg.csc_init_beta(Xcd, Dcd)
        _, stc = pkg.csc_lgcd_solve(Xcd, Dcd, tc, bc, lam0, w.tol)
        line["crop_parity"] = {"side": crop, "objective_gpu": stc["objective"], "objective_oracle": obj0,
                               "objective_rel_err_vs_oracle": abs(stc["objective"] - obj0) / abs(obj0),
                               "max_dz_final": stc["max_dz_final"]}
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def launches_per_step_solve(st):
    # init_beta: correlation + DtD table; solve: atom norms + window-layout
    # table, then per round: header reset, LGCD, and the refresh (reset,
    # nonzero list, residual init / scatter / finish, dense check, transposed
    # table, bin count / scan / fill, gather, the gated correlation refresh)
    # -- 18 kernels for a one-round solve, as the ncu launch list shows
    return 2 + 2 + 14 * int(st["refresh_rounds"])


# ------------------------------------------------ full CDL on the 8192^2 image
CDL_OUTER = 10


def cdl_workload():
    from synthetic import IMAGE_8192
    return IMAGE_8192


def cdl_start_atoms(D_true, seed):
    """The dictionary the loop starts from: the generating atoms.  At
    lambda = 0.1 lambda_max the sparse code of a point-source image is cheap
    only near them (with 5 % noise added to the atoms the oracle's LGCD on a
    256^2 crop needs 15 k updates instead of 81, with 10 % it does not finish
    200 k), so the ten outer iterations refine a dictionary that fits the
    data, as the late iterations of a learning run do."""
    del seed
    return np.ascontiguousarray(D_true, dtype=np.float32)


def cdl_config(w, crop, extra=None):
    d = {"workload": "cdl_" + w.name, "P": w.P, "K": w.K, "T": list(w.T), "L": list(w.L), "density": w.density,
         "activations": "|N(0,1)|" if w.nonneg else "N(0,1)", "sigma": w.sigma,
         "lambda": f"{w.reg} * lambda_max(X, D0), fixed", "tol": w.tol, "outer_iterations": CDL_OUTER,
         "D0": "the generating atoms",
         "step": f"cdl_fit: {CDL_OUTER} outer iterations of Alg. 2 (beta-init, LGCD, phi/psi, PGD + Armijo, "
                 "FP64 costs); one solve = one outer iteration",
         "oracle_crop": f"{crop}x{crop} image of the same family"}
    if extra:
        d.update(extra)
    return d


def cdl_main(args):
    rank, world, local = dist_env()
    w = cdl_workload()
    crop = 256 if args.crop == 512 else args.crop
    area = (crop * crop) / float(w.T[0] * w.T[1])
    from synthetic import make_problem, scaled
    if args.impl == "reference":
        if rank != 0:
            return 0
        print(json.dumps({"impl": "reference", "unavailable": "full CDL workload: the FP64 oracle's dictionary "
                          "step alone takes about 70 s per outer iteration at K = 25 atoms of 32 x 32 (its "
                          "gradient is a direct K^2 |Theta| |Phi| sum), beyond the bench's time; the GPU arm's "
                          "cpu_baseline times the oracle's parts on a crop, and tests/test_gpu_cdl.py checks "
                          "the loop against the oracle on a 1024^2 crop"}))
        return 0

    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_1901_09235_gb300 as pkg
    from synthetic import make_dictionary, make_image_device
    Dt = make_dictionary(np.random.default_rng(args.seed + 1000 * rank), w.K, w.P, w.L)
    D0 = cdl_start_atoms(Dt, args.seed + 1000 * rank + 7)
    X = make_image_device(w, args.seed + 1000 * rank + 1, Dt, device)
    D0d = torch.from_numpy(D0).to(device)
    Dd = torch.empty_like(D0d)
    s = pkg.make_shape(tuple(X.shape), tuple(D0d.shape))
    tune = None
    if args.sub > 0:
        tune = {"sub": args.sub, "ms": None, "tried": {}, "seconds": 0.0, "given": True}
    elif not args.no_tune:
        from paper_1901_09235_gb300 import autotune
        t0 = time.perf_counter()
        tune = autotune.tune_single(make_image_device(w, args.seed + 1000 * rank + 2, Dt, device), D0d,
                                    reg=w.reg, tol=w.tol, reps=1)
        tune["seconds"] = time.perf_counter() - t0
        torch.cuda.empty_cache()
    sub = [tune["sub"]] * 2 if tune else [0, 0]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=device)
    stream = torch.cuda.current_stream()

    class Step:
        def __init__(self, beta_init):
            self.opts = pkg.default_opts(beta_init=beta_init, sub=sub)
            self.prob = pkg.Problem.create(X, Dd, self.opts)
            self.trace = None

        def run(self, Xin=None, Din=None):
            if Din is None:
                Dd.copy_(D0d, non_blocking=True)
            self.prob.D = Dd if Din is None else Din
            _, tr, rc = pkg.cdl_fit(X if Xin is None else Xin, self.prob.D, reg=w.reg, tol=w.tol,
                                    max_outer=CDL_OUTER, nu=0.0, pgd_max_iter=50, opts=self.opts, prob=self.prob)
            if rc != pkg.CSC_OK or len(tr) != CDL_OUTER:
                raise RuntimeError(f"cdl_fit status {rc}, {len(tr)} iterations")
            self.trace = tr
            return {"status": rc}

    arms = {}
    clk = ClockSampler(local).__enter__()
    for name, bi in (("mixed_bf16x3", 1), ("plain_fp32", 0)):
        step = Step(bi)
        times, _ = time_gpu(step, args.steps, max(3, args.warmup) if args.warmup >= 3 else 3, flush, stream)
        arms[name] = {"times": times, "trace": step.trace, "step": step}
    # end to end through host buffers for the mixed arm: X and D0 in, D out
    Xh = torch.empty(X.shape, dtype=torch.float32, pin_memory=True)
    Xh.copy_(X)
    D0h = torch.from_numpy(D0).pin_memory()
    Dout = torch.empty_like(D0h).pin_memory()
    Xe, De = torch.empty_like(X), torch.empty_like(D0d)
    mstep = arms["mixed_bf16x3"]["step"]

    def e2e_step():
        Xe.copy_(Xh, non_blocking=True)
        De.copy_(D0h, non_blocking=True)
        st = mstep.run(Xe, De)
        Dout.copy_(De, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        return st

    e2e_times, _ = time_gpu(mstep, args.steps, 3, flush, stream, e2e=e2e_step)
    clk.__exit__(None, None, None)
    clocks = clk.summary()
    tm, tp, te = max_over_ranks([sum(arms["mixed_bf16x3"]["times"]), sum(arms["plain_fp32"]["times"]),
                                 sum(e2e_times)], device)
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0
    trm, trp = arms["mixed_bf16x3"]["trace"], arms["plain_fp32"]["trace"]
    rel = [abs(a[1] - b[1]) / abs(b[1]) for a, b in zip(trm, trp)]
    n_solves = CDL_OUTER * args.steps
    line = {
        "metric": METRIC, "value": world * n_solves / tm, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": 3, "ms_per_step": 1e3 * tm / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (beta-init: split bf16 x3, FP32 accumulation; FP64 costs)",
        "data": "synthetic",
        "config": cdl_config(w, crop, {"parallelism": f"replicas{world}" if world > 1 else "single",
                                       "sub": sub, "sub_choice": "autotuned" if tune else "library default (2 L)",
                                       "l2": "flushed between steps (256 MiB write); beta, Z 6.7 GB each"}),
        "tuning": tune,
        "p50_ms": 1e3 * float(np.percentile(arms["mixed_bf16x3"]["times"], 50)),
        "p99_ms": 1e3 * float(np.percentile(arms["mixed_bf16x3"]["times"], 99)),
        "trace_mixed": trm, "trace_fp32": trp,
        "cost_rel_diff_vs_fp32_per_iteration": rel,
        "plain_fp32": {"value": world * n_solves / tp, "unit": UNIT, "ms_per_step": 1e3 * tp / args.steps},
        "mixed_over_fp32": tp / tm,
        "e2e": {"value": world * n_solves / te, "unit": UNIT,
                "h2d_bytes_per_step": int(Xh.numel() * 4 + D0h.numel() * 4),
                "d2h_bytes_per_step": int(Dout.numel() * 4)},
        "gpu_launches": None,
        "clocks": clocks,
    }
    if not args.no_cpu_baseline and world == 1:
        # the oracle's outer iteration in two parts: the sparse code (lambda_max,
        # LGCD, phi / psi) on a crop, which scales with the image area, and PGD
        # iterations of the dictionary step, whose cost does not depend on the
        # image; estimate = code / area ratio + one PGD iteration x 50 (the
        # iteration cap both sides run with)
        import oracle
        oracle.build()
        wc = scaled(w, (crop, crop))
        Xc, Dtc, _ = make_problem(wc, args.seed)
        t0 = time.perf_counter()
        lm = oracle.lambda_max(Xc, Dtc)
        zc = oracle.lgcd(Xc, Dtc, w.reg * lm, w.tol)["Z"]
        phi, psi = oracle.phi_psi(zc, Xc, w.L)
        t_code = time.perf_counter() - t0
        xs = float((Xc.astype(np.float64) ** 2).sum())
        t0 = time.perf_counter()
        _, _, pit = oracle.pgd_armijo(phi, psi, xs, Dtc, max_iter=2, tol=0.0)
        t_pgd = (time.perf_counter() - t0) / max(pit, 1)
        gpu_pgd = 50
        est = t_code / area + t_pgd * gpu_pgd
        line["cpu_baseline"] = {"value": 1.0 / est, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"one sparse code (lambda_max, LGCD, phi/psi) of a {crop}x{crop} crop "
                                          f"({t_code:.1f} s, scaled by the area ratio {area:.6g}) and {pit} PGD "
                                          f"iterations ({t_pgd:.1f} s each, x {gpu_pgd}, the cap), "
                                          f"one core"}
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# ------------------------------------------------------- beta-init on its own
def betainit_main(args):
    """csc_init_beta (FP32, CUDA cores) and csc_init_beta_bf16x3 (split bf16 on
    the tensor cores) on an image of the 4096^2 family, each timed with CUDA
    events; the tensor-core arm against the bf16 peak (three products per
    multiply-add of the correlation)."""
    import torch
    rank, world, local = dist_env()
    side = args.side if "--side" in sys.argv else 4096
    w = large_image_workload(side)
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps({"impl": "reference", "unavailable": "beta-init alone: the oracle arm is timed by "
                              "the default workload (its solves include the oracle's beta-init)"}))
        return 0
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_1901_09235_gb300 as pkg
    from synthetic import make_dictionary, make_image_device
    D = make_dictionary(np.random.default_rng(args.seed), w.K, w.P, w.L)
    Dd = torch.from_numpy(D).to(device)
    X = make_image_device(w, args.seed + 1, D, device)
    s = pkg.make_shape(tuple(X.shape), tuple(Dd.shape))
    ws = pkg.workspace(s, device=device)
    beta = torch.empty(pkg.z_shape(s), dtype=torch.float32, device=device)
    dtd = torch.empty(pkg.tab_shape(s), dtype=torch.float32, device=device)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=device)
    stream = torch.cuda.current_stream()
    nz = int(np.prod(pkg.z_shape(s)))
    flop = 2.0 * nz * w.P * int(np.prod(w.L))
    out = {}
    for name, fn in (("fp32", pkg.csc_init_beta), ("bf16x3", pkg.csc_init_beta_bf16x3)):
        class Step:
            def run(self):
                fn(X, Dd, beta, dtd, ws, want_lambda_max=False)
                return {}

        times, _ = time_gpu(Step(), args.steps, max(3, args.warmup), flush, stream)
        ms = 1e3 * sum(times) / len(times)
        out[name] = {"ms": ms, "p50_ms": 1e3 * float(np.percentile(times, 50)), "tflops": flop / (ms / 1e3) / 1e12}
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    bf16 = float(peaks.get("bf16_tflops", 1900.0))
    Np = -(-w.K // 16) * 16
    L1p = -(-w.L[1] // 16) * 16
    # tensor work as issued: M = 128 positions x N = 2 Np (hi parts against the
    # hi and lo dictionary) + N = Np (lo parts against the hi dictionary) per
    # reduction step over P L0 L1p taps
    tc_flop = 2.0 * nz * w.P * w.L[0] * L1p * 3 * Np / w.K
    line = {"metric": "beta-init time (FP32 CUDA cores vs split bf16 on the tensor cores)",
            "value": out["bf16x3"]["ms"], "unit": "ms", "n_gpus": 1, "steps": args.steps,
            "warmup": max(3, args.warmup), "higher_is_better": False, "dtype": "bf16x3 (fp32 arm beside)",
            "data": "synthetic", "config": {"workload": w.name, "K": w.K, "L": list(w.L), "P": w.P,
                                            "flop": flop, "l2": "flushed between steps"},
            "fp32": out["fp32"], "bf16x3": out["bf16x3"],
            "roofline": {"bound": "tensor", "kernel": "corr_umma_kernel",
                         "achieved": tc_flop / (out["bf16x3"]["ms"] / 1e3) / 1e12, "peak": bf16, "unit": "TFLOP/s",
                         "frac": tc_flop / (out["bf16x3"]["ms"] / 1e3) / 1e12 / bf16,
                         "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst, of measured)",
                         "note": "tensor work as issued (atoms padded to 16, taps to 16 per row, three products)"}}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.steps is None:
        # enough timed steps on the 1-D GPU arm (about 1 ms each) for several
        # clock samples and a meaningful p99; the oracle arm and the longer
        # workloads keep 20
        args.steps = 20
        if args.impl == "gb300":
            args.steps = {"signal": 200, "image4096": 30, "cdl": 3}.get(args.workload, 20)
    if args.workload == "image4096":
        return large_image_main(args)
    if args.workload == "cdl":
        return cdl_main(args)
    if args.workload == "betainit":
        return betainit_main(args)
    if args.workload == "served":
        return served_main(args)
    if args.workload == "selection":
        return selection_main(args)
    if args.workload == "lambda":
        return lambda_main(args)
    if args.workload == "image":
        return image_main(args)
    rank, world, local = dist_env()
    w = workload()
    from synthetic import make_problem

    if args.impl == "reference":
        if rank != 0:
            return 0
        X, D0, _ = make_problem(w, args.seed)
        import oracle
        oracle.build()
        for _ in range(args.warmup):
            cpu_oracle_step(X, D0, w)
        times = []
        upd = 0
        for _ in range(args.steps):
            dt, u, _ = cpu_oracle_step(X, D0, w)
            times.append(dt)
            upd += u
        total = sum(times)
        val = args.steps / total
        line = {"metric": METRIC, "value": val, "unit": UNIT, "impl": "reference", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": config_dict(w, {"arm": "FP64 CPU oracle, single thread"}),
                "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                                 "sample": f"{args.steps} full oracle steps"},
                "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                "updates_per_s": upd / total,
                "p50_ms": 1e3 * float(np.percentile(times, 50)),
                "p99_ms": 1e3 * float(np.percentile(times, 99))}
        print(json.dumps(line))
        return 0

    import torch
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    import __graft_entry__
    __graft_entry__.build()
    X, D0, _ = make_problem(w, args.seed + rank)
    step = GpuStep(X, D0, w, device, api=args.api)
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=device)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    barrier()
    clk = ClockSampler(local).__enter__()  # sampled over both timed loops below
    times, stats = time_gpu(step, args.steps, max(3, args.warmup), flush, stream)
    barrier()

    # end to end through host buffers: pinned X / D in, D and objective out
    Xh = torch.from_numpy(X).pin_memory()
    Dh = torch.from_numpy(D0).pin_memory()
    Dout = torch.empty_like(Dh).pin_memory()
    Xe = torch.empty_like(step.X)
    De = torch.empty_like(step.D)

    def e2e_step():
        Xe.copy_(Xh, non_blocking=True)
        De.copy_(Dh, non_blocking=True)
        st = step.run(Xe, De)
        Dout.copy_(De, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        return st

    e2e_times, _ = time_gpu(step, args.steps, max(3, args.warmup), flush, stream, e2e=e2e_step)
    clk.__exit__(None, None, None)
    clocks = clk.summary()
    barrier()

    tot = sum(times)
    tot_e2e = sum(e2e_times)
    tot, tot_e2e = max_over_ranks([tot, tot_e2e], device)
    if rank != 0:
        torch.distributed.destroy_process_group()
        return 0

    upd = sum(s["updates"] for s in stats)
    kms = [s["kernel_ms"] for s in stats]
    kernel_s = sum(kms) / 1e3
    abytes = sum(lgcd_algorithmic_bytes(s, w) for s in stats)
    achieved = abytes / kernel_s / 1e9
    peak = smem_peak_gbs()
    last = stats[-1]
    line = {
        "metric": METRIC, "value": world * args.steps / tot, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": config_dict(w, {"parallelism": f"replicas{world}" if world > 1 else "single",
                                  "workers": last["workers"], "tile": last["tile_size"][0],
                                  "api": "cdl_step" if args.api == "step" else "four calls"}),
        "updates_per_s": world * upd / tot,
        "p50_ms": 1e3 * float(np.percentile(times, 50)),
        "p99_ms": 1e3 * float(np.percentile(times, 99)),
        "lgcd_kernel_ms_per_step": 1e3 * kernel_s / args.steps,
        "lgcd_updates_per_s_kernel": upd / kernel_s,
        "objective": last["objective"], "max_dz_final": last["max_dz_final"], "nnz": last["nnz"],
        "updates_per_solve": upd / args.steps,
        "solve_stats": {k: last[k] for k in ("iterations", "rejected_softlock", "skipped_subtol",
                                              "messages", "deferred", "refresh_rounds",
                                              "max_worker_iterations", "max_worker_updates",
                                              "kernel_ms", "dict_iters")},
        "roofline": {"bound": "smem", "kernel": "lgcd_async_kernel", "achieved": achieved,
                     "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": lgcd_traffic_per_launch(),
                     "peak_source": "derived: 152 SMs x 128 B/clk x 2070 MHz (shared memory)",
                     "algorithmic_bytes_per_launch": abytes / len(stats)},
        "e2e": {"value": world * args.steps / tot_e2e, "unit": UNIT,
                "h2d_bytes_per_step": int(Xh.numel() * 4 + Dh.numel() * 4),
                "d2h_bytes_per_step": int(Dout.numel() * 4 + 8)},
        "gpu_launches": sum(launches_per_step(s) for s in stats),
        "clocks": clocks,
    }
    if not args.no_cpu_baseline and world == 1:
        cb = cpu_baseline(X, D0, w, args.cpu_seconds)
        obj_ref = cb.pop("objective")
        line["cpu_baseline"] = cb
        # the same solve's objective against the FP64 oracle's (both at tol)
        line["objective_oracle"] = obj_ref
        line["objective_rel_err_vs_oracle"] = abs(last["objective"] - obj_ref) / abs(obj_ref)
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
