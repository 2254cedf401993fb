"""Sub-domain and stop-margin autotuner for batched LGCD solves.

The LGCD worker scans one sub-domain C_m per iteration (Alg. 1); Section 3
takes |C_m| of side 2 L, and the soft-lock acceptance analysis of Section 4
ties the rate of rejected border updates to the sub-domain and tile sizes, so
the best size depends on the image size and the atoms.  This tuner times
candidate sub-domain sides (seeded at 2 L: L, 4L/3, 2L, 8L/3, 4L) and stop
margins (the fraction of tol at which workers stop before the fresh-beta
check) for each image-size class, through the persistent queue (the path the
server uses), on synthetic images drawn like the workload, and keeps the
fastest.  A class's cost is the device time of its jobs plus the host time of
each extra refresh round a candidate needs.

The table maps a size class to options; it can be saved to and loaded from
JSON.  Every solve runs in the CUDA library; this module only times them.
"""
from __future__ import annotations

import json
import math
import time

# image-side classes: upper bounds (inclusive); the last class is open
CLASS_BOUNDS = (96, 192, 384, 768, 1536)


def size_class(side: int) -> int:
    for i, b in enumerate(CLASS_BOUNDS):
        if side <= b:
            return i
    return len(CLASS_BOUNDS)


def class_side(c: int, lo: int = 64, hi: int = 2048) -> int:
    """A representative side of class c: the geometric middle of its range."""
    a = lo if c == 0 else CLASS_BOUNDS[c - 1] + 1
    b = CLASS_BOUNDS[c] if c < len(CLASS_BOUNDS) else hi
    return int(round(math.sqrt(a * b)))


def sub_candidates(L: int):
    return sorted({max(L, s) for s in (L, (4 * L + 2) // 3, 2 * L, (8 * L + 2) // 3, 4 * L)})


def opts_for(table: dict, side: int, base=None):
    """SolveOpts for an image of the given side from a tuning table (None or
    a missing class: the library's defaults)."""
    from . import default_opts
    kw = dict(base or {})
    entry = (table or {}).get(str(size_class(side)))
    if entry:
        kw["sub"] = [entry["sub"], entry["sub"]]
        kw["stop_margin"] = entry["stop_margin"]
    return default_opts(**kw)


def save(table: dict, path: str):
    with open(path, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)


def load_table(path: str) -> dict:
    with open(path) as f:
        return json.load(f)


def tune(D, make_image, classes=None, margins=(0.99, 0.95, 0.9), reps: int = 2, reg: float = 0.1,
         tol: float = 1e-4, max_rounds: int = 4, run_seconds: float = 600.0, log=None, ctas_per_sm: int = 0):
    """Tune every class (default: all) for atoms D (K, P, L0, L1) on the
    device, through a queue of the given density (as the server will run it).  make_image(side, seed) returns a device float32 image
    (P, side, side).  Returns {class: {"sub", "stop_margin", "ms", "side",
    "tried": {...}}}."""
    import torch
    from . import Queue, csc_init_beta, csc_refresh_beta, default_opts, make_shape, workspace
    K, P, L0, L1 = D.shape
    if L0 != L1:
        raise ValueError("square atoms only")
    classes = list(range(len(CLASS_BOUNDS) + 1)) if classes is None else list(classes)
    subs = sub_candidates(L0)
    cur = torch.cuda.current_stream(D.device)
    # every buffer is allocated, and every copy warmed up, before the queue
    # starts: nothing may allocate or load a kernel beside the persistent one
    imgs, bufs = {}, {}
    dtd = None
    for c in classes:
        side = class_side(c)
        imgs[c] = []
        for r in range(reps):
            X = make_image(side, 1000 * c + r)
            beta0, dtd, lm = csc_init_beta(X, D)
            imgs[c].append((X, beta0, reg * lm))
        s = make_shape(tuple(imgs[c][0][0].shape), tuple(D.shape))
        beta = torch.empty_like(imgs[c][0][1])
        beta.copy_(imgs[c][0][1])
        bufs[c] = (beta, torch.empty_like(beta), workspace(s, device=D.device))
    cur.synchronize()
    table = {}
    with Queue(D, dtd, max_jobs=len(classes) * len(subs) * len(margins) * reps * (max_rounds + 1) + 8,
               ctl_slots=8, run_seconds=run_seconds, ctas_per_sm=ctas_per_sm) as q:
        for c in classes:
            side = class_side(c)
            beta, Z, ws = bufs[c]
            tried = {}
            for sub in subs:
                for m in margins:
                    o = default_opts(sub=[sub, sub], stop_margin=m)
                    total = 0.0
                    ok = True
                    for X, beta0, lam in imgs[c]:
                        beta.copy_(beta0)
                        cur.synchronize()
                        st = q.wait(q.submit(beta, Z, lam, tol, opts=o), timeout=120.0)
                        total += st["kernel_ms"]
                        for _ in range(max_rounds):
                            if st["status"] != 0:
                                ok = False
                                break
                            t0 = time.perf_counter()
                            _, mdz, _ = csc_refresh_beta(X, D, Z, lam, beta=beta, ws=ws)
                            total += 1e3 * (time.perf_counter() - t0)
                            if mdz < tol:
                                break
                            st = q.wait(q.submit(beta, Z, lam, tol, warm_start=True, opts=o), timeout=120.0)
                            total += st["kernel_ms"]
                        else:
                            ok = False
                    if ok:
                        tried[f"{sub}/{m}"] = total / len(imgs[c])
                    if log:
                        log(f"class {c} (side {side}) sub {sub} margin {m}: "
                            f"{total / len(imgs[c]):.2f} ms{'' if ok else ' (failed)'}")
            if not tried:
                continue
            best = min(tried, key=tried.get)
            bs, bm = best.split("/")
            table[str(c)] = {"sub": int(bs), "stop_margin": float(bm), "ms": tried[best], "side": side,
                             "tried": tried}
    return table


def single_candidates(L: int):
    """Sub-domain sides for single solves: L/2, 3L/4, L, 4L/3 and the paper's 2L."""
    return sorted({max(1, s) for s in (L // 2, (3 * L) // 4, L, (4 * L + 2) // 3, 2 * L)})


def tune_single(X, D, reg: float = 0.1, tol: float = 1e-4, reps: int = 2, candidates=None, log=None):
    """Sub-domain side for single solves (csc_init_beta + csc_lgcd_solve with
    its fresh-beta check) of images like X (P, T0, T1; square atoms): each
    candidate side is timed with CUDA events on the current stream over `reps`
    solves, after one untimed solve, and the fastest is kept.  X should be a
    tuning image drawn like the workload, not the one to be solved.  Returns
    {"sub": side, "ms": mean ms per solve, "tried": {side: ms}}."""
    import torch
    from . import CSC_OK, csc_init_beta, csc_lgcd_solve, default_opts, make_shape, tab_shape, workspace, z_shape
    K, P, L0, L1 = D.shape
    if L0 != L1:
        raise ValueError("square atoms only")
    s = make_shape(tuple(X.shape), tuple(D.shape))
    beta = torch.empty(z_shape(s), dtype=torch.float32, device=X.device)
    Z = torch.empty_like(beta)
    dtd = torch.empty(tab_shape(s), dtype=torch.float32, device=X.device)
    ws = workspace(s, device=X.device)
    tried = {}
    for sub in candidates or single_candidates(L0):
        o = default_opts(sub=[sub, sub])
        ms = []
        for r in range(reps + 1):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            _, _, lm = csc_init_beta(X, D, beta, dtd, ws)
            _, st = csc_lgcd_solve(X, D, dtd, beta, reg * lm, tol, Z=Z, opts=o, ws=ws)
            b.record()
            b.synchronize()
            if st["status"] != CSC_OK:
                break
            if r > 0:
                ms.append(a.elapsed_time(b))
        else:
            tried[sub] = sum(ms) / len(ms)
        if log:
            log(f"sub {sub}: {tried.get(sub, float('nan')):.2f} ms")
    if not tried:
        raise RuntimeError("no sub-domain candidate converged")
    best = min(tried, key=tried.get)
    return {"sub": best, "ms": tried[best], "tried": tried}
