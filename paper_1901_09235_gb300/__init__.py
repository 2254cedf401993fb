"""Python binding of the GB300 CSC library (``include/dicodile_gb.h``).

Argument marshalling only: every step of the computation runs in the CUDA
library ``lib/libdicodile_gb.so``.  Tensors are torch CUDA tensors (float32,
or float64 for the ``_f64`` calls), contiguous, laid out as the header states:

  1-D: X (P, T),      D (K, P, L),      Z / beta (K, T - L + 1)
  2-D: X (P, T0, T1), D (K, P, L0, L1), Z / beta (K, T0 - L0 + 1, T1 - L1 + 1)

Calls are enqueued on the current torch stream.  If the library is missing
the functions raise; there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libdicodile_gb.so")

CSC_OK, CSC_ERR_INVALID, CSC_ERR_CUDA, CSC_NOT_CONVERGED = 0, 1, 2, 3
CSC_ERR_TIMEOUT, CSC_ERR_DIVERGED, CSC_ERR_UNIMPLEMENTED, CSC_ERR_WORKSPACE = 4, 5, 6, 7
MODE_ASYNC, MODE_PHASED, MODE_NOLOCK = 0, 1, 2


class Shape(C.Structure):
    _fields_ = [("d", C.c_int), ("P", C.c_int), ("K", C.c_int),
                ("T", C.c_int * 2), ("L", C.c_int * 2)]


class SolveOpts(C.Structure):
    _fields_ = [("tile", C.c_int * 2), ("sub", C.c_int * 2), ("mode", C.c_int),
                ("max_workers", C.c_int), ("max_updates", C.c_longlong),
                ("timeout_s", C.c_double), ("beta_refresh", C.c_int),
                ("divergence_guard", C.c_int), ("warm_start", C.c_int), ("placement", C.c_int),
                ("beta_init", C.c_int), ("stop_margin", C.c_double)]


class SolveStats(C.Structure):
    _fields_ = [("updates", C.c_longlong), ("iterations", C.c_longlong),
                ("rejected_softlock", C.c_longlong), ("skipped_subtol", C.c_longlong),
                ("messages", C.c_longlong), ("refresh_rounds", C.c_longlong),
                ("workers", C.c_int), ("placement", C.c_int), ("tiles", C.c_int * 2),
                ("tile_size", C.c_int * 2),
                ("max_dz_final", C.c_double), ("objective", C.c_double),
                ("nnz", C.c_longlong), ("kernel_ms", C.c_double), ("deferred", C.c_longlong),
                ("max_worker_iterations", C.c_longlong), ("max_worker_updates", C.c_longlong),
                ("last_active_wave", C.c_longlong), ("t_first_pause_us", C.c_double),
                ("t_exit_us", C.c_double), ("wakeups", C.c_longlong),
                ("phase_cycles", C.c_longlong * 6), ("candidates", C.c_longlong), ("status", C.c_int)]

    _arrays = ("tiles", "tile_size", "phase_cycles")

    def as_dict(self):
        out = {name: getattr(self, name) for name, _ in self._fields_}
        for name in self._arrays:
            out[name] = list(out[name])
        return out


class CscError(RuntimeError):
    """A failed call; ``stats`` holds the solve statistics when a solve failed."""

    def __init__(self, status: int, where: str, stats: dict | None = None):
        self.status = status
        self.stats = stats
        msg = status_string(status) if _lib is not None else str(status)
        if status == CSC_ERR_CUDA and _lib is not None:
            msg += f" (cudaError {_lib.csc_last_cuda_error()})"
        super().__init__(f"{where}: {msg}")


_lib = None


def library_path() -> str:
    return LIB_PATH


def load():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run paper_1901_09235_gb300.build)")
    lib = C.CDLL(LIB_PATH)
    p, i, d, sz = C.c_void_p, C.c_int, C.c_double, C.c_size_t
    S, O, ST = C.POINTER(Shape), C.POINTER(SolveOpts), C.POINTER(SolveStats)
    sig = {
        "csc_default_opts": (None, [O]),
        "csc_workspace_size": (i, [S, O, C.POINTER(sz)]),
        "csc_init_beta": (i, [S, p, p, p, p, C.POINTER(d), p, sz, p]),
        "csc_init_beta_f64": (i, [S, p, p, p, p, C.POINTER(d), p, sz, p]),
        "csc_init_beta_bf16x3": (i, [S, p, p, p, p, C.POINTER(d), p, sz, p]),
        "csc_lgcd_solve": (i, [S, p, p, p, p, p, C.c_float, C.c_float, O, p, sz, ST, p]),
        "csc_lgcd_solve_f64": (i, [S, p, p, p, p, p, d, d, O, p, sz, ST, p]),
        "csc_objective": (i, [S, p, p, p, d, C.POINTER(d), p, sz, p]),
        "cdl_dict_stats": (i, [S, p, p, p, p, p, sz, p]),
        "csc_sparse_code": (i, [S, p, p, p, p, C.c_longlong, C.POINTER(C.c_longlong), p, sz, p]),
        "cdl_dict_update": (i, [S, p, p, d, p, i, d, C.POINTER(d), C.POINTER(i), p, sz, p]),
        "cdl_fit": (i, [S, p, p, p, p, p, p, p, d, d, i, d, i, d, O, p, sz, C.POINTER(d), C.POINTER(i), p]),
        "cdl_step": (i, [S, p, p, p, p, p, p, p, d, d, d, d, i, d, O, p, sz, ST, C.POINTER(d), C.POINTER(d),
                         C.POINTER(i), p]),
        "csc_refresh_beta": (i, [S, p, p, p, C.c_float, p, C.POINTER(d), C.POINTER(d), p, sz, p]),
        "csc_rcd_solve": (i, [S, p, p, p, p, C.c_float, p, C.c_longlong, C.POINTER(C.c_longlong), p, sz, p]),
        "csc_queue_workspace_size": (i, [S, i, i, i, C.POINTER(sz), C.POINTER(sz)]),
        "csc_queue_create": (i, [S, p, p, O, i, i, i, p, sz, p, sz, d, p, p, C.POINTER(p)]),
        "csc_queue_create_deferred": (i, [S, p, p, O, i, i, i, p, sz, p, sz, d, p, p, C.POINTER(p)]),
        "csc_queue_start": (i, [p, i]),
        "csc_queue_submit": (i, [p, i, i, p, p, C.c_float, C.c_float, i, O, C.POINTER(i)]),
        "csc_queue_poll": (i, [p, i, ST]),
        "csc_queue_close": (i, [p]),
        "csc_queue_inspect": (i, [p, i, C.POINTER(C.c_longlong)]),
        "csc_status_string": (C.c_char_p, [i]),
        "csc_last_cuda_error": (i, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_string(status: int) -> str:
    return load().csc_status_string(int(status)).decode()


def _check(rc: int, where: str, soft=(), stats=None):
    if rc != CSC_OK and rc not in soft:
        raise CscError(rc, where, stats)
    return rc


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _need(t, dtype, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def make_shape(X_shape, D_shape) -> Shape:
    """csc_shape from the tensor shapes of X and D."""
    s = Shape()
    if len(X_shape) == 2:
        P, T = X_shape
        K, P2, L = D_shape
        s.d, s.P, s.K = 1, P, K
        s.T[0], s.T[1], s.L[0], s.L[1] = T, 1, L, 1
    elif len(X_shape) == 3:
        P, T0, T1 = X_shape
        K, P2, L0, L1 = D_shape
        s.d, s.P, s.K = 2, P, K
        s.T[0], s.T[1], s.L[0], s.L[1] = T0, T1, L0, L1
    else:
        raise ValueError("X must be (P, T) or (P, T0, T1)")
    if P2 != P:
        raise ValueError("D and X disagree on P")
    return s


def z_shape(s: Shape):
    if s.d == 1:
        return (s.K, s.T[0] - s.L[0] + 1)
    return (s.K, s.T[0] - s.L[0] + 1, s.T[1] - s.L[1] + 1)


def tab_shape(s: Shape):
    if s.d == 1:
        return (s.K, s.K, 2 * s.L[0] - 1)
    return (s.K, s.K, 2 * s.L[0] - 1, 2 * s.L[1] - 1)


def default_opts(**kw) -> SolveOpts:
    o = SolveOpts()
    load().csc_default_opts(C.byref(o))
    for k, v in kw.items():
        if k in ("tile", "sub"):
            arr = getattr(o, k)
            vals = list(v) + [0] * (2 - len(v))
            arr[0], arr[1] = vals[0], vals[1]
        else:
            setattr(o, k, v)
    return o


def workspace_size(shape: Shape, opts: SolveOpts | None = None) -> int:
    n = C.c_size_t(0)
    _check(load().csc_workspace_size(C.byref(shape), C.byref(opts) if opts else None, C.byref(n)),
           "csc_workspace_size")
    return int(n.value)


def workspace(shape: Shape, opts: SolveOpts | None = None, device=None):
    """A caller-owned device workspace (uint8 tensor) for ``shape``."""
    import torch
    return torch.empty(workspace_size(shape, opts), dtype=torch.uint8, device=device or "cuda")


def csc_init_beta(X, D, beta=None, dtd=None, ws=None, stream=None, want_lambda_max=True):
    """beta = D~ * X, the D^T D table and lambda_max (csc_init_beta)."""
    import torch
    f64 = X.dtype == torch.float64
    dt = torch.float64 if f64 else torch.float32
    _need(X, dt, "X")
    _need(D, dt, "D")
    s = make_shape(tuple(X.shape), tuple(D.shape))
    if beta is None:
        beta = torch.empty(z_shape(s), dtype=dt, device=X.device)
    if dtd is None:
        dtd = torch.empty(tab_shape(s), dtype=dt, device=X.device)
    if ws is None:
        ws = workspace(s, device=X.device)
    lm = C.c_double(0.0)
    fn = load().csc_init_beta_f64 if f64 else load().csc_init_beta
    _check(fn(C.byref(s), _ptr(X), _ptr(D), _ptr(beta), _ptr(dtd),
              C.byref(lm) if want_lambda_max else None, _ptr(ws), ws.numel(), _stream(stream)),
           "csc_init_beta")
    return beta, dtd, (lm.value if want_lambda_max else None)



def csc_init_beta_bf16x3(X, D, beta=None, dtd=None, ws=None, stream=None, want_lambda_max=True):
    """csc_init_beta with the correlation on the tensor cores in split-bf16
    precision (csc_init_beta_bf16x3); float32 tensors only."""
    import torch
    _need(X, torch.float32, "X")
    _need(D, torch.float32, "D")
    s = make_shape(tuple(X.shape), tuple(D.shape))
    if beta is None:
        beta = torch.empty(z_shape(s), dtype=torch.float32, device=X.device)
    if dtd is None:
        dtd = torch.empty(tab_shape(s), dtype=torch.float32, device=X.device)
    if ws is None:
        ws = workspace(s, device=X.device)
    lm = C.c_double(0.0)
    _check(load().csc_init_beta_bf16x3(C.byref(s), _ptr(X), _ptr(D), _ptr(beta), _ptr(dtd),
                                       C.byref(lm) if want_lambda_max else None, _ptr(ws), ws.numel(),
                                       _stream(stream)), "csc_init_beta_bf16x3")
    return beta, dtd, (lm.value if want_lambda_max else None)

def csc_lgcd_solve(X, D, dtd, beta, lam: float, tol: float, Z=None, opts: SolveOpts | None = None,
                   ws=None, stream=None):
    """LGCD with soft-locks (csc_lgcd_solve).  beta is updated in place.
    Returns (Z, stats dict).  NOT_CONVERGED / DIVERGED are reported in
    stats['status']; other failures raise CscError."""
    import torch
    f64 = X.dtype == torch.float64
    dt = torch.float64 if f64 else torch.float32
    for t, n in ((X, "X"), (D, "D"), (dtd, "dtd"), (beta, "beta")):
        _need(t, dt, n)
    s = make_shape(tuple(X.shape), tuple(D.shape))
    if Z is None:
        Z = torch.empty(z_shape(s), dtype=dt, device=X.device)
    _need(Z, dt, "Z")
    if opts is None:
        opts = default_opts()
    if ws is None:
        ws = workspace(s, opts, device=X.device)
    st = SolveStats()
    fn = load().csc_lgcd_solve_f64 if f64 else load().csc_lgcd_solve
    rc = fn(C.byref(s), _ptr(X), _ptr(D), _ptr(dtd), _ptr(beta), _ptr(Z), lam, tol, C.byref(opts),
            _ptr(ws), ws.numel(), C.byref(st), _stream(stream))
    stats = st.as_dict()
    _check(rc, "csc_lgcd_solve", soft=(CSC_NOT_CONVERGED, CSC_ERR_DIVERGED), stats=stats)
    return Z, stats


def csc_objective(X, D, Z, lam: float, ws=None, stream=None) -> float:
    import torch
    for t, n in ((X, "X"), (D, "D"), (Z, "Z")):
        _need(t, torch.float32, n)
    s = make_shape(tuple(X.shape), tuple(D.shape))
    if ws is None:
        ws = workspace(s, device=X.device)
    out = C.c_double(0.0)
    _check(load().csc_objective(C.byref(s), _ptr(X), _ptr(D), _ptr(Z), float(lam), C.byref(out),
                                _ptr(ws), ws.numel(), _stream(stream)), "csc_objective")
    return out.value


def csc_refresh_beta(X, D, Z, lam: float, beta=None, ws=None, stream=None):
    """beta recomputed from scratch for Z, with max |dZ| (the KKT test) and
    the objective (csc_refresh_beta).  Returns (beta, max_dz, objective)."""
    import torch
    for t, n in ((X, "X"), (D, "D"), (Z, "Z")):
        _need(t, torch.float32, n)
    s = make_shape(tuple(X.shape), tuple(D.shape))
    if beta is None:
        beta = torch.empty(z_shape(s), dtype=torch.float32, device=X.device)
    _need(beta, torch.float32, "beta")
    if ws is None:
        ws = workspace(s, device=X.device)
    mdz, obj = C.c_double(0.0), C.c_double(0.0)
    _check(load().csc_refresh_beta(C.byref(s), _ptr(X), _ptr(D), _ptr(Z), float(lam), _ptr(beta),
                                   C.byref(mdz), C.byref(obj), _ptr(ws), ws.numel(), _stream(stream)),
           "csc_refresh_beta")
    return beta, mdz.value, obj.value


def csc_rcd_solve(X_shape, D, dtd, beta, Z, lam: float, coords, ws=None, stream=None) -> int:
    """Coordinate descent over the flat indices ``coords`` (a uint32-valued
    CUDA tensor, k |Omega| + s), in order (csc_rcd_solve).  beta and Z are
    updated in place.  Returns the number of coordinates that changed."""
    import torch
    for t, n in ((D, "D"), (dtd, "dtd"), (beta, "beta"), (Z, "Z")):
        _need(t, torch.float32, n)
    if not isinstance(coords, torch.Tensor) or not coords.is_cuda or coords.dtype not in (torch.int32,
                                                                                        torch.uint32):
        raise TypeError("coords must be a CUDA int32 / uint32 tensor")
    if not coords.is_contiguous():
        raise ValueError("coords must be contiguous")
    s = make_shape(tuple(X_shape), tuple(D.shape))
    if ws is None:
        ws = workspace(s, device=D.device)
    upd = C.c_longlong(0)
    _check(load().csc_rcd_solve(C.byref(s), _ptr(D), _ptr(dtd), _ptr(beta), _ptr(Z), float(lam), _ptr(coords),
                                coords.numel(), C.byref(upd), _ptr(ws), ws.numel(), _stream(stream)),
           "csc_rcd_solve")
    return upd.value


class Queue:
    """Many 2-D solves of uneven size in one persistent launch (csc_queue_*).

    D (K, P, L0, L1) and its D^T D table stay resident.  Each job brings its
    own beta (from csc_init_beta*, ready on the submitting stream) and Z, which
    the kernel updates in place.  The kernel runs on its own stream and the
    control copies on a second one; both are non-blocking streams.  While the
    queue is open nothing may wait for the whole device (torch.cuda.synchronize,
    the legacy default stream of a blocking stream): the kernel ends only on
    close() or after run_seconds.  ctas_per_sm: 2 (0, the default) leaves room
    beside the queue for the tensor-core beta-init; 3 runs more tiles at once
    and leaves room for the FP32 calls only.  start=False makes the queue
    without launching its kernel: jobs submitted before start() are published
    before it runs, and start(drain=True) lets it end by itself once they are
    done (no host copy has to overlap the running kernel)."""

    def __init__(self, D, dtd, max_jobs: int = 1024, ctl_slots: int = 256, run_seconds: float = 120.0,
                 opts: SolveOpts | None = None, ctas_per_sm: int = 0, start: bool = True):
        import torch
        _need(D, torch.float32, "D")
        _need(dtd, torch.float32, "dtd")
        if D.dim() != 4:
            raise ValueError("D must be (K, P, L0, L1)")
        K, P, L0, L1 = D.shape
        s = Shape()
        s.d, s.P, s.K = 2, P, K
        s.T[0], s.T[1], s.L[0], s.L[1] = L0, L1, L0, L1
        self.atoms, self.D, self.dtd = s, D, dtd
        lib = load()
        db, hb = C.c_size_t(0), C.c_size_t(0)
        _check(lib.csc_queue_workspace_size(C.byref(s), int(max_jobs), int(ctl_slots), int(ctas_per_sm),
                                            C.byref(db), C.byref(hb)), "csc_queue_workspace_size")
        self.ws = torch.empty(db.value, dtype=torch.uint8, device=D.device)
        self.host = torch.zeros(hb.value, dtype=torch.uint8, pin_memory=True)
        self.kernel_stream = torch.cuda.Stream(device=D.device)
        self.side_stream = torch.cuda.Stream(device=D.device)
        self.side_stream.wait_stream(torch.cuda.current_stream(D.device))
        self.kernel_stream.wait_stream(torch.cuda.current_stream(D.device))
        self._opts = opts
        self._jobs = {}
        h = C.c_void_p(0)
        create = lib.csc_queue_create if start else lib.csc_queue_create_deferred
        _check(create(C.byref(s), _ptr(D), _ptr(dtd), C.byref(opts) if opts else None,
                      int(max_jobs), int(ctl_slots), int(ctas_per_sm), _ptr(self.ws), self.ws.numel(),
                      C.c_void_p(self.host.data_ptr()), self.host.numel(), float(run_seconds),
                      C.c_void_p(self.kernel_stream.cuda_stream), C.c_void_p(self.side_stream.cuda_stream),
                      C.byref(h)), "csc_queue_create")
        self._h = h

    def start(self, drain: bool = True):
        """Launch the kernel of a queue made with start=False (csc_queue_start).
        drain: it ends by itself after the jobs submitted so far, and takes no
        more."""
        if self._h is None:
            raise RuntimeError("queue closed")
        _check(load().csc_queue_start(self._h, int(bool(drain))), "csc_queue_start")

    def submit(self, beta, Z, lam: float, tol: float, warm_start: bool = False, stream=None,
               opts: SolveOpts | None = None) -> int:
        """Queue one image; beta (K, Z0, Z1) must be complete on `stream` (the
        current stream by default).  opts: this job's solve options (None: the
        queue's).  Returns the job index."""
        import torch
        _need(beta, torch.float32, "beta")
        _need(Z, torch.float32, "Z")
        if self._h is None:
            raise RuntimeError("queue closed")
        K, L0, L1 = self.atoms.K, self.atoms.L[0], self.atoms.L[1]
        if beta.dim() != 3 or beta.shape[0] != K or tuple(Z.shape) != tuple(beta.shape):
            raise ValueError("beta and Z must both be (K, Z0, Z1)")
        src = stream if stream is not None else torch.cuda.current_stream(beta.device)
        self.side_stream.wait_stream(src)
        T0, T1 = beta.shape[1] + L0 - 1, beta.shape[2] + L1 - 1
        j = C.c_int(-1)
        _check(load().csc_queue_submit(self._h, int(T0), int(T1), _ptr(beta), _ptr(Z), float(lam),
                                       float(tol), int(bool(warm_start)), C.byref(opts) if opts else None,
                                       C.byref(j)), "csc_queue_submit")
        self._jobs[j.value] = (beta, Z)  # keep the buffers alive while the kernel uses them
        return j.value

    def poll(self, job: int):
        """The job's statistics once it has completed, else None (no CUDA call)."""
        st = SolveStats()
        rc = load().csc_queue_poll(self._h, int(job), C.byref(st))
        if rc < 0:
            raise CscError(-rc, "csc_queue_poll")
        if rc == 0:
            return None
        self._jobs.pop(int(job), None)
        return st.as_dict()

    def inspect(self, job: int) -> dict:
        """Device-side state of a job (csc_queue_inspect), for a stalled queue."""
        out = (C.c_longlong * 8)()
        _check(load().csc_queue_inspect(self._h, int(job), out), "csc_queue_inspect")
        keys = ("prefix", "W", "claimed", "done", "njobs", "next_slot", "grid", "complete")
        return dict(zip(keys, list(out)))

    def wait(self, job: int, timeout: float = 60.0):
        import time
        t_end = time.monotonic() + timeout
        while True:
            r = self.poll(job)
            if r is not None:
                return r
            if time.monotonic() > t_end:
                raise TimeoutError(f"queue job {job} did not complete in {timeout} s: {self.inspect(job)}")
            time.sleep(20e-6)

    def close(self):
        if self._h is not None:
            h, self._h = self._h, None
            _check(load().csc_queue_close(h), "csc_queue_close")
            self._jobs.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        # a queue dropped without close() would keep its kernel running until
        # run_seconds; stop it (best effort: the CUDA context may already be gone)
        try:
            if getattr(self, "_h", None) is not None:
                self.close()
        except Exception:
            pass


def cdl_dict_stats(Z, X, D_shape, phi=None, psi=None, ws=None, stream=None):
    """phi = Z~ * Z on Phi and psi = Z~ * X on Theta (cdl_dict_stats)."""
    import torch
    _need(Z, torch.float32, "Z")
    _need(X, torch.float32, "X")
    s = make_shape(tuple(X.shape), tuple(D_shape))
    if phi is None:
        phi = torch.empty(tab_shape(s), dtype=torch.float32, device=X.device)
    if psi is None:
        psi = torch.empty(tuple(D_shape), dtype=torch.float32, device=X.device)
    if ws is None:
        ws = workspace(s, device=X.device)
    _check(load().cdl_dict_stats(C.byref(s), _ptr(Z), _ptr(X), _ptr(phi), _ptr(psi), _ptr(ws),
                                 ws.numel(), _stream(stream)), "cdl_dict_stats")
    return phi, psi


def sparse_code(Z, X_shape, D_shape, out=None, ws=None, stream=None):
    """The nonzeros of Z in (position, atom) order (csc_sparse_code): returns
    (k, s, values, nnz) with k, s int32 and values float32 device tensors of
    nnz entries (views of `out`, a (k, s, values) triple of capacity cap, when
    given; when the count exceeds cap, a CscError with the count in .stats)."""
    import torch
    _need(Z, torch.float32, "Z")
    s = make_shape(tuple(X_shape), tuple(D_shape))
    if ws is None:
        ws = workspace(s, device=Z.device)
    n = C.c_longlong(0)
    lib = load()
    if out is None:
        rc = lib.csc_sparse_code(C.byref(s), _ptr(Z), None, None, None, 0, C.byref(n), _ptr(ws), ws.numel(),
                                 _stream(stream))
        if rc not in (CSC_OK, CSC_ERR_WORKSPACE):
            _check(rc, "csc_sparse_code")
        cap = max(1, n.value)
        out = (torch.empty(cap, dtype=torch.int32, device=Z.device),
               torch.empty(cap, dtype=torch.int32, device=Z.device),
               torch.empty(cap, dtype=torch.float32, device=Z.device))
    kb, sb, vb = out
    cap = min(kb.numel(), sb.numel(), vb.numel())
    rc = lib.csc_sparse_code(C.byref(s), _ptr(Z), _ptr(kb), _ptr(sb), _ptr(vb), cap, C.byref(n), _ptr(ws),
                             ws.numel(), _stream(stream))
    if rc != CSC_OK:
        raise CscError(rc, "csc_sparse_code", {"nnz": n.value, "cap": cap})
    m = n.value
    return kb[:m], sb[:m], vb[:m], m


def cdl_dict_update(phi, psi, x_sqnorm: float, D, X_shape, max_iter: int = 50, tol: float = 1e-8,
                    ws=None, stream=None):
    """PGD + Armijo on D in place (cdl_dict_update).  Returns (F, iterations)."""
    import torch
    for t, n in ((phi, "phi"), (psi, "psi"), (D, "D")):
        _need(t, torch.float32, n)
    s = make_shape(tuple(X_shape), tuple(D.shape))
    if ws is None:
        ws = workspace(s, device=D.device)
    f = C.c_double(0.0)
    it = C.c_int(0)
    _check(load().cdl_dict_update(C.byref(s), _ptr(phi), _ptr(psi), float(x_sqnorm), _ptr(D),
                                  int(max_iter), float(tol), C.byref(f), C.byref(it), _ptr(ws),
                                  ws.numel(), _stream(stream)), "cdl_dict_update")
    return f.value, it.value


def cdl_fit(X, D, reg: float = 0.1, tol: float = 1e-4, max_outer: int = 10, nu: float = 0.0,
            pgd_max_iter: int = 50, pgd_tol: float = 1e-8, opts: SolveOpts | None = None, prob=None,
            stream=None):
    """Dictionary learning (cdl_fit): D is updated in place.  Returns
    (Z, trace of (cost after CSC, cost after the dictionary step), status)."""
    import torch
    _need(X, torch.float32, "X")
    _need(D, torch.float32, "D")
    if prob is None:
        prob = Problem.create(X, D, opts)
    s = prob.shape
    tr = (C.c_double * (2 * max_outer))()
    n = C.c_int(0)
    rc = load().cdl_fit(C.byref(s), _ptr(X), _ptr(D), _ptr(prob.Z), _ptr(prob.beta), _ptr(prob.dtd),
                        _ptr(prob.phi), _ptr(prob.psi), float(reg), float(tol), int(max_outer), float(nu),
                        int(pgd_max_iter), float(pgd_tol), C.byref(opts) if opts else None,
                        _ptr(prob.ws), prob.ws.numel(), tr, C.byref(n), _stream(stream))
    _check(rc, "cdl_fit", soft=(CSC_NOT_CONVERGED,))
    trace = [(tr[2 * i], tr[2 * i + 1]) for i in range(n.value)]
    return prob.Z, trace, rc


def cdl_step(X, D, prob, reg: float = 0.1, tol: float = 1e-4, x_sqnorm: float | None = None,
             pgd_max_iter: int = 50, pgd_tol: float = 1e-8, opts: SolveOpts | None = None, stream=None,
             lam: float | None = None):
    """One pass of the loop body of Alg. 2 in one call (cdl_step): beta-init,
    LGCD with the given lambda (``lam``) or lambda = reg * lambda_max(X, D),
    phi / psi and the dictionary step, into the buffers of ``prob`` (a
    Problem of the same shapes); D is updated in place.  x_sqnorm None: summed
    on the device.  Returns (Z, stats): the solve statistics plus 'lambda',
    'dict_F' and 'dict_iters'."""
    import torch
    _need(X, torch.float32, "X")
    _need(D, torch.float32, "D")
    s = prob.shape
    st = SolveStats()
    lam_out, fd, it = C.c_double(0.0), C.c_double(0.0), C.c_int(0)
    rc = load().cdl_step(C.byref(s), _ptr(X), _ptr(D), _ptr(prob.Z), _ptr(prob.beta), _ptr(prob.dtd),
                         _ptr(prob.phi), _ptr(prob.psi), float(reg), float(lam or 0.0), float(tol),
                         -1.0 if x_sqnorm is None else float(x_sqnorm),
                         int(pgd_max_iter), float(pgd_tol), C.byref(opts) if opts else None, _ptr(prob.ws),
                         prob.ws.numel(), C.byref(st), C.byref(lam_out), C.byref(fd), C.byref(it),
                         _stream(stream))
    stats = st.as_dict()
    _check(rc, "cdl_step", soft=(CSC_NOT_CONVERGED,), stats=stats)
    stats["lambda"], stats["dict_F"], stats["dict_iters"] = lam_out.value, fd.value, it.value
    return prob.Z, stats


@dataclass
class Problem:
    """Device-resident buffers of one CSC problem (inputs stay in HBM)."""
    X: object
    D: object
    shape: Shape
    ws: object
    beta: object = None
    dtd: object = None
    Z: object = None
    phi: object = None
    psi: object = None

    @classmethod
    def create(cls, X, D, opts=None):
        import torch
        s = make_shape(tuple(X.shape), tuple(D.shape))
        p = cls(X=X, D=D, shape=s, ws=workspace(s, opts, device=X.device))
        p.beta = torch.empty(z_shape(s), dtype=X.dtype, device=X.device)
        p.Z = torch.empty_like(p.beta)
        p.dtd = torch.empty(tab_shape(s), dtype=X.dtype, device=X.device)
        p.phi = torch.empty(tab_shape(s), dtype=torch.float32, device=X.device)
        p.psi = torch.empty(tuple(D.shape), dtype=torch.float32, device=X.device)
        return p


def cdl_dict_stats_noalloc(Z, X, D_shape, phi=None, psi=None, stream=None):
    """phi and psi like cdl_dict_stats, for callers that cannot allocate device
    memory: the library's built-in scratch array is used instead of a caller
    workspace (the output tensors are still the caller's).  Calls that overlap
    on the GPU must be serialised by the caller."""
    import torch
    _need(Z, torch.float32, "Z")
    _need(X, torch.float32, "X")
    lib = load()
    fn = lib.cdl_dict_stats_noalloc
    fn.restype = C.c_int
    fn.argtypes = [C.POINTER(Shape), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    s = make_shape(tuple(X.shape), tuple(D_shape))
    if phi is None:
        phi = torch.empty(tab_shape(s), dtype=torch.float32, device=X.device)
    if psi is None:
        psi = torch.empty(tuple(D_shape), dtype=torch.float32, device=X.device)
    _check(fn(C.byref(s), _ptr(Z), _ptr(X), _ptr(phi), _ptr(psi), _stream(stream)),
           "cdl_dict_stats_noalloc")
    return phi, psi
