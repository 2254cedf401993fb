"""FP64 CPU oracle for the DiCoDiLe CSC / dictionary-update path.

TEST INFRASTRUCTURE ONLY.  The oracle is a plain, sequential C restatement of
the paper's definitions and of Alg. 1 (LGCD), used to check the CUDA library.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  The CUDA library never calls it and shares no code
with it.

Arrays follow the layouts documented at the top of ``oracle.c``; a 1-D signal
is passed with a leading singleton spatial axis (T0 = L0 = 1).  Inputs are
converted to contiguous float64 before the call.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` with gcc (no fast-math, no
    FMA contraction, so every product and sum rounds as written)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11",
                               "-ffp-contract=off", "-fno-fast-math",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        d, i, ll = C.c_double, C.c_int, C.c_longlong
        p = C.c_void_p
        sig = {
            "orc_beta_init": (None, [i, i, i, i, i, i, p, p, p]),
            "orc_dtd": (None, [i, i, i, i, p, p]),
            "orc_atom_sqnorms": (None, [i, i, i, i, p, p]),
            "orc_lambda_max": (d, [i, i, i, i, i, i, p, p]),
            "orc_reconstruct": (None, [i, i, i, i, i, i, p, p, p]),
            "orc_objective": (d, [i, i, i, i, i, i, p, p, p, d]),
            "orc_beta_from_Z": (None, [i, i, i, i, i, i, p, p, p, p]),
            "orc_max_dz": (d, [i, i, i, p, p, p, d]),
            "orc_lgcd_tiled": (i, [i, i, i, i, i, i, p, p, d, d, i, i, i, i, ll,
                                   p, p, p, p, ll, p, p, p, p, p]),
            "orc_phi_psi": (None, [i, i, i, i, i, i, p, p, p, p]),
            "orc_dict_grad": (None, [i, i, i, i, p, p, p, p]),
            "orc_dict_objective": (d, [i, i, i, i, p, p, d, p]),
            "orc_pgd_armijo": (i, [i, i, i, i, p, p, d, p, i, d, p]),
            "orc_beta_at": (None, [i, i, i, i, i, i, p, p, ll, p, p, p]),
            "orc_beta_from_Z_at": (None, [i, i, i, i, i, i, p, p, p, ll, p, p, p]),
            "orc_objective_sparse": (d, [i, i, i, i, i, i, p, p, p, d]),
            "orc_objective_nz": (d, [i, i, i, i, i, i, p, p, C.c_longlong, p, p, p, p, d]),
            "orc_rcd": (ll, [i, i, i, i, i, i, p, d, p, ll, p, p]),
            "orc_phi_psi_nz": (i, [i, i, i, i, i, i, p, ll, p, p, p, p, p, p]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _geom(X: np.ndarray, D: np.ndarray):
    """(P, K, T0, T1, L0, L1) from X (P x T or P x T0 x T1) and D (K x P x L...)."""
    if X.ndim == 2:
        P, T1 = X.shape
        T0 = 1
        K, P2, L1 = D.shape
        L0 = 1
    else:
        P, T0, T1 = X.shape
        K, P2, L0, L1 = D.shape
    assert P2 == P
    return P, K, T0, T1, L0, L1


def _zshape(X, D):
    P, K, T0, T1, L0, L1 = _geom(X, D)
    return (K, T1 - L1 + 1) if X.ndim == 2 else (K, T0 - L0 + 1, T1 - L1 + 1)


def beta_init(X, D):
    """beta = D~ * X on the valid activation domain (Alg. 1 initialisation)."""
    X, D = _f64(X), _f64(D)
    g = _geom(X, D)
    beta = np.zeros(_zshape(X, D))
    _load().orc_beta_init(*g, _ptr(X), _ptr(D), _ptr(beta))
    return beta


def dtd(D, d: int):
    """C[k][k2][delta] = sum_p sum_tau D_kp[tau] D_k2p[tau+delta] (Eq. beta_update)."""
    D = _f64(D)
    if d == 1:
        K, P, L1 = D.shape
        L0 = 1
    else:
        K, P, L0, L1 = D.shape
    out = np.zeros((K, K, 2 * L0 - 1, 2 * L1 - 1))
    _load().orc_dtd(P, K, L0, L1, _ptr(D), _ptr(out))
    return out if d == 2 else out[:, :, 0, :].copy()


def atom_sqnorms(D):
    D = _f64(D)
    K, P = D.shape[:2]
    L = D.shape[2:]
    L0, L1 = (1, L[0]) if len(L) == 1 else L
    out = np.zeros(K)
    _load().orc_atom_sqnorms(P, K, L0, L1, _ptr(D), _ptr(out))
    return out


def lambda_max(X, D) -> float:
    X, D = _f64(X), _f64(D)
    return float(_load().orc_lambda_max(*_geom(X, D), _ptr(X), _ptr(D)))


def reconstruct(Z, D, T):
    """(Z * D) on the signal domain of size T (a tuple)."""
    Z, D = _f64(Z), _f64(D)
    K, P = D.shape[:2]
    X = np.zeros((P,) + tuple(T))
    _load().orc_reconstruct(*_geom(X, D), _ptr(Z), _ptr(D), _ptr(X))
    return X


def objective(X, D, Z, lam: float) -> float:
    X, D, Z = _f64(X), _f64(D), _f64(Z)
    return float(_load().orc_objective(*_geom(X, D), _ptr(X), _ptr(D), _ptr(Z), float(lam)))


def beta_from_Z(X, D, Z):
    X, D, Z = _f64(X), _f64(D), _f64(Z)
    beta = np.zeros(_zshape(X, D))
    _load().orc_beta_from_Z(*_geom(X, D), _ptr(X), _ptr(D), _ptr(Z), _ptr(beta))
    return beta


def max_dz(beta, Z, nrm, lam: float) -> float:
    beta, Z, nrm = _f64(beta), _f64(Z), _f64(nrm)
    K = beta.shape[0]
    sp = beta.shape[1:]
    Z0, Z1 = (1, sp[0]) if len(sp) == 1 else sp
    return float(_load().orc_max_dz(K, Z0, Z1, _ptr(beta), _ptr(Z), _ptr(nrm), float(lam)))


def kkt(X, D, Z, lam: float) -> float:
    """max |ST(beta,lambda)/||D_k||^2 - Z| with beta recomputed from scratch."""
    return max_dz(beta_from_Z(X, D, Z), Z, atom_sqnorms(D), lam)


def lgcd(X, D, lam: float, eps: float, sub=None, tile=None, max_updates: int = 0,
         trace_cap: int = 0):
    """LGCD (Alg. 1); with ``tile`` the checkerboard-phased tiled schedule.

    ``sub`` / ``tile`` are per-dimension sizes (tuples of length d); None means
    the default sub-domain 2L and a single tile.  Returns a dict with Z, beta,
    status (0 converged, 1 max_updates reached), n_updates, n_iters and, when
    ``trace_cap`` > 0, the first ``trace_cap`` accepted updates."""
    X, D = _f64(X), _f64(D)
    g = _geom(X, D)
    d = X.ndim - 1
    sub0, sub1 = (0, 0) if sub is None else ((1, sub[0]) if d == 1 else tuple(sub))
    t0, t1 = (0, 0) if tile is None else ((1, tile[0]) if d == 1 else tuple(tile))
    Z = np.zeros(_zshape(X, D))
    beta = np.zeros_like(Z)
    nu, ni = C.c_longlong(0), C.c_longlong(0)
    cap = int(trace_cap)
    tk = np.zeros(max(cap, 1), np.int32)
    ts = np.zeros(max(cap, 1), np.int64)
    tzo, tzn, tb = (np.zeros(max(cap, 1)) for _ in range(3))
    st = _load().orc_lgcd_tiled(*g, _ptr(X), _ptr(D), float(lam), float(eps), t0, t1, sub0, sub1,
                                int(max_updates), _ptr(Z), _ptr(beta), C.byref(nu), C.byref(ni),
                                cap, _ptr(tk), _ptr(ts), _ptr(tzo), _ptr(tzn), _ptr(tb))
    out = dict(Z=Z, beta=beta, status=int(st), n_updates=int(nu.value), n_iters=int(ni.value))
    if cap > 0:
        n = min(cap, out["n_updates"])
        out["trace"] = dict(k0=tk[:n], s0=ts[:n], z_old=tzo[:n], z_new=tzn[:n], beta=tb[:n])
    return out


def rcd(X, D, lam: float, coords, Z=None, beta=None):
    """Coordinate descent over the flat indices ``coords`` (k |Omega| + s), in
    order (the RCD baseline of Section 5.1 when the order is random).  Starts
    from ``Z`` / ``beta`` (default: Z = 0, beta = D~ * X) and returns
    (Z, beta, number of coordinates that changed)."""
    X, D = _f64(X), _f64(D)
    g = _geom(X, D)
    if Z is None:
        Z = np.zeros(_zshape(X, D))
        beta = beta_init(X, D)
    Z, beta = _f64(Z).copy(), _f64(beta).copy()
    cs = np.ascontiguousarray(coords, dtype=np.uint32)
    n = _load().orc_rcd(*g, _ptr(D), float(lam), _ptr(cs), len(cs), _ptr(Z), _ptr(beta))
    if n < 0:
        raise ValueError("coordinate index outside K x Omega")
    return Z, beta, int(n)


def phi_psi(Z, X, L):
    """phi (Eq. phi, restricted to Phi) and psi = Z~ * X restricted to Theta."""
    Z, X = _f64(Z), _f64(X)
    K = Z.shape[0]
    d = X.ndim - 1
    L0, L1 = (1, L[0]) if d == 1 else tuple(L)
    P = X.shape[0]
    T0, T1 = (1, X.shape[1]) if d == 1 else X.shape[1:]
    phi = np.zeros((K, K, 2 * L0 - 1, 2 * L1 - 1))
    psi = np.zeros((K, P, L0, L1))
    _load().orc_phi_psi(P, K, T0, T1, L0, L1, _ptr(Z), _ptr(X), _ptr(phi), _ptr(psi))
    if d == 1:
        return phi[:, :, 0, :].copy(), psi[:, :, 0, :].copy()
    return phi, psi


def _dict_geom(D):
    K, P = D.shape[:2]
    L = D.shape[2:]
    L0, L1 = (1, L[0]) if len(L) == 1 else L
    return P, K, L0, L1


def dict_grad(phi, psi, D):
    phi, psi, D = _f64(phi), _f64(psi), _f64(D)
    g = np.zeros_like(D)
    _load().orc_dict_grad(*_dict_geom(D), _ptr(phi), _ptr(psi), _ptr(D), _ptr(g))
    return g


def dict_objective(phi, psi, x_sqnorm: float, D) -> float:
    phi, psi, D = _f64(phi), _f64(psi), _f64(D)
    return float(_load().orc_dict_objective(*_dict_geom(D), _ptr(phi), _ptr(psi),
                                            float(x_sqnorm), _ptr(D)))


def pgd_armijo(phi, psi, x_sqnorm: float, D, max_iter: int = 50, tol: float = 1e-8):
    """PGD with Armijo backtracking on D (Alg. 2).  Returns (D, F, iterations)."""
    phi, psi = _f64(phi), _f64(psi)
    D = _f64(D).copy()
    f = C.c_double(0.0)
    it = _load().orc_pgd_armijo(*_dict_geom(D), _ptr(phi), _ptr(psi), float(x_sqnorm),
                                _ptr(D), int(max_iter), float(tol), C.byref(f))
    return D, float(f.value), int(it)


def _coords(ks, ss):
    ks = np.ascontiguousarray(np.asarray(ks, dtype=np.int32))
    ss = np.ascontiguousarray(np.asarray(ss, dtype=np.int64))
    assert ks.shape == ss.shape
    return ks, ss


def beta_at(X, D, ks, ss):
    """beta_k[s] of the initialisation at listed (k, row-major s)."""
    X, D = _f64(X), _f64(D)
    ks, ss = _coords(ks, ss)
    out = np.zeros(len(ks))
    _load().orc_beta_at(*_geom(X, D), _ptr(X), _ptr(D), len(ks), _ptr(ks), _ptr(ss), _ptr(out))
    return out


def beta_from_Z_at(X, D, Z, ks, ss):
    """beta from its definition for the current Z at listed (k, s)."""
    X, D, Z = _f64(X), _f64(D), _f64(Z)
    ks, ss = _coords(ks, ss)
    out = np.zeros(len(ks))
    _load().orc_beta_from_Z_at(*_geom(X, D), _ptr(X), _ptr(D), _ptr(Z), len(ks), _ptr(ks),
                               _ptr(ss), _ptr(out))
    return out


def objective_sparse(X, D, Z, lam: float) -> float:
    X, D, Z = _f64(X), _f64(D), _f64(Z)
    return float(_load().orc_objective_sparse(*_geom(X, D), _ptr(X), _ptr(D), _ptr(Z), float(lam)))


def objective_nz(X, D, k, i, j, z, lam: float) -> float:
    """Eq. csc from the nonzeros of Z given as index arrays (k, i, j) and
    values z (for 1-D problems i is all zeros and j the position)."""
    X, D = _f64(X), _f64(D)
    k, i, j = (np.ascontiguousarray(np.asarray(v), dtype=np.int64) for v in (k, i, j))
    z = _f64(np.asarray(z))
    if not (len(k) == len(i) == len(j) == len(z)):
        raise ValueError("index and value arrays differ in length")
    return float(_load().orc_objective_nz(*_geom(X, D), _ptr(X), _ptr(D), len(z), _ptr(k), _ptr(i),
                                          _ptr(j), _ptr(z), float(lam)))


def phi_psi_nz(X, L, K, k, i, j, z):
    """phi and psi from the nonzeros of Z given as index arrays (k, i, j) and
    values z (1-D problems: i all zeros, j the position), for activation maps
    too large for the dense routine.  Shapes as ``phi_psi`` returns them."""
    X = _f64(X)
    d = X.ndim - 1
    L0, L1 = (1, L[0]) if d == 1 else tuple(L)
    P = X.shape[0]
    T0, T1 = (1, X.shape[1]) if d == 1 else X.shape[1:]
    k, i, j = (np.ascontiguousarray(np.asarray(v), dtype=np.int64) for v in (k, i, j))
    z = _f64(np.asarray(z))
    if not (len(k) == len(i) == len(j) == len(z)):
        raise ValueError("index and value arrays differ in length")
    phi = np.zeros((K, K, 2 * L0 - 1, 2 * L1 - 1))
    psi = np.zeros((K, P, L0, L1))
    rc = _load().orc_phi_psi_nz(P, K, T0, T1, L0, L1, _ptr(X), len(z), _ptr(k), _ptr(i), _ptr(j), _ptr(z),
                                _ptr(phi), _ptr(psi))
    if rc != 0:
        raise ValueError("nonzero index outside the activation domain")
    if d == 1:
        return phi[:, :, 0, :].copy(), psi[:, :, 0, :].copy()
    return phi, psi


def cdl(X, D0, reg: float, tol: float, n_outer: int, pgd_max_iter: int = 50, pgd_tol: float = 1e-8):
    """The outer loop of Alg. 2 with the routines above: Z by LGCD from zero
    (lambda = reg * lambda_max(X, D0), fixed), then phi/psi and PGD-Armijo on
    D.  Returns (D, Z, [(cost after CSC, cost after the dictionary step)])."""
    X = _f64(X)
    D = _f64(D0).copy()
    lam = reg * lambda_max(X, D)
    L = D.shape[2:]
    xs = float(np.sum(X ** 2))
    trace = []
    Z = None
    for _ in range(n_outer):
        Z = lgcd(X, D, lam, tol)["Z"]
        c1 = objective(X, D, Z, lam)
        phi, psi = phi_psi(Z, X, L)
        D, f, _ = pgd_armijo(phi, psi, xs, D, max_iter=pgd_max_iter, tol=pgd_tol)
        trace.append((c1, f + lam * float(np.abs(Z).sum())))
    return D, Z, trace
