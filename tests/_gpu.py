"""Helpers shared by the GPU parity tests."""
import numpy as np

U32 = 2.0 ** -24


def gamma(n: int, u: float = U32) -> float:
    """gamma_n = n u / (1 - n u): the classical bound on the relative error
    of an n-term floating-point dot product (recursive or fused summation)."""
    return n * u / (1.0 - n * u)


def dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    return t.detach().cpu().numpy()


def support_mismatch(z_a, z_b, tol, factor=100.0):
    """Coordinates nonzero in exactly one of the two solutions; each must be
    small (|Z| <= factor * tol in the solution that keeps it)."""
    a = z_a != 0
    b = z_b != 0
    diff = a ^ b
    vals = np.where(a & ~b, np.abs(z_a), np.where(b & ~a, np.abs(z_b), 0.0))
    return int(diff.sum()), float(vals.max()) if diff.any() else 0.0


def max_window_nonzeros(Z, L):
    """The largest number of nonzeros of Z (all atoms) within one window
    V(s) = prod [s_i - L_i + 1, s_i + L_i - 1] (integral image)."""
    Zs = np.asarray(Z)
    Zs = Zs if Zs.ndim == 3 else Zs[:, None, :]
    L0, L1 = (1, L[0]) if len(L) == 1 else tuple(L)
    cnt = (Zs != 0).sum(axis=0).astype(np.int64)
    n0, n1 = cnt.shape
    c = np.zeros((n0 + 1, n1 + 1), np.int64)
    c[1:, 1:] = cnt.cumsum(0).cumsum(1)
    i = np.arange(n0)
    j = np.arange(n1)
    i0, i1 = np.maximum(i - L0 + 1, 0), np.minimum(i + L0, n0)
    j0, j1 = np.maximum(j - L1 + 1, 0), np.minimum(j + L1, n1)
    win = c[i1][:, j1] - c[i0][:, j1] - c[i1][:, j0] + c[i0][:, j0]
    return int(win.max()) if win.size else 0


def kkt_fp64_within_bound(orc, X, D, Z, lam, tol, ks=None, ss=None):
    """The KKT test of the oracle against the GPU's.

    The GPU ends a solve only when max |dZ| < tol holds on a beta it
    recomputes in FP32 from Z, in one of two ways: the correlation of the
    residual (R = X - Z * D summed in FP64 and rounded to FP32,
    beta_k[s] = sum over the n = P |Theta| taps of D_kp[tau] R_p[s + tau] in
    FP32, plus ||D_k||^2 Z_k[s]) or, on global-memory tiles, the initial beta
    minus the table times Z (beta_k[s] = beta0_k[s] - sum over the m nonzeros
    (k', s') of Z within V(s), (k', s') != (k, s), of C[k][k'][s - s'] Z_k'[s'],
    with beta0 and C themselves n-term FP32 correlations).  Either FP32 value
    differs from its FP64 counterpart by at most
        |d beta| <= gamma_{n+m+3} (sum |D_kp[tau]| (|X| + |Z| * |D|)_p[s + tau] + ||D_k||^2 |Z_k[s]|)
    and |d dZ| <= |d beta| / ||D_k||^2 + gamma_3 (|Z'| + |Z|) for the scaling
    and the subtraction (dZ = ST(beta, lambda) / ||D_k||^2 - Z), m being the
    largest count of nonzeros of Z in one window.  So on the oracle's FP64
    beta every coordinate must satisfy
        |dZ_64| < tol + |d dZ|,
    which is what this returns (True / False) together with the largest
    |dZ_64| and the largest bound, at the listed coordinates (k, row-major s)
    or everywhere."""
    X64, D64, Z64 = (np.asarray(a, dtype=np.float64) for a in (X, D, Z))
    K = D64.shape[0]
    n = int(np.prod(D64.shape[1:]))
    m = max_window_nonzeros(Z64, D64.shape[2:])
    nrm = orc.atom_sqnorms(D64)
    Zf = Z64.reshape(K, -1)
    if ks is None:
        b64 = orc.beta_from_Z(X64, D64, Z64).reshape(K, -1)
        # sum |D| (|X| + |Z| * |D|) = beta_from_Z(|X|, |D|, -|Z|) + ||D||^2 |Z|
        babs = orc.beta_from_Z(np.abs(X64), np.abs(D64), -np.abs(Z64)).reshape(K, -1) + nrm[:, None] * np.abs(Zf)
        nk = nrm[:, None]
        z = Zf
    else:
        ks, ss = np.asarray(ks), np.asarray(ss)
        b64 = orc.beta_from_Z_at(X64, D64, Z64, ks, ss)
        babs = orc.beta_from_Z_at(np.abs(X64), np.abs(D64), -np.abs(Z64), ks, ss) + nrm[ks] * np.abs(Zf[ks, ss])
        nk = nrm[ks]
        z = Zf[ks, ss]
    zn = np.sign(b64) * np.maximum(np.abs(b64) - lam, 0.0) / nk
    dz = np.abs(zn - z)
    bound = gamma(n + m + 3) * (babs + nk * np.abs(z)) / nk + gamma(3) * (np.abs(zn) + np.abs(z))
    return bool(np.all(dz < tol + bound)), float(dz.max()), float(bound.max())
