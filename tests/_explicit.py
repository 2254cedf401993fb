"""Independent, explicit-matrix restatement of the CSC problem for tiny inputs.

The convolutional model X = Z * D (Eq. model) is a linear map; here it is
materialised column by column as a dense matrix A whose column (k, s) is the
library convolution of a unit impulse at s with atom k.  The LASSO of Eq. csc
then reads 1/2 ||x - A z||^2 + lambda ||z||_1 and is solved by textbook FISTA.
Nothing here calls the oracle: these helpers are the things the oracle is
pinned against.
"""
from __future__ import annotations

import numpy as np
from scipy.signal import convolve


def design_matrix(D: np.ndarray, T: tuple) -> np.ndarray:
    """A with A[:, (k,s)] = vec(e_s * D_k) (all channels), s over the valid domain."""
    D = np.asarray(D, np.float64)
    K, P = D.shape[:2]
    L = D.shape[2:]
    Tz = tuple(t - l + 1 for t, l in zip(T, L))
    cols = []
    for k in range(K):
        for s in np.ndindex(*Tz):
            imp = np.zeros(Tz)
            imp[s] = 1.0
            col = np.stack([convolve(imp, D[k, p], mode="full") for p in range(P)])
            assert col.shape[1:] == tuple(T)
            cols.append(col.ravel())
    return np.stack(cols, axis=1)


def lasso_objective(A, x, z, lam):
    r = x - A @ z
    return 0.5 * float(r @ r) + lam * float(np.abs(z).sum())


def soft(u, lam):
    return np.sign(u) * np.maximum(np.abs(u) - lam, 0.0)


def fista(A, x, lam, n_iter=200_000, tol=1e-15):
    """FISTA with function-value restart on 1/2||x - Az||^2 + lam ||z||_1."""
    Lip = np.linalg.norm(A, 2) ** 2
    z = np.zeros(A.shape[1])
    y = z.copy()
    t = 1.0
    f_old = lasso_objective(A, x, z, lam)
    for _ in range(n_iter):
        g = A.T @ (A @ y - x)
        z_new = soft(y - g / Lip, lam / Lip)
        f_new = lasso_objective(A, x, z_new, lam)
        if f_new > f_old:  # restart momentum
            t = 1.0
            y = z.copy()
            continue
        t_new = 0.5 * (1 + np.sqrt(1 + 4 * t * t))
        y = z_new + ((t - 1) / t_new) * (z_new - z)
        if np.max(np.abs(z_new - z)) < tol:
            z = z_new
            break
        z, t, f_old = z_new, t_new, f_new
    return z


def beta_explicit(A, x, z):
    """beta = A^T (x - A z) + diag(A^T A) z (the definition of beta, Section 3)."""
    return A.T @ (x - A @ z) + (A * A).sum(axis=0) * z


def cd_explicit(A, x, lam, eps, order_blocks, max_sweeps=100_000):
    """Coordinate descent on the explicit LASSO where each step takes the
    block ``order_blocks[m]`` (a list of column indices, visited cyclically),
    picks its largest |dz| (first index on ties) and applies it if >= eps.
    Stops after a full cycle of blocks that applied nothing."""
    n = A.shape[1]
    z = np.zeros(n)
    nrm = (A * A).sum(axis=0)
    r = x.copy()
    M = len(order_blocks)
    quiet = 0
    m = 0
    updates = 0
    for _ in range(max_sweeps * M):
        cols = order_blocks[m]
        b = A[:, cols].T @ r + nrm[cols] * z[cols]
        znew = soft(b, lam) / nrm[cols]
        dz = np.abs(znew - z[cols])
        j = int(np.argmax(dz))
        if dz[j] >= eps:
            c = cols[j]
            r -= A[:, c] * (znew[j] - z[c])
            z[c] = znew[j]
            quiet = 0
            updates += 1
        else:
            quiet += 1
        m = (m + 1) % M
        if quiet >= M:
            break
    return z, updates
