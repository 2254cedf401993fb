"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws inputs: a dictionary of unit-norm Gaussian atoms, a
Bernoulli-Gaussian activation map and a noisy observation X = Z * D + noise
(the convolutional model, Eq. model).  It contains none of the solver's
arithmetic and is shared, as a source of identical input bytes, by the CUDA
path, the oracle and the benchmark.

Inputs are returned as float32 arrays: both sides read the same fp32 values
(the oracle widens them to float64 exactly).  Layouts:
  1-D: X (P, T),      D (K, P, L),      Z (K, T - L + 1)
  2-D: X (P, T0, T1), D (K, P, L0, L1), Z (K, T0 - L0 + 1, T1 - L1 + 1)
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Workload:
    """One problem family: sizes and the generating distribution."""
    name: str
    P: int
    K: int
    T: tuple
    L: tuple
    density: float
    sigma: float
    nonneg: bool = False
    reg: float = 0.1          # lambda = reg * lambda_max
    tol: float = 1e-4         # stop when max |dZ| < tol
    amp: float = 1.0          # standard deviation of the nonzero activations


# The workloads named in the project's benchmark configuration.
IMAGE_64 = Workload("csc2d_64x64_P1_K5_L8", 1, 5, (64, 64), (8, 8), 0.01, 0.1)
SIGNAL_200K = Workload("csc1d_T200000_P5_K10_L64", 5, 10, (200_000,), (64,), 0.005, 0.1)
IMAGE_4096 = Workload("csc2d_4096x4096_P1_K25_L32", 1, 25, (4096, 4096), (32, 32), 1e-4, 0.05,
                      nonneg=True)
IMAGE_8192 = Workload("csc2d_8192x8192_P1_K25_L32", 1, 25, (8192, 8192), (32, 32), 5e-5, 0.05,
                      nonneg=True)
SERVED_ATOMS = dict(P=3, K=16, L=(12, 12), density=0.002, sigma=0.1)
# coordinate-selection comparison on one worker (Section 5.1): 7 channels, 25
# atoms of 250, rho = 0.007, activations N(0, 10^2), noise variance 1
SELECTION_150L = Workload("selection_T150L_P7_K25_L250", 7, 25, (150 * 250,), (250,), 0.007, 1.0, amp=10.0)
SELECTION_750L = Workload("selection_T750L_P7_K25_L250", 7, 25, (750 * 250,), (250,), 0.007, 1.0, amp=10.0)


def scaled(w: Workload, T: tuple, name: str | None = None) -> Workload:
    """The same family at another signal size (used for small parity cases)."""
    return Workload(name or f"{w.name}@{'x'.join(map(str, T))}", w.P, w.K, tuple(T), w.L,
                    w.density, w.sigma, w.nonneg, w.reg, w.tol)


def make_dictionary(rng: np.random.Generator, K: int, P: int, L: tuple) -> np.ndarray:
    """K atoms of P x L with i.i.d. N(0,1) entries, each scaled to unit L2 norm."""
    D = rng.standard_normal((K, P) + tuple(L))
    nrm = np.sqrt((D.reshape(K, -1) ** 2).sum(axis=1))
    D /= nrm.reshape((K,) + (1,) * (D.ndim - 1))
    return D.astype(np.float32)


def _full_conv(z: np.ndarray, d: np.ndarray) -> np.ndarray:
    """Full linear convolution of one activation map with one atom channel."""
    if z.ndim == 1:
        return np.convolve(z, d, mode="full")
    from scipy.signal import fftconvolve
    return fftconvolve(z, d, mode="full")


def make_problem(w: Workload, seed: int, D: np.ndarray | None = None):
    """Draw (X, D, Z_true) for workload ``w`` from ``numpy.random.default_rng(seed)``.

    Z_true ~ Bernoulli(density) x N(0,1) (absolute value when ``nonneg``),
    X = Z_true * D + N(0, sigma^2).  A dictionary may be passed in to keep it
    resident across requests."""
    rng = np.random.default_rng(seed)
    if D is None:
        D = make_dictionary(rng, w.K, w.P, w.L)
    T = tuple(w.T)
    Tz = tuple(t - l + 1 for t, l in zip(T, w.L))
    n = int(np.prod(Tz))
    Z = np.zeros((w.K,) + Tz, dtype=np.float32 if w.density < 0.05 else np.float64)
    if w.density < 0.05:
        # i.i.d. Bernoulli(density) per coordinate, drawn as a binomial count
        # and a uniform subset of positions per atom
        for k in range(w.K):
            cnt = int(rng.binomial(n, w.density))
            pos = rng.choice(n, size=cnt, replace=False)
            amp = w.amp * rng.standard_normal(cnt)
            Z[k].reshape(-1)[pos] = np.abs(amp) if w.nonneg else amp
    else:
        mask = rng.random((w.K,) + Tz) < w.density
        amp = w.amp * rng.standard_normal((w.K,) + Tz)
        if w.nonneg:
            amp = np.abs(amp)
        Z[...] = np.where(mask, amp, 0.0)
    X = np.zeros((w.P,) + T)
    D64 = D.astype(np.float64)
    for k in range(w.K):
        idx = np.nonzero(Z[k])
        nnz = len(idx[0])
        if nnz == 0:
            continue
        if nnz * int(np.prod(w.L)) < 8 * int(np.prod(Tz)):
            # sparse map: add each nonzero's shifted atom
            z = Z[k][idx].astype(np.float64)
            for off in np.ndindex(*w.L):
                tgt = tuple(i + o for i, o in zip(idx, off))
                for p in range(w.P):
                    np.add.at(X[p], tgt, z * D64[(k, p) + off])
        else:
            for p in range(w.P):
                X[p] += _full_conv(Z[k], D64[k, p])
    X += w.sigma * rng.standard_normal(X.shape)
    return X.astype(np.float32), D, Z.astype(np.float32, copy=False)


def make_image_device(w: Workload, seed: int, D: np.ndarray, device="cuda"):
    """A 2-D observation for benchmark inputs too large to build on the host:
    Z is drawn as in ``make_problem`` (the same sequence from the same seed),
    and X = Z * D + noise is formed on ``device`` in float32 (a transposed
    convolution of Z with the atoms, then N(0, sigma^2) from torch's generator
    seeded from the same stream).  Returns X as a float32 device tensor."""
    import torch
    rng = np.random.default_rng(seed)
    if len(w.T) != 2:
        raise ValueError("2-D workloads only")
    Tz = tuple(t - l + 1 for t, l in zip(w.T, w.L))
    n = int(np.prod(Tz))
    Zd = torch.zeros((w.K, n), dtype=torch.float32, device=device)
    for k in range(w.K):
        cnt = int(rng.binomial(n, w.density))
        pos = rng.choice(n, size=cnt, replace=False)
        amp = w.amp * rng.standard_normal(cnt)
        if w.nonneg:
            amp = np.abs(amp)
        Zd[k, torch.from_numpy(pos).to(device)] = torch.from_numpy(amp.astype(np.float32)).to(device)
    Dd = torch.from_numpy(np.ascontiguousarray(D, dtype=np.float32)).to(device)
    X = torch.nn.functional.conv_transpose2d(Zd.view((1, w.K) + Tz), Dd)[0]
    g = torch.Generator(device=device)
    g.manual_seed(int(rng.integers(1 << 62)))
    X += w.sigma * torch.randn(X.shape, generator=g, device=device, dtype=torch.float32)
    return X.contiguous()


def served_sizes(n: int, seed: int, lo: int = 64, hi: int = 2048):
    """Square image sides, log-uniform in [lo, hi], rounded to integers."""
    rng = np.random.default_rng(seed)
    return np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), size=n))).astype(int)


def poisson_arrivals(n: int, rate_hz: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_hz, size=n))
