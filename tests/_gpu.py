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
