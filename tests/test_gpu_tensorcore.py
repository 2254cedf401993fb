"""beta-init on the tensor cores (tcgen05, split-bf16 products, FP32
accumulation) against the oracle's correlation (Alg. 1 initialisation).

The bound follows from the splitting: with x = x_hi + x_lo + e_x,
|e_x| <= 2^-18 |x| (two bf16 roundings), the computed x_hi d_hi + x_hi d_lo
+ x_lo d_hi differs from x d by at most (2^-18 + 2^-17) |x||d| plus the
FP32 accumulation over n = P L0 roundup(L1, 16) products (two gamma_n for
the tensor core's summation order).  Summed over the window the bound is
(2^-16 + 2 gamma_n) times the correlation of |X| with |D|, elementwise."""
import numpy as np
import pytest

from synthetic import SIGNAL_200K, Workload, make_problem, scaled
from tests._gpu import dev, gamma, host

pytestmark = pytest.mark.gpu

CASES = [
    Workload("tc1d", P=5, K=10, T=(3001,), L=(64,), density=0.005, sigma=0.1),
    Workload("tc2d", P=2, K=5, T=(70, 150), L=(8, 12), density=0.01, sigma=0.1),
    Workload("tc25", P=1, K=25, T=(150, 290), L=(32, 32), density=1e-3, sigma=0.05, nonneg=True),
    Workload("tcserved", P=3, K=16, T=(97, 131), L=(12, 12), density=0.002, sigma=0.1),
    Workload("tc1tap", P=1, K=3, T=(200,), L=(1,), density=0.05, sigma=0.1),
    # rows of X on 16-byte boundaries (T1 a multiple of 4): the builders' 16-byte
    # loads, ragged last tiles included
    Workload("tc1d_x4", P=5, K=10, T=(3004,), L=(64,), density=0.005, sigma=0.1),
    Workload("tc25_x4", P=1, K=25, T=(150, 292), L=(32, 32), density=1e-3, sigma=0.05, nonneg=True),
    Workload("tcserved_x4", P=3, K=16, T=(97, 132), L=(12, 12), density=0.002, sigma=0.1),
]


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1901_09235_gb300 as p
    from paper_1901_09235_gb300 import build
    build.build()
    p.load()
    return p


@pytest.mark.parametrize("w", CASES, ids=[w.name for w in CASES])
def test_beta_init_bf16x3_within_split_bound(pkg, orc, w):
    X, D, _ = make_problem(w, 51)
    beta, dtd, lmax = pkg.csc_init_beta_bf16x3(dev(X), dev(D))
    ref = orc.beta_init(X, D)
    absref = orc.beta_init(np.abs(X), np.abs(D))
    n = w.P * (w.L[0] if len(w.L) == 2 else 1) * (-(-w.L[-1] // 16) * 16)
    bound = (2.0 ** -16 + 2 * gamma(n)) * absref + 1e-30
    err = np.abs(host(beta).astype(np.float64) - ref)
    assert np.all(err <= bound), (err / bound).max()
    assert abs(lmax - np.abs(ref).max()) <= bound.max()
    # the D^T D table is the FP32 path's
    _, dtd32, _ = pkg.csc_init_beta(dev(X), dev(D))
    np.testing.assert_array_equal(host(dtd), host(dtd32))


def test_beta_init_bf16x3_signal_200k(pkg, orc):
    """The 1-D bench workload at full size: sampled outputs against the oracle."""
    w = SIGNAL_200K
    X, D, _ = make_problem(w, 0)
    beta, _, _ = pkg.csc_init_beta_bf16x3(dev(X), dev(D))
    bh = host(beta)
    rng = np.random.default_rng(7)
    ks = rng.integers(0, w.K, 400)
    ss = rng.integers(0, bh.shape[1], 400)
    ref = orc.beta_at(X, D, ks, ss)
    absref = orc.beta_at(np.abs(X), np.abs(D), ks, ss)
    bound = (2.0 ** -16 + 2 * gamma(w.P * 64)) * absref
    assert np.all(np.abs(bh[ks, ss].astype(np.float64) - ref) <= bound)
