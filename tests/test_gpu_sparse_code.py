"""csc_sparse_code: the nonzeros of a solved Z as a (position, atom)-ordered
list, checked against numpy's own listing of the same Z, plus the count-only
and too-small-capacity paths."""
import numpy as np
import pytest

from synthetic import Workload, make_problem
from tests._gpu import dev, host

pytestmark = pytest.mark.gpu

W2 = Workload("sc2d", P=2, K=5, T=(150, 170), L=(8, 8), density=0.01, sigma=0.1)
W1 = Workload("sc1d", P=3, K=4, T=(3000,), L=(32,), density=0.01, sigma=0.1)


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


def _listing(Z):
    """(k, s, value) of the nonzeros of Z (K x positions), positions
    ascending, atoms ascending within a position."""
    Zf = Z.reshape(Z.shape[0], -1)
    s, k = np.nonzero(Zf.T)  # row-major over (position, atom)
    return k.astype(np.int32), s.astype(np.int32), Zf[k, s]


@pytest.mark.parametrize("w", [W2, W1], ids=["2d", "1d"])
def test_sparse_code_lists_the_nonzeros_in_order(pkg, w):
    X, D, _ = make_problem(w, 51)
    Xd, Dd = dev(X), dev(D)
    beta, dtd, lmax = pkg.csc_init_beta(Xd, Dd)
    Z, st = pkg.csc_lgcd_solve(Xd, Dd, dtd, beta, 0.1 * lmax, 1e-4)
    Zh = host(Z)
    k, s, v, n = pkg.sparse_code(Z, X.shape, D.shape)
    kr, sr, vr = _listing(Zh)
    assert n == len(kr) == st["nnz"] > 0
    assert np.array_equal(host(k), kr) and np.array_equal(host(s), sr)
    assert np.array_equal(host(v), vr)  # the stored bits, copied


def test_sparse_code_capacity_and_empty(pkg):
    import torch
    X, D, _ = make_problem(W2, 52)
    Xd, Dd = dev(X), dev(D)
    beta, dtd, lmax = pkg.csc_init_beta(Xd, Dd)
    Z, st = pkg.csc_lgcd_solve(Xd, Dd, dtd, beta, 0.1 * lmax, 1e-4)
    n = st["nnz"]
    small = tuple(torch.empty(n - 1, dtype=t, device=Z.device) for t in (torch.int32, torch.int32, torch.float32))
    with pytest.raises(pkg.CscError) as e:
        pkg.sparse_code(Z, X.shape, D.shape, out=small)
    assert e.value.status == pkg.CSC_ERR_WORKSPACE and e.value.stats["nnz"] == n
    k, s, v, m = pkg.sparse_code(torch.zeros_like(Z), X.shape, D.shape, out=small)
    assert m == 0 and k.numel() == 0
