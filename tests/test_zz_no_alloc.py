"""The allocation-free form of the dictionary statistics.

Some callers cannot allocate device memory when they need phi and psi (a
plugin whose host application owns every device allocation, a service that
reserves all of its memory at start-up).  cdl_dict_stats_noalloc serves them
from a scratch array built into the library.  These tests call it through the
C ABI and check it against cdl_dict_stats (caller workspace) on two calls in a
row with different problems, so that anything the first call leaves in the
shared array would show up in the second.  This file is collected last."""
import ctypes as C

import numpy as np
import pytest

from synthetic import Workload, make_problem

pytestmark = pytest.mark.gpu

W_A = Workload("na1d", P=5, K=10, T=(3001,), L=(64,), density=0.005, sigma=0.1)
W_B = Workload("na2d", P=2, K=5, T=(70, 150), L=(8, 12), density=0.01, sigma=0.1)


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1901_09235_gb300 as p
    from paper_1901_09235_gb300 import build
    build.build()
    lib = p.load()
    fn = lib.cdl_dict_stats_noalloc
    fn.restype = C.c_int
    fn.argtypes = [C.POINTER(p.Shape), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    return p


def _noalloc(pkg, Z, X, D_shape):
    """Direct C-ABI call with caller-owned output buffers and no workspace."""
    import torch
    s = pkg.make_shape(tuple(X.shape), tuple(D_shape))
    phi = torch.full(pkg.tab_shape(s), float("nan"), dtype=torch.float32, device=X.device)
    psi = torch.full(tuple(D_shape), float("nan"), dtype=torch.float32, device=X.device)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = pkg.load().cdl_dict_stats_noalloc(C.byref(s), C.c_void_p(Z.data_ptr()), C.c_void_p(X.data_ptr()),
                                           C.c_void_p(phi.data_ptr()), C.c_void_p(psi.data_ptr()), stream)
    assert rc == pkg.CSC_OK, pkg.status_string(rc)
    torch.cuda.synchronize()
    return phi.cpu().numpy(), psi.cpu().numpy()


def _close(got, ref):
    np.testing.assert_allclose(got, ref, rtol=1e-6, atol=1e-6 * max(1.0, float(np.abs(ref).max())))


def test_noalloc_matches_workspace_form_twice(pkg):
    import torch
    for w, seed in ((W_A, 31), (W_B, 32), (W_A, 33)):
        X, D, Z = make_problem(w, seed)
        Xd, Zd = torch.from_numpy(X).cuda(), torch.from_numpy(Z).cuda()
        phi_ref, psi_ref = pkg.cdl_dict_stats(Zd, Xd, D.shape)
        phi_ref, psi_ref = phi_ref.cpu().numpy(), psi_ref.cpu().numpy()
        phi, psi = _noalloc(pkg, Zd, Xd, D.shape)
        _close(phi, phi_ref)
        _close(psi, psi_ref)


def test_noalloc_rejects_problems_beyond_its_scratch(pkg):
    import torch
    s = pkg.make_shape((1, 512, 512), (25, 1, 32, 32))  # phi accumulators alone exceed the array
    dummy = torch.zeros(4, dtype=torch.float32, device="cuda")
    p = C.c_void_p(dummy.data_ptr())
    rc = pkg.load().cdl_dict_stats_noalloc(C.byref(s), p, p, p, p, None)
    assert rc == pkg.CSC_ERR_WORKSPACE


def test_noalloc_holds_more_nonzeros_than_the_workspace_list(pkg, orc):
    """The nonzero list takes whatever the fixed array leaves after the
    accumulators: a Z with more nonzeros than the workspace form's list
    (max(2^16, K |Omega| / 16) entries) still fits, and phi / psi match the
    FP64 oracle within the bounds of their FP32 and FP64 sums."""
    import torch
    from tests._gpu import gamma
    w = Workload("na_dense", P=1, K=4, T=(300_000,), L=(16,), density=0.08, sigma=0.1)
    X, D, Z = make_problem(w, 34)
    nnz = int((Z != 0).sum())
    nz = Z.size
    assert nnz > max(1 << 16, nz // 16) and nnz * 12 < (7 << 20)
    Xd, Zd = torch.from_numpy(X).cuda(), torch.from_numpy(Z).cuda()
    phi, psi = _noalloc(pkg, Zd, Xd, D.shape)
    pr, sr = orc.phi_psi(Z, X, w.L)
    pa, sa = orc.phi_psi(np.abs(Z), np.abs(X), w.L)
    assert np.all(np.abs(phi - pr) <= 2.0 ** -24 * np.abs(pr) + 1e-12 * pa)
    assert np.all(np.abs(psi - sr) <= gamma(65) * sa + 1e-12 * np.abs(sr).max())
