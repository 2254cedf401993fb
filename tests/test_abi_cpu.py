"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, exports every function declared in include/*.h, and rejects
invalid shapes before touching a device."""
import ctypes as C
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1901_09235_gb300 import build
    build.build()
    import paper_1901_09235_gb300 as pkg
    return pkg.load()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        names |= set(re.findall(r"CSC_API\s+[\w\s\*]+?\b(\w+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("csc_init_beta", "csc_lgcd_solve", "cdl_dict_stats", "cdl_dict_update"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1901_09235_gb300 import library_path
    out = subprocess.run(["nm", "-D", "--defined-only", library_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (\w+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert getattr(lib, n) is not None


def test_status_strings_and_defaults(lib):
    import paper_1901_09235_gb300 as pkg
    assert pkg.status_string(0) == "ok"
    assert "workspace" in pkg.status_string(7)
    o = pkg.default_opts()
    assert o.mode == pkg.MODE_ASYNC and o.beta_refresh == 2 and o.timeout_s > 0


@pytest.mark.parametrize("bad", [
    dict(d=3, P=1, K=1, T=(8, 1), L=(2, 1)),
    dict(d=1, P=0, K=1, T=(8, 1), L=(2, 1)),
    dict(d=1, P=1, K=1, T=(8, 1), L=(9, 1)),
    dict(d=1, P=1, K=1, T=(8, 2), L=(2, 1)),
    dict(d=2, P=1, K=1, T=(8, 8), L=(2, 9)),
])
def test_invalid_shapes_rejected_on_host(lib, bad):
    import paper_1901_09235_gb300 as pkg
    s = pkg.Shape()
    s.d, s.P, s.K = bad["d"], bad["P"], bad["K"]
    s.T[0], s.T[1] = bad["T"]
    s.L[0], s.L[1] = bad["L"]
    n = C.c_size_t(0)
    assert lib.csc_workspace_size(C.byref(s), None, C.byref(n)) == pkg.CSC_ERR_INVALID
    rc = lib.csc_init_beta(C.byref(s), None, None, None, None, None, None, 0, None)
    assert rc == pkg.CSC_ERR_INVALID


def test_workspace_size_grows_with_problem(lib):
    import paper_1901_09235_gb300 as pkg
    a = pkg.workspace_size(pkg.make_shape((1, 64, 64), (5, 1, 8, 8)))
    b = pkg.workspace_size(pkg.make_shape((1, 256, 256), (5, 1, 8, 8)))
    assert 0 < a < b


def test_null_pointers_rejected(lib):
    import paper_1901_09235_gb300 as pkg
    s = pkg.make_shape((2, 100), (3, 2, 5))
    st = pkg.SolveStats()
    rc = lib.csc_lgcd_solve(C.byref(s), None, None, None, None, None, 0.1, 1e-4, None, None, 0,
                            C.byref(st), None)
    assert rc == pkg.CSC_ERR_INVALID
    assert lib.cdl_dict_stats(C.byref(s), None, None, None, None, None, 0, None) == pkg.CSC_ERR_INVALID


def test_sparse_code_arguments_rejected_on_host(lib):
    """csc_sparse_code validates its pointers, capacity and workspace size
    before any device work."""
    import paper_1901_09235_gb300 as pkg
    s = pkg.make_shape((1, 64, 64), (5, 1, 8, 8))
    n = C.c_longlong(-1)
    fake = C.c_void_p(0x1000)  # never dereferenced: every case fails on the host
    ws_need = pkg.workspace_size(s)

    def call(Z=fake, k=fake, sv=fake, v=fake, cap=16, nnz=True, ws=fake, ws_bytes=ws_need):
        return lib.csc_sparse_code(C.byref(s), Z, k, sv, v, cap, C.byref(n) if nnz else None, ws, ws_bytes, None)

    assert call(Z=None) == pkg.CSC_ERR_INVALID
    assert call(nnz=False) == pkg.CSC_ERR_INVALID
    assert call(ws=None) == pkg.CSC_ERR_INVALID
    assert call(cap=-1) == pkg.CSC_ERR_INVALID
    for missing in ("k", "sv", "v"):
        assert call(**{missing: None}) == pkg.CSC_ERR_INVALID, missing
    assert call(ws_bytes=1024) == pkg.CSC_ERR_WORKSPACE
    bad = pkg.make_shape((1, 64, 64), (5, 1, 8, 8))
    bad.K = 0
    assert lib.csc_sparse_code(C.byref(bad), fake, fake, fake, fake, 16, C.byref(n), fake, ws_need,
                               None) == pkg.CSC_ERR_INVALID


def test_option_and_queue_arguments_rejected_on_host(lib):
    """Out-of-range solve options and queue densities are refused before any
    device work (the pointers below are never dereferenced)."""
    import paper_1901_09235_gb300 as pkg
    s = pkg.make_shape((2, 100), (3, 2, 5))
    st = pkg.SolveStats()
    fake = [C.c_void_p(16 * (i + 1)) for i in range(6)]
    for bad in (-0.1, 1.5, float("nan")):
        o = pkg.default_opts(stop_margin=bad)
        rc = lib.csc_lgcd_solve(C.byref(s), fake[0], fake[1], fake[2], fake[3], fake[4], 0.1, 1e-4,
                                C.byref(o), fake[5], 1 << 30, C.byref(st), None)
        assert rc == pkg.CSC_ERR_INVALID, bad
    atoms = pkg.Shape()
    atoms.d, atoms.P, atoms.K = 2, 3, 16
    atoms.T[0] = atoms.T[1] = atoms.L[0] = atoms.L[1] = 12
    db, hb = C.c_size_t(0), C.c_size_t(0)
    for dens in (1, 4, -2):
        assert lib.csc_queue_workspace_size(C.byref(atoms), 8, 4, dens, C.byref(db), C.byref(hb)) == \
            pkg.CSC_ERR_INVALID
    sizes = []
    for dens in (0, 2, 3):
        assert lib.csc_queue_workspace_size(C.byref(atoms), 8, 4, dens, C.byref(db), C.byref(hb)) == pkg.CSC_OK
        sizes.append(db.value)
    # the default is two CTAs per SM; three need larger per-slot control areas
    assert sizes[0] == sizes[1] < sizes[2]


def test_cdl_step_arguments_rejected_on_host(lib):
    """The fused loop-body call refuses missing buffers, neither a positive
    lambda nor a positive reg, a non-positive tol, a NaN ||X||^2 and a short
    workspace before any device work (the pointers below are never
    dereferenced)."""
    import paper_1901_09235_gb300 as pkg
    s = pkg.make_shape((2, 100), (3, 2, 5))
    st = pkg.SolveStats()
    fake = [C.c_void_p(16 * (i + 1)) for i in range(8)]
    need = pkg.workspace_size(s)

    def call(ptrs=fake[:7], reg=0.1, lam=0.0, tol=1e-4, xs=1.0, ws=fake[7], ws_bytes=need):
        lo, fd, it = C.c_double(0), C.c_double(0), C.c_int(0)
        return lib.cdl_step(C.byref(s), *ptrs, reg, lam, tol, xs, 50, 1e-8, None, ws, ws_bytes, C.byref(st),
                            C.byref(lo), C.byref(fd), C.byref(it), None)

    for i in range(7):
        ptrs = list(fake[:7])
        ptrs[i] = None
        assert call(ptrs=ptrs) == pkg.CSC_ERR_INVALID, i
    assert call(ws=None) == pkg.CSC_ERR_INVALID
    for reg in (0.0, -1.0, float("nan")):
        assert call(reg=reg) == pkg.CSC_ERR_INVALID
        assert call(reg=reg, lam=float("nan")) == pkg.CSC_ERR_INVALID
    assert call(tol=0.0) == pkg.CSC_ERR_INVALID
    assert call(xs=float("nan")) == pkg.CSC_ERR_INVALID
    bad_opts = pkg.default_opts(beta_init=2)
    lo, fd, it = C.c_double(0), C.c_double(0), C.c_int(0)
    assert lib.cdl_step(C.byref(s), *fake[:7], 0.1, 0.0, 1e-4, 1.0, 50, 1e-8, C.byref(bad_opts), fake[7], need,
                        C.byref(st), C.byref(lo), C.byref(fd), C.byref(it), None) == pkg.CSC_ERR_INVALID
    assert call(ws_bytes=1024) == pkg.CSC_ERR_WORKSPACE


def test_every_compute_call_refuses_null_buffers_on_the_host(lib):
    """Each entry point that takes device buffers checks them before any
    device work: with a valid shape and null buffers it returns
    CSC_ERR_INVALID (never CSC_ERR_CUDA, which would mean it reached the
    device first)."""
    import paper_1901_09235_gb300 as pkg
    s = pkg.make_shape((2, 40, 40), (3, 2, 5, 5))
    d, n = C.c_double(0.0), C.c_longlong(0)
    it = C.c_int(0)
    st = pkg.SolveStats()
    o = pkg.default_opts()
    calls = {
        "csc_init_beta": lambda: lib.csc_init_beta(C.byref(s), None, None, None, None, None, None, 0, None),
        "csc_init_beta_f64": lambda: lib.csc_init_beta_f64(C.byref(s), None, None, None, None, None, None, 0,
                                                           None),
        "csc_init_beta_bf16x3": lambda: lib.csc_init_beta_bf16x3(C.byref(s), None, None, None, None, None, None,
                                                                 0, None),
        "csc_lgcd_solve": lambda: lib.csc_lgcd_solve(C.byref(s), None, None, None, None, None, 0.1, 1e-4,
                                                     C.byref(o), None, 0, C.byref(st), None),
        "csc_lgcd_solve_f64": lambda: lib.csc_lgcd_solve_f64(C.byref(s), None, None, None, None, None, 0.1, 1e-4,
                                                             C.byref(o), None, 0, C.byref(st), None),
        "csc_objective": lambda: lib.csc_objective(C.byref(s), None, None, None, 0.1, C.byref(d), None, 0, None),
        "cdl_dict_stats": lambda: lib.cdl_dict_stats(C.byref(s), None, None, None, None, None, 0, None),
        "cdl_dict_update": lambda: lib.cdl_dict_update(C.byref(s), None, None, 1.0, None, 10, 1e-8, C.byref(d),
                                                       C.byref(it), None, 0, None),
        "csc_refresh_beta": lambda: lib.csc_refresh_beta(C.byref(s), None, None, None, 0.1, None, C.byref(d),
                                                         C.byref(d), None, 0, None),
        "csc_rcd_solve": lambda: lib.csc_rcd_solve(C.byref(s), None, None, None, None, 0.1, None, 10, C.byref(n),
                                                   None, 0, None),
        "csc_sparse_code": lambda: lib.csc_sparse_code(C.byref(s), None, None, None, None, 0, C.byref(n), None,
                                                       0, None),
        "cdl_fit": lambda: lib.cdl_fit(C.byref(s), None, None, None, None, None, None, None, 0.1, 1e-4, 2, 0.0,
                                       10, 1e-8, C.byref(o), None, 0, None, C.byref(it), None),
    }
    for name, call in calls.items():
        assert call() == pkg.CSC_ERR_INVALID, name
