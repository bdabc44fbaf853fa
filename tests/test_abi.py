"""C ABI checks that need no GPU: the library builds/loads, exports every symbol the headers
declare, validates arguments and sizes workspaces without touching a device."""
import ctypes as C
import glob
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1606_09402_gb300 import _lib, build
    build.build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_1606_09402_gb300 import _lib
    headers = glob.glob(os.path.join(ROOT, "include", "*.h"))
    assert headers
    names = set()
    for h in headers:
        names.update(_lib.declared_symbols(h))
    assert "qb_ei_dense" in names and "qb_fp_dense" in names
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_status_strings(lib):
    assert lib.qb_status_str(0) == b"QB_OK"
    assert lib.qb_status_str(-5) == b"QB_ERR_WORKSPACE"
    assert lib.qb_status_str(12345) == b"QB_UNKNOWN_STATUS"


def _dense(m, n, dtype=0):
    from paper_1606_09402_gb300 import _lib
    return _lib.qb_dense(m=m, n=n, ld=n, dtype=dtype, reserved=0, a=C.c_void_p(16),
                         a_lo=C.c_void_p(32), src_norm2=float("nan"))


def _opts(**kw):
    from paper_1606_09402_gb300 import _lib
    o = dict(tol=1e-3, relative=1, b=64, P=1, row_by_row=1, seed=1, rank_cap=0, l_tilde=0,
             prec=0, flags=0)
    o.update(kw)
    return _lib.qb_opts(**o)


def test_workspace_query_scales(lib):
    d = _dense(2000, 1000)
    o = _opts(b=20)
    ei = lib.qb_dense_workspace(C.byref(d), C.byref(o), 0)
    fp = lib.qb_dense_workspace(C.byref(d), C.byref(o), 1)
    assert 0 < ei < fp
    # FP holds G (m x l~) and H (n x l~) in float64
    lt = 50 * 20
    assert fp >= 8 * (2000 + 1000) * lt


def test_invalid_arguments_rejected(lib):
    d = _dense(100, 50)
    for bad in (_opts(b=0), _opts(b=65), _opts(P=-1), _opts(tol=-1.0), _opts(prec=7)):
        assert lib.qb_dense_workspace(C.byref(d), C.byref(bad), 0) == 0
    # mixed precision needs bf16/f32 storage, fp64 needs f64 storage
    assert lib.qb_dense_workspace(C.byref(d), C.byref(_opts(prec=1)), 0) == 0
    assert lib.qb_dense_workspace(C.byref(_dense(100, 50, 3)), C.byref(_opts(prec=0)), 0) == 0
    info = (C.c_char * 128)()
    rc = lib.qb_ei_dense(C.byref(d), C.byref(_opts(b=0)), None, 100, None, 50, None, 0, None, None)
    assert rc == -1
    rc = lib.qb_ei_dense(C.byref(d), C.byref(_opts()), C.c_void_p(64), 10, C.c_void_p(64), 50,
                         None, 0, None, None)
    assert rc == -1   # ldq < m
    assert lib.qb_omega(10, 0, 4, 1, 9, None, 10, None) == -1
    del info


def test_csr_workspace(lib):
    from paper_1606_09402_gb300 import _lib
    s = _lib.qb_csr(m=1000, n=500, nnz=20000, rowptr=C.c_void_p(16), colind=C.c_void_p(16),
                    dtype=0, reserved=0, val=C.c_void_p(16))
    o = _opts(b=32)
    ws = lib.qb_csr_workspace(C.byref(s), C.byref(o), 0)
    assert ws > 20000 * (4 + 8)  # CSC copy of A
