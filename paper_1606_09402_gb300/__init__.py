"""GB300-native fixed-precision randomized QB factorisation (randQB_EI / randQB_FP).

Thin Python binding over the C ABI of libqb.so (include/qb.h): it only marshals arguments.
PyTorch provides device memory and the current CUDA stream; every step of the factorisation
runs in the library's CUDA kernels.

    Q, B, info = qb_fp_dense(A, tol=1e-3, b=64, P=1, seed=9402)         # float64 A
    hi, lo, norms = quantize_bf16x2(A64)                                    # mixed precision
    Q, B, info = qb_fp_dense(hi, tol=1e-3, b=64, P=1, seed=9402, a_lo=lo,
                             src_norm2=norms[0], prec="mixed")
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

from . import _lib

__all__ = ["qb_ei_dense", "qb_fp_dense", "qb_ei_csr", "qb_fp_csr", "qb_ei_coo", "qb_fp_coo",
           "qb_omega",
           "quantize_bf16x2", "qb_apass_sketch", "qb_apass_trans", "qb_fixed_rank_fwd",
           "qb_fixed_rank_bwd", "QBFixedRank", "qb_ei_batched", "qb_svd_from_qb", "QBError",
           "QBInfo",
           "launch_count", "status_str"]


class QBError(RuntimeError):
    def __init__(self, code: int, where: str):
        lib = _lib.load()
        msg = lib.qb_status_str(code).decode()
        if code == _lib.QB_ERR_CUDA:
            msg += " (" + lib.qb_last_cuda_error().decode() + ")"
        super().__init__(f"{where}: {msg}")
        self.code = code


@dataclass
class QBInfo:
    status: int
    rank: int
    err2_est: float
    err_est: float
    normA2: float
    passes: int
    omega_cols: int
    status_bits: int
    blocks: int
    launches: int

    @property
    def converged(self) -> bool:
        return self.status in (_lib.QB_OK, _lib.QB_WARN_TOL_FLOOR)


def status_str(code: int) -> str:
    return _lib.load().qb_status_str(code).decode()


def launch_count() -> int:
    return int(_lib.load().qb_launch_count())


def profile_last() -> dict:
    """Per-phase device milliseconds of the last call made with flags=QB_FLAG_PROFILE (2), or of
    the last qb_apass_sketch / qb_apass_trans call (phase "sketch" / "trans")."""
    buf = (C.c_double * len(_lib.PHASES))()
    _lib.load().qb_profile_last(buf, len(_lib.PHASES))
    return dict(zip(_lib.PHASES, (float(x) for x in buf)))


def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dtype_code(t) -> int:
    torch = _torch()
    return {torch.float64: _lib.QB_F64, torch.float32: _lib.QB_F32,
            torch.bfloat16: _lib.QB_BF16}[t.dtype]


def _opts(tol, b, P, seed, relative, rank_cap, l_tilde, row_by_row, prec, flags=0):
    return _lib.qb_opts(tol=float(tol), relative=int(bool(relative)), b=int(b), P=int(P),
                        row_by_row=int(bool(row_by_row)), seed=int(seed) & ((1 << 64) - 1),
                        rank_cap=int(rank_cap or 0), l_tilde=int(l_tilde or 0),
                        prec=_lib.QB_PREC_MIXED if prec == "mixed" else _lib.QB_PREC_FP64,
                        flags=int(flags))


def _check_dev(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise ValueError("tensors must live on a CUDA device")


def _alloc_out(m, n, cap, prec, device, out):
    torch = _torch()
    dt = torch.float64 if prec != "mixed" else torch.float32
    if out is not None:
        Q, B = out
        assert Q.dtype == dt and B.dtype == dt and Q.shape[1] == m and B.shape[1] == n
        assert Q.shape[0] >= cap and B.shape[0] >= cap
        return Q, B
    # Q is column-major m x cap: stored as a (cap, m) row-major tensor (Q^T)
    Qt = torch.empty(max(cap, 1), m, dtype=dt, device=device)
    B = torch.empty(max(cap, 1), n, dtype=dt, device=device)
    return Qt, B


def _info(rc, inf):
    return QBInfo(rc, int(inf.rank), float(inf.err2_est), float(inf.err_est), float(inf.normA2),
                  int(inf.passes), int(inf.omega_cols), int(inf.status_bits), int(inf.blocks),
                  int(inf.launches))


def _dense_call(fn, name, A, tol, b, P, seed, relative, rank_cap, l_tilde, row_by_row, prec,
                a_lo, src_norm2, stream, out, workspace, flags=0, a_lo_ready=None):
    torch = _torch()
    lib = _lib.load()
    _check_dev(A, a_lo)
    assert A.dim() == 2 and A.stride(1) == 1, "A must be row-major (contiguous rows)"
    m, n = A.shape
    if a_lo is not None:
        assert a_lo.shape == A.shape and a_lo.stride() == A.stride() and a_lo.dtype == torch.bfloat16
        dt = _lib.QB_BF16X2
    else:
        dt = _dtype_code(A)
    d = _lib.qb_dense(m=m, n=n, ld=A.stride(0), dtype=dt, reserved=0, a=A.data_ptr(),
                      a_lo=a_lo.data_ptr() if a_lo is not None else None,
                      src_norm2=float("nan") if src_norm2 is None else float(src_norm2),
                      a_lo_ready=a_lo_ready.cuda_event if a_lo_ready is not None else None)
    o = _opts(tol, b, P, seed, relative, rank_cap, l_tilde, row_by_row, prec, flags)
    algo = 1 if name.startswith("qb_fp") else 0
    wsb = lib.qb_dense_workspace(C.byref(d), C.byref(o), algo)
    if wsb == 0:
        raise QBError(_lib.QB_ERR_INVALID_ARG, name + " workspace query")
    cap = min(m, n) if not rank_cap or rank_cap <= 0 else min(m, n, int(rank_cap))
    Qt, B = _alloc_out(m, n, cap, prec, A.device, out)
    ws = workspace if workspace is not None and workspace.numel() >= wsb else \
        torch.empty(wsb, dtype=torch.uint8, device=A.device)
    inf = _lib.qb_info()
    with torch.cuda.device(A.device):
        rc = fn(C.byref(d), C.byref(o), C.c_void_p(Qt.data_ptr()), Qt.stride(0),
                C.c_void_p(B.data_ptr()), B.stride(0), C.c_void_p(ws.data_ptr()), ws.numel(),
                C.byref(inf), _stream_ptr(stream))
    if rc < 0:
        raise QBError(rc, name)
    info = _info(rc, inf)
    k = info.rank
    return Qt[:k].T, B[:k], info


def qb_ei_dense(A, tol, b, P=0, seed=0, relative=True, rank_cap=None, row_by_row=True,
                prec="fp64", a_lo=None, src_norm2=None, stream=None, out=None, workspace=None,
                flags=0, a_lo_ready=None):
    """randQB_EI (Algorithm 2) on a dense row-major A; returns (Q, B, QBInfo).

    Q is an m x rank view (column-major storage), B a rank x n row-major view.  a_lo_ready: an
    optional torch.cuda.Event recorded after a_lo's last write on another stream; the call waits
    on it right before its first read of a_lo."""
    return _dense_call(_lib.load().qb_ei_dense, "qb_ei_dense", A, tol, b, P, seed, relative,
                       rank_cap, None, row_by_row, prec, a_lo, src_norm2, stream, out, workspace,
                       flags, a_lo_ready)


def qb_fp_dense(A, tol, b, P=0, seed=0, relative=True, rank_cap=None, l_tilde=None,
                row_by_row=True, prec="fp64", a_lo=None, src_norm2=None, stream=None, out=None,
                workspace=None, flags=0, a_lo_ready=None):
    """randQB_FP (Algorithm 4) on a dense row-major A; returns (Q, B, QBInfo).  a_lo_ready as in
    qb_ei_dense: the power scheme's sketches read A_hi only, so A_lo can still be arriving."""
    return _dense_call(_lib.load().qb_fp_dense, "qb_fp_dense", A, tol, b, P, seed, relative,
                       rank_cap, l_tilde, row_by_row, prec, a_lo, src_norm2, stream, out,
                       workspace, flags, a_lo_ready)


def _csr_call(fn, name, rowptr, colind, val, shape, tol, b, P, seed, relative, rank_cap, l_tilde,
              row_by_row, stream, workspace, flags=0):
    torch = _torch()
    lib = _lib.load()
    _check_dev(rowptr, colind, val)
    assert rowptr.dtype == torch.int32 and colind.dtype == torch.int32
    m, n = shape
    prec = "fp64" if val.dtype == torch.float64 else "mixed"
    s = _lib.qb_csr(m=m, n=n, nnz=colind.numel(), rowptr=rowptr.data_ptr(),
                    colind=colind.data_ptr(), dtype=_dtype_code(val), reserved=0,
                    val=val.data_ptr())
    o = _opts(tol, b, P, seed, relative, rank_cap, l_tilde, row_by_row, prec, flags)
    algo = 1 if name.startswith("qb_fp") else 0
    wsb = lib.qb_csr_workspace(C.byref(s), C.byref(o), algo)
    if wsb == 0:
        raise QBError(_lib.QB_ERR_INVALID_ARG, name + " workspace query")
    cap = min(m, n) if not rank_cap or rank_cap <= 0 else min(m, n, int(rank_cap))
    Qt, B = _alloc_out(m, n, cap, prec, val.device, None)
    ws = workspace if workspace is not None and workspace.numel() >= wsb else \
        torch.empty(wsb, dtype=torch.uint8, device=val.device)
    inf = _lib.qb_info()
    with torch.cuda.device(val.device):
        rc = fn(C.byref(s), C.byref(o), C.c_void_p(Qt.data_ptr()), Qt.stride(0),
                C.c_void_p(B.data_ptr()), B.stride(0), C.c_void_p(ws.data_ptr()), ws.numel(),
                C.byref(inf), _stream_ptr(stream))
    if rc < 0:
        raise QBError(rc, name)
    info = _info(rc, inf)
    k = info.rank
    return Qt[:k].T, B[:k], info


def qb_ei_csr(rowptr, colind, val, shape, tol, b, P=0, seed=0, relative=True, rank_cap=None,
              row_by_row=True, stream=None, workspace=None, flags=0):
    """randQB_EI on a CSR matrix (int32 indices; float64 values -> fp64 path, float32 -> mixed)."""
    return _csr_call(_lib.load().qb_ei_csr, "qb_ei_csr", rowptr, colind, val, shape, tol, b, P,
                     seed, relative, rank_cap, None, row_by_row, stream, workspace, flags)


def qb_fp_csr(rowptr, colind, val, shape, tol, b, P=0, seed=0, relative=True, rank_cap=None,
              l_tilde=None, row_by_row=True, stream=None, workspace=None, flags=0):
    """randQB_FP on a CSR matrix."""
    return _csr_call(_lib.load().qb_fp_csr, "qb_fp_csr", rowptr, colind, val, shape, tol, b, P,
                     seed, relative, rank_cap, l_tilde, row_by_row, stream, workspace, flags)


def _coo_call(fn, name, row, col, val, shape, tol, b, P, seed, relative, rank_cap, l_tilde,
              row_by_row, stream, workspace, flags=0):
    torch = _torch()
    lib = _lib.load()
    _check_dev(row, col, val)
    assert row.dtype == torch.int32 and col.dtype == torch.int32
    assert row.numel() == col.numel() == val.numel()
    m, n = shape
    prec = "fp64" if val.dtype == torch.float64 else "mixed"
    s = _lib.qb_coo(m=m, n=n, nnz=val.numel(), row=row.data_ptr(), col=col.data_ptr(),
                    dtype=_dtype_code(val), reserved=0, val=val.data_ptr())
    o = _opts(tol, b, P, seed, relative, rank_cap, l_tilde, row_by_row, prec, flags)
    algo = 1 if name.startswith("qb_fp") else 0
    wsb = lib.qb_coo_workspace(C.byref(s), C.byref(o), algo)
    if wsb == 0:
        raise QBError(_lib.QB_ERR_INVALID_ARG, name + " workspace query")
    cap = min(m, n) if not rank_cap or rank_cap <= 0 else min(m, n, int(rank_cap))
    Qt, B = _alloc_out(m, n, cap, prec, val.device, None)
    ws = workspace if workspace is not None and workspace.numel() >= wsb else \
        torch.empty(wsb, dtype=torch.uint8, device=val.device)
    inf = _lib.qb_info()
    with torch.cuda.device(val.device):
        rc = fn(C.byref(s), C.byref(o), C.c_void_p(Qt.data_ptr()), Qt.stride(0),
                C.c_void_p(B.data_ptr()), B.stride(0), C.c_void_p(ws.data_ptr()), ws.numel(),
                C.byref(inf), _stream_ptr(stream))
    if rc < 0:
        raise QBError(rc, name)
    info = _info(rc, inf)
    k = info.rank
    return Qt[:k].T, B[:k], info


def qb_ei_coo(row, col, val, shape, tol, b, P=0, seed=0, relative=True, rank_cap=None,
              row_by_row=True, stream=None, workspace=None, flags=0):
    """randQB_EI on a COO matrix (int32 row / col indices, each (row, col) at most once, any
    order, sorted by row fastest; float64 values -> fp64 path, float32 -> mixed)."""
    return _coo_call(_lib.load().qb_ei_coo, "qb_ei_coo", row, col, val, shape, tol, b, P, seed,
                     relative, rank_cap, None, row_by_row, stream, workspace, flags)


def qb_fp_coo(row, col, val, shape, tol, b, P=0, seed=0, relative=True, rank_cap=None,
              l_tilde=None, row_by_row=True, stream=None, workspace=None, flags=0):
    """randQB_FP on a COO matrix."""
    return _coo_call(_lib.load().qb_fp_coo, "qb_fp_coo", row, col, val, shape, tol, b, P, seed,
                     relative, rank_cap, l_tilde, row_by_row, stream, workspace, flags)


def qb_omega(n, col0, w, seed, dtype=None, device="cuda", stream=None):
    """Omega rows 0..n-1, global columns col0..col0+w-1, as an n x w tensor (column-major)."""
    torch = _torch()
    dtype = dtype or torch.float64
    out_t = torch.empty(max(w, 1), max(n, 1), dtype=dtype, device=device)  # Omega^T row-major
    rc = _lib.load().qb_omega(n, col0, w, int(seed) & ((1 << 64) - 1), _dtype_code(out_t),
                              C.c_void_p(out_t.data_ptr()), out_t.stride(0), _stream_ptr(stream))
    if rc < 0:
        raise QBError(rc, "qb_omega")
    return out_t[:w, :n].T


def quantize_bf16x2(A, stream=None):
    """float64 row-major A -> (hi, lo, norms) with A ~= hi + lo (bf16 each) and
    norms = (||A||^2, ||A - hi - lo||^2, ||A - hi||^2) in float64."""
    torch = _torch()
    _check_dev(A)
    assert A.dtype == torch.float64 and A.stride(1) == 1
    m, n = A.shape
    hi = torch.empty(m, n, dtype=torch.bfloat16, device=A.device)
    lo = torch.empty(m, n, dtype=torch.bfloat16, device=A.device)
    lib = _lib.load()
    wsb = lib.qb_quantize_workspace(m, n)
    ws = torch.empty(wsb, dtype=torch.uint8, device=A.device)
    norms = (C.c_double * 3)()
    rc = lib.qb_quantize_bf16x2(C.c_void_p(A.data_ptr()), m, n, A.stride(0),
                                C.c_void_p(hi.data_ptr()), C.c_void_p(lo.data_ptr()), n, norms,
                                C.c_void_p(ws.data_ptr()), wsb, _stream_ptr(stream))
    if rc < 0:
        raise QBError(rc, "qb_quantize_bf16x2")
    return hi, lo, tuple(float(x) for x in norms)


def _dense_desc(A, a_lo=None, src_norm2=None):
    torch = _torch()
    assert A.dim() == 2 and A.stride(1) == 1, "A must be row-major (contiguous rows)"
    m, n = A.shape
    if a_lo is not None:
        assert a_lo.shape == A.shape and a_lo.stride() == A.stride() and a_lo.dtype == torch.bfloat16
        dt = _lib.QB_BF16X2
    else:
        dt = _dtype_code(A)
    return _lib.qb_dense(m=m, n=n, ld=A.stride(0), dtype=dt, reserved=0, a=A.data_ptr(),
                         a_lo=a_lo.data_ptr() if a_lo is not None else None,
                         src_norm2=float("nan") if src_norm2 is None else float(src_norm2))


def _apass(trans, A, V, precise, a_lo, stream):
    torch = _torch()
    lib = _lib.load()
    _check_dev(A, V, a_lo)
    d = _dense_desc(A, a_lo)
    m, n = A.shape
    rows_in, rows_out = (m, n) if trans else (n, m)
    w = V.shape[1]
    assert V.shape[0] == rows_in
    out_dt = torch.float64 if A.dtype == torch.float64 else torch.float32
    Vt = V.T.contiguous().to(out_dt)            # column-major V stored as V^T row-major
    Yt = torch.empty(max(w, 1), rows_out, dtype=out_dt, device=A.device)
    wsb = lib.qb_apass_workspace(C.byref(d), w)
    if wsb == 0:
        raise QBError(_lib.QB_ERR_INVALID_ARG, "qb_apass_workspace")
    ws = torch.empty(wsb, dtype=torch.uint8, device=A.device)
    with torch.cuda.device(A.device):
        if trans:
            rc = lib.qb_apass_trans(C.byref(d), C.c_void_p(Vt.data_ptr()), rows_in, w,
                                    int(precise), C.c_void_p(Yt.data_ptr()), rows_out,
                                    C.c_void_p(ws.data_ptr()), wsb, _stream_ptr(stream))
        else:
            rc = lib.qb_apass_sketch(C.byref(d), C.c_void_p(Vt.data_ptr()), rows_in, w,
                                     C.c_void_p(Yt.data_ptr()), rows_out,
                                     C.c_void_p(ws.data_ptr()), wsb, _stream_ptr(stream))
    if rc < 0:
        raise QBError(rc, "qb_apass_trans" if trans else "qb_apass_sketch")
    return Yt[:w].T


def qb_apass_sketch(A, V, a_lo=None, stream=None):
    """Y = A V (one pass over a dense row-major A; float32 V/Y for bf16 A, float64 otherwise)."""
    return _apass(False, A, V, False, a_lo, stream)


def qb_apass_trans(A, V, precise=1, a_lo=None, stream=None):
    """Z = A^T V (one pass over a dense row-major A).  For bf16 hi+lo A: precise=0 uses A_hi and
    bf16(V), 1 the three hi/lo products, 2 (A_hi + A_lo) with bf16(V)."""
    return _apass(True, A, V, precise, a_lo, stream)


def _fixed_ws(lib, d, k, prec_code, device):
    torch = _torch()
    wsb = lib.qb_fixed_rank_workspace(C.byref(d), k, prec_code)
    if wsb == 0:
        raise QBError(_lib.QB_ERR_INVALID_ARG, "qb_fixed_rank_workspace")
    return torch.empty(wsb, dtype=torch.uint8, device=device)


def qb_fixed_rank_fwd(A, k, seed, a_lo=None, stream=None):
    """Fixed-rank QB map (Omega = Philox columns 0..k-1): returns Q (m x k), B (k x n), R (k x k).
    float64 A -> float64 path; bf16 A (optionally with a_lo) -> mixed path, float32 outputs."""
    torch = _torch()
    lib = _lib.load()
    _check_dev(A, a_lo)
    d = _dense_desc(A, a_lo)
    m, n = A.shape
    f64 = A.dtype == torch.float64
    prec = _lib.QB_PREC_FP64 if f64 else _lib.QB_PREC_MIXED
    dt = torch.float64 if f64 else torch.float32
    Qt = torch.empty(k, m, dtype=dt, device=A.device)      # Q column-major
    B = torch.empty(k, n, dtype=dt, device=A.device)
    Rt = torch.empty(k, k, dtype=dt, device=A.device)      # R column-major
    ws = _fixed_ws(lib, d, k, prec, A.device)
    with torch.cuda.device(A.device):
        rc = lib.qb_fixed_rank_fwd(C.byref(d), k, int(seed) & ((1 << 64) - 1), prec,
                                   C.c_void_p(Qt.data_ptr()), m, C.c_void_p(B.data_ptr()), n,
                                   C.c_void_p(Rt.data_ptr()), k, C.c_void_p(ws.data_ptr()),
                                   ws.numel(), _stream_ptr(stream))
    if rc < 0:
        raise QBError(rc, "qb_fixed_rank_fwd")
    return Qt.T, B, Rt.T


def qb_fixed_rank_bwd(A, k, seed, Q, R, GQ, GB, a_lo=None, stream=None):
    """dL/dA for L with dL/dQ = GQ (m x k), dL/dB = GB (k x n); Q, R from qb_fixed_rank_fwd."""
    torch = _torch()
    lib = _lib.load()
    _check_dev(A, a_lo, Q, R, GQ, GB)
    d = _dense_desc(A, a_lo)
    m, n = A.shape
    f64 = A.dtype == torch.float64
    prec = _lib.QB_PREC_FP64 if f64 else _lib.QB_PREC_MIXED
    dt = torch.float64 if f64 else torch.float32
    Qc = Q.to(dt).T.contiguous()        # column-major Q stored as Q^T
    Rc = R.to(dt).T.contiguous()
    GQc = GQ.to(dt).T.contiguous()
    GBr = GB.to(dt).contiguous()        # row-major k x n
    GA = torch.empty(m, n, dtype=dt, device=A.device)
    ws = _fixed_ws(lib, d, k, prec, A.device)
    with torch.cuda.device(A.device):
        rc = lib.qb_fixed_rank_bwd(C.byref(d), k, int(seed) & ((1 << 64) - 1), prec,
                                   C.c_void_p(Qc.data_ptr()), m, C.c_void_p(Rc.data_ptr()), k,
                                   C.c_void_p(GQc.data_ptr()), m, C.c_void_p(GBr.data_ptr()), n,
                                   C.c_void_p(GA.data_ptr()), n, C.c_void_p(ws.data_ptr()),
                                   ws.numel(), _stream_ptr(stream))
    if rc < 0:
        raise QBError(rc, "qb_fixed_rank_bwd")
    return GA


def qb_ei_batched(As, tols, seed=0, rank_cap=None, relative=True, row_by_row=True, stream=None,
                  outs=None, workspace=None):
    """Batched randQB_EI (b = 16, P = 0) over a list of float32 row-major CUDA matrices with
    per-matrix tolerances; returns a list of (Q_t, B_t, QBInfo).  Matrix t uses seed + t."""
    torch = _torch()
    lib = _lib.load()
    count = len(As)
    descs = (_lib.qb_dense * count)()
    for t, A in enumerate(As):
        _check_dev(A)
        assert A.dtype == torch.float32 and A.stride(1) == 1
        descs[t] = _dense_desc(A)
    tol_arr = (C.c_double * count)(*[float(x) for x in tols])
    o = _opts(0.0, 16, 0, seed, relative, rank_cap, None, row_by_row, "mixed")
    if outs is None:
        outs = []
        for A in As:
            m, n = A.shape
            cap = min(m, n) if not rank_cap else min(m, n, int(rank_cap))
            outs.append((torch.empty(cap, m, dtype=torch.float32, device=A.device),
                         torch.empty(cap, n, dtype=torch.float32, device=A.device)))
    qp = (C.c_void_p * count)(*[q.data_ptr() for q, _ in outs])
    bp = (C.c_void_p * count)(*[b.data_ptr() for _, b in outs])
    ldq = (C.c_int64 * count)(*[q.stride(0) for q, _ in outs])
    ldb = (C.c_int64 * count)(*[b.stride(0) for _, b in outs])
    wsb = lib.qb_ei_batched_workspace(count, descs, C.byref(o))
    if wsb == 0:
        raise QBError(_lib.QB_ERR_INVALID_ARG, "qb_ei_batched_workspace")
    ws = workspace if workspace is not None and workspace.numel() >= wsb else \
        torch.empty(wsb, dtype=torch.uint8, device=As[0].device)
    infos = (_lib.qb_info * count)()
    with torch.cuda.device(As[0].device):
        rc = lib.qb_ei_batched(count, descs, tol_arr, C.byref(o), qp, ldq, bp, ldb,
                               C.c_void_p(ws.data_ptr()), ws.numel(), infos, _stream_ptr(stream))
    if rc < 0:
        raise QBError(rc, "qb_ei_batched")
    res = []
    for t in range(count):
        inf = infos[t]
        st = _lib.QB_OK
        if inf.status_bits & _lib.QB_BIT_NOT_CONVERGED:
            st = _lib.QB_NOT_CONVERGED
        elif inf.status_bits & _lib.QB_BIT_TOL_FLOOR:
            st = _lib.QB_WARN_TOL_FLOOR
        info = _info(st, inf)
        k = info.rank
        q, b = outs[t]
        res.append((q[:k].T, b[:k], info))
    return res


def qb_svd_from_qb(Q, B, want_u=True, want_v=True, stream=None):
    """SVD from a QB factorisation: (U, S, V, sweeps) with A ~ Q B = U diag(S) V^T, U = Q U~
    (m x k), V (n x k), S descending (float64).  Q, B as returned by the qb_* calls (float64 or
    float32, Q an m x k view of column-major storage, B k x n row-major)."""
    torch = _torch()
    lib = _lib.load()
    _check_dev(Q, B)
    m, k = Q.shape
    k2, n = B.shape
    assert k == k2 and Q.dtype == B.dtype
    f64 = Q.dtype == torch.float64
    prec = _lib.QB_PREC_FP64 if f64 else _lib.QB_PREC_MIXED
    Qc = Q if (Q.stride(0) == 1 and Q.stride(1) >= m) else Q.T.contiguous().T   # column-major
    Bc = B if B.stride(1) == 1 else B.contiguous()
    S = torch.empty(k, dtype=torch.float64, device=Q.device)
    Ut = torch.empty(k, m, dtype=Q.dtype, device=Q.device) if want_u else None
    Vt = torch.empty(k, n, dtype=Q.dtype, device=Q.device) if want_v else None
    wsb = lib.qb_svd_workspace(m, n, k, prec)
    if wsb == 0:
        raise QBError(_lib.QB_ERR_INVALID_ARG, "qb_svd_workspace")
    ws = torch.empty(wsb, dtype=torch.uint8, device=Q.device)
    sweeps = C.c_int32(0)
    with torch.cuda.device(Q.device):
        rc = lib.qb_svd_from_qb(m, n, k, prec, C.c_void_p(Qc.data_ptr()), Qc.stride(1),
                                C.c_void_p(Bc.data_ptr()), Bc.stride(0), C.c_void_p(S.data_ptr()),
                                C.c_void_p(Ut.data_ptr()) if want_u else None, m,
                                C.c_void_p(Vt.data_ptr()) if want_v else None, n,
                                C.c_void_p(ws.data_ptr()), wsb, C.byref(sweeps),
                                _stream_ptr(stream))
    if rc < 0:
        raise QBError(rc, "qb_svd_from_qb")
    return (Ut.T if want_u else None), S, (Vt.T if want_v else None), int(sweeps.value)


def batched_set_plan(cfg=None):
    """Pin the batched call's launch plan: cfg = (rows per thread 1|2, columns per thread 1|2,
    sketch CTAs per SM, B-pass CTAs per SM); None returns to the autotuner."""
    lib = _lib.load()
    if cfg is None:
        rc = lib.qb_batched_set_plan(None)
    else:
        arr = (C.c_int32 * 4)(*[int(x) for x in cfg])
        rc = lib.qb_batched_set_plan(arr)
    if rc < 0:
        raise QBError(rc, "qb_batched_set_plan")


def batched_last_plan() -> dict:
    """The last batched call's plan: tile shape, grids, whether it tuned and reused a graph."""
    out = (C.c_int32 * 8)()
    _lib.load().qb_batched_last_plan(out, 8)
    keys = ("rows_per_thread", "cols_per_thread", "sketch_grid", "bpass_grid", "tuned",
            "graph_reused", "tuner_entries")
    return dict(zip(keys, (int(x) for x in out[:7])))


def _autograd_function():
    torch = _torch()

    class QBFixedRank(torch.autograd.Function):
        """(Q, B) = QBFixedRank.apply(A, k, seed): the fixed-rank QB map with Omega fixed by the
        seed; backward runs the library's adjoint (Omega regenerated, Y not stored).  The gradient
        is returned in A's dtype."""

        @staticmethod
        def forward(ctx, A, k, seed):
            Q, B, R = qb_fixed_rank_fwd(A, k, seed)
            ctx.save_for_backward(A, Q, R)
            ctx.k, ctx.seed = k, seed
            return Q, B

        @staticmethod
        def backward(ctx, gQ, gB):
            A, Q, R = ctx.saved_tensors
            if gQ is None:
                gQ = torch.zeros_like(Q)
            if gB is None:
                gB = torch.zeros(ctx.k, A.shape[1], dtype=Q.dtype, device=A.device)
            GA = qb_fixed_rank_bwd(A, ctx.k, ctx.seed, Q, R, gQ, gB)
            return GA.to(A.dtype), None, None

    return QBFixedRank


def __getattr__(name):
    if name == "QBFixedRank":
        f = _autograd_function()
        globals()["QBFixedRank"] = f
        return f
    raise AttributeError(name)
