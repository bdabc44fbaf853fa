"""ctypes view of the C ABI in include/qb.h (structures, prototypes, library loading).

Loading fails loudly when libqb.so is missing: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libqb.so")

QB_OK = 0
QB_NOT_CONVERGED = 1
QB_WARN_TOL_FLOOR = 2
QB_ERR_INVALID_ARG = -1
QB_ERR_NONFINITE = -2
QB_ERR_CUDA = -3
QB_ERR_BREAKDOWN = -4
QB_ERR_WORKSPACE = -5
QB_ERR_TIMEOUT = -6
QB_ERR_UNSUPPORTED = -7

QB_BIT_BREAKDOWN = 1
QB_BIT_TOL_FLOOR = 2
QB_BIT_NOT_CONVERGED = 4

QB_F64, QB_F32, QB_BF16, QB_BF16X2 = 0, 1, 2, 3
QB_FLAG_SIMT_APASS, QB_FLAG_PROFILE, QB_FLAG_WHOLE_BATCH = 1, 2, 4
PHASES = ("omega", "sketch", "trans", "power_orth", "projections", "cholqr2", "fp_b_formula",
          "indicator")
QB_PREC_FP64, QB_PREC_MIXED = 0, 1


class qb_dense(C.Structure):
    _fields_ = [("m", C.c_int64), ("n", C.c_int64), ("ld", C.c_int64), ("dtype", C.c_int32),
                ("reserved", C.c_int32), ("a", C.c_void_p), ("a_lo", C.c_void_p),
                ("src_norm2", C.c_double), ("a_lo_ready", C.c_void_p)]


class qb_csr(C.Structure):
    _fields_ = [("m", C.c_int64), ("n", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.c_void_p),
                ("colind", C.c_void_p), ("dtype", C.c_int32), ("reserved", C.c_int32),
                ("val", C.c_void_p)]


class qb_coo(C.Structure):
    _fields_ = [("m", C.c_int64), ("n", C.c_int64), ("nnz", C.c_int64), ("row", C.c_void_p),
                ("col", C.c_void_p), ("dtype", C.c_int32), ("reserved", C.c_int32),
                ("val", C.c_void_p)]


class qb_opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("relative", C.c_int32), ("b", C.c_int32), ("P", C.c_int32),
                ("row_by_row", C.c_int32), ("seed", C.c_uint64), ("rank_cap", C.c_int64),
                ("l_tilde", C.c_int64), ("prec", C.c_int32), ("flags", C.c_int32)]


class qb_info(C.Structure):
    _fields_ = [("rank", C.c_int64), ("err2_est", C.c_double), ("err_est", C.c_double),
                ("normA2", C.c_double), ("passes", C.c_int64), ("omega_cols", C.c_int64),
                ("status_bits", C.c_int32), ("blocks", C.c_int32), ("launches", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# name -> (restype, argtypes)
_P = C.c_void_p
_I64 = C.c_int64
_SIG = {
    "qb_status_str": (C.c_char_p, [C.c_int32]),
    "qb_last_cuda_error": (C.c_char_p, []),
    "qb_launch_count": (C.c_int64, []),
    "qb_profile_last": (C.c_int32, [C.POINTER(C.c_double), C.c_int32]),
    "qb_dense_workspace": (C.c_size_t, [C.POINTER(qb_dense), C.POINTER(qb_opts), C.c_int32]),
    "qb_ei_dense": (C.c_int32, [C.POINTER(qb_dense), C.POINTER(qb_opts), _P, _I64, _P, _I64, _P,
                                C.c_size_t, C.POINTER(qb_info), _P]),
    "qb_fp_dense": (C.c_int32, [C.POINTER(qb_dense), C.POINTER(qb_opts), _P, _I64, _P, _I64, _P,
                                C.c_size_t, C.POINTER(qb_info), _P]),
    "qb_csr_workspace": (C.c_size_t, [C.POINTER(qb_csr), C.POINTER(qb_opts), C.c_int32]),
    "qb_ei_csr": (C.c_int32, [C.POINTER(qb_csr), C.POINTER(qb_opts), _P, _I64, _P, _I64, _P,
                              C.c_size_t, C.POINTER(qb_info), _P]),
    "qb_fp_csr": (C.c_int32, [C.POINTER(qb_csr), C.POINTER(qb_opts), _P, _I64, _P, _I64, _P,
                              C.c_size_t, C.POINTER(qb_info), _P]),
    "qb_coo_workspace": (C.c_size_t, [C.POINTER(qb_coo), C.POINTER(qb_opts), C.c_int32]),
    "qb_ei_coo": (C.c_int32, [C.POINTER(qb_coo), C.POINTER(qb_opts), _P, _I64, _P, _I64, _P,
                              C.c_size_t, C.POINTER(qb_info), _P]),
    "qb_fp_coo": (C.c_int32, [C.POINTER(qb_coo), C.POINTER(qb_opts), _P, _I64, _P, _I64, _P,
                              C.c_size_t, C.POINTER(qb_info), _P]),
    "qb_omega": (C.c_int32, [_I64, _I64, _I64, C.c_uint64, C.c_int32, _P, _I64, _P]),
    "qb_apass_workspace": (C.c_size_t, [C.POINTER(qb_dense), _I64]),
    "qb_apass_sketch": (C.c_int32, [C.POINTER(qb_dense), _P, _I64, _I64, _P, _I64, _P, C.c_size_t,
                                    _P]),
    "qb_apass_trans": (C.c_int32, [C.POINTER(qb_dense), _P, _I64, _I64, C.c_int32, _P, _I64, _P,
                                   C.c_size_t, _P]),
    "qb_apass_sketch_noalloc": (C.c_int32, [C.POINTER(qb_dense), _P, _I64, _I64, _P, _I64, _P]),
    "qb_fixed_rank_workspace": (C.c_size_t, [C.POINTER(qb_dense), _I64, C.c_int32]),
    "qb_fixed_rank_fwd": (C.c_int32, [C.POINTER(qb_dense), _I64, C.c_uint64, C.c_int32, _P, _I64,
                                      _P, _I64, _P, _I64, _P, C.c_size_t, _P]),
    "qb_fixed_rank_bwd": (C.c_int32, [C.POINTER(qb_dense), _I64, C.c_uint64, C.c_int32, _P, _I64,
                                      _P, _I64, _P, _I64, _P, _I64, _P, _I64, _P, C.c_size_t, _P]),
    "qb_ei_batched_workspace": (C.c_size_t, [C.c_int32, C.POINTER(qb_dense), C.POINTER(qb_opts)]),
    "qb_ei_batched": (C.c_int32, [C.c_int32, C.POINTER(qb_dense), C.POINTER(C.c_double),
                                  C.POINTER(qb_opts), C.POINTER(C.c_void_p), C.POINTER(C.c_int64),
                                  C.POINTER(C.c_void_p), C.POINTER(C.c_int64), _P, C.c_size_t,
                                  C.POINTER(qb_info), _P]),
    "qb_svd_workspace": (C.c_size_t, [_I64, _I64, _I64, C.c_int32]),
    "qb_svd_from_qb": (C.c_int32, [_I64, _I64, _I64, C.c_int32, _P, _I64, _P, _I64, _P, _P, _I64,
                                   _P, _I64, _P, C.c_size_t, C.POINTER(C.c_int32), _P]),
    "qb_batched_set_plan": (C.c_int32, [C.POINTER(C.c_int32)]),
    "qb_batched_last_plan": (C.c_int32, [C.POINTER(C.c_int32), C.c_int32]),
    "qb_quantize_workspace": (C.c_size_t, [_I64, _I64]),
    "qb_quantize_bf16x2": (C.c_int32, [_P, _I64, _I64, _I64, _P, _P, _I64,
                                       C.POINTER(C.c_double), _P, C.c_size_t, _P]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libqb.so and attach the prototypes above; raises if the library is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libqb.so not built ({path}); run __graft_entry__.build() or "
                           "python -m paper_1606_09402_gb300.build")
    lib = C.CDLL(path)
    for name, (res, args) in _SIG.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def declared_symbols(header: str) -> list[str]:
    """Function names declared in a C header of this project (used by the ABI tests)."""
    import re
    txt = open(header).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(qb_[a-z0-9_]+)\s*\(", txt)))
