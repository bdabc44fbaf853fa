"""SVD from a QB factorisation, the plain definition (Sect. 2, the approximate SVD).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  With B = U~ S V~^T (LAPACK SVD of the
small k x n B), A ~ Q B = (Q U~) S V~^T: the leading columns of Q U~ and V~ and the leading
entries of S approximate the singular triplets of A.  Followed by randQB_FP at P = 0 (Algorithm 3,
whose G and H the paper forms in one sweep over a row-major A) this is the single-pass SVD of
Sect. 5.3.
"""
from __future__ import annotations

import numpy as np


def svd_from_qb(Q: np.ndarray, B: np.ndarray):
    """Returns (U, s, V) with Q B = U diag(s) V^T, s descending, U = Q U~ (m x k), V (n x k)."""
    Ut, s, Vt = np.linalg.svd(np.asarray(B, dtype=np.float64), full_matrices=False)
    return np.asarray(Q, dtype=np.float64) @ Ut, s, Vt.T
