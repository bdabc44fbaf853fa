"""Seeded synthetic inputs shared by the CUDA-path tests, the benchmark and the oracle tests.

This module only draws test matrices, sparse patterns and cotangents from fixed seeds.  It holds
none of the QB method's arithmetic (no sketching, no orthonormalisation, no indicator): the
random test matrix Omega that the method itself draws is produced separately on each side from
the Philox4x32-10 definition.

Workload recipes (the paper's synthetic test matrices, Sect. 5.2 and Sect. 5.1):

* dense  A = U diag(sigma) V^T with U, V orthonormal columns from the QR of seeded N(0,1)
  matrices ("Haar-like"), spectra
    - ``sigma_pow(p)``   sigma_j = j^-p         (Matrix 1 uses p = 2; the 2000x2000 case p = 1.5)
    - ``sigma_exp(tau, floor)``  sigma_j = exp(-j/tau) + floor  (Matrix 2: tau = 7)
    - ``sigma_s()``      sigma_j = 1e-4 + 1/(1 + exp(j - 30))   (Matrix 3)
  j counts from 1.
* sparse CSR with Poisson row lengths, Zipf-distributed distinct column indices mapped through a
  seeded permutation, log-normal values.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

__all__ = [
    "sigma_pow", "sigma_exp", "sigma_s", "dense_from_spectrum", "dense_low_rank",
    "dense_from_spectrum_torch", "csr_zipf", "batched_specs", "cotangents", "svd_rank",
]


# ----------------------------------------------------------------------------- spectra
def sigma_pow(n: int, p: float, scale: float = 1.0) -> np.ndarray:
    j = np.arange(1, n + 1, dtype=np.float64)
    return scale * j ** (-p)


def sigma_exp(n: int, tau: float, floor: float = 0.0) -> np.ndarray:
    j = np.arange(1, n + 1, dtype=np.float64)
    return np.exp(-j / tau) + floor


def sigma_s(n: int, center: float = 30.0, floor: float = 1e-4) -> np.ndarray:
    j = np.arange(1, n + 1, dtype=np.float64)
    return floor + np.exp(-np.logaddexp(0.0, j - center))  # 1 / (1 + e^(j - center))


def svd_rank(sigma: np.ndarray, tol: float) -> int:
    """Smallest k with sqrt(sum_{j>k} sigma_j^2) < tol * ||sigma||_2 (strict, relative)."""
    s2 = np.asarray(sigma, dtype=np.float64) ** 2
    total = s2.sum()
    tail = np.concatenate([np.cumsum(s2[::-1])[::-1], [0.0]])  # tail[k] = sum_{j>k}
    ok = np.nonzero(tail < (tol * tol) * total)[0]
    return int(ok[0])


# ----------------------------------------------------------------------------- dense
def _orthonormal(rng: np.random.Generator, rows: int, cols: int) -> np.ndarray:
    g = rng.standard_normal((rows, cols))
    q, _ = np.linalg.qr(g)
    return q


def dense_from_spectrum(m: int, n: int, sigma: np.ndarray, seed: int, dtype=np.float64) -> np.ndarray:
    """A = U diag(sigma) V^T, U (m x r), V (n x r) orthonormal, r = len(sigma) <= min(m, n).

    Row-major (C-contiguous) float64 unless ``dtype`` says otherwise.
    """
    r = len(sigma)
    assert r <= min(m, n)
    rng = np.random.default_rng(seed)
    u = _orthonormal(rng, m, r)
    v = _orthonormal(rng, n, r)
    a = (u * np.asarray(sigma, dtype=np.float64)[None, :]) @ v.T
    return np.ascontiguousarray(a, dtype=dtype)


def dense_low_rank(m: int, n: int, r: int, seed: int) -> np.ndarray:
    """Exactly rank-r float64 matrix with singular values 1 .. 1/r (linear)."""
    sigma = np.linspace(1.0, 1.0 / r, r)
    return dense_from_spectrum(m, n, sigma, seed)


def dense_from_spectrum_torch(m: int, n: int, sigma, seed: int, device, dtype=None,
                              work_dtype=None):
    """Large-scale variant of ``dense_from_spectrum`` drawn on a torch device.

    U and V come from the QR of seeded N(0,1) matrices computed in ``work_dtype`` (default
    float32: orthonormality ~1e-6, which perturbs the singular values relatively by the same
    amount; float64 keeps them to ~1e-15) on ``device``; the product is formed in the same type
    and returned as ``dtype`` (default float64), row-major.
    """
    import torch

    dtype = dtype or torch.float64
    wd = work_dtype or torch.float32
    r = len(sigma)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        s = torch.as_tensor(np.asarray(sigma, dtype=np.float64), device=device).to(wd)
        gu = torch.randn(m, r, generator=gen, device=device, dtype=torch.float32).to(wd)
        u, _ = torch.linalg.qr(gu)
        del gu
        gv = torch.randn(n, r, generator=gen, device=device, dtype=torch.float32).to(wd)
        v, _ = torch.linalg.qr(gv)
        del gv
        a = torch.empty(m, n, device=device, dtype=dtype)
        # form A in row blocks to bound the float32 temporary
        step = max(1, min(m, (1 << 28) // max(n, 1)))
        us = u * s[None, :]
        for r0 in range(0, m, step):
            r1 = min(m, r0 + step)
            a[r0:r1].copy_(us[r0:r1] @ v.T)
        return a
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


# ----------------------------------------------------------------------------- sparse
@dataclass
class CSR:
    m: int
    n: int
    rowptr: np.ndarray  # int32 [m+1]
    colind: np.ndarray  # int32 [nnz]
    val: np.ndarray     # float32 or float64 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.colind, self.rowptr), shape=(self.m, self.n))


def csr_zipf(m: int, n: int, mean_len: float, zipf_s: float, seed: int,
             val_dtype=np.float32, merge_duplicates: bool = False) -> CSR:
    """Row lengths ~ Poisson(mean_len) (capped at n); columns Zipf(zipf_s) over ranks 1..n drawn
    without repetition inside a row (duplicates are redrawn), rank -> column id through a seeded
    permutation; values log-normal(0, 1).  Column indices are sorted inside each row.

    ``merge_duplicates=True`` is the other reading of the recipe: the Poisson(mean_len) draws of a
    row keep their repeats and repeated columns are merged by summing their log-normal values
    (about 31% of the draws collide at Zipf(1.1), so the matrix has fewer nonzeros and more weight
    in the hot columns)."""
    if merge_duplicates:
        return _csr_zipf_merged(m, n, mean_len, zipf_s, seed, val_dtype)
    rng = np.random.default_rng(seed)
    lens = np.minimum(rng.poisson(mean_len, size=m), n).astype(np.int64)
    ranks = np.arange(1, n + 1, dtype=np.float64)
    cdf = np.cumsum(ranks ** (-zipf_s))
    cdf /= cdf[-1]
    perm = rng.permutation(n).astype(np.int64)
    keys = np.empty(0, dtype=np.int64)        # sorted, unique keys row * n + rank
    have = np.zeros(m, dtype=np.int64)
    # draw, dedupe per row, redraw what is missing; only the new draws are sorted and merged into
    # the kept keys, which gives the same key set as re-sorting everything each round
    pending_rows = np.repeat(np.arange(m, dtype=np.int64), lens)
    for _ in range(64):
        if pending_rows.size == 0:
            break
        u = rng.random(pending_rows.size)
        c = np.minimum(np.searchsorted(cdf, u, side="right"), n - 1)
        new = np.sort(pending_rows * n + c)
        if new.size:
            new = new[np.concatenate(([True], new[1:] != new[:-1]))]
        pos = np.searchsorted(keys, new)
        if keys.size:
            present = keys[np.minimum(pos, keys.size - 1)] == new
            new = new[~present]
            pos = pos[~present]
        keys = np.insert(keys, pos, new)
        have += np.bincount(new // n, minlength=m)
        missing = lens - have
        pending_rows = np.repeat(np.arange(m, dtype=np.int64), np.maximum(missing, 0))
    # sort by (row, column id): the pairs are distinct, so one sort of row * n + column does it
    rc = np.sort((keys // n) * n + perm[keys % n])
    r_of = rc // n
    cols = rc % n
    counts = np.bincount(r_of, minlength=m)
    rowptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    vals = rng.lognormal(0.0, 1.0, size=cols.size).astype(val_dtype)
    return CSR(m, n, rowptr.astype(np.int32), cols.astype(np.int32), vals)


def _csr_zipf_merged(m, n, mean_len, zipf_s, seed, val_dtype):
    rng = np.random.default_rng(seed)
    lens = rng.poisson(mean_len, size=m).astype(np.int64)
    ranks = np.arange(1, n + 1, dtype=np.float64)
    cdf = np.cumsum(ranks ** (-zipf_s))
    cdf /= cdf[-1]
    perm = rng.permutation(n).astype(np.int64)
    rows = np.repeat(np.arange(m, dtype=np.int64), lens)
    c = np.minimum(np.searchsorted(cdf, rng.random(rows.size), side="right"), n - 1)
    vals = rng.lognormal(0.0, 1.0, size=rows.size)
    keys = rows * n + perm[c]
    order = np.argsort(keys, kind="stable")
    keys, vals = keys[order], vals[order]
    first = np.concatenate(([True], keys[1:] != keys[:-1])) if keys.size else np.zeros(0, bool)
    starts = np.nonzero(first)[0]
    uk = keys[starts]
    uv = np.add.reduceat(vals, starts) if keys.size else vals
    r_of = uk // n
    counts = np.bincount(r_of, minlength=m)
    rowptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return CSR(m, n, rowptr.astype(np.int32), (uk % n).astype(np.int32), uv.astype(val_dtype))


# ----------------------------------------------------------------------------- batched
@dataclass
class BatchSpec:
    m: int
    n: int
    scale: float
    tol: float
    seed: int


def batched_specs(count: int, seed: int, lo: int = 256, hi: int = 4096,
                  tols=(1e-2, 1e-3)) -> list[BatchSpec]:
    """Per-matrix shapes m, n ~ U[lo, hi], spectrum scale ~ U[1, 100], tolerance from ``tols``."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        m = int(rng.integers(lo, hi + 1))
        n = int(rng.integers(lo, hi + 1))
        scale = float(rng.uniform(1.0, 100.0))
        tol = float(tols[int(rng.integers(0, len(tols)))])
        out.append(BatchSpec(m, n, scale, tol, seed * 100003 + i))
    return out


# ----------------------------------------------------------------------------- cotangents
def cotangents(m: int, n: int, k: int, seed: int):
    """Seeded N(0,1) cotangents G_Q (m x k) and G_B (k x n), float64."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((m, k)), rng.standard_normal((k, n))


def table4_matrix_spectra(n: int):
    """The three spectra of Table 4 / Sect. 5.2 (Matrix 1, 2, 3) for an n x n matrix."""
    return {"M1": sigma_pow(n, 2.0), "M2": sigma_exp(n, 7.0), "M3": sigma_s(n)}
