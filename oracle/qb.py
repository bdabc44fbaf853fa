"""Plain float64 CPU oracle for randQB_EI / randQB_FP (Yu, Gu, Li, arXiv:1606.09402).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package; only the test
suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs of
``bench.py`` use it.  It shares no code with the CUDA library.

Every routine takes the steps of the paper in its order and notation; numpy's matmul, LAPACK
Householder QR (``numpy.linalg.qr``) and scipy.sparse products serve as single steps.  ``A`` may
be a dense row-major float64 array or a scipy.sparse matrix (the same code serves both).

Readings of points the paper leaves open (each one is tested in ``tests/test_oracle_*.py``):
  * orth(X) is the Householder QR with R's diagonal made non-negative (columns of Q flipped);
    QB products do not depend on this sign choice.
  * Stopping rule: strict E < eps^2 (Alg. 1, Alg. 2; Alg. 4 writes sqrt(E) < eps, the same test).
    ``relative=True`` means eps = tol * ||A||_F (the criterion of the experiments, Sect. 5.4).
  * Row-by-row truncation (Sect. 3.1): rows of B_i are subtracted in order and the row whose
    subtraction makes E < eps^2 is kept; rank = (i-1) b + j.
  * A matrix with ||A||_F = 0 returns rank 0 (the loop would otherwise never meet E < 0).
  * Power scheme for randQB_EI (the paper only points at Martinsson-Voronin): per block, on the
    implicit residual A - QB:  Y = A Om_i - Q (B Om_i);  P times { Y = orth(Y);
    Z = orth(A^T Y - B^T (Q^T Y));  Y = A Z - Q (B Z) }; then Algorithm 2 continues with
    Q_i = orth(Y), the re-orthogonalisation and B_i = Q_i^T A.
  * randQB_FP when l~ columns do not reach the tolerance (Sect. 4.3 "re-generate Omega and
    rerun"): batch q draws global Omega columns [q l~, (q+1) l~); its P power iterations act on
    the implicit residual (for q = 0 this is exactly the power loop of Algorithm 4), then G = A Omega,
    H = A^T G and the blocked loop continues with the existing Q, B.
  * Theorem 3 floor: eps <= sqrt(4 u / delta) ||A||_F with u = 2^-53, delta = 0.01 raises the
    warning status QB_WARN_TOL_FLOOR (=2) on an otherwise converged result.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .philox import omega as _omega

QB_OK = 0
QB_NOT_CONVERGED = 1
QB_WARN_TOL_FLOOR = 2

U_FP64 = 2.0 ** -53
THM3_DELTA = 0.01


def _dense(x):
    return x.toarray() if hasattr(x, "toarray") else np.asarray(x)


def frob2(A) -> float:
    """||A||_F^2 as the sum of squares of the entries (Sect. 2; Theorem 3 discussion)."""
    if hasattr(A, "data") and hasattr(A, "tocsr"):
        d = np.asarray(A.data, dtype=np.float64)
        return float(np.dot(d, d))
    a = np.asarray(A, dtype=np.float64).ravel()
    return float(np.dot(a, a))


def qr_pos(X: np.ndarray):
    """Economic Householder QR with diag(R) >= 0."""
    Q, R = np.linalg.qr(X, mode="reduced")
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s[None, :], R * s[:, None]


def orth(X: np.ndarray) -> np.ndarray:
    """Orthonormal basis of range(X) (Fig. 1 "orth")."""
    return qr_pos(X)[0]


def thm3_floor(normA2: float, u: float = U_FP64, delta: float = THM3_DELTA) -> float:
    """Theorem 3: eps must exceed sqrt(4 u / delta) ||A||_F for E to have relative error <= delta."""
    return np.sqrt(4.0 * u / delta) * np.sqrt(normA2)


@dataclass
class QBResult:
    Q: np.ndarray
    B: np.ndarray
    rank: int
    E: float                  # the indicator ||A||^2 - sum ||B_i||^2 at exit
    normA2: float
    status: int
    passes: int               # passes over A (Table 1 accounting)
    omega_cols: int           # global Omega columns drawn
    E_hist: list = field(default_factory=list)  # E after each accepted row
    omega_used: np.ndarray | None = None        # FP: the (power-processed) Omega of batch 0

    @property
    def err_est(self) -> float:
        return float(np.sqrt(max(self.E, 0.0)))


def _eps_abs(tol: float, relative: bool, normA2: float) -> float:
    return tol * np.sqrt(normA2) if relative else tol


def _row_by_row(E: float, Bi: np.ndarray, eps2: float, hist: list, row_by_row: bool):
    """Row-by-row scheme of Sect. 3.1: subtract ||B_i(j,:)||^2 row by row; return
    (E, rows kept, stopped)."""
    rows = Bi.shape[0]
    if not row_by_row:
        E = E - float(np.sum(Bi * Bi))
        hist.append(E)
        return E, rows, E < eps2
    for j in range(rows):
        E = E - float(np.dot(Bi[j], Bi[j]))
        hist.append(E)
        if E < eps2:
            return E, j + 1, True
    return E, rows, False


def _cap(rank_cap, m, n):
    c = min(m, n)
    return c if rank_cap is None else min(int(rank_cap), c)


# ----------------------------------------------------------------------------- randQB (Fig. 1a)
def randqb(A, l: int, seed: int, P: int = 0, Omega=None):
    """Basic randQB: Q = orth(A Omega), optional power scheme, B = Q^T A."""
    m, n = A.shape
    Om = _omega(n, 0, l, seed) if Omega is None else Omega
    Q = orth(A @ Om)
    for _ in range(P):
        Qt = orth(A.T @ Q)
        Q = orth(A @ Qt)
    B = np.asarray((A.T @ Q).T)
    return Q, B


# ----------------------------------------------------------------------------- randQB_b (Fig. 1b)
def randqb_b(A, tol: float, b: int, seed: int, P: int = 0, relative: bool = True,
             rank_cap=None, fixed_rank=None) -> QBResult:
    """Blocked randQB of Martinsson-Voronin with an explicit residual, as Sect. 2 and 3.2
    describe it (Fig. 1b itself is not available): Q_i = orth(A Om_i) on the residual A, power
    steps on the residual, re-orthogonalise against Q, B_i = Q_i^T A, A <- A - Q_i B_i; stop once
    ||A||_F < eps."""
    R = _dense(A).astype(np.float64, copy=True)
    m, n = R.shape
    normA2 = frob2(R)
    eps = _eps_abs(tol, relative, normA2)
    cap = _cap(fixed_rank if fixed_rank is not None else rank_cap, m, n)
    Q = np.zeros((m, 0))
    B = np.zeros((0, n))
    k = 0
    status = QB_NOT_CONVERGED
    while k < cap:
        bi = min(b, cap - k)
        Om = _omega(n, k, bi, seed)
        Qi = orth(R @ Om)
        for _ in range(P):
            Qi = orth(R @ orth(R.T @ Qi))
        Qi = orth(Qi - Q @ (Q.T @ Qi))
        Bi = Qi.T @ R
        Q = np.hstack([Q, Qi])
        B = np.vstack([B, Bi])
        R = R - Qi @ Bi
        k += bi
        if fixed_rank is None and frob2(R) < eps * eps:
            status = QB_OK
            break
    return QBResult(Q, B, k, frob2(R), normA2, status, 0, k)


# ----------------------------------------------------------------------------- randQB_EI (Alg. 2)
def randqb_ei(A, tol: float, b: int, seed: int, P: int = 0, relative: bool = True,
              rank_cap=None, row_by_row: bool = True, reorth: bool = True,
              fixed_rank=None, omega_fn=None, A_sketch=None) -> QBResult:
    """Algorithm 2 with the row-by-row stop and the power-scheme reading in the module header.

    ``fixed_rank=k`` runs exactly k columns with no tolerance test (the fixed-rank version used by
    Proposition 2).  ``omega_fn(col0, w)`` replaces the Philox Omega (equivalence tests only).
    ``A_sketch`` (default A) is the matrix the sketch and power steps multiply by; B_i = Q_i^T A
    and the indicator always use A.  A sketch only has to capture a span, so a perturbed copy
    (A rounded to bf16) still gives a valid QB of A; this models a representation that streams a
    reduced copy of A for the sketches.
    """
    m, n = A.shape
    As = A if A_sketch is None else A_sketch
    normA2 = frob2(A)
    eps = _eps_abs(tol, relative, normA2)
    eps2 = eps * eps
    cap = _cap(fixed_rank if fixed_rank is not None else rank_cap, m, n)
    Q = np.zeros((m, 0))
    B = np.zeros((0, n))
    E = normA2
    hist: list = []
    k = 0
    passes = 0
    drawn = 0
    status = QB_NOT_CONVERGED
    if normA2 == 0.0 and fixed_rank is None:
        return QBResult(Q, B, 0, 0.0, 0.0, QB_OK, 0, 0, hist)
    while k < cap:
        bi = min(b, cap - k)
        drawn = k + bi
        Om = _omega(n, k, bi, seed) if omega_fn is None else omega_fn(k, bi)
        Y = As @ Om - Q @ (B @ Om)
        passes += 1
        for _ in range(P):
            Y = orth(Y)
            Z = orth(np.asarray(As.T @ Y) - B.T @ (Q.T @ Y))
            Y = As @ Z - Q @ (B @ Z)
            passes += 2
        Qi = orth(Y)
        if reorth:
            Qi = orth(Qi - Q @ (Q.T @ Qi))
        Bi = np.asarray((A.T @ Qi).T)             # B_i = Q_i^T A, no residual needed
        passes += 1
        if fixed_rank is None:
            E, keep, stop = _row_by_row(E, Bi, eps2, hist, row_by_row)
        else:
            E, keep, stop = _row_by_row(E, Bi, -np.inf, hist, True)   # record, never stop
        Q = np.hstack([Q, Qi[:, :keep]])
        B = np.vstack([B, Bi[:keep]])
        k += keep
        if stop:
            status = QB_OK
            break
    if status == QB_OK and eps <= thm3_floor(normA2):
        status = QB_WARN_TOL_FLOOR
    return QBResult(Q, B, k, E, normA2, status, passes, drawn, hist)


# ----------------------------------------------------------------------------- randQB_FP (Alg. 3/4)
def randqb_fp(A, tol: float, b: int, seed: int, P: int = 0, l_tilde=None,
              relative: bool = True, rank_cap=None, row_by_row: bool = True,
              reorth: bool = True, fixed_rank=None, omega_fn=None, A_sketch=None) -> QBResult:
    """Algorithm 4 (Algorithm 3 when ``reorth=False``) with the row-by-row stop.

    ``l_tilde`` defaults to 50 b (Sect. 5.4), clamped to the rank cap.  ``A_sketch`` (default A)
    is the matrix the power steps and G = A_sketch Omega multiply by; H = A^T G uses A.  The B_i
    formula of Sect. 4.2 needs only H = A^T G for the G it is given and B = Q^T A, so B_i is still
    Q_i^T A with Q_i = orth(G_i - Q B Omega_i).
    """
    m, n = A.shape
    As = A if A_sketch is None else A_sketch
    normA2 = frob2(A)
    eps = _eps_abs(tol, relative, normA2)
    eps2 = eps * eps
    cap = _cap(fixed_rank if fixed_rank is not None else rank_cap, m, n)
    lt = 50 * b if l_tilde is None else int(l_tilde)
    lt = max(1, min(lt, cap))
    Q = np.zeros((m, 0))
    B = np.zeros((0, n))
    E = normA2
    hist: list = []
    k = 0
    passes = 0
    status = QB_NOT_CONVERGED
    omega_used = None
    if normA2 == 0.0 and fixed_rank is None:
        return QBResult(Q, B, 0, 0.0, 0.0, QB_OK, 0, 0, hist)
    q = 0
    drawn = 0
    stop = False
    while k < cap and not stop:
        w = min(lt, cap - k)
        col0 = q * lt
        Om = _omega(n, col0, w, seed) if omega_fn is None else omega_fn(col0, w)
        drawn = col0 + w
        for _ in range(P):
            G = orth(As @ Om - Q @ (B @ Om))
            Om = orth(np.asarray(As.T @ G) - B.T @ (Q.T @ G))
            passes += 2
        if q == 0:
            omega_used = Om.copy()
        G = As @ Om
        H = np.asarray(A.T @ G)
        passes += 1
        for c0 in range(0, w, b):
            bi = min(b, w - c0)
            Om_i = Om[:, c0:c0 + bi]
            Y = G[:, c0:c0 + bi] - Q @ (B @ Om_i)
            Qi, Ri = qr_pos(Y)
            if reorth:
                # re-orthogonalisation of Sect. 4.2: [Q_i, R~_i] = qr(Q_i - Q Q^T Q_i),
                # R_i = R~_i R_i, B_i = R_i^-T (H_i^T - Y_i^T Q B - Om_i^T B^T B)
                Qi, Rt = qr_pos(Qi - Q @ (Q.T @ Qi))
                Ri = Rt @ Ri
                S = H[:, c0:c0 + bi].T - (Y.T @ Q) @ B - Om_i.T @ (B.T @ B)
            else:
                # Algorithm 3: B_i = R_i^-T (H_i^T - Om_i^T B^T B)
                S = H[:, c0:c0 + bi].T - Om_i.T @ (B.T @ B)
            Bi = np.linalg.solve(Ri.T, S)                         # R_i^{-T} (...)
            if fixed_rank is None:
                E, keep, stop = _row_by_row(E, Bi, eps2, hist, row_by_row)
            else:
                E, keep, stop = _row_by_row(E, Bi, -np.inf, hist, True)   # record, never stop
            Q = np.hstack([Q, Qi[:, :keep]])
            B = np.vstack([B, Bi[:keep]])
            k += keep
            if stop:
                status = QB_OK
                break
        q += 1
    if status == QB_OK and eps <= thm3_floor(normA2):
        status = QB_WARN_TOL_FLOOR
    return QBResult(Q, B, k, E, normA2, status, passes, drawn, hist, omega_used)


# ----------------------------------------------------------------------------- fixed-rank map
def qb_fixed_rank(A, k: int, seed: int, Omega=None):
    """The fixed-rank QB map A -> (Q, B) with Omega fixed: Y = A Omega (n x k Philox columns
    0..k-1 unless ``Omega`` is given), Y = Q R with diag(R) > 0, B = Q^T A.  Equal in exact arithmetic to k columns of
    randQB / randQB_EI / randQB_FP at P = 0 (Proposition 2)."""
    m, n = A.shape
    Om = _omega(n, 0, k, seed) if Omega is None else Omega
    Y = A @ Om
    Q, R = qr_pos(Y)
    B = np.asarray((A.T @ Q).T)
    return Q, B, R


def qb_fixed_rank_adjoint(A, k: int, seed: int, GQ: np.ndarray, GB: np.ndarray, Omega=None):
    """Gradient of L = <G_Q, Q> + <G_B, B> for the fixed-rank QB map (Omega fixed).

    The paper has no adjoint; this is reverse-mode differentiation of the three steps above:
      B = Q^T A              ->  Qbar = G_Q + A G_B^T,      Abar += Q G_B
      Y = Q R (R unused)     ->  M = -Qbar^T Q,  Ybar = (Qbar + Q copyltu(M)) R^{-T},
                                 copyltu(M) = tril(M) + tril(M, -1)^T
      Y = A Omega            ->  Abar += Ybar Omega^T
    """
    m, n = A.shape
    Om = _omega(n, 0, k, seed) if Omega is None else Omega
    Y = A @ Om
    Q, R = qr_pos(Y)
    Qbar = GQ + A @ GB.T
    M = -(Qbar.T @ Q)
    C = np.tril(M) + np.tril(M, -1).T
    Ybar = np.linalg.solve(R, (Qbar + Q @ C).T).T       # (.) R^{-T}
    return Q @ GB + Ybar @ Om.T


def orth_loss(Q: np.ndarray) -> float:
    """||Q^T Q - I||_inf (footnote of Sect. 3.3)."""
    k = Q.shape[1]
    if k == 0:
        return 0.0
    D = Q.T @ Q - np.eye(k)
    return float(np.max(np.sum(np.abs(D), axis=1)))
