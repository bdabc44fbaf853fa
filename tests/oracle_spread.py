"""How far apart two faithful float64 evaluations of the same QB factorisation land.

Test infrastructure (uses the float64 oracle).  The oracle is run on A and on row-permuted copies
P A.  In exact arithmetic the results agree up to that permutation: G = (P A) Omega = P (A Omega),
the Householder QR of P G is P times the QR of G, and H = (P A)^T (P G) = A^T G.  In float64 every
inner product over the rows of A (the QR, H = A^T G, B_i = Q_i^T A, the projections) sums in a
different order, so the spread of the results measures the rounding error the algorithm itself
carries at this input.  For randQB_FP that error is amplified by about (sigma_1 / sigma_k)^2
through the B_i formula (Remark 4.1), so the spread can exceed 1e-10 relative, and no float64
implementation can then be held closer than that to the oracle.
"""
from __future__ import annotations

import numpy as np

import oracle

PARITY = 1e-10          # the float64 parity target: ||QB_gpu - QB_cpu||_F / ||A||_F
SPREAD_FACTOR = 10.0    # a bound above the target is at most this multiple of the measured spread


def common_qb(Q1, B1, Q2, B2):
    """QB of both results over their common leading rank (the rows of B that both kept)."""
    k = min(Q1.shape[1], Q2.shape[1])
    return Q1[:, :k] @ B1[:k], Q2[:, :k] @ B2[:k]


def spread(A, alg, tol, b, perms=4, seed_perm=1, **kw):
    """Largest ||QB(A) - P^T QB(P A)||_F / ||A||_F over `perms` random row permutations P, with
    the oracle's randQB_EI (alg "ei") or randQB_FP ("fp"); returns (spread, reference result)."""
    f = oracle.randqb_ei if alg == "ei" else oracle.randqb_fp
    ref = f(A, tol, b, **kw)
    nA = np.linalg.norm(A)
    rng = np.random.default_rng(seed_perm)
    worst = 0.0
    for _ in range(perms):
        p = rng.permutation(A.shape[0])
        r = f(A[p], tol, b, **kw)
        Qp = np.empty_like(r.Q)
        Qp[p] = r.Q                                  # undo the row permutation of Q
        X, Y = common_qb(ref.Q, ref.B, Qp, r.B)
        worst = max(worst, float(np.linalg.norm(X - Y) / nA))
    return worst, ref


def parity_bound(measured_spread):
    """The float64 parity bound for a case: 1e-10, or, where two float64 evaluations of the oracle
    itself already disagree by more than a tenth of that, SPREAD_FACTOR times their disagreement."""
    return max(PARITY, SPREAD_FACTOR * measured_spread)
