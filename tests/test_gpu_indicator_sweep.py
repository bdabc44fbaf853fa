"""Fig. 2 / Theorem 3 on the GPU: the error indicator E = ||A||^2 - sum ||B_i||^2 against the true
error ||A - Q B||^2 and the loss of orthogonality ||Q^T Q - I||_inf as the rank l grows, for
randQB_EI (b = 10) on n x n matrices with sigma_j = exp(-j / tau), through the C ABI.

Theorem 3: the rounding of E is about 4 u ||A||^2, so E is within 1% of the true squared error
while that error exceeds 4 u ||A||^2 / 0.01, i.e. (2.1e-7)^2 ||A||^2 in float64 (u = 2^-53).  On
the mixed path Q and B are float32 (u = 2^-24): the same argument puts the 1% threshold at
(4.9e-3)^2 ||A||^2.  Below the threshold E only has to stay within a few u ||A||^2 of the error.

E_l for intermediate l is formed here from the rows of the returned B in float64 (the same
subtraction the library's indicator kernel makes block by block); the library's own E at exit is
checked against it."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1606_09402_gb300 as qb  # noqa: E402

U64 = 2.0 ** -53
U32 = 2.0 ** -24


def _sweep(A, Q, B, normA2, ls):
    rn = (B.double() ** 2).sum(dim=1).cpu().numpy()
    out = []
    for l in ls:
        E = normA2 - float(np.sum(rn[:l]))
        err2 = 0.0
        for r0 in range(0, A.shape[0], 2048):
            D = A[r0:r0 + 2048].double() - Q[r0:r0 + 2048, :l].double() @ B[:l].double()
            err2 += float((D * D).sum())
        Ql = Q[:, :l].double()
        orth = float((Ql.T @ Ql - torch.eye(l, dtype=torch.float64, device=A.device))
                     .abs().sum(dim=1).max())
        out.append((l, E / normA2, err2 / normA2, orth))
    return out


@pytest.mark.parametrize("n,tau,lmax", [(3000, 20.0, 600), (6000, 60.0, 1500)])
def test_fig2_fp64(n, tau, lmax):
    sigma = synth.sigma_exp(n, tau)
    A = synth.dense_from_spectrum_torch(n, n, sigma, n, "cuda", dtype=torch.float64,
                                        work_dtype=torch.float64)
    # tol 0: the loop runs until E drops below zero through rounding (the point where Fig. 2's
    # log plot loses the indicator) or the rank cap
    Q, B, info = qb.qb_ei_dense(A, 0.0, 10, P=0, seed=20, rank_cap=lmax)
    assert info.rank >= lmax // 2
    ls = list(range(10, info.rank + 1, max(10, info.rank // 20)))
    rows = _sweep(A, Q, B, info.normA2, ls + [info.rank])
    # the library's own E at exit is the float64 subtraction of all rows of B
    assert abs(rows[-1][1] * info.normA2 - info.err2_est) <= 1e-13 * info.normA2
    thr = 4 * U64 / 0.01
    seen_above = seen_below = False
    for l, e, err2, orth in rows:
        if err2 > thr:
            seen_above = True
            assert abs(e - err2) <= 0.01 * err2, (l, e, err2)
        else:
            seen_below = True
            assert abs(e - err2) <= 8 * U64 * (1 + l / 100), (l, e, err2)
        assert orth <= 1e-12, (l, orth)
    assert seen_above and seen_below


def test_fig2_mixed():
    n, tau, lmax = 3000, 20.0, 400
    sigma = synth.sigma_exp(n, tau)
    A = synth.dense_from_spectrum_torch(n, n, sigma, n, "cuda", dtype=torch.float64,
                                        work_dtype=torch.float64)
    hi, lo, norms = qb.quantize_bf16x2(A)
    Q, B, info = qb.qb_ei_dense(hi, 0.0, 10, P=0, seed=20, rank_cap=lmax, a_lo=lo,
                                src_norm2=norms[0], prec="mixed")
    assert info.rank >= 100
    rows = _sweep(A, Q, B, norms[0], list(range(10, info.rank + 1, 20)))
    thr = 4 * U32 / 0.01
    seen_above = False
    for l, e, err2, orth in rows:
        if err2 > thr:
            seen_above = True
            assert abs(e - err2) <= 0.01 * err2, (l, e, err2)
        else:
            assert abs(e - err2) <= 8 * U32, (l, e, err2)
        assert orth <= 1e-5, (l, orth)
    assert seen_above
