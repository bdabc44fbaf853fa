"""SVD from QB on the GPU (qb_svd_from_qb, Sect. 2) against the oracle's definition on the same
Q, B, through the C ABI; and the single-pass SVD of Sect. 5.3 (randQB_FP at P = 0, l = 60, top 50
singular values of Matrix 1 and Matrix 2) against the known spectrum and the oracle.

Bounds: the GPU forms W = B B^T and diagonalises it by Jacobi rotations in float64, so s_j carries
about u k s_1^2 / s_j of absolute error (the Gram squares the condition number; Jacobi's own error
is backward-stable in W); the test allows 10 times that plus 1e-14 s_1."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1606_09402_gb300 as qb  # noqa: E402

U64 = 2.0 ** -53


def _s_bound(s_ref, k):
    return 10 * U64 * k * s_ref[0] ** 2 / np.maximum(s_ref, 1e-300) + 1e-14 * s_ref[0]


def _check_svd(Q, B, U, S, V, tol_rec=1e-10):
    Qh, Bh = Q.double().cpu().numpy(), B.double().cpu().numpy()
    Ur, sr, Vr = oracle.svd_from_qb(Qh, Bh)
    s = S.cpu().numpy()
    k = len(sr)
    assert np.all(np.abs(s - sr) <= _s_bound(sr, k)), np.max(np.abs(s - sr) / _s_bound(sr, k))
    Uh, Vh = U.double().cpu().numpy(), V.double().cpu().numpy()
    QB = Qh @ Bh
    assert np.linalg.norm(Uh * s @ Vh.T - QB) <= tol_rec * np.linalg.norm(QB)
    # U = Q U~ is orthonormal; V~ = B^T U~ S^-1 for the well-separated leading triplets
    assert np.max(np.abs(Uh.T @ Uh - np.eye(k))) <= 1e-12
    lead = int(np.sum(s >= 1e-3 * s[0]))
    assert np.max(np.abs(Vh[:, :lead].T @ Vh[:, :lead] - np.eye(lead))) <= 1e-9
    # the leading singular vectors match the oracle's up to sign where the gaps are wide
    gap = np.append(np.abs(np.diff(sr[: lead + 1])) / sr[0], np.inf)   # gap below s_j
    for j in range(min(lead, 10)):
        if gap[j] > 1e-3 and (j == 0 or gap[j - 1] > 1e-3):
            c = abs(float(Uh[:, j] @ Ur[:, j]))
            assert abs(c - 1) <= 1e-9, (j, c)


@pytest.mark.parametrize("m,n,k", [(300, 200, 37), (1000, 3000, 128), (513, 257, 257)])
def test_svd_from_qb_fp64_matches_oracle(m, n, k):
    sigma = synth.sigma_exp(min(m, n), 20.0, 1e-8)
    A = synth.dense_from_spectrum(m, n, sigma, seed=m + n)
    Q, B, info = qb.qb_fp_dense(torch.tensor(A, device="cuda"), 0.0, 16, P=1, seed=4, rank_cap=k)
    assert info.rank == k
    U, S, V, sweeps = qb.qb_svd_from_qb(Q, B)
    assert 1 <= sweeps <= 40
    _check_svd(Q, B, U, S, V)


def test_svd_from_qb_odd_and_tiny_orders():
    """k = 1 (no rotation), k = 2 (one pair), k = 3 (odd: one index sits out each step)."""
    A = synth.dense_from_spectrum(80, 60, synth.sigma_exp(60, 5.0), seed=2)
    for k in (1, 2, 3):
        Q, B, info = qb.qb_ei_dense(torch.tensor(A, device="cuda"), 0.0, 4, seed=1, rank_cap=k)
        assert info.rank == k
        U, S, V, _ = qb.qb_svd_from_qb(Q, B)
        _check_svd(Q, B, U, S, V)


def test_svd_from_qb_mixed():
    """Float32 Q, B (the mixed path's outputs): W with exact products in float32-pair sums, the
    eigendecomposition in float64, U and V formed in float32."""
    A = synth.dense_from_spectrum(2000, 1500, synth.sigma_exp(1500, 40.0, 1e-6), seed=12)
    Ad = torch.tensor(A, device="cuda")
    hi, lo, norms = qb.quantize_bf16x2(Ad)
    Q, B, info = qb.qb_fp_dense(hi, 1e-3, 32, P=1, seed=3, a_lo=lo, src_norm2=norms[0],
                                prec="mixed")
    U, S, V, _ = qb.qb_svd_from_qb(Q, B)
    Qh, Bh = Q.double().cpu().numpy(), B.double().cpu().numpy()
    _, sr, _ = oracle.svd_from_qb(Qh, Bh)
    s = S.cpu().numpy()
    assert np.max(np.abs(s - sr)) <= 1e-6 * sr[0]
    QB = Qh @ Bh
    rec = U.double().cpu().numpy() * s @ V.double().cpu().numpy().T
    assert np.linalg.norm(rec - QB) <= 1e-5 * np.linalg.norm(QB)


@pytest.mark.parametrize("mat", ["M1", "M2"])
def test_single_pass_svd_top50(mat):
    """Sect. 5.3 / Figs. 9-10: randQB_FP at P = 0 (G and H from the same Omega, one sweep in the
    paper's row-major setting), l = 50 + 10 oversampling, top 50 singular values; GPU float64
    against the oracle on the same A (same Omega), and both against the known spectrum."""
    n = 2000
    sigma = synth.table4_matrix_spectra(n)[mat]
    A = synth.dense_from_spectrum(n, n, sigma, seed=5)
    Q, B, info = qb.qb_fp_dense(torch.tensor(A, device="cuda"), 0.0, 10, P=0, seed=3,
                                rank_cap=60, l_tilde=60)
    assert info.rank == 60
    _, S, _, _ = qb.qb_svd_from_qb(Q, B, want_u=False, want_v=False)
    s = S.cpu().numpy()
    r = oracle.randqb_fp(A, 0.0, 10, seed=3, P=0, fixed_rank=60, l_tilde=60)
    _, sr, _ = oracle.svd_from_qb(r.Q, r.B)
    assert np.max(np.abs(s[:50] - sr[:50]) / sigma[:50]) <= 1e-9
    assert np.all(s <= sigma[:60] * (1 + 1e-10))           # interlacing: B = Q^T A
    top10 = np.max(np.abs(s[:10] - sigma[:10]) / sigma[:10])
    assert top10 <= (5e-3 if mat == "M1" else 1e-5)
