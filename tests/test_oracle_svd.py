"""Pins of the oracle's SVD from QB (Sect. 2) and of the single-pass setting of Sect. 5.3, on the
CPU: the exact SVD of exactly low-rank inputs, singular-value interlacing for B = Q^T A, and the
accuracy pattern Figs. 9/10 report for the top singular values of Matrix 1 and Matrix 2."""
import numpy as np
import pytest

import oracle
import synth


def test_exact_low_rank_gives_the_exact_svd():
    """A of rank 12 with known singular values: a QB of rank 20 holds A exactly, so its SVD is A's
    (the singular values, and U S V^T = A)."""
    sigma = np.linspace(3.0, 0.25, 12)
    A = synth.dense_from_spectrum(150, 90, sigma, seed=17)
    r = oracle.randqb_ei(A, 0.0, 5, seed=2, fixed_rank=20)
    U, s, V = oracle.svd_from_qb(r.Q, r.B)
    assert np.allclose(s[:12], sigma, rtol=1e-12, atol=0)
    assert np.all(s[12:] <= 1e-13 * sigma[0])
    assert np.linalg.norm(U * s @ V.T - A) <= 1e-12 * np.linalg.norm(A)
    assert np.linalg.norm(U.T @ U - np.eye(20)) <= 1e-12
    assert np.linalg.norm(V[:, :12].T @ V[:, :12] - np.eye(12)) <= 1e-12


def test_interlacing_and_reconstruction():
    """B = Q^T A with orthonormal Q: sigma_j(B) <= sigma_j(A) for every j; U diag(s) V^T = Q B."""
    sigma = synth.sigma_pow(120, 1.0)
    A = synth.dense_from_spectrum(200, 120, sigma, seed=3)
    r = oracle.randqb_fp(A, 0.0, 8, seed=4, fixed_rank=40)
    U, s, V = oracle.svd_from_qb(r.Q, r.B)
    assert np.all(s <= sigma[:40] * (1 + 1e-12))
    assert np.linalg.norm(U * s @ V.T - r.Q @ r.B) <= 1e-12 * np.linalg.norm(A)
    assert np.all(np.diff(s) <= 0)


@pytest.mark.parametrize("mat,p0_top10,p1_gain", [("M1", 5e-3, 1e3), ("M2", 1e-5, 1e3)])
def test_single_pass_top_singular_values(mat, p0_top10, p1_gain):
    """Sect. 5.3: randQB_FP at P = 0 (single pass) with l = 50 + 10 oversampling; the top
    singular values are accurate on the fast-decaying Matrix 2 and moderately so on the slowly
    decaying Matrix 1, and one power iteration (P = 1) improves them by orders of magnitude."""
    n = 2000
    sigma = synth.table4_matrix_spectra(n)[mat]
    A = synth.dense_from_spectrum(n, n, sigma, seed=5)
    errs = []
    for P in (0, 1):
        r = oracle.randqb_fp(A, 0.0, 10, seed=3, P=P, fixed_rank=60, l_tilde=60)
        _, s, _ = oracle.svd_from_qb(r.Q, r.B)
        assert np.all(s <= sigma[:60] * (1 + 1e-12))
        errs.append(np.max(np.abs(s[:10] - sigma[:10]) / sigma[:10]))
    assert errs[0] <= p0_top10
    assert errs[1] * p1_gain <= errs[0]


def test_planted_mistake_in_svd_from_qb_is_seen():
    """Returning Q V~ instead of Q U~ breaks the reconstruction pin."""
    A = synth.dense_from_spectrum(60, 60, synth.sigma_exp(60, 6.0), seed=9)
    r = oracle.randqb_ei(A, 0.0, 5, seed=2, fixed_rank=15)
    Ut, s, Vt = np.linalg.svd(r.B, full_matrices=False)
    bad_U = r.Q @ Vt[:, :15].T[:15] if Vt.shape[1] >= 15 else None
    U, s2, V = oracle.svd_from_qb(r.Q, r.B)
    assert np.linalg.norm(U * s2 @ V.T - r.Q @ r.B) <= 1e-12 * np.linalg.norm(A)
    assert np.linalg.norm(bad_U * s @ Vt - r.Q @ r.B) > 1e-3 * np.linalg.norm(A)
