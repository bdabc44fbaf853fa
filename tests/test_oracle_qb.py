"""Pins for the float64 oracle of randQB_EI / randQB_FP against what the paper and the
mathematics fix: Theorem 1/2, Propositions 1 and 2, Table 4's SVD ranks, the Eckart-Young floor,
exact low rank, orthogonality, Theorem 3, and the fixed-rank adjoint (finite differences and
torch autograd)."""
import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def qb_diff(r1, r2, A):
    return np.linalg.norm(r1.Q @ r1.B - r2.Q @ r2.B) / np.linalg.norm(A)


@pytest.fixture(scope="module")
def A_exp():
    return synth.dense_from_spectrum(90, 70, synth.sigma_exp(70, 8.0), seed=11)


# ----------------------------------------------------------------------------- Theorem 1 / 2
@pytest.mark.parametrize("alg", ["ei", "fp"])
@pytest.mark.parametrize("P", [0, 1])
def test_indicator_equals_direct_residual(alg, P):
    A = synth.dense_from_spectrum(64, 48, synth.sigma_exp(48, 6.0), seed=2)
    f = oracle.randqb_ei if alg == "ei" else oracle.randqb_fp
    r = f(A, 1e-5, 5, seed=7, P=P)
    normA2 = oracle.frob2(A)
    assert len(r.E_hist) == r.rank
    for k in range(1, r.rank + 1):
        direct = np.linalg.norm(A - r.Q[:, :k] @ r.B[:k]) ** 2
        assert abs(r.E_hist[k - 1] - direct) <= 1e-12 * normA2


def test_frob2_is_sum_of_squares():
    A = np.arange(12.0).reshape(3, 4) - 5.0
    assert oracle.frob2(A) == float(sum(x * x for x in A.ravel()))
    S = sp.random(30, 20, density=0.2, random_state=1, format="csr")
    assert abs(oracle.frob2(S) - np.sum(S.toarray() ** 2)) < 1e-13


# ----------------------------------------------------------------------------- Proposition 1
@pytest.mark.parametrize("P", [0, 1])
def test_ei_equals_blocked_randqb(A_exp, P):
    k = 23  # not a multiple of b
    r_ei = oracle.randqb_ei(A_exp, 0.0, 5, seed=3, P=P, fixed_rank=k)
    r_b = oracle.randqb_b(A_exp, 0.0, 5, seed=3, P=P, fixed_rank=k)
    assert r_ei.rank == r_b.rank == k
    assert qb_diff(r_ei, r_b, A_exp) <= 1e-12


def test_ei_tolerance_rank_matches_blocked_randqb(A_exp):
    r_ei = oracle.randqb_ei(A_exp, 1e-3, 4, seed=3, row_by_row=False)
    r_b = oracle.randqb_b(A_exp, 1e-3, 4, seed=3)
    assert r_ei.rank == r_b.rank
    assert qb_diff(r_ei, r_b, A_exp) <= 1e-12


# ----------------------------------------------------------------------------- Proposition 2
def test_fp_without_reorth_equals_ei_without_reorth(A_exp):
    r_fp = oracle.randqb_fp(A_exp, 0.0, 5, seed=4, reorth=False, fixed_rank=20)
    r_ei = oracle.randqb_ei(A_exp, 0.0, 5, seed=4, reorth=False, fixed_rank=20)
    assert qb_diff(r_fp, r_ei, A_exp) <= 1e-10


def test_fp_equals_ei_and_randqb(A_exp):
    r_fp = oracle.randqb_fp(A_exp, 0.0, 5, seed=4, fixed_rank=20)
    r_ei = oracle.randqb_ei(A_exp, 0.0, 5, seed=4, fixed_rank=20)
    Q, B = oracle.randqb(A_exp, 20, seed=4)
    assert qb_diff(r_fp, r_ei, A_exp) <= 1e-10
    assert np.linalg.norm(r_fp.Q @ r_fp.B - Q @ B) / np.linalg.norm(A_exp) <= 1e-10


def test_fp_tolerance_path_equals_ei(A_exp):
    r_fp = oracle.randqb_fp(A_exp, 1e-4, 6, seed=8)
    r_ei = oracle.randqb_ei(A_exp, 1e-4, 6, seed=8)
    assert r_fp.rank == r_ei.rank
    assert qb_diff(r_fp, r_ei, A_exp) <= 1e-10


def test_fp_power_equals_ei_on_processed_omega(A_exp):
    r_fp = oracle.randqb_fp(A_exp, 0.0, 5, seed=9, P=1, l_tilde=25, fixed_rank=25)
    Om1 = r_fp.omega_used
    r_ei = oracle.randqb_ei(A_exp, 0.0, 5, seed=0, P=0, fixed_rank=25,
                            omega_fn=lambda c0, w: Om1[:, c0:c0 + w])
    assert qb_diff(r_fp, r_ei, A_exp) <= 1e-10


def test_fp_multiple_batches_reach_tolerance():
    A = synth.dense_from_spectrum(120, 100, synth.sigma_exp(100, 15.0), seed=5)
    for P in (0, 1):
        r = oracle.randqb_fp(A, 1e-3, 4, seed=1, P=P, l_tilde=12)
        assert r.status == oracle.QB_OK
        assert r.omega_cols > 12
        assert np.linalg.norm(A - r.Q @ r.B) < 1e-3 * np.linalg.norm(A)
        assert abs(r.E - np.linalg.norm(A - r.Q @ r.B) ** 2) <= 1e-12 * r.normA2


# ----------------------------------------------------------------------------- Table 4
def _table4():
    rows = []
    with open(os.path.join(GOLDEN, "table4_svd_ranks.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            m, n, eps, r_svd, r_ei, r_fp = line.split()
            rows.append((m, int(n), float(eps), int(r_svd), int(r_ei), int(r_fp)))
    return rows


def test_table4_svd_ranks_closed_form():
    rows = _table4()
    assert len(rows) == 6
    for mat, n, eps, r_svd, r_ei, r_fp in rows:
        sigma = synth.table4_matrix_spectra(n)[mat]
        assert synth.svd_rank(sigma, eps) == r_svd, (mat, eps)
        # the randomized ranks the paper prints never beat the SVD (Eckart-Young)
        assert r_ei >= r_svd and r_fp >= r_svd


@pytest.mark.parametrize("mat,eps", [("M1", 1e-2), ("M2", 1e-4), ("M2", 1e-5), ("M3", 1e-2)])
@pytest.mark.parametrize("alg", ["ei", "fp"])
def test_fixed_precision_on_table4_spectra(mat, eps, alg):
    n = 400
    sigma = synth.table4_matrix_spectra(n)[mat]
    A = 37.5 * synth.dense_from_spectrum(n, n, sigma, seed=42)   # scale must not matter
    f = oracle.randqb_ei if alg == "ei" else oracle.randqb_fp
    r = f(A, eps, 10, seed=1, P=1)
    r_svd = synth.svd_rank(sigma, eps)
    err = np.linalg.norm(A - r.Q @ r.B) / np.linalg.norm(A)
    assert r.status == oracle.QB_OK
    assert err < eps                       # the fixed-precision guarantee
    assert r_svd <= r.rank <= r_svd + 3    # close to optimal with P = 1 (Table 4: +0..+15)


# ----------------------------------------------------------------------------- Eckart-Young, low rank
@pytest.mark.parametrize("alg", ["ei", "fp"])
def test_eckart_young_floor(alg):
    sigma = synth.sigma_pow(80, 1.0)
    A = synth.dense_from_spectrum(100, 80, sigma, seed=6)
    f = oracle.randqb_ei if alg == "ei" else oracle.randqb_fp
    for k in (5, 17, 40):
        r = f(A, 0.0, 6, seed=2, fixed_rank=k)
        floor = np.sqrt(np.sum(sigma[k:] ** 2))
        assert np.linalg.norm(A - r.Q @ r.B) >= floor * (1 - 1e-12)


@pytest.mark.parametrize("r_true", [30, 27])
@pytest.mark.parametrize("alg", ["ei", "fp"])
def test_exact_low_rank_stops_at_true_rank(r_true, alg):
    A = synth.dense_low_rank(70, 60, r_true, seed=r_true)
    f = oracle.randqb_ei if alg == "ei" else oracle.randqb_fp
    r = f(A, 1e-6, 10, seed=3)
    assert r.rank == r_true
    assert abs(r.E) <= 4 * 1.11e-16 * r.normA2   # Theorem 3's bound on the rounding of E
    assert np.linalg.norm(A - r.Q @ r.B) ** 2 <= 1e-20 * r.normA2


def test_orthogonality_and_row_by_row(A_exp):
    A = synth.dense_from_spectrum(400, 300, synth.sigma_exp(300, 40.0), seed=12)
    for f in (oracle.randqb_ei, oracle.randqb_fp):
        r = f(A, 1e-4, 16, seed=5)
        assert oracle.orth_loss(r.Q) <= 1e-13
        eps2 = (1e-4) ** 2 * r.normA2
        assert r.E_hist[-1] < eps2 <= r.E_hist[-2]   # stop at the first crossing row
        assert r.rank % 16 != 0 or r.rank == 0       # arbitrary integer rank here


def test_zero_matrix_and_loose_tolerance():
    Z = np.zeros((20, 10))
    for f in (oracle.randqb_ei, oracle.randqb_fp):
        r = f(Z, 0.1, 4, seed=1)
        assert r.rank == 0 and r.status == oracle.QB_OK
    A = synth.dense_from_spectrum(20, 10, synth.sigma_pow(10, 1.0), seed=1)
    r = oracle.randqb_ei(A, 1.5, 4, seed=1)   # tol >= 1: one row already meets it
    assert r.rank == 1


def test_rank_cap_not_converged():
    A = synth.dense_from_spectrum(50, 40, synth.sigma_pow(40, 0.5), seed=2)
    for f in (oracle.randqb_ei, oracle.randqb_fp):
        r = f(A, 1e-6, 4, seed=1, rank_cap=10)
        assert r.rank == 10 and r.status == oracle.QB_NOT_CONVERGED
        assert abs(r.E - np.linalg.norm(A - r.Q @ r.B) ** 2) <= 1e-12 * r.normA2


# ----------------------------------------------------------------------------- Theorem 3
def test_theorem3_floor():
    vals = {}
    with open(os.path.join(GOLDEN, "theorem3.txt")) as f:
        for line in f:
            if not line.startswith("#") and line.strip():
                k, v = line.split()
                vals[k] = float(v)
    floor = oracle.thm3_floor(1.0, u=vals["eps_mach"], delta=vals["delta"])
    assert round(floor, 8) == pytest.approx(vals["floor_rel"], abs=0.05e-7)
    A = synth.dense_low_rank(30, 20, 5, seed=1)
    r = oracle.randqb_ei(A, 1e-8, 4, seed=1)
    assert r.status == oracle.QB_WARN_TOL_FLOOR


def test_indicator_accuracy_above_theorem3_floor():
    # Fig. 2 setting scaled down: sigma_j = exp(-j/20); the relative error of E stays below
    # delta = 1% while E / ||A||^2 > (2.1e-7)^2.
    A = synth.dense_from_spectrum(300, 300, synth.sigma_exp(300, 20.0), seed=3)
    r = oracle.randqb_ei(A, 0.0, 10, seed=2, fixed_rank=300)
    normA2 = r.normA2
    for k in range(10, 300, 10):
        direct = np.linalg.norm(A - r.Q[:, :k] @ r.B[:k]) ** 2
        if direct / normA2 > 4.4e-14:
            assert abs(r.E_hist[k - 1] - direct) <= 0.01 * direct


# ----------------------------------------------------------------------------- sparse input
@pytest.mark.parametrize("alg", ["ei", "fp"])
def test_sparse_equals_dense(alg):
    csr = synth.csr_zipf(300, 200, 12.0, 1.1, seed=4, val_dtype=np.float64)
    S = csr.to_scipy()
    D = S.toarray()
    f = oracle.randqb_ei if alg == "ei" else oracle.randqb_fp
    rs = f(S, 0.5, 8, seed=2, P=1, rank_cap=64)
    rd = f(D, 0.5, 8, seed=2, P=1, rank_cap=64)
    assert rs.rank == rd.rank
    assert qb_diff(rs, rd, D) <= 1e-12


def test_csr_generator_shape():
    csr = synth.csr_zipf(2000, 1000, 20.0, 1.1, seed=1)
    assert csr.rowptr.dtype == np.int32 and csr.colind.dtype == np.int32
    lens = np.diff(csr.rowptr)
    assert abs(lens.mean() - 20.0) < 1.0
    for i in range(0, 2000, 97):
        cols = csr.colind[csr.rowptr[i]:csr.rowptr[i + 1]]
        assert np.all(np.diff(cols) > 0)  # distinct, sorted
    counts = np.bincount(csr.colind, minlength=1000)
    assert counts.max() > 20 * counts.mean()   # Zipf hot columns


# ----------------------------------------------------------------------------- adjoint
def _loss(A, k, seed, GQ, GB):
    Q, B, _ = oracle.qb_fixed_rank(A, k, seed)
    return float(np.sum(GQ * Q) + np.sum(GB * B))


def test_fixed_rank_map_equals_randqb():
    A = synth.dense_from_spectrum(80, 60, synth.sigma_pow(60, 1.0), seed=3)
    Q, B, R = oracle.qb_fixed_rank(A, 12, seed=5)
    r = oracle.randqb_ei(A, 0.0, 4, seed=5, fixed_rank=12)
    assert np.linalg.norm(Q @ B - r.Q @ r.B) / np.linalg.norm(A) <= 1e-12
    assert np.all(np.diag(R) > 0)


def test_adjoint_finite_differences():
    m, n, k = 48, 36, 6
    A = synth.dense_from_spectrum(m, n, synth.sigma_pow(36, 1.0), seed=4)
    GQ, GB = synth.cotangents(m, n, k, seed=5)
    Abar = oracle.qb_fixed_rank_adjoint(A, k, 7, GQ, GB)
    rng = np.random.default_rng(0)
    h = 1e-6
    for _ in range(3):
        V = rng.standard_normal((m, n))
        fd = (_loss(A + h * V, k, 7, GQ, GB) - _loss(A - h * V, k, 7, GQ, GB)) / (2 * h)
        an = float(np.sum(Abar * V))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))


def test_adjoint_matches_torch_autograd():
    torch = pytest.importorskip("torch")
    m, n, k = 512, 384, 32
    A = synth.dense_from_spectrum(m, n, synth.sigma_pow(384, 1.0), seed=8)
    GQ, GB = synth.cotangents(m, n, k, seed=9)
    Om = oracle.omega(n, 0, k, 3)
    At = torch.tensor(A, dtype=torch.float64, requires_grad=True)
    Y = At @ torch.tensor(Om)
    Q, R = torch.linalg.qr(Y)
    s = torch.sign(torch.diagonal(R))
    Q = Q * s[None, :]
    B = Q.T @ At
    L = (torch.tensor(GQ) * Q).sum() + (torch.tensor(GB) * B).sum()
    L.backward()
    ref = At.grad.numpy()
    ours = oracle.qb_fixed_rank_adjoint(A, k, 3, GQ, GB)
    assert np.linalg.norm(ours - ref) <= 1e-10 * np.linalg.norm(ref)


# ----------------------------------------------------------------------------- reduced sketch copy
def _bf16(X):
    """Round float64 entries to bfloat16 (round to nearest even) and back (test-side model of a
    reduced copy of A; the product path has its own kernel for this)."""
    u = np.ascontiguousarray(X, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("alg", ["ei", "fp"])
def test_sketch_copy_still_gives_qb_of_a(alg):
    """With the sketches taken on bf16(A) (a span only), Theorem 1 and B = Q^T A still hold for A
    itself: for randQB_FP because the B_i formula of Sect. 4.2 needs only H = A^T G for the G it
    uses.  A mistake that formed H or B_i from the sketch copy breaks both checks."""
    A = synth.dense_from_spectrum(300, 200, synth.sigma_exp(200, 20.0, 1e-6), seed=31)
    As = _bf16(A)
    assert np.linalg.norm(A - As) > 1e-4 * np.linalg.norm(A)
    f = oracle.randqb_ei if alg == "ei" else oracle.randqb_fp
    r = f(A, 1e-3, 10, seed=3, P=1, A_sketch=As)
    assert r.status in (0, 2)
    nA2 = r.normA2
    assert np.linalg.norm(r.B - r.Q.T @ A) <= 1e-10 * np.sqrt(nA2)
    assert abs(r.E - np.linalg.norm(A - r.Q @ r.B) ** 2) <= 1e-12 * nA2
    assert oracle.orth_loss(r.Q) <= 1e-12
    # the sketch copy changes Q (a different span), not its validity
    r0 = f(A, 1e-3, 10, seed=3, P=1)
    assert np.linalg.norm(r0.Q @ r0.B - r.Q @ r.B) > 1e-8 * np.sqrt(nA2)
