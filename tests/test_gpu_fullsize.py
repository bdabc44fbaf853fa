"""The benchmark workload at full size, with the inputs and the call that bench.py times.

The workload: dense 40000 x 20000, sigma_j = exp(-j/200) + 1e-6 (j <= 4096), on the mixed path
(A as bf16 hi + lo), b = 64, P = 1, relative tol 1e-3, l~ = 3200, rank cap 4096.

The float64 oracle cannot factor this size inside a test.  The checks are therefore properties
that hold at any size, plus outputs computed one by one:

* ||A - QB||_F / ||A||_F < tol, in float64 on the GPU: the tolerance the algorithms promise.
* The rank is at least the SVD-optimal rank for tol (Eckart-Young, from the spectrum) and
  within 10% of it.
* |E - ||A - QB||_F^2| <= 4 u_32 ||A||_F^2: Theorem 1's identity within Theorem 3's float32
  bound.
* ||Q^T Q - I||_max <= 1e-4 (float32 Q).
* randQB_EI, whose B_i = Q_i^T A comes straight from the precise pass: 256 sampled entries of B
  against float64 dot products of the stored Q's and A's columns, within 1e-5 of |Q|^T |A| (the
  bar of the single-pass tests).
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1606_09402_gb300 as qb  # noqa: E402

M, N, R = 40000, 20000, 4096
TOL, B, P, L_TILDE, CAP = 1e-3, 64, 1, 3200, 4096
SEED_A, SEED_OMEGA = 1606, 9402
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def workload():
    sigma = synth.sigma_exp(R, 200.0, 1e-6)
    A64 = synth.dense_from_spectrum_torch(M, N, sigma, SEED_A, "cuda", dtype=torch.float64)
    hi, lo, norms = qb.quantize_bf16x2(A64)
    yield A64, hi, lo, norms[0], sigma
    del A64, hi, lo
    torch.cuda.empty_cache()


def _svd_rank(sigma, tol):
    """Smallest k with sum_{j > k} sigma_j^2 < tol^2 sum_j sigma_j^2 (Eckart-Young)."""
    s2 = np.sort(np.asarray(sigma, dtype=np.float64))[::-1] ** 2
    tails = s2.sum() - np.cumsum(s2)          # tails[k - 1] = sum over j > k
    return int(np.argmax(tails < tol * tol * s2.sum())) + 1


@pytest.mark.parametrize("alg", ["fp", "ei"])
def test_full_size_workload(workload, alg):
    A64, hi, lo, normA2, sigma = workload
    kw = dict(P=P, seed=SEED_OMEGA, a_lo=lo, src_norm2=normA2, prec="mixed", rank_cap=CAP)
    if alg == "fp":
        Q, Bm, info = qb.qb_fp_dense(hi, TOL, B, l_tilde=L_TILDE, **kw)
    else:
        Q, Bm, info = qb.qb_ei_dense(hi, TOL, B, **kw)
    assert info.converged, info
    k = info.rank
    k_opt = _svd_rank(sigma, TOL)
    assert k_opt <= k <= 1.1 * k_opt, (k, k_opt)

    Bd = Bm.double()
    err2 = 0.0
    for r0 in range(0, M, 4096):
        D = A64[r0:r0 + 4096] - Q[r0:r0 + 4096].double() @ Bd
        err2 += float((D * D).sum())
    del D, Bd
    assert err2 < TOL * TOL * normA2, (err2 / normA2) ** 0.5
    assert abs(info.err2_est - err2) <= 4 * U32 * normA2, (info.err2_est, err2)

    Qd = Q.double()
    G = Qd.T @ Qd
    G.diagonal().sub_(1.0)
    assert G.abs().max().item() <= 1e-4
    del Qd, G

    if alg == "ei":
        rng = np.random.default_rng(3)
        ii = rng.integers(0, k, 256)
        jj = rng.integers(0, N, 256)
        Qc = Q[:, torch.tensor(ii, device="cuda")].double().cpu().numpy()   # M x 256
        Ac = A64[:, torch.tensor(jj, device="cuda")].cpu().numpy()          # M x 256
        ref = np.einsum("ri,ri->i", Qc, Ac)
        scale = np.einsum("ri,ri->i", np.abs(Qc), np.abs(Ac))
        got = Bm[torch.tensor(ii, device="cuda"), torch.tensor(jj, device="cuda")]
        got = got.double().cpu().numpy()
        assert np.all(np.abs(got - ref) <= 1e-5 * scale), np.max(np.abs(got - ref) / scale)
