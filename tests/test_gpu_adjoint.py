"""The fixed-rank QB map and its adjoint on the GPU (through the C ABI) against the float64
oracle, which is itself pinned by central finite differences and torch autograd
(tests/test_oracle_qb.py); plus finite differences of the GPU forward and the autograd.Function."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1606_09402_gb300 as qb  # noqa: E402


@pytest.fixture(scope="module")
def small():
    m, n, k = 512, 384, 32
    A = synth.dense_from_spectrum(m, n, synth.sigma_pow(384, 1.0), seed=8)
    GQ, GB = synth.cotangents(m, n, k, seed=9)
    return A, GQ, GB, k


def test_fixed_rank_forward_fp64(small):
    A, _, _, k = small
    Q, B, R = qb.qb_fixed_rank_fwd(torch.tensor(A).cuda(), k, 3)
    Qr, Br, Rr = oracle.qb_fixed_rank(A, k, 3)
    QB = (Q @ B).cpu().numpy()
    assert np.linalg.norm(QB - Qr @ Br) / np.linalg.norm(A) <= 1e-10
    assert np.linalg.norm(Q.cpu().numpy() - Qr) <= 1e-9 * np.sqrt(k)
    assert np.linalg.norm(R.cpu().numpy() - Rr) <= 1e-10 * np.linalg.norm(Rr)


def test_fixed_rank_adjoint_fp64_matches_oracle(small):
    A, GQ, GB, k = small
    Ad = torch.tensor(A).cuda()
    Q, B, R = qb.qb_fixed_rank_fwd(Ad, k, 3)
    GA = qb.qb_fixed_rank_bwd(Ad, k, 3, Q, R, torch.tensor(GQ).cuda(), torch.tensor(GB).cuda())
    ref = oracle.qb_fixed_rank_adjoint(A, k, 3, GQ, GB)
    assert np.linalg.norm(GA.cpu().numpy() - ref) <= 1e-10 * np.linalg.norm(ref)


def test_fixed_rank_adjoint_finite_differences_on_gpu(small):
    A, GQ, GB, k = small
    Ad = torch.tensor(A).cuda()
    GQd, GBd = torch.tensor(GQ).cuda(), torch.tensor(GB).cuda()
    Q, B, R = qb.qb_fixed_rank_fwd(Ad, k, 3)
    GA = qb.qb_fixed_rank_bwd(Ad, k, 3, Q, R, GQd, GBd)
    V = np.random.default_rng(1).standard_normal(A.shape)
    V = torch.tensor(V / np.linalg.norm(V)).cuda()     # unit direction
    h = 1e-5

    def loss(X):
        Qx, Bx, _ = qb.qb_fixed_rank_fwd(X, k, 3)
        return float((GQd * Qx).sum() + (GBd * Bx).sum())

    fd = (loss(Ad + h * V) - loss(Ad - h * V)) / (2 * h)
    an = float((GA * V).sum())
    assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))


def test_autograd_function(small):
    A, GQ, GB, k = small
    Ad = torch.tensor(A).cuda().requires_grad_(True)
    Q, B = qb.QBFixedRank.apply(Ad, k, 3)
    L = (torch.tensor(GQ).cuda() * Q).sum() + (torch.tensor(GB).cuda() * B).sum()
    L.backward()
    ref = oracle.qb_fixed_rank_adjoint(A, k, 3, GQ, GB)
    assert np.linalg.norm(Ad.grad.cpu().numpy() - ref) <= 1e-10 * np.linalg.norm(ref)


def test_fixed_rank_fp64_ragged_panels():
    """k = 150: three panels (64, 64, 22) of the blocked QR, the multi-panel Gram-Schmidt, and the
    column-parallel triangular inverse of the backward at k > 128."""
    m, n, k = 700, 500, 150
    A = synth.dense_from_spectrum(m, n, synth.sigma_pow(n, 1.0), seed=12)
    GQ, GB = synth.cotangents(m, n, k, seed=13)
    Ad = torch.tensor(A).cuda()
    Q, B, R = qb.qb_fixed_rank_fwd(Ad, k, 4)
    Qr, Br, Rr = oracle.qb_fixed_rank(A, k, 4)
    assert np.linalg.norm((Q @ B).cpu().numpy() - Qr @ Br) / np.linalg.norm(A) <= 1e-10
    assert np.linalg.norm(Q.cpu().numpy() - Qr) <= 1e-9 * np.sqrt(k)
    assert np.linalg.norm(R.cpu().numpy() - Rr) <= 1e-10 * np.linalg.norm(Rr)
    GA = qb.qb_fixed_rank_bwd(Ad, k, 4, Q, R, torch.tensor(GQ).cuda(), torch.tensor(GB).cuda())
    ref = oracle.qb_fixed_rank_adjoint(A, k, 4, GQ, GB)
    assert np.linalg.norm(GA.cpu().numpy() - ref) <= 1e-10 * np.linalg.norm(ref)


@pytest.mark.parametrize("m,n,k", [(2048, 1536, 64), (1000, 904, 150), (8192, 8192, 256)])
def test_fixed_rank_mixed_bf16(m, n, k):
    """BF16 storage with float32 accumulation against the float64 oracle evaluated on the same
    (bf16-valued) A and the same bf16-rounded Omega."""
    sigma = 1.0 / np.arange(1, min(m, n) + 1)
    A = synth.dense_from_spectrum_torch(m, n, sigma, 1606, "cuda", dtype=torch.float32)
    Ab = A.to(torch.bfloat16)
    GQ, GB = synth.cotangents(m, n, k, seed=5)
    Q, B, R = qb.qb_fixed_rank_fwd(Ab, k, 9)
    GA = qb.qb_fixed_rank_bwd(Ab, k, 9, Q, R, torch.tensor(GQ).cuda(), torch.tensor(GB).cuda())
    A64 = Ab.double().cpu().numpy()
    Om = torch.tensor(oracle.omega_f32(n, 0, k, 9)).to(torch.bfloat16).double().numpy()
    Qr, Br, _ = oracle.qb_fixed_rank(A64, k, 9, Omega=Om)
    ref = oracle.qb_fixed_rank_adjoint(A64, k, 9, GQ, GB, Omega=Om)
    QB = (Q.double() @ B.double()).cpu().numpy()
    assert np.linalg.norm(QB - Qr @ Br) / np.linalg.norm(A64) <= 1e-5
    Rr = oracle.qb_fixed_rank(A64, k, 9, Omega=Om)[2]
    assert np.linalg.norm(R.double().cpu().numpy() - Rr) <= 5e-4 * np.linalg.norm(Rr)
    err = np.linalg.norm(GA.double().cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err <= 2e-3, err
