"""Batched randQB_EI (one launch per stage over all matrices, conditional CUDA graph loop) against
the float64 oracle run matrix by matrix, on the batched workload's structure: uneven shapes,
sigma_j = s j^-2 with a per-matrix scale s, per-matrix tolerance from {1e-2, 1e-3}."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1606_09402_gb300 as qb  # noqa: E402


def _batch(count, seed, lo, hi):
    specs = synth.batched_specs(count, seed, lo=lo, hi=hi)
    mats = []
    for s in specs:
        r = min(s.m, s.n, 256)
        A = synth.dense_from_spectrum(s.m, s.n, synth.sigma_pow(r, 2.0, s.scale), s.seed)
        mats.append(A.astype(np.float32))
    return specs, mats


def test_batched_matches_oracle_per_matrix():
    specs, mats = _batch(12, 3, 100, 700)
    As = [torch.tensor(A).cuda() for A in mats]
    res = qb.qb_ei_batched(As, [s.tol for s in specs], seed=40)
    for t, (s, A, (Q, B, info)) in enumerate(zip(specs, mats, res)):
        A64 = A.astype(np.float64)
        assert info.converged, (t, info)
        err = np.linalg.norm(A64 - (Q.double() @ B.double()).cpu().numpy()) / np.linalg.norm(A64)
        assert err < s.tol, (t, err, s.tol)
        ref = oracle.randqb_ei(A64, s.tol, 16, seed=40 + t)
        sv = synth.sigma_pow(min(s.m, s.n, 256), 2.0, s.scale)
        assert synth.svd_rank(sv, s.tol) <= info.rank <= int(1.15 * ref.rank) + 2, (t, info.rank, ref.rank)
        assert abs(info.err2_est - err ** 2 * info.normA2) <= 4 * 2.0 ** -24 * info.normA2


def test_batched_uneven_and_rank_cap():
    rng = np.random.default_rng(5)
    mats = [rng.standard_normal((m, n)).astype(np.float32) for m, n in
            [(300, 17), (17, 300), (64, 64), (513, 129)]]
    As = [torch.tensor(A).cuda() for A in mats]
    res = qb.qb_ei_batched(As, [1e-6] * 4, seed=1, rank_cap=40)
    for A, (Q, B, info) in zip(mats, res):
        cap = min(A.shape[0], A.shape[1], 40)
        assert info.rank == cap
        Qh = Q.double().cpu().numpy()
        assert oracle.orth_loss(Qh) < 1e-4
        Bh = B.double().cpu().numpy()
        assert np.linalg.norm(Bh - Qh.T @ A) <= 1e-5 * np.linalg.norm(A)
