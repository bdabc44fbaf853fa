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


def test_batched_autotuner_choice_is_used_and_graph_reused():
    """The first call on a new batch-shape bucket tunes the two A-streaming stages and records its
    choice; the next call with the same shapes (and workspace) reuses both the choice and the
    captured iteration graph and gives the same result bit for bit.  Every pinned plan gives the
    same result too: the tile shape changes no summation order."""
    specs, mats = _batch(10, 17, 300, 1400)
    As = [torch.tensor(A).cuda() for A in mats]
    tols = [s.tol for s in specs]
    outs = [(torch.empty(min(A.shape), A.shape[0], device="cuda"),
             torch.empty(min(A.shape), A.shape[1], device="cuda")) for A in mats]
    import ctypes as C
    from paper_1606_09402_gb300 import _lib
    lib = _lib.load()
    descs = (_lib.qb_dense * len(As))(*[qb._dense_desc(A) for A in As])
    o = qb._opts(0.0, 16, 0, 40, True, None, None, True, "mixed")
    ws = torch.empty(lib.qb_ei_batched_workspace(len(As), descs, C.byref(o)), dtype=torch.uint8,
                     device="cuda")
    qb.batched_set_plan(None)
    r1 = qb.qb_ei_batched(As, tols, seed=40, outs=outs, workspace=ws)
    p1 = qb.batched_last_plan()
    snap = [(Q.clone(), B.clone(), i.rank) for Q, B, i in r1]
    r2 = qb.qb_ei_batched(As, tols, seed=40, outs=outs, workspace=ws)
    p2 = qb.batched_last_plan()
    assert p2["tuned"] == 0 and p2["graph_reused"] == 1
    for key in ("rows_per_thread", "cols_per_thread", "sketch_grid", "bpass_grid"):
        assert p1[key] == p2[key], (key, p1, p2)
    assert p1["rows_per_thread"] in (1, 2) and p1["cols_per_thread"] in (1, 2)
    for (Q, B, i), (Qs, Bs, k) in zip(r2, snap):
        assert i.rank == k and torch.equal(Q, Qs) and torch.equal(B, Bs)
    try:
        for cfg in [(1, 1, 4, 4), (2, 2, 16, 8), (2, 1, 8, 16)]:
            qb.batched_set_plan(cfg)
            r3 = qb.qb_ei_batched(As, tols, seed=40, outs=outs, workspace=ws)
            p3 = qb.batched_last_plan()
            assert (p3["rows_per_thread"], p3["cols_per_thread"]) == cfg[:2] and p3["tuned"] == 0
            for (Q, B, i), (Qs, Bs, k) in zip(r3, snap):
                assert i.rank == k and torch.equal(Q, Qs) and torch.equal(B, Bs), cfg
    finally:
        qb.batched_set_plan(None)


def test_batched_workload_every_matrix_meets_its_tolerance():
    """The benchmark's batch itself (256 float32 matrices, m, n ~ U[256, 4096], sigma_j = s j^-2,
    tol in {1e-2, 1e-3}): every converged matrix's true error is below its tolerance.  The stop
    test keeps a 2 u ||A||^2 margin for the rounding of ||B||^2 (Theorem 3); it holds only while
    Q stays orthonormal to ~u, since E misses tr(B^T (Q^T Q - I) B) of the true error."""
    specs = synth.batched_specs(256, 1606)
    mats = [synth.dense_from_spectrum_torch(s.m, s.n, synth.sigma_pow(min(s.m, s.n, 512), 2.0,
                                                                      s.scale),
                                            s.seed, "cuda", dtype=torch.float32) for s in specs]
    res = qb.qb_ei_batched(mats, [s.tol for s in specs], seed=9402)
    worst = 0.0
    for t, (s, A, (Q, B, info)) in enumerate(zip(specs, mats, res)):
        assert info.converged, (t, info)
        A64 = A.double()
        err = float(torch.linalg.norm(A64 - Q.double() @ B.double()) / torch.linalg.norm(A64))
        worst = max(worst, err / s.tol)
        assert err < s.tol, (t, s.m, s.n, s.tol, info.rank, err)
        Qd = Q.double()
        orth = float((Qd.T @ Qd - torch.eye(info.rank, dtype=torch.float64, device="cuda"))
                     .abs().max())
        assert orth <= 1e-6, (t, orth)
    assert worst < 1.0
