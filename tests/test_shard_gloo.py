"""Row-sharded randQB_EI on CPU ranks (gloo, world size 2 and 3): the multi-GPU design of the hot
path, tested without GPUs.

Each rank holds a block of A's rows (uneven blocks).  Per block of Algorithm 2:
  * Y_p = A_p Omega_i - Q_p (B Omega_i) is local (Omega and B are replicated);
  * the power step's A^T Y = sum_p A_p^T Y_p and Q^T Y = sum_p Q_p^T Y_p are all-reduced (n x b and
    k x b); Z = orth(.) is formed on every rank from the same reduced values;
  * orth(Y) is CholeskyQR2 over the ranks: W = sum_p Y_p^T Y_p (all-reduced b x b Gram), R from a
    Cholesky of W on every rank, Y_p <- Y_p R^-1, twice; the re-orthogonalisation coefficients
    Q^T Q_i are one more k x b all-reduce;
  * B_i = sum_p Q_{i,p}^T A_p is one b x n all-reduce, and the indicator of Theorem 1 with the
    row-by-row stop of Sect. 3.1 runs on every rank on the same B_i.
The gathered Q and the replicated B must reproduce the float64 oracle's randqb_ei: the same rank
and the same QB up to rounding (CholeskyQR2 and Householder QR with a positive diagonal give
the same Q for a full-rank block).  Every rank forms the replicated quantities (R, Z, B_i, E)
from the same all-reduced float64 values."""
import os
import socket

import numpy as np
import pytest

import oracle
import synth
from oracle import qb as oqb

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _allreduce(x):
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64))
    torch.distributed.all_reduce(t)
    return t.numpy()


def _cholqr_dist(Yp):
    """One CholeskyQR pass over the ranks: W = sum_p Y_p^T Y_p, W = R^T R, Y_p R^-1."""
    W = _allreduce(Yp.T @ Yp)
    R = np.linalg.cholesky(W).T
    return np.linalg.solve(R.T, Yp.T).T


def _orth_dist(Yp):
    return _cholqr_dist(_cholqr_dist(Yp))


def _sharded_ei(Ap, n, normA2, tol, b, seed, P, cap):
    """Algorithm 2 on the local rows Ap; returns (local Q rows, B, rank, E)."""
    eps2 = (tol * np.sqrt(normA2)) ** 2
    Qp = np.zeros((Ap.shape[0], 0))
    B = np.zeros((0, n))
    E = normA2
    k = 0
    hist = []
    while k < cap:
        bi = min(b, cap - k)
        Om = oqb._omega(n, k, bi, seed)
        Yp = Ap @ Om - Qp @ (B @ Om)
        for _ in range(P):
            Yp = _orth_dist(Yp)
            AtY = _allreduce(Ap.T @ Yp)
            QtY = _allreduce(Qp.T @ Yp)
            Z = oracle.orth(AtY - B.T @ QtY)
            Yp = Ap @ Z - Qp @ (B @ Z)
        Qi = _orth_dist(Yp)
        if k > 0:
            Qi = _orth_dist(Qi - Qp @ _allreduce(Qp.T @ Qi))
        Bi = _allreduce(Qi.T @ Ap)
        E, keep, stop = oqb._row_by_row(E, Bi, eps2, hist, True)
        Qp = np.hstack([Qp, Qi[:, :keep]])
        B = np.vstack([B, Bi[:keep]])
        k += keep
        if stop:
            break
    return Qp, B, k, E


def _worker(rank, world, port, cfg, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m, n, tol, b, seed, P = cfg
        A = synth.dense_from_spectrum(m, n, synth.sigma_exp(min(m, n), 12.0, 1e-8), seed=61)
        # uneven row blocks
        cuts = [0] + [int(m * (p + 1) / world) + (7 if p + 1 < world else 0) for p in range(world)]
        cuts[-1] = m
        Ap = A[cuts[rank]:cuts[rank + 1]]
        normA2 = float(_allreduce(np.array([oracle.frob2(Ap)]))[0])
        Qp, B, k, E = _sharded_ei(Ap, n, normA2, tol, b, seed, P, min(m, n))
        np.save(os.path.join(out_dir, f"Q{rank}.npy"), Qp)
        if rank == 0:
            np.save(os.path.join(out_dir, "B.npy"), B)
            np.save(os.path.join(out_dir, "kE.npy"), np.array([k, E]))
    finally:
        torch.distributed.destroy_process_group()


@pytest.mark.timeout(600)
@pytest.mark.parametrize("world,P", [(2, 0), (2, 1), (3, 1)])
def test_row_sharded_ei_matches_oracle(tmp_path, world, P):
    m, n, tol, b, seed = 500, 300, 1e-3, 16, 77
    ctx = torch.multiprocessing.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, (m, n, tol, b, seed, P), str(tmp_path)))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=540)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    Q = np.vstack([np.load(tmp_path / f"Q{r}.npy") for r in range(world)])
    B = np.load(tmp_path / "B.npy")
    k, E = np.load(tmp_path / "kE.npy")
    A = synth.dense_from_spectrum(m, n, synth.sigma_exp(min(m, n), 12.0, 1e-8), seed=61)
    ref = oracle.randqb_ei(A, tol, b, seed=seed, P=P)
    assert int(k) == ref.rank and Q.shape[1] == ref.rank
    nA = np.linalg.norm(A)
    assert np.linalg.norm(Q @ B - ref.Q @ ref.B) <= 1e-10 * nA
    assert abs(E - ref.E) <= 1e-12 * ref.normA2
    assert oracle.orth_loss(Q) <= 1e-12
    assert np.linalg.norm(A - Q @ B) < tol * nA
