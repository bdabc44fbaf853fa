"""GPU parity of the COO paths (Sect. 5.1: the sparse matrix in coordinate format) against the
float64 CPU oracle, through the C ABI: the sparse workload's structure (Poisson row lengths,
Zipf column popularity, log-normal values), triplets sorted by row and shuffled (any order is
accepted), empty rows and columns, a long hot column (its entries span several 256-nonzero
chunks of the column-sorted copy), and the CSR path on the same matrix."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import scipy.sparse as sp  # noqa: E402

import paper_1606_09402_gb300 as qb  # noqa: E402


def _coo_dev(rows, cols, vals):
    return (torch.tensor(np.asarray(rows, dtype=np.int32)).cuda(),
            torch.tensor(np.asarray(cols, dtype=np.int32)).cuda(),
            torch.tensor(vals).cuda())


def _zipf_coo(m, n, mean, seed):
    csr = synth.csr_zipf(m, n, mean, 1.1, seed=seed, val_dtype=np.float64)
    S = csr.to_scipy().tocoo()
    return S, csr


@pytest.mark.parametrize("alg", ["ei", "fp"])
@pytest.mark.parametrize("P", [0, 1])
@pytest.mark.parametrize("order", ["row", "shuffled"])
def test_coo_fp64_parity(alg, P, order):
    S, _ = _zipf_coo(3000, 1500, 30.0, 909)
    r, c, v = S.row, S.col, S.data
    if order == "shuffled":
        p = np.random.default_rng(1).permutation(len(v))
        r, c, v = r[p], c[p], v[p]
    f = qb.qb_ei_coo if alg == "ei" else qb.qb_fp_coo
    g = oracle.randqb_ei if alg == "ei" else oracle.randqb_fp
    Q, B, info = f(*_coo_dev(r, c, v), S.shape, 0.5, 32, P=P, seed=77, rank_cap=256)
    ref = g(S.tocsr(), 0.5, 32, seed=77, P=P, rank_cap=256)
    assert info.rank == ref.rank and info.status == ref.status
    diff = np.linalg.norm((Q.double() @ B.double()).cpu().numpy() - ref.Q @ ref.B) / \
        np.sqrt(oracle.frob2(S.tocsr()))
    assert diff <= 1e-10
    assert abs(info.normA2 - oracle.frob2(S.tocsr())) <= 1e-12 * info.normA2


def test_coo_empty_rows_and_hot_column():
    rng = np.random.default_rng(3)
    m, n = 517, 389
    dense = rng.standard_normal((m, n)) * (rng.random((m, n)) < 0.02)
    dense[10:20] = 0.0          # empty rows
    dense[:, 40:44] = 0.0       # empty columns
    dense[:, 5] = 1.0           # a fully dense hot column: 517 entries, three 256-chunks
    S = sp.coo_matrix(dense)
    p = np.random.default_rng(2).permutation(S.nnz)
    for f, g in ((qb.qb_ei_coo, oracle.randqb_ei), (qb.qb_fp_coo, oracle.randqb_fp)):
        Q, B, info = f(*_coo_dev(S.row[p], S.col[p], S.data[p]), (m, n), 0.3, 7, P=1, seed=5)
        ref = g(sp.csr_matrix(dense), 0.3, 7, seed=5, P=1)
        assert info.rank == ref.rank
        diff = np.linalg.norm((Q @ B).cpu().numpy() - ref.Q @ ref.B) / np.linalg.norm(dense)
        assert diff <= 1e-10


def test_coo_mixed_matches_csr_mixed():
    """float32 values (the mixed path): COO and CSR run the same loop on the same matrix; their
    passes sum in different orders, so the results agree to float32 rounding, not bit for bit."""
    S, csr = _zipf_coo(4000, 2000, 40.0, 31)
    v32 = S.data.astype(np.float32)
    Qc, Bc, ic = qb.qb_ei_coo(*_coo_dev(S.row, S.col, v32), S.shape, 0.5, 32, P=1, seed=3,
                              rank_cap=512)
    rp = torch.tensor(csr.rowptr).cuda()
    ci = torch.tensor(csr.colind).cuda()
    vc = torch.tensor(csr.val.astype(np.float32)).cuda()
    Qr, Br, ir = qb.qb_ei_csr(rp, ci, vc, S.shape, 0.5, 32, P=1, seed=3, rank_cap=512)
    assert abs(ic.rank - ir.rank) <= 1
    k = min(ic.rank, ir.rank)
    X = (Qc[:, :k].double() @ Bc[:k].double()).cpu().numpy()
    Y = (Qr[:, :k].double() @ Br[:k].double()).cpu().numpy()
    assert np.linalg.norm(X - Y) <= 1e-4 * np.sqrt(oracle.frob2(S.tocsr()))
    A = S.toarray().astype(np.float32).astype(np.float64)
    err = np.linalg.norm(A - (Qc.double() @ Bc.double()).cpu().numpy()) / np.linalg.norm(A)
    assert ic.converged and err < 0.5
