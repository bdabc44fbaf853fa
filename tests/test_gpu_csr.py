"""GPU parity of the sparse (CSR) paths against the float64 CPU oracle (scipy.sparse products),
through the C ABI, on the sparse workload's structure: Poisson row lengths, Zipf column
popularity (hot columns), log-normal values."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1606_09402_gb300 as qb  # noqa: E402


def _dev(csr, dtype):
    return (torch.tensor(csr.rowptr).cuda(), torch.tensor(csr.colind).cuda(),
            torch.tensor(csr.val.astype(dtype)).cuda())


@pytest.mark.parametrize("alg", ["ei", "fp"])
@pytest.mark.parametrize("P", [0, 1])
def test_csr_fp64_parity(alg, P):
    csr = synth.csr_zipf(3000, 1500, 30.0, 1.1, seed=909, val_dtype=np.float64)
    S = csr.to_scipy()
    rp, ci, v = _dev(csr, np.float64)
    f = qb.qb_ei_csr if alg == "ei" else qb.qb_fp_csr
    g = oracle.randqb_ei if alg == "ei" else oracle.randqb_fp
    Q, B, info = f(rp, ci, v, (csr.m, csr.n), 0.5, 32, P=P, seed=77, rank_cap=256)
    ref = g(S, 0.5, 32, seed=77, P=P, rank_cap=256)
    assert info.rank == ref.rank and info.status == ref.status
    D = S.toarray()
    diff = np.linalg.norm((Q.double() @ B.double()).cpu().numpy() - ref.Q @ ref.B) / np.linalg.norm(D)
    assert diff <= 1e-10
    assert abs(info.normA2 - oracle.frob2(S)) <= 1e-12 * info.normA2


def test_csr_ragged_and_empty_rows():
    rng = np.random.default_rng(3)
    m, n = 517, 389
    dense = rng.standard_normal((m, n)) * (rng.random((m, n)) < 0.02)
    dense[10:20] = 0.0          # empty rows
    dense[:, 5] = 1.0           # one fully dense (hot) column
    import scipy.sparse as sp
    S = sp.csr_matrix(dense)
    rp = torch.tensor(S.indptr.astype(np.int32)).cuda()
    ci = torch.tensor(S.indices.astype(np.int32)).cuda()
    v = torch.tensor(S.data).cuda()
    for f, g in ((qb.qb_ei_csr, oracle.randqb_ei), (qb.qb_fp_csr, oracle.randqb_fp)):
        Q, B, info = f(rp, ci, v, (m, n), 0.3, 7, P=1, seed=5)
        ref = g(S, 0.3, 7, seed=5, P=1)
        assert info.rank == ref.rank
        diff = np.linalg.norm((Q @ B).cpu().numpy() - ref.Q @ ref.B) / np.linalg.norm(dense)
        assert diff <= 1e-10


@pytest.mark.parametrize("alg", ["ei", "fp"])
def test_csr_mixed_float32(alg):
    csr = synth.csr_zipf(4000, 2000, 40.0, 1.1, seed=11, val_dtype=np.float32)
    S = csr.to_scipy().astype(np.float64)
    rp, ci, v = _dev(csr, np.float32)
    f = qb.qb_ei_csr if alg == "ei" else qb.qb_fp_csr
    Q, B, info = f(rp, ci, v, (csr.m, csr.n), 0.5, 32, P=1, seed=3, rank_cap=512)
    assert info.status == 0
    D = S.toarray()
    err = np.linalg.norm(D - (Q.double() @ B.double()).cpu().numpy()) / np.linalg.norm(D)
    assert err < 0.5
    ref = (oracle.randqb_ei if alg == "ei" else oracle.randqb_fp)(S, 0.5, 32, seed=3, P=1,
                                                                   rank_cap=512)
    assert abs(info.rank - ref.rank) <= 2


@pytest.mark.parametrize("alg", ["ei", "fp"])
def test_csr_long_rows_and_wide_slices(alg):
    """Rows and columns many times longer than one long-row segment (a full row of 4000 nonzeros,
    a half row, two full columns), and pass widths that fill 128-column staging slices and leave
    ragged ones (EI: w = b = 48; FP: l~ = 300), in float64 against the oracle."""
    import scipy.sparse as sp
    rng = np.random.default_rng(21)
    m, n = 700, 4000
    dense = rng.standard_normal((m, n)) * (rng.random((m, n)) < 0.01)
    dense[3, :] = rng.standard_normal(n)
    dense[100, ::2] = 1.0 + rng.random(n // 2)
    dense[:, 7] = rng.standard_normal(m)
    dense[:, 11] = 2.0
    S = sp.csr_matrix(dense)
    rp = torch.tensor(S.indptr.astype(np.int32)).cuda()
    ci = torch.tensor(S.indices.astype(np.int32)).cuda()
    v = torch.tensor(S.data).cuda()
    if alg == "ei":
        Q, B, info = qb.qb_ei_csr(rp, ci, v, (m, n), 0.2, 48, P=1, seed=8, rank_cap=480)
        ref = oracle.randqb_ei(S, 0.2, 48, seed=8, P=1, rank_cap=480)
    else:
        Q, B, info = qb.qb_fp_csr(rp, ci, v, (m, n), 0.2, 48, P=1, seed=8, rank_cap=480,
                                  l_tilde=300)
        ref = oracle.randqb_fp(S, 0.2, 48, seed=8, P=1, rank_cap=480, l_tilde=300)
    assert info.rank == ref.rank and info.status == ref.status
    diff = np.linalg.norm((Q @ B).cpu().numpy() - ref.Q @ ref.B) / np.linalg.norm(dense)
    assert diff <= 1e-10
