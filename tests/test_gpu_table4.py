"""Table 4 (Sect. 5.4) on the GPU: the three 8000 x 8000 test matrices of Sect. 5.2 with their
exact spectra, randQB_EI and randQB_FP at P = 1 (b = 10; b = 40 on the last row, as the table
does), through the C ABI.

The paper prints, per row, the SVD-optimal rank under the relative criterion
||A - QB||_F < eps ||A||_F and the ranks its randomized runs reached (its own Omega, Matlab).  The
golden file holds those numbers (and a CPU test reproduces the SVD column from the spectra in
closed form).  Here each GPU result must:
  * meet the tolerance, with the true error computed in float64 on the device;
  * have rank >= the SVD-optimal rank (Eckart-Young);
  * stay at most 2% (at least 3) above the rank the paper printed for the same algorithm: the
    excess over the SVD rank depends on the spectrum and on b, P, not on the particular Omega;
  * on the float64 path, for the rows of small rank, equal the float64 oracle (rank and
    ||QB_gpu - QB_cpu||_F / ||A||_F <= 1e-10, same Omega).
The mixed path runs the rows whose tolerance lies above the float32 stop margin (Theorem 3)."""
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1606_09402_gb300 as qb  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table4_svd_ranks.txt")
N = 8000
SEED_A = {"M1": 801, "M2": 802, "M3": 803}
SEED_OMEGA = 1654


def _rows():
    rows = []
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            m, n, eps, r_svd, r_ei, r_fp = line.split()
            rows.append((m, int(n), float(eps), int(r_svd), int(r_ei), int(r_fp)))
    return rows


ROWS = _rows()


@pytest.fixture(scope="module")
def mats():
    spectra = synth.table4_matrix_spectra(N)
    return {k: synth.dense_from_spectrum_torch(N, N, spectra[k], SEED_A[k], "cuda",
                                               dtype=torch.float64, work_dtype=torch.float64)
            for k in ("M1", "M2", "M3")}


def _true_err(A, Q, B):
    err2 = 0.0
    for r0 in range(0, A.shape[0], 2000):
        D = A[r0:r0 + 2000] - Q[r0:r0 + 2000].double() @ B.double()
        err2 += float((D * D).sum())
    return (err2 / float((A * A).sum())) ** 0.5


@pytest.mark.parametrize("row", ROWS, ids=[f"{r[0]}-{r[2]:g}" for r in ROWS])
@pytest.mark.parametrize("alg", ["ei", "fp"])
def test_table4_fp64(mats, row, alg):
    mat, n, eps, r_svd, r_ei, r_fp = row
    b = 40 if eps == 1.5e-3 else 10
    A = mats[mat]
    f = qb.qb_ei_dense if alg == "ei" else qb.qb_fp_dense
    Q, B, info = f(A, eps, b, P=1, seed=SEED_OMEGA)
    assert info.status == 0 and info.converged
    err = _true_err(A, Q, B)
    assert err < eps, (row, err)
    paper = r_ei if alg == "ei" else r_fp
    assert r_svd <= info.rank <= paper + max(3, 0.02 * paper), (row, info.rank, paper)
    if info.rank <= 100:
        Ah = A.cpu().numpy()
        ref = (oracle.randqb_ei if alg == "ei" else oracle.randqb_fp)(Ah, eps, b,
                                                                     seed=SEED_OMEGA, P=1)
        assert info.rank == ref.rank
        diff = np.linalg.norm((Q.double() @ B.double()).cpu().numpy() - ref.Q @ ref.B) / \
            np.linalg.norm(Ah)
        assert diff <= 1e-10, (row, diff)


# the mixed path's sketches read the bf16 A_hi, whose rounding leaves about
# (u_bf16^2 / 3)(k / n)(1 + sqrt(n / m))^2 ||A||^2 behind; at eps = 1.5e-3 and k ~ 1590 of 8000 that
# is ~40% of eps^2, so only the rows with eps = 1e-2 are held to the paper's ranks here
MIXED_ROWS = [r for r in ROWS if r[2] >= 1e-2]


@pytest.mark.parametrize("row", MIXED_ROWS, ids=[f"{r[0]}-{r[2]:g}" for r in MIXED_ROWS])
@pytest.mark.parametrize("alg", ["ei", "fp"])
def test_table4_mixed(mats, row, alg):
    mat, n, eps, r_svd, r_ei, r_fp = row
    b = 40 if eps == 1.5e-3 else 10
    A = mats[mat]
    hi, lo, norms = qb.quantize_bf16x2(A)
    f = qb.qb_ei_dense if alg == "ei" else qb.qb_fp_dense
    Q, B, info = f(hi, eps, b, P=1, seed=SEED_OMEGA, a_lo=lo, src_norm2=norms[0], prec="mixed")
    assert info.converged
    err = _true_err(A, Q, B)
    assert err < eps, (row, err)
    paper = r_ei if alg == "ei" else r_fp
    assert r_svd <= info.rank <= paper + max(3, 0.02 * paper), (row, info.rank)
