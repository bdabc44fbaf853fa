"""GPU parity of the dense paths against the float64 CPU oracle, through the C ABI.

Float64 path: ||QB_gpu - QB_cpu||_F / ||A||_F <= 1e-10 and the same rank (the rank may differ by
one only where E sits within 1e-12 ||A||^2 of eps^2).  Mixed path: the achieved error
||A - QB||_F / ||A||_F (float64, on the CPU) is below the tolerance and the rank is close to the
oracle's.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1606_09402_gb300 as qb  # noqa: E402

from oracle_spread import PARITY, common_qb, parity_bound, spread  # noqa: E402


def _qb(Q, B):
    return (Q.double() @ B.double()).cpu().numpy()


def _check_parity(A, res, ref, tol_rel, label="", bound=PARITY):
    """QB and E against the oracle.  A rank that differs by one is allowed only where E sits within
    1e-12 ||A||^2 of eps^2 (a numerical tie of the stopping test); QB is then still compared over
    the common leading rank, where both results hold the same blocks."""
    Q, B, info = res
    normA = np.linalg.norm(A)
    if info.rank != ref.rank:
        eps2 = (tol_rel ** 2) * ref.normA2
        near = min(abs(e - eps2) for e in ref.E_hist[max(0, min(info.rank, ref.rank) - 2):])
        assert abs(info.rank - ref.rank) <= 1 and near <= 1e-12 * ref.normA2, \
            (label, info.rank, ref.rank)
    X, Y = common_qb(Q.double().cpu().numpy(), B.double().cpu().numpy(), ref.Q, ref.B)
    diff = np.linalg.norm(X - Y) / normA
    assert diff <= bound, (label, diff, bound)
    if info.rank == ref.rank:
        assert abs(info.err2_est - ref.E) <= max(1e-10, bound) * ref.normA2, \
            (label, info.err2_est, ref.E)


# ----------------------------------------------------------------------------- Omega
def test_omega_f64_matches_oracle():
    for (n, c0, w, seed) in [(1000, 0, 37, 9402), (777, 13, 20, (1 << 40) + 3), (5, 3, 1, 0)]:
        g = qb.qb_omega(n, c0, w, seed, dtype=torch.float64).cpu().numpy()
        r = oracle.omega(n, c0, w, seed)
        np.testing.assert_allclose(g, r, rtol=1e-13, atol=1e-13)


def test_omega_f32_and_bf16():
    n, c0, w, seed = 3000, 5, 24, 77
    g = qb.qb_omega(n, c0, w, seed, dtype=torch.float32).cpu().numpy().astype(np.float64)
    r = oracle.omega_f32(n, c0, w, seed).astype(np.float64)
    err = np.abs(g - r) / (1 + np.abs(r))
    assert np.quantile(err, 0.999) < 1e-5 and err.max() < 1e-3
    gb = qb.qb_omega(n, c0, w, seed, dtype=torch.bfloat16).float().cpu().numpy()
    assert np.max(np.abs(gb - g) / (1 + np.abs(g))) < 2.0 ** -8


# ----------------------------------------------------------------------------- 2000 x 2000 workload
@pytest.fixture(scope="module")
def A2000():
    return synth.dense_from_spectrum(2000, 2000, synth.sigma_pow(2000, 1.5), seed=1606)


@pytest.mark.parametrize("alg", ["ei", "fp"])
@pytest.mark.parametrize("P", [0, 1])
@pytest.mark.parametrize("tol", [0.05, 2e-3])
def test_fp64_parity_2000(A2000, alg, P, tol):
    Ad = torch.tensor(A2000, device="cuda")
    f = qb.qb_ei_dense if alg == "ei" else qb.qb_fp_dense
    g = oracle.randqb_ei if alg == "ei" else oracle.randqb_fp
    res = f(Ad, tol, 20, P=P, seed=9402)
    ref = g(A2000, tol, 20, seed=9402, P=P)
    assert res[2].status == ref.status
    _check_parity(A2000, res, ref, tol, f"{alg} P={P} tol={tol}")


# ----------------------------------------------------------------------------- ragged shapes, edge cases
@pytest.mark.parametrize("alg", ["ei", "fp"])
@pytest.mark.parametrize("m,n,b,P,tol,cap,lt", [
    (517, 389, 7, 1, 1e-3, None, None),     # ragged tiles, b not a power of two
    (389, 517, 64, 0, 1e-4, None, 100),      # wide A, full-width blocks, several FP batches
    (130, 70, 16, 2, 1e-6, 40, None),        # rank cap reached -> not converged
    (65, 1, 3, 0, 1e-2, None, None),         # single column
])
def test_fp64_parity_ragged(alg, m, n, b, P, tol, cap, lt):
    k = min(m, n)
    sigma = synth.sigma_exp(k, max(k / 8.0, 1.0))
    A = synth.dense_from_spectrum(m, n, sigma, seed=m * 7 + n)
    Ad = torch.tensor(A, device="cuda")
    if alg == "ei":
        res = qb.qb_ei_dense(Ad, tol, b, P=P, seed=5, rank_cap=cap)
        ref = oracle.randqb_ei(A, tol, b, seed=5, P=P, rank_cap=cap)
    else:
        res = qb.qb_fp_dense(Ad, tol, b, P=P, seed=5, rank_cap=cap, l_tilde=lt)
        ref = oracle.randqb_fp(A, tol, b, seed=5, P=P, rank_cap=cap, l_tilde=lt)
    assert res[2].status == ref.status
    # 1e-10, unless two float64 runs of the oracle itself (A and row-permuted A) already disagree
    # by more than 1e-11: randQB_FP's B_i formula amplifies rounding by (sigma_1 / sigma_k)^2
    # (Remark 4.1); at 389 x 517 (rank 389, sigma_1 / sigma_k ~ 3e3) the oracle's own spread is 3e-9
    sp, _ = spread(A, alg, tol, b, seed=5, P=P, rank_cap=cap,
                   **({} if alg == "ei" else {"l_tilde": lt}))
    _check_parity(A, res, ref, tol, f"{alg} {m}x{n} spread={sp:.1e}", parity_bound(sp))


@pytest.mark.parametrize("P", [0, 1, 2])
def test_ei_passes_follow_table1(P):
    """randQB_EI reads A 2 + 2P times per block (Table 1): the sketch, 2P power steps, B_i."""
    A = synth.dense_from_spectrum(600, 400, synth.sigma_exp(400, 40.0), seed=8)
    _, _, info = qb.qb_ei_dense(torch.tensor(A, device="cuda"), 1e-3, 16, P=P, seed=2)
    assert info.blocks >= 3
    assert info.passes == (2 + 2 * P) * info.blocks


@pytest.mark.parametrize("alg", ["ei", "fp"])
@pytest.mark.parametrize("r_true", [30, 27])
def test_exact_low_rank(alg, r_true):
    A = synth.dense_low_rank(300, 200, r_true, seed=r_true)
    f = qb.qb_ei_dense if alg == "ei" else qb.qb_fp_dense
    Q, B, info = f(torch.tensor(A, device="cuda"), 1e-6, 10, seed=3)
    assert info.rank == r_true
    assert abs(info.err2_est) <= 4 * 1.11e-16 * info.normA2 * 10
    assert np.linalg.norm(A - _qb(Q, B)) ** 2 <= 1e-18 * info.normA2


@pytest.mark.parametrize("alg", ["ei", "fp"])
def test_zero_and_loose_and_nonfinite(alg):
    f = qb.qb_ei_dense if alg == "ei" else qb.qb_fp_dense
    Z = torch.zeros(50, 40, dtype=torch.float64, device="cuda")
    Q, B, info = f(Z, 0.1, 8, seed=1)
    assert info.rank == 0 and info.status == 0
    A = synth.dense_from_spectrum(50, 40, synth.sigma_pow(40, 1.0), seed=1)
    Q, B, info = f(torch.tensor(A, device="cuda"), 1.5, 8, seed=1)
    assert info.rank == 1
    A[3, 4] = np.nan
    with pytest.raises(qb.QBError) as e:
        f(torch.tensor(A, device="cuda"), 0.1, 8, seed=1)
    assert e.value.code == -2


def test_indicator_matches_direct_residual():
    A = synth.dense_from_spectrum(400, 300, synth.sigma_exp(300, 30.0), seed=4)
    for f in (qb.qb_ei_dense, qb.qb_fp_dense):
        Q, B, info = f(torch.tensor(A, device="cuda"), 1e-5, 16, P=1, seed=2)
        direct = np.linalg.norm(A - _qb(Q, B)) ** 2
        assert abs(info.err2_est - direct) <= 1e-12 * info.normA2
        Qh = Q.cpu().numpy()
        assert oracle.orth_loss(Qh) <= 1e-12


# ----------------------------------------------------------------------------- FP chunks vs whole batch
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_fp_chunked_matches_whole_batch(prec):
    """The default randQB_FP forms the Omega batch in 512-column chunks as the loop reaches them;
    orth is column-causal, so Q, B must equal the whole-batch evaluation (QB_FLAG_WHOLE_BATCH,
    Algorithm 4 as written) up to rounding, and (float64) the oracle's."""
    m, n, b = 2000, 1500, 32
    sigma = synth.sigma_exp(1500, 150.0, 1e-6)
    A = synth.dense_from_spectrum(m, n, sigma, seed=404)
    tol = 1e-2
    Ad = torch.tensor(A, device="cuda")
    kw = dict(P=1, seed=21)
    if prec == "mixed":
        hi, lo, norms = qb.quantize_bf16x2(Ad)
        args = (hi, tol, b)
        kw.update(prec="mixed", a_lo=lo, src_norm2=norms[0])
    else:
        args = (Ad, tol, b)
    Qc, Bc, ic = qb.qb_fp_dense(*args, **kw)
    Qw, Bw, iw = qb.qb_fp_dense(*args, flags=4, **kw)     # QB_FLAG_WHOLE_BATCH
    assert ic.rank > 512            # the loop crossed at least one chunk boundary
    assert ic.converged and iw.converged
    assert ic.omega_cols < iw.omega_cols == min(50 * b, n)
    # reads of A (Table 1's unit, with G and H as two reads): 2 + 2P per 512-column chunk formed;
    # the whole batch takes 1 + 2P for the power scheme and G, plus one per 512-column piece of H
    # formed as the loop reaches it
    assert ic.passes == (2 + 2 * 1) * -(-ic.omega_cols // 512)
    assert iw.passes == (1 + 2 * 1) + -(-(iw.blocks * b) // 512)
    nA = np.linalg.norm(A)
    if prec == "fp64":
        assert ic.rank == iw.rank
        diff = np.linalg.norm(_qb(Qc, Bc) - _qb(Qw, Bw)) / nA
        sp, ref = spread(A, "fp", tol, b, perms=2, seed=21, P=1)
        assert diff <= parity_bound(sp), (diff, sp)
        assert ic.rank == ref.rank
        _check_parity(A, (Qc, Bc, ic), ref, tol, "fp chunked", parity_bound(sp))
    else:
        assert abs(ic.rank - iw.rank) <= 2
        for Q, B in ((Qc, Bc), (Qw, Bw)):
            assert np.linalg.norm(A - _qb(Q, B)) / nA < tol


# ----------------------------------------------------------------------------- mixed precision
U32 = 2.0 ** -24


def _bf16(X):
    """float64 -> bfloat16 (round to nearest even) -> float64, test-side."""
    u = np.ascontiguousarray(X, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _check_mixed_rank(A, hi, tol, b, seed, P, alg, rank):
    """The mixed path's rank against the float64 oracle run on the mixed path's representation:
    sketches of the bf16 A_hi the kernels stream (B_i and H from A itself), the bf16-rounded
    float32 Omega the kernels draw, and the stop test's margin E < eps^2 - 2 u_32 ||A||^2 written
    as a tolerance.  What is left between the two is float32 Q, B and the GPU's operand roundings
    (2^-17 of each term): 2% of the rank, or 4, covers it."""
    n = A.shape[1]
    f = oracle.randqb_ei if alg == "ei" else oracle.randqb_fp
    om = lambda c0, w: _bf16(oracle.omega_f32(n, c0, w, seed).astype(np.float64))  # noqa: E731
    emu = f(A, float(np.sqrt(tol ** 2 - 2 * U32)), b, seed=seed, P=P,
            A_sketch=hi.double().cpu().numpy(), omega_fn=om)
    assert abs(rank - emu.rank) <= max(4, 0.02 * emu.rank), (alg, rank, emu.rank)

@pytest.fixture(scope="module")
def A_mixed():
    return synth.dense_from_spectrum(3000, 2000, synth.sigma_exp(2000, 60.0, 1e-6), seed=7)


@pytest.mark.parametrize("alg", ["ei", "fp"])
def test_mixed_reaches_tolerance(A_mixed, alg):
    A = A_mixed
    tol = 1e-3
    Ad = torch.tensor(A, device="cuda")
    hi, lo, norms = qb.quantize_bf16x2(Ad)
    assert abs(norms[0] - oracle.frob2(A)) <= 1e-12 * norms[0]
    assert norms[1] <= 1e-9 * norms[0]
    f = qb.qb_ei_dense if alg == "ei" else qb.qb_fp_dense
    Q, B, info = f(hi, tol, 32, P=1, seed=11, a_lo=lo, src_norm2=norms[0], prec="mixed")
    # converged; tol 1e-3 is below the Theorem 3 floor for float32 B (4.9e-3), hence status 2
    assert info.status == 2 and info.converged
    err = np.linalg.norm(A - _qb(Q, B)) / np.linalg.norm(A)
    assert err < tol
    ref = (oracle.randqb_ei if alg == "ei" else oracle.randqb_fp)(A, tol, 32, seed=11, P=1)
    # the mixed path never stops below the float64 oracle's rank; its excess (461 against 420 on
    # this spectrum) comes from its representation, which the oracle reproduces in float64
    assert info.rank >= ref.rank - 2
    _check_mixed_rank(A, hi, tol, 32, 11, 1, alg, info.rank)
    # the indicator tracks the true error (Theorem 1) within Theorem 3's bound for float32 B
    assert abs(info.err2_est - (err ** 2) * info.normA2) <= 4 * 2.0 ** -24 * info.normA2


def test_quantize_bf16x2_split():
    A = np.random.default_rng(0).standard_normal((300, 257))
    Ad = torch.tensor(A, device="cuda")
    hi, lo, norms = qb.quantize_bf16x2(Ad)
    rec = hi.double() + lo.double()
    rel = np.abs(rec.cpu().numpy() - A) / np.abs(A)
    assert rel.max() <= 2.0 ** -16
    assert abs(norms[0] - np.sum(A * A)) <= 1e-12 * norms[0]
    assert abs(norms[2] - np.sum((A - hi.double().cpu().numpy()) ** 2)) <= 1e-9 * norms[2]


@pytest.fixture(scope="module")
def A_tall():
    return synth.dense_from_spectrum(70000, 1024, synth.sigma_exp(1024, 20.0, 1e-6), seed=19)


@pytest.mark.parametrize("alg", ["ei", "fp"])
def test_mixed_tall_panels(A_tall, alg):
    """m = 70000 rows: the fused CholeskyQR slices (461 rows per CTA) exceed the rows a CTA holds
    in shared memory, so each phase streams them in tiles.  Same bar as the resident case:
    converged, true error below tol, rank close to the float64 oracle's (140), Q orthonormal to
    float32 accuracy, and the indicator within Theorem 3's float32 bound of the true error.

    n = 1024 keeps the rank small against n: the sketches read bf16 A_hi, and every captured
    direction is rotated by the quantisation error D = A - A_hi, leaving about ||D||_2^2 of energy
    behind, k ||D||_2^2 ~ (u_bf16^2 / 3)(k / n)(1 + sqrt(n / m))^2 ||A||^2 in all; at n = 256 and
    k ~ 140 that floor (1.7e-6 ||A||^2) is above tol^2 and the mixed path cannot converge."""
    A = A_tall
    tol = 1e-3
    Ad = torch.tensor(A, device="cuda")
    hi, lo, norms = qb.quantize_bf16x2(Ad)
    del Ad
    f = qb.qb_ei_dense if alg == "ei" else qb.qb_fp_dense
    Q, B, info = f(hi, tol, 32, P=1, seed=4, a_lo=lo, src_norm2=norms[0], prec="mixed")
    assert info.converged
    err = np.linalg.norm(A - _qb(Q, B)) / np.linalg.norm(A)
    assert err < tol
    ref = (oracle.randqb_ei if alg == "ei" else oracle.randqb_fp)(A, tol, 32, seed=4, P=1)
    assert info.rank >= ref.rank - 2
    _check_mixed_rank(A, hi, tol, 32, 4, 1, alg, info.rank)
    Qd = Q.double()
    orth = (Qd.T @ Qd - torch.eye(info.rank, dtype=torch.float64, device="cuda")).abs().max().item()
    assert orth <= 1e-4
    assert abs(info.err2_est - (err ** 2) * info.normA2) <= 4 * 2.0 ** -24 * info.normA2


@pytest.mark.parametrize("alg", ["ei", "fp"])
def test_a_lo_ready_event(A_mixed, alg):
    """A_lo still arriving when the call starts: a second stream first spins (~20 ms of device
    clock cycles) and only then copies A_lo from the host, recording the event the call receives.
    The call must wait for it before its first read of A_lo: Q, B and the rank are bit-identical
    to the call on a fully resident A_lo (a missed wait would read the zeros A_lo starts from)."""
    A = torch.tensor(A_mixed, device="cuda")
    hi, lo, norms = qb.quantize_bf16x2(A)
    del A
    f = qb.qb_ei_dense if alg == "ei" else qb.qb_fp_dense
    Q0, B0, i0 = f(hi, 1e-3, 32, P=1, seed=21, a_lo=lo, src_norm2=norms[0], prec="mixed")
    Q0, B0 = Q0.clone(), B0.clone()
    lo_h = lo.cpu().pin_memory()
    lo_d = torch.zeros_like(lo)
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    ready = torch.cuda.Event()
    with torch.cuda.stream(side):
        torch.cuda._sleep(40_000_000)
        lo_d.copy_(lo_h, non_blocking=True)
        ready.record(side)
    Q1, B1, i1 = f(hi, 1e-3, 32, P=1, seed=21, a_lo=lo_d, src_norm2=norms[0], prec="mixed",
                   a_lo_ready=ready)
    torch.cuda.synchronize()
    assert i1.rank == i0.rank and i1.status == i0.status
    assert torch.equal(Q1, Q0) and torch.equal(B1, B0)


@pytest.mark.parametrize("alg", ["ei", "fp"])
def test_mixed_ill_conditioned_blocks(alg):
    """sigma_j = exp(-j / 10): inside one 64-column block the singular values fall by
    e^6.4 ~ 600, so both Q_i panels (rank ~70: the first block, and the second, which gets one
    CholeskyQR pass before its re-orthogonalisation) reach kappa above the float32 factor's
    weak-pivot limit (~100) and go through the float64 refactor of the fused CholeskyQR.  The
    result must still meet the tolerance, with a rank close to the float64 oracle's and Q
    orthonormal to float32 accuracy."""
    A = synth.dense_from_spectrum(4000, 3000, synth.sigma_exp(3000, 10.0, 1e-9), seed=33)
    tol = 1e-3
    Ad = torch.tensor(A, device="cuda")
    hi, lo, norms = qb.quantize_bf16x2(Ad)
    del Ad
    f = qb.qb_ei_dense if alg == "ei" else qb.qb_fp_dense
    Q, B, info = f(hi, tol, 64, P=1, seed=5, a_lo=lo, src_norm2=norms[0], prec="mixed")
    assert info.converged
    err = np.linalg.norm(A - _qb(Q, B)) / np.linalg.norm(A)
    assert err < tol, err
    ref = (oracle.randqb_ei if alg == "ei" else oracle.randqb_fp)(A, tol, 64, seed=5, P=1)
    assert ref.rank - 2 <= info.rank <= ref.rank + max(4, 0.05 * ref.rank), (info.rank, ref.rank)
    Qd = Q.double()
    orth = float(torch.linalg.norm(Qd.T @ Qd - torch.eye(Q.shape[1], device=Q.device, dtype=torch.float64)))
    assert orth < 1e-4, orth
