"""The tensor-core passes over dense A (tcgen05 + TMA), through the C ABI, against float64
products computed on the CPU.  Covers the stream-K schedule (one column tile), the raster
schedule (many units), the hybrid schedule (whole raster waves, then the k-blocks of the
remaining units split across all CTAs), ragged tails in every dimension, and the hi/lo passes."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1606_09402_gb300 as qb  # noqa: E402


def _bf16(x):
    return torch.tensor(x, dtype=torch.float32).to(torch.bfloat16)


def _rel_err(got, ref, scale):
    return float(np.max(np.abs(got - ref) / scale))


@pytest.mark.parametrize("m,n,w", [
    (1000, 776, 64),     # stream-K, ragged m
    (777, 1000, 20),     # w below one column tile
    (4099, 2048, 200),   # two column tiles, ragged
    (16384, 1024, 2560), # raster schedule (>= 8 units per SM)
    (300, 136, 1),       # single column
])
def test_sketch_bf16(m, n, w):
    rng = np.random.default_rng(m + n + w)
    A = rng.standard_normal((m, n)).astype(np.float32)
    V = rng.standard_normal((n, w)).astype(np.float32)
    Ad = _bf16(A).cuda()
    Y = qb.qb_apass_sketch(Ad, torch.tensor(V).cuda()).cpu().numpy().astype(np.float64)
    Ah = Ad.double().cpu().numpy()
    Vh = _bf16(V).double().numpy()              # the kernel rounds V to bf16
    ref = Ah @ Vh
    scale = np.abs(Ah) @ np.abs(Vh) + 1e-30
    assert _rel_err(Y, ref, scale) < 1e-5


@pytest.mark.parametrize("m,n,w,precise", [
    (2000, 1000, 64, True),
    (2000, 1000, 64, False),
    (2000, 1000, 64, 2),
    (1024, 8192, 1000, 2),
    (1500, 777 + 7, 33, True),     # ragged n (multiple of 8 for TMA rows), ragged w
    (1024, 16384, 2560, True),     # raster schedule
    (40000, 256, 64, True),        # long reduction split across many CTAs
])
def test_trans_bf16(m, n, w, precise):
    rng = np.random.default_rng(m * 3 + n + w)
    A = rng.standard_normal((m, n))
    V = rng.standard_normal((m, w)).astype(np.float32)
    Ad = torch.tensor(A).cuda()
    hi, lo, _ = qb.quantize_bf16x2(Ad)
    Z = qb.qb_apass_trans(hi, torch.tensor(V).cuda(), precise=int(precise), a_lo=lo)
    Z = Z.cpu().numpy().astype(np.float64)
    Vd = V.astype(np.float64)
    if precise:
        # (A_hi + A_lo)^T V: exact float32 V (precise 1) or bf16(V) (precise 2)
        Ahl = hi.double().cpu().numpy() + lo.double().cpu().numpy()
        if precise == 2:
            Vd = _bf16(V).double().numpy()
        ref = Ahl.T @ Vd
        scale = np.abs(Ahl.T) @ np.abs(Vd) + 1e-30
        assert _rel_err(Z, ref, scale) < 1e-5
        if precise is True:
            assert np.linalg.norm(Z - A.T @ Vd) / np.linalg.norm(A.T @ Vd) < 1e-5
    else:
        Ah = hi.double().cpu().numpy()
        ref = Ah.T @ _bf16(V).double().numpy()
        scale = np.abs(Ah.T) @ np.abs(_bf16(V).double().numpy()) + 1e-30
        assert _rel_err(Z, ref, scale) < 1e-5


@pytest.mark.parametrize("kind", ["sketch", "trans_two_term"])
def test_hybrid_schedule(kind):
    """Shapes whose last raster wave is partial, which the hybrid schedule splits: a sketch of
    20000 rows at w = 512 (157 x 2 units of 128 x 256 on 152 CTAs) and the transposed pass of
    randQB_FP's H chunk at 20000 output rows, w = 512, G held as two-term bf16 values (157 x 4
    units of 128 x 128: the pattern of the 40000 x 20000 step)."""
    rng = np.random.default_rng(17 if kind == "sketch" else 18)
    if kind == "sketch":
        m, n, w = 20000, 4096, 512
        A = rng.standard_normal((m, n)).astype(np.float32)
        V = rng.standard_normal((n, w)).astype(np.float32)
        Ad = _bf16(A).cuda()
        Y = qb.qb_apass_sketch(Ad, torch.tensor(V).cuda()).cpu().numpy().astype(np.float64)
        Ah = Ad.double().cpu().numpy()
        Vh = _bf16(V).double().numpy()
        ref = Ah @ Vh
        scale = np.abs(Ah) @ np.abs(Vh) + 1e-30
        assert _rel_err(Y, ref, scale) < 1e-5
    else:
        m, n, w = 4096, 20000, 512
        A = rng.standard_normal((m, n))
        Vt = torch.tensor(rng.standard_normal((m, w)).astype(np.float32))
        v_hi = Vt.to(torch.bfloat16).float()
        V2 = v_hi + (Vt - v_hi).to(torch.bfloat16).float()     # 16 significant bits
        hi, lo, _ = qb.quantize_bf16x2(torch.tensor(A).cuda())
        Z = qb.qb_apass_trans(hi, V2.cuda(), precise=3, a_lo=lo).cpu().numpy().astype(np.float64)
        Ahl = hi.double().cpu().numpy() + lo.double().cpu().numpy()
        Vd = V2.double().numpy()
        ref = Ahl.T @ Vd
        scale = np.abs(Ahl.T) @ np.abs(Vd) + 1e-30
        assert _rel_err(Z, ref, scale) < 1e-5


def test_fp64_apass_matches_numpy():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((333, 211))
    V = rng.standard_normal((211, 17))
    W = rng.standard_normal((333, 9))
    Ad = torch.tensor(A).cuda()
    Y = qb.qb_apass_sketch(Ad, torch.tensor(V).cuda()).cpu().numpy()
    Z = qb.qb_apass_trans(Ad, torch.tensor(W).cuda()).cpu().numpy()
    np.testing.assert_allclose(Y, A @ V, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(Z, A.T @ W, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("precise", [0, 1])
def test_long_reduction_has_no_drift(precise):
    """Positive data over a 40000-long reduction: the mean signed relative error must stay at
    rounding level.  (A single tensor-core accumulation chain of that length drifts toward zero by
    about -3.4e-6; the kernels flush short chains into registers.)"""
    rng = np.random.default_rng(1)
    m, n, w = 40000, 512, 64
    a = (np.abs(rng.standard_normal((m, n))) + 0.5).astype(np.float32)
    v = (np.abs(rng.standard_normal((m, w))) + 0.5).astype(np.float32)
    A = _bf16(a).cuda()
    Vb = _bf16(v).float().cuda()
    lo = torch.zeros_like(A) if precise else None
    Z = qb.qb_apass_trans(A, Vb, precise=precise, a_lo=lo).double().cpu().numpy()
    ref = A.double().cpu().numpy().T @ Vb.double().cpu().numpy()
    r = (Z - ref) / ref
    assert abs(r.mean()) < 1e-7, r.mean()
    Y = qb.qb_apass_sketch(A.T.contiguous(), Vb).double().cpu().numpy()
    r = (Y - ref) / ref
    assert abs(r.mean()) < 1e-7, r.mean()
