"""The allocation-free sketch entry point (qb_apass_sketch_noalloc) against the workspace entry
point (qb_apass_sketch), through the C ABI.

Some callers cannot allocate device memory or hand the library a workspace (for example a
process whose device memory is already carved up by its own pool).  The no-alloc variant keeps
its scratch in a fixed device array inside the library; this file checks that two calls in a row
(different shapes, so stale contents of the shared array would show) give the same result as the
ordinary entry point, and that calls beyond the array's size limit are refused.  It is collected
last so a failure here leaves every other test already run."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)


def _call_noalloc(lib, qb, A, V):
    m, n = A.shape
    w = V.shape[1]
    d = qb._dense_desc(A)
    Vt = V.T.contiguous()                      # V column-major n x w
    Yt = torch.full((w, m), float("nan"), dtype=torch.float32, device=A.device)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.qb_apass_sketch_noalloc(C.byref(d), C.c_void_p(Vt.data_ptr()), n, w,
                                     C.c_void_p(Yt.data_ptr()), m, stream)
    return rc, Yt.T


def test_noalloc_sketch_matches_workspace_entry_point():
    from paper_1606_09402_gb300 import _lib, build
    build.build()
    lib = _lib.load()
    import paper_1606_09402_gb300 as qb

    rng = np.random.default_rng(7)
    for m, n, w in [(3000, 2048, 64), (1500, 784, 40)]:
        A = torch.tensor(rng.standard_normal((m, n)), dtype=torch.float32).to(torch.bfloat16).cuda()
        V = torch.tensor(rng.standard_normal((n, w)), dtype=torch.float32).cuda()
        ref = qb.qb_apass_sketch(A, V).double().cpu().numpy()
        rc, Y = _call_noalloc(lib, qb, A, V)
        assert rc == 0, lib.qb_status_str(rc)
        Y = Y.double().cpu().numpy()
        scale = (np.abs(A.double().cpu().numpy()) @
                 np.abs(V.to(torch.bfloat16).double().cpu().numpy())) + 1e-30
        assert np.max(np.abs(Y - ref) / scale) < 1e-5


def test_noalloc_rejects_sizes_beyond_its_array():
    from paper_1606_09402_gb300 import _lib
    lib = _lib.load()
    import paper_1606_09402_gb300 as qb
    A = torch.zeros(256, 256, dtype=torch.bfloat16, device="cuda")
    V = torch.zeros(256, 65, dtype=torch.float32, device="cuda")
    rc, _ = _call_noalloc(lib, qb, A, V)
    assert rc == -5   # QB_ERR_WORKSPACE: w above the fixed array's limit


def test_noalloc_size_limit_boundary():
    """Both sides of the array's size limit at w = 64: n = 49144 is the largest width whose bf16
    copy of V (align8(n) * 64 * 2 bytes) fits beside the 10 MiB + 256 bytes of partial tiles and
    flag in the 16 MiB array, and it runs and matches the workspace entry point; n = 49152 (the
    next multiple of 8) is refused before any launch."""
    from paper_1606_09402_gb300 import _lib
    lib = _lib.load()
    import paper_1606_09402_gb300 as qb

    rng = np.random.default_rng(11)
    m, w = 128, 64
    for n, ok in [(49144, True), (49152, False)]:
        A = torch.tensor(rng.standard_normal((m, n)), dtype=torch.float32).to(torch.bfloat16).cuda()
        V = torch.tensor(rng.standard_normal((n, w)), dtype=torch.float32).cuda()
        rc, Y = _call_noalloc(lib, qb, A, V)
        if not ok:
            assert rc == -5, (n, rc)   # QB_ERR_WORKSPACE
            continue
        assert rc == 0, (n, lib.qb_status_str(rc))
        ref = qb.qb_apass_sketch(A, V).double().cpu().numpy()
        scale = (np.abs(A.double().cpu().numpy()) @
                 np.abs(V.to(torch.bfloat16).double().cpu().numpy())) + 1e-30
        assert np.max(np.abs(Y.double().cpu().numpy() - ref) / scale) < 1e-5
