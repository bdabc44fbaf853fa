"""Benchmark: time-to-tolerance of mixed-precision randQB_FP on one GB300, next to the float64
randQB_FP path, the narrow A-pass bandwidth and the float64 CPU oracle.

Workload (one "step" = one complete fixed-precision factorisation, inputs resident in HBM):
  A = U diag(sigma) V^T, 40000 x 20000, sigma_j = exp(-j/200) + 1e-6 (j <= 4096; the omitted
  tail carries 1.6e-8 of the energy of ||A||^2 = 99.5, far below eps^2 = 1e-6 ||A||^2), U, V from
  the QR of seeded N(0,1) matrices; b = 64, P = 1, relative tolerance 1e-3, Omega seed 9402,
  l~ = 50 b = 3200.  Mixed path: A stored as bf16 hi + lo (quantised once from float64, not
  timed), BF16 tensor-core passes, float32 Q/B, float64 indicator, adaptive b x b Cholesky.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--no-fp64] [--quick]
N > 1 runs N independent replicas (the factorisation of one matrix does not shard across GPUs
here), one per rank under torchrun.  Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "time-to-tolerance (s) and A-pass HBM GB/s, mixed-precision vs FP64 randQB_FP"
M, N = 40000, 20000
RANK_SPECTRUM = 4096
TOL, B, P, SEED_A, SEED_OMEGA = 1e-3, 64, 1, 1606, 9402
L_TILDE = 50 * B
RANK_CAP = 4096
# DRAM bytes of one k_tc_prec<128, true, 2, 2> launch (w = 512) at 40000 x 20000: ncu
# (dram__bytes_read.sum + dram__bytes_write.sum, one pass) on the first H chunk of one mixed
# randQB_FP step, 4.23 GB + 44.4 MB, against 3.32 GB algorithmic (A hi + lo 3.2 GB, G's two bf16
# terms 82 MB, H 41 MB): the 20 units the hybrid schedule splits read A without L2 sharing.
PREC_TRAFFIC_BYTES = 4.274e9
PREC_TRAFFIC_NOTE = ("ncu dram bytes (one pass) of the first k_tc_prec<128,1,2,2> launch of a "
                     "40000x20000 step: 4.23 GB read + 44.4 MB written; algorithmic 3.32 GB")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the float64 comparison run")
    ap.add_argument("--quick", action="store_true", help="smaller workload (smoke only)")
    ap.add_argument("--steps-only", action="store_true",
                    help="time the mixed randQB_FP steps only (no side measurements); for profiling")
    ap.add_argument("--profile-small", nargs="?", const="fp", default=None,
                    choices=["fp", "ei", "csr", "coo", "batched", "adjoint", "adjoint8192", "svd"],
                    help="small cases for ncu section captures: two mixed randQB_FP (fp) or "
                         "randQB_EI (ei) factorisations of a 16384 x 8192 matrix; the sparse "
                         "passes on a 50000 x 25000 Zipf CSR / COO matrix (csr, coo); a batch of "
                         "32 matrices (batched); the 4096 x 4096 fixed-rank map and adjoint "
                         "(adjoint; adjoint8192 at the benchmark's 8192 x 8192 for one-pass "
                         "launch lists); the SVD from a rank-1024 QB (svd)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class Clocks:
    """nvidia-smi sampler for the timed region (SM clock, throttle reasons)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- inputs
def make_inputs(torch, dev, quick):
    import synth
    m, n = (4000, 2000) if quick else (M, N)
    r = min(RANK_SPECTRUM, n)
    sigma = synth.sigma_exp(r, 200.0, 1e-6)
    A64 = synth.dense_from_spectrum_torch(m, n, sigma, SEED_A, dev, dtype=torch.float64)
    return A64, sigma


def timed(torch, fn, steps, warmup, ws, stream):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        fn()
    ev1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    return ev0.elapsed_time(ev1) / 1e3 / steps


def event_time(torch, fn, reps, stream):
    """Average device time of fn() over reps launches, CUDA events on the launching stream."""
    fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3 / reps


def pass_time(torch, qb, fn, reps, phase):
    """Average device time of one pass over A: the library records CUDA events on the launching
    stream around each single-pass call's work (the operand split, the tensor-core kernel, the
    stream-K fix-up) and reports them through profile_last(); the binding's own transposes and
    each call's host round trip fall outside."""
    fn()
    torch.cuda.synchronize()
    total = 0.0
    for _ in range(reps):
        fn()
        total += qb.profile_last()[phase]
    return total / 1e3 / reps


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), or "" if neither says."""
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return ""


def oracle_cores():
    """Threads the oracle's BLAS actually uses (threadpoolctl when present, else the CPU count)."""
    cores = os.cpu_count()
    try:
        from threadpoolctl import threadpool_info
        cores = max((i.get("num_threads") or 0) for i in threadpool_info()) or cores
    except Exception:
        pass
    return cores


def cpu_baseline(A_host):
    """The float64 oracle's randQB_FP on the whole workload, one run, timed on the host cores.

    No sample is scaled: the oracle's cost is dominated by the n x n product B^T B of the B_i
    formula in every block (Sect. 4.2), which does not shrink with a row sample (measured: 111 s at
    4000 rows, 114 s at 8000 rows, 175 s at all 40000 rows on 8 x86 cores)."""
    import numpy as np

    import oracle
    As = np.ascontiguousarray(A_host)
    t0 = time.perf_counter()
    r = oracle.randqb_fp(As, TOL, B, seed=SEED_OMEGA, P=P, l_tilde=L_TILDE, rank_cap=RANK_CAP)
    t = time.perf_counter() - t0
    m, n = As.shape
    return {"value": t, "unit": "s", "cores": oracle_cores(), "kind": "oracle", "cpu": cpu_model(),
            "sample": f"the whole {m}x{n} workload, one oracle randQB_FP run (float64 "
                      f"numpy/LAPACK), rank {r.rank}, measured, not scaled"}


def run_batched(torch, qb, dev, stream):
    """The batched workload: 256 float32 matrices (seed 1606), b = 16, P = 0; one call factorises
    all of them (conditional CUDA graph).  Spectra are truncated at j <= 512 (the tail beyond
    carries < 3e-9 of ||A||^2)."""
    import numpy as np

    import synth
    specs = synth.batched_specs(256, 1606)
    mats = []
    for s in specs:
        r = min(s.m, s.n, 512)
        mats.append(synth.dense_from_spectrum_torch(s.m, s.n, synth.sigma_pow(r, 2.0, s.scale),
                                                    s.seed, dev, dtype=torch.float32))
    tols = [s.tol for s in specs]
    outs = [(torch.empty(min(s.m, s.n), s.m, device=dev), torch.empty(min(s.m, s.n), s.n, device=dev))
            for s in specs]
    import ctypes as C
    from paper_1606_09402_gb300 import _lib
    lib = _lib.load()
    descs = (_lib.qb_dense * len(mats))(*[qb._dense_desc(A) for A in mats])
    o = qb._opts(0.0, 16, 0, 9402, True, None, None, True, "mixed")
    ws = torch.empty(lib.qb_ei_batched_workspace(len(mats), descs, C.byref(o)), dtype=torch.uint8,
                     device=dev)
    # warm-up: the first call tunes the A-streaming stages for this batch shape and captures the
    # iteration graph; the timed calls reuse both
    res = qb.qb_ei_batched(mats, tols, seed=9402, outs=outs, workspace=ws)
    plan_first = qb.batched_last_plan()
    torch.cuda.synchronize()
    times = []
    for _ in range(3):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = qb.qb_ei_batched(mats, tols, seed=9402, outs=outs, workspace=ws)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    plan = qb.batched_last_plan()
    ranks = [r[2].rank for r in res]
    ok = sum(1 for r in res if r[2].converged)
    a_bytes = sum(4.0 * s.m * s.n for s in specs)
    # true error of every result (float64, verification only)
    worst = 0.0
    for t in range(len(specs)):
        A = mats[t].double()
        Q, B, _ = res[t]
        worst = max(worst, float(torch.linalg.norm(A - Q.double() @ B.double()) / torch.linalg.norm(A)) / tols[t])
    # bytes of A the A-streaming stages read: each block of matrix t reads A_t twice
    a_read = sum(2.0 * 4.0 * s.m * s.n * r[2].blocks for s, r in zip(specs, res))
    t_med = statistics.median(times)
    pk, _ = peaks()
    return {"matrices": len(specs), "time_s": t_med, "converged": ok,
            "rank_min": int(min(ranks)), "rank_max": int(max(ranks)),
            "blocks_total": int(sum(r[2].blocks for r in res)),
            "a_bytes_per_sweep": a_bytes, "a_bytes_read": a_read,
            "a_read_gbs": a_read / t_med / 1e9, "a_read_frac_of_hbm": a_read / t_med / 1e9 / pk["hbm_gbs"],
            "worst_err_over_tol": worst, "plan": plan, "plan_first_call": plan_first,
            "note": "one graph launch per call; the timed calls reuse the graph and the tuned plan"}


def run_sparse(torch, qb, dev, stream):
    """The sparse workload: CSR 200000 x 100000, Poisson(100) row lengths, Zipf(1.1) columns,
    log-normal float32 values (seed 909), b = 32, P = 1, relative tol 0.5, rank cap 1024;
    randQB_EI and randQB_FP time-to-tolerance, and the A-pass bandwidth of EI from its phase
    times (the CSR passes run in the sketch and transposed phases)."""
    import numpy as np

    import synth
    csr = synth.csr_zipf(200000, 100000, 100.0, 1.1, seed=909, val_dtype=np.float32)
    rp = torch.tensor(csr.rowptr, device=dev)
    ci = torch.tensor(csr.colind, device=dev)
    v = torch.tensor(csr.val, device=dev)
    shape = (csr.m, csr.n)
    kw = dict(P=1, seed=9402, rank_cap=1024)
    out = {"m": csr.m, "n": csr.n, "nnz": int(ci.numel()), "b": 32, "P": 1, "tol": 0.5}
    for name, f in (("ei", qb.qb_ei_csr), ("fp", qb.qb_fp_csr)):
        f(rp, ci, v, shape, 0.5, 32, **kw)                   # warm-up
        torch.cuda.synchronize()
        t = event_time(torch, lambda: f(rp, ci, v, shape, 0.5, 32, **kw), 3, stream)
        _, _, info = f(rp, ci, v, shape, 0.5, 32, flags=2, **kw)
        ph = qb.profile_last()
        out[name] = {"time_to_tol_s": t, "rank": info.rank, "passes": info.passes,
                     "status": info.status, "err_rel_est": info.err_est / info.normA2 ** 0.5,
                     "pass_ms": ph["sketch"] + ph["trans"]}
    a_bytes = 8.0 * out["nnz"] + 4.0 * (csr.m + 1)
    ei = out["ei"]
    out["a_bytes_per_pass"] = a_bytes
    out["ei_pass_gbs"] = ei["passes"] * a_bytes / (ei["pass_ms"] * 1e-3) / 1e9
    # the same matrix as COO triplets sorted by row (Sect. 5.1's coordinate format)
    lens = np.diff(csr.rowptr.astype(np.int64))
    row = torch.tensor(np.repeat(np.arange(csr.m, dtype=np.int32), lens), device=dev)
    for name, f in (("coo_ei", qb.qb_ei_coo), ("coo_fp", qb.qb_fp_coo)):
        f(row, ci, v, shape, 0.5, 32, **kw)                   # warm-up
        torch.cuda.synchronize()
        t = event_time(torch, lambda: f(row, ci, v, shape, 0.5, 32, **kw), 3, stream)
        _, _, info = f(row, ci, v, shape, 0.5, 32, flags=2, **kw)
        ph = qb.profile_last()
        out[name] = {"time_to_tol_s": t, "rank": info.rank, "passes": info.passes,
                     "status": info.status, "pass_ms": ph["sketch"] + ph["trans"]}
    out["coo_ei"]["pass_gbs"] = (out["coo_ei"]["passes"] * (12.0 * out["nnz"]) /
                                 (out["coo_ei"]["pass_ms"] * 1e-3) / 1e9)
    del row
    # the merged-duplicates reading of the generator: converges at tol 0.5 well under the cap
    mc = synth.csr_zipf(200000, 100000, 100.0, 1.1, seed=909, val_dtype=np.float32,
                        merge_duplicates=True)
    rpm = torch.tensor(mc.rowptr, device=dev)
    cim = torch.tensor(mc.colind, device=dev)
    vm = torch.tensor(mc.val, device=dev)
    merged = {"nnz": int(cim.numel()), "note": "duplicate Zipf draws merged (summed values)"}
    for name, f in (("ei", qb.qb_ei_csr), ("fp", qb.qb_fp_csr)):
        f(rpm, cim, vm, shape, 0.5, 32, **kw)
        torch.cuda.synchronize()
        t = event_time(torch, lambda: f(rpm, cim, vm, shape, 0.5, 32, **kw), 3, stream)
        _, _, info = f(rpm, cim, vm, shape, 0.5, 32, **kw)
        merged[name] = {"time_to_tol_s": t, "rank": info.rank, "passes": info.passes,
                        "status": info.status, "err_rel_est": info.err_est / info.normA2 ** 0.5}
    out["merged_duplicates"] = merged
    return out


def run_adjoint(torch, qb, dev, stream):
    """Fixed-rank k = 256 QB of an 8192 x 8192 bf16 A (sigma_j = 1/j): forward and backward."""
    import numpy as np

    import synth
    m = n = 8192
    k = 256
    A = synth.dense_from_spectrum_torch(m, n, 1.0 / np.arange(1, n + 1), 1606, dev,
                                        dtype=torch.float32).to(torch.bfloat16)
    GQ, GB = synth.cotangents(m, n, k, seed=5)
    GQ = torch.tensor(GQ, dtype=torch.float32, device=dev)
    GB = torch.tensor(GB, dtype=torch.float32, device=dev)
    Q, B, R = qb.qb_fixed_rank_fwd(A, k, 9)
    qb.qb_fixed_rank_bwd(A, k, 9, Q, R, GQ, GB)
    tf = event_time(torch, lambda: qb.qb_fixed_rank_fwd(A, k, 9), 3, stream)
    tb = event_time(torch, lambda: qb.qb_fixed_rank_bwd(A, k, 9, Q, R, GQ, GB), 3, stream)
    # algorithmic work: the forward is two passes over A (Y = A Omega, B = Q^T A), 4 m n k flops
    # and 2 m n bf16 bytes each; the backward is A G_B^T and the K = 2k product for Abar
    # (6 m n k flops), reading A once and writing the float32 Abar
    pk, src = peaks()
    fl_f, by_f = 4.0 * m * n * k, 2.0 * m * n * 2
    fl_b, by_b = 6.0 * m * n * k, m * n * 2.0 + m * n * 4.0
    frac = lambda fl, by, t: {"tflops": fl / t / 1e12, "gbs": by / t / 1e9,
                              "tensor_frac": fl / t / 1e12 / pk["bf16_tflops"],
                              "hbm_frac": by / t / 1e9 / pk["hbm_gbs"]}
    return {"m": m, "n": n, "k": k, "forward_s": tf, "backward_s": tb,
            "forward": frac(fl_f, by_f, tf), "backward": frac(fl_b, by_b, tb),
            "peak_source": src + " (burst bf16, copy bandwidth)"}


def run_paper_dense(torch, qb, dev, stream):
    """The paper's dense runtime experiment (Sect. 5.1, Fig. 3): n x n with n = 32000, l = 200
    columns, b = 20, P = 0 and 1.  The paper notes that the spectrum is immaterial for this
    comparison; A = U diag(1/j) V^T with j <= 512 (U, V from seeded Gaussian QR).  Fixed rank: tol
    0 and a rank cap of 200, so every run forms exactly 200 columns (status QB_NOT_CONVERGED).
    Float64 path on the float64 A, mixed path on its bf16 hi + lo split.  The paper's times
    (2 x 12-core Xeon E5-2630, MKL, float64, P = 0): randQB_FP 8.01 s, randQB_EI 13.47 s."""
    import numpy as np

    import synth
    n = 32000
    A64 = synth.dense_from_spectrum_torch(n, n, 1.0 / np.arange(1, 513), 3200, dev,
                                          dtype=torch.float64)
    hi, lo, norms = qb.quantize_bf16x2(A64)
    out = {"n": n, "l": 200, "b": 20,
           "paper_s": {"fp_P0": 8.01, "ei_P0": 13.47,
                       "hardware": "2 x 12-core Intel Xeon E5-2630 @ 2.30 GHz, MKL, float64"}}
    for prec in ("fp64", "mixed"):
        for alg, f in (("ei", qb.qb_ei_dense), ("fp", qb.qb_fp_dense)):
            for P in (0, 1):
                if prec == "fp64":
                    call = lambda: f(A64, 0.0, 20, P=P, seed=SEED_OMEGA, rank_cap=200)  # noqa: E731
                else:
                    call = lambda: f(hi, 0.0, 20, P=P, seed=SEED_OMEGA, rank_cap=200, a_lo=lo,  # noqa: E731
                                     src_norm2=norms[0], prec="mixed")
                _, _, info = call()
                t = event_time(torch, call, 1 if prec == "fp64" else 3, stream)
                out[f"{prec}_{alg}_P{P}"] = {"time_s": t, "rank": info.rank,
                                             "passes": info.passes,
                                             "err_rel_est": info.err_est / info.normA2 ** 0.5}
    del A64, hi, lo
    torch.cuda.empty_cache()
    return out


# ----------------------------------------------------------------------------- reference arm
def run_reference(args, ws, rank):
    """The oracle's randQB_FP on the same workload, timed on the host cores: each timed step is one
    complete run on the whole matrix (about two minutes on 16 cores), and the timed steps stop once
    150 s are spent so the arm ends within a few minutes.  Warm-up steps run on a 500-row slice:
    the oracle has nothing to compile, they only start the BLAS threads and fill the caches."""
    if rank != 0:
        return
    import numpy as np
    import torch

    import oracle
    import synth
    m, n = (4000, 2000) if args.quick else (M, N)
    r = min(RANK_SPECTRUM, n)
    sigma = synth.sigma_exp(r, 200.0, 1e-6)
    # the same A as the GPU arm when a GPU is present, else the float64 CPU generator
    if torch.cuda.is_available():
        A = synth.dense_from_spectrum_torch(m, n, sigma, SEED_A, "cuda:0").cpu().numpy()
        torch.cuda.empty_cache()
    else:
        A = synth.dense_from_spectrum(m, n, sigma, SEED_A)
    for _ in range(args.warmup):
        oracle.randqb_fp(A[:500], TOL, B, seed=SEED_OMEGA, P=P, l_tilde=L_TILDE,
                         rank_cap=RANK_CAP)
    times = []
    rank_out = None
    for _ in range(max(1, args.steps)):
        t0 = time.perf_counter()
        res = oracle.randqb_fp(A, TOL, B, seed=SEED_OMEGA, P=P, l_tilde=L_TILDE, rank_cap=RANK_CAP)
        times.append(time.perf_counter() - t0)
        rank_out = res.rank
        if sum(times) > 150:      # keep the whole run within a few minutes
            break
    v = statistics.mean(times)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": ws,
            "steps": len(times), "warmup": args.warmup, "ms_per_step": v * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": config_dict(m, n),
            "cpu_baseline": {"value": v, "unit": "s", "cores": oracle_cores(), "kind": "oracle",
                             "cpu": cpu_model(),
                             "sample": f"the whole {m}x{n} workload per step (rank {rank_out}), "
                                       f"measured, not scaled; warm-up on rows 0..499"},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    _ = np


def config_dict(m, n):
    return {"workload": f"dense {m}x{n} sigma_j=exp(-j/200)+1e-6, randQB_FP mixed (bf16 hi+lo A), "
                        f"b={B}, P={P}, relative tol={TOL}, l~={L_TILDE}",
            "m": m, "n": n, "b": B, "P": P, "tol": TOL, "l_tilde": L_TILDE, "rank_cap": RANK_CAP,
            "seed_A": SEED_A, "seed_omega": SEED_OMEGA, "parallelism": "replicas",
            "l2": "inputs larger than L2 (A hi+lo = 3.2 GB)"}


# ----------------------------------------------------------------------------- our arm
def run_ours(args, ws, rank, local):
    import numpy as np
    import torch

    import paper_1606_09402_gb300 as qb

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    A64, sigma = make_inputs(torch, dev, args.quick)
    m, n = A64.shape
    hi, lo, norms = qb.quantize_bf16x2(A64)
    normA2 = norms[0]
    dt = torch.float32
    Qt = torch.empty(RANK_CAP, m, dtype=dt, device=dev)
    Bm = torch.empty(RANK_CAP, n, dtype=dt, device=dev)
    out = {}

    def step():
        out["r"] = qb.qb_fp_dense(hi, TOL, B, P=P, seed=SEED_OMEGA, a_lo=lo, src_norm2=normA2,
                                  prec="mixed", rank_cap=RANK_CAP, l_tilde=L_TILDE,
                                  out=(Qt, Bm), workspace=out.get("ws"))

    # workspace once (the binding reuses it)
    import ctypes as C
    from paper_1606_09402_gb300 import _lib
    d = qb._dense_desc(hi, lo, normA2)
    o = qb._opts(TOL, B, P, SEED_OMEGA, True, RANK_CAP, L_TILDE, True, "mixed")
    wsb = _lib.load().qb_dense_workspace(C.byref(d), C.byref(o), 1)
    out["ws"] = torch.empty(wsb, dtype=torch.uint8, device=dev)

    l0 = qb.launch_count()
    with Clocks(local) as ck:
        t_step = timed(torch, step, args.steps, args.warmup, ws, stream)
    launches = qb.launch_count() - l0
    Q, Bf, info = out["r"]
    # one extra, untimed factorisation with phase events (QB_FLAG_PROFILE) for the breakdown
    qb.qb_fp_dense(hi, TOL, B, P=P, seed=SEED_OMEGA, a_lo=lo, src_norm2=normA2, prec="mixed",
                   rank_cap=RANK_CAP, l_tilde=L_TILDE, out=(Qt, Bm), workspace=out["ws"], flags=2)
    phases = qb.profile_last()
    if args.steps_only:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": t_step, "unit": "s", "rank": info.rank,
                              "launches_per_step": launches / (args.steps + args.warmup),
                              "phases_ms": phases}))
        return
    # timed-region launches only: the warmup steps launched the same count per step
    per_step = launches / (args.steps + args.warmup)
    gpu_launches = int(round(per_step * args.steps))

    # achieved error (float64, verification only; untimed)
    err2 = 0.0
    for r0 in range(0, m, 4096):
        r1 = min(m, r0 + 4096)
        D = A64[r0:r1] - (Q[r0:r1].double() @ Bf.double())
        err2 += float((D * D).sum())
    err_rel = (err2 / normA2) ** 0.5

    # ---- kernel-level: the A passes measured with CUDA events on the launching stream
    pk, pk_src = peaks()
    hbm = pk["hbm_gbs"]
    reps = 3 if args.quick else 10
    Om = torch.randn(n, L_TILDE, device=dev, dtype=torch.float32)
    G = torch.randn(m, L_TILDE, device=dev, dtype=torch.float32)
    t_sk_wide = pass_time(torch, qb, lambda: qb.qb_apass_sketch(hi, Om), reps, "sketch")
    # the precise transposed pass of the step: one 512-column chunk of H = A^T G, G held as
    # two-term bf16 values (precise=3, four tensor-core products per output)
    Gc = torch.randn(m, 512, device=dev, dtype=torch.float32)
    t_prec = pass_time(torch, qb, lambda: qb.qb_apass_trans(hi, Gc, precise=3, a_lo=lo), reps,
                       "trans")
    Om64 = torch.randn(n, B, device=dev, dtype=torch.float32)
    G64 = torch.randn(m, B, device=dev, dtype=torch.float32)
    t_sk_nar = pass_time(torch, qb, lambda: qb.qb_apass_sketch(hi, Om64), reps, "sketch")
    t_tr_nar = pass_time(torch, qb, lambda: qb.qb_apass_trans(hi, G64, precise=1, a_lo=lo), reps,
                         "trans")
    # the setup quantisation float64 A -> bf16 hi + lo, outside time-to-tolerance
    t_quant = event_time(torch, lambda: qb.quantize_bf16x2(A64), reps, stream)
    flops_wide = 2.0 * m * n * L_TILDE
    a_hi_bytes = 2.0 * m * n
    tf_sk = flops_wide / t_sk_wide / 1e12
    tf_prec = 2.0 * m * n * 512 / t_prec / 1e12
    gbs_nar_sk = (a_hi_bytes + 4.0 * (n + m) * B) / t_sk_nar / 1e9
    gbs_nar_tr = (2 * a_hi_bytes + 4.0 * (n + m) * B) / t_tr_nar / 1e9

    # ---- float64 randQB_FP on the same A (the comparison path): one warm-up run, one timed
    # with CUDA events; its float64 sketch pass against a measured float64 GEMM rate
    fp64 = None
    if not args.no_fp64:
        Q64 = torch.empty(RANK_CAP, m, dtype=torch.float64, device=dev)
        B64 = torch.empty(RANK_CAP, n, dtype=torch.float64, device=dev)
        res64 = {}

        def step64():
            res64["r"] = qb.qb_fp_dense(A64, TOL, B, P=P, seed=SEED_OMEGA, rank_cap=RANK_CAP,
                                        l_tilde=L_TILDE, out=(Q64, B64))
        t64 = event_time(torch, step64, 1, stream)
        inf64 = res64["r"][2]
        del Q64, B64
        # the float64 peak of this GPU: cuBLAS DGEMM 4096^3, best of 3 (CUDA events)
        X = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
        best = min(event_time(torch, lambda: X @ X, 1, stream) for _ in range(3))
        dgemm_tf = 2.0 * 4096 ** 3 / best / 1e12
        del X
        V64 = torch.randn(n, 512, dtype=torch.float64, device=dev)
        t_sk64 = pass_time(torch, qb, lambda: qb.qb_apass_sketch(A64, V64), 3, "sketch")
        sk64_tf = 2.0 * m * n * 512 / t_sk64 / 1e12
        del V64
        fp64 = {"time_to_tol_s": t64, "rank": inf64.rank,
                "err_est": inf64.err_est / normA2 ** 0.5, "status": inf64.status,
                "timing": "one warm-up run, then one run timed with CUDA events",
                "dgemm_tflops_measured": dgemm_tf,
                "sketch_pass_w512": {"kernel": "k_gemm2 (float64 SIMT), G = A Omega, w = 512",
                                     "ms": t_sk64 * 1e3, "achieved_tflops": sk64_tf,
                                     "frac_of_dgemm": sk64_tf / dgemm_tf}}

    # ---- mixed randQB_EI on the same A (narrow passes)
    ei = None
    try:
        def step_ei():
            out["e"] = qb.qb_ei_dense(hi, TOL, B, P=P, seed=SEED_OMEGA, a_lo=lo, src_norm2=normA2,
                                      prec="mixed", rank_cap=RANK_CAP, out=(Qt, Bm))
        t_ei = timed(torch, step_ei, max(1, args.steps // 2), 1, 1, stream)
        ie = out["e"][2]
        ei = {"time_to_tol_s": t_ei, "rank": ie.rank, "passes": ie.passes}
    except Exception as e:  # pragma: no cover
        ei = {"error": str(e)}

    # ---- batched: 256 float32 matrices, m, n ~ U[256, 4096], sigma_j = s j^-2, tol in {1e-2, 1e-3}
    batched = None if args.quick else run_batched(torch, qb, dev, stream)
    # ---- fixed-rank adjoint: 8192 x 8192 bf16, k = 256, sigma_j = 1/j
    adjoint = None if args.quick else run_adjoint(torch, qb, dev, stream)
    # ---- sparse: CSR 200000 x 100000, nnz ~ 2e7
    sparse = None if args.quick else run_sparse(torch, qb, dev, stream)
    # ---- the paper's dense runtime shape: n = 32000, l = 200, b = 20
    paper_dense = None if args.quick else run_paper_dense(torch, qb, dev, stream)

    # ---- end to end through the public API with host buffers (pinned)
    hi_h = hi.cpu().pin_memory()
    lo_h = lo.cpu().pin_memory()
    hi_d = torch.empty_like(hi)
    lo_d = torch.empty_like(lo)
    Qh = torch.empty(RANK_CAP, m, dtype=dt).pin_memory()
    Bh = torch.empty(RANK_CAP, n, dtype=dt).pin_memory()
    d2h = {"b": 0}

    # A_hi first on the call's stream; A_lo on a second stream right after it, overlapping the
    # power scheme's sketches (which read A_hi only); the call waits on lo_ready before its first
    # read of A_lo.  Both copies are inside the timed region.
    side = torch.cuda.Stream(device=dev)
    hi_ready = torch.cuda.Event()
    lo_ready = torch.cuda.Event()

    def step_e2e():
        hi_d.copy_(hi_h, non_blocking=True)
        hi_ready.record(stream)
        side.wait_event(hi_ready)
        with torch.cuda.stream(side):
            lo_d.copy_(lo_h, non_blocking=True)
            lo_ready.record(side)
        Qx, Bx, ix = qb.qb_fp_dense(hi_d, TOL, B, P=P, seed=SEED_OMEGA, a_lo=lo_d,
                                    src_norm2=normA2, prec="mixed", rank_cap=RANK_CAP,
                                    l_tilde=L_TILDE, out=(Qt, Bm), workspace=out["ws"],
                                    a_lo_ready=lo_ready)
        k = ix.rank
        Qh[:k].copy_(Qt[:k], non_blocking=True)
        Bh[:k].copy_(Bm[:k], non_blocking=True)
        d2h["b"] = 4 * k * (m + n)

    t_e2e = timed(torch, step_e2e, max(1, args.steps // 2), 1, 1, stream)

    # ---- max over ranks
    if ws > 1:
        tt = torch.tensor([t_step], device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        t_step = float(tt.item())
    if rank != 0:
        return

    # the passes are timed alone (pass_time: CUDA events around one single-pass call), so the
    # burst figure is their peak; the sustained one is kept beside it for reference
    burst = pk["bf16_tflops"]
    sustained = pk.get("bf16_tflops_sustained", burst)
    A_host = A64.cpu().numpy()
    del A64
    torch.cuda.empty_cache()
    cpu = cpu_baseline(A_host)
    line = {
        "metric": METRIC, "value": t_step, "unit": "s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": config_dict(m, n),
        "result": {"rank": info.rank, "status": info.status, "err_est": info.err_est / normA2 ** 0.5,
                   "err_true": err_rel, "passes": info.passes, "blocks": info.blocks,
                   "svd_rank": 1382 if not args.quick else None},
        "roofline": {"bound": "tensor",
                     "kernel": "k_tc_prec: precise H = (A_hi + A_lo)^T G chunk (w = 512), "
                               "4 bf16 tensor-core products per output",
                     "achieved": tf_prec, "peak": burst, "unit": "TFLOP/s",
                     "frac": tf_prec / burst, "traffic": PREC_TRAFFIC_BYTES if not args.quick else None,
                     "traffic_note": PREC_TRAFFIC_NOTE,
                     "algorithmic": "2 m n w flops per launch (the product, not the 4 issued)",
                     "issued_frac": 4 * tf_prec / burst, "ms_per_launch": t_prec * 1e3,
                     "frac_of_sustained": tf_prec / sustained,
                     "peak_source": f"{pk_src} bf16_tflops (burst: the pass is timed alone)"},
        "roofline_sketch": {"bound": "tensor", "kernel": "k_tc_gemm: sketch G = A_hi Omega "
                                                         "(w = l~ = 3200)",
                            "achieved": tf_sk, "peak": burst, "unit": "TFLOP/s",
                            "frac": tf_sk / burst, "ms_per_launch": t_sk_wide * 1e3,
                            "peak_source": f"{pk_src} bf16_tflops (burst)"},
        "apass": {"sketch_narrow_gbs": gbs_nar_sk, "trans_narrow_precise_gbs": gbs_nar_tr,
                  "hbm_peak_gbs": hbm, "sketch_narrow_frac": gbs_nar_sk / hbm,
                  "trans_narrow_frac": gbs_nar_tr / hbm, "w": B,
                  "sketch_wide_ms": t_sk_wide * 1e3, "peak_source": pk_src,
                  "timing": "CUDA events the library records on the launching stream around "
                            "each single-pass call (operand split, kernel, fix-up)"},
        "phases_ms": phases,
        "setup_ms": {"quantize_bf16x2": t_quant * 1e3,
                     "note": "float64 A -> bf16 hi + lo with the norms; not in time-to-tolerance"},
        "fp64_randqb_fp": fp64,
        "mixed_randqb_ei": ei,
        "batched_ei_256": batched,
        "fixed_rank_adjoint_8192": adjoint,
        "sparse_csr_200000x100000": sparse,
        "paper_dense_32000": paper_dense,
        "e2e": {"value": t_e2e, "unit": "s", "h2d_bytes_per_step": int(2 * hi.numel() * 2),
                "d2h_bytes_per_step": int(d2h["b"])},
        "gpu_launches": gpu_launches,
        "clocks": ck.summary(),
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    _ = np


def run_profile_small(alg):
    """The small case of the mixed randQB_FP (alg "fp") or randQB_EI (alg "ei": its passes are the
    narrow w = b ones) step for ncu captures: A 16384 x 8192 (sigma_j = exp(-j/100) + 1e-6,
    j <= 2048), b = 64, P = 1, tol 1e-3; A hi+lo = 537 MB, larger than L2."""
    import torch

    import paper_1606_09402_gb300 as qb
    import synth
    A = synth.dense_from_spectrum_torch(16384, 8192, synth.sigma_exp(2048, 100.0, 1e-6), 3, "cuda")
    hi, lo, norms = qb.quantize_bf16x2(A)
    del A
    torch.cuda.synchronize()
    f = qb.qb_fp_dense if alg == "fp" else qb.qb_ei_dense
    for _ in range(2):
        _, _, info = f(hi, TOL, B, P=P, seed=1, prec="mixed", a_lo=lo, src_norm2=norms[0],
                       rank_cap=1600)
        torch.cuda.synchronize()
        print("rank", info.rank, "status", info.status, flush=True)


def run_profile_other(kind):
    """Small cases of the other kernel families for ncu captures (each exits 0 on success)."""
    import numpy as np
    import torch

    import paper_1606_09402_gb300 as qb
    import synth
    dev = "cuda"
    if kind in ("csr", "coo"):
        # 50000 x 25000, Poisson(100) rows, Zipf(1.1) columns: CSR 40 MB (> L2 with X staging)
        c = synth.csr_zipf(50000, 25000, 100.0, 1.1, seed=909, val_dtype=np.float32)
        rp, ci, v = (torch.tensor(c.rowptr, device=dev), torch.tensor(c.colind, device=dev),
                     torch.tensor(c.val, device=dev))
        for _ in range(2):
            if kind == "csr":
                _, _, info = qb.qb_ei_csr(rp, ci, v, (c.m, c.n), 0.5, 32, P=1, seed=1, rank_cap=128)
            else:
                row = torch.tensor(np.repeat(np.arange(c.m, dtype=np.int32),
                                             np.diff(c.rowptr.astype(np.int64))), device=dev)
                _, _, info = qb.qb_ei_coo(row, ci, v, (c.m, c.n), 0.5, 32, P=1, seed=1,
                                          rank_cap=128)
            torch.cuda.synchronize()
            print("rank", info.rank, "status", info.status, flush=True)
    elif kind == "batched":
        specs = synth.batched_specs(32, 1606)
        mats = [synth.dense_from_spectrum_torch(s.m, s.n, synth.sigma_pow(min(s.m, s.n, 512), 2.0,
                                                                          s.scale),
                                                s.seed, dev, dtype=torch.float32) for s in specs]
        for _ in range(2):
            res = qb.qb_ei_batched(mats, [s.tol for s in specs], seed=9402)
            torch.cuda.synchronize()
            print("ranks", [r[2].rank for r in res[:8]], flush=True)
    elif kind in ("adjoint", "adjoint8192"):
        m = n = 4096 if kind == "adjoint" else 8192
        k = 256
        A = synth.dense_from_spectrum_torch(m, n, 1.0 / np.arange(1, n + 1), 1606, dev,
                                            dtype=torch.float32).to(torch.bfloat16)
        GQ, GB = synth.cotangents(m, n, k, seed=5)
        GQ = torch.tensor(GQ, dtype=torch.float32, device=dev)
        GB = torch.tensor(GB, dtype=torch.float32, device=dev)
        for _ in range(2):
            Q, B, R = qb.qb_fixed_rank_fwd(A, k, 9)
            GA = qb.qb_fixed_rank_bwd(A, k, 9, Q, R, GQ, GB)
            torch.cuda.synchronize()
            print("grad norm", float(GA.double().norm()), flush=True)
    elif kind == "svd":
        A = synth.dense_from_spectrum_torch(8192, 4096, synth.sigma_exp(4096, 300.0), 7, dev)
        Q, B, info = qb.qb_fp_dense(A, 0.0, 64, P=1, seed=2, rank_cap=1024)
        for _ in range(2):
            _, S, _, sweeps = qb.qb_svd_from_qb(Q, B)
            torch.cuda.synchronize()
            print("sweeps", sweeps, "s1", float(S[0]), flush=True)


def main():
    args = parse()
    if args.profile_small in ("fp", "ei"):
        run_profile_small(args.profile_small)
        return
    if args.profile_small:
        run_profile_other(args.profile_small)
        return
    ws, rank, local = dist_env()
    if ws > 1:
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        torch.distributed.init_process_group(backend)
    if args.impl == "reference":
        if ws > 1 and rank != 0:
            return
        run_reference(args, ws, rank)
        return
    run_ours(args, ws, rank, local)
    if ws > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
