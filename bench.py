"""Benchmark of the BLWS path: Robust PCA solves/s and latency on one GPU.

One step = one complete Robust PCA solve (inexact ALM, every SVT by BLWS:
start block, block Lanczos products, block coefficients, residuals,
CholeskyQR2, T_k eigen-solve, Ritz lift, threshold and count, fused epilogue)
on the 2000 x 2000, rank-100, 10%-corrupted synthetic workload (seeded), run
to tol 1e-7.  The timed region holds only device work on inputs already in
HBM; L2 is flushed (a 512 MB write) between steps, outside the timed events.

Prints ONE JSON line (rank 0).  --impl reference times the FP64 CPU oracle
(full-SVD inexact ALM) on the host cores instead, on a bounded sample.
Under torchrun (N > 1) every rank solves its own instances (replicas: the
solves are independent) and rank 0 reports the aggregate.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (m, n, rank, corrupted fraction)
    "rpca_2000x2000_r100": (2000, 2000, 100, 0.10),
    "rpca_20000x200_r5": (20000, 200, 5, 0.10),
    "rpca_200x200_r10": (200, 200, 10, 0.05),
}
DEFAULT = "rpca_2000x2000_r100"
WORKLOAD_MN = {k: v[0] * v[1] for k, v in WORKLOADS.items()}
PRECISIONS = {"fp64": 0, "mixed": 1, "fp64tc": 2}
MC_WORKLOADS = {
    # name: (m, n, rank, observed fraction)
    "mc_5000x5000_r50": (5000, 5000, 50, 0.10),
}
# DRAM bytes (read + write) of one product with the augmented matrix, both
# gemm_f64_kernel<double, ., 0, 32, 8> launches, from one ncu capture of the
# 2000 x 2000 workload at b = 101 with the current FP64 GEMM kernel
APPLY_TRAFFIC = {"rpca_2000x2000_r100": 33622016 + 33624320}
APPLY_TRAFFIC_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of the two gemm_f64_kernel "
                        "<double,{0,1},0,32,8> launches of blws_apply (b=101), bench.py --profile-apply")


MODE_DTYPE = {
    "fp64": "f64 throughout (DFMA products)",
    "mixed": "tf32x3 tensor-core products (hi+lo split, f32 sums of <= 256 terms, f64 beyond), f64 "
             "Cholesky/eigen/count (the eigen refinement's products as fp64-equivalent digit planes); "
             "fp64-equivalent digit-plane products for everything once the residual < 1e-5",
    "fp64tc": "fp64-equivalent products: 7 bf16 digit planes per operand on tcgen05 (exact f32 sums of "
              "256 terms, ~1e-14 relative); Cholesky, eigen stage and count f64",
}
LEG_KEY = {"fp64": "fp64_dfma", "mixed": "mixed_precision", "fp64tc": "fp64_tensor_core"}
# tensor-core work per multiply-add of the product with W~: 28 BF16 digit-pair
# MMAs (FP64-equivalent mode), 3 TF32 MMAs (mixed mode); 2 flops each
TENSOR_MMAS = {"fp64tc": 28, "mixed": 3}
# DRAM bytes (read + write) of one launch of the digit-plane kernel for the
# 2000 x 2000 product at b = 101 (2 K splits, 128 CTAs), from one ncu capture of
# the current kernel (bench.py --profile-apply --precision fp64tc)
OZ_TRAFFIC = {"rpca_2000x2000_r100": 120623616 + 3644672}
OZ_TRAFFIC_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one oz_kernel launch of blws_apply "
                     "(b=101, the eight-drain-warp kernel), bench.py --profile-apply --precision fp64tc")


def measured_peaks():
    """The measured peaks of this machine (HBM copy GB/s, bf16 TFLOP/s
    burst and sustained), else the recipe's fallback figures."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": d["hbm_gbs"], "bf16": d["bf16_tflops"], "bf16_sustained": d["bf16_tflops_sustained"],
                "source": "of measured (MEASURED_PEAKS.json)"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16": 1900.0, "bf16_sustained": 1700.0, "source": "of fallback"}


# kernel kind of the mode's products with W~ (blws_timing_records): FP64 DFMA,
# split TF32, digit planes.  The mixed mode's refinement tail and every mode's
# norm estimate of the tensor-core modes run digit-plane products too; the
# roofline is the mode's own kernel's.
MODE_KIND = {"fp64": 0, "mixed": 1, "fp64tc": 2}


def steady_state(records, kind=None, work=None):
    """The timed products of the given kernel kind at the solves' steady block
    width: those of work `work` (2 m n b at the final b) when there are any,
    else the size that takes the most device time (the small products of the
    norm estimate and the wider ones of the first iterations are left out):
    (count, mean ms, work each)."""
    recs = [(t, w) for t, w, k in records or [] if kind is None or k == kind]
    if not recs:
        return 0, 0.0, 0.0
    tot = {}
    for t, w in recs:
        tot[w] = tot.get(w, 0.0) + t
    w0 = work if work in tot else max(tot, key=lambda w: (tot[w], w))
    ts = [t for t, w in recs if w == w0]
    return len(ts), float(np.mean(ts)), w0


def roofline(torch, mode, ms, launches, work, clocks, workload, b, records=None):
    """Roofline object of the dominant kernel, the product with W~ (step a2),
    from the device times the library's event timing measured around each of
    them in the timed solves: the products of the block width that takes the
    most of the kernel's time (b = 101 on the 2000 x 2000 workload), with the
    rate over all products (the norm estimate's and the first iterations'
    included) beside it."""
    if not launches or ms <= 0:
        return None
    all_tflops = 2.0 * work / (ms / 1e3) / 1e12  # FP64-equivalent rate over every product
    n_ss, ms_ss, w_ss = steady_state(records, MODE_KIND[mode], 2.0 * WORKLOAD_MN[workload] * b)
    if n_ss:
        launches, work, ms = n_ss, w_ss * n_ss, ms_ss * n_ss
        b = int(round(w_ss / (2.0 * WORKLOAD_MN[workload])))
    per = ms / launches / 1e3  # seconds per product
    if mode == "fp64":
        peak, sms, mhz = fp64_peak_gflops(torch, clocks.get("sm_max_mhz"))
        achieved = 2.0 * work / launches / per / 1e9
        return {"kernel": "gemm_f64 x 2 (P = [W X_v; W^T X_u], b=%d)" % b, "bound": "alu",
                "achieved": achieved, "peak": peak, "unit": "GFLOP/s", "frac": achieved / peak,
                "traffic": APPLY_TRAFFIC.get(workload) if b == 101 else None,
                "traffic_source": APPLY_TRAFFIC_SOURCE if b == 101 else None,
                "launches": launches, "us_per_launch": per * 1e6,
                "algorithmic": "2 x (2 m n b) FP64 flops per product",
                "peak_source": "FP64 derived from unit counts: %d SMs x 2 DFMA/clk x 2 x %.0f MHz "
                               "(MEASURED_PEAKS.json has no FP64 figure)" % (sms, mhz)}
    pk = measured_peaks()
    mmas = TENSOR_MMAS[mode]
    achieved = 2.0 * mmas * work / launches / per / 1e12
    # timed inside long solves: the sustained bf16 figure; TF32 at half the bf16 rate
    peak = pk["bf16_sustained"] * (0.5 if mode == "mixed" else 1.0)
    kern = "oz_kernel (digit-plane products, both halves of P in one launch)" if mode == "fp64tc" else \
        "tc_tf32x3_kernel (split-TF32 products, both halves of P in one launch)"
    tr = OZ_TRAFFIC.get(workload) if mode == "fp64tc" and b == 101 else None
    return {"kernel": kern + ", b=%d" % b, "bound": "tensor", "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak, "traffic": tr,
            "traffic_source": OZ_TRAFFIC_SOURCE if tr else None,
            "launches": launches, "us_per_launch": per * 1e6,
            "algorithmic": "%d x 2 x (2 m n b) %s tensor flops per product (b unpadded)"
                           % (mmas, "bf16" if mode == "fp64tc" else "tf32"),
            "fp64_equivalent_tflops": 2.0 * work / launches / per / 1e12,
            "all_products_fp64_equivalent_tflops": all_tflops,
            "peak_source": "bf16 sustained %s%s" % (pk["source"], ", x 0.5 for tf32 (nominal ratio)"
                                                     if mode == "mixed" else "")}


def fp64_peak_gflops(torch, sm_max_mhz):
    """FP64 peak derived from unit counts: SMs (read from the device) x 2 DFMA
    per clock per SM x 2 flops x the maximum SM clock (sampled by nvidia-smi,
    else the GB300's 2070 MHz)."""
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = sm_max_mhz or 2070.0
    return sms * 2 * 2 * mhz * 1e6 / 1e9, sms, mhz


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def max_over_ranks(dist, local, device):
    """The largest of a per-rank value over all ranks (the slowest rank sets the
    job's time); `local` itself with no process group."""
    if dist is None:
        return float(local)
    import torch
    t = torch.tensor([float(local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world_size, units_per_rank, ms):
    """Whole-job throughput: the units all ranks processed over the job's time."""
    return world_size * units_per_rank / (ms / 1e3)


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def blas_threads():
    """Host threads the oracle's LAPACK/BLAS calls use (OpenBLAS: every core
    unless an environment variable caps it)."""
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        v = os.environ.get(var)
        if v and v.isdigit():
            return int(v)
    return os.cpu_count()


def cpu_oracle_solve(D, tol):
    """One complete solve of the FP64 oracle (inexact ALM with a full LAPACK SVD
    in every iteration) on the host cores, timed; its A and E are the reference
    every GPU leg's relerr_vs_oracle is taken against."""
    import oracle
    t0 = time.perf_counter()
    out = oracle.rpca_ialm_full(D, tol=tol)
    dt = time.perf_counter() - t0
    return {"value": 1.0 / dt, "unit": "solves/s", "cores": blas_threads(), "kind": "oracle",
            "ms_per_solve": dt * 1e3, "iters": out["iters"], "rank": out["rank"],
            "sample": "one complete solve of the same workload to tol %g (%d inexact-ALM iterations, "
                      "full LAPACK SVD each, %.1f s)" % (tol, out["iters"], dt)}, out


def relerr_to(torch, X, ref):
    """||X - ref||_F / ||ref||_F, X a CUDA tensor and ref a host array."""
    R = torch.from_numpy(np.ascontiguousarray(ref)).to(X.device)
    return float(torch.linalg.norm(X - R) / torch.linalg.norm(R))


def fullsvd_gpu_sample(torch, Dg, lam, iters_full, sample_iters=2):
    """The same inexact-ALM host rules with a library FP64 SVD (cuSOLVER
    through torch.linalg.svd) on the same GPU: the plain full-SVD SVT the
    method replaces.  A comparison leg only (never on the product path):
    timed over a bounded number of iterations, scaled to a full solve."""
    m, n = Dg.shape
    D = Dg.contiguous()
    norm_two = float(torch.linalg.matrix_norm(D, ord=2))
    J = max(norm_two, float(D.abs().max()) / lam)
    Y = D / J
    E = torch.zeros_like(D)
    A = torch.zeros_like(D)
    mu = 1.25 / norm_two
    torch.cuda.synchronize()
    times = []
    for it in range(sample_iters + 1):
        t0 = time.perf_counter()
        W = D - A + Y / mu
        E = torch.sign(W) * torch.clamp(W.abs() - lam / mu, min=0.0)
        U, S, Vh = torch.linalg.svd(D - E + Y / mu, full_matrices=False)
        th = torch.clamp(S - 1.0 / mu, min=0.0)
        A = (U * th) @ Vh
        Z = D - A - E
        Y = Y + mu * Z
        mu = mu * 1.5
        float(torch.linalg.norm(Z))  # the host reads the residual each iteration
        torch.cuda.synchronize()
        if it:  # the first iteration also warms the library up
            times.append(time.perf_counter() - t0)
    per_iter = float(np.mean(times))
    return {"value": 1.0 / (per_iter * iters_full), "unit": "solves/s", "ms_per_iter": per_iter * 1e3,
            "sample": "%d inexact-ALM iterations with a full FP64 SVD (torch.linalg.svd) on the same "
                      "GPU, scaled to %d iterations" % (sample_iters, iters_full)}


def run_mc(args):
    """Matrix completion, m = n = 5000, rank 50, 10% observed (2.5M entries, CSR int32):
    SVT of [Cai08] with every SVT by BLWS over the CSR operator, to tol 1e-4.  Prints its
    own JSON line (metric mc_solves_per_s)."""
    import torch
    from paper_1012_0365_gb300 import blws, synthetic as syn
    m, n, r, frac = MC_WORKLOADS[args.workload]
    P = syn.mc_problem(m, n, r, frac, seed=0)
    rowptr = torch.from_numpy(P["rowptr"]).cuda()
    cols = torch.from_numpy(P["cols"]).cuda()
    vals = torch.from_numpy(P["vals"]).cuda()
    prec = PRECISIONS[args.precision]
    ctx = blws.Context(k=args.k, precision=prec, tune=args.tune)
    flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    max_rank = 4 * r
    if args.profile_solve:  # one untimed solve, for a profiler's launch list
        l0 = ctx.launches
        U, th, V, info = ctx.mc_solve(m, n, rowptr, cols, vals, max_rank=max_rank)
        torch.cuda.synchronize()
        return {"profile": "solve", "workload": args.workload, "iters": info["iters"],
                "launches": ctx.launches - l0}
    for _ in range(args.warmup):
        U, th, V, info = ctx.mc_solve(m, n, rowptr, cols, vals, max_rank=max_rank)
    ms = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        U, th, V, info = ctx.mc_solve(m, n, rowptr, cols, vals, max_rank=max_rank)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    # relerr of X = U diag(th) V^T against the planted M = ML MR^T, both formed on the device
    # (the expansion ||X||^2 + ||M||^2 - 2 <X, M> cancels to rounding noise at 1e-4)
    with torch.no_grad():
        Mg = torch.from_numpy(P["ML"]).cuda() @ torch.from_numpy(P["MR"]).cuda().t()
        Xg = (U * th) @ V.t()
        rel = float(torch.linalg.norm(Xg - Mg) / torch.linalg.norm(Mg))
        del Mg, Xg
    # the sparse product [S X_v; S^T X_u] at b = rank + 1, with the CSC mirror built once
    b = r + 1
    mirror = ctx.csc_mirror(m, n, rowptr, cols)
    X = blws.colmajor(torch.randn(m + n, b, dtype=torch.float64, device="cuda"))
    Pm = blws.empty_colmajor(m + n, b)
    for _ in range(2):
        ctx.apply_sparse(m, n, rowptr, cols, vals, X, P=Pm, mirror=mirror)
    reps = 10
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        ctx.apply_sparse(m, n, rowptr, cols, vals, X, P=Pm, mirror=mirror)
    e1.record(stream)
    e1.synchronize()
    spmm_ms = e0.elapsed_time(e1) / reps
    nnz = int(vals.numel())
    flops = 4.0 * nnz * b
    achieved = flops / (spmm_ms / 1e3) / 1e9
    peak = fp64_peak_gflops(torch, None)[0]
    lat = np.array(ms)
    return {"metric": "mc_solves_per_s", "value": args.steps / (float(np.sum(ms)) / 1e3), "unit": "solves/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(ms)),
            "higher_is_better": True, "dtype": ["f64", "mixed", "f64 (tensor-core digits)"][prec], "data": "synthetic",
            "config": {"workload": args.workload, "m": m, "n": n, "rank": r, "observed": frac, "nnz": nnz,
                       "tol": 1e-4, "k": args.k, "l2": "flushed between steps (512 MB write)"},
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "solve": {"iters": info["iters"], "rank": info["rank"], "residual": info["residual"],
                      "relerr_vs_planted": rel},
            "roofline": {"kernel": "spmm_rows (S X_v and S^T X_u, b=%d)" % b, "bound": "alu",
                         "achieved": achieved, "peak": peak, "unit": "GFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "ms_per_product": spmm_ms,
                         "note": "blws_apply on the sparse operator with a prebuilt CSC mirror (includes "
                                 "the row-major copy of X)"}}


def mc_oracle_parity(torch):
    """Matrix completion against the FP64 oracle on a small case (200 x 200,
    rank 5, 6 samples per degree of freedom): SVT of [Cai08] run to tol 1e-8
    on both sides approaches the unique minimiser, where the iterates can be
    compared (the oracle takes a full LAPACK SVD per iteration)."""
    import oracle
    from paper_1012_0365_gb300 import blws, synthetic as syn
    m = n = 200
    r = 5
    P = syn.mc_problem(m, n, r, 6 * r * (m + n - r) / (m * n), seed=0)
    ctx = blws.Context(k=3)
    U, th, V, info = ctx.mc_solve(m, n, torch.from_numpy(P["rowptr"]).cuda(), torch.from_numpy(P["cols"]).cuda(),
                                  torch.from_numpy(P["vals"]).cuda(), max_rank=60, tol=1e-8, max_iter=3000)
    ref = oracle.mc_svt_full(m, n, P["rows"], P["cols"], P["vals"], tol=1e-8, max_iter=3000)
    X = ((U * th) @ V.t()).cpu().numpy()
    Xr = (ref["U"] * ref["th"]) @ ref["V"].T
    return {"workload": "mc_200x200_r5_6dof", "tol": 1e-8, "iters": info["iters"], "oracle_iters": ref["iters"],
            "relerr_vs_oracle": float(np.linalg.norm(X - Xr) / np.linalg.norm(Xr))}


def run_ablation(args):
    """Variants of the method (its own JSON line): on the 2000x2000 rank-100 RPCA
    workload, the number of Lanczos blocks k, the mixed start [U;V]/sqrt2 against
    the standard start [U;0] (Section 4.1), and warm starts against a cold
    (random-start) block Lanczos in every outer iteration; then the paper's size
    sweeps as GPU reruns: RPCA m = n in {500, 1000, 2000, 3000}, rank 10%, 10%
    corrupted, against full-SVD SVT on the same GPU (Table 1 pattern), and MC
    m = n from 5000 to 30000 at the (rank, samples per degree of freedom) pairs
    of the Table 2 pattern; and BL_EVD of a symmetric matrix (evd_sequence)."""
    import torch
    from paper_1012_0365_gb300 import blws, synthetic as syn

    def rpca_case(m, rank, ctx_kw, steps, max_iter=1000, amp=50.0):
        D, L0, _ = syn.rpca_problem(m, m, rank, 0.10, amp=amp, seed=0)
        Dg = blws.colmajor(torch.from_numpy(D))
        ctx = blws.Context(**ctx_kw)
        A = blws.empty_colmajor(m, m)
        E = blws.empty_colmajor(m, m)
        kw = dict(tol=1e-7, A=A, E=E, max_iter=max_iter, allow_noconv=True)
        _, _, info = ctx.rpca_solve(Dg, **kw)
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            _, _, info = ctx.rpca_solve(Dg, **kw)
            e1.record()
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        L0g = torch.from_numpy(L0).cuda()
        rel = float(torch.linalg.norm(A - L0g) / torch.linalg.norm(L0g))
        out = {"ms_per_solve": float(np.mean(ms)), "iters": info["iters"], "rank": info["rank"],
               "status": info["status"], "residual": info["residual"], "relerr_vs_planted": rel}
        return out, Dg, info

    res = {"metric": "ablation", "unit": "ms/solve", "n_gpus": 1, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "rpca_2000x2000_r100 variants; size sweeps", "tol_rpca": 1e-7}}
    base = {"precision": 0}
    res["k_sweep"] = {str(k): rpca_case(2000, 100, dict(base, k=k), 2)[0] for k in (2, 3, 4)}
    default = res["k_sweep"]["3"]  # k = 3, mixed start, warm restarts
    res["start"] = {"mixed [U;V]/sqrt2": default,
                    "standard [U;0]": rpca_case(2000, 100, dict(base, start=1), 2)[0]}
    # a cold (seeded Gaussian) block Lanczos of k_cold blocks in every outer iteration,
    # capped at 100 iterations: status -4 with the residual reached when it stalls
    res["warm"] = {"warm (BLWS), k=3": default,
                   "cold every iteration, k_cold=4": rpca_case(2000, 100, dict(base, warm=0), 1, max_iter=100)[0],
                   "cold every iteration, k_cold=8": rpca_case(2000, 100, dict(base, warm=0, k_cold=8), 1,
                                                               max_iter=100)[0]}
    # Table 1 pattern: rank 10% of m, 10% of the entries corrupted, values in [-500, 500]
    sweep = []
    for m in (500, 1000, 2000, 3000):
        r = max(1, int(round(0.10 * m)))
        out, Dg, info = rpca_case(m, r, base, 2, amp=500.0)
        full = fullsvd_gpu_sample(torch, Dg, 1.0 / math.sqrt(m), info["iters"])
        out.update({"m": m, "rank": r, "fullsvd_ms_per_solve": 1e3 / full["value"],
                    "speedup": 1e3 / full["value"] / out["ms_per_solve"]})
        sweep.append(out)
    res["rpca_size_sweep"] = sweep
    # Table 2 pattern: (m, r, samples per degree of freedom s / d_r)
    mcs = []
    for m, r, spd in ((5000, 10, 6), (5000, 50, 5), (5000, 100, 4), (10000, 10, 6), (10000, 50, 5),
                      (20000, 10, 6), (30000, 10, 6)):
        frac = spd * r * (2 * m - r) / (m * m)
        P = syn.mc_problem(m, m, r, frac, seed=0)
        ctx = blws.Context(precision=0)
        rp, cc, vv = (torch.from_numpy(P[x]).cuda() for x in ("rowptr", "cols", "vals"))
        # early SVT iterates can carry many more values above tau than the rank
        cap = min(m, max(4 * r, 200))
        try:
            U, th, V, info = ctx.mc_solve(m, m, rp, cc, vv, max_rank=cap)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            U, th, V, info = ctx.mc_solve(m, m, rp, cc, vv, max_rank=cap)
            e1.record()
            e1.synchronize()
        except blws.BlwsError as e:  # reported, not hidden: the sweep goes on
            mcs.append({"m": m, "rank": r, "s_per_dof": spd, "observed": frac, "error": str(e)})
            continue
        # ||U diag(th) V^T - ML MR^T||_F from the QR factors of [U th, -ML] and [V, MR]
        with torch.no_grad():
            ML, MR = torch.from_numpy(P["ML"]).cuda(), torch.from_numpy(P["MR"]).cuda()
            _, R1 = torch.linalg.qr(torch.cat([U * th, -ML], 1))
            _, R2 = torch.linalg.qr(torch.cat([V, MR], 1))
            _, R3 = torch.linalg.qr(ML)
            _, R4 = torch.linalg.qr(MR)
            rel = float(torch.linalg.norm(R1 @ R2.t()) / torch.linalg.norm(R3 @ R4.t()))
        mcs.append({"m": m, "rank": r, "s_per_dof": spd, "observed": frac, "ms_per_solve": e0.elapsed_time(e1),
                    "iters": info["iters"], "status": info["status"], "relerr_vs_planted": rel})
    res["mc_size_sweep"] = mcs
    res["bl_evd"] = evd_sequence(torch, blws, syn)
    return res


def evd_sequence(torch, blws, syn, m=4000, rank=150, r=100, calls=6, delta=1e-3):
    """BL_EVD on a symmetric W (Section 4's BLWS definition applied to a partial
    EVD): a sequence W_i = W + i delta E of nearby symmetric matrices, the
    leading r = 100 eigenpairs of each, warm-started from the previous call's
    (k = 3), against a cold block Lanczos per call (k_cold = 4) and a full FP64
    EVD by the library (torch.linalg.eigh, cuSOLVER) on the same GPU.  The
    accuracy is the largest error of the eigenvalues above eps against the
    library's, relative to the largest eigenvalue."""
    W0, npos = syn.symmetric_problem(m, rank, seed=0)
    G = syn.gaussian_block(m, m, seed=1)
    W0g = blws.colmajor(torch.from_numpy(W0))
    Eg = blws.colmajor(torch.from_numpy((G + G.T) / 2))
    lam_ref = torch.linalg.eigvalsh(W0g).flip(0)
    eps = float(0.5 * (lam_ref[npos - 1] + lam_ref[npos]))
    seq = [blws.colmajor(W0g + (i * delta) * Eg) for i in range(calls)]
    ctx = blws.Context(k=3)

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        e1.synchronize()
        return out, e0.elapsed_time(e1)

    U, lam, c = ctx.blws_evd(seq[0], eps, r)          # the first call is cold
    warm_ms, cold_ms, lib_ms, err_w, err_c = [], [], [], 0.0, 0.0
    for Wi in seq[1:]:
        ref, t = timed(lambda: torch.linalg.eigvalsh(Wi))
        lib_ms.append(t)
        ref = ref.flip(0)
        (U, lam, c), t = timed(lambda: ctx.blws_evd(Wi, eps, r, U))
        warm_ms.append(t)
        scale = float(ref.abs().max())
        err_w = max(err_w, float((lam[:c] - ref[:c]).abs().max()) / scale)
        (_, lamc, cc), t = timed(lambda: ctx.blws_evd(Wi, eps, r))
        cold_ms.append(t)
        err_c = max(err_c, float((lamc[:cc] - ref[:cc]).abs().max()) / scale)
    return {"m": m, "r": r, "count_above_eps": c, "calls": calls - 1, "delta": delta,
            "warm_k3_ms": float(np.mean(warm_ms)), "warm_max_relerr": err_w,
            "cold_k4_ms": float(np.mean(cold_ms)), "cold_max_relerr": err_c,
            "library_full_evd_ms": float(np.mean(lib_ms))}


def run_batch(args):
    """Uneven instances (m, n ~ U{100..1000}, rank 5% of min(m, n), 5-10%
    corruption) solved by the library's server: all submitted at once, solved
    concurrently by --workers workers.  Compared with the same instances solved
    one at a time through one context.  Prints its own JSON line."""
    import torch
    from paper_1012_0365_gb300 import blws, synthetic as syn
    specs = syn.batched_rpca_specs(args.batch_count, seed=0)
    probs = [syn.rpca_problem(s["m"], s["n"], s["rank"], s["frac"], seed=s["seed"]) for s in specs]
    Ds = [blws.colmajor(torch.from_numpy(p[0])) for p in probs]
    prec = PRECISIONS[args.precision]
    srv = blws.Server(workers=args.workers, precision=prec, grid_sms=args.grid_sms,
                      graphs=args.graphs, tune=args.tune)
    # warm-up: the workers' first solves; with the autotuner, every instance once
    # (each size bucket is timed the first time it is met, outside the timed region)
    warm = Ds if args.tune else Ds[:args.workers]
    for t in [srv.submit_rpca(D, tol=args.tol) for D in warm]:
        srv.wait(t)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tickets = [srv.submit_rpca(D, tol=args.tol) for D in Ds]
    outs = [srv.wait(t) for t in tickets]
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    rel = [float(torch.linalg.norm(A - torch.from_numpy(p[1]).cuda()) / np.linalg.norm(p[1]))
           for (A, _, _), p in zip(outs, probs)]
    ok = sum(1 for _, _, i in outs if i["status"] == 0)
    # one at a time, one context, on a sample of the same instances
    ctx = blws.Context(k=args.k, precision=prec, graphs=args.graphs, tune=args.tune)
    sample = min(len(Ds), 32)
    for D in Ds[:2]:
        ctx.rpca_solve(D, tol=args.tol)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for D in Ds[:sample]:
        ctx.rpca_solve(D, tol=args.tol)
    torch.cuda.synchronize()
    seq = sample / (time.perf_counter() - t1)
    lat = np.array([i["queue_ms"] + i["run_ms"] for _, _, i in outs])
    return {"metric": "rpca_batched_solves_per_s", "value": len(Ds) / wall, "unit": "solves/s",
            "n_gpus": 1, "higher_is_better": True, "dtype": ["f64", "mixed", "f64 (tensor-core digits)"][prec],
            "data": "synthetic",
            "config": {"workload": "rpca_batch_%d_uneven_100_1000" % len(Ds), "workers": args.workers,
                       "grid_sms": args.grid_sms, "graphs": args.graphs, "tune": args.tune,
                       "tuned_buckets": blws.Context.tune_count(),
                       "tol": args.tol, "k": args.k},
            "wall_s": wall, "solved_ok": ok, "relerr_vs_planted": {"median": float(np.median(rel)),
                                                                   "max": float(np.max(rel))},
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "peak_running": st["peak_running"],
            "sequential": {"value": seq, "unit": "solves/s", "sample": "%d of the instances, one at a "
                           "time through one context" % sample},
            "speedup_vs_sequential": (len(Ds) / wall) / seq}


def run_serve(args):
    """Serving: a Poisson stream of mixed RPCA / MC requests (a pool of seeded
    problems reused round-robin) at offered rates swept around the measured
    capacity; per rate the achieved solves/s and the p50 / p99 latency
    (submit to result).  Prints its own JSON line."""
    import torch
    from paper_1012_0365_gb300 import blws, synthetic as syn
    specs = syn.serving_specs(args.pool, seed=1)
    pool = []
    for sp in specs:
        if sp["kind"] == "rpca":
            D = syn.rpca_problem(sp["m"], sp["n"], sp["rank"], sp["frac"], seed=sp["seed"])[0]
            pool.append(("rpca", blws.colmajor(torch.from_numpy(D)), sp))
        else:
            P = syn.mc_problem(sp["m"], sp["n"], sp["rank"], sp["frac"], seed=sp["seed"])
            pool.append(("mc", (sp["m"], sp["n"], torch.from_numpy(P["rowptr"]).cuda(),
                                torch.from_numpy(P["cols"]).cuda(), torch.from_numpy(P["vals"]).cuda()),
                         sp))
    prec = PRECISIONS[args.precision]
    srv = blws.Server(workers=args.workers, precision=prec)

    def submit(item):
        kind, data, sp = item
        if kind == "rpca":
            return srv.submit_rpca(data, tol=args.tol)
        # output capacity: SVT's early iterates can hold many more values above tau than
        # the final rank when the sampling is thin (s / d_r near 3)
        return srv.submit_mc(*data, max_rank=min(max(4 * sp["rank"], sp["rank"] + 100), min(sp["m"], sp["n"])))

    for t in [submit(it) for it in pool]:  # warm-up, and every worker context sized
        srv.wait(t)
    t0 = time.perf_counter()
    outs = [srv.wait(t) for t in [submit(it) for it in pool]]
    capacity = len(pool) / (time.perf_counter() - t0)
    rng = np.random.default_rng(2)
    sweep = []
    for frac in args.serve_rates:
        rate = frac * capacity
        gaps = rng.exponential(1.0 / rate, size=args.serve_requests)
        arrivals = np.cumsum(gaps)
        tickets = [None] * len(arrivals)
        start = time.perf_counter()

        def producer():
            for i, ta in enumerate(arrivals):
                delay = start + ta - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                tickets[i] = submit(pool[i % len(pool)])

        th = threading.Thread(target=producer)
        th.start()
        lat, bad, statuses = [], 0, {}
        for i in range(len(arrivals)):
            while tickets[i] is None:
                time.sleep(0.0005)
            out = srv.wait(tickets[i])
            info = out[-1]
            lat.append(info["queue_ms"] + info["run_ms"])
            bad += info["status"] != 0
            if info["status"] != 0:
                statuses[str(info["status"])] = statuses.get(str(info["status"]), 0) + 1
        th.join()
        span = time.perf_counter() - start
        lat = np.array(lat)
        sweep.append({"offered_per_s": rate, "offered_frac_of_capacity": frac,
                      "achieved_per_s": len(arrivals) / span, "p50_ms": float(np.percentile(lat, 50)),
                      "p99_ms": float(np.percentile(lat, 99)), "failed": int(bad),
                      "failed_statuses": statuses})
    st = srv.stats()
    srv.close()
    n_rpca = sum(1 for k, _, _ in pool if k == "rpca")
    return {"metric": "serving_solves_per_s_and_latency", "value": capacity, "unit": "solves/s",
            "n_gpus": 1, "higher_is_better": True, "dtype": ["f64", "mixed", "f64 (tensor-core digits)"][prec],
            "data": "synthetic",
            "config": {"workload": "serve_mixed_rpca%d_mc%d" % (n_rpca, len(pool) - n_rpca),
                       "workers": args.workers, "requests_per_rate": args.serve_requests,
                       "tol_rpca": args.tol, "tol_mc": 1e-4},
            "pool": [{"kind": k, "m": sp["m"], "n": sp["n"], "rank": sp["rank"],
                      "frac": round(sp["frac"], 3)} for k, _, sp in pool],
            "sweep": sweep, "peak_running": st["peak_running"], "budget_bytes": st["budget"],
            "peak_in_use_bytes": st["peak_in_use"]}


def run_reference(args, ws, rank):
    """--impl reference: the FP64 CPU oracle (full-SVD inexact ALM) on the host
    cores, on the same workload.  One step is one outer iteration of the oracle
    (its full SVD dominates and costs the same in every iteration); the
    set-up (||D||_2 by a full SVD, Y_0, mu_0) is timed once, apart.  W warm-up
    iterations run untimed, then K timed ones; the solves/s figure is
    1 / (set-up + iterations-per-solve x mean iteration time), with the
    oracle's own iteration count on this workload (--ref-iters)."""
    from paper_1012_0365_gb300 import synthetic as syn
    import oracle
    if rank != 0:
        return None
    if args.workload not in WORKLOADS:
        return {"impl": "reference", "unavailable": "the CPU reference arm is defined on the RPCA workloads"}
    m, n, r, f = WORKLOADS[args.workload]
    D, L0, _ = syn.rpca_problem(m, n, r, f, seed=0)
    stamps = []
    t0 = time.perf_counter()
    oracle.rpca_ialm_full(D, tol=0.0, max_iter=args.warmup + args.steps,
                          progress=lambda: stamps.append(time.perf_counter()))
    setup = stamps[0] - t0
    iters = np.diff(np.array(stamps))           # one entry per outer iteration
    timed = iters[args.warmup:args.warmup + args.steps]
    per_iter = float(np.mean(timed))
    solve_s = setup + args.ref_iters * per_iter
    value = 1.0 / solve_s
    return {"metric": "rpca_solves_per_s", "value": value, "unit": "solves/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * per_iter,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "m": m, "n": n, "rank": r, "corrupt": f,
                       "tol": args.tol, "step": "one outer inexact-ALM iteration of the oracle"},
            "ms_per_solve": 1e3 * solve_s, "setup_ms": 1e3 * setup,
            "cpu_baseline": {"kind": "oracle", "cores": blas_threads(), "value": value,
                             "unit": "solves/s",
                             "sample": "%d timed inexact-ALM iterations (full LAPACK SVD each) after %d "
                                       "untimed, plus the set-up timed once; a solve = set-up + %d "
                                       "iterations" % (args.steps, args.warmup, args.ref_iters)},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="blws", choices=["blws", "reference"])
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS) + sorted(MC_WORKLOADS))
    ap.add_argument("--tol", type=float, default=1e-7)
    ap.add_argument("--k", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fullsvd", action="store_true", help="skip the full-SVD GPU comparison leg")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision measurement")
    ap.add_argument("--no-extra-legs", action="store_true",
                    help="skip the matrix-completion, batch and serving sub-objects of the default line")
    ap.add_argument("--ref-iters", type=int, default=25)
    ap.add_argument("--profile-solve", action="store_true",
                    help="run one untimed solve only (for ncu launch lists)")
    ap.add_argument("--profile-apply", action="store_true",
                    help="run the block product with W~ a few times only (for ncu captures)")
    ap.add_argument("--headline", default="fp64tc", choices=["fp64", "mixed", "fp64tc"],
                    help="precision mode of the headline value (the others become sub-objects)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed", "fp64tc"],
                    help="context precision of --profile-solve / --profile-apply / --batch / --serve")
    ap.add_argument("--batch", action="store_true", help="uneven batch through the server (own JSON line)")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--serve", action="store_true", help="Poisson serving sweep (own JSON line)")
    ap.add_argument("--ablation", action="store_true",
                    help="variants of the method and the paper's size sweeps (own JSON line)")
    ap.add_argument("--pool", type=int, default=12)
    ap.add_argument("--serve-requests", type=int, default=24)
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[0.25, 0.5, 1.0, 1.5])
    ap.add_argument("--workers", type=int, default=16)
    ap.add_argument("--grid-sms", type=int, default=0,
                    help="SMs each worker context sizes its grids for (0: all)")
    ap.add_argument("--graphs", type=int, default=1, choices=(0, 1),
                    help="replay CUDA graphs of the outer-iteration phases (1, default) or launch directly")
    ap.add_argument("--tune", type=int, default=1, choices=(0, 1),
                    help="CUDA-core product tiles from the timed autotuner (1, default) or the fixed rule")
    args = ap.parse_args()
    ws, rank = dist_env()

    if args.impl == "reference":
        out = run_reference(args, ws, rank)
        if out is not None:
            print(json.dumps(out))
        return
    if args.workload in MC_WORKLOADS and args.impl != "reference":
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        print(json.dumps(run_mc(args)))
        return
    if args.batch or args.serve or args.ablation:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        print(json.dumps(run_ablation(args) if args.ablation else run_batch(args) if args.batch else run_serve(args)))
        return

    import torch
    from paper_1012_0365_gb300 import blws, synthetic as syn

    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local_rank)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    m, n, r, f = WORKLOADS[args.workload]
    D, L0, S0 = syn.rpca_problem(m, n, r, f, seed=rank)
    Dh = torch.from_numpy(D.T.copy()).pin_memory()  # column-major host copy
    Dg = blws.empty_colmajor(m, n)
    Dg.t().copy_(Dh)
    A = blws.empty_colmajor(m, n)
    E = blws.empty_colmajor(m, n)
    Ah = torch.empty((n, m), dtype=torch.float64).pin_memory()
    Eh = torch.empty((n, m), dtype=torch.float64).pin_memory()
    head = PRECISIONS[args.headline]
    ctx = blws.Context(k=args.k, device=local_rank, precision=head, graphs=args.graphs, tune=args.tune)
    flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def solve(c=None):
        return (c or ctx).rpca_solve(Dg, tol=args.tol, A=A, E=E)

    if args.profile_solve or args.profile_apply:
        ctx = blws.Context(k=args.k, device=local_rank, precision=PRECISIONS[args.precision],
                           graphs=args.graphs, tune=args.tune)
        if args.profile_solve:
            l0 = ctx.launches
            _, _, info = solve()
            print(json.dumps({"profile": "solve", "precision": args.precision, "iters": info["iters"],
                              "launches": ctx.launches - l0}))
        else:
            b = r + 1
            X = blws.colmajor(torch.randn(m + n, b, dtype=torch.float64, device="cuda"))
            for _ in range(3):
                ctx.apply(Dg, X)
            print(json.dumps({"profile": "apply", "b": b}))
        torch.cuda.synchronize()
        return

    for _ in range(args.warmup):
        _, _, info = solve()
    torch.cuda.synchronize()

    # ---- device-timed steps (inputs resident in HBM) ----
    sampler = ClockSampler(local_rank)
    sampler.start()
    step_ms = []
    launches0 = ctx.launches
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    ctx.timing_start()  # events around every product with W~ (step a2) in the timed steps
    for _ in range(args.steps):
        flush.zero_()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        _, _, info = solve()
        ev1.record(stream)
        ev1.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall0
    apply_ms, apply_n, apply_work = ctx.timing_stop()
    apply_recs = ctx.timing_records()
    launches = ctx.launches - launches0
    clocks = sampler.stop()
    total_ms = max_over_ranks(dist, float(np.sum(step_ms)), "cuda")
    value = job_rate(ws, args.steps, total_ms)
    relerr = float(torch.linalg.norm(A - torch.from_numpy(L0).cuda()) / np.linalg.norm(L0))
    kept = {args.headline: (A.clone(), E.clone())}  # for the relerr against the oracle, below

    # ---- end to end through the public API with host buffers ----
    e2e_ms = []
    for _ in range(max(2, args.steps // 2)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Dg.t().copy_(Dh, non_blocking=True)
        _, _, _ = solve()
        Ah.copy_(A.t(), non_blocking=True)
        Eh.copy_(E.t(), non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_val = job_rate(ws, 1, max_over_ranks(dist, float(np.mean(e2e_ms)), "cuda"))
    roof = roofline(torch, args.headline, apply_ms, apply_n, apply_work, clocks, args.workload,
                    info["rank"] + 1, apply_recs)

    # ---- the other precision modes, each as a sub-object ----
    legs = {}
    if not args.no_mixed:
        for mode in [x for x in ("fp64", "mixed", "fp64tc") if x != args.headline]:
            c2 = blws.Context(k=args.k, device=local_rank, precision=PRECISIONS[mode], graphs=args.graphs,
                              tune=args.tune)
            for _ in range(args.warmup):
                solve(c2)
            ms2 = []
            c2.timing_start()
            for _ in range(args.steps):
                flush.zero_()
                ev0 = torch.cuda.Event(enable_timing=True)
                ev1 = torch.cuda.Event(enable_timing=True)
                ev0.record(stream)
                _, _, i2 = solve(c2)
                ev1.record(stream)
                ev1.synchronize()
                ms2.append(ev0.elapsed_time(ev1))
            a_ms, a_n, a_work = c2.timing_stop()
            a_recs = c2.timing_records()
            kept[mode] = (A.clone(), E.clone())
            legs[mode] = {
                "value": job_rate(ws, args.steps, max_over_ranks(dist, float(np.sum(ms2)), "cuda")),
                "unit": "solves/s", "ms_per_step": float(np.mean(ms2)),
                "latency_ms": {"p50": float(np.percentile(ms2, 50)), "p99": float(np.percentile(ms2, 99))},
                "dtype": MODE_DTYPE[mode], "iters": i2["iters"], "mixed_iters": i2["mixed_iters"],
                "residual": i2["residual"],
                "relerr_vs_planted": float(torch.linalg.norm(A - torch.from_numpy(L0).cuda()) / np.linalg.norm(L0)),
                "roofline": roofline(torch, mode, a_ms, a_n, a_work, clocks, args.workload, i2["rank"] + 1,
                                     a_recs)}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    fullsvd = None
    if not args.no_fullsvd and ws == 1:
        lam = 1.0 / math.sqrt(max(m, n))
        fullsvd = fullsvd_gpu_sample(torch, Dg, lam, info["iters"])
    # the other workloads of the metric, each as a compact sub-object: matrix
    # completion (5000^2, rank 50, 10% observed), the uneven batch (256
    # instances through the server) and one rate of the serving loop
    extra = {}
    if not args.no_extra_legs and ws == 1:
        sub = argparse.Namespace(**vars(args))
        sub.workload, sub.precision, sub.steps, sub.warmup, sub.profile_solve = (
            "mc_5000x5000_r50", "fp64", 3, 1, False)
        mcl = run_mc(sub)
        extra["mc"] = {k: mcl[k] for k in ("value", "unit", "ms_per_step", "latency_ms", "solve",
                                             "roofline", "config")}
        extra["mc"]["steps"], extra["mc"]["warmup"] = sub.steps, sub.warmup
        extra["mc"]["oracle_parity"] = mc_oracle_parity(torch)
        sub = argparse.Namespace(**vars(args))
        sub.precision, sub.batch_count, sub.workers = "fp64tc", 256, 16
        bl = run_batch(sub)
        extra["batch"] = {k: bl[k] for k in ("value", "unit", "config", "solved_ok", "relerr_vs_planted",
                                             "latency_ms", "sequential", "speedup_vs_sequential")}
        sub = argparse.Namespace(**vars(args))
        sub.precision, sub.serve_rates, sub.serve_requests, sub.workers = "fp64", [0.5], 24, 16
        sv = run_serve(sub)
        extra["serve"] = {"capacity_solves_per_s": sv["value"], "config": sv["config"],
                          "rate": sv["sweep"][0]}
    cpu = None
    rel_oracle = {}
    if not args.no_cpu_baseline and ws == 1:
        cpu, ref = cpu_oracle_solve(D, args.tol)
        for mode, (Am, Em) in kept.items():
            rel_oracle[mode] = {"A": relerr_to(torch, Am, ref["A"]), "E": relerr_to(torch, Em, ref["E"])}
    lat = np.array(step_ms)
    out = {
        "metric": "rpca_solves_per_s",
        "value": value,
        "unit": "solves/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": float(np.mean(step_ms)),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "m": m, "n": n, "rank": r, "corrupt": f,
                   "tol": args.tol, "k": args.k, "precision": args.headline,
                   "arithmetic": MODE_DTYPE[args.headline],
                   "l2": "flushed between steps (512 MB write)",
                   "graphs": args.graphs, "tune": args.tune,
                   "parallelism": "replicas" if ws > 1 else "single"},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "max": float(lat.max())},
        "solve": {"iters": info["iters"], "rank": info["rank"], "nnzE": info["nnzE"],
                  "residual": info["residual"], "relerr_vs_planted": relerr,
                  "relerr_vs_oracle": rel_oracle.get(args.headline)},
        "e2e": {"value": e2e_val, "unit": "solves/s", "h2d_bytes_per_step": m * n * 8,
                "d2h_bytes_per_step": 2 * m * n * 8},
        "gpu_launches": int(launches),
        "roofline": roof,
        "clocks": clocks,
        "wall_s": t_wall,
    }
    if cpu:
        out["cpu_baseline"] = cpu
    for mode, leg in legs.items():
        leg["relerr_vs_oracle"] = rel_oracle.get(mode)
        out[LEG_KEY[mode]] = leg
    if fullsvd:
        out["fullsvd_same_gpu"] = fullsvd
        out["fullsvd_same_gpu"]["blws_speedup"] = value / fullsvd["value"]
    out.update(extra)
    print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
