"""Benchmark: Newton iterations per second and time to a relative gap of
1e-8 of the primal-dual affine scaling solve on the dense LP m = 8192,
n = 32768 with A stored in BF16 (columns scaled by U(0.1, 10)), seeded
synthetic data; the mixed-precision form (tensor-core normal matrix, FP32
factor, FP64 refinement) beside the plain FP64 GPU form.

One step = one pass of the whole per-iteration path: D = x/s, r = A x,
M = A D A', Cholesky, triangular solves and FP64 refinement, directions,
psi and the step.  `value` times K such steps of the mixed form from the
seeded start (the first K iterations of a solve, restarted after
convergence); the line also carries both forms' full solves to the gap
(time to gap, iterations, objective, whole-solve iterations per second).

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
(full Newton iterations from the same seeded start) instead.  --gpus N > 1
(under torchrun) runs N independent replicas, one LP per GPU: the single-LP
path does not shard.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import lpgen  # noqa: E402

METRIC = "Newton iters/s & time-to-gap-1e-8, mixed vs FP64 GPU, m=8192 n=32768"
UNIT = "Newton iters/s"
DEFAULT_WORKLOAD = "dense_8192x32768_bf16_colscaled"
ALPHA = 0.95
CSRC = os.path.join(ROOT, "paper_1502_03543_gb300", "csrc")

FORM_DTYPE_LABEL = {"fp64": "f64", "fp32_ir": "f32-f64", "bf16_ir": "bf16-f32-f64", "tf32_ir": "tf32-f32-f64"}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return dict(hbm=p["hbm_gbs"], bf16=p["bf16_tflops"], bf16_sus=p.get("bf16_tflops_sustained", p["bf16_tflops"]),
                    sm_max_mhz=p.get("sm_max_mhz", 2070.0), source="measured")
    return dict(hbm=6800.0, bf16=1900.0, bf16_sus=1700.0, sm_max_mhz=2070.0, source="fallback")


def probe_peaks(device="cuda", n=8192):
    """Dense matmul peaks of the dtypes without a measured figure:
    torch.matmul (cuBLAS) at n^3, best of a few launches timed with CUDA
    events after one warm-up: TF32 (FP32 with TF32 allowed), FP32 (TF32
    off) and FP64.  Returns TFLOP/s (2 n^3 flops per product)."""
    import torch
    saved = torch.backends.cuda.matmul.allow_tf32
    out = {}
    try:
        for name, dt, tf32, reps in (("tf32", torch.float32, True, 10), ("fp32", torch.float32, False, 5),
                                     ("fp64", torch.float64, False, 3)):
            torch.backends.cuda.matmul.allow_tf32 = tf32
            g = torch.Generator(device=device).manual_seed(7)
            a = torch.randn(n, n, dtype=dt, device=device, generator=g)
            b = torch.randn(n, n, dtype=dt, device=device, generator=g)
            c = torch.matmul(a, b)
            torch.cuda.synchronize()
            best = math.inf
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b, out=c)
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1))
            out[name] = round(2.0 * n ** 3 / (best * 1e-3) / 1e12, 2)
            del a, b, c
    finally:
        torch.backends.cuda.matmul.allow_tf32 = saved
        torch.cuda.empty_cache()
    out["how"] = "torch.matmul %d^3 per dtype, best of 10/5/3 after one warm-up, CUDA events, in this run" % n
    return out


# DRAM bytes (read + write) per launch of the BF16 normal-matrix kernel from
# one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum, a single
# pass, one launch) of `bench.py --kernel normal --steps 1 --warmup 1` on this
# workload.  Valid only for the kernel source it was captured on: the digest
# of its sources must match, else the roofline reports traffic as null.
SYRK_TRAFFIC_CAPTURES = {("dense_8192x32768_bf16_colscaled", 3): dict(bytes=10270291456 + 132332800,
                                                                       digest="2ab6bed042edf37a")}
SYRK_SOURCES = ("syrk_tc.cu", "syrk_tc.cuh", "tc_util.cuh")


def syrk_source_digest():
    h = hashlib.sha1()
    for f in SYRK_SOURCES:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def syrk_traffic(workload, terms):
    cap = SYRK_TRAFFIC_CAPTURES.get((workload, terms))
    if cap and cap["digest"] == syrk_source_digest():
        return float(cap["bytes"])
    return None


def form_terms(form, splits):
    """Products per K step of the tensor-core normal matrix: BF16, the split
    terms of D.*A (default 3); TF32, 3 (TF32 x 3, the default) or 1."""
    if form == "bf16_ir":
        return splits or 3
    if form == "tf32_ir":
        return 1 if splits == 1 else 3
    return 1


def fp32_simt_peak(peaks):
    """152 SMs x 128 FP32 lanes x 2 flops x the maximum SM clock (TFLOP/s)."""
    return 152 * 128 * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12


def syrk_roofline(form, m, n, splits, ms_per_launch, peaks, workload=None):
    """Roofline record of the normal-matrix kernel.  Algorithmic work is one
    lower-triangle product, m(m+1)/2 entries of n multiply-adds (m(m+1)n
    flops, FMA = 2); the tensor-core forms execute that product once per
    split term of D.*A, reported separately as executed work.  Peaks: BF16
    sustained from MEASURED_PEAKS.json; TF32, FP32 and FP64 from this run's
    matmul probe when present."""
    terms = splits if form in ("bf16_ir", "tf32_ir") else 1
    flops = float(m) * (m + 1) * n
    achieved = flops / (ms_per_launch * 1e-3) / 1e12
    if form == "bf16_ir":
        bound, peak, note = "tensor", peaks["bf16_sus"], "bf16 dense, sustained, of %s" % peaks["source"]
    elif form == "tf32_ir":
        if "tf32" in peaks:
            bound, peak, note = "tensor", peaks["tf32"], "tf32 dense, burst, of measured (matmul probe)"
        else:
            bound, peak, note = "tensor", peaks["bf16_sus"] * 1.1 / 2.25, "tf32 = bf16 sustained x 1.1/2.25 nominal"
    elif form == "fp32_ir":
        if "fp32" in peaks:
            bound, peak, note = "alu", peaks["fp32"], "fp32 dense, burst, of measured (matmul probe)"
        else:
            bound, peak, note = "alu", fp32_simt_peak(peaks), "fp32 SIMT from unit counts"
    else:
        if "fp64" in peaks:
            bound, peak, note = "alu", peaks["fp64"], "fp64 dense, burst, of measured (matmul probe)"
        else:
            bound, peak, note = "alu", 1.25, "fp64 nominal 1.25 TFLOP/s"
    traffic = syrk_traffic(workload, terms) if form == "bf16_ir" else None
    rec = dict(bound=bound, achieved=round(achieved, 3), peak=round(peak, 3), unit="TFLOP/s",
               frac=round(achieved / peak, 4), traffic=traffic, kernel="normal-matrix k_syrk_tc (a3)",
               peak_note=note, algorithmic_flops_per_launch=flops, ms_per_launch=round(ms_per_launch, 4),
               split_terms=terms, executed_flops_per_launch=flops * terms,
               executed_frac=round(achieved * terms / peak, 4))
    if traffic is not None:
        # algorithmic bytes: A, the split planes of D.*A (terms), the lower triangle of M (FP32)
        alg = 2.0 * m * n * (1 + terms) + 4.0 * m * (m + 1) / 2
        rec["traffic_note"] = ("ncu dram bytes read+write per launch; algorithmic %.3g B (A, %d planes of D.*A, lower M),"
                               " ratio %.2f" % (alg, terms, traffic / alg))
    return rec


def chol_roofline(form, m, ms_per_launch, peaks):
    """Roofline record of the Cholesky factor: m^3/3 flops.  The FP32 tile
    factor of the mixed forms runs its trailing products (~97% of the flops)
    on the tensor cores as six BF16 products per FP32-grade product, so its
    roof is the sustained BF16 peak / 6; the fraction of the FP32 peak is
    given beside it.  The FP64 form's factor runs on the FP64 pipes."""
    flops = float(m) ** 3 / 3.0
    achieved = flops / (ms_per_launch * 1e-3) / 1e12
    if form == "fp64":
        peak = peaks.get("fp64", 1.25)
        note = "fp64 dense, burst, of measured (matmul probe)" if "fp64" in peaks else "fp64 nominal 1.25 TFLOP/s"
        return dict(bound="alu", achieved=round(achieved, 3), peak=round(peak, 3), unit="TFLOP/s",
                    frac=round(achieved / peak, 4), traffic=None, kernel="blocked FP64 Cholesky (a4)",
                    peak_note=note, algorithmic_flops_per_launch=flops, ms_per_launch=round(ms_per_launch, 4))
    peak = peaks["bf16_sus"] / 6.0
    simt = peaks.get("fp32", fp32_simt_peak(peaks))
    return dict(bound="tensor", achieved=round(achieved, 3), peak=round(peak, 3), unit="TFLOP/s",
                frac=round(achieved / peak, 4), traffic=None, kernel="k_chol_tiles<float> (a4)",
                peak_note="FP32-grade products as 6 BF16 MMAs: bf16 dense sustained / 6, of %s; the factor "
                          "is bound by its chain of diagonal tasks" % peaks["source"],
                fp32_peak=round(simt, 3), fp32_frac=round(achieved / simt, 4),
                algorithmic_flops_per_launch=flops, ms_per_launch=round(ms_per_launch, 4))


def stop_margin(gap, tol):
    """|log10(|gap| / tol)| of a finished solve: how far its last gap sits
    from the stop threshold (a run within 1e-3 of it is flagged: one more or
    one fewer iteration there is rounding, not the method).  A negative gap
    (c'x < b'y: the iterate has drifted off primal feasibility) is measured
    by its magnitude and reported beside it."""
    if not (gap != 0 and tol > 0) or math.isnan(gap):
        return None
    return abs(math.log10(abs(gap) / tol))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.tmp,
                                         stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        self.tmp.flush()
        rows = []
        with open(self.tmp.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.tmp.name)
        if not rows:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["unavailable"], samples=0)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, name in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(name)
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(smax) if smax else None,
                    reasons=sorted(reasons), samples=len(rows))


def oracle_iterations(lp, count, budget_s=None):
    """Full Newton iterations of the FP64 CPU oracle from the seeded start
    (direction, psi, theta, step: the algorithm of Section III, nothing
    projected), timed one by one.  Runs `count` iterations, or, when the
    first one shows that `count` would not fit budget_s, as many as fit (at
    least one).  Returns (list of seconds per iteration, threads used)."""
    import oracle
    A64 = lp.A64
    x, y, s = lp.x0.copy(), lp.y0.copy(), lp.s0.copy()
    secs = []
    while len(secs) < count:
        t0 = time.perf_counter()
        d = oracle.direction(A64, x, s)
        th = oracle.theta(oracle.psi(x, s, d["dx"], d["ds"]), ALPHA)
        x, y, s = oracle.step(x, y, s, d["dx"], d["dy"], d["ds"], th)
        secs.append(time.perf_counter() - t0)
        if budget_s is not None and len(secs) == 1 and count > 1:
            count = max(1, min(count, int(budget_s // max(secs[0], 1e-9))))
    return secs, oracle.threads()


def replica_rate(local_elapsed, steps, world, device="cpu"):
    """Whole-job rate of N independent replicas: every rank ran `steps`
    iterations; the job took as long as the slowest rank (max over ranks).
    Returns (iterations per second over all ranks, max elapsed seconds)."""
    import torch
    t = torch.tensor([float(local_elapsed)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    elapsed_max = float(t.item())
    return steps * world / elapsed_max, elapsed_max


def dist_info():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def bench_config(lp, workload, form, splits, world):
    """The config dict of both arms: the workload and the form it is run in."""
    return dict(workload=workload, m=lp.m, n=lp.n, a_storage=lp.storage, form=form,
                splits=splits if form in ("bf16_ir", "tf32_ir") else None, alpha=ALPHA,
                tol=lpgen.WORKLOADS[workload]["tol"],
                steps_from="seeded interior start: the first K iterations of a solve (restart after convergence)",
                l2="inputs larger than L2 (A is %d MB)" % (lp.m * lp.n * lp.A_store.itemsize // 2 ** 20),
                parallelism="replicas" if world > 1 else "single")


def run_reference(args):
    """The reference arm: the FP64 CPU oracle, as it stands, timed on the
    host cores over full Newton iterations from the seeded start.  Each step
    is one whole iteration; W warm-up iterations and K timed ones are run
    when the first iteration shows that they fit --ref-budget seconds, else
    as many timed iterations as fit (at least one) and no warm-up.  `steps`
    and `warmup` report what was run."""
    world, rank, _ = dist_info()
    if rank != 0:
        return
    lp = lpgen.workload(args.workload, seed=0)
    secs, cores = oracle_iterations(lp, 1)
    first = secs[0]
    if (args.warmup + args.steps) * first <= args.ref_budget:
        warm = args.warmup
        secs, cores = oracle_iterations(lp, args.warmup + args.steps)
        timed = secs[warm:]
    else:
        warm = 0
        timed, cores = oracle_iterations(lp, args.steps, budget_s=args.ref_budget)
    sec = sum(timed) / len(timed)
    value = 1.0 / sec
    splits = form_terms(args.form, args.splits)
    sample = ("%d full Newton iteration(s) %d..%d of the solve from the seeded start at %dx%d, each timed whole "
              "(direction, psi, step), after %d untimed" % (len(timed), warm, warm + len(timed) - 1, lp.m, lp.n,
                                                             warm))
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=args.gpus, steps=len(timed), warmup=warm,
                ms_per_step=sec * 1e3, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64",
                data="synthetic", impl="reference",
                config=bench_config(lp, args.workload, args.form, splits, world),
                requested=dict(steps=args.steps, warmup=args.warmup, budget_s=args.ref_budget),
                cpu_baseline=dict(value=value, unit=UNIT, cores=cores, kind="oracle", sample=sample,
                                  seconds_per_iteration=[round(t, 3) for t in timed]),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line))


def run_normal_only(args):
    """Times the normal-matrix stage alone (pdas_form_normal: D = x/s and
    M = A D A' at the seeded start), for kernel profiles and the roofline.
    --tier2: the FP64 tier's formation instead (the handle is moved to the
    tier by one direction under dspread_refactor = 1e-300): the tensor-core
    digit planes when the kept columns fit them (BF16 A), else double-float."""
    import torch

    import paper_1502_03543_gb300 as P
    from paper_1502_03543_gb300 import build as B

    B.build()
    lp = lpgen.workload(args.workload, seed=0)
    a_dtype = torch.bfloat16 if lp.storage == "bf16" else {"f64": torch.float64, "f32": torch.float32}[lp.storage]
    if lp.storage == "bf16":
        A = torch.from_numpy(lp.A_store.view(np.int16)).view(torch.bfloat16).cuda()
    else:
        A = torch.from_numpy(np.ascontiguousarray(lp.A_store)).cuda()
    x = torch.from_numpy(lp.x0).cuda()
    s = torch.from_numpy(lp.s0).cuda()
    opts = {"splits": args.splits} if args.splits else {}
    if args.tier2:
        opts["dspread_refactor"] = 1e-300
    S = P.Solver(lp.m, lp.n, args.form, a_dtype, **opts)
    if args.tier2:
        _, _, _, info = S.direction(A, x, s)
        normal_form = info["normal_form"]
    factor = args.kernel == "factor"
    for _ in range(args.warmup):
        S.form_normal(A, x, s)
        if factor:
            S.factor()
    torch.cuda.synchronize()
    fms = 0.0
    S.profile_enable(True)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        S.form_normal(A, x, s)
        if factor:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            S.factor()
            e1.record()
            torch.cuda.synchronize()
            fms += e0.elapsed_time(e1)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    prof = S.profile_read()
    S.close()
    ms = prof["ms"]["normal"] / max(1, prof["calls"]["normal"])
    splits = form_terms(args.form, args.splits)
    peaks = load_peaks()
    if args.tier2:
        # algorithmic m(m+1)n flops; the digit planes execute 30 pair products
        flops = float(lp.m) * (lp.m + 1) * lp.n
        terms = 30 if normal_form == 4 else 1
        achieved = flops / (ms * 1e-3) / 1e12
        roof = dict(bound="tensor" if normal_form == 4 else "alu", achieved=round(achieved, 3),
                    peak=peaks["bf16_sus"], unit="TFLOP/s", frac=round(achieved / peaks["bf16_sus"], 4),
                    traffic=None, kernel="FP64-tier normal matrix (normal_form %d)" % normal_form,
                    executed_frac=round(achieved * terms / peaks["bf16_sus"], 4), pair_products=terms,
                    peak_note="bf16 dense, sustained, of %s" % peaks["source"])
    else:
        roof = syrk_roofline(args.form, lp.m, lp.n, splits, ms, peaks, args.workload)
    out = dict(kernel="normal-matrix", workload=args.workload, form=args.form, splits=splits, ms_per_launch=ms,
               launches=prof["launches"], wall_s=wall, roofline=roof)
    if factor:
        fac_ms = fms / args.steps
        out["factor_ms"] = fac_ms
        if args.tier2:
            # the FP64 tier's factor: FP64 panels, trailing updates from 34 digit-pair
            # products on the tensor cores; algorithmic m^3/3 flops, also against the FP64 peak
            peaks["fp64"] = probe_peaks(n=4096)["fp64"]
            alg = float(lp.m) ** 3 / 3.0
            ach = alg / (fac_ms * 1e-3) / 1e12
            out["factor_roofline"] = dict(
                bound="tensor", achieved=round(ach, 3), peak=peaks["bf16_sus"], unit="TFLOP/s",
                frac=round(ach / peaks["bf16_sus"], 4), traffic=None,
                kernel="FP64-tier factor (k_dig_diag, k_dig_panel_rows, k_dig_update)",
                executed_frac=round(34 * ach / peaks["bf16_sus"], 4), pair_products=34,
                fp64_peak=peaks["fp64"], fp64_multiple=round(ach / peaks["fp64"], 3),
                algorithmic_flops_per_launch=alg, ms_per_launch=round(fac_ms, 4),
                peak_note="bf16 dense, sustained, of %s; fp64_peak: torch.matmul FP64 4096^3 in this run; "
                          "fp64_multiple = achieved / fp64_peak" % peaks["source"])
        else:
            out["factor_roofline"] = chol_roofline(args.form, lp.m, fac_ms, peaks)
    print(json.dumps(out))


def timed_solve(P, torch, lp, A, a_dtype, form, stream, tol, opts):
    """One full solve from the seeded start through pdas_solve, timed with
    CUDA events on the handle's stream, with the library's per-stage times."""
    dv = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    b, c = dv(lp.b), dv(lp.c)
    x, y, s = dv(lp.x0), dv(lp.y0), dv(lp.s0)
    with P.Solver(lp.m, lp.n, form, a_dtype, stream=stream, **opts) as S:
        torch.cuda.synchronize()
        S.profile_enable(True)
        ta, tb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ta.record(stream)
        out = S.solve(A, b, c, x, y, s, alpha=ALPHA, tol=tol)
        tb.record(stream)
        torch.cuda.synchronize()
        prof = S.profile_read()
    secs = ta.elapsed_time(tb) / 1e3
    margin = stop_margin(out["rel_gap"], tol)
    return dict(form=form, seconds=round(secs, 4), iters=out["iters"], status=out["status_name"],
                rel_gap=out["rel_gap"], objective=float(torch.dot(c, x).item()),
                whole_solve_iters_per_s=round(out["iters"] / secs, 4) if secs > 0 else None,
                stop_margin=round(margin, 4) if margin is not None else None,
                near_threshold=bool(margin is not None and margin < 1e-3), gap_negative=bool(out["rel_gap"] < 0),
                stages_s={k: round(v / 1e3, 3) for k, v in prof["ms"].items() if v},
                gpu_launches=prof["launches"]), (x, y, s)


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1502_03543_gb300 as P
    from paper_1502_03543_gb300 import build as B

    world, rank, local = dist_info()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    B.build()
    w = lpgen.WORKLOADS[args.workload]
    lp = lpgen.workload(args.workload, seed=rank)  # one independent LP per replica
    m, n = lp.m, lp.n
    if lp.storage == "bf16":
        A = torch.from_numpy(lp.A_store.view(np.int16)).view(torch.bfloat16).cuda()
        a_dtype = torch.bfloat16
    else:
        A = torch.from_numpy(np.ascontiguousarray(lp.A_store)).cuda()
        a_dtype = A.dtype
    peaks = load_peaks()
    if not args.no_peak_probe:
        probe = probe_peaks()
        peaks.update({k: v for k, v in probe.items() if k != "how"})
    else:
        probe = None
    dv = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    b, c = dv(lp.b), dv(lp.c)
    x0, y0, s0 = dv(lp.x0), dv(lp.y0), dv(lp.s0)
    x, y, s = x0.clone(), y0.clone(), s0.clone()
    stream = torch.cuda.current_stream()
    opts = {}
    if args.splits:
        opts["splits"] = args.splits
    if args.dspread is not None:
        opts["dspread_refactor"] = args.dspread
    S = P.Solver(m, n, args.form, a_dtype, stream=stream, **opts)
    splits = form_terms(args.form, S.options.splits)

    def restart():
        x.copy_(x0)
        y.copy_(y0)
        s.copy_(s0)

    def one_step():
        st, info = S.step(A, b, c, x, y, s, alpha=ALPHA, raise_on_error=True)
        if st == 2 or info["rel_gap"] < w["tol"]:
            restart()  # converged: the next step starts a fresh solve of the same LP
        return info

    # warm-up from the seeded start
    restart()
    for _ in range(args.warmup):
        one_step()
    restart()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    infos = []
    S.profile_enable(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            infos.append(one_step())
        ev1.record(stream)
        torch.cuda.synchronize()
    prof = S.profile_read()
    S.profile_enable(False)
    elapsed = ev0.elapsed_time(ev1) / 1e3
    value, elapsed_max = replica_rate(elapsed, args.steps, world, device="cuda")

    # end to end through the public API with host buffers: per step the
    # iterate goes up from pinned host memory and comes back down.
    hx, hy, hs = (torch.from_numpy(a.copy()).pin_memory() for a in (lp.x0, lp.y0, lp.s0))
    ox, oy, os_ = (torch.empty_like(a).pin_memory() for a in (hx, hy, hs))
    restart()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for k in range(args.steps):
        src = (hx, hy, hs) if k == 0 else (ox, oy, os_)
        x.copy_(src[0], non_blocking=True)
        y.copy_(src[1], non_blocking=True)
        s.copy_(src[2], non_blocking=True)
        one_step()
        ox.copy_(x, non_blocking=True)
        oy.copy_(y, non_blocking=True)
        os_.copy_(s, non_blocking=True)
        torch.cuda.synchronize()
    e2e_elapsed = time.perf_counter() - t0
    e2e_value, _ = replica_rate(e2e_elapsed, args.steps, world, device="cuda")
    vec_bytes = 8 * (2 * n + m)
    S.close()

    # the metric's second half: full solves to the gap from the seeded start,
    # the mixed form and the plain FP64 GPU form, each through pdas_solve
    ttg, ttg64, comparison = None, None, None
    if not args.no_time_to_gap:
        ttg, _ = timed_solve(P, torch, lp, A, a_dtype, args.form, stream, w["tol"], opts)
        if args.form != "fp64" and not args.no_fp64_arm:
            ttg64, _ = timed_solve(P, torch, lp, A, a_dtype, "fp64", stream, w["tol"], {})
            comparison = dict(
                mixed_s=ttg["seconds"], fp64_s=ttg64["seconds"], speedup=round(ttg64["seconds"] / ttg["seconds"], 3),
                iters_mixed=ttg["iters"], iters_fp64=ttg64["iters"],
                iteration_counts_equal=ttg["iters"] == ttg64["iters"],
                objective_rel_diff=abs(ttg["objective"] - ttg64["objective"]) / abs(ttg64["objective"]),
                note="both stop after the first step with rel_gap < tol; iteration counts can differ by one when "
                     "either run ends close to the threshold (see stop_margin)")

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    normal_ms = prof["ms"]["normal"] / max(1, prof["calls"]["normal"])
    factor_ms = prof["ms"]["factor"] / max(1, prof["calls"]["factor"])
    # the dominant kernel of the step is reported as "roofline"; both records
    # are listed under "rooflines"
    roofs = [syrk_roofline(args.form, m, n, splits, normal_ms, peaks, args.workload),
             chol_roofline(args.form, m, factor_ms, peaks)]
    roof = max(roofs, key=lambda r: r["ms_per_launch"])
    stages = {k: round(v / max(1, args.steps), 4) for k, v in prof["ms"].items()}
    clocks = clk.summary()
    fp64_steps = sum(i["used_fp64"] for i in infos)
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=elapsed_max * 1e3 / args.steps, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype=FORM_DTYPE_LABEL[args.form], data="synthetic",
                config=bench_config(lp, args.workload, args.form, splits, world),
                window=dict(iterations="0..%d of the solve from the seeded start" % (args.steps - 1)
                            if args.steps <= (ttg or {}).get("iters", args.steps) else
                            "the solve from the seeded start, restarted after convergence",
                            fp32_tier_steps=args.steps - fp64_steps, fp64_tier_steps=fp64_steps,
                            note="value covers these iterations only; whole_solve_iters_per_s covers a full solve"),
                roofline=roof, rooflines=roofs, stages_ms_per_step=stages,
                refine_sweeps=[i["refine_sweeps"] for i in infos], used_fp64=[i["used_fp64"] for i in infos],
                gpu_launches=prof["launches"],
                e2e=dict(value=e2e_value, unit=UNIT, h2d_bytes_per_step=vec_bytes, d2h_bytes_per_step=vec_bytes),
                clocks=clocks)
    if probe:
        line["peaks_probe"] = probe
    if ttg:
        line["time_to_gap"] = ttg
        line["whole_solve_iters_per_s"] = ttg["whole_solve_iters_per_s"]
    if ttg64:
        line["time_to_gap_fp64"] = ttg64
        line["mixed_vs_fp64"] = comparison
    if not args.no_cpu_baseline and world == 1:
        secs, cores = oracle_iterations(lp, 1)
        line["cpu_baseline"] = dict(value=1.0 / secs[0], unit=UNIT, cores=cores, kind="oracle",
                                    sample="the first Newton iteration of the solve from the seeded start at %dx%d, "
                                           "timed whole (direction, psi, step)" % (m, n),
                                    seconds_per_iteration=[round(t, 3) for t in secs])
    if not args.no_batches and world == 1:
        # the two batch workloads, timed after the headline region (their own
        # modes, --batch and --batch-adjoint, print the full records)
        bt = measure_batch(3, 1)
        line["batch_512_f32"] = dict(value=round(bt["value"], 1), unit=bt["unit"], ms_per_batch=bt["ms_per_batch"],
                                     iterations_per_batch=bt["iterations_per_batch"], statuses=bt["statuses"],
                                     steps=3, warmup=1)
        ad = measure_batch_adjoint(3, 1)
        line["adjoint_256_f32"] = dict(forward_ms=ad["forward_ms"], adjoint_ms=ad["adjoint_ms"],
                                       adjoint_lps_per_s=round(ad["adjoint_lps_per_s"], 1),
                                       adjoint_statuses=ad["adjoint_statuses"], steps=3, warmup=1)
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def measure_batch(steps, warmup):
    """The batch configuration (512 LPs, m ~ U{16..256}, n = m U{2..4}, FP32,
    gap 1e-7) through pdas_batch: K timed graph replays after W warm-up
    replays, each from the seeded starts.  Returns a record (not the headline
    metric: total Newton iterations of all LPs per second)."""
    import torch

    import paper_1502_03543_gb300 as P
    from paper_1502_03543_gb300 import build as B

    B.build()
    spec = lpgen.BATCHES["batch_512_f32"]
    lps = lpgen.batch(spec["count"], seed=spec["seed"], storage=spec["storage"])
    pk = lpgen.pack(lps)
    dv = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    A = torch.from_numpy(np.ascontiguousarray(pk["A"], dtype=np.float32)).cuda()
    b, c = dv(pk["b"]), dv(pk["c"])
    x0, y0, s0 = dv(pk["x0"]), dv(pk["y0"]), dv(pk["s0"])
    x, y, s = x0.clone(), y0.clone(), s0.clone()
    S = P.BatchSolver(pk["m"], pk["n"], A, b, c, x, y, s, tol=spec["tol"])
    times, iters, out = [], 0, None
    for k in range(warmup + steps):
        x.copy_(x0)
        y.copy_(y0)
        s.copy_(s0)
        out = S.solve()
        if k >= warmup:
            times.append(out["ms"])
            iters += int(out["iters"].sum())
    cfg = S.config()
    S.close()
    ms = float(np.sum(times))
    st, cnt = np.unique(out["status"], return_counts=True)
    return dict(metric="Newton iters/s (batch of 512 small LPs)", value=iters / (ms * 1e-3),
                unit="Newton iters/s", ms_per_batch=ms / len(times), steps=steps, warmup=warmup,
                iterations_per_batch=iters // len(times), higher_is_better=True,
                config=dict(workload="batch_512_f32", count=len(lps), tol=spec["tol"], alpha=0.95,
                            buckets=[dict(m_bound=m_, threads=t_, lps=n_) for m_, t_, n_ in cfg]),
                statuses={str(int(a)): int(b_) for a, b_ in zip(st, cnt)},
                fp64_tier_iterations=int(out["fp64_iters"].sum()),
                slowest_lp_ms=float(out["time_us"].max() * 1e-3))


def run_batch(args):
    print(json.dumps(measure_batch(args.steps, args.warmup)))


def measure_batch_adjoint(steps, warmup):
    """The differentiable batch (256 LPs of 128 x 384, FP32, gap 1e-6; loss
    sum_i w_i' x*_i, w ~ N(0,1)): the batch solve and pdas_batch_backward
    (every LP's adjoint in one launch per bucket), K timed repetitions after
    W warm-ups, each from the seeded starts.  Returns a record."""
    import torch

    import paper_1502_03543_gb300 as P
    from paper_1502_03543_gb300 import build as B

    B.build()
    spec = lpgen.BATCHES["adjoint_256_f32"]
    sizes = (np.full(spec["count"], spec["m"]), np.full(spec["count"], spec["n"]))
    lps = lpgen.batch(spec["count"], storage=spec["storage"], sizes=sizes)
    pk = lpgen.pack(lps)
    dv = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    A = torch.from_numpy(np.ascontiguousarray(pk["A"], dtype=np.float32)).cuda()
    b, c = dv(pk["b"]), dv(pk["c"])
    x0, y0, s0 = dv(pk["x0"]), dv(pk["y0"]), dv(pk["s0"])
    x, y, s = x0.clone(), y0.clone(), s0.clone()
    w = dv(np.random.default_rng(0).standard_normal(int(pk["n"].sum())))
    S = P.BatchSolver(pk["m"], pk["n"], A, b, c, x, y, s, tol=spec["tol"])
    fwd, bwd = [], []
    for k in range(warmup + steps):
        x.copy_(x0)
        y.copy_(y0)
        s.copy_(s0)
        out = S.solve()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dA, db, dc, status = S.backward(w)
        t1 = time.perf_counter()
        if k >= warmup:
            fwd.append(out["ms"])
            bwd.append((t1 - t0) * 1e3)
    S.close()
    return dict(metric="differentiable batch: forward solve and batched adjoint (256 LPs of 128x384)",
                forward_ms=float(np.mean(fwd)), adjoint_ms=float(np.mean(bwd)),
                adjoint_lps_per_s=spec["count"] / (float(np.mean(bwd)) * 1e-3),
                forward_statuses={str(int(a)): int(n) for a, n in zip(*np.unique(out["status"],
                                                                                 return_counts=True))},
                adjoint_statuses={str(int(a)): int(n) for a, n in zip(*np.unique(status,
                                                                                 return_counts=True))},
                iterations_per_batch=int(out["iters"].sum()), steps=steps, warmup=warmup,
                adjoint_timing="host wall clock around pdas_batch_backward (it synchronises its stream)",
                config=dict(workload="adjoint_256_f32", count=spec["count"], m=spec["m"], n=spec["n"],
                            tol=spec["tol"], alpha=ALPHA))


def run_batch_adjoint(args):
    print(json.dumps(measure_batch_adjoint(args.steps, args.warmup)))


def run_woodbury(args):
    """The paper's own solver of the normal equations (the Egidi-Maponi
    rank-one recurrence from (A A')^{-1} A, pdas_woodbury.h) against the
    library's FP64 direction on the same workload at the seeded start: one
    JSON line with both times, their agreement and the recurrence's roofline
    (4 m flops per column and step: a dot product and an axpy, FP64)."""
    import torch

    import paper_1502_03543_gb300 as P
    from paper_1502_03543_gb300 import build as B

    B.build()
    lp = lpgen.workload(args.workload, seed=0)
    if lp.storage == "bf16":
        A = torch.from_numpy(lp.A_store.view(np.int16)).view(torch.bfloat16).cuda()
    else:
        A = torch.from_numpy(np.ascontiguousarray(lp.A_store)).cuda()
    dv = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    x, s = dv(lp.x0), dv(lp.s0)
    D = x / s
    ev = lambda: torch.cuda.Event(enable_timing=True)
    with P.Solver(lp.m, lp.n, "fp64", A.dtype) as S:
        r = S.gemv(A, x)
        for _ in range(max(1, args.warmup)):
            S.direction(A, x, s)
        e0, e1 = ev(), ev()
        e0.record()
        for _ in range(args.steps):
            _, dy_chol, _, _ = S.direction(A, x, s)
        e1.record()
        torch.cuda.synchronize()
        chol_ms = e0.elapsed_time(e1) / args.steps
    with P.WoodburySolver(lp.m, lp.n, A.dtype) as W:
        e0, e1 = ev(), ev()
        e0.record()
        W.prepare(A)
        e1.record()
        torch.cuda.synchronize()
        prep_ms = e0.elapsed_time(e1)
        W.solve(A, D, r)  # warm-up
        e0, e1 = ev(), ev()
        e0.record()
        for _ in range(args.steps):
            dy_wb, min_den = W.solve(A, D, r)
        e1.record()
        torch.cuda.synchronize()
        wb_ms = e0.elapsed_time(e1) / args.steps
    m, n = lp.m, lp.n
    flops = 4.0 * m * n * (n + 1) / 2.0
    peaks = load_peaks()
    probe = probe_peaks() if not args.no_peak_probe else {}
    peak = probe.get("fp64", 1.25)
    achieved = flops / (wb_ms * 1e-3) / 1e12
    diff = float((dy_wb - dy_chol).abs().max() / dy_chol.abs().max())
    print(json.dumps(dict(metric="normal-equations solve: Woodbury recurrence vs Cholesky direction (FP64)",
                          workload=args.workload, m=m, n=n, woodbury_solve_ms=round(wb_ms, 3),
                          woodbury_prepare_ms=round(prep_ms, 3), cholesky_direction_ms=round(chol_ms, 3),
                          dy_max_rel_diff=diff, min_den=min_den, steps=args.steps,
                          roofline=dict(bound="alu", achieved=round(achieved, 4), peak=peak, unit="TFLOP/s",
                                        frac=round(achieved / peak, 4), traffic=None,
                                        kernel="k_wb_step (the rank-one recurrence)",
                                        peak_note="fp64 dense, burst, of measured (matmul probe)" if probe else
                                        "fp64 nominal", algorithmic_flops_per_solve=flops,
                                        hbm_bytes_per_solve=16.0 * m * n * (n + 1) / 2.0,
                                        hbm_peak=peaks["hbm"]))))


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(lpgen.WORKLOADS))
    ap.add_argument("--form", default="bf16_ir", choices=sorted(FORM_DTYPE_LABEL))
    ap.add_argument("--splits", type=int, default=0)
    ap.add_argument("--dspread", type=float, default=None, help="dspread_refactor option (<= 0 disables)")
    ap.add_argument("--no-time-to-gap", action="store_true", help="skip the full solves to the gap")
    ap.add_argument("--no-fp64-arm", action="store_true", help="skip the plain FP64 form's full solve")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-peak-probe", action="store_true", help="skip the TF32/FP32/FP64 matmul probe")
    ap.add_argument("--no-batches", action="store_true",
                    help="skip the summaries of the batch and differentiable-batch workloads")
    ap.add_argument("--ref-budget", type=float, default=200.0,
                    help="reference arm: seconds of oracle iterations to fit the run into")
    ap.add_argument("--kernel", choices=["step", "normal", "factor"], default="step",
                    help="normal: time only the normal-matrix stage; factor: also the Cholesky (for profiles)")
    ap.add_argument("--tier2", action="store_true", help="--kernel normal: the FP64 tier's formation")
    ap.add_argument("--batch", action="store_true", help="time the 512-LP batch configuration instead")
    ap.add_argument("--batch-adjoint", action="store_true",
                    help="time the differentiable batch (256 LPs, forward and batched adjoint) instead")
    ap.add_argument("--woodbury", action="store_true",
                    help="time the paper's rank-one (Woodbury) solver against the Cholesky direction instead")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours" and args.kernel == "step" and not (args.batch or args.woodbury or
                                                                                  args.batch_adjoint):
        ap.error("--warmup must be >= 3")
    if args.batch:
        run_batch(args)
    elif args.woodbury:
        run_woodbury(args)
    elif args.batch_adjoint:
        run_batch_adjoint(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.kernel in ("normal", "factor"):
        run_normal_only(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
