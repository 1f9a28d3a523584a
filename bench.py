"""Benchmark: Newton iterations per second of the primal-dual affine scaling
solve (one step = one pass of the whole per-iteration path: D = x/s, r = A x,
M = A D A', Cholesky, triangular solves / FP64 refinement, directions, psi and
the step) on the dense LP m = 8192, n = 32768 with A stored in BF16
(columns scaled by U(0.1, 10)), seeded synthetic data.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on a bounded sample of the same workload instead.  --gpus N > 1 (under
torchrun) runs N independent replicas, one LP per GPU: the single-LP path
does not shard.
"""
from __future__ import annotations

import argparse
import json
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

FORM_DTYPE_LABEL = {"fp64": "f64", "fp32_ir": "f32-f64", "bf16_ir": "bf16-f32-f64", "tf32_ir": "tf32-f32-f64"}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return dict(hbm=p["hbm_gbs"], bf16=p["bf16_tflops"], bf16_sus=p.get("bf16_tflops_sustained", p["bf16_tflops"]),
                    sm_max_mhz=p.get("sm_max_mhz", 2070.0), source="measured")
    return dict(hbm=6800.0, bf16=1900.0, bf16_sus=1700.0, sm_max_mhz=2070.0, source="fallback")


# DRAM bytes (read + write) per launch of the normal-matrix kernel from one
# ncu capture (dram__bytes_read.sum + dram__bytes_write.sum, one pass) of
# `bench.py --kernel normal` on this workload; profiles/syrk_tc_bf16x3_8192x32768.md.
# Valid only for the kernel as captured.  The kernel's source has changed
# since (the TF32 template parameters; the BF16 loads and tile order are as
# captured), so the roofline reports traffic as null and this figure under
# traffic_at_capture until a new capture.
SYRK_TRAFFIC_AT_CAPTURE = {("dense_8192x32768_bf16_colscaled", 3): 10.32e9 + 0.131e9}


def form_terms(form, splits):
    """Products per K step of the tensor-core normal matrix: BF16, the split
    terms of D.*A (default 3); TF32, 3 (TF32 x 3, the default) or 1."""
    if form == "bf16_ir":
        return splits or 3
    if form == "tf32_ir":
        return 1 if splits == 1 else 3
    return 1


def syrk_roofline(form, m, n, splits, ms_per_launch, peaks, workload=None):
    """Roofline record of the normal-matrix kernel.  Algorithmic work is one
    lower-triangle product, m(m+1)/2 entries of n multiply-adds (m^2 n flops,
    FMA = 2); the tensor-core forms execute that product once per split term
    of D.*A, reported separately as executed work."""
    terms = splits if form in ("bf16_ir", "tf32_ir") else 1
    flops = float(m) * (m + 1) * n
    achieved = flops / (ms_per_launch * 1e-3) / 1e12
    if form == "bf16_ir":
        bound, peak, note = "tensor", peaks["bf16_sus"], "bf16 dense, sustained, of %s" % peaks["source"]
    elif form == "tf32_ir":
        bound, peak, note = "tensor", peaks["bf16_sus"] * 1.1 / 2.25, "tf32 = bf16 sustained x 1.1/2.25 nominal ratio"
    elif form == "fp32_ir":
        bound, peak, note = "alu", fp32_simt_peak(peaks), "FP32 SIMT from unit counts"
    else:
        bound, peak, note = "alu", 1.25, "FP64 nominal 1.25 TFLOP/s (no measured FP64 peak)"
    traffic = None
    captured = SYRK_TRAFFIC_AT_CAPTURE.get((workload, terms)) if form == "bf16_ir" else None
    return dict(bound=bound, achieved=round(achieved, 3), peak=round(peak, 3), unit="TFLOP/s",
                frac=round(achieved / peak, 4), traffic=traffic, kernel="normal-matrix k_syrk_tc (a3)",
                peak_note=note, algorithmic_flops_per_launch=flops, ms_per_launch=round(ms_per_launch, 4),
                split_terms=terms, executed_flops_per_launch=flops * terms,
                executed_frac=round(achieved * terms / peak, 4), traffic_at_capture=captured)


def fp32_simt_peak(peaks):
    """152 SMs x 128 FP32 lanes x 2 flops x the maximum SM clock (TFLOP/s)."""
    return 152 * 128 * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12


def chol_roofline(form, m, ms_per_launch, peaks):
    """Roofline record of the Cholesky factor: m^3/3 flops.  The FP32 tile
    factor of the mixed forms runs its trailing products (~97% of the flops)
    on the tensor cores as six BF16 products per FP32-grade product, so its
    roof is the sustained BF16 peak / 6; the fraction of the FP32 SIMT peak is
    given beside it.  The FP64 form's factor runs on the FP64 pipes."""
    flops = float(m) ** 3 / 3.0
    achieved = flops / (ms_per_launch * 1e-3) / 1e12
    if form == "fp64":
        return dict(bound="alu", achieved=round(achieved, 3), peak=1.25, unit="TFLOP/s",
                    frac=round(achieved / 1.25, 4), traffic=None, kernel="blocked FP64 Cholesky (a4)",
                    peak_note="FP64 nominal 1.25 TFLOP/s (no measured FP64 peak)",
                    algorithmic_flops_per_launch=flops, ms_per_launch=round(ms_per_launch, 4))
    peak = peaks["bf16_sus"] / 6.0
    simt = fp32_simt_peak(peaks)
    return dict(bound="tensor", achieved=round(achieved, 3), peak=round(peak, 3), unit="TFLOP/s",
                frac=round(achieved / peak, 4), traffic=None, kernel="k_chol_tiles<float> (a4)",
                peak_note="FP32-grade products as 6 BF16 MMAs: bf16 dense sustained / 6, of %s; the factor "
                          "is bound by its chain of diagonal tasks" % peaks["source"],
                fp32_simt_peak=round(simt, 3), fp32_simt_frac=round(achieved / simt, 4),
                algorithmic_flops_per_launch=flops, ms_per_launch=round(ms_per_launch, 4))


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


def oracle_sample(lp, band_rows=64, chol_m=2048):
    """Time the FP64 CPU oracle on a bounded sample of one Newton iteration of
    this LP and project the full iteration.  Returns (seconds per iteration,
    cores, description)."""
    import oracle
    A64 = lp.A64
    m, n = A64.shape
    x, s = lp.x0, lp.s0
    t = {}
    t0 = time.perf_counter()
    D = oracle.scaling(x, s)
    r = oracle.gemv(A64, x)
    t["rhs"] = time.perf_counter() - t0
    # normal matrix: a band of the last rows (the longest), scaled by entries
    band = min(band_rows, m)
    p0 = m - band
    t0 = time.perf_counter()
    oracle.normal_rows(A64, D, p0, m)
    t_band = time.perf_counter() - t0
    band_entries = sum(p + 1 for p in range(p0, m))
    t["normal"] = t_band * (m * (m + 1) / 2) / band_entries
    # Cholesky and triangular solves on a chol_m x chol_m normal matrix of the
    # same family, scaled by (m / chol_m)^3 and (m / chol_m)^2
    mc = min(chol_m, m)
    nc = min(n, 4 * mc)
    Mc = oracle.normal_matrix(A64[:mc, :nc], D[:nc])
    t0 = time.perf_counter()
    Lc, fail = oracle.cholesky(Mc)
    t["factor"] = (time.perf_counter() - t0) * (m / mc) ** 3
    t0 = time.perf_counter()
    oracle.backward(Lc, oracle.forward(Lc, r[:mc]))
    t["solve"] = (time.perf_counter() - t0) * (m / mc) ** 2
    t0 = time.perf_counter()
    dy = np.zeros(m)
    w = oracle.gemv_t(A64, dy)
    ds = -w
    dx = D * w - x
    t["direction"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    p = oracle.psi(x, s, dx, ds)
    oracle.step(x, lp.y0, s, dx, dy, ds, oracle.theta(p, ALPHA))
    t["step"] = time.perf_counter() - t0
    total = sum(t.values())
    desc = ("one Newton iteration at %dx%d projected from: full A x, A'dy, psi and step; normal-matrix rows "
            "%d..%d (%d of %d lower entries) scaled by entry count; Cholesky + triangular solves of a %dx%d "
            "normal matrix scaled by (m/%d)^3 and ^2" % (m, n, p0, m - 1, band_entries, m * (m + 1) // 2, mc, mc,
                                                          mc))
    return total, oracle.threads(), desc, {k: round(v, 3) for k, v in t.items()}


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


def run_reference(args):
    world, rank, _ = dist_info()
    if rank != 0:
        return
    lp = lpgen.workload(args.workload, seed=0)
    samples = []
    for i in range(args.warmup + args.steps):
        sec, cores, desc, parts = oracle_sample(lp, band_rows=16, chol_m=1024)
        if i >= args.warmup:
            samples.append(sec)
    sec = sum(samples) / len(samples)
    value = 1.0 / sec
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=args.gpus, steps=args.steps, warmup=args.warmup,
                ms_per_step=sec * 1e3, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64",
                data="synthetic", impl="reference",
                config=dict(workload=args.workload, m=lp.m, n=lp.n, alpha=ALPHA, l2="inputs larger than L2"),
                cpu_baseline=dict(value=value, unit=UNIT, cores=cores, kind="oracle", sample=desc),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line))


def run_normal_only(args):
    """Times the normal-matrix stage alone (pdas_form_normal: D = x/s and
    M = A D A' at the seeded start), for kernel profiles and the roofline."""
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
    S = P.Solver(lp.m, lp.n, args.form, a_dtype, **opts)
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
    roof = syrk_roofline(args.form, lp.m, lp.n, splits, ms, peaks, args.workload)
    out = dict(kernel="normal-matrix", workload=args.workload, form=args.form, splits=splits, ms_per_launch=ms,
               launches=prof["launches"], wall_s=wall, roofline=roof)
    if factor:
        out["factor_ms"] = fms / args.steps
        out["factor_roofline"] = chol_roofline(args.form, lp.m, fms / args.steps, peaks)
    print(json.dumps(out))


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
        info = one_step()
        ox.copy_(x, non_blocking=True)
        oy.copy_(y, non_blocking=True)
        os_.copy_(s, non_blocking=True)
        torch.cuda.synchronize()
    e2e_elapsed = time.perf_counter() - t0
    e2e_value, _ = replica_rate(e2e_elapsed, args.steps, world, device="cuda")
    vec_bytes = 8 * (2 * n + m)

    ttg = None
    # the metric's second half: one full solve from the seeded start (on by
    # default for the mixed forms, ~9 s at 8192 x 32768; the FP64 form's
    # ~110 s solve only with --time-to-gap)
    if args.time_to_gap or (args.form != "fp64" and not args.no_time_to_gap):
        restart()
        torch.cuda.synchronize()
        ta, tb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ta.record(stream)
        out = S.solve(A, b, c, x, y, s, alpha=ALPHA, tol=w["tol"])
        tb.record(stream)
        torch.cuda.synchronize()
        secs = ta.elapsed_time(tb) / 1e3
        ttg = dict(seconds=secs, iters=out["iters"], status=out["status_name"], rel_gap=out["rel_gap"],
                   objective=float(torch.dot(c, x).item()))
    S.close()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    peaks = load_peaks()
    normal_ms = prof["ms"]["normal"] / max(1, prof["calls"]["normal"])
    factor_ms = prof["ms"]["factor"] / max(1, prof["calls"]["factor"])
    # the dominant kernel of the step is reported as "roofline"; both records
    # are listed under "rooflines"
    roofs = [syrk_roofline(args.form, m, n, splits, normal_ms, peaks, args.workload),
             chol_roofline(args.form, m, factor_ms, peaks)]
    roof = max(roofs, key=lambda r: r["ms_per_launch"])
    stages = {k: round(v / max(1, args.steps), 4) for k, v in prof["ms"].items()}
    clocks = clk.summary()
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=elapsed_max * 1e3 / args.steps, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype=FORM_DTYPE_LABEL[args.form], data="synthetic",
                config=dict(workload=args.workload, m=m, n=n, a_storage=lp.storage, form=args.form,
                            splits=splits if args.form in ("bf16_ir", "tf32_ir") else None, alpha=ALPHA,
                            steps_from="seeded interior start (restart after convergence)",
                            l2="inputs larger than L2 (A is %d MB)" % (A.numel() * A.element_size() // 2 ** 20),
                            parallelism="replicas" if world > 1 else "single"),
                roofline=roof, rooflines=roofs, stages_ms_per_step=stages,
                refine_sweeps=[i["refine_sweeps"] for i in infos], used_fp64=[i["used_fp64"] for i in infos],
                gpu_launches=prof["launches"],
                e2e=dict(value=e2e_value, unit=UNIT, h2d_bytes_per_step=vec_bytes, d2h_bytes_per_step=vec_bytes),
                clocks=clocks)
    if ttg:
        line["time_to_gap"] = ttg
    if not args.no_cpu_baseline and world == 1:
        sec, cores, desc, parts = oracle_sample(lp)
        line["cpu_baseline"] = dict(value=1.0 / sec, unit=UNIT, cores=cores, kind="oracle", sample=desc,
                                    projected_seconds_per_iter=round(sec, 2), parts_s=parts)
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def run_batch(args):
    """The batch configuration (512 LPs, m ~ U{16..256}, n = m U{2..4}, FP32,
    gap 1e-7) through pdas_batch: K timed graph replays after W warm-up
    replays, each from the seeded starts; prints one JSON line (not the
    headline metric: total Newton iterations of all LPs per second)."""
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
    for k in range(args.warmup + args.steps):
        x.copy_(x0)
        y.copy_(y0)
        s.copy_(s0)
        out = S.solve()
        if k >= args.warmup:
            times.append(out["ms"])
            iters += int(out["iters"].sum())
    cfg = S.config()
    S.close()
    ms = float(np.sum(times))
    st, cnt = np.unique(out["status"], return_counts=True)
    print(json.dumps(dict(metric="Newton iters/s (batch of 512 small LPs)", value=iters / (ms * 1e-3),
                          unit="Newton iters/s", ms_per_batch=ms / len(times), steps=args.steps, warmup=args.warmup,
                          iterations_per_batch=iters // len(times), higher_is_better=True,
                          config=dict(workload="batch_512_f32", count=len(lps), tol=spec["tol"], alpha=0.95,
                                      buckets=[dict(m_bound=m_, threads=t_, lps=n_) for m_, t_, n_ in cfg]),
                          statuses={str(int(a)): int(b_) for a, b_ in zip(st, cnt)},
                          fp64_tier_iterations=int(out["fp64_iters"].sum()),
                          slowest_lp_ms=float(out["time_us"].max() * 1e-3))))


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
    ap.add_argument("--time-to-gap", action="store_true",
                    help="also time one full solve to the gap tolerance (default for the mixed forms)")
    ap.add_argument("--no-time-to-gap", action="store_true", help="skip the full solve of the mixed forms")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--kernel", choices=["step", "normal", "factor"], default="step",
                    help="normal: time only the normal-matrix stage; factor: also the Cholesky (for profiles)")
    ap.add_argument("--batch", action="store_true", help="time the 512-LP batch configuration instead")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours" and args.kernel == "step" and not args.batch:
        ap.error("--warmup must be >= 3")
    if args.batch:
        run_batch(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.kernel in ("normal", "factor"):
        run_normal_only(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
