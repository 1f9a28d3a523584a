"""The benchmark's JSON contract, checked on the CPU: the reference arm
(the oracle timed on the host cores) prints one line with the keys its
readers expect, and the roofline helpers report what they claim."""
import json
import os
import subprocess
import sys

from conftest import ROOT

sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_reference_arm_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "dense_64x128_f64", "--steps", "2", "--warmup", "1"], capture_output=True, text=True,
                         check=True, cwd=ROOT, timeout=600).stdout
    lines = [l for l in out.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "Newton iters/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert abs(d["ms_per_step"] - 1e3 / d["value"]) <= 1e-6 * d["ms_per_step"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    assert d["e2e"] == dict(value=d["value"], unit=d["unit"], h2d_bytes_per_step=0, d2h_bytes_per_step=0)
    assert d["config"]["workload"] == "dense_64x128_f64" and d["config"]["m"] == 64 and d["config"]["n"] == 128


def test_syrk_roofline_arithmetic():
    peaks = dict(bf16_sus=1740.5, source="measured")
    r = bench.syrk_roofline("bf16_ir", 8192, 32768, 3, 4.93, peaks)
    flops = 8192.0 * 8193 * 32768
    assert r["algorithmic_flops_per_launch"] == flops and r["split_terms"] == 3
    assert abs(r["achieved"] - flops / 4.93e-3 / 1e12) < 1e-3
    assert abs(r["frac"] - r["achieved"] / 1740.5) < 1e-4
    assert abs(r["executed_frac"] - 3 * r["achieved"] / 1740.5) < 1e-4
    t = bench.syrk_roofline("tf32_ir", 2048, 8192, bench.form_terms("tf32_ir", 0), 0.188, peaks)
    assert t["split_terms"] == 3 and abs(t["peak"] - 1740.5 * 1.1 / 2.25) < 1e-3


def test_form_terms():
    assert bench.form_terms("bf16_ir", 0) == 3 and bench.form_terms("bf16_ir", 2) == 2
    assert bench.form_terms("tf32_ir", 0) == 3 and bench.form_terms("tf32_ir", 1) == 1
    assert bench.form_terms("tf32_ir", 3) == 3 and bench.form_terms("fp64", 0) == 1


def test_stop_margin_and_traffic_record():
    assert abs(bench.stop_margin(7.66e-9, 1e-8) - 0.1158) < 1e-3
    assert bench.stop_margin(0.0, 1e-8) is None
    assert abs(bench.stop_margin(-9.5e-9, 1e-8) - 0.0223) < 1e-3
    # the SYRK traffic figure is reported only for the kernel source it was captured on
    t = bench.syrk_traffic("dense_8192x32768_bf16_colscaled", 3)
    cap = bench.SYRK_TRAFFIC_CAPTURES[("dense_8192x32768_bf16_colscaled", 3)]
    assert t == (cap["bytes"] if cap["digest"] == bench.syrk_source_digest() else None)
    assert bench.syrk_traffic("dense_4096x16384_bf16_colscaled", 3) is None
    peaks = dict(bf16_sus=1708.8, source="measured", tf32=900.0, fp32=70.0, fp64=1.1)
    assert bench.syrk_roofline("tf32_ir", 2048, 8192, 3, 0.2, peaks)["peak"] == 900.0
    assert bench.syrk_roofline("fp64", 2048, 8192, 1, 30.0, peaks)["peak"] == 1.1
    assert bench.chol_roofline("fp64", 8192, 190.0, peaks)["peak"] == 1.1


def test_both_arms_share_the_config():
    import lpgen
    lp = lpgen.workload("dense_64x128_f64", 0)
    a = bench.bench_config(lp, "dense_64x128_f64", "bf16_ir", 3, 1)
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "dense_64x128_f64", "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                         check=True, cwd=ROOT, timeout=600).stdout
    assert json.loads(out.strip().splitlines()[-1])["config"] == a
