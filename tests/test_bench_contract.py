"""The benchmark's JSON contract, on the CPU: the reference arm (the oracle timed on a bounded
sample) prints one line with the keys the driver reads, and the roofline of a stage is taken
against the unit that bounds it."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "config", "e2e", "cpu_baseline"):
        assert k in d, k
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    assert d["config"]["workload"].startswith("mie-N64-M128")


def test_roofline_picks_the_bounding_unit():
    clk = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}
    tensor_stage = {"name": "recon_part", "ms": 100.0, "launches": 3, "flops": 4.4e12,
                    "bytes": 1e9, "tc_flops": 1.2e14}
    fp64_stage = {"name": "eigen", "ms": 150.0, "launches": 10, "flops": 6.2e10,
                  "bytes": 4e8, "tc_flops": 0.0}
    r = bench.roofline([tensor_stage, fp64_stage], clk, "mixed")
    assert r["bound"] == "alu" and r["kernel_stage"] == "eigen"
    assert abs(r["achieved"] - 6.2e10 / 0.150 / 1e12) < 1e-9
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    r = bench.roofline([dict(tensor_stage, ms=200.0), fp64_stage], clk, "mixed")
    assert r["bound"] == "tensor" and r["kernel_stage"] == "recon_part"
    # achieved: the algorithmic (FP64-equivalent) rate; peak: the BF16 rate scaled by the
    # algorithmic FLOPs per slice-product FLOP, so frac is also the slice products' BF16 fraction
    assert abs(r["achieved"] - 4.4e12 / 0.200 / 1e12) < 1e-9
    assert abs(r["slice_products_tflops"] - 1.2e14 / 0.200 / 1e12) < 1e-9
    assert abs(r["peak"] - r["bf16_peak"] * 4.4e12 / 1.2e14) < 1e-9
    assert abs(r["frac"] - r["slice_products_tflops"] / r["bf16_peak"]) < 1e-12
    assert r["unit"] == "TFLOP/s"


def test_roofline_headline_skips_a_concurrent_stage():
    # the side-stream stage's time spans its fork to its join and overlaps the eigen stage:
    # it is reported per stage, never as the headline's dominant stage
    clk = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}
    side = {"name": "side_ops", "ms": 400.0, "launches": 18, "flops": 1e12, "bytes": 1e9,
            "tc_flops": 2.8e13}
    fp64_stage = {"name": "eigen", "ms": 110.0, "launches": 14, "flops": 6.2e10,
                  "bytes": 4e8, "tc_flops": 0.0}
    r = bench.roofline([side, fp64_stage], clk, "mixed")
    assert r["kernel_stage"] == "eigen"
    entry = next(e for e in r["per_stage"] if e["stage"] == "side_ops")
    assert "concurrent" in entry
