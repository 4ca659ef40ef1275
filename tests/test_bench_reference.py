"""The benchmark's reference arm (the oracle timed on the host cores) keeps the
one-line JSON contract; it needs no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "flip_L4", "--steps", "1",
                        "--warmup", "0", "--reference-seconds", "1"], cwd=ROOT, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "flip_L4"
    assert d["metric"] == json.load(open(os.path.join(ROOT, "BASELINE.json")))["metric"]


def test_reference_config_has_the_cuda_arms_keys():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "flip_L4", "--steps", "1",
                        "--warmup", "0", "--reference-seconds", "1"], cwd=ROOT, capture_output=True, text=True,
                       timeout=300)
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["config"]["parallelism"] == "replicas1"


def test_sweep_roofline_of_a_pflip_cycle():
    """The flip / p-flip workload's roofline from per-kind kernel times (no GPU)."""
    sys.path.insert(0, ROOT)
    import bench
    import toric3d_inputs as inp
    w = inp.WORKLOADS["pflip_L32"]
    q, S, steps = inp.n_bits(32), 100_000, 2
    prof = {k: (0.0, 0) for k in ("noise", "syndrome", "flip", "pflip", "bp_step", "bp_decide", "logical", "layout",
                                  "cnn")}
    prof.update(noise=(12.6, 2), syndrome=(14.0, 2), flip=(9.0, 8), pflip=(4.0, 4))
    r = bench.sweep_roofline(prof, w, q, S, steps, 40.0, 6780.0, "test", {"sm_mhz": 2070.0})
    assert r["kernel"] == "k_syndrome" and abs(r["ms_per_application"] - 7.0) < 1e-9
    assert r["bound"] in ("alu", "hbm") and 0 < r["frac"] < 1
    flip = r["kernels_hbm_frac"]["flip"]             # 0.5 B x qubits x S per 1.125 ms application (4 F per cycle)
    assert abs(flip - 0.5 * q * S / 1.125e-3 / 1e9 / 6780.0) < 1e-9
    assert 0 < r["cycle_hbm_frac"] < 1


def test_sweep_roofline_cycle_bound_and_flip_traffic():
    """The cycle's combined bound is the sum over its kernels of the slower of the byte and
    issue bounds, and the flip's DRAM traffic figure applies at the captured noise rates only."""
    sys.path.insert(0, ROOT)
    import dataclasses
    import bench
    import toric3d_inputs as inp
    w = inp.WORKLOADS["pflip_L32"]
    q, S, steps = inp.n_bits(32), 100_000, 5
    prof = {k: (0.0, 0) for k in ("noise", "syndrome", "flip", "pflip", "bp_step", "bp_decide", "logical", "layout",
                                  "cnn")}
    prof.update(noise=(11.4, 5), syndrome=(13.0, 5), flip=(20.5, 20), pflip=(8.5, 10))
    ms = 55.3
    r = bench.sweep_roofline(prof, w, q, S, steps, ms, 6780.0, "test", {"sm_mhz": 2070.0})
    assert r["kernel"] == "k_flip_tiled"
    words = (S + 63) // 64
    hbm, issue = 6780.0e9, 152 * 4 * 2070.0e6
    b = bench.SWEEP_BYTES
    i = bench.SWEEP_INST
    want = (max(b["noise"] * q * S / hbm, i["noise"] * q * words / issue)
            + max(b["syndrome"] * q * S / hbm, i["syndrome"] * q * words / issue)
            + 4 * b["flip"] * q * S / hbm
            + max((b["pflip"] - bench.PFLIP_APPLY_BYTES) * q * S / hbm, i["pflip"] * (q // 3) * words / issue)
            + bench.PFLIP_APPLY_BYTES * q * S / hbm)
    assert abs(r["cycle_bound_ms"] - 1e3 * want) < 1e-9
    assert abs(r["cycle_roofline_frac"] - want / (ms / 1e3 / steps)) < 1e-12
    assert abs(r["traffic"] - bench.FLIP_TRAFFIC * q * S) < 1.0
    # another noise rate: no instruction counts and no traffic figure for it
    w2 = dataclasses.replace(w, p=0.05, q=0.05)
    r2 = bench.sweep_roofline(prof, w2, q, S, steps, ms, 6780.0, "test", {"sm_mhz": 2070.0})
    assert r2["traffic"] is None and "cycle_bound_ms" not in r2
