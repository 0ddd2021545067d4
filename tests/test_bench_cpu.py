"""The benchmark's CPU baselines on a tiny sample (no GPU): the paper-style
blocked CPU M2L (per-class BLAS products) must reproduce the oracle."""
import pytest


def test_nablk_baseline_matches_oracle():
    import bench
    import oracle
    oracle.build_c()
    ref, loc = bench.cpu_oracle_sample(ntargets=48, seed=3, with_locals=True)
    out = bench.cpu_nablk_sample(ntargets=48, seed=3, ref=loc)
    assert out["rel_l2_vs_oracle"] < 1e-13, out
    assert out["value"] > 0 and ref["value"] > 0
    info = bench.host_info()
    assert info["cpu_count"] >= 1 and info["model"]


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference runs the oracle on the host and prints one JSON
    line with the keys of the benchmark contract (no GPU needed)."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["steps"] == 1 and line["warmup"] == 3 and line["n_gpus"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["value"] == line["value"] and line["e2e"]["h2d_bytes_per_step"] == 0
