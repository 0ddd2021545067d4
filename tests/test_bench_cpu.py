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
