"""The batched-trees workload: 64 independent octrees (N log-uniform in
[1e4, 1e6], uniform cube and sphere surface alternating, leaf levels 3-6,
ell in {4, 5, 6}), kernel 1/sqrt(r^2 + c^2) with c = 0.01, FP32; all levels of
all trees in ONE persistent launch on the CUDA cores, or one per order on the
tensor cores (TF32x3, BF16x3), captured in a CUDA graph and replayed.
Checked against the oracle on sampled targets of every problem."""
import numpy as np
import pytest

import oracle
from gpu_helpers import TOL, device

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

C = 0.01


@pytest.fixture(scope="module")
def m2l():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()
    from paper_1210_7292_gb300 import m2l as mod
    return mod


def _problems(m2l, ntrees):
    from paper_1210_7292_gb300 import synth
    ops_cache, probs = {}, []
    for spec in synth.batched_tree_specs(ntrees, seed=4):
        pts, _ = synth.tree_points(spec)
        ell = spec["ell"]
        for L in range(2, spec["leaf_level"] + 1):
            cells = synth.occupied_cells(pts, L)
            key = (ell, L)
            if key not in ops_cache:
                ops_cache[key] = m2l.m2l_precompute(m2l.M2L_K_INV_SQRT_R2C2, ell, 0.0, oracle.cell_width(L), C)
            ijk = torch.from_numpy(cells).to(device())
            off, src = m2l.m2l_build_lists(ijk, ijk)
            lv = m2l.Level(oracle.cell_width(L), ijk, ijk, off, src, L)
            w = synth.gaussian_vectors(len(cells), ell ** 3, seed=spec["seed"] * 10 + L)
            probs.append({"ops": ops_cache[key], "lv": lv, "cells": cells, "w": w, "ell": ell, "L": L})
    return probs, ops_cache


def _check_sampled(probs, outs, rng, nsamp=6):
    worst = 0.0
    ops_o = {}
    for pr, out in zip(probs, outs):
        if pr["lv"].nnz == 0:
            assert float(out.abs().max()) == 0.0
            continue
        cells, ell, L = pr["cells"], pr["ell"], pr["L"]
        samp = np.unique(rng.choice(len(cells), min(nsamp, len(cells)), replace=False))
        off, src = oracle.interaction_lists(cells[samp], cells)
        if (ell, L) not in ops_o:
            ops_o[(ell, L)] = oracle.operator_table(ell, 2, C, L)
        ref = oracle.m2l_apply(ops_o[(ell, L)], cells[samp], cells, off, src, pr["w"])
        got = out[torch.from_numpy(samp).to(device())].double().cpu().numpy()
        if np.abs(ref).max() > 0:
            worst = max(worst, oracle.rel_l2(got, ref))
    return worst


def test_batched_trees_one_launch_and_graph(m2l):
    probs, _ = _problems(m2l, 64)
    assert len(probs) > 64
    plans = [m2l.m2l_plan_create(p["ops"], p["lv"]) for p in probs]
    ins = [torch.from_numpy(p["w"]).to(device(), torch.float32) for p in probs]
    outs = [torch.zeros(p["lv"].struct.ncells_tgt, p["ell"] ** 3, dtype=torch.float32, device=device()) for p in probs]
    batch = m2l.m2l_batch_create(plans, ins, outs, "fp32")
    info = m2l.m2l_batch_info(batch)
    assert info["tile_width"] in (32, 64) and info["tiles"] > 0
    before = m2l.m2l_launch_count()
    m2l.m2l_batch_run(batch)
    assert m2l.m2l_launch_count() - before == 1          # one persistent launch for all problems
    torch.cuda.synchronize()
    worst = _check_sampled(probs, outs, np.random.default_rng(5))
    assert worst < TOL["fp32"], worst
    eager = [o.clone() for o in outs]
    # capture the launch in a CUDA graph and replay it twice: outputs accumulate
    for o in outs:
        o.zero_()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            m2l.m2l_batch_run(batch, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    for o in outs:
        o.zero_()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    m2l.m2l_sync_status(probs[0]["ops"])
    for o, e in zip(outs, eager):
        if float(e.abs().max()) > 0:
            assert float((o - 2 * e).norm() / (2 * e).norm()) < 1e-5
    nint = sum(p["lv"].nnz for p in probs)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(5):
        g.replay()
    t1.record()
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / 5
    print("batched: %d problems, %d interactions, tile width %d, graph replay %.3f ms, %.3e interactions/s"
          % (len(probs), nint, info["tile_width"], ms, nint / ms * 1e3))


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
def test_batched_trees_tensor_cores(m2l, prec):
    """The same 64 trees on the tcgen05 tensor cores: one persistent launch per
    order (ell^3 = 64, 125, 216) over every tree and level of that order, tile
    shapes from the autotuner, sampled targets against the oracle, and two
    replays of a CUDA graph of the run giving twice the eager result."""
    probs, _ = _problems(m2l, 64)
    plans = [m2l.m2l_plan_create(p["ops"], p["lv"]) for p in probs]
    ins = [torch.from_numpy(p["w"]).to(device(), torch.float32) for p in probs]
    outs = [torch.zeros(p["lv"].struct.ncells_tgt, p["ell"] ** 3, dtype=torch.float32, device=device()) for p in probs]
    batch = m2l.m2l_batch_create(plans, ins, outs, prec)
    groups = m2l.m2l_batch_groups(batch)
    assert sorted(g[0] for g in groups) == sorted({p["ell"] ** 3 for p in probs})
    for _, nt, eg in groups:
        assert nt in (32, 64) and eg in (1, 2)
    before = m2l.m2l_launch_count()
    m2l.m2l_batch_run(batch)
    # per order: gather of the inputs, one persistent tensor-core launch, scatter of the outputs
    assert m2l.m2l_launch_count() - before == 3 * len(groups)
    torch.cuda.synchronize()
    m2l.m2l_sync_status(probs[0]["ops"])
    worst = _check_sampled(probs, outs, np.random.default_rng(7))
    assert worst < TOL[prec], worst
    eager = [o.clone() for o in outs]
    for o in outs:
        o.zero_()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            m2l.m2l_batch_run(batch, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    for o in outs:
        o.zero_()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    m2l.m2l_sync_status(probs[0]["ops"])
    for o, e in zip(outs, eager):
        if float(e.abs().max()) > 0:
            assert float((o - 2 * e).norm() / (2 * e).norm()) < 1e-5
    nint = sum(p["lv"].nnz for p in probs)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(5):
        g.replay()
    t1.record()
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / 5
    print("batched %s: %d problems, %d interactions, groups %s, graph replay %.3f ms, %.3e interactions/s"
          % (prec, len(probs), nint, groups, ms, nint / ms * 1e3))


def test_apply_batch_entry_point(m2l):
    probs, _ = _problems(m2l, 6)
    ins = [torch.from_numpy(p["w"]).to(device(), torch.float32) for p in probs]
    outs = [torch.zeros(p["lv"].struct.ncells_tgt, p["ell"] ** 3, dtype=torch.float32, device=device()) for p in probs]
    m2l.m2l_apply_batch([p["ops"] for p in probs], [p["lv"] for p in probs], ins, outs, "fp32")
    worst = _check_sampled(probs, outs, np.random.default_rng(6))
    assert worst < TOL["fp32"], worst
    # FP64 through the same persistent kernel
    ins64 = [torch.from_numpy(p["w"]).to(device()) for p in probs]
    outs64 = [torch.zeros(p["lv"].struct.ncells_tgt, p["ell"] ** 3, dtype=torch.float64, device=device()) for p in probs]
    m2l.m2l_apply_batch([p["ops"] for p in probs], [p["lv"] for p in probs], ins64, outs64, "fp64")
    worst = _check_sampled(probs, outs64, np.random.default_rng(6))
    assert worst < TOL["fp64"], worst
    # a tensor-core precision through the same entry point (a batch per call)
    outs_tc = [torch.zeros_like(o) for o in outs]
    m2l.m2l_apply_batch([p["ops"] for p in probs], [p["lv"] for p in probs], ins, outs_tc, "tf32x3")
    worst = _check_sampled(probs, outs_tc, np.random.default_rng(6))
    assert worst < TOL["tf32x3"], worst
