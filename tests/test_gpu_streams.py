"""Concurrent levels: per-level plans re-classified (m2l_plan_classify) and
applied on separate CUDA streams after m2l_ops_prepare, against the oracle;
and a plan re-classified with another level's lists."""
import numpy as np
import pytest

import oracle
from gpu_helpers import TOL, device, gpu_ops, make_level, oracle_ops, pruned_cells

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def m2l():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()
    from paper_1210_7292_gb300 import m2l as mod
    return mod


@pytest.mark.parametrize("split", [False, True])
@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "tf32x3"])
def test_levels_on_concurrent_streams(m2l, prec, split):
    """Levels 2-4 of a pruned tree, ell = 4, 1/r (one homogeneous operator set),
    classified and applied on three streams at once, twice in a row.  With
    split, the levels classify as soon as the tables are rebuilt, while the
    operators are assembled and prepared on the current stream."""
    ell = 4
    ops = gpu_ops(m2l, ell, 0, 2)
    data = {}
    for level, keep in ((2, 1.0), (3, 0.8), (4, 0.4)):
        cells = pruned_cells(level, keep, seed=50 + level)
        w = np.random.default_rng(60 + level).standard_normal((len(cells), ell ** 3))
        lv = make_level(m2l, cells, level)
        data[level] = (cells, w, lv)
    plans = {L: m2l.m2l_plan_create(ops, data[L][2]) for L in data}
    streams = {L: torch.cuda.Stream() for L in data}
    outs = {}
    for rep in range(2):
        cur = torch.cuda.current_stream()
        tables = torch.cuda.Event()
        if split:
            m2l.m2l_ops_rebuild_tables(ops, cur)
            tables.record(cur)
            m2l.m2l_ops_rebuild_operators(ops, cur)
        else:
            m2l.m2l_ops_rebuild(ops, cur)
        m2l.m2l_ops_prepare(ops, prec, cur)
        ready = torch.cuda.Event()
        ready.record(cur)
        for L, (cells, w, lv) in data.items():
            s = streams[L]
            s.wait_event(tables if split else ready)
            with torch.cuda.stream(s):
                outs[L] = torch.zeros(len(cells), ell ** 3, dtype=torch.float32, device=device())
                win = torch.from_numpy(w).to(device(), torch.float32)
            m2l.m2l_plan_classify(plans[L], lv, s)
            s.wait_event(ready)
            m2l.m2l_plan_apply(plans[L], win, outs[L], prec, stream=s)
            done = torch.cuda.Event()
            done.record(s)
            cur.wait_event(done)
        torch.cuda.synchronize()
        m2l.m2l_sync_status(ops)
        for L, (cells, w, lv) in data.items():
            off, src = oracle.interaction_lists(cells, cells)
            ref = oracle.m2l_apply(oracle_ops(ell, 0, L), cells, cells, off, src, w)
            err = oracle.rel_l2(outs[L].double().cpu().numpy(), ref)
            assert err < TOL[prec], (rep, L, prec, err)


def test_plan_reclassified_with_another_level(m2l):
    """A plan created on level 4 and re-classified with level 3's lists (fewer
    entries, same buffers) applies level 3; then level 4 again."""
    ell = 3
    ops = gpu_ops(m2l, ell, 1, 3)
    c4, c3 = pruned_cells(4, 0.5, 71), pruned_cells(3, 0.9, 72)
    lv4, lv3 = make_level(m2l, c4, 4), make_level(m2l, c3, 3)
    plan = m2l.m2l_plan_create(ops, lv4)
    for cells, lv, level in ((c3, lv3, 3), (c4, lv4, 4)):
        m2l.m2l_plan_classify(plan, lv)
        w = np.random.default_rng(level).standard_normal((len(cells), ell ** 3))
        out = torch.zeros(len(cells), ell ** 3, dtype=torch.float64, device=device())
        m2l.m2l_plan_apply(plan, torch.from_numpy(w).to(device()), out, "fp64")
        m2l.m2l_sync_status(ops)
        off, src = oracle.interaction_lists(cells, cells)
        ref = oracle.m2l_apply(oracle_ops(ell, 1, level), cells, cells, off, src, w)
        assert oracle.rel_l2(out.cpu().numpy(), ref) < TOL["fp64"]
        counts, _ = m2l.m2l_plan_query(plan)
        assert int(counts.sum()) == len(src)
