"""A level split by target ranges, each range applied through the library as a
level of its own: targets = the range, sources = the cells its lists read
(ncells_tgt != ncells_src, lists re-indexed into the gathered sources), as
one rank of the sharded path would run it after the multipole exchange
(target cells are independent, Eq. (7); the halo is |t|_inf <= 3, Sec. 3.2).
The concatenated shards are compared with the oracle's unsharded level."""
import numpy as np
import pytest

import oracle
from gpu_helpers import TOL, device, gpu_ops, pruned_cells

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


@pytest.mark.parametrize("world", [2, 3, 4])
@pytest.mark.parametrize("full", [True, False])
def test_sharded_level_matches_oracle(m2l, world, full):
    from paper_1210_7292_gb300 import shard, synth
    ell, level = 4, 4
    cells = synth.full_grid(level) if full else pruned_cells(level, 0.7, 41)
    w = synth.gaussian_vectors(len(cells), ell ** 3, seed=42)
    off, src = oracle.interaction_lists(cells, cells)
    ref = oracle.m2l_apply(oracle.operator_table(ell, oracle.KIND_INV_R, 0.0, level), cells, cells, off, src, w)
    ops = gpu_ops(m2l, ell, 0, level)
    for prec, dt in (("fp64", torch.float64), ("fp32", torch.float32), ("bf16x3", torch.float32)):
        parts = []
        for rank in range(world):
            sh = shard.shard_level(off, src, rank, world)
            t0, t1, need = sh["t0"], sh["t1"], sh["needed"]
            assert len(need) != t1 - t0          # a shard's source set is not its target set
            tgt = torch.from_numpy(np.ascontiguousarray(cells[t0:t1])).to(device())
            srcs = torch.from_numpy(np.ascontiguousarray(cells[need])).to(device())
            lv = m2l.Level(oracle.cell_width(level), tgt, srcs, torch.from_numpy(sh["offsets"]).to(device()),
                           torch.from_numpy(sh["sources"]).to(device()), level)
            assert lv.struct.ncells_tgt == t1 - t0 and lv.struct.ncells_src == len(need)
            halo = torch.from_numpy(np.ascontiguousarray(w[need])).to(device(), dt)
            loc = torch.zeros(t1 - t0, ell ** 3, dtype=dt, device=device())
            m2l.m2l_apply_level(ops, lv, halo, loc, prec)
            m2l.m2l_sync_status(ops)
            parts.append(loc.double().cpu().numpy())
        got = np.concatenate(parts, axis=0)
        err = oracle.rel_l2(got, ref)
        print("%d shards (%s, %d cells), %s: rel L2 vs oracle %.2e" % (world, "full" if full else "pruned",
                                                                       len(cells), prec, err))
        assert err < TOL[prec], (prec, err)
