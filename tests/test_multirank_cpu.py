"""Multi-rank paths on CPU (gloo, world size 2): the sharding of one level by
target ranges with the multipole all-gather, and the timing helpers of the
benchmark (barrier, max over ranks).  The oracle stands in for each rank's
apply, so the sharded result must equal the unsharded one bit for bit."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist

    import bench
    import oracle
    from paper_1210_7292_gb300 import shard, synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    level, ell = 3, 3
    rng = np.random.default_rng(21)
    cells = synth.full_grid(level)
    cells = np.ascontiguousarray(cells[rng.random(len(cells)) < 0.8])
    w = synth.gaussian_vectors(len(cells), ell ** 3, seed=22)
    off, src = oracle.interaction_lists(cells, cells)
    ranges = shard.target_ranges(len(cells), world)
    sh = shard.shard_level(off, src, rank, world)
    t0, t1 = ranges[rank]
    mine = torch.from_numpy(w[t0:t1])                       # this rank owns these multipoles
    halo = shard.exchange_multipoles(mine, ranges, sh["needed"]).numpy()
    ops = oracle.operator_table(ell, 0, 0.0, level)
    loc = oracle.m2l_apply(ops, cells[t0:t1], cells[sh["needed"]], sh["offsets"], sh["sources"], halo)
    # the benchmark's helpers
    bench.barrier(world)
    tmax = bench.max_over_ranks(world, float(rank + 1), torch.device("cpu"))
    np.save(os.path.join(out_dir, "loc%d.npy" % rank), loc)
    np.save(os.path.join(out_dir, "tmax%d.npy" % rank), np.array([tmax]))
    dist.destroy_process_group()


def test_two_rank_sharded_level_equals_unsharded(tmp_path):
    import torch.multiprocessing as mp

    import oracle
    from paper_1210_7292_gb300 import shard, synth
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    level, ell = 3, 3
    rng = np.random.default_rng(21)
    cells = synth.full_grid(level)
    cells = np.ascontiguousarray(cells[rng.random(len(cells)) < 0.8])
    w = synth.gaussian_vectors(len(cells), ell ** 3, seed=22)
    off, src = oracle.interaction_lists(cells, cells)
    full = oracle.m2l_apply(oracle.operator_table(ell, 0, 0.0, level), cells, cells, off, src, w)
    got = np.concatenate([np.load(tmp_path / ("loc%d.npy" % r)) for r in range(world)])
    assert np.array_equal(got, full)
    for r in range(world):
        assert float(np.load(tmp_path / ("tmax%d.npy" % r))[0]) == float(world)
    # ranges tile the targets
    rs = shard.target_ranges(len(cells), world)
    assert rs[0][0] == 0 and rs[-1][1] == len(cells) and rs[0][1] == rs[1][0]


def test_shard_halo_is_bounded():
    """A rank reads sources within three cells of its range (|t|_inf <= 3)."""
    import oracle
    from paper_1210_7292_gb300 import shard, synth
    cells = synth.full_grid(4)
    off, src = oracle.interaction_lists(cells, cells)
    for world in (2, 3, 4):
        for r in range(world):
            sh = shard.shard_level(off, src, r, world)
            tz = cells[sh["t0"]:sh["t1"], 2]
            sz = cells[sh["needed"], 2]
            assert sz.min() >= tz.min() - 3 and sz.max() <= tz.max() + 3
            # re-indexed lists address the same global sources in the same order
            glob = sh["needed"][sh["sources"]]
            assert np.array_equal(glob, src[off[sh["t0"]]:off[sh["t1"]]])
