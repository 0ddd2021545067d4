"""m2l_apply_level_noalloc, the entry point for callers that cannot allocate
device memory while they run, checked through the C ABI against the oracle
(plain FP64 M2L with directly assembled operators).

The cases cover two calls in a row on levels of different sizes (stale
buckets left in the shared scratch array by the first call would show up as
a mismatch in the second), the largest order the scratch holds (ell = 6), a
level just below the entry limit of 524,288 list entries, an empty level, and
the device memory: once the first call on the device has looked up the
scratch array, a call leaves the free device memory unchanged.
This file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import TOL, device, gpu_ops, make_level, pruned_cells

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NOALLOC_MAX_NNZ = 1 << 19


@pytest.fixture(scope="module")
def m2l():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()
    from paper_1210_7292_gb300 import m2l as mod
    return mod


def _oracle_locals(ell, cells, level, w, f0):
    off, src = oracle.interaction_lists(cells, cells)
    ops = oracle.operator_table(ell, oracle.KIND_INV_R, 0.0, level)
    return f0 + oracle.m2l_apply(ops, cells, cells, off, src, w), len(src)


def _noalloc(m2l, ops, cells, level, ell, seed):
    """One call on seeded multipoles and non-zero starting locals; returns
    (locals before, locals after, multipoles) on the host in FP64."""
    from paper_1210_7292_gb300 import synth
    lv = make_level(m2l, cells, level)
    w = synth.gaussian_vectors(len(cells), ell ** 3, seed=seed).astype(np.float32)
    f0 = synth.gaussian_vectors(len(cells), ell ** 3, seed=seed + 1).astype(np.float32)
    wd = torch.from_numpy(w).to(device())
    fd = torch.from_numpy(f0).to(device())
    m2l.m2l_apply_level_noalloc(ops, lv, wd, fd)
    m2l.m2l_sync_status(ops)
    return f0.astype(np.float64), fd.double().cpu().numpy(), w.astype(np.float64), lv.nnz


def test_noalloc_matches_oracle_twice(m2l):
    from paper_1210_7292_gb300 import synth
    ell = 5
    ops = gpu_ops(m2l, ell, 0, 3)
    for cells, level in ((synth.full_grid(3), 3), (pruned_cells(3, 0.5, 17), 3)):
        f0, got, w, nnz = _noalloc(m2l, ops, cells, level, ell, seed=len(cells))
        ref, nref = _oracle_locals(ell, cells, level, w, f0)
        assert nnz == nref
        err = oracle.rel_l2(got - f0, ref - f0)
        print("noalloc ell=%d, %d cells, %d entries: rel L2 vs oracle %.2e" % (ell, len(cells), nnz, err))
        assert err < TOL["fp32"], err


def test_noalloc_largest_order(m2l):
    """ell = 6 fills the scratch's operator layout (216 nodes padded to 224 x 256)."""
    from paper_1210_7292_gb300 import synth
    ell, level = 6, 3
    ops = gpu_ops(m2l, ell, 0, level)
    cells = synth.full_grid(level)
    f0, got, w, _ = _noalloc(m2l, ops, cells, level, ell, seed=61)
    ref, _ = _oracle_locals(ell, cells, level, w, f0)
    err = oracle.rel_l2(got - f0, ref - f0)
    print("noalloc ell=6: rel L2 vs oracle %.2e" % err)
    assert err < TOL["fp32"], err


def test_noalloc_near_the_entry_limit(m2l):
    """A pruned level-4 grid with 523,600 list entries, 688 below the limit,
    fills the scratch's bucket arrays almost to their end."""
    ell, level = 4, 4
    cells = pruned_cells(level, 0.945, 7)
    ops = gpu_ops(m2l, ell, 0, level)
    f0, got, w, nnz = _noalloc(m2l, ops, cells, level, ell, seed=71)
    assert 520000 < nnz <= NOALLOC_MAX_NNZ
    ref, nref = _oracle_locals(ell, cells, level, w, f0)
    assert nnz == nref
    err = oracle.rel_l2(got - f0, ref - f0)
    print("noalloc %d entries: rel L2 vs oracle %.2e" % (nnz, err))
    assert err < TOL["fp32"], err


def test_noalloc_empty_levels_leave_locals_unchanged(m2l):
    ell = 4
    ops = gpu_ops(m2l, ell, 0, 3)
    lone = np.array([[3, 3, 3]], dtype=np.int32)        # one cell: no far-field pair
    f0, got, _, nnz = _noalloc(m2l, ops, lone, 3, ell, seed=81)
    assert nnz == 0 and np.array_equal(got, f0)
    none = np.zeros((0, 3), dtype=np.int32)            # no cells at all
    f0, got, _, nnz = _noalloc(m2l, ops, none, 3, ell, seed=82)
    assert nnz == 0 and got.shape == (0, ell ** 3)


def test_noalloc_leaves_free_device_memory_unchanged(m2l):
    """After the first call on this device (which looks up the scratch array),
    further calls allocate nothing: cudaMemGetInfo reports the same free bytes
    before and after each of two calls."""
    from paper_1210_7292_gb300 import synth
    ell, level = 5, 3
    cells = synth.full_grid(level)
    ops = gpu_ops(m2l, ell, 0, level)
    lv = make_level(m2l, cells, level)
    wd = torch.from_numpy(synth.gaussian_vectors(len(cells), ell ** 3, seed=91)).to(device(), torch.float32)
    fd = torch.zeros(len(cells), ell ** 3, dtype=torch.float32, device=device())
    m2l.m2l_apply_level_noalloc(ops, lv, wd, fd)        # first call: set-up on this device
    m2l.m2l_sync_status(ops)
    for _ in range(2):
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        m2l.m2l_apply_level_noalloc(ops, lv, wd, fd)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, (free0, free1)
    m2l.m2l_sync_status(ops)


def test_noalloc_rejects_beyond_its_limits(m2l):
    from paper_1210_7292_gb300 import synth
    ops7 = gpu_ops(m2l, 7, 0, 3)
    cells = synth.full_grid(2)
    lv = make_level(m2l, cells, 2)
    z = torch.zeros(len(cells), 343, dtype=torch.float32, device=device())
    with pytest.raises(m2l.M2LError) as ei:
        m2l.m2l_apply_level_noalloc(ops7, lv, z, z.clone())
    assert ei.value.status == m2l.M2L_EUNSUPPORTED
    ops4 = gpu_ops(m2l, 4, 0, 4)
    big = make_level(m2l, synth.full_grid(4), 4)     # 584,136 entries > 524,288
    z = torch.zeros(4096, 64, dtype=torch.float32, device=device())
    with pytest.raises(m2l.M2LError) as ei:
        m2l.m2l_apply_level_noalloc(ops4, big, z, z.clone())
    assert ei.value.status == m2l.M2L_EINVAL
