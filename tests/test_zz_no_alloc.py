"""m2l_apply_level_noalloc, the entry point for callers that cannot allocate
device memory while they run, checked through the C ABI against
m2l_apply_level (FP32) on two calls in a row.

The second call uses a smaller level than the first, so stale buckets left in
the shared scratch array by the first call would show up as a mismatch.
This file is collected last on purpose.
"""
import numpy as np
import pytest

from gpu_helpers import TOL, device, gpu_ops, make_level, pruned_cells

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


def _rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_apply_level_twice(m2l):
    from paper_1210_7292_gb300 import synth
    ell = 5
    cases = [(synth.full_grid(3), 3), (pruned_cells(3, 0.5, 17), 3)]
    ops = gpu_ops(m2l, ell, 0, 3)
    for cells, level in cases:
        lv = make_level(m2l, cells, level)
        w = torch.from_numpy(synth.gaussian_vectors(len(cells), ell ** 3, seed=len(cells))).to(device(),
                                                                                             torch.float32)
        ref = torch.zeros(len(cells), ell ** 3, dtype=torch.float32, device=device())
        m2l.m2l_apply_level(ops, lv, w, ref, "fp32")
        got = torch.zeros_like(ref)
        m2l.m2l_apply_level_noalloc(ops, lv, w, got)
        m2l.m2l_sync_status(ops)
        err = _rel_l2(got.double().cpu().numpy(), ref.double().cpu().numpy())
        assert err < TOL["fp32"], err


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
