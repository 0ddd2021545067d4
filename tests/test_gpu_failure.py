"""Failure detection without a GPU fault: a bounded device wait is made to run
out by a test switch (the producers withhold their first stage signal), the
kernel returns on its own, the host reads M2L_ETIMEOUT, and the context stays
usable for a correct apply afterwards."""
import time

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


def test_bounded_wait_reports_timeout_and_context_survives(m2l):
    level, ell = 3, 4
    cells = pruned_cells(level, 0.6, 50)
    lv = make_level(m2l, cells, level)
    ops = gpu_ops(m2l, ell, 0, level)
    w = np.random.default_rng(51).standard_normal((len(cells), ell ** 3))
    wd = torch.from_numpy(w).to(device(), torch.float32)
    m2l.m2l_ops_set_debug(ops, m2l.M2L_DEBUG_STALL_PRODUCER)
    loc = torch.zeros(len(cells), ell ** 3, dtype=torch.float32, device=device())
    t0 = time.time()
    m2l.m2l_apply_level(ops, lv, wd, loc, "bf16x3")
    with pytest.raises(m2l.M2LError) as ei:
        m2l.m2l_sync_status(ops)
    elapsed = time.time() - t0
    assert ei.value.status == m2l.M2L_ETIMEOUT
    assert elapsed < 30.0
    # the status word was cleared and the context works
    m2l.m2l_ops_set_debug(ops, 0)
    m2l.m2l_sync_status(ops)
    off, src = oracle.interaction_lists(cells, cells)
    ref = oracle.m2l_apply(oracle_ops(ell, 0, level), cells, cells, off, src, w)
    loc.zero_()
    m2l.m2l_apply_level(ops, lv, wd, loc, "bf16x3")
    m2l.m2l_sync_status(ops)
    assert oracle.rel_l2(loc.double().cpu().numpy(), ref) < TOL["bf16x3"]
