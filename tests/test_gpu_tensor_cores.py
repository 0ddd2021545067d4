"""Parity of the tcgen05 tensor-core precisions (TF32, BF16x3, TF32x3) with the
CPU oracle, through the C ABI.  Tolerances per precision in gpu_helpers.TOL."""
import numpy as np
import pytest

import oracle
from gpu_helpers import TOL, device, gpu_ops, make_level, oracle_ops, pruned_cells

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TC = ["tf32", "bf16x3", "tf32x3"]


@pytest.fixture(scope="module")
def m2l():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()
    from paper_1210_7292_gb300 import m2l as mod
    return mod


def _apply(m2l, ops, lv, w, prec, out_fp64=False, init=None):
    dt_out = torch.float64 if out_fp64 else torch.float32
    loc = torch.zeros(lv.struct.ncells_tgt, w.shape[1], dtype=dt_out, device=device())
    if init is not None:
        loc += torch.from_numpy(init).to(device(), dt_out)
    m2l.m2l_apply_level(ops, lv, torch.from_numpy(w).to(device(), torch.float32), loc, prec, out_fp64)
    m2l.m2l_sync_status(ops)
    return loc.double().cpu().numpy()


def _check(got, ref, prec):
    err = oracle.rel_l2(got, ref)
    assert err < TOL[prec], (prec, err)
    assert np.max(np.abs(got - ref)) < 50 * TOL[prec] * np.max(np.abs(ref))
    return err


@pytest.mark.parametrize("prec", TC)
def test_tc_config1_level3(m2l, prec):
    from paper_1210_7292_gb300 import synth
    level, ell = 3, 4
    cells = synth.full_grid(level)
    w = synth.gaussian_vectors(len(cells), ell ** 3, seed=1)
    lv = make_level(m2l, cells, level)
    ops = gpu_ops(m2l, ell, 0, level)
    off, src = oracle.interaction_lists(cells, cells)
    ref = oracle.m2l_apply(oracle_ops(ell, 0, level), cells, cells, off, src, w)
    err = _check(_apply(m2l, ops, lv, w, prec), ref, prec)
    print("config1 %s rel L2 %.3e" % (prec, err))


@pytest.mark.parametrize("prec", TC)
@pytest.mark.parametrize("ell,kind,level,keep", [(5, 0, 4, 0.5), (3, 1, 4, 0.7), (5, 2, 3, 0.9), (2, 0, 2, 1.0),
                                                 (4, 1, 5, 0.03)])
def test_tc_pruned_levels(m2l, prec, ell, kind, level, keep):
    cells = pruned_cells(level, keep, seed=ell * 7 + level)
    rng = np.random.default_rng(ell + 100)
    w = rng.standard_normal((len(cells), ell ** 3))
    init = rng.standard_normal((len(cells), ell ** 3))
    lv = make_level(m2l, cells, level)
    ops = gpu_ops(m2l, ell, kind, level)
    off, src = oracle.interaction_lists(cells, cells)
    ref = oracle.m2l_apply(oracle_ops(ell, kind, level), cells, cells, off, src, w, locals_in=init)
    _check(_apply(m2l, ops, lv, w, prec, init=init), ref, prec)


@pytest.mark.parametrize("prec", TC)
def test_tc_fp64_locals_and_adjoint(m2l, prec):
    level, ell = 3, 5
    cells = pruned_cells(level, 0.75, 31)
    rng = np.random.default_rng(9)
    w = rng.standard_normal((len(cells), ell ** 3))
    lv = make_level(m2l, cells, level)
    ops = gpu_ops(m2l, ell, 0, level)
    off, src = oracle.interaction_lists(cells, cells)
    K = oracle_ops(ell, 0, level)
    _check(_apply(m2l, ops, lv, w, prec, out_fp64=True), oracle.m2l_apply(K, cells, cells, off, src, w), prec)
    ref = oracle.m2l_apply_adjoint(K, cells, cells, off, src, w, len(cells))
    out = torch.zeros(len(cells), ell ** 3, dtype=torch.float32, device=device())
    m2l.m2l_apply_level_adjoint(ops, lv, torch.from_numpy(w).to(device(), torch.float32), out, prec)
    m2l.m2l_sync_status(ops)
    _check(out.double().cpu().numpy(), ref, prec)


def test_tc_level5_sampled(m2l):
    """The benchmark's launch: full level 5, ell = 5, 1/r; 48 sampled targets."""
    from paper_1210_7292_gb300 import synth
    level, ell = 5, 5
    cells = synth.full_grid(level)
    w = synth.gaussian_vectors(len(cells), ell ** 3, seed=2)
    lv = make_level(m2l, cells, level)
    ops = gpu_ops(m2l, ell, 0, level)
    got = {p: _apply(m2l, ops, lv, w, p) for p in TC}
    rng = np.random.default_rng(8)
    samp = np.unique(np.concatenate([[0, len(cells) - 1], rng.choice(len(cells), 46, replace=False)]))
    off, src = oracle.interaction_lists(cells[samp], cells)
    ref = oracle.m2l_apply(oracle_ops(ell, 0, level), cells[samp], cells, off, src, w)
    for p in TC:
        err = _check(got[p][samp], ref, p)
        print("level5 %s rel L2 %.3e" % (p, err))


@pytest.mark.parametrize("prec", TC)
@pytest.mark.parametrize("ell,kind,level,keep", [(6, 2, 3, 0.6), (7, 1, 3, 0.5), (8, 0, 3, 0.15)])
def test_tc_large_orders(m2l, prec, ell, kind, level, keep):
    """ell = 6..8: the operator is streamed through a ring of swizzled blocks and
    the accumulator spans two to four M tiles (ragged last tile included).  Every
    precision fits shared memory, ell 8 TF32x3 with a two-slot ring."""
    cells = pruned_cells(level, keep, seed=ell * 3 + kind)
    rng = np.random.default_rng(ell + 7)
    w = rng.standard_normal((len(cells), ell ** 3))
    lv = make_level(m2l, cells, level)
    ops = gpu_ops(m2l, ell, kind, level)
    off, src = oracle.interaction_lists(cells, cells)
    ref = oracle.m2l_apply(oracle_ops(ell, kind, level), cells, cells, off, src, w)
    got = _apply(m2l, ops, lv, w, prec)
    err = _check(got, ref, prec)
    print("ell %d %s rel L2 %.3e" % (ell, prec, err))


def test_tc_unsupported_requests_refused(m2l):
    cells = pruned_cells(3, 0.3, 2)
    lv = make_level(m2l, cells, 3)
    ops = gpu_ops(m2l, 4, 0, 3, eps=1e-4)
    w = np.zeros((len(cells), 64))
    with pytest.raises(m2l.M2LError) as ei:
        _apply(m2l, ops, lv, w, "tf32")
    assert ei.value.status == m2l.M2L_EUNSUPPORTED
