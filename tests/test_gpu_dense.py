"""The target-stationary tensor-core kernel (full levels of at least 16384
cells, ell <= 5) against the oracle, through the C ABI: full and nearly full
levels 5 and 6 (domain boundary, a ragged last unit per octant, empty
columns), the three kernels of the
configurations, FP64 locals, accumulation into non-zero locals, the adjoint,
agreement with the operator-bucketed kernel on the same plan, and the bounded
wait of its failure path."""
import time

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


_ORACLE = {}
_LISTS = {}


def _lists(cells):
    key = (len(cells), cells.tobytes().__hash__())
    if key not in _LISTS:
        _LISTS[key] = oracle.interaction_lists(cells, cells)
    return _LISTS[key]


def _oracle_level(ell, kind, level, cells, w, init=None, adjoint=False):
    """The oracle's (adjoint) level, cached across the precisions of one case."""
    key = (ell, kind, level, len(cells), float(w[0, 0]), adjoint)
    if key not in _ORACLE:
        off, src = _lists(cells)
        K = oracle_ops(ell, kind, level)
        _ORACLE[key] = (oracle.m2l_apply_adjoint(K, cells, cells, off, src, w, len(cells)) if adjoint
                        else oracle.m2l_apply(K, cells, cells, off, src, w))
    return _ORACLE[key] if init is None else _ORACLE[key] + init


def _check(got, ref, prec):
    err = oracle.rel_l2(got, ref)
    assert err < TOL[prec], (prec, err)
    assert np.max(np.abs(got - ref)) < 50 * TOL[prec] * np.max(np.abs(ref))
    return err


def _plan_apply(m2l, plan, w, prec, n_out, out_fp64=False, init=None):
    dt = torch.float64 if out_fp64 else torch.float32
    loc = torch.zeros(n_out, w.shape[1], dtype=dt, device=device())
    if init is not None:
        loc += torch.from_numpy(init).to(device(), dt)
    m2l.m2l_plan_apply(plan, torch.from_numpy(w).to(device(), torch.float32), loc, prec, out_fp64)
    m2l.m2l_sync_status(plan.ops)
    return loc.double().cpu().numpy()


@pytest.mark.parametrize("prec", TC)
@pytest.mark.parametrize("ell,kind,level,keep", [(2, 0, 5, 1.0), (3, 2, 5, 0.93), (4, 1, 5, 0.9)])
def test_dense_matches_oracle(m2l, prec, ell, kind, level, keep):
    from paper_1210_7292_gb300 import synth
    cells = synth.full_grid(level) if keep == 1.0 else pruned_cells(level, keep, seed=ell * 11 + level)
    rng = np.random.default_rng(ell + 300)
    w = rng.standard_normal((len(cells), ell ** 3))
    init = rng.standard_normal((len(cells), ell ** 3))
    lv = make_level(m2l, cells, level)
    ops = gpu_ops(m2l, ell, kind, level)
    plan = m2l.m2l_plan_create(ops, lv)
    info = m2l.m2l_plan_kernel_info(plan)
    assert info["dense"], info
    ref = _oracle_level(ell, kind, level, cells, w, init=init)
    err = _check(_plan_apply(m2l, plan, w, prec, len(cells), init=init), ref, prec)
    print("dense %s ell=%d kind=%d level=%d keep=%.2f (%d cells, %d units of %d): rel L2 %.2e"
          % (prec, ell, kind, level, keep, len(cells), info["units"], info["unit_width"], err))


@pytest.mark.parametrize("prec", TC)
def test_dense_fp64_locals_adjoint_and_bucketed_agree(m2l, prec):
    """One plan applied by both tensor-core kernels (the bucketed one through
    the M2L_DEBUG_NO_DENSE switch), FP64 locals, and the adjoint plan."""
    from paper_1210_7292_gb300 import synth
    ell, level = 4, 5
    cells = synth.full_grid(level)
    w = synth.gaussian_vectors(len(cells), ell ** 3, seed=301)
    lv = make_level(m2l, cells, level)
    ops = gpu_ops(m2l, ell, 0, level)
    plan = m2l.m2l_plan_create(ops, lv)
    adj = m2l.m2l_plan_create(ops, lv, adjoint=True)
    assert m2l.m2l_plan_kernel_info(plan)["dense"] and m2l.m2l_plan_kernel_info(adj)["dense"]
    ref = _oracle_level(ell, 0, level, cells, w)
    dense = _plan_apply(m2l, plan, w, prec, len(cells), out_fp64=True)
    _check(dense, ref, prec)
    m2l.m2l_ops_set_debug(ops, m2l.M2L_DEBUG_NO_DENSE)
    bucketed = _plan_apply(m2l, plan, w, prec, len(cells), out_fp64=True)
    m2l.m2l_ops_set_debug(ops, 0)
    _check(bucketed, ref, prec)
    assert oracle.rel_l2(dense, bucketed) < TOL[prec]
    ref_adj = _oracle_level(ell, 0, level, cells, w, adjoint=True)
    _check(_plan_apply(m2l, adj, w, prec, len(cells)), ref_adj, prec)


def test_dense_level5_sampled_and_repeatable(m2l):
    """The benchmark's level (full level 5, ell = 5, 1/r) in BF16x3: sampled
    targets against the oracle, and two applies bit-identical."""
    from paper_1210_7292_gb300 import synth
    ell, level = 5, 5
    cells = synth.full_grid(level)
    w = synth.gaussian_vectors(len(cells), ell ** 3, seed=302)
    lv = make_level(m2l, cells, level)
    ops = gpu_ops(m2l, ell, 0, level)
    plan = m2l.m2l_plan_create(ops, lv)
    info = m2l.m2l_plan_kernel_info(plan)
    assert info["dense"]
    a = _plan_apply(m2l, plan, w, "bf16x3", len(cells))
    b = _plan_apply(m2l, plan, w, "bf16x3", len(cells))
    assert np.array_equal(a, b)        # one write per (target, node): no order-dependent sums
    rng = np.random.default_rng(303)
    samp = np.unique(np.concatenate([[0, len(cells) - 1], rng.choice(len(cells), 62, replace=False)]))
    off, src = oracle.interaction_lists(cells[samp], cells)
    ref = oracle.m2l_apply(oracle_ops(ell, 0, level), cells[samp], cells, off, src, w)
    err = _check(a[samp], ref, "bf16x3")
    print("dense level 5 bf16x3 (%d units of %d): rel L2 %.2e" % (info["units"], info["unit_width"], err))


def test_dense_level6_sampled(m2l):
    """A full level 6 (262,144 cells, the differentiation workload's level),
    ell = 3, 1/r^4, TF32x3 and BF16x3, sampled targets against the oracle."""
    from paper_1210_7292_gb300 import synth
    ell, level = 3, 6
    cells = synth.full_grid(level)
    w = synth.gaussian_vectors(len(cells), ell ** 3, seed=306)
    lv = make_level(m2l, cells, level)
    ops = gpu_ops(m2l, ell, 1, level)
    plan = m2l.m2l_plan_create(ops, lv)
    info = m2l.m2l_plan_kernel_info(plan)
    assert info["dense"]
    rng = np.random.default_rng(307)
    samp = np.unique(np.concatenate([[0, len(cells) - 1], rng.choice(len(cells), 94, replace=False)]))
    off, src = oracle.interaction_lists(cells[samp], cells)
    ref = oracle.m2l_apply(oracle_ops(ell, 1, level), cells[samp], cells, off, src, w)
    for prec in ("tf32x3", "bf16x3"):
        got = _plan_apply(m2l, plan, w, prec, len(cells))
        err = _check(got[samp], ref, prec)
        print("dense level 6 %s (%d units of %d): rel L2 %.2e" % (prec, info["units"], info["unit_width"], err))


def test_sparse_and_small_levels_keep_the_bucketed_kernel(m2l):
    from paper_1210_7292_gb300 import synth
    for cells, level in ((pruned_cells(5, 0.4, 304), 5), (synth.full_grid(4), 4)):
        lv = make_level(m2l, cells, level)
        plan = m2l.m2l_plan_create(gpu_ops(m2l, 4, 0, level), lv)
        assert not m2l.m2l_plan_kernel_info(plan)["dense"], (level, len(cells))


def test_dense_bounded_wait_reports_timeout(m2l):
    """The failure switch on the dense kernel: its producer withholds the first
    stage, the MMA warp's bounded wait runs out, the kernel returns, the host
    reads M2L_ETIMEOUT and a correct apply follows on the same context."""
    from paper_1210_7292_gb300 import synth
    ell, level = 2, 5
    cells = synth.full_grid(level)
    w = synth.gaussian_vectors(len(cells), ell ** 3, seed=305)
    lv = make_level(m2l, cells, level)
    ops = gpu_ops(m2l, ell, 0, level)
    plan = m2l.m2l_plan_create(ops, lv)
    assert m2l.m2l_plan_kernel_info(plan)["dense"]
    m2l.m2l_ops_set_debug(ops, m2l.M2L_DEBUG_STALL_PRODUCER)
    loc = torch.zeros(len(cells), ell ** 3, dtype=torch.float32, device=device())
    t0 = time.time()
    m2l.m2l_plan_apply(plan, torch.from_numpy(w).to(device(), torch.float32), loc, "bf16x3")
    with pytest.raises(m2l.M2LError) as ei:
        m2l.m2l_sync_status(ops)
    assert ei.value.status == m2l.M2L_ETIMEOUT and time.time() - t0 < 30.0
    m2l.m2l_ops_set_debug(ops, 0)
    off, src = oracle.interaction_lists(cells, cells)
    ref = oracle.m2l_apply(oracle_ops(ell, 0, level), cells, cells, off, src, w)
    _check(_plan_apply(m2l, plan, w, "bf16x3", len(cells)), ref, "bf16x3")


def test_dense_repeated_and_near_entries_reported(m2l):
    """On the dense path a repeated (X, t) entry and a near-field entry are
    skipped and reported (M2L_EINVAL); every other entry is applied."""
    from paper_1210_7292_gb300 import synth
    ell, level = 2, 5
    cells = synth.full_grid(level)
    off, src = _lists(cells)
    bad = src.copy()
    r1, r2 = 100, 20000
    bad[off[r1] + 1] = src[off[r1]]                    # row r1: its first (X, t) twice
    nb = cells[r2] + np.array([1, 0, 0]) if cells[r2][0] < (1 << level) - 1 else cells[r2] - np.array([1, 0, 0])
    near = int(np.flatnonzero((cells == nb).all(axis=1))[0])
    bad[off[r2]] = near                                # row r2: a near-field neighbour
    keep = np.ones(len(src), dtype=bool)
    keep[[off[r1] + 1, off[r2]]] = False
    good_off = np.concatenate([[0], np.cumsum([keep[off[i]:off[i + 1]].sum() for i in range(len(cells))])])
    good_src = src[keep]
    ijk = torch.from_numpy(np.ascontiguousarray(cells, dtype=np.int32)).to(device())
    lv = m2l.Level(oracle.cell_width(level), ijk, ijk, torch.from_numpy(off).to(device()),
                   torch.from_numpy(bad).to(device()), level)
    ops = gpu_ops(m2l, ell, 0, level)
    plan = m2l.m2l_plan_create(ops, lv)
    assert m2l.m2l_plan_kernel_info(plan)["dense"]
    w = synth.gaussian_vectors(len(cells), ell ** 3, seed=306)
    loc = torch.zeros(len(cells), ell ** 3, dtype=torch.float32, device=device())
    m2l.m2l_plan_apply(plan, torch.from_numpy(w).to(device(), torch.float32), loc, "bf16x3")
    with pytest.raises(m2l.M2LError) as ei:
        m2l.m2l_sync_status(ops)
    assert ei.value.status == m2l.M2L_EINVAL
    ref = oracle.m2l_apply(oracle_ops(ell, 0, level), cells, cells, good_off.astype(np.int32), good_src, w)
    _check(loc.cpu().double().numpy(), ref, "bf16x3")
    m2l.m2l_sync_status(ops)   # cleared


@pytest.mark.parametrize("adjoint", [False, True])
def test_buckets_derived_from_dense_classification(m2l, adjoint):
    """A full level is classified for the dense kernel only; asking for its
    operator buckets derives them on the device.  As a set, the derived records
    (source, target, g) are the oracle's classification of the level's list
    (the transposed list for the adjoint), and the per-operator counts match."""
    from paper_1210_7292_gb300 import synth
    level = 5
    cells = synth.full_grid(level)
    lv = make_level(m2l, cells, level)
    plan = m2l.m2l_plan_create(gpu_ops(m2l, 3, 0, level), lv, adjoint=adjoint)
    assert m2l.m2l_plan_kernel_info(plan)["dense"]
    counts, recs = m2l.m2l_plan_query(plan)
    off, src = _lists(cells)
    tgt = np.repeat(np.arange(len(cells)), np.diff(off))
    if adjoint:
        tgt, src = src.astype(np.int64), tgt
    t = cells[tgt].astype(np.int64) - cells[src].astype(np.int64)
    code = oracle.lut343()[(t[:, 0] + 3) + 7 * (t[:, 1] + 3) + 49 * (t[:, 2] + 3)].astype(np.int64)
    assert np.array_equal(counts, np.bincount(code & 0xFF, minlength=16))
    exp = np.stack([src, tgt, code >> 8], axis=1).astype(np.int64)
    got = recs.astype(np.int64)
    key = lambda a: np.lexsort((a[:, 2], a[:, 1], a[:, 0]))
    assert np.array_equal(got[key(got)], exp[key(exp)])
    # records of one operator are grouped, and within it each target's entries are consecutive
    p_of = np.repeat(np.arange(16), counts)
    assert np.array_equal(p_of, code[np.lexsort((code & 0xFF,))] & 0xFF)
    for p in range(16):
        tg = got[p_of == p, 1]
        starts = np.flatnonzero(np.diff(tg) != 0).size + 1
        assert starts == np.unique(tg).size, p
