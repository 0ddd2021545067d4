"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Index and permutation work is compared bit for bit; floating-point results
element by element against the oracle within the tolerance of each precision
(gpu_helpers.TOL, relative L2 over the level plus a max-abs bound).
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import KIND_C, TOL, device, gpu_ops, make_level, oracle_ops, pruned_cells

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


# ---------------------------------------------------------------- tables (a2)
@pytest.mark.parametrize("ell", [2, 3, 4, 5, 6, 7, 8])
def test_tables_bit_exact(m2l, ell):
    ops = m2l.m2l_precompute(m2l.M2L_K_INV_R, ell)
    ranks, sigma, lut = m2l.m2l_ops_query(ops)
    assert np.array_equal(sigma.astype(np.int64), oracle.sigma_tables(ell))
    assert np.array_equal(lut, oracle.lut343())
    assert np.all(ranks == ell ** 3)


# ---------------------------------------------------------------- operators (a1)
@pytest.mark.parametrize("ell,kind", [(4, 0), (5, 0), (7, 1), (5, 2), (8, 0)])
def test_operators_match_direct_assembly(m2l, ell, kind):
    level = 3
    ops = gpu_ops(m2l, ell, kind, level)
    K = m2l.m2l_ops_copy_operators(ops)
    info = m2l.m2l_ops_info(ops)
    w = oracle.cell_width(level)
    scale = (w / info["ref_width"]) ** info["homogeneity_degree"] if kind != 2 else 1.0
    for p, t in enumerate(oracle.t_sym_list()):
        ref = oracle.operator_for_t(ell, kind, KIND_C[kind], level, t)
        rel = np.max(np.abs(K[p] * scale - ref)) / np.max(np.abs(ref))
        assert rel < 1e-14, (p, t, rel)
    # and every one of the 316 operators through the tables (Eq. (25))
    _, sigma, lut = m2l.m2l_ops_query(ops)
    for t in oracle.transfer_vectors()[::7]:
        v = int(lut[oracle.t_slot(t)])
        p, g = v & 0xFF, v >> 8
        ref = oracle.operator_for_t(ell, kind, KIND_C[kind], level, t)
        s = sigma[g].astype(np.int64)
        rel = np.max(np.abs(K[p][np.ix_(s, s)] * scale - ref)) / np.max(np.abs(ref))
        assert rel < 1e-14


# ---------------------------------------------------------------- lists and classification (a3)
@pytest.mark.parametrize("level,keep,seed", [(2, 1.0, 0), (3, 1.0, 0), (4, 0.5, 1), (5, 0.05, 2)])
def test_lists_bit_exact(m2l, level, keep, seed):
    cells = pruned_cells(level, keep, seed)
    lv = make_level(m2l, cells, level)
    off_o, src_o = oracle.interaction_lists(cells, cells)
    assert np.array_equal(lv.il_offsets.cpu().numpy(), off_o)
    assert np.array_equal(lv.il_sources.cpu().numpy(), src_o)


def _expected_buckets(cells, off, src):
    lut = oracle.lut343()
    recs = []
    for x in range(len(cells)):
        for e in range(off[x], off[x + 1]):
            y = int(src[e])
            t = tuple(int(v) for v in cells[x] - cells[y])
            code = int(lut[oracle.t_slot(t)])
            recs.append((code & 0xFF, y, x, code >> 8))
    recs.sort(key=lambda r: r[0])   # stable: list order inside a bucket
    counts = np.bincount([r[0] for r in recs], minlength=16)
    return counts, np.array([r[1:] for r in recs], dtype=np.int32)


@pytest.mark.parametrize("adjoint", [False, True])
def test_classification_bit_exact(m2l, adjoint):
    level = 3
    cells = pruned_cells(level, 0.8, 5)
    lv = make_level(m2l, cells, level)
    ops = m2l.m2l_precompute(m2l.M2L_K_INV_R, 3)
    plan = m2l.m2l_plan_create(ops, lv, adjoint=adjoint)
    counts, recs = m2l.m2l_plan_query(plan)
    off, src = oracle.interaction_lists(cells, cells)
    if adjoint:
        # transposed list: rows over sources, ascending target inside a row
        pairs = sorted((int(src[e]), x) for x in range(len(cells)) for e in range(off[x], off[x + 1]))
        toff = np.zeros(len(cells) + 1, dtype=np.int64)
        for y, _ in pairs:
            toff[y + 1] += 1
        off, src = np.cumsum(toff), np.array([x for _, x in pairs], dtype=np.int32)
    exp_counts, exp_recs = _expected_buckets(cells, off, src)
    assert np.array_equal(counts, exp_counts)
    assert np.array_equal(recs, exp_recs)


# ---------------------------------------------------------------- apply (a4-a6)
def _run_apply(m2l, ops, lv, w, prec, locals_fp64=False, init=None):
    dt_in = torch.float64 if prec == "fp64" else torch.float32
    dt_out = torch.float64 if (prec == "fp64" or locals_fp64) else torch.float32
    n3 = w.shape[1]
    loc = torch.zeros(lv.struct.ncells_tgt, n3, dtype=dt_out, device=device())
    if init is not None:
        loc += torch.from_numpy(init).to(device(), dt_out)
    m2l.m2l_apply_level(ops, lv, torch.from_numpy(w).to(device(), dt_in), loc, prec, locals_fp64)
    m2l.m2l_sync_status(ops)
    return loc.double().cpu().numpy()


def _compare(got, ref, tol):
    err = oracle.rel_l2(got, ref)
    assert err < tol, err
    assert np.max(np.abs(got - ref)) < 50 * tol * np.max(np.abs(ref))
    return err


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_config1_plain_level3(m2l, prec):
    """Full level 3 of [-1,1]^3, ell = 4, 1/r, multipoles N(0,1) (seed 1)."""
    from paper_1210_7292_gb300 import synth
    level, ell = 3, 4
    cells = synth.full_grid(level)
    w = synth.gaussian_vectors(len(cells), ell ** 3, seed=1)
    lv = make_level(m2l, cells, level)
    assert lv.nnz == 53352
    ops = gpu_ops(m2l, ell, 0, level)
    off, src = oracle.interaction_lists(cells, cells)
    ref = oracle.m2l_apply(oracle_ops(ell, 0, level), cells, cells, off, src, w)
    got = _run_apply(m2l, ops, lv, w, prec)
    _compare(got, ref, TOL[prec])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("ell,kind,level,keep", [(3, 0, 4, 0.6), (5, 1, 4, 0.3), (6, 2, 3, 0.9), (7, 0, 3, 0.5),
                                                 (2, 0, 2, 1.0)])
def test_apply_pruned_levels(m2l, prec, ell, kind, level, keep):
    """Pruned levels: ragged buckets, several tiles per bucket, ragged last tile."""
    cells = pruned_cells(level, keep, seed=ell * 10 + level)
    rng = np.random.default_rng(ell)
    w = rng.standard_normal((len(cells), ell ** 3))
    init = rng.standard_normal((len(cells), ell ** 3))
    lv = make_level(m2l, cells, level)
    ops = gpu_ops(m2l, ell, kind, level)
    off, src = oracle.interaction_lists(cells, cells)
    ref = oracle.m2l_apply(oracle_ops(ell, kind, level), cells, cells, off, src, w, locals_in=init)
    got = _run_apply(m2l, ops, lv, w, prec, init=init)
    _compare(got, ref, TOL[prec])


def test_order_8(m2l):
    """ell = 8 (512 nodes): FP32 runs with 32-column tiles; FP64 does not fit
    shared memory and is refused with M2L_EUNSUPPORTED."""
    level, ell = 3, 8
    cells = pruned_cells(level, 0.2, 8)
    w = np.random.default_rng(8).standard_normal((len(cells), ell ** 3))
    lv = make_level(m2l, cells, level)
    ops = gpu_ops(m2l, ell, 1, level)
    off, src = oracle.interaction_lists(cells, cells)
    ref = oracle.m2l_apply(oracle_ops(ell, 1, level), cells, cells, off, src, w)
    _compare(_run_apply(m2l, ops, lv, w, "fp32"), ref, TOL["fp32"])
    with pytest.raises(m2l.M2LError) as ei:
        _run_apply(m2l, ops, lv, w, "fp64")
    assert ei.value.status == m2l.M2L_EUNSUPPORTED


def test_classify_then_apply_classified(m2l):
    level, ell = 3, 4
    cells = pruned_cells(level, 0.85, 13)
    w = np.random.default_rng(6).standard_normal((len(cells), ell ** 3))
    lv = make_level(m2l, cells, level)
    ops = gpu_ops(m2l, ell, 0, level)
    off, src = oracle.interaction_lists(cells, cells)
    ref = oracle.m2l_apply(oracle_ops(ell, 0, level), cells, cells, off, src, w)
    loc = torch.zeros(len(cells), ell ** 3, dtype=torch.float64, device=device())
    m2l.m2l_classify_level(ops, lv)
    m2l.m2l_apply_classified(ops, torch.from_numpy(w).to(device()), loc, "fp64")
    m2l.m2l_sync_status(ops)
    _compare(loc.cpu().numpy(), ref, TOL["fp64"])


def test_fp32_products_fp64_locals(m2l):
    level, ell = 3, 5
    cells = pruned_cells(level, 0.7, 3)
    w = np.random.default_rng(0).standard_normal((len(cells), ell ** 3))
    lv = make_level(m2l, cells, level)
    ops = gpu_ops(m2l, ell, 0, level)
    off, src = oracle.interaction_lists(cells, cells)
    ref = oracle.m2l_apply(oracle_ops(ell, 0, level), cells, cells, off, src, w)
    got = _run_apply(m2l, ops, lv, w, "fp32", locals_fp64=True)
    _compare(got, ref, TOL["fp32"])


def test_empty_and_degenerate_lists(m2l):
    ops = gpu_ops(m2l, 4, 0, 2)
    # a level whose cells are all neighbours: empty lists
    cells = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 1]], dtype=np.int32)
    lv = make_level(m2l, cells, 2)
    assert lv.nnz == 0
    got = _run_apply(m2l, ops, lv, np.ones((3, 64)), "fp32")
    assert np.all(got == 0)
    # one target with one source
    cells = np.array([[0, 0, 0], [3, 2, 0]], dtype=np.int32)
    lv = make_level(m2l, cells, 2)
    assert lv.nnz == 2
    w = np.random.default_rng(1).standard_normal((2, 64))
    off, src = oracle.interaction_lists(cells, cells)
    ref = oracle.m2l_apply(oracle_ops(4, 0, 2), cells, cells, off, src, w)
    _compare(_run_apply(m2l, ops, lv, w, "fp64"), ref, TOL["fp64"])


def test_bad_list_entry_reported(m2l):
    """A near-field pair in the list is skipped and reported; the rest is applied."""
    ops = gpu_ops(m2l, 3, 0, 2)
    cells = np.array([[0, 0, 0], [1, 0, 0], [3, 3, 3]], dtype=np.int32)
    ijk = torch.from_numpy(cells).to(device())
    off = torch.tensor([0, 2, 2, 2], dtype=torch.int32, device=device())
    src = torch.tensor([1, 2], dtype=torch.int32, device=device())   # (0,0,0)<-(1,0,0) is near
    lv = m2l.Level(oracle.cell_width(2), ijk, ijk, off, src, 2)
    loc = torch.zeros(3, 27, dtype=torch.float64, device=device())
    w = np.random.default_rng(2).standard_normal((3, 27))
    m2l.m2l_apply_level(ops, lv, torch.from_numpy(w).to(device()), loc, "fp64")
    with pytest.raises(m2l.M2LError) as ei:
        m2l.m2l_sync_status(ops)
    assert ei.value.status == m2l.M2L_EINVAL
    good_off = np.array([0, 1, 1, 1], dtype=np.int32)
    ref = oracle.m2l_apply(oracle_ops(3, 0, 2), cells, cells, good_off, np.array([2], np.int32), w)
    _compare(loc.cpu().numpy(), ref, TOL["fp64"])
    m2l.m2l_sync_status(ops)   # cleared


def test_width_mismatch_rejected_for_non_homogeneous(m2l):
    ops = gpu_ops(m2l, 3, 2, 3)
    cells = pruned_cells(2, 1.0, 0)
    lv = make_level(m2l, cells, 2)   # width of level 2, operators built for level 3
    loc = torch.zeros(len(cells), 27, device=device())
    with pytest.raises(m2l.M2LError) as ei:
        m2l.m2l_apply_level(ops, lv, torch.zeros(len(cells), 27, device=device()), loc, "fp32")
    assert ei.value.status == m2l.M2L_EINVAL


# ---------------------------------------------------------------- adjoint
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_adjoint_matches_oracle_transpose(m2l, prec):
    level, ell = 3, 4
    cells = pruned_cells(level, 0.7, 9)
    g = np.random.default_rng(3).standard_normal((len(cells), ell ** 3))
    lv = make_level(m2l, cells, level)
    ops = gpu_ops(m2l, ell, 0, level)
    off, src = oracle.interaction_lists(cells, cells)
    ref = oracle.m2l_apply_adjoint(oracle_ops(ell, 0, level), cells, cells, off, src, g, len(cells))
    dt = torch.float64 if prec == "fp64" else torch.float32
    out = torch.zeros(len(cells), ell ** 3, dtype=dt, device=device())
    m2l.m2l_apply_level_adjoint(ops, lv, torch.from_numpy(g).to(device(), dt), out, prec)
    m2l.m2l_sync_status(ops)
    _compare(out.double().cpu().numpy(), ref, TOL[prec])


# ---------------------------------------------------------------- low rank
@pytest.mark.parametrize("trunc", ["frobenius", "spectral"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("ell,kind,eps", [(5, 0, 1e-5), (7, 1, 1e-7)])
def test_lowrank_matches_oracle(m2l, prec, ell, kind, eps, trunc):
    """Step a1 by the device's one-sided Jacobi SVD: the ranks under either
    truncation criterion equal the oracle's (LAPACK SVD), the truncated
    operators agree to 1e-12 s_1, and the apply matches the oracle's."""
    level = 3
    cells = pruned_cells(level, 0.4, 21)
    w = np.random.default_rng(4).standard_normal((len(cells), ell ** 3))
    lv = make_level(m2l, cells, level)
    ops = gpu_ops(m2l, ell, kind, level, eps=eps, truncation=trunc)
    assert m2l.m2l_ops_truncation(ops) == trunc
    sweeps = m2l.m2l_ops_svd_sweeps(ops)
    assert 0 < sweeps.min() and sweeps.max() < 100
    ranks, _, _ = m2l.m2l_ops_query(ops)
    tsym = oracle.t_sym_list()
    full = oracle.operator_table(ell, kind, KIND_C[kind], level)
    for p, t in enumerate(tsym):
        s = np.linalg.svd(full[oracle.t_slot(t)], compute_uv=False)
        assert ranks[p] == oracle.truncation_rank(s, eps, trunc)
        U, V = m2l.m2l_ops_copy_lowrank(ops, p)
        info = m2l.m2l_ops_info(ops)
        sc = (oracle.cell_width(level) / info["ref_width"]) ** info["homogeneity_degree"]
        Ko, Vo, r = oracle.lowrank(full[oracle.t_slot(t)], eps, trunc)
        assert np.allclose(sc * U @ V.T, Ko @ Vo.T, rtol=0, atol=1e-12 * s[0])
        # the device's factor columns are orthogonal: V orthonormal, U = U_K Sigma
        assert np.abs(V.T @ V - np.eye(r)).max() < 1e-12
        G = U.T @ U
        assert np.abs(G - np.diag(np.diag(G))).max() < 1e-12 * G[0, 0]
    off, src = oracle.interaction_lists(cells, cells)
    ops_lr, _ = oracle.lowrank_operator_table(full, eps, trunc)
    ref = oracle.m2l_apply(ops_lr, cells, cells, off, src, w)
    _compare(_run_apply(m2l, ops, lv, w, prec), ref, TOL[prec])


# ---------------------------------------------------------------- plans
def test_plan_apply_repeats(m2l):
    level, ell = 3, 4
    cells = pruned_cells(level, 0.9, 12)
    w = np.random.default_rng(5).standard_normal((len(cells), ell ** 3))
    lv = make_level(m2l, cells, level)
    ops = gpu_ops(m2l, ell, 0, level)
    plan = m2l.m2l_plan_create(ops, lv)
    off, src = oracle.interaction_lists(cells, cells)
    ref = oracle.m2l_apply(oracle_ops(ell, 0, level), cells, cells, off, src, w)
    loc = torch.zeros(len(cells), ell ** 3, dtype=torch.float64, device=device())
    wd = torch.from_numpy(w).to(device())
    for _ in range(2):
        m2l.m2l_plan_apply(plan, wd, loc, "fp64")
    m2l.m2l_sync_status(ops)
    _compare(loc.cpu().numpy(), 2 * ref, TOL["fp64"])


# ---------------------------------------------------------------- full-size workload, sampled
def test_config2_level5_sampled_targets(m2l):
    """Full level 5 (32768 cells, 5 398 920 interactions), ell = 5, 1/r, in the
    launch configuration the benchmark times; 48 sampled targets against the oracle."""
    from paper_1210_7292_gb300 import synth
    level, ell = 5, 5
    cells = synth.full_grid(level)
    w = synth.gaussian_vectors(len(cells), ell ** 3, seed=2)
    lv = make_level(m2l, cells, level)
    assert lv.nnz == 5398920
    ops = gpu_ops(m2l, ell, 0, level)
    got = {p: _run_apply(m2l, ops, lv, w, p) for p in ("fp64", "fp32")}
    rng = np.random.default_rng(7)
    samp = np.sort(rng.choice(len(cells), 48, replace=False))
    samp[0] = 0                       # a corner cell
    samp[-1] = 16 + 32 * (16 + 32 * 16)  # an interior cell
    samp = np.unique(samp)
    off, src = oracle.interaction_lists(cells[samp], cells)
    ref = oracle.m2l_apply(oracle_ops(ell, 0, level), cells[samp], cells, off, src, w)
    for p in ("fp64", "fp32"):
        _compare(got[p][samp], ref, TOL[p])
