"""SA and SArcmp on the GPU (m2l_sa_*, Sec. 4.1, Eqs. (17)-(19)) against the
oracle's factorisation of the same operators: the rank r and the per-core
recompression ranks exactly, the represented operators U C_t B^T element by
element, and the apply over a level against the oracle's cell-by-cell M2L
with the oracle's SA operators."""
import numpy as np
import pytest

import oracle
from gpu_helpers import KIND_C, device, gpu_ops, make_level, pruned_cells

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


def _scale(m2l, ops, level):
    info = m2l.m2l_ops_info(ops)
    if info["homogeneity_degree"] == 0:
        return 1.0
    return (oracle.cell_width(level) / info["ref_width"]) ** info["homogeneity_degree"]


CASES = [(4, 0, 1e-4, False), (5, 0, 1e-5, False), (5, 0, 1e-5, True), (5, 1, 1e-6, True), (4, 2, 1e-5, True),
         (3, 0, 1e-3, True), (3, 0, 0.0, False)]


@pytest.mark.parametrize("trunc", ["frobenius", "spectral"])
@pytest.mark.parametrize("ell,kind,eps,rcmp", CASES)
def test_sa_factors_match_oracle(m2l, ell, kind, eps, rcmp, trunc):
    """The device's Jacobi SVDs of K_col, K_row^T and of every core give the
    oracle's (LAPACK's) ranks under either truncation criterion."""
    level = 3
    ops = gpu_ops(m2l, ell, kind, level, truncation=trunc)
    sa = m2l.m2l_sa_create(ops, eps, rcmp)
    r, nrc, rt = m2l.m2l_sa_info(sa)
    table, sa_ref, ranks = oracle.sa_operator_table(oracle.operator_table(ell, kind, KIND_C[kind], level), eps, rcmp,
                                                    trunc)
    assert r == sa_ref["r"]
    if rcmp:
        expect = np.where((ranks > 0) & (ranks < r), ranks, 0)
        assert np.array_equal(rt, expect)
        assert nrc == int(np.count_nonzero(expect))
    else:
        assert nrc == 0 and not rt.any()
    U, B, X, Y = m2l.m2l_sa_copy_factors(sa)
    # the bases are orthonormal (right singular vectors)
    assert np.abs(U.T @ U - np.eye(r)).max() < 1e-12
    assert np.abs(B.T @ B - np.eye(r)).max() < 1e-12
    s = _scale(m2l, ops, level)
    worst = 0.0
    for t in oracle.transfer_vectors():
        sl = oracle.t_slot(t)
        k = int(rt[sl])
        C = X[sl] if k == 0 else X[sl][:, :k] @ Y[sl][:, :k].T
        K = s * (U @ C @ B.T)
        worst = max(worst, np.abs(K - table[sl]).max() / np.abs(table[sl]).max())
    print("ell=%d kind=%d eps=%g rcmp=%d: r=%d, %d cores recompressed, max rel diff %.2e"
          % (ell, kind, eps, rcmp, r, nrc, worst))
    assert worst < 1e-9, worst


def _apply_case(m2l, ell, kind, eps, rcmp, level, keep, seed, precision, locals_fp64=False):
    cells = pruned_cells(level, keep, seed)
    lv = make_level(m2l, cells, level)
    ops = gpu_ops(m2l, ell, kind, level)
    sa = m2l.m2l_sa_create(ops, eps, rcmp)
    rng = np.random.default_rng(seed + 100)
    n3 = ell ** 3
    w = rng.standard_normal((len(cells), n3))
    f0 = rng.standard_normal((len(cells), n3))
    table, _, _ = oracle.sa_operator_table(oracle.operator_table(ell, kind, KIND_C[kind], level), eps, rcmp)
    off, src = lv.il_offsets.cpu().numpy(), lv.il_sources.cpu().numpy()
    ref = oracle.m2l_apply(table, cells, cells, off, src, w, f0)
    tin = torch.float64 if precision == "fp64" else torch.float32
    tout = torch.float64 if (precision == "fp64" or locals_fp64) else torch.float32
    wd = torch.from_numpy(w).to(device(), tin)
    fd = torch.from_numpy(f0).to(device(), tout)
    m2l.m2l_sa_apply_level(sa, lv, wd, fd, precision, locals_fp64)
    m2l.m2l_sync_status(ops)
    got = fd.double().cpu().numpy()
    return oracle.rel_l2(got - f0, ref - f0), got, ref


@pytest.mark.parametrize("ell,kind,eps,rcmp,level,keep,seed", [
    (4, 0, 1e-4, False, 3, 1.0, 1), (5, 0, 1e-5, True, 4, 0.3, 2), (5, 1, 1e-6, True, 3, 0.7, 3),
    (4, 2, 1e-5, True, 3, 0.9, 4), (3, 0, 0.0, False, 4, 0.2, 5)])
def test_sa_apply_fp64_matches_oracle(m2l, ell, kind, eps, rcmp, level, keep, seed):
    err, _, _ = _apply_case(m2l, ell, kind, eps, rcmp, level, keep, seed, "fp64")
    print("SA apply fp64 ell=%d kind=%d eps=%g rcmp=%d: rel L2 %.2e" % (ell, kind, eps, rcmp, err))
    assert err < 1e-9, err


@pytest.mark.parametrize("locals_fp64", [False, True])
@pytest.mark.parametrize("ell,kind,eps,rcmp", [(5, 0, 1e-5, False), (5, 1, 1e-6, True)])
def test_sa_apply_fp32_matches_oracle(m2l, ell, kind, eps, rcmp, locals_fp64):
    err, _, _ = _apply_case(m2l, ell, kind, eps, rcmp, 4, 0.25, 6, "fp32", locals_fp64)
    print("SA apply fp32 ell=%d kind=%d eps=%g rcmp=%d out64=%d: rel L2 %.2e" % (ell, kind, eps, rcmp,
                                                                                 locals_fp64, err))
    assert err < 2e-5, err


def test_sa_full_rank_equals_blocked_apply(m2l):
    """eps = 0 keeps r = n3: U C_t B^T = K_t exactly, so SA gives the M2L itself."""
    ell, level = 4, 3
    cells = pruned_cells(level, 0.8, 7)
    lv = make_level(m2l, cells, level)
    ops = gpu_ops(m2l, ell, 0, level)
    sa = m2l.m2l_sa_create(ops, 0.0, True)
    r, nrc, _ = m2l.m2l_sa_info(sa)
    assert r == ell ** 3 and nrc == 0
    w = torch.from_numpy(np.random.default_rng(8).standard_normal((len(cells), ell ** 3))).to(device())
    f_sa = torch.zeros_like(w)
    f_bl = torch.zeros_like(w)
    m2l.m2l_sa_apply_level(sa, lv, w, f_sa, "fp64")
    m2l.m2l_apply_level(ops, lv, w, f_bl, "fp64")
    m2l.m2l_sync_status(ops)
    assert oracle.rel_l2(f_sa.cpu().numpy(), f_bl.cpu().numpy()) < 1e-12


def test_sa_bad_list_and_empty_level(m2l):
    ell, level = 3, 3
    cells = pruned_cells(level, 1.0, 9)
    lv = make_level(m2l, cells, level)
    ops = gpu_ops(m2l, ell, 0, level)
    sa = m2l.m2l_sa_create(ops, 1e-3)
    w = torch.ones((len(cells), ell ** 3), dtype=torch.float32, device=device())
    f = torch.zeros_like(w)
    # an entry pointing at the target itself (t = 0) is not a far-field pair
    lv.il_sources[0] = 0
    m2l.m2l_sa_apply_level(sa, lv, w, f, "fp32")
    with pytest.raises(m2l.M2LError) as ei:
        m2l.m2l_sync_status(ops)
    assert ei.value.status == m2l.M2L_EINVAL
    # an empty level is a no-op
    e = torch.zeros((0, 3), dtype=torch.int32, device=device())
    off = torch.zeros(1, dtype=torch.int32, device=device())
    src = torch.zeros(0, dtype=torch.int32, device=device())
    empty = m2l.Level(oracle.cell_width(level), e, e, off, src, level)
    z = torch.zeros((0, ell ** 3), dtype=torch.float32, device=device())
    m2l.m2l_sa_apply_level(sa, empty, z, z, "fp32")
    m2l.m2l_sync_status(ops)
    with pytest.raises(m2l.M2LError) as ei:
        m2l.m2l_sa_create(ops, 1.5)
    assert ei.value.status == m2l.M2L_EINVAL


@pytest.mark.parametrize("prec,tol", [("bf16x3", 2e-5), ("tf32x3", 2e-5), ("tf32", 2e-3)])
@pytest.mark.parametrize("ell,kind,eps,rcmp", [(5, 0, 1e-5, False), (5, 1, 1e-6, True), (4, 2, 1e-5, True)])
def test_sa_apply_tensor_cores(m2l, ell, kind, eps, rcmp, prec, tol):
    """The cores on the tcgen05 kernel (one class per transfer vector) against the
    oracle's SA operators; BF16x3 and TF32x3 reach FP32-level error."""
    err, _, _ = _apply_case(m2l, ell, kind, eps, rcmp, 4, 0.25, 6, prec, True)
    print("SA apply %s ell=%d kind=%d eps=%g rcmp=%d: rel L2 %.2e" % (prec, ell, kind, eps, rcmp, err))
    assert err < tol, err
