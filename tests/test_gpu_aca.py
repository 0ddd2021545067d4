"""The ACA + truncated SVD precompute on the GPU (m2l_precompute_aca): the
ranks equal those of the SVD precompute and of the oracle's ACA (Sec. 5: both
routes end with the same ranks), every factorisation is within the
truncation bound eps s_1 of its operator, and the low-rank apply with these
factors agrees with the SVD-factor apply and with the exact M2L to O(eps)."""
import numpy as np
import pytest

import oracle
from gpu_helpers import KIND_C, device, make_level, pruned_cells

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


def _ops(m2l, fn, ell, kind, eps, level):
    w = oracle.cell_width(level)
    return fn(kind, ell, eps, w if kind == 2 else 0.0, KIND_C[kind])


@pytest.mark.parametrize("ell,kind,eps", [(3, 0, 1e-3), (5, 0, 1e-5), (5, 1, 1e-6), (6, 2, 1e-6), (7, 1, 1e-7),
                                          (8, 0, 1e-8)])
def test_aca_ranks_and_bound(m2l, ell, kind, eps):
    level = 3
    ops_a = _ops(m2l, m2l.m2l_precompute_aca, ell, kind, eps, level)
    ops_s = _ops(m2l, m2l.m2l_precompute, ell, kind, eps, level)
    ranks_a = m2l.m2l_ops_query(ops_a)[0]
    ranks_s = m2l.m2l_ops_query(ops_s)[0]
    terms, sweeps = m2l.m2l_ops_aca_info(ops_a)
    K = m2l.m2l_ops_copy_operators(ops_a)
    ref_ranks = []
    worst = 0.0
    for p, t in enumerate(oracle.t_sym_list()):
        Kp = oracle.operator_for_t(ell, kind, KIND_C[kind], level, t)
        _, _, r = oracle.lowrank(Kp, eps)
        _, _, ra, _ = oracle.aca_lowrank(Kp, eps)
        assert ra == r
        ref_ranks.append(r)
        U, V = m2l.m2l_ops_copy_lowrank(ops_a, p)
        s1 = np.linalg.norm(K[p], 2)
        worst = max(worst, np.linalg.norm(K[p] - U @ V.T, 2) / s1)
    print("ell=%d kind=%d eps=%g: ranks %s, ACA terms %d-%d, Jacobi sweeps <= %d, max |K - UV^T|_2 / s1 = %.2e"
          % (ell, kind, eps, list(ranks_a), terms.min(), terms.max(), sweeps.max(), worst))
    assert list(ranks_a) == list(ranks_s) == ref_ranks
    assert np.all(terms >= ranks_a) and sweeps.max() < 60
    assert worst <= 1.01 * eps


@pytest.mark.parametrize("ell,kind,eps", [(5, 0, 1e-5), (7, 1, 1e-7)])
def test_aca_apply(m2l, ell, kind, eps):
    level = 4
    cells = pruned_cells(level, 0.3, 3)
    lv = make_level(m2l, cells, level)
    w = torch.from_numpy(np.random.default_rng(4).standard_normal((len(cells), ell ** 3))).to(device())
    outs = {}
    for name, fn in (("aca", m2l.m2l_precompute_aca), ("svd", m2l.m2l_precompute)):
        ops = _ops(m2l, fn, ell, kind, eps, level)
        f = torch.zeros_like(w)
        m2l.m2l_apply_level(ops, lv, w, f, "fp64")
        m2l.m2l_sync_status(ops)
        outs[name] = f.cpu().numpy()
    off, src = lv.il_offsets.cpu().numpy(), lv.il_sources.cpu().numpy()
    exact = oracle.m2l_apply(oracle.operator_table(ell, kind, KIND_C[kind], level), cells, cells, off, src,
                             w.cpu().numpy())
    e_aca = oracle.rel_l2(outs["aca"], exact)
    e_svd = oracle.rel_l2(outs["svd"], exact)
    d = oracle.rel_l2(outs["aca"], outs["svd"])
    print("apply ell=%d eps=%g: ACA vs exact %.2e, SVD vs exact %.2e, ACA vs SVD %.2e" % (ell, eps, e_aca, e_svd, d))
    assert e_aca < 10 * eps and d < 10 * eps
