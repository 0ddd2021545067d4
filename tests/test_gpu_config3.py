"""The mixed-precision workload: N = 4,000,000 particles on the ellipsoid
surface with semi-axes (1, 0.5, 0.25), charges N(0,1) (seed 3), uniform-depth
octree to level 6 with empty cells pruned, ell = 7 (343 nodes), kernel 1/r^4,
per-operator truncated SVD at eps = 1e-7 (Eq. (20)).

Level 6 is applied with the low-rank and the full-rank operators in FP64 and
FP32 on the CUDA cores and compared on sampled targets with the oracle's
per-pair truncated operators; the relative L2 error of each precision
against the FP64 oracle is printed; the full-rank operators also run in the
tensor-core precisions (TF32, split BF16, split TF32 with FP32 accumulation),
and so do the low-rank factors (two tensor-core passes, Z = V_p^T W_p then
(U_p Sigma_p) Z), against the oracle's truncated operators."""
import numpy as np
import pytest

import oracle
from gpu_helpers import TOL, device

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


def test_config3_level6_lowrank_and_full(m2l):
    from paper_1210_7292_gb300 import synth
    ell, level, eps = 7, 6, 1e-7
    pts, q = synth.ellipsoid_surface(4_000_000, (1.0, 0.5, 0.25), seed=3)
    cells = synth.occupied_cells(pts, level)
    ijk = torch.from_numpy(cells).to(device())
    off, src = m2l.m2l_build_lists(ijk, ijk)
    lv = m2l.Level(oracle.cell_width(level), ijk, ijk, off, src, level)
    print("config3 level 6: %d non-empty cells, %d interactions" % (len(cells), lv.nnz))
    assert 4000 < len(cells) < 8000
    w = synth.gaussian_vectors(len(cells), ell ** 3, seed=33)
    ops_lr = m2l.m2l_precompute(m2l.M2L_K_INV_R4, ell, eps)
    ops_full = m2l.m2l_precompute(m2l.M2L_K_INV_R4, ell)
    ranks, _, _ = m2l.m2l_ops_query(ops_lr)
    tsym = oracle.t_sym_list()
    full_o = oracle.operator_table(ell, 1, 0.0, level)
    mult = {p: 0 for p in tsym}
    for t in oracle.transfer_vectors():
        mult[oracle.p_vector(t)] += 1
    mean_rank = sum(ranks[i] * mult[t] for i, t in enumerate(tsym)) / 316.0
    print("config3 ranks per operator:", list(ranks), "multiplicity-weighted mean %.1f" % mean_rank)
    assert 15 <= ranks.min() and ranks.max() <= 120
    rng = np.random.default_rng(34)
    samp = np.unique(rng.choice(len(cells), 40, replace=False))
    so, ss = oracle.interaction_lists(cells[samp], cells)
    lr_o, ranks_o = oracle.lowrank_operator_table(full_o, eps)
    ref_lr = oracle.m2l_apply(lr_o, cells[samp], cells, so, ss, w)
    ref_full = oracle.m2l_apply(full_o, cells[samp], cells, so, ss, w)
    # the truncation changes the result by about eps relative (Eckart-Young)
    assert oracle.rel_l2(ref_lr, ref_full) < 1e-5
    idx = torch.from_numpy(samp).to(device())
    errs = {}
    for name, ops in (("lowrank", ops_lr), ("full", ops_full)):
        for prec in ("fp64", "fp32"):
            dt = torch.float64 if prec == "fp64" else torch.float32
            loc = torch.zeros(len(cells), ell ** 3, dtype=torch.float64, device=device())
            m2l.m2l_apply_level(ops, lv, torch.from_numpy(w).to(device(), dt), loc, prec, locals_fp64=True)
            m2l.m2l_sync_status(ops)
            got = loc[idx].cpu().numpy()
            ref = ref_lr if name == "lowrank" else ref_full
            errs[(name, prec)] = oracle.rel_l2(got, ref)
            assert errs[(name, prec)] < TOL[prec], (name, prec, errs[(name, prec)])
    print("config3 rel L2 vs FP64 oracle:", {"%s/%s" % k: "%.2e" % v for k, v in errs.items()})
    # the tensor-core precisions on the full-rank operators (FP32 accumulation)
    for prec in ("tf32", "bf16x3", "tf32x3"):
        loc = torch.zeros(len(cells), ell ** 3, dtype=torch.float64, device=device())
        m2l.m2l_apply_level(ops_full, lv, torch.from_numpy(w).to(device(), torch.float32), loc, prec,
                            locals_fp64=True)
        m2l.m2l_sync_status(ops_full)
        errs[("full", prec)] = oracle.rel_l2(loc[idx].cpu().numpy(), ref_full)
        assert errs[("full", prec)] < TOL[prec], (prec, errs[("full", prec)])
    print("config3 tensor-core rel L2 vs FP64 oracle:",
          {p: "%.2e" % errs[("full", p)] for p in ("tf32", "bf16x3", "tf32x3")})
    # the tensor-core precisions on the low-rank factors (two passes)
    for prec in ("tf32", "bf16x3", "tf32x3"):
        loc = torch.zeros(len(cells), ell ** 3, dtype=torch.float64, device=device())
        m2l.m2l_apply_level(ops_lr, lv, torch.from_numpy(w).to(device(), torch.float32), loc, prec,
                            locals_fp64=True)
        m2l.m2l_sync_status(ops_lr)
        errs[("lowrank", prec)] = oracle.rel_l2(loc[idx].cpu().numpy(), ref_lr)
        assert errs[("lowrank", prec)] < TOL[prec], (prec, errs[("lowrank", prec)])
    print("config3 low-rank tensor-core rel L2 vs FP64 oracle:",
          {p: "%.2e" % errs[("lowrank", p)] for p in ("tf32", "bf16x3", "tf32x3")})


@pytest.mark.parametrize("ell,kind,level,keep,eps", [(5, 0, 3, 1.0, 1e-5), (6, 1, 3, 0.7, 1e-6), (5, 2, 4, 0.4, 1e-4)])
@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3", "tf32"])
def test_lowrank_tensor_cores_match_oracle(m2l, ell, kind, level, keep, eps, prec):
    """The low-rank tensor-core apply on whole levels (ell 5-6, three kernels,
    full and pruned levels, the adjoint too) against the oracle's truncated
    operators."""
    from gpu_helpers import KIND_C, gpu_ops, make_level, pruned_cells
    from paper_1210_7292_gb300 import synth
    cells = synth.full_grid(level) if keep == 1.0 else pruned_cells(level, keep, seed=ell + 13 * level)
    w = synth.gaussian_vectors(len(cells), ell ** 3, seed=91 + ell)
    lv = make_level(m2l, cells, level)
    ops = gpu_ops(m2l, ell, kind, level, eps=eps)
    off, src = oracle.interaction_lists(cells, cells)
    K, _ = oracle.lowrank_operator_table(oracle.operator_table(ell, kind, KIND_C[kind], level), eps)
    ref = oracle.m2l_apply(K, cells, cells, off, src, w)
    loc = torch.zeros(len(cells), ell ** 3, dtype=torch.float32, device=device())
    m2l.m2l_apply_level(ops, lv, torch.from_numpy(w).to(device(), torch.float32), loc, prec)
    m2l.m2l_sync_status(ops)
    err = oracle.rel_l2(loc.double().cpu().numpy(), ref)
    assert err < TOL[prec], err
    ref_adj = oracle.m2l_apply_adjoint(K, cells, cells, off, src, w, len(cells))
    adj = torch.zeros_like(loc)
    m2l.m2l_apply_level_adjoint(ops, lv, torch.from_numpy(w).to(device(), torch.float32), adj, prec)
    m2l.m2l_sync_status(ops)
    err_adj = oracle.rel_l2(adj.double().cpu().numpy(), ref_adj)
    assert err_adj < TOL[prec], err_adj
    print("low-rank %s ell=%d kind=%d level=%d: rel L2 %.2e, adjoint %.2e" % (prec, ell, kind, level, err, err_adj))
