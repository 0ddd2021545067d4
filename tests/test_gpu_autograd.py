"""Differentiation through the M2L translation: the hand-written adjoint behind
torch.autograd.Function, checked against the oracle's transposed apply,
central finite differences and torch.autograd.gradcheck."""
import numpy as np
import pytest

import oracle
from gpu_helpers import device, gpu_ops, make_level, oracle_ops, pruned_cells

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()
    from paper_1210_7292_gb300 import autograd, m2l
    return m2l, autograd


def test_gradcheck_fp64_small(mods):
    m2l, ag = mods
    level, ell = 3, 2
    cells = pruned_cells(level, 0.5, 40)
    lv = make_level(m2l, cells, level)
    op = ag.M2LLevelOperator(gpu_ops(m2l, ell, 0, level), lv, "fp64")
    w = torch.randn(len(cells), ell ** 3, dtype=torch.float64, device=device(), requires_grad=True)
    # the map is linear, so a large step is exact; it keeps the rounding noise of the
    # atomic accumulation (order-dependent in the last bits) far below the tolerance
    assert torch.autograd.gradcheck(op, (w,), eps=1e-2, atol=1e-8, rtol=1e-7, nondet_tol=1e-10)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 2e-6), ("bf16x3", 5e-5), ("tf32x3", 2e-6)])
def test_dot_product_identity(mods, prec, tol):
    m2l, ag = mods
    level, ell = 4, 4
    cells = pruned_cells(level, 0.6, 41)
    lv = make_level(m2l, cells, level)
    op = ag.M2LLevelOperator(gpu_ops(m2l, ell, 0, level), lv, prec)
    g = torch.Generator(device="cpu").manual_seed(3)
    w = torch.randn(len(cells), ell ** 3, generator=g, dtype=torch.float64).to(device(), op.dtype)
    gl = torch.randn(len(cells), ell ** 3, generator=g, dtype=torch.float64).to(device(), op.dtype)
    a = float((gl.double() * op.apply_forward(w).double()).sum())
    b = float((op.apply_adjoint(gl).double() * w.double()).sum())
    assert abs(a - b) <= tol * (abs(a) + abs(b)), (a, b)


def test_config5_level6_gradient(mods):
    """Full level 6 (262 144 cells, 46 298 376 interactions), ell = 5, 1/r, FP32
    forward and backward; loss = sum(W * locals), w ~ N(0,1) seed 5, W ~ N(0,1) seed 6.
    The gradient is checked on sampled source cells against the oracle's FP64
    transposed apply and, for a few entries, against central differences."""
    m2l, ag = mods
    from paper_1210_7292_gb300 import synth
    level, ell = 6, 5
    cells = synth.full_grid(level)
    lv = make_level(m2l, cells, level)
    assert lv.nnz == 46298376
    ops = gpu_ops(m2l, ell, 0, level)
    op = ag.M2LLevelOperator(ops, lv, "fp32")
    w_np = synth.gaussian_vectors(len(cells), ell ** 3, seed=5)
    W_np = synth.gaussian_vectors(len(cells), ell ** 3, seed=6)
    w = torch.from_numpy(w_np).to(device(), torch.float32).requires_grad_(True)
    W = torch.from_numpy(W_np).to(device(), torch.float32)
    loss = (W * op(w)).sum()
    loss.backward()
    grad = w.grad.double().cpu().numpy()
    m2l.m2l_sync_status(ops)

    # oracle: g_Y = sum over targets X with Y in list(X) of K_{X-Y}^T W_X, FP64
    rng = np.random.default_rng(13)
    samp = np.unique(np.concatenate([[0, len(cells) - 1], rng.choice(len(cells), 30, replace=False)]))
    off_s, src_s = oracle.interaction_lists(cells[samp], cells)     # the far-field relation is symmetric
    touched = np.unique(src_s)
    pos = {int(y): i for i, y in enumerate(samp)}
    off_t, src_t = oracle.interaction_lists(cells[touched], cells)
    t_off = [0]
    t_src = []
    for i in range(len(touched)):
        keep = [pos[int(y)] for y in src_t[off_t[i]:off_t[i + 1]] if int(y) in pos]
        t_src.extend(keep)
        t_off.append(len(t_src))
    ref = oracle.m2l_apply_adjoint(oracle_ops(ell, 0, level), cells[touched], cells[samp],
                                   np.array(t_off, np.int32), np.array(t_src, np.int32), W_np[touched], len(samp))
    err = oracle.rel_l2(grad[samp], ref)
    assert err < 5e-6, err

    # Central differences, h = 1e-3, summed over the targets the perturbed source
    # touches (the others cancel).  (i) Through the FP64 forward: the map is linear, so
    # the difference quotient is the exact derivative up to FP64 rounding, and the FP32
    # gradient must match it to FP32 accuracy.  (ii) Through the FP32 forward: each
    # product column is re-rounded in FP32 when w changes, which leaves noise of about
    # u32 * |F| * sqrt(#locals touched) / (2 h) ~ 6 on a derivative of ~1e2 here, so
    # this quotient is only held to 10 %.
    h = 1e-3
    w64 = w.detach().double()
    for y, b in [(int(samp[3]), 7), (int(samp[-1]), 100), (0, 0)]:
        tl = oracle.interaction_lists(cells[[y]], cells)[1]
        for prec, tol in (("fp64", 1e-4), ("fp32", 0.1)):
            vals = []
            for sgn in (1.0, -1.0):
                wp = (w64 if prec == "fp64" else w.detach()).clone()
                wp[y, b] += sgn * h
                loc = torch.zeros(len(cells), ell ** 3, dtype=torch.float64, device=device())
                m2l.m2l_plan_apply(op.fwd, wp, loc, prec, out_fp64=True)
                vals.append(float((W[tl].double() * loc[tl]).sum()))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - grad[y, b]) <= tol * max(1.0, abs(grad[y, b])), (prec, y, b, fd, grad[y, b])
