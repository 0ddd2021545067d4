"""The bbFMM matvec on the GPU (m2l_fmm_*): P2M, M2M, M2L per level, L2L,
L2P and the near field against the oracle's FMM of the same tree (multipoles
per level, potentials at sampled particles) and against the direct sum."""
import numpy as np
import pytest

import oracle
from gpu_helpers import KIND_C, device

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


def _ops(m2l, ell, kind, leaf):
    if kind == 2:   # not homogeneous: one operator set per level width
        return {L: m2l.m2l_precompute(kind, ell, 0.0, oracle.cell_width(L), KIND_C[kind]) for L in range(2, leaf + 1)}
    return m2l.m2l_precompute(kind, ell, 0.0, 0.0, KIND_C[kind])


def _gpu_fmm(m2l, pts, q, ell, kind, leaf, prec="fp64"):
    dt = torch.float64 if prec == "fp64" else torch.float32
    xyz = torch.from_numpy(np.ascontiguousarray(pts)).to(device(), dt)
    qq = torch.from_numpy(np.ascontiguousarray(q)).to(device(), dt)
    fmm = m2l.m2l_fmm_create(_ops(m2l, ell, kind, leaf), xyz, leaf)
    phi = torch.zeros(len(q), dtype=dt, device=device())
    m2l.m2l_fmm_evaluate(fmm, xyz, qq, phi, prec)
    torch.cuda.synchronize()
    return fmm, phi.double().cpu().numpy()


@pytest.mark.parametrize("geometry,n,ell,kind,leaf", [("cube", 3000, 4, 0, 3), ("ellipsoid", 20000, 4, 1, 4),
                                                       ("cube", 6000, 5, 2, 3), ("sphere", 12000, 3, 0, 4)])
def test_fmm_fp64_matches_oracle(m2l, geometry, n, ell, kind, leaf):
    from paper_1210_7292_gb300 import synth
    if geometry == "cube":
        pts, q = synth.uniform_cube(n, seed=31)
    elif geometry == "ellipsoid":
        pts, q = synth.ellipsoid_surface(n, seed=32)
    else:
        pts, q = synth.sphere_surface(n, seed=33)
    fmm, phi = _gpu_fmm(m2l, pts, q, ell, kind, leaf)
    c = KIND_C[kind]
    up = oracle.UpwardPass(ell, leaf, pts, q)
    # the tree: kept cells and multipoles per level (P2M, M2M)
    for L in range(2, leaf + 1):
        ijk, W, _ = m2l.m2l_fmm_query(fmm, L)
        cells, Wref = up.levels[L]
        assert np.array_equal(ijk, cells), L
        assert oracle.rel_l2(W, Wref) < 1e-12, (L, oracle.rel_l2(W, Wref))
    # potentials at sampled particles (M2L, L2L, L2P, near field)
    samp = np.sort(np.random.default_rng(5).choice(n, 150, replace=False))
    ref = oracle.fmm_at_samples(up, kind, c, oracle.fmm_oracle_locals(up, kind, c), samp)
    err = oracle.rel_l2(phi[samp], ref)
    assert err < 1e-11, err
    # and the FMM approximates the direct sum to its interpolation order
    exact = oracle.direct_sum(kind, c, pts[samp], pts, q)
    approx = oracle.rel_l2(phi[samp], exact)
    print("%s n=%d ell=%d kind=%d leaf=%d: vs oracle FMM %.2e, vs direct sum %.2e" % (geometry, n, ell, kind, leaf,
                                                                                   err, approx))
    assert approx < 10.0 ** (2 - ell), approx


@pytest.fixture(scope="module")
def fp32_case():
    """40,000 uniform particles, ell = 5, leaf level 4, 1/r: the oracle's FMM
    potentials and the direct sum at 200 sampled particles."""
    from paper_1210_7292_gb300 import synth
    pts, q = synth.uniform_cube(40000, seed=34)
    up = oracle.UpwardPass(5, 4, pts, q)
    samp = np.sort(np.random.default_rng(6).choice(len(q), 200, replace=False))
    ref = oracle.fmm_at_samples(up, 0, 0.0, oracle.fmm_oracle_locals(up, 0, 0.0), samp)
    exact = oracle.direct_sum(0, 0.0, pts[samp], pts, q)
    return pts, q, samp, ref, exact


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("tf32x3", 1e-5), ("bf16x3", 1e-4)])
def test_fmm_fp32_precisions(m2l, fp32_case, prec, tol):
    """FP32 passes with the M2L in each FP32-accurate precision against the
    oracle's FMM (FP64, directly assembled operators) at sampled particles,
    and at equal error: the error against the direct sum stays within 10 % of
    the oracle FMM's own."""
    pts, q, samp, ref, exact = fp32_case
    _, phi = _gpu_fmm(m2l, pts, q, 5, 0, 4, prec)
    err = oracle.rel_l2(phi[samp], ref)
    e_gpu, e_ref = oracle.rel_l2(phi[samp], exact), oracle.rel_l2(ref, exact)
    print("FMM %s: vs oracle FMM %.2e; vs direct sum %.3e (oracle FMM %.3e)" % (prec, err, e_gpu, e_ref))
    assert err < tol, err
    assert e_gpu <= 1.10 * e_ref, (e_gpu, e_ref)


def test_fmm_info_and_bad_arguments(m2l):
    from paper_1210_7292_gb300 import synth
    pts, q = synth.uniform_cube(20000, seed=35)
    fmm, _ = _gpu_fmm(m2l, pts, q, 3, 0, 3)
    leaf, nc, nz = m2l.m2l_fmm_info(fmm)
    assert leaf == 3 and nc[2] == 64 and nc[3] == 512 and nz[2] == 3096 and nz[3] == 53352
    xyz = torch.from_numpy(pts).to(device())
    qq = torch.from_numpy(q).to(device())
    phi = torch.zeros(len(q), dtype=torch.float64, device=device())
    with pytest.raises(m2l.M2LError) as ei:
        m2l.m2l_fmm_evaluate(fmm, xyz, qq, phi, "bf16x3")   # FP64 FMM with an FP32 product
    assert ei.value.status == m2l.M2L_EINVAL
    with pytest.raises(m2l.M2LError) as ei:
        m2l.m2l_fmm_create(m2l.m2l_precompute(0, 3), xyz, 9)
    assert ei.value.status == m2l.M2L_EINVAL
