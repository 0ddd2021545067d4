"""Pins of the dFMM oracle (oracle/dfmm_oracle.py) to facts the paper and the
mathematics fix, independent of the oracle's own formulas:

* k = 0 turns the Helmholtz operator into the 1/r operator of the bbFMM
  oracle (its C assembly from absolute nodes);
* the 48 signed axis permutations map K_t onto K_{p(t)} for transfer vectors
  far outside [-3, 3]^3 (the kernel is radial; Sec. 4.2.1);
* Eq. (10): with the cone direction, the interpolation error of K^u decays in
  ell at a rate that does not depend on k w, while the plain kernel and the
  reversed direction degrade as k w grows;
* Eqs. (11)-(14): directional P2M, M2L with K (not K^u) and L2P reproduce the
  direct sum of one separated pair;
* Alg. 1: the level-wise lists equal the literal recursion from the roots, and
  near and far fields cover every pair of leaves exactly once;
* the cones partition the directions and nest from level to level;
* the cell-by-cell M2L equals a brute-force sum with operators assembled from
  the cells' own interpolation points.
"""
import itertools

import numpy as np
import pytest

import oracle

d = oracle.dfmm


def test_k0_reduces_to_the_laplace_operator():
    for ell, level, t in [(3, 3, (2, 0, 0)), (4, 4, (3, -2, 1)), (5, 2, (-3, 3, -3))]:
        K = d.dfmm_operator_for_t(ell, 0.0, level, t)
        ref = oracle.operator_for_t(ell, 0, 0.0, level, t)
        assert np.abs(K.imag).max() == 0.0
        assert np.abs(K.real - ref).max() <= 1e-13 * np.abs(ref).max()


def test_symmetries_hold_for_large_transfer_vectors():
    g = np.random.default_rng(1)
    ell, k, level = 4, 32.0, 4
    for _ in range(12):
        t = tuple(int(v) for v in g.integers(-12, 13, 3))
        if max(abs(v) for v in t) < 2:
            continue
        p = oracle.p_vector(t)
        assert p == d.canonical_t(t)
        s = oracle.sigma_of_t(t, ell)
        Kt = d.dfmm_operator_for_t(ell, k, level, t)
        Kp = d.dfmm_operator_for_t(ell, k, level, p)
        assert np.abs(Kt - Kp[np.ix_(s, s)]).max() <= 1e-13 * np.abs(Kt).max()


def _pair(level, t, k):
    w = d.level_width(level, 2.0)
    m = d.cone_m(k, w)
    u = d.cone_direction(m, d.cone_index(m, t))
    X = np.asarray(t) + 40
    Y = np.full(3, 40)
    return w, u, oracle.cell_center(X, level), oracle.cell_center(Y, level)


def test_directional_interpolation_is_independent_of_kw():
    k = 32.0
    errs = {}
    for level, t in [(5, (3, 1, 1)), (4, (5, 1, 0)), (3, (9, 2, 1))]:   # k w = 2, 4, 8
        w, u, xc, yc = _pair(level, t, k)
        assert d.admissible(k, w, t)
        e = [d.interpolation_error(ell, k, u, xc, yc, w) for ell in (3, 5, 7)]
        assert e[0] > 10 * e[1] > 100 * e[2]            # exponential decay in ell
        errs[level] = e[2]
        plain = d.interpolation_error(7, k, np.zeros(3), xc, yc, w)
        reversed_ = d.interpolation_error(7, k, -u, xc, yc, w)
        if k * w >= 4:
            assert plain > 50 * e[2] and reversed_ > 1000 * e[2]
    assert max(errs.values()) < 10 * min(errs.values())   # the same rate at k w = 2, 4, 8
    assert max(errs.values()) < 1e-5


def test_fast_summation_of_one_pair_matches_direct_sum():
    k, level, t = 32.0, 3, (9, 2, 1)
    w, u, xc, yc = _pair(level, t, k)
    g = np.random.default_rng(2)
    xs = xc + w * (g.random((40, 3)) - 0.5)
    ys = yc + w * (g.random((50, 3)) - 0.5)
    q = g.standard_normal(50)
    exact = d.helmholtz_direct(k, xs, ys, q)
    errs = []
    for ell in (5, 7, 9):
        W = d.dfmm_p2m(ell, k, u, ys, q, yc, w)
        F = d.dfmm_operator(ell, k, xc, yc, w) @ W
        f = d.dfmm_l2p(ell, k, u, xs, xc, w, F)
        errs.append(oracle.rel_l2(f, exact))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-6, errs
    # the M2L takes the plain kernel: K^u in its place gives a wrong sum
    W = d.dfmm_p2m(7, k, u, ys, q, yc, w)
    xn, yn = oracle.cell_nodes(7, xc, w), oracle.cell_nodes(7, yc, w)
    Ku = d.helmholtz_directional(k, u, xn[:, None, :], yn[None, :, :])
    assert oracle.rel_l2(d.dfmm_l2p(7, k, u, xs, xc, w, Ku @ W), exact) > 0.1


def _tiny_tree(n=120, seed=3, leaf=5):
    from paper_1210_7292_gb300 import synth
    pts, _ = synth.sphere_surface(n, seed=seed)
    return {L: synth.occupied_cells(pts, L) for L in range(leaf + 1)}


def _csr_from_far(far_L, ncells, C):
    rows = [far_L.get((x, c), []) for x in range(ncells) for c in range(C)]
    off = np.zeros(len(rows) + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(r) for r in rows])
    return off, np.asarray([y for r in rows for y in r], dtype=np.int64)


@pytest.mark.parametrize("k", [8.0, 3.0])
def test_level_lists_equal_the_recursion_of_alg1(k):
    leaf = 5
    cells = _tiny_tree(leaf=leaf)
    far, near = d.separate_recursive(cells, leaf, k, 2.0)
    total = 0
    for L in range(leaf + 1):
        C, off, src = d.directional_lists(cells[L], L, k, 2.0)
        assert C == d.n_cones(k, d.level_width(L, 2.0))
        off_r, src_r = _csr_from_far(far[L], len(cells[L]), C)
        assert np.array_equal(off, off_r) and np.array_equal(src, src_r), L
        total += len(src)
    assert total > 0 and near


def test_near_and_far_cover_every_leaf_pair_once():
    leaf, k = 5, 8.0
    cells = _tiny_tree(leaf=leaf)
    far, near = d.separate_recursive(cells, leaf, k, 2.0)
    covered = {L: set() for L in far}
    for L in far:
        for (x, _c), ys in far[L].items():
            for y in ys:
                covered[L].add((x, y))
    index = {L: {tuple(int(v) for v in c): i for i, c in enumerate(cells[L])} for L in cells}
    leaves = cells[leaf]
    for xi, X in enumerate(leaves):
        for yi, Y in enumerate(leaves):
            n = int(yi in near.get(xi, []))
            for L in range(leaf + 1):
                sh = leaf - L
                ax = index[L][tuple(int(v) >> sh for v in X)]
                ay = index[L][tuple(int(v) >> sh for v in Y)]
                n += int((ax, ay) in covered[L])
            assert n == 1, (X, Y, n)


def test_cones_partition_and_nest():
    for m in (1, 2, 4, 8):
        hit = set()
        for t in itertools.product(range(-9, 10), repeat=3):
            if max(abs(v) for v in t) < 2:
                continue
            c = d.cone_index(m, t)
            assert 0 <= c < 6 * m * m
            hit.add(c)
            # the direction lies in the face square around u_c (gnomonic half-width 1/m)
            u = d.cone_direction(m, c)
            f = int(np.argmax(np.abs(u)))
            v = np.asarray(t, dtype=np.float64) / abs(t[f])
            uu = u / abs(u[f])
            assert np.sign(t[f]) == np.sign(u[f])
            assert np.abs(v - uu).max() <= 1.0 / m + 1e-12
            if m > 1:   # nested: the cone of the coarser level contains it
                cp = d.cone_index(m // 2, t)
                face, rem = divmod(c, m * m)
                ib, ia = divmod(rem, m)
                assert cp == face * (m // 2) ** 2 + (ib // 2) * (m // 2) + ia // 2
        if m <= 4:
            assert len(hit) == 6 * m * m


def test_m2l_matches_brute_force():
    k, level, ell = 8.0, 3, 2
    cells = _tiny_tree(n=200, seed=4, leaf=level)[level]
    C, off, src = d.directional_lists(cells, level, k, 2.0)
    assert len(src) > 0
    g = np.random.default_rng(5)
    W = g.standard_normal((len(cells) * C, ell ** 3)) + 1j * g.standard_normal((len(cells) * C, ell ** 3))
    F = d.dfmm_m2l_apply(ell, k, level, cells, cells, C, off, src, W)
    w = d.level_width(level, 2.0)
    ref = np.zeros_like(F)
    for e in range(len(cells) * C):
        x = e // C
        for j in range(off[e], off[e + 1]):
            y = src[j]
            xn = oracle.cell_nodes(ell, oracle.cell_center(cells[x], level), w)
            yn = oracle.cell_nodes(ell, oracle.cell_center(cells[y], level), w)
            for a in range(ell ** 3):
                for b in range(ell ** 3):
                    r = np.sqrt(((xn[a] - yn[b]) ** 2).sum())
                    ref[e, a] += np.exp(1j * k * r) / r * W[y * C + e % C, b]
    assert oracle.rel_l2(F, ref) < 1e-13


@pytest.mark.parametrize("geometry", ["sphere", "oblate", "prolate"])
def test_list_sizes_match_the_paper(geometry):
    """The paper's geometries (boxes of side 64, k = 1) are, on the unit domain,
    surfaces with the same axis ratios and k = 32: only k times the domain width
    enters.  |T| and |T_sym| of the directional lists are the printed ones at
    every printed level, for the sphere, the oblate and the prolate spheroid
    (high- and low-frequency levels)."""
    import json
    import os
    from paper_1210_7292_gb300 import synth
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "dfmm_list_sizes.json")))
    geo = gold["geometry"]
    k = geo["wavenumber"] * geo["box"] / 2.0
    g = gold["geometries"][geometry]
    axes = tuple(0.999 * a for a in g["semi_axes_over_half_box"])
    if geometry == "sphere":
        pts, _ = synth.sphere_surface(g["particles"], seed=g["seed"])
    else:
        pts, _ = synth.ellipsoid_surface(g["particles"], axes, seed=g["seed"])
    for L in g["reproduced_levels"]:
        ref = g["levels"][str(L)]
        cells = synth.occupied_cells(pts, L)
        C, off, src = d.directional_lists(cells, L, k, 2.0)
        x = np.repeat(np.arange(len(off) - 1) // C, np.diff(off))
        T = np.unique(cells[x].astype(np.int64) - cells[src].astype(np.int64), axis=0)
        Tsym = {d.canonical_t(t) for t in T}
        assert [len(T), len(Tsym)] == ref, (geometry, L)
