"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: counts the
paper prints, closed forms, invariants of the reflection group, library
routines (numpy's Chebyshev module, SVD), brute force on tiny inputs, and the
convergence of the whole FMM to the direct sum.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle as o

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden():
    with open(os.path.join(GOLDEN, "paper_counts.json")) as f:
        return json.load(f)


def _signed_perms():
    """All 48 signed axis permutations as 3x3 integer matrices (brute force)."""
    out = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            M = np.zeros((3, 3), dtype=int)
            for r in range(3):
                M[r, perm[r]] = signs[r]
            out.append(M)
    return out


# ---------------------------------------------------------------- counts
def test_paper_counts():
    g = _golden()
    T = o.transfer_vectors()
    assert len(T) == g["distinct_transfer_vectors_per_level"]["value"]
    assert len(o.t_sym_list()) == g["unique_operators_bbfmm"]["value"]
    near = [t for t in itertools.product(range(-1, 2), repeat=3)]
    assert len(near) == g["near_field_per_cell"]["value"]
    # an interior cell at level 4: its list holds the 216 children of the parent's
    # 27 neighbours minus its own 27 neighbours
    cells = o.full_grid_cells(4)
    off, src = o.interaction_lists(cells, cells)
    sizes = np.diff(off)
    assert sizes.max() == g["max_far_per_cell"]["value"]
    assert g["children_near_and_far"]["value"] - g["near_field_per_cell"]["value"] == sizes.max()
    flips = {o.g_index(t) % 8 for t in T}
    orders = {o.g_index(t) // 8 for t in T}
    assert len(flips) == g["axial_octants"]["value"]
    assert len(orders) == g["diagonal_cones"]["value"]


def test_tsym_is_orbit_representatives():
    """T_sym holds exactly one vector of each orbit of T under the 48 reflections."""
    T = set(o.transfer_vectors())
    G = _signed_perms()
    orbits = set()
    for t in T:
        orbits.add(frozenset(tuple(int(v) for v in M @ np.array(t)) for M in G))
    assert sum(len(orb) for orb in orbits) == len(T) == 316
    tsym = o.t_sym_list()
    assert len(orbits) == len(tsym)
    for orb in orbits:
        reps = [t for t in orb if t in tsym]
        assert len(reps) == 1
        for t in orb:
            assert o.p_vector(t) == reps[0]
    # multiplicities n_p of Alg. 2 are orbit sizes 48 / |stabiliser|
    mult = {o.p_vector(t): 0 for t in T}
    for t in T:
        mult[o.p_vector(t)] += 1
    for p, n in mult.items():
        stab = sum(1 for M in G if tuple(int(v) for v in M @ np.array(p)) == p)
        assert n * stab == 48


def test_level_totals_closed_form():
    """Full-grid list totals equal A^3 - B^3 with per-axis pair counts (separability)."""
    for L in (2, 3, 4):
        n = 1 << L
        A = sum(1 for x in range(n) for y in range(n) if abs((x >> 1) - (y >> 1)) <= 1)
        B = sum(1 for x in range(n) for y in range(n) if abs(x - y) <= 1)
        cells = o.full_grid_cells(L)
        off, src = o.interaction_lists(cells, cells)
        assert off[-1] == A ** 3 - B ** 3
    # the level-3 total is the config-1 interaction count
    assert (40 ** 3 - 22 ** 3) == 53352


def test_lists_match_brute_force_on_pruned_level():
    """Candidate enumeration equals the all-pairs admissibility test (level 3, pruned)."""
    rng = np.random.default_rng(11)
    cells = o.full_grid_cells(3)
    keep = rng.random(len(cells)) < 0.6
    cells = cells[keep]
    off, src = o.interaction_lists(cells, cells)
    for x in range(len(cells)):
        brute = [y for y in range(len(cells))
                 if o.is_far_pair(tuple(cells[x]), tuple(cells[y]))]
        assert list(src[off[x]:off[x + 1]]) == brute


# ---------------------------------------------------------------- nodes
def test_chebyshev_roots_closed_forms():
    assert np.allclose(o.cheb_roots(1), [0.0])
    assert np.allclose(o.cheb_roots(2), [-1 / np.sqrt(2), 1 / np.sqrt(2)], rtol=0, atol=1e-15)
    assert np.allclose(o.cheb_roots(3), [-np.sqrt(3) / 2, 0.0, np.sqrt(3) / 2], rtol=0, atol=1e-15)
    for ell in range(1, 10):
        r = o.cheb_roots(ell)
        assert np.all(np.diff(r) > 0)
        coef = np.zeros(ell + 1)
        coef[ell] = 1.0
        assert np.max(np.abs(np.polynomial.chebyshev.chebval(r, coef))) < 1e-13
        ref = np.sort(np.polynomial.chebyshev.chebroots(coef))
        assert np.allclose(r, ref, rtol=0, atol=1e-12)


def test_index_map_x_fastest():
    for ell in (2, 3, 5):
        mi = o.multi_indices(ell)
        assert len({tuple(r) for r in mi}) == ell ** 3
        assert tuple(mi[1]) == (1, 0, 0)
        assert tuple(mi[ell]) == (0, 1, 0)
        assert tuple(mi[ell * ell]) == (0, 0, 1)
        for j in range(ell ** 3):
            assert o.m_of(mi[j], ell) == j


def test_lagrange_basis_properties():
    for ell in (2, 3, 5, 7):
        xi = o.cheb_roots(ell)
        assert np.allclose(o.lagrange_1d(ell, xi), np.eye(ell), atol=1e-13)
        x = np.linspace(-1, 1, 37)
        L = o.lagrange_1d(ell, x)
        assert np.allclose(L.sum(axis=1), 1.0, atol=1e-12)


def test_interpolation_exact_below_degree_ell():
    """S_ell reproduces tensor polynomials of degree < ell per axis (Eq. (2))."""
    rng = np.random.default_rng(3)
    for ell in (3, 4, 6):
        center, w = np.array([0.3, -0.2, 0.1]), 0.5
        nodes = o.cell_nodes(ell, center, w)
        pts = center + 0.5 * w * rng.uniform(-1, 1, (50, 3))
        S = o.interp_matrix(ell, pts, center, w)
        for deg in itertools.product(range(ell), repeat=3):
            f = lambda p: np.prod(p ** np.array(deg), axis=1)
            assert np.allclose(S @ f(nodes), f(pts), rtol=1e-10, atol=1e-12)
        # one degree higher is not reproduced
        f = lambda p: p[:, 0] ** ell
        assert np.max(np.abs(S @ f(nodes) - f(pts))) > 1e-6


def test_m2m_equals_direct_p2m_to_parent():
    rng = np.random.default_rng(5)
    ell = 4
    pts = rng.uniform(-1, 1, (400, 3))
    q = rng.standard_normal(400)
    cells4, W4 = o.p2m(ell, 4, pts, q)
    parents, W3 = o.m2m(ell, cells4, W4)
    cells3, W3d = o.p2m(ell, 3, pts, q)
    assert np.array_equal(parents, cells3)
    assert np.allclose(W3, W3d, rtol=1e-11, atol=1e-11)


# ---------------------------------------------------------------- symmetry
def test_model_example_2d():
    """The 2-D model example of Sec. 4.2.1 (Fig. 1, Fig. 2), embedded with t3 = 0."""
    g = _golden()["model_example_2d"]
    ell = g["ell"]
    ref, ax, dg, comb = (tuple(g[k]) + (0,) for k in ("t_ref", "t_axial", "t_diag", "t_combined"))
    assert o.p_vector(ax) == ref and o.p_vector(dg) == ref and o.p_vector(comb) == ref
    mi = o.multi_indices(ell)
    flip1 = [o.m_of((ell - 1 - a[0], a[1], a[2]), ell) for a in mi]      # Eq. (21)
    swap12 = [o.m_of((a[1], a[0], a[2]), ell) for a in mi]              # Eq. (22)
    assert list(o.sigma_of_t(ax, ell)) == flip1
    assert list(o.sigma_of_t(dg, ell)) == swap12
    # (-1, 2): axial flip first, then the diagonal swap (reflections do not commute)
    first_flip_then_swap = [o.m_of((a[1], ell - 1 - a[0], a[2]), ell) for a in mi]
    first_swap_then_flip = [o.m_of((ell - 1 - a[1], a[0], a[2]), ell) for a in mi]
    assert list(o.sigma_of_t(comb, ell)) == first_flip_then_swap
    assert first_flip_then_swap != first_swap_then_flip
    for level in (2, 3):
        Kr = o.operator_for_t(ell, 0, 0.0, level, ref)
        for t in (ax, dg, comb):
            s = o.sigma_of_t(t, ell)
            Kt = o.operator_for_t(ell, 0, 0.0, level, t)
            assert np.allclose(Kt, Kr[np.ix_(s, s)], rtol=1e-14, atol=0)
            # entries themselves differ before the permutation (Sec. 4.2.1)
            assert not np.allclose(Kt, Kr, rtol=1e-6)


def test_sigma_tables_group_properties():
    for ell in (2, 3, 4, 5):
        T = o.transfer_vectors()
        tab = o.sigma_tables(ell)
        assert tab.shape == (48, ell ** 3)
        for g in range(48):
            assert sorted(tab[g]) == list(range(ell ** 3))
        assert len({tuple(r) for r in tab}) == 48
        for t in T:
            assert np.array_equal(o.sigma_of_t(t, ell), tab[o.g_index(t)])
            if o.in_z_sym(t):
                assert np.array_equal(o.sigma_of_t(t, ell), np.arange(ell ** 3))
        assert {o.g_index(t) for t in T} == set(range(48))


@pytest.mark.parametrize("ell,kind", [(3, 0), (4, 0), (5, 0), (4, 1), (4, 2)])
def test_reflection_identity_all_316(ell, kind):
    """K_t[a, b] = K_{p(t)}[sigma_t(a), sigma_t(b)] for every t (Eq. (25)).

    The reverse orientation (sigma_t^{-1}) must fail exactly for the sigma
    that are not involutions, which pins the reading of P_t.
    """
    c = 0.01 if kind == 2 else 0.0
    level = 3
    ops = o.operator_table(ell, kind, c, level)
    lut = o.lut343()
    tsym = o.t_sym_list()
    n_fail_inverse = 0
    n_non_involution = 0
    for t in o.transfer_vectors():
        s = o.t_slot(t)
        p, g = int(lut[s]) & 0xFF, int(lut[s]) >> 8
        assert tsym[p] == o.p_vector(t)
        sig = o.sigma_of_t(t, ell)
        Kp = ops[o.t_slot(tsym[p])]
        Kt = ops[s]
        rel = np.max(np.abs(Kp[np.ix_(sig, sig)] - Kt)) / np.max(np.abs(Kt))
        assert rel < 4e-15
        inv = np.argsort(sig)
        if np.max(np.abs(Kp[np.ix_(inv, inv)] - Kt)) / np.max(np.abs(Kt)) > 1e-10:
            n_fail_inverse += 1
        if not np.array_equal(sig[sig], np.arange(ell ** 3)):
            n_non_involution += 1
    assert n_fail_inverse == n_non_involution > 0


def test_lut_encoding():
    lut = o.lut343()
    for t in itertools.product(range(-3, 4), repeat=3):
        v = int(lut[o.t_slot(t)])
        if max(map(abs, t)) <= 1:
            assert v == 0xFFFF
        else:
            assert (v & 0xFF) < 16 and (v >> 8) < 48


def test_transpose_identity():
    """K_{-t} = K_t^T: the kernel is symmetric, K(x, y) = K(y, x)."""
    ops = o.operator_table(4, 0, 0.0, 3)
    for t in o.transfer_vectors():
        mt = tuple(-v for v in t)
        A, B = ops[o.t_slot(t)], ops[o.t_slot(mt)]
        assert np.max(np.abs(A - B.T)) <= 1e-15 * np.max(np.abs(A))


@pytest.mark.parametrize("kind,n", [(0, -1), (1, -4)])
def test_homogeneity_across_levels(kind, n):
    """K(alpha r) = alpha^n K(r) (Sec. 3.2): halving the width scales K_t by 2^-n."""
    assert o.homogeneity_degree(kind) == n
    for t in [(2, 0, 0), (3, -1, 2), (-3, -3, -3)]:
        K3 = o.operator_for_t(4, kind, 0.0, 3, t)
        K4 = o.operator_for_t(4, kind, 0.0, 4, t)
        assert np.allclose(K4, K3 * 2.0 ** (-n), rtol=1e-13, atol=0)


def test_singular_values_invariant_under_reflection():
    ops = o.operator_table(4, 0, 0.0, 2)
    tsym = o.t_sym_list()
    for t in o.transfer_vectors():
        s1 = np.linalg.svd(ops[o.t_slot(t)], compute_uv=False)
        s2 = np.linalg.svd(ops[o.t_slot(o.p_vector(t))], compute_uv=False)
        assert np.allclose(s1, s2, rtol=1e-12, atol=1e-12 * s1[0])
    assert len(tsym) == 16


def test_eckart_young_truncation():
    """Spectral reading: s_r > eps s_1 >= s_{r+1} and |K - U V^T|_2 = s_{r+1};
    Frobenius reading: |K - U V^T|_F <= eps |K|_F < |K - K_{r-1}|_F, both
    norms taken of the difference matrix itself (Eckart-Young)."""
    ops = o.operator_table(5, 1, 0.0, 3)
    for t in [(2, 0, 0), (3, 1, -2), (-3, 3, 3)]:
        K = ops[o.t_slot(t)]
        s = np.linalg.svd(K, compute_uv=False)
        nf = np.linalg.norm(K, "fro")
        for eps in (1e-3, 1e-6, 1e-9):
            U, V, r = o.lowrank(K, eps, o.SPECTRAL)
            assert s[r - 1] > eps * s[0]
            if r < len(s):
                assert s[r] <= eps * s[0]
                err2 = np.linalg.norm(K - U @ V.T, 2)
                assert abs(err2 - s[r]) <= 1e-9 * s[0]
            U, V, r = o.lowrank(K, eps, o.FROBENIUS)
            assert np.linalg.norm(K - U @ V.T, "fro") <= eps * nf * (1 + 1e-9) + 1e-14 * nf
            Um, Vm, _ = o.lowrank(K, 0.0)
            K_rm1 = (Um[:, :r - 1]) @ Vm[:, :r - 1].T
            assert np.linalg.norm(K - K_rm1, "fro") > eps * nf
            # the Frobenius tail keeps at least as many terms as the spectral reading
            assert r >= o.truncation_rank(s, eps, o.SPECTRAL)
    for crit in (o.SPECTRAL, o.FROBENIUS):
        assert o.truncation_rank(np.array([3.0, 2.0, 1.0]), 0.0, crit) == 3
    # hand-checkable cases: s = (1, 0.1, 0.01); tails^2 = 1.0101, 0.0101, 1e-4
    sv = np.array([1.0, 0.1, 0.01])
    assert o.truncation_rank(sv, 0.05, o.SPECTRAL) == 2        # 0.1 > 0.05 >= 0.01
    assert o.truncation_rank(sv, 0.05, o.FROBENIUS) == 2       # 1e-4 <= 0.0025 * 1.0101 < 0.0101
    assert o.truncation_rank(sv, 0.0099, o.FROBENIUS) == 3     # 1e-4 > 0.0099^2 * 1.0101
    assert o.truncation_rank(sv, 0.0099, o.SPECTRAL) == 3
    with pytest.raises(ValueError):
        o.truncation_rank(sv, 0.1, "nuclear")
    # a cut inside a cluster of equal values moves past it: tails^2 of
    # (1, .5, .5, .1) are 1.51, .51, .26, .01; eps^2 1.51 = .3058 puts the cut at 2
    assert o.truncation_rank(np.array([1.0, 0.5, 0.5, 0.1]), 0.45, o.FROBENIUS) == 3
    assert o.truncation_rank(np.array([1.0, 0.5, 0.49, 0.1]), 0.45, o.FROBENIUS) == 2
    assert o.truncation_rank(np.array([1.0, 0.5, 0.5, 0.1]), 0.3, o.SPECTRAL) == 3


def _prolate_column_lists(level):
    """Cells and far-field interactions of the 2 x 2 x 2^level column the
    prolate spheroid of Sec. 5 crosses at levels 2-4 (cube of side 64 around the
    6.4 x 6.4 x 64 box; x and y in the two cells next to the origin)."""
    n = 1 << level
    mid = n // 2
    cells = np.array([(x, y, z) for z in range(n) for y in (mid - 1, mid) for x in (mid - 1, mid)], dtype=np.int32)
    off, src = o.interaction_lists(cells, cells)
    counts = {}
    for i in range(len(cells)):
        for j in src[off[i]:off[i + 1]]:
            t = tuple(int(v) for v in cells[i] - cells[j])
            counts[t] = counts.get(t, 0) + 1
    return len(cells), counts


def test_paper_costs_per_level_prolate_acc9():
    """The paper's printed M2L costs per level (Sec. 5.2, bbFMM, prolate sphere,
    Acc 9: ell = 9, eps = 1e-9, Laplace kernel) from the oracle's lists and
    ranks, under the Frobenius-tail reading of "accuracy eps":

    * SA: one rank r for all C_t (the larger of the ranks of K_row and K_col over
      the level's T); cost = cells (4 l^3 r - l^3) + interactions 2 r^2.  The
      interaction term alone is (cost_3 - 2 cost_2) / 96 = 2 r^2 -> r = 216.
    * SArcmp: cost = cells (4 l^3 r - l^3) + sum over interactions r_t (4 r - 1).
    * IA: cost = sum over interactions r_t (4 l^3 - 1), the ranks from ACA
      stopped at eps_ACA = eps followed by the truncated SVD (Sec. 5: the
      precomputation by ACA).  The plain SVD gives 12 more (0.2 %).

    The spectral reading misses all three (SA r = 189, 9 % fewer IA flops),
    so the pin tells the two readings apart.
    """
    with open(os.path.join(GOLDEN, "paper_costs_prolate_acc9.json")) as f:
        g = json.load(f)
    ell, eps = 9, 1e-9
    n3 = ell ** 3
    lists = {L: _prolate_column_lists(L) for L in g["levels"]}
    # levels 2-4: 16/32/64 cells, 96/288/672 interactions; the IA costs scale 1 : 3 : 7
    assert [lists[L][0] for L in g["levels"]] == [16, 32, 64]
    assert [sum(lists[L][1].values()) for L in g["levels"]] == [96, 288, 672]
    assert [c // g["IA"][0] for c in g["IA"]] == [1, 3, 7] and all(c % g["IA"][0] == 0 for c in g["IA"])
    # the same 36 transfer vectors at every level; ranks are level-independent for 1/r
    T = sorted(lists[2][1])
    assert len(T) == 36 and all(sorted(lists[L][1]) == T for L in g["levels"])
    ops = {o.t_slot(t): o.operator_for_t(ell, o.KIND_INV_R, 0.0, 2, t) for t in T}

    def costs(criterion, aca_ranks):
        sa = o.sa_factors(ops, eps, criterion, ts=T)
        r = sa["r"]
        _, rt = o.sa_recompress(sa["C"], r, eps, criterion, ts=T)
        if aca_ranks:
            ria = {t: o.aca_lowrank(ops[o.t_slot(t)], eps, criterion, eps_factor=1.0)[2] for t in T}
        else:
            ria = {t: o.lowrank(ops[o.t_slot(t)], eps, criterion)[2] for t in T}
        out = {"r": r, "SA": [], "SArcmp": [], "IA": []}
        for L in g["levels"]:
            ncell, cnt = lists[L]
            nint = sum(cnt.values())
            cell_part = ncell * (4 * n3 * r - n3)
            out["SA"].append(cell_part + nint * 2 * r * r)
            out["SArcmp"].append(cell_part + sum(cnt[t] * rt[o.t_slot(t)] * (4 * r - 1) for t in T))
            out["IA"].append(sum(cnt[t] * ria[t] * (4 * n3 - 1) for t in T))
        return out

    fro = costs(o.FROBENIUS, aca_ranks=True)
    assert fro["r"] == 216
    assert fro["SA"] == g["SA"]
    assert fro["SArcmp"] == g["SArcmp"]
    assert fro["IA"] == g["IA"]
    fro_svd = costs(o.FROBENIUS, aca_ranks=False)
    assert fro_svd["SA"] == g["SA"] and fro_svd["SArcmp"] == g["SArcmp"]
    assert all(0 < a / b - 1 < 0.003 for a, b in zip(fro_svd["IA"], g["IA"]))
    spec = costs(o.SPECTRAL, aca_ranks=False)
    assert spec["r"] != 216 and spec["SA"] != g["SA"] and spec["SArcmp"] != g["SArcmp"]
    assert all(a / b < 0.95 for a, b in zip(spec["IA"], g["IA"]))


# ---------------------------------------------------------------- kernels / direct sum
def test_direct_sum_closed_form():
    x = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0]])
    y = np.array([[0.0, 0.0, 0.0], [3.0, 0.0, 4.0]])
    q = np.array([2.0, 5.0])
    d01 = np.sqrt(9 + 16 + 0.0)   # x0 to y1
    d10 = np.sqrt(0 + 16 + 16.0)  # x1 to y1
    d11 = 5.0                     # x1 to y0
    f = o.direct_sum(0, 0.0, x, y, q)
    assert np.allclose(f, [5.0 / d01, 2.0 / d11 + 5.0 / d10], rtol=1e-15)
    f = o.direct_sum(1, 0.0, x, y, q)
    assert np.allclose(f, [5.0 / d01 ** 4, 2.0 / d11 ** 4 + 5.0 / d10 ** 4], rtol=1e-15)
    f = o.direct_sum(2, 0.5, x, y, q)
    # the coincident pair is skipped for every kernel, softened or not
    assert np.allclose(f, [5.0 / np.sqrt(25 + 0.25),
                           2.0 / np.sqrt(25.25) + 5.0 / np.sqrt(32.25)], rtol=1e-15)


# ---------------------------------------------------------------- M2L apply
def test_single_pair_interpolation_converges():
    """P2M -> M2L (oracle K_t) -> L2P between two well-separated cells approaches
    the direct sum (Eq. (5)); a transposed or mis-signed K_t would not."""
    rng = np.random.default_rng(7)
    level = 3
    w = o.cell_width(level)
    X, Y = np.array([3, 3, 3]), np.array([1, 4, 2])
    t = tuple(int(v) for v in X - Y)
    cx, cy = o.cell_center(X, level), o.cell_center(Y, level)
    ys = cy + 0.5 * w * rng.uniform(-1, 1, (40, 3))
    xs = cx + 0.5 * w * rng.uniform(-1, 1, (30, 3))
    q = rng.standard_normal(40)
    exact = o.direct_sum(0, 0.0, xs, ys, q)
    errs = []
    for ell in (2, 3, 4, 5, 6, 7):
        W = o.interp_matrix(ell, ys, cy, w).T @ q
        K = o.operator_for_t(ell, 0, 0.0, level, t)
        F = K @ W
        f = o.l2p(ell, xs, cx, w, F)
        errs.append(o.rel_l2(f, exact))
        Kwrong = o.operator_for_t(ell, 0, 0.0, level, tuple(-v for v in t))
        if ell >= 4:
            assert o.rel_l2(o.l2p(ell, xs, cx, w, Kwrong @ W), exact) > 100 * errs[-1]
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-5


def test_fmm_converges_to_direct_sum():
    """The whole FMM with oracle M2L at levels 2-3 vs the direct N^2 sum:
    the error falls with ell (Sec. 5.1, roughly a decade per order)."""
    rng = np.random.default_rng(2)
    N = 1500
    pts = rng.uniform(-1, 1, (N, 3))
    q = rng.uniform(-1, 1, N)
    samp = np.arange(0, N, 15)
    exact = o.direct_sum(0, 0.0, pts[samp], pts, q)
    errs = []
    for ell in (2, 3, 4, 5):
        up = o.UpwardPass(ell, 3, pts, q)
        loc = o.fmm_oracle_locals(up, 0, 0.0)
        errs.append(o.rel_l2(o.fmm_at_samples(up, 0, 0.0, loc, samp), exact))
    assert all(b < 0.5 * a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-4


def test_adjoint_dot_product_identity():
    rng = np.random.default_rng(4)
    ell = 3
    cells = o.full_grid_cells(3)
    cells = cells[rng.random(len(cells)) < 0.7]
    off, src = o.interaction_lists(cells, cells)
    ops = o.operator_table(ell, 0, 0.0, 3)
    w = rng.standard_normal((len(cells), ell ** 3))
    g = rng.standard_normal((len(cells), ell ** 3))
    Mw = o.m2l_apply(ops, cells, cells, off, src, w)
    Mtg = o.m2l_apply_adjoint(ops, cells, cells, off, src, g, len(cells))
    a, b = float(np.sum(g * Mw)), float(np.sum(Mtg * w))
    assert abs(a - b) <= 1e-13 * (abs(a) + abs(b))


def test_apply_matches_pairwise_assembly_tiny():
    """Brute force on a tiny level: every pair assembled from its own cells' nodes."""
    rng = np.random.default_rng(8)
    ell, level = 2, 2
    cells = o.full_grid_cells(level)
    off, src = o.interaction_lists(cells, cells)
    w = rng.standard_normal((len(cells), ell ** 3))
    ops = o.operator_table(ell, 0, 0.0, level)
    f = o.m2l_apply(ops, cells, cells, off, src, w)
    wd = o.cell_width(level)
    ref = np.zeros_like(f)
    for x in range(len(cells)):
        xn = o.cell_nodes(ell, o.cell_center(cells[x], level), wd)
        for e in range(off[x], off[x + 1]):
            y = src[e]
            yn = o.cell_nodes(ell, o.cell_center(cells[y], level), wd)
            D = np.linalg.norm(xn[:, None, :] - yn[None, :, :], axis=2)
            ref[x] += (1.0 / D) @ w[y]
    assert np.allclose(f, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


def test_apply_rejects_near_field_pair():
    cells = np.array([[0, 0, 0], [1, 0, 0]], dtype=np.int32)
    ops = o.operator_table(2, 0, 0.0, 2)
    with pytest.raises(ValueError):
        o.m2l_apply(ops, cells, cells, np.array([0, 1, 1], np.int32), np.array([1], np.int32),
                    np.zeros((2, 8)))


def test_rel_err_definition():
    assert o.rel_l2([1.0, 2.0], [1.0, 2.0]) == 0.0
    assert abs(o.rel_l2([0.0, 0.0], [3.0, 4.0]) - 1.0) < 1e-15


# ---------------------------------------------------------------------------
# SA / SArcmp (Sec. 4.1)
# ---------------------------------------------------------------------------
def _ops_l4():
    return o.operator_table(4, 0, 0.0, 3)


def test_sa_three_forms_of_c_agree():
    """Eq. (18): C_t = U^* K_t B = Sigma V_t^* B = U^* A_t Gamma (exact even
    after truncation: the residuals are orthogonal to U and to B)."""
    sa = o.sa_factors(_ops_l4(), 1e-6)
    assert 0 < sa["r"] < 64
    for t in o.transfer_vectors()[::7]:
        sl = o.t_slot(t)
        c = sa["C"][sl]
        scale = np.abs(c).max()
        assert np.abs(sa["C_sigma_v"][sl] - c).max() < 1e-12 * scale
        assert np.abs(sa["C_a_gamma"][sl] - c).max() < 1e-12 * scale


def test_sa_error_bound_and_exact_limit():
    """||K_t - U C_t B^*||_2 <= s_{r+1}(K_row) + s_{r+1}(K_col) for every t; with
    eps = 0 the representation is exact."""
    ops = _ops_l4()
    for eps in (1e-3, 1e-6):
        table, sa, _ = o.sa_operator_table(ops, eps)
        r = sa["r"]
        bound = sa["s_row"][r] + sa["s_col"][r] if r < len(sa["s_row"]) else 0.0
        for t in o.transfer_vectors():
            sl = o.t_slot(t)
            err = np.linalg.norm(ops[sl] - table[sl], 2)
            assert err <= bound * (1 + 1e-8) + 1e-13 * np.linalg.norm(ops[sl], 2), (eps, t, err, bound)
    table, sa, _ = o.sa_operator_table(ops, 0.0)
    assert sa["r"] == 64
    for t in o.transfer_vectors()[::11]:
        sl = o.t_slot(t)
        assert np.abs(table[sl] - ops[sl]).max() < 1e-12 * np.abs(ops[sl]).max()


def test_sa_rank_decreases_with_eps():
    ops = _ops_l4()
    ranks = [o.sa_factors(ops, e)["r"] for e in (1e-9, 1e-6, 1e-3, 1e-1)]
    assert all(a >= b for a, b in zip(ranks, ranks[1:])) and ranks[0] > ranks[-1]


@pytest.mark.parametrize("criterion", ["spectral", "frobenius"])
def test_sarcmp_recompression(criterion):
    """Eq. (19): a recompressed C_t has rank r_t < r/2 and differs from C_t by
    its truncated tail (Eckart-Young: the (r_t+1)-th singular value in the
    2-norm, the root sum of squares of the tail in the Frobenius norm), within
    eps of C_t in the criterion's norm; the others are kept whole."""
    ops = _ops_l4()
    eps = 1e-4
    sa = o.sa_factors(ops, eps, criterion)
    C2, ranks = o.sa_recompress(sa["C"], sa["r"], eps, criterion)
    n_re = 0
    for t in o.transfer_vectors():
        sl = o.t_slot(t)
        sv = np.linalg.svd(sa["C"][sl], compute_uv=False)
        if ranks[sl] < sa["r"]:
            n_re += 1
            k = ranks[sl]
            assert 2 * k < sa["r"]
            err = np.linalg.norm(C2[sl] - sa["C"][sl], 2)
            assert abs(err - sv[k]) <= 1e-10 * sv[0]
            errf = np.linalg.norm(C2[sl] - sa["C"][sl], "fro")
            assert abs(errf - np.sqrt(np.sum(sv[k:] ** 2))) <= 1e-10 * sv[0]
            if criterion == "spectral":
                assert sv[k] <= eps * sv[0]
            else:
                assert errf <= eps * np.linalg.norm(sa["C"][sl], "fro") * (1 + 1e-9)
        else:
            assert np.array_equal(C2[sl], sa["C"][sl])
    assert n_re > 0


# ---------------------------------------------------------------- ACA + truncated SVD
def test_aca_recovers_an_exact_low_rank_matrix():
    g = np.random.default_rng(11)
    K = g.standard_normal((60, 7)) @ g.standard_normal((7, 50))
    U, V = o.aca(K, 1e-14)
    assert U.shape[1] <= 8
    assert np.abs(U @ V.T - K).max() < 1e-11 * np.abs(K).max()


def test_aca_interpolates_its_pivot_rows_and_columns():
    """A cross approximation reproduces K exactly on every pivot row and column."""
    K = o.operator_for_t(5, 0, 0.0, 3, (3, 1, 0))
    U, V, piv = o.aca(K, 1e-6, return_pivots=True)
    S = U @ V.T
    scale = np.abs(K).max()
    for i, j in piv:
        assert np.abs(S[i, :] - K[i, :]).max() < 1e-12 * scale
        assert np.abs(S[:, j] - K[:, j]).max() < 1e-12 * scale


@pytest.mark.parametrize("criterion", ["spectral", "frobenius"])
@pytest.mark.parametrize("ell,kind,eps", [(5, 0, 1e-5), (7, 1, 1e-7), (6, 2, 1e-6), (3, 0, 1e-3)])
def test_aca_then_svd_gives_the_svd_ranks(ell, kind, eps, criterion):
    """Sec. 5: ACA followed by a truncated SVD ends with the same ranks as the SVD
    (where the SVD's cut moved past a cluster of equal singular values, which
    the ACA approximant no longer holds equal, by that cluster at most);
    the error stays within the truncation bound of the ACA approximant S plus
    the ACA residual, |K - U V^T| <= |K - S| + eps |S| (triangle inequality; the
    2-norm for the spectral reading, the Frobenius norm for the Frobenius one),
    and the ACA residual stays below the target accuracy eps |K| (its stop
    test bounds a term, not the residual: at ell 7, t = (2, 0, 0) it ends at
    0.56 eps |K|_F)."""
    c = 0.01 if kind == 2 else 0.0
    nrm = 2 if criterion == "spectral" else "fro"
    for t in o.t_sym_list():
        K = o.operator_for_t(ell, kind, c, 3, t)
        _, _, r = o.lowrank(K, eps, criterion)
        U, V, ra, k = o.aca_lowrank(K, eps, criterion)
        sk = np.linalg.svd(K, compute_uv=False)
        assert ra == r or (ra < r and sk[ra - 1] - sk[r - 1] <= o.CLUSTER_GAP * sk[0]), (t, r, ra)
        Ua, Va = o.aca(K, o.ACA_EPS_FACTOR * eps)
        S = Ua @ Va.T
        res = np.linalg.norm(K - S, nrm)
        assert np.linalg.norm(K - U @ V.T, nrm) <= (res + eps * np.linalg.norm(S, nrm)) * (1 + 1e-9)
        assert res <= eps * np.linalg.norm(K, nrm)
        assert k < K.shape[0]
