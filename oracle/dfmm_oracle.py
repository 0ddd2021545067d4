"""FP64 CPU oracle of the directional FMM (dFMM) M2L for the Helmholtz kernel.

TEST INFRASTRUCTURE ONLY.  Imported by ``tests/`` and by the CPU legs of
``bench.py``; never by the library or its binding, with which it shares no
code.  Everything is recomputed from the definitions of Sec. 2.1.2 (dFMM),
Sec. 3 (near and far field, Alg. 1) and Sec. 4.2 (symmetries) of Messner,
Bramas, Coulaud, Darve, "Optimized M2L kernels for the Chebyshev
interpolation based fast multipole method".

What it computes:

* the Helmholtz kernel K(x, y) = exp(i k |x - y|) / |x - y| (Eq. (33), the
  4 pi dropped like the other kernels) and its directional form
  K^u(x, y) = K(x, y) exp(-i k u.(x - y)) (Eq. (9));
* the low/high-frequency regime of a level, the two admissibility criteria,
  the cones of directions and the per-cone (directional) far-field lists
  that Alg. 1 produces on a uniform-depth octree;
* directional P2M and L2P (Eqs. (12) and (14)) for one cell;
* the dFMM M2L (Eq. (13)): F^u_X += K_t W^u_Y for every pair of a
  directional list, cell by cell, with K_t assembled from kernel values at
  the interpolation points (no symmetry, no blocking).

Readings, where the paper defers to its reference on the directional FMM:

* D1 regime: a level of cell width w is high-frequency when k w >= 1 (the
  paper's table of list sizes has k w = 1 in hf and k w = 1/2 in lf).
* D2 admissibility: at an lf level, |t|_inf >= 2 (the bbFMM rule); at an hf
  level, additionally |c_X - c_Y| > max(k w^2, 2 w) (the O(k w^2) separation,
  strict, never below two cell widths), evaluated as
  (t.t) w w > (k w w)(k w w) and t.t > 4 in FP64.  With it the paper's table
  of list sizes is reproduced exactly, for all three geometries and every
  printed level.
* D3 cones: the unit sphere is split through the faces of the cube [-1, 1]^3,
  each face into m x m squares, m the smallest power of two >= k w (cone
  aperture O(1/(k w)), halved from one level to the next coarser one:
  nested).  The cone of a pair is the square hit by the ray along
  c_X - c_Y, from source to target: that orientation makes
  |x - y| - u.(x - y) small and K^u smooth over the pair.  Computed in
  integers from t: face axis f = the first axis with the largest |t_i|,
  side s = (t_f < 0), on the other two axes a < b the squares
  floor((t_a + |t_f|) m / (2 |t_f|)) clamped to m - 1; cone index
  (2 f + s) m^2 + i_b m + i_a.
* D4 one expansion per (cell, cone) of the level, stored densely as
  [ncells][n_cones][ell^3]; an lf level has a single cone.
"""
from __future__ import annotations

import numpy as np

from .m2l_oracle import cell_center, cell_nodes, interp_matrix


# --------------------------------------------------------------------------
# kernels (Eq. (33), Eq. (9))
# --------------------------------------------------------------------------
def helmholtz(k: float, r):
    """exp(i k r) / r."""
    r = np.asarray(r, dtype=np.float64)
    return np.exp(1j * k * r) / r


def helmholtz_directional(k: float, u, x, y):
    """K^u(x, y) = exp(i k (|x - y| - u.(x - y))) / |x - y| (Eq. (9)); x, y [..., 3]."""
    d = np.asarray(x, dtype=np.float64) - np.asarray(y, dtype=np.float64)
    r = np.linalg.norm(d, axis=-1)
    return np.exp(1j * k * (r - d @ np.asarray(u, dtype=np.float64))) / r


# --------------------------------------------------------------------------
# regimes, admissibility, cones (Sec. 2.1.2, Sec. 3.2; readings D1-D3)
# --------------------------------------------------------------------------
def is_high_frequency(k: float, w: float) -> bool:
    """D1: the level of width w is in the high-frequency regime."""
    return k * w >= 1.0


def admissible(k: float, w: float, t) -> bool:
    """D2: cells of width w with transfer vector t are separated (far field)."""
    tinf = max(abs(int(v)) for v in t)
    if tinf < 2:
        return False
    if not is_high_frequency(k, w):
        return True
    tt = float(sum(int(v) * int(v) for v in t))
    return tt * w * w > (k * w * w) * (k * w * w) and tt > 4.0


def cone_m(k: float, w: float) -> int:
    """D3: squares per cube-face edge at an hf level (0 at an lf level)."""
    if not is_high_frequency(k, w):
        return 0
    m = 1
    while m < k * w:
        m *= 2
    return m


def n_cones(k: float, w: float) -> int:
    m = cone_m(k, w)
    return 6 * m * m if m else 1


def cone_index(m: int, t) -> int:
    """D3: the cone of the direction c_X - c_Y = w t, in integer arithmetic."""
    if m == 0:
        return 0
    t = [int(v) for v in t]
    at = [abs(v) for v in t]
    f = at.index(max(at))
    s = 1 if t[f] < 0 else 0
    a, b = [i for i in range(3) if i != f]
    T = at[f]
    ia = min((t[a] + T) * m // (2 * T), m - 1)
    ib = min((t[b] + T) * m // (2 * T), m - 1)
    return (2 * f + s) * m * m + ib * m + ia


def cone_direction(m: int, c: int) -> np.ndarray:
    """Unit direction u_c through the centre of cone c's face square (D3)."""
    face, rem = divmod(c, m * m)
    f, s = divmod(face, 2)
    ib, ia = divmod(rem, m)
    a, b = [i for i in range(3) if i != f]
    v = np.zeros(3)
    v[f] = -1.0 if s else 1.0
    v[a] = -1.0 + (2 * ia + 1) / m
    v[b] = -1.0 + (2 * ib + 1) / m
    return v / np.linalg.norm(v)


# --------------------------------------------------------------------------
# interaction lists (Alg. 1 on a uniform-depth octree)
# --------------------------------------------------------------------------
def level_width(level: int, domain_width: float) -> float:
    return domain_width / (1 << level)


def separate_recursive(cells_by_level: dict, leaf_level: int, k: float, domain_width: float):
    """Alg. 1 run literally from the pair of roots: a pair is put in the
    directional far field (hf, by cone), in the far field (lf) or, at the
    leaves, in the near field; otherwise every pair of non-empty children is
    tested.  Small trees only (pure Python recursion).

    Returns (far, near): far[level][(x, c)] -> sorted source indices,
    near[x] -> sorted leaf indices; x, y index cells_by_level[level].
    """
    index = {L: {tuple(int(v) for v in c): i for i, c in enumerate(cells_by_level[L])}
             for L in cells_by_level}
    children = {}
    for L in range(leaf_level):
        ch = {}
        for c, i in index[L + 1].items():
            ch.setdefault(tuple(v >> 1 for v in c), []).append(c)
        children[L] = ch
    far = {L: {} for L in range(leaf_level + 1)}
    near = {}

    def visit(L, X, Y):
        w = level_width(L, domain_width)
        t = tuple(a - b for a, b in zip(X, Y))
        if admissible(k, w, t):
            c = cone_index(cone_m(k, w), t)
            far[L].setdefault((index[L][X], c), []).append(index[L][Y])
            return
        if L == leaf_level:
            near.setdefault(index[L][X], []).append(index[L][Y])
            return
        for Xc in children[L].get(X, []):
            for Yc in children[L].get(Y, []):
                visit(L + 1, Xc, Yc)

    root = tuple(int(v) for v in cells_by_level[0][0])
    visit(0, root, root)
    for L in far:
        for key in far[L]:
            far[L][key].sort()
    for key in near:
        near[key].sort()
    return far, near


def admissible_many(k: float, w: float, t: np.ndarray) -> np.ndarray:
    """admissible() for an integer array t [..., 3] (same FP64 expression)."""
    t = np.asarray(t, dtype=np.int64)
    ok = np.abs(t).max(axis=-1) >= 2
    if not is_high_frequency(k, w):
        return ok
    tt = (t * t).sum(axis=-1).astype(np.float64)
    return ok & (tt * w * w > (k * w * w) * (k * w * w)) & (tt > 4.0)


def directional_lists(cells: np.ndarray, level: int, k: float, domain_width: float):
    """The lists of one level as Alg. 1 leaves them, written per level: Y is in
    the (directional) far field of X at `level` when the pair is admissible
    there and no pair of their ancestors (levels 0 .. level - 1) is.

    Returns (n_cones, offsets int32 [ncells * n_cones + 1] over target
    expansions e = x * n_cones + c, sources int32 [nnz] ascending within each
    expansion).
    """
    w = level_width(level, domain_width)
    C = n_cones(k, w)
    m = cone_m(k, w)
    cells = np.asarray(cells, dtype=np.int64)
    side = 1 << level
    lookup = np.full(side ** 3, -1, dtype=np.int64)
    lookup[cells[:, 0] + side * cells[:, 1] + side * side * cells[:, 2]] = np.arange(len(cells))
    # reach: the parents are not admissible, so |t_p|_inf < max(2, 2 k w) and
    # |t|_inf <= 2 |t_p|_inf + 1
    R = 2 * int(np.ceil(max(2.0, 2.0 * k * w))) + 1
    r = np.arange(-R, R + 1)
    dz, dy, dx = np.meshgrid(r, r, r, indexing="ij")
    T = np.stack([dx.ravel(), dy.ravel(), dz.ravel()], axis=1)
    T = T[admissible_many(k, w, T)]
    cone_of = np.array([cone_index(m, t) for t in T], dtype=np.int64)
    rows = [[] for _ in range(len(cells) * C)]
    for x, X in enumerate(cells):
        Y = X[None, :] - T
        inside = np.all((Y >= 0) & (Y < side), axis=1)
        Yi, Ti, ci = Y[inside], T[inside], cone_of[inside]
        y = lookup[Yi[:, 0] + side * Yi[:, 1] + side * side * Yi[:, 2]]
        keep = y >= 0
        for l in range(level):
            sh = level - l
            tp = (X[None, :] >> sh) - (Yi >> sh)
            keep &= ~admissible_many(k, level_width(l, domain_width), tp)
        for yy, cc in zip(y[keep], ci[keep]):
            rows[x * C + int(cc)].append(int(yy))
    offsets = np.zeros(len(rows) + 1, dtype=np.int32)
    srcs = []
    for e, rr in enumerate(rows):
        rr.sort()
        srcs.extend(rr)
        offsets[e + 1] = offsets[e] + len(rr)
    return C, offsets, np.asarray(srcs, dtype=np.int32)


# --------------------------------------------------------------------------
# operators and the M2L (Eq. (13), Eq. (15))
# --------------------------------------------------------------------------
def dfmm_operator(ell: int, k: float, x_center, y_center, w: float) -> np.ndarray:
    """(K)_{m(alpha) n(beta)} = K(xbar_alpha, ybar_beta), complex [ell^3, ell^3],
    from the absolute interpolation points of two cells of width w."""
    xn = cell_nodes(ell, x_center, w)
    yn = cell_nodes(ell, y_center, w)
    r = np.linalg.norm(xn[:, None, :] - yn[None, :, :], axis=-1)
    return helmholtz(k, r)


def dfmm_operator_for_t(ell: int, k: float, level: int, t, lo: float = -1.0, domain_width: float = 2.0):
    """K_t of a level: the operator of the pair X = (R, R, R) + t, Y = (R, R, R)
    (translation invariance, Sec. 3.2)."""
    R = 64
    X = np.asarray(t, dtype=np.int64) + R
    Y = np.full(3, R, dtype=np.int64)
    w = level_width(level, domain_width)
    return dfmm_operator(ell, k, cell_center(X, level, lo, domain_width), cell_center(Y, level, lo, domain_width), w)


def dfmm_m2l_apply(ell: int, k: float, level: int, tgt_ijk, src_ijk, cones: int, offsets, sources, W,
                   locals_in=None, lo: float = -1.0, domain_width: float = 2.0) -> np.ndarray:
    """F[x * C + c] += K_{t(X, Y)} W[y * C + c] over the directional lists (Eq. (13)).

    W: complex [nsrc * C, ell^3]; returns complex [ntgt * C, ell^3].  The
    operator of each transfer vector is assembled once and reused for every
    pair that has it.
    """
    n3 = ell ** 3
    tgt = np.asarray(tgt_ijk, dtype=np.int64)
    src = np.asarray(src_ijk, dtype=np.int64)
    F = np.zeros((len(tgt) * cones, n3), dtype=np.complex128) if locals_in is None \
        else np.array(locals_in, dtype=np.complex128)
    W = np.asarray(W, dtype=np.complex128)
    cache = {}
    for e in range(len(tgt) * cones):
        x, c = divmod(e, cones)
        for j in range(int(offsets[e]), int(offsets[e + 1])):
            y = int(sources[j])
            t = tuple(int(v) for v in tgt[x] - src[y])
            if t not in cache:
                cache[t] = dfmm_operator_for_t(ell, k, level, t, lo, domain_width)
            F[e] += cache[t] @ W[y * cones + c]
    return F


def canonical_t(t) -> tuple:
    """p(t): |t| sorted descending (the reference cone of Sec. 4.2.1), any size."""
    return tuple(sorted((abs(int(v)) for v in t), reverse=True))


def t_sym_of_lists(tgt_ijk, src_ijk, offsets, sources, cones: int) -> list:
    """T_sym of a level's lists: the distinct p(t) over all entries, ascending."""
    tgt = np.asarray(tgt_ijk, dtype=np.int64)
    src = np.asarray(src_ijk, dtype=np.int64)
    out = set()
    for e in range(len(offsets) - 1):
        x = e // cones
        for j in range(int(offsets[e]), int(offsets[e + 1])):
            out.add(canonical_t(tgt[x] - src[int(sources[j])]))
    return sorted(out)


# --------------------------------------------------------------------------
# directional P2M / L2P for one cell (Eqs. (12), (14))
# --------------------------------------------------------------------------
def dfmm_p2m(ell: int, k: float, u, pts, q, center, w: float) -> np.ndarray:
    """W^u_beta = exp(i k u.ybar_beta) sum_j S(y_j, ybar_beta) exp(-i k u.y_j) q_j."""
    u = np.asarray(u, dtype=np.float64)
    S = interp_matrix(ell, np.asarray(pts), center, w)           # [n, ell^3]
    nodes = cell_nodes(ell, center, w)
    return np.exp(1j * k * (nodes @ u)) * (S.T @ (np.exp(-1j * k * (np.asarray(pts) @ u)) * q))


def dfmm_l2p(ell: int, k: float, u, pts, center, w: float, F) -> np.ndarray:
    """f_i = exp(i k u.x_i) sum_alpha S(x_i, xbar_alpha) exp(-i k u.xbar_alpha) F^u_alpha."""
    u = np.asarray(u, dtype=np.float64)
    S = interp_matrix(ell, np.asarray(pts), center, w)
    nodes = cell_nodes(ell, center, w)
    return np.exp(1j * k * (np.asarray(pts) @ u)) * (S @ (np.exp(-1j * k * (nodes @ u)) * F))


def helmholtz_direct(k: float, targets, sources, q) -> np.ndarray:
    """sum_j K(x_i, y_j) q_j (Eq. (1)), all pairs (the sets must not overlap)."""
    d = np.asarray(targets)[:, None, :] - np.asarray(sources)[None, :, :]
    return helmholtz(k, np.linalg.norm(d, axis=-1)) @ np.asarray(q)


def interpolation_error(ell: int, k: float, u, x_center, y_center, w: float, npts: int = 60, seed: int = 0):
    """max |K^u(x, y) - sum S(x, xbar) K^u(xbar, ybar) S(y, ybar)| / max |K^u| over
    random x in X and y in Y (Eq. (10))."""
    g = np.random.default_rng(seed)
    xs = np.asarray(x_center) + w * (g.random((npts, 3)) - 0.5)
    ys = np.asarray(y_center) + w * (g.random((npts, 3)) - 0.5)
    xn = cell_nodes(ell, x_center, w)
    yn = cell_nodes(ell, y_center, w)
    Kn = helmholtz_directional(k, u, xn[:, None, :], yn[None, :, :])
    approx = interp_matrix(ell, xs, x_center, w) @ Kn @ interp_matrix(ell, ys, y_center, w).T
    exact = helmholtz_directional(k, u, xs[:, None, :], ys[None, :, :])
    return float(np.abs(approx - exact).max() / np.abs(exact).max())

