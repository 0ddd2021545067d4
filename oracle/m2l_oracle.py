"""FP64 CPU oracle of the black-box Chebyshev FMM M2L translation.

TEST INFRASTRUCTURE ONLY.  This module exists to check the CUDA path; it is
imported by ``tests/``, by ``__graft_entry__.smoke()`` and by the CPU-baseline
leg of ``bench.py``, and by nothing else.  It shares no code, table or helper
with the CUDA library: every quantity here is recomputed from the paper's
definitions (Messner, Bramas, Coulaud, Darve, "Optimized M2L kernels for the
Chebyshev interpolation based fast multipole method").

What it computes, each function citing its source:

* Chebyshev roots and tensor nodes (Sec. 2.1, Eqs. (2)-(3)), the index map
  m(alpha) (Eq. (16)).
* Kernel functions (Sec. 1, Eq. (33)); the configs use 1/r, 1/r^4 and
  1/sqrt(r^2+c^2), all without the 4*pi factor.
* Transfer vectors and interaction lists (Sec. 3.1-3.2, Table 1): Y is in the
  far field of X when the parents are neighbours and |X - Y|_inf >= 2.
* M2L operators K_t assembled directly from kernel evaluations at absolute node
  coordinates (Eq. (15)), 316 per level, no symmetry, no homogeneity scaling.
* The symmetry maps of Sec. 4.2.1: axial and diagonal multi-index
  permutations (Eqs. (26)-(27)), T_sym (Eqs. (23)-(24)) and p(t).
* Cell-by-cell M2L f_X += K_t w_Y (Eq. (7)) and its adjoint, in plain C loops.
* Truncated SVD per operator (Eq. (20)); the single low-rank approximation
  SA of all operators and its recompression SArcmp (Sec. 4.1).
* P2M/M2M (Eq. (6)), L2L/L2P (Eq. (8)), P2P and the direct sum (Eq. (1)).

Readings of the paper taken where it is silent or garbled (each stated where
it is used): roots in ascending order; P_t oriented so that
K_t[a, b] = K_{p(t)}[sigma_t(a), sigma_t(b)]; ties of |t_i| broken by a stable
sort (lower axis first); SVD truncated at the smallest r whose Frobenius
tail is within eps of the Frobenius norm, sum_{i>r} s_i^2 <= eps^2 sum s_i^2
(the spectral reading s_{r+1} <= eps s_1 is an option).
"""
from __future__ import annotations

import ctypes
import itertools
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "m2l_oracle.c")
_SO = os.path.join(_HERE, "libm2l_oracle.so")

KIND_INV_R, KIND_INV_R4, KIND_INV_SQRT_R2C2 = 0, 1, 2


# --------------------------------------------------------------------------
# the C loops
# --------------------------------------------------------------------------
def build_c(force: bool = False) -> str:
    """Compile the plain C loops of the oracle (no fused multiply-add)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=c99", "-shared", "-fPIC",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


_lib_handle = None


def _lib():
    global _lib_handle
    if _lib_handle is None:
        lib = ctypes.CDLL(build_c())
        P = ctypes.c_void_p
        lib.oracle_assemble_pair.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, P, P, P]
        lib.oracle_assemble_pair.restype = None
        for fn in (lib.oracle_m2l_apply, lib.oracle_m2l_apply_adjoint):
            fn.argtypes = [ctypes.c_int, P, ctypes.c_int, P, P, P, P, P, P]
            fn.restype = ctypes.c_long
        lib.oracle_direct_sum.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_long, P,
                                          ctypes.c_long, P, P, P]
        lib.oracle_direct_sum.restype = None
        _lib_handle = lib
    return _lib_handle


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


# --------------------------------------------------------------------------
# Chebyshev nodes and index maps (Sec. 2.1, Sec. 3.1)
# --------------------------------------------------------------------------
def cheb_roots(ell: int) -> np.ndarray:
    """The ell roots of T_ell(x) = cos(ell * arccos x) on [-1, 1], ascending.

    Sec. 2.1 prints T_ell(x) = cos(arccos x); the ell in front of arccos is read
    back in.  The roots are cos((2k-1) pi / (2 ell)), k = 1..ell; they are
    returned in ascending order, the order in which the multi-index grows
    along +e_i in Fig. 1.
    """
    k = np.arange(1, ell + 1, dtype=np.float64)
    return np.sort(np.cos((2.0 * k - 1.0) * np.pi / (2.0 * ell)))


def multi_indices(ell: int) -> np.ndarray:
    """[ell^3, 3] zero-based multi-indices alpha, row j holding m^{-1}(j).

    Eq. (16) with m(alpha) = (alpha_1 - 1) + (alpha_2 - 1) ell + (alpha_3 - 1) ell^2 + 1,
    written zero-based: row m holds (alpha_1, alpha_2, alpha_3) - 1.
    """
    out = np.empty((ell ** 3, 3), dtype=np.int64)
    for a3 in range(ell):
        for a2 in range(ell):
            for a1 in range(ell):
                out[a1 + a2 * ell + a3 * ell * ell] = (a1, a2, a3)
    return out


def m_of(alpha, ell: int) -> int:
    """Zero-based m(alpha) of Eq. (16) for a zero-based multi-index."""
    return int(alpha[0]) + int(alpha[1]) * ell + int(alpha[2]) * ell * ell


def cell_width(level: int, domain_width: float = 2.0) -> float:
    """Width of a cell at `level` of a uniform octree over a cube of side domain_width."""
    return domain_width / (1 << level)


def cell_center(ijk, level: int, lo: float = -1.0, domain_width: float = 2.0) -> np.ndarray:
    """Centre of the cell with integer coordinates ijk at `level`: lo + w (ijk + 1/2)."""
    w = cell_width(level, domain_width)
    return lo + w * (np.asarray(ijk, dtype=np.float64) + 0.5)


def cell_nodes(ell: int, center, width: float) -> np.ndarray:
    """[ell^3, 3] absolute interpolation points xbar_alpha of a cell, in m() order.

    Tensor product of the roots (Eq. (3)) mapped affinely onto the cell
    (the map Phi of Sec. 2.1): xbar = center + (width / 2) xi.
    """
    xi = cheb_roots(ell)
    mi = multi_indices(ell)
    ref = xi[mi]  # [ell^3, 3]
    return np.asarray(center, dtype=np.float64)[None, :] + 0.5 * width * ref


# --------------------------------------------------------------------------
# kernels (Sec. 1, Eq. (33))
# --------------------------------------------------------------------------
def kernel_r(kind: int, c: float, r):
    r = np.asarray(r, dtype=np.float64)
    if kind == KIND_INV_R:
        return 1.0 / r
    if kind == KIND_INV_R4:
        r2 = r * r
        return 1.0 / (r2 * r2)
    if kind == KIND_INV_SQRT_R2C2:
        return 1.0 / np.sqrt(r * r + c * c)
    raise ValueError("unknown kernel kind %r" % kind)


def homogeneity_degree(kind: int):
    """Degree n of K(alpha r) = alpha^n K(r) (Sec. 3.2), or None if not homogeneous."""
    return {KIND_INV_R: -1, KIND_INV_R4: -4}.get(kind)


# --------------------------------------------------------------------------
# transfer vectors and the symmetry maps (Sec. 3.1, 3.2, 4.2.1)
# --------------------------------------------------------------------------
def transfer_vectors() -> list:
    """T: every t in [-3,3]^3 with |t|_inf >= 2, i.e. |t| > sqrt(3) (Sec. 3.2).

    These are the far-field transfer vectors of the union of the eight
    children's interaction lists, 7^3 - 3^3 of them.
    """
    return [t for t in itertools.product(range(-3, 4), repeat=3) if max(map(abs, t)) >= 2]


def in_z_sym(t) -> bool:
    """Membership in the reference cone Z^3_sym: t1 >= t2 >= t3 >= 0 (Eq. (23))."""
    return t[0] >= t[1] >= t[2] >= 0


def t_sym_list() -> list:
    """T_sym = T intersected with Z^3_sym (Eq. (24)), sorted lexicographically ascending.

    The ascending lexicographic order fixes the operator index p used by the
    tables of the library interface.
    """
    return sorted(t for t in transfer_vectors() if in_z_sym(t))


def axial_permutation(t, alpha, ell: int):
    """pi^A_t of Eq. (26): flip component i (alpha_i -> ell - (alpha_i - 1)) when t_i < 0.

    alpha is zero-based here, so the flip reads alpha_i -> ell - 1 - alpha_i.
    t_i = 0 falls in the t_i >= 0 branch (no flip).
    """
    return tuple((ell - 1 - alpha[i]) if t[i] < 0 else alpha[i] for i in range(3))


def diagonal_order(t) -> tuple:
    """Axis order (i, j, k) with |t_i| >= |t_j| >= |t_k| (Eq. (27)).

    Ties |t_i| = |t_j| are broken by a stable sort: the lower axis comes first.
    """
    return tuple(sorted(range(3), key=lambda i: -abs(t[i])))


def diagonal_permutation(t, alpha):
    """pi^D_t of Eq. (27): (alpha_1, alpha_2, alpha_3) -> (alpha_i, alpha_j, alpha_k)."""
    i, j, k = diagonal_order(t)
    return (alpha[i], alpha[j], alpha[k])


def p_vector(t) -> tuple:
    """p(t) in T_sym: the reflection of t into the reference cone.

    Applying the axial reflections (absolute values) and then the diagonal
    ones (components sorted by modulus, descending) maps t onto the cone
    t1 >= t2 >= t3 >= 0 (Sec. 4.2.1, Fig. 5).
    """
    i, j, k = diagonal_order(t)
    a = [abs(x) for x in t]
    return (a[i], a[j], a[k])


def sigma_of_t(t, ell: int) -> np.ndarray:
    """sigma_t(j) = m(pi_t(m^{-1}(j))) with pi_t = pi^D_t o pi^A_t (Eqs. (28)-(29)).

    Reading of the orientation: with this sigma,
    K_t[a, b] = K_{p(t)}[sigma_t(a), sigma_t(b)], i.e. the reflected point of
    node a of the cell pair t is node sigma_t(a) of the pair p(t).
    """
    mi = multi_indices(ell)
    out = np.empty(ell ** 3, dtype=np.int64)
    for j in range(ell ** 3):
        alpha = tuple(int(v) for v in mi[j])
        out[j] = m_of(diagonal_permutation(t, axial_permutation(t, alpha, ell)), ell)
    return out


def g_index(t) -> int:
    """Index of the signed axis permutation of t: 8 * perm_id + flip_mask.

    flip_mask has bit i set when t_i < 0 (the octant of Eq. (26)); perm_id is
    the position of the axis order of Eq. (27) among the six permutations of
    (0, 1, 2) in lexicographic order.  sigma_t depends on t only through this
    index, so 48 tables cover all of T.
    """
    perms = list(itertools.permutations(range(3)))
    flip = sum(1 << i for i in range(3) if t[i] < 0)
    return 8 * perms.index(diagonal_order(t)) + flip


def sigma_of_g(g: int, ell: int) -> np.ndarray:
    """The sigma table of signed permutation g (flip mask g % 8, axis order g // 8)."""
    perms = list(itertools.permutations(range(3)))
    order = perms[g // 8]
    flip = g % 8
    mi = multi_indices(ell)
    out = np.empty(ell ** 3, dtype=np.int64)
    for j in range(ell ** 3):
        a = [int(v) for v in mi[j]]
        a = [(ell - 1 - a[i]) if (flip >> i) & 1 else a[i] for i in range(3)]
        out[j] = m_of((a[order[0]], a[order[1]], a[order[2]]), ell)
    return out


def sigma_tables(ell: int) -> np.ndarray:
    """[48, ell^3] sigma tables indexed by g."""
    return np.stack([sigma_of_g(g, ell) for g in range(48)])


def lut343() -> np.ndarray:
    """uint16 table over t in [-3,3]^3 at slot (t1+3) + 7 (t2+3) + 49 (t3+3).

    Entry p | (g << 8) for far-field t, 0xFFFF for |t|_inf <= 1.
    """
    tsym = t_sym_list()
    out = np.full(343, 0xFFFF, dtype=np.uint16)
    for t in transfer_vectors():
        out[t_slot(t)] = tsym.index(p_vector(t)) | (g_index(t) << 8)
    return out


def t_slot(t) -> int:
    return (t[0] + 3) + 7 * (t[1] + 3) + 49 * (t[2] + 3)


# --------------------------------------------------------------------------
# M2L operators (Eq. (15)), assembled directly
# --------------------------------------------------------------------------
def assemble_pair(ell: int, kind: int, c: float, xnodes: np.ndarray, ynodes: np.ndarray) -> np.ndarray:
    """(K)_{m(alpha) n(beta)} = K(xbar_alpha, ybar_beta) for two node sets (Eq. (15))."""
    n3 = ell ** 3
    x = np.ascontiguousarray(xnodes, dtype=np.float64)
    y = np.ascontiguousarray(ynodes, dtype=np.float64)
    out = np.empty((n3, n3), dtype=np.float64)
    _lib().oracle_assemble_pair(kind, float(c), n3, _ptr(x), _ptr(y), _ptr(out))
    return out


def operator_for_t(ell: int, kind: int, c: float, level: int, t, lo: float = -1.0,
                   domain_width: float = 2.0, x_cell=(3, 3, 3)) -> np.ndarray:
    """K_t at `level`, assembled from the absolute nodes of the pair X, Y = X - t.

    X defaults to the cell (3, 3, 3), so that X - t has non-negative integer
    coordinates for every t in [-3, 3]^3.  By translation invariance of the
    kernel (Sec. 3.2) this is the operator of every cell pair with transfer
    vector t at this level.
    """
    w = cell_width(level, domain_width)
    x_cell = np.asarray(x_cell, dtype=np.int64)
    y_cell = x_cell - np.asarray(t, dtype=np.int64)
    xn = cell_nodes(ell, cell_center(x_cell, level, lo, domain_width), w)
    yn = cell_nodes(ell, cell_center(y_cell, level, lo, domain_width), w)
    return assemble_pair(ell, kind, c, xn, yn)


def operator_table(ell: int, kind: int, c: float, level: int, lo: float = -1.0,
                   domain_width: float = 2.0) -> np.ndarray:
    """[343, ell^3, ell^3]: the 316 operators of T at their t-slots, zeros elsewhere."""
    n3 = ell ** 3
    ops = np.zeros((343, n3, n3), dtype=np.float64)
    for t in transfer_vectors():
        ops[t_slot(t)] = operator_for_t(ell, kind, c, level, t, lo, domain_width)
    return ops


FROBENIUS, SPECTRAL = "frobenius", "spectral"
CLUSTER_GAP = 1e-12   # singular values closer than this (relative to s_1) are one cluster


def truncation_rank(s: np.ndarray, eps: float, criterion: str = FROBENIUS) -> int:
    """Truncation rank at "accuracy eps" (Eq. (20) and Sec. 4.1), s descending.

    frobenius: the smallest r with sum_{i>r} s_i^2 <= eps^2 sum_i s_i^2, i.e.
      |K - K_r|_F <= eps |K|_F.  With it the paper's printed per-level costs of
      SA and SArcmp (Sec. 5.2, bbFMM, prolate sphere, Acc 9) come out exactly.
    spectral: the smallest r with s_{r+1} <= eps s_1, i.e. |K - K_r|_2 <= eps |K|_2.

    The truncated SVD is unique only when s_r > s_{r+1}.  A cut that would
    split a cluster of equal singular values (operators with a symmetry have
    such pairs) moves past the cluster: r grows while s_r - s_{r+1} <=
    CLUSTER_GAP s_1, a gap no SVD in double precision resolves.
    """
    s = np.asarray(s, dtype=np.float64)
    n = len(s)
    if eps <= 0.0:
        return n
    if criterion == SPECTRAL:
        r = int(np.count_nonzero(s > eps * s[0]))
    elif criterion == FROBENIUS:
        # tail[r] = sum_{i >= r} s_i^2 (0-based), summed from the smallest value up
        tail = np.zeros(n + 1)
        for i in range(n - 1, -1, -1):
            tail[i] = tail[i + 1] + s[i] * s[i]
        r = n
        for k in range(n + 1):
            if tail[k] <= eps * eps * tail[0]:
                r = k
                break
    else:
        raise ValueError("unknown truncation criterion %r" % (criterion,))
    while 0 < r < n and s[r - 1] - s[r] <= CLUSTER_GAP * s[0]:
        r += 1
    return r


def lowrank(K: np.ndarray, eps: float, criterion: str = FROBENIUS):
    """Truncated SVD K ~ U_t V_t^T of Eq. (20), U_t = U_r Sigma_r, V_t = V_r.

    Returns (U_t, V_t, rank).
    """
    U, s, Vt = np.linalg.svd(K)
    r = truncation_rank(s, eps, criterion)
    return U[:, :r] * s[None, :r], Vt[:r, :].T.copy(), r


def lowrank_operator_table(ops: np.ndarray, eps: float, criterion: str = FROBENIUS):
    """Replace every stored operator by its rank-r_t truncation U_t V_t^T.

    Returns (table, ranks) where ranks[slot] is r_t (0 for unused slots).
    """
    out = np.zeros_like(ops)
    ranks = np.zeros(343, dtype=np.int64)
    for t in transfer_vectors():
        s = t_slot(t)
        U, V, r = lowrank(ops[s], eps, criterion)
        out[s] = U @ V.T
        ranks[s] = r
    return out, ranks


# --------------------------------------------------------------------------
# ACA followed by a truncated SVD (Sec. 4.1 and Sec. 5: the cheaper route to
# the factors of Eq. (20); the algorithm is Bebendorf's partially pivoted ACA)
# --------------------------------------------------------------------------
ACA_EPS_FACTOR = 0.01   # reading: ACA stops at eps_ACA = 0.01 eps before the truncated SVD


def aca(K: np.ndarray, eps_aca: float, kmax: int = None, return_pivots: bool = False):
    """Adaptive cross approximation with partial pivoting, K ~ sum_k u_k v_k^T.

    Steps, in order: take pivot row i (row 0 first), form its residual row
    r = K[i, :] - sum_l u_l[i] v_l; take the column j of largest |r_j| (the
    first on ties); if r_j = 0 the row is exhausted: move to the first unused
    row without adding a term; else v_k = r / r_j and u_k = the residual of
    column j.  The Frobenius norm of the approximant S_k is updated
    incrementally; stop when |u_k| |v_k| <= eps_aca |S_k|_F.  The next pivot
    row is the unused row of largest |u_k[i]| (the first on ties).

    Returns (U [m, k], V [n, k]) and, with return_pivots, the pivot rows and
    columns of the k terms.
    """
    K = np.asarray(K, dtype=np.float64)
    m, n = K.shape
    kmax = min(m, n) if kmax is None else kmax
    us, vs, piv = [], [], []
    used = np.zeros(m, dtype=bool)
    i = 0
    norm2 = 0.0
    while len(us) < kmax:
        used[i] = True
        r = K[i, :].copy()
        for u, v in zip(us, vs):
            r -= u[i] * v
        j = int(np.argmax(np.abs(r)))
        if r[j] == 0.0:
            free = np.flatnonzero(~used)
            if len(free) == 0:
                break
            i = int(free[0])
            continue
        v = r / r[j]
        u = K[:, j].copy()
        for ul, vl in zip(us, vs):
            u -= vl[j] * ul
        cross = sum((ul @ u) * (vl @ v) for ul, vl in zip(us, vs))
        uu, vv = float(u @ u), float(v @ v)
        norm2 += 2.0 * cross + uu * vv
        us.append(u)
        vs.append(v)
        piv.append((i, j))
        if np.sqrt(uu * vv) <= eps_aca * np.sqrt(norm2):
            break
        cand = np.where(used, -1.0, np.abs(u))
        if cand.max() < 0.0:
            break
        i = int(np.argmax(cand))
    U = np.stack(us, axis=1) if us else np.zeros((m, 0))
    V = np.stack(vs, axis=1) if vs else np.zeros((n, 0))
    return (U, V, piv) if return_pivots else (U, V)


def aca_lowrank(K: np.ndarray, eps: float, criterion: str = FROBENIUS, eps_factor: float = None):
    """ACA at eps_ACA = eps_factor eps (default ACA_EPS_FACTOR), then the
    truncated SVD of the approximant (QR of both factors, SVD of the small
    core), truncated with the criterion of Eq. (20).
    Returns (U_t = U_r Sigma_r, V_t, rank, aca_terms)."""
    Ua, Va = aca(K, (ACA_EPS_FACTOR if eps_factor is None else eps_factor) * eps)
    Qu, Ru = np.linalg.qr(Ua)
    Qv, Rv = np.linalg.qr(Va)
    W, s, Zt = np.linalg.svd(Ru @ Rv.T)
    r = max(1, truncation_rank(s, eps, criterion))
    return (Qu @ W[:, :r]) * s[None, :r], Qv @ Zt[:r, :].T, r, Ua.shape[1]


# --------------------------------------------------------------------------
# single low-rank approximation (SA) and its recompression (SArcmp), Sec. 4.1
# --------------------------------------------------------------------------
def sa_factors(ops: np.ndarray, eps: float, criterion: str = FROBENIUS, ts=None):
    """SA of Sec. 4.1, Eqs. (17)-(18), for the operators of a level's T.

    The operators of T (default: all 316, in the order of transfer_vectors())
    are joined as a row K_row = [K_t1, ..., K_t|T|] and as a column
    K_col = [K_t1; ...; K_t|T|];
    K_row ~ U Sigma V^*, K_col ~ A Gamma B^* by truncated SVDs.  The paper gives
    one rank r for both; it is read here as the larger of the two truncation
    ranks at accuracy eps (same criterion as Eq. (20)).  Then
    K_t ~ U C_t B^* with C_t = U^* K_t B.

    Returns dict: U [n3, r], B [n3, r], C [343, r, r] at the t-slots (zeros
    elsewhere), r, the singular values of K_row and K_col, and, for the pins,
    Sigma V_t^* B and U^* A_t Gamma (the paper's two other forms of C_t).
    """
    ts = transfer_vectors() if ts is None else list(ts)
    Ks = [ops[t_slot(t)] for t in ts]
    n3 = Ks[0].shape[0]
    Urow, s_row, Vh_row = np.linalg.svd(np.concatenate(Ks, axis=1), full_matrices=False)
    Acol, s_col, Bh_col = np.linalg.svd(np.concatenate(Ks, axis=0), full_matrices=False)
    r = max(truncation_rank(s_row, eps, criterion), truncation_rank(s_col, eps, criterion))
    U, B = Urow[:, :r], Bh_col[:r, :].T
    C = np.zeros((343, r, r))
    C_sv = np.zeros((343, r, r))
    C_ag = np.zeros((343, r, r))
    for i, t in enumerate(ts):
        sl = t_slot(t)
        C[sl] = U.T @ Ks[i] @ B
        C_sv[sl] = (s_row[:r, None] * Vh_row[:r, i * n3:(i + 1) * n3]) @ B
        C_ag[sl] = U.T @ (Acol[i * n3:(i + 1) * n3, :r] * s_col[None, :r])
    return {"U": U, "B": B, "C": C, "r": r, "s_row": s_row, "s_col": s_col, "C_sigma_v": C_sv,
            "C_a_gamma": C_ag}


def sa_recompress(C: np.ndarray, r: int, eps: float, criterion: str = FROBENIUS, ts=None):
    """SArcmp, Eq. (19) of Sec. 4.1.1: each C_t ~ Ubar_t Vbar_t^* with rank
    r_t (same criterion at accuracy eps, relative to C_t's own singular
    values), kept only when r_t < r / 2; otherwise C_t stays as it is.

    Returns (table [343, r, r] of the represented C_t, ranks [343]: r_t, or r
    where C_t is kept whole, 0 at unused slots).
    """
    out = np.zeros_like(C)
    ranks = np.zeros(343, dtype=np.int64)
    for t in (transfer_vectors() if ts is None else ts):
        sl = t_slot(t)
        u, sv, vh = np.linalg.svd(C[sl])
        rt = truncation_rank(sv, eps, criterion)
        if 2 * rt < r:
            out[sl] = (u[:, :rt] * sv[None, :rt]) @ vh[:rt, :]
            ranks[sl] = rt
        else:
            out[sl] = C[sl]
            ranks[sl] = r
    return out, ranks


def sa_operator_table(ops: np.ndarray, eps: float, recompress: bool = False, criterion: str = FROBENIUS):
    """The SA (or SArcmp) operators U C_t B^* at the t-slots, for m2l_apply.

    Returns (table [343, n3, n3], sa dict, recompression ranks or None).
    """
    sa = sa_factors(ops, eps, criterion)
    C, ranks = (sa_recompress(sa["C"], sa["r"], eps, criterion) if recompress else (sa["C"], None))
    out = np.zeros_like(ops)
    for t in transfer_vectors():
        sl = t_slot(t)
        out[sl] = sa["U"] @ C[sl] @ sa["B"].T
    return out, sa, ranks


# --------------------------------------------------------------------------
# interaction lists (Sec. 3.2, Alg. 1 for asymptotically smooth kernels)
# --------------------------------------------------------------------------
def is_far_pair(x, y) -> bool:
    """Y is in the far field (interaction list) of X at the same level.

    The parents are neighbours (|P(X) - P(Y)|_inf <= 1) and X, Y are not
    (|X - Y|_inf >= 2, i.e. |t| > sqrt(3) in Sec. 3.2).
    """
    px = [v >> 1 for v in x]
    py = [v >> 1 for v in y]
    if max(abs(a - b) for a, b in zip(px, py)) > 1:
        return False
    return max(abs(a - b) for a, b in zip(x, y)) >= 2


def interaction_lists(tgt_ijk: np.ndarray, src_ijk: np.ndarray):
    """CSR interaction lists at one level: for each target (in array order) the
    indices of the source cells in its far field, ascending.

    Candidates are the children of the parent's 27 neighbours (Sec. 3.2); a
    candidate is kept when it exists in src_ijk and passes is_far_pair.
    Returns (offsets int32 [ntgt+1], sources int32 [nnz]).
    """
    index = {tuple(int(v) for v in c): i for i, c in enumerate(np.asarray(src_ijk))}
    offsets = [0]
    sources = []
    for x in np.asarray(tgt_ijk):
        x = tuple(int(v) for v in x)
        px = [v >> 1 for v in x]
        found = []
        for d in itertools.product(range(-1, 2), repeat=3):
            for ch in itertools.product(range(2), repeat=3):
                y = tuple(2 * (px[i] + d[i]) + ch[i] for i in range(3))
                j = index.get(y)
                if j is not None and is_far_pair(x, y):
                    found.append(j)
        sources.extend(sorted(found))
        offsets.append(len(sources))
    return np.asarray(offsets, dtype=np.int32), np.asarray(sources, dtype=np.int32)


def full_grid_cells(level: int) -> np.ndarray:
    """Integer coordinates of all cells of a full uniform level, x fastest."""
    n = 1 << level
    g = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), axis=-1)
    return np.ascontiguousarray(g.transpose(2, 1, 0, 3).reshape(-1, 3).astype(np.int32))


# --------------------------------------------------------------------------
# the M2L translation (Eq. (7)) and its adjoint
# --------------------------------------------------------------------------
def m2l_apply(ops: np.ndarray, tgt_ijk, src_ijk, offsets, sources, multipoles,
              locals_in=None) -> np.ndarray:
    """Cell-by-cell M2L: locals[X] += K_{t(X,Y)} multipoles[Y] (Eq. (7)), FP64."""
    n3 = ops.shape[-1]
    tgt = np.ascontiguousarray(tgt_ijk, dtype=np.int32)
    src = np.ascontiguousarray(src_ijk, dtype=np.int32)
    off = np.ascontiguousarray(offsets, dtype=np.int32)
    srcs = np.ascontiguousarray(sources, dtype=np.int32)
    w = np.ascontiguousarray(multipoles, dtype=np.float64)
    ntgt = tgt.shape[0]
    f = np.zeros((ntgt, n3)) if locals_in is None else np.array(locals_in, dtype=np.float64)
    opsc = np.ascontiguousarray(ops, dtype=np.float64)
    rc = _lib().oracle_m2l_apply(n3, _ptr(opsc), ntgt, _ptr(tgt), _ptr(src), _ptr(off),
                                 _ptr(srcs), _ptr(w), _ptr(f))
    if rc != 0:
        raise ValueError("list entry %d is not a far-field pair" % (-1 - rc))
    return f


def m2l_apply_adjoint(ops: np.ndarray, tgt_ijk, src_ijk, offsets, sources, grad_locals,
                      nsrc: int) -> np.ndarray:
    """Transpose of m2l_apply: grad_multipoles[Y] += K_t^T grad_locals[X]."""
    n3 = ops.shape[-1]
    tgt = np.ascontiguousarray(tgt_ijk, dtype=np.int32)
    src = np.ascontiguousarray(src_ijk, dtype=np.int32)
    off = np.ascontiguousarray(offsets, dtype=np.int32)
    srcs = np.ascontiguousarray(sources, dtype=np.int32)
    gx = np.ascontiguousarray(grad_locals, dtype=np.float64)
    gy = np.zeros((nsrc, n3))
    opsc = np.ascontiguousarray(ops, dtype=np.float64)
    rc = _lib().oracle_m2l_apply_adjoint(n3, _ptr(opsc), tgt.shape[0], _ptr(tgt), _ptr(src),
                                         _ptr(off), _ptr(srcs), _ptr(gx), _ptr(gy))
    if rc != 0:
        raise ValueError("list entry %d is not a far-field pair" % (-1 - rc))
    return gy


# --------------------------------------------------------------------------
# interpolation: S_ell, P2M/M2M, L2L/L2P (Eqs. (3), (6), (8))
# --------------------------------------------------------------------------
def lagrange_1d(ell: int, x) -> np.ndarray:
    """[npts, ell] one-dimensional S_ell(x, xi_k) on reference coordinates in [-1, 1].

    The paper defers the formula of S_ell to its reference [fong09a]; it is
    read here as the Lagrange basis on the ell Chebyshev roots,
    L_k(x) = prod_{j != k} (x - xi_j) / (xi_k - xi_j), the unique interpolant
    of degree ell - 1 (equal, in exact arithmetic, to the Chebyshev-sum form).
    """
    xi = cheb_roots(ell)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    out = np.ones((x.shape[0], ell))
    for k in range(ell):
        for j in range(ell):
            if j != k:
                out[:, k] *= (x - xi[j]) / (xi[k] - xi[j])
    return out


def interp_matrix(ell: int, pts: np.ndarray, center, width: float) -> np.ndarray:
    """[npts, ell^3] S_ell(x, xbar_alpha) of Eq. (3) for points of one cell.

    Points are mapped to the reference cube by the inverse of Phi.
    """
    ref = (np.asarray(pts, dtype=np.float64) - np.asarray(center)[None, :]) / (0.5 * width)
    mi = multi_indices(ell)
    L = [lagrange_1d(ell, ref[:, d]) for d in range(3)]
    return L[0][:, mi[:, 0]] * L[1][:, mi[:, 1]] * L[2][:, mi[:, 2]]


def leaf_coords(pts: np.ndarray, level: int, lo: float = -1.0, domain_width: float = 2.0) -> np.ndarray:
    """Integer leaf-cell coordinates of particles (cells half-open, top face clamped)."""
    n = 1 << level
    w = cell_width(level, domain_width)
    ijk = np.floor((np.asarray(pts) - lo) / w).astype(np.int64)
    return np.clip(ijk, 0, n - 1)


def p2m(ell: int, level: int, pts: np.ndarray, q: np.ndarray, lo: float = -1.0,
        domain_width: float = 2.0, chunk: int = 200000):
    """P2M of Eq. (6): W_beta = sum_j S(y_j, ybar_beta) w_j per non-empty leaf.

    Returns (cells [ncells, 3] int32 sorted by linear index x-fastest,
    multipoles [ncells, ell^3]).
    """
    n = 1 << level
    w = cell_width(level, domain_width)
    ijk = leaf_coords(pts, level, lo, domain_width)
    lin = ijk[:, 0] + n * ijk[:, 1] + n * n * ijk[:, 2]
    ulin, inv = np.unique(lin, return_inverse=True)
    cells = np.stack([ulin % n, (ulin // n) % n, ulin // (n * n)], axis=1).astype(np.int32)
    W = np.zeros((len(ulin), ell ** 3))
    for s in range(0, len(pts), chunk):
        e = min(len(pts), s + chunk)
        centers = lo + w * (ijk[s:e] + 0.5)
        ref = (pts[s:e] - centers) / (0.5 * w)
        mi = multi_indices(ell)
        L = [lagrange_1d(ell, ref[:, d]) for d in range(3)]
        S = L[0][:, mi[:, 0]] * L[1][:, mi[:, 1]] * L[2][:, mi[:, 2]]
        np.add.at(W, inv[s:e], S * q[s:e, None])
    return cells, W


def child_to_parent_matrices(ell: int) -> np.ndarray:
    """[8, ell^3, ell^3] S(ybar^child_beta', ybar^parent_beta) per child octant.

    Child octant o = ox + 2 oy + 4 oz.  Entry [o, beta', beta] is the parent's
    interpolation polynomial beta evaluated at the child's node beta', in the
    parent's reference cube (parent width 2, child width 1, child centre +-1/2).
    """
    out = np.empty((8, ell ** 3, ell ** 3))
    for o in range(8):
        off = np.array([(o >> d) & 1 for d in range(3)], dtype=np.float64) - 0.5
        child_nodes = cell_nodes(ell, off, 1.0)
        out[o] = interp_matrix(ell, child_nodes, np.zeros(3), 2.0)
    return out


def m2m(ell: int, child_cells: np.ndarray, child_W: np.ndarray):
    """M2M of Eq. (6) with the children's nodes as the "particles" carrying W.

    Returns (parent cells sorted by linear index, parent multipoles).
    """
    S8 = child_to_parent_matrices(ell)
    child_cells = np.asarray(child_cells, dtype=np.int64)
    par = child_cells >> 1
    octant = (child_cells[:, 0] & 1) + 2 * (child_cells[:, 1] & 1) + 4 * (child_cells[:, 2] & 1)
    n = int(par.max()) + 1 if len(par) else 1
    lin = par[:, 0] + n * par[:, 1] + n * n * par[:, 2]
    ulin, inv = np.unique(lin, return_inverse=True)
    parents = np.stack([ulin % n, (ulin // n) % n, ulin // (n * n)], axis=1).astype(np.int32)
    Wp = np.zeros((len(ulin), ell ** 3))
    for o in range(8):
        sel = octant == o
        np.add.at(Wp, inv[sel], child_W[sel] @ S8[o])
    return parents, Wp


def l2l(ell: int, parent_F: np.ndarray, octant: int) -> np.ndarray:
    """L2L of Eq. (8): the child's nodes receive the parent's interpolant,
    F^child_alpha' = sum_alpha S(xbar^child_alpha', xbar^parent_alpha) F^parent_alpha."""
    return child_to_parent_matrices(ell)[octant] @ parent_F


def l2p(ell: int, pts: np.ndarray, center, width: float, F: np.ndarray) -> np.ndarray:
    """L2P of Eq. (8): f_i = sum_alpha S(x_i, xbar_alpha) F_alpha."""
    return interp_matrix(ell, pts, center, width) @ F


def direct_sum(kind: int, c: float, targets: np.ndarray, sources: np.ndarray, q: np.ndarray) -> np.ndarray:
    """Eq. (1): f_i = sum_j K(x_i, y_j) w_j, exact coincidences skipped."""
    x = np.ascontiguousarray(targets, dtype=np.float64)
    y = np.ascontiguousarray(sources, dtype=np.float64)
    w = np.ascontiguousarray(q, dtype=np.float64)
    f = np.zeros(x.shape[0])
    _lib().oracle_direct_sum(kind, float(c), x.shape[0], _ptr(x), y.shape[0], _ptr(y), _ptr(w), _ptr(f))
    return f


def rel_l2(approx, exact) -> float:
    """Relative L2 error (Eq. (34)), read with a squared denominator:
    (sum |f - fbar|^2 / sum |f|^2)^(1/2).  Real or complex values."""
    cplx = np.iscomplexobj(approx) or np.iscomplexobj(exact)
    dt = np.complex128 if cplx else np.float64
    a = np.asarray(approx, dtype=dt).ravel()
    e = np.asarray(exact, dtype=dt).ravel()
    den = float(np.sum(np.abs(e) ** 2))
    num = float(np.sum(np.abs(a - e) ** 2))
    return float(np.sqrt(num / den)) if den > 0 else float(np.sqrt(float(np.sum(np.abs(a) ** 2))))


# --------------------------------------------------------------------------
# an FMM evaluation at sampled particles, for the accuracy checks
# --------------------------------------------------------------------------
class UpwardPass:
    """Multipoles of every level 2..leaf of a uniform-depth octree with empty cells pruned.

    levels[L] = (cells [n, 3] int32 sorted x-fastest, multipoles [n, ell^3]).
    """

    def __init__(self, ell, leaf_level, pts, q, lo=-1.0, domain_width=2.0):
        self.ell, self.leaf_level, self.lo, self.domain_width = ell, leaf_level, lo, domain_width
        self.pts, self.q = np.asarray(pts, dtype=np.float64), np.asarray(q, dtype=np.float64)
        self.levels = {}
        cells, W = p2m(ell, leaf_level, self.pts, self.q, lo, domain_width)
        self.levels[leaf_level] = (cells, W)
        for L in range(leaf_level - 1, 1, -1):
            cells, W = m2m(ell, cells, W)
            self.levels[L] = (cells, W)

    def far_field_lists(self, level):
        cells = self.levels[level][0]
        return interaction_lists(cells, cells)


def fmm_at_samples(up: UpwardPass, kind: int, c: float, locals_by_level: dict,
                   sample_idx: np.ndarray) -> np.ndarray:
    """Potential at the sampled particles from M2L locals of levels 2..leaf.

    For a sampled particle in leaf X: descend from level 2 to the leaf, the
    local of each level being its own M2L result plus the L2L of its parent's
    (Eq. (8)); then L2P at the particle plus the direct near field over the
    <= 27 neighbour leaves (Sec. 3.2), the particle itself skipped.
    locals_by_level[L] is [ncells_L, ell^3] in the order of up.levels[L][0].
    """
    ell, Lf = up.ell, up.leaf_level
    pts, q = up.pts, up.q
    leaf_ijk = leaf_coords(pts, Lf, up.lo, up.domain_width)
    n = 1 << Lf
    leaf_lin = leaf_ijk[:, 0] + n * leaf_ijk[:, 1] + n * n * leaf_ijk[:, 2]
    order = np.argsort(leaf_lin, kind="stable")
    sorted_lin = leaf_lin[order]
    index = {L: {tuple(int(v) for v in cc): i for i, cc in enumerate(up.levels[L][0])}
             for L in range(2, Lf + 1)}
    S8 = child_to_parent_matrices(ell)
    out = np.empty(len(sample_idx))
    for si, i in enumerate(sample_idx):
        xi = pts[i]
        leaf = leaf_ijk[i]
        F = None
        for L in range(2, Lf + 1):
            cell = tuple(int(v) for v in (leaf >> (Lf - L)))
            own = locals_by_level[L][index[L][cell]]
            if F is None:
                F = own.copy()
            else:
                octant = (cell[0] & 1) + 2 * (cell[1] & 1) + 4 * (cell[2] & 1)
                F = S8[octant] @ F + own
        w = cell_width(Lf, up.domain_width)
        center = cell_center(leaf, Lf, up.lo, up.domain_width)
        f = float(l2p(ell, xi[None, :], center, w, F)[0])
        near = 0.0
        for d in itertools.product(range(-1, 2), repeat=3):
            nb = leaf + np.array(d)
            if np.any(nb < 0) or np.any(nb >= n):
                continue
            lin = nb[0] + n * nb[1] + n * n * nb[2]
            a = np.searchsorted(sorted_lin, lin, side="left")
            b = np.searchsorted(sorted_lin, lin, side="right")
            if b > a:
                js = order[a:b]
                js = js[js != i]
                near += float(direct_sum(kind, c, xi[None, :], pts[js], q[js])[0])
        out[si] = f + near
    return out


def fmm_oracle_locals(up: UpwardPass, kind: int, c: float, eps: float = 0.0,
                      criterion: str = FROBENIUS) -> dict:
    """M2L locals of every level 2..leaf by the oracle (directly assembled operators)."""
    out = {}
    for L in range(2, up.leaf_level + 1):
        cells, W = up.levels[L]
        off, src = interaction_lists(cells, cells)
        ops = operator_table(up.ell, kind, c, L, up.lo, up.domain_width)
        if eps > 0:
            ops, _ = lowrank_operator_table(ops, eps, criterion)
        out[L] = m2l_apply(ops, cells, cells, off, src, W)
    return out
