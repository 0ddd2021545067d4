/*
 * m2l.h -- C ABI of the GB300 (sm_103a) M2L library.
 *
 * The library computes the multipole-to-local (M2L) translation of the
 * black-box Chebyshev fast multipole method for one octree level at a time,
 * following Messner, Bramas, Coulaud and Darve, "Optimized M2L kernels for
 * the Chebyshev interpolation based fast multipole method":
 *
 *   F_alpha = sum_beta K(xbar_alpha, ybar_beta) W_beta            (Eq. (7))
 *
 * for every far-field pair (X, Y) of the level.  The 316 operators K_t of a
 * level (Eq. (15)) are expressed as permutations of 16 unique ones
 * (Eq. (25), Sec. 4.2.1); interactions sharing an operator are blocked into
 * matrix-matrix products (Alg. 2, Sec. 4.2.3), optionally on per-operator
 * SVD-compressed factors (Eq. (20), Sec. 4.2).
 *
 * Steps of the translation, as the entry points below name them:
 *   a1  the 16 unique operators K_p in FP64 (Eq. (15)), optionally with their
 *       truncated SVD factors (Eq. (20));
 *   a2  the 48 symmetry permutations sigma_g and the table t -> (p, g) over
 *       the 343 transfer vectors (Eqs. (23)-(29), Sec. 4.2.1);
 *   a3  classification: each list entry's t, its (p, g), and the entries
 *       bucketed by operator (Alg. 2, first loop);
 *   a4  gather and permute: W_p[sigma_g(b)][c] = w_Y[b] (Eq. (30), the same
 *       loop);
 *   a5  the blocked product F_p = K_p W_p per operator (Eq. (31), Alg. 2,
 *       second loop);
 *   a6  un-permute and add into the locals: f[a] += F_p[sigma_g(a)][c]
 *       (Eq. (32), Alg. 2, third loop).
 *
 * Conventions shared by every entry point:
 *  - Pointers named "device" are CUDA device pointers owned by the caller;
 *    "host" pointers are ordinary host memory owned by the caller.  The
 *    library owns m2l_ops and m2l_plan objects and the workspace inside them.
 *  - Streams are cudaStream_t values passed as void* (NULL = legacy default
 *    stream).  Every device operation is stream-ordered on that stream; apply
 *    calls return before the GPU has finished.
 *  - Node vectors (multipoles W, locals F) are row-major [ncells][ell^3];
 *    within a vector, node alpha = (a1, a2, a3) (zero-based) sits at
 *    m(alpha) = a1 + a2*ell + a3*ell^2 (Eq. (16), x fastest).
 *  - Chebyshev nodes on the reference interval are the roots of T_ell in
 *    ascending order, -cos((2k+1) pi / (2 ell)), k = 0..ell-1 (Sec. 2.1).
 *  - The transfer vector of a pair is t = X - Y (target minus source) in
 *    integer cell coordinates (Sec. 3.1).  Every list entry must satisfy
 *    |t|_inf in {2, 3}.
 *  - An m2l_ops object belongs to the device that was current when it was
 *    built.  Every entry point that launches work with it (directly, or through
 *    a plan, batch, FMM or SA object built from it) first checks that the
 *    calling thread's current device is that device and returns M2L_EINVAL,
 *    launching nothing, when it is not.  Vectors, lists and streams passed
 *    with it must live on the same device.
 *  - No exception crosses the ABI: every entry point returns an m2l_status;
 *    m2l_last_error() gives a message for the calling thread.  Errors found
 *    by a kernel (a list entry that is not a far-field pair, an index out of
 *    range, a wait that timed out) set a status word on the device; the
 *    entries concerned are skipped and m2l_sync_status() reports the error.
 */
#ifndef M2L_H
#define M2L_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    M2L_OK = 0,
    M2L_EINVAL = 1,        /* bad argument, or a bad interaction list found on the device */
    M2L_ENOMEM = 2,        /* a device allocation failed */
    M2L_ECUDA = 3,         /* a CUDA runtime or library call failed */
    M2L_ETIMEOUT = 4,      /* a bounded device wait gave up (kernel returned early) */
    M2L_EUNSUPPORTED = 5   /* valid request the library cannot serve (e.g. order too large) */
} m2l_status;

/* Kernel functions (Sec. 1; Eq. (33) with the 4*pi factor dropped). */
typedef enum {
    M2L_K_INV_R = 0,          /* 1/r, homogeneous of degree -1 */
    M2L_K_INV_R4 = 1,         /* 1/r^4, homogeneous of degree -4 */
    M2L_K_INV_SQRT_R2C2 = 2   /* 1/sqrt(r^2 + c^2), not homogeneous */
} m2l_kernel_type;

typedef struct {
    int type;   /* m2l_kernel_type */
    double c;   /* used by M2L_K_INV_SQRT_R2C2 only */
} m2l_kernel;

/* Truncation criterion of "accuracy eps" for the low-rank factors (Eq. (20)),
 * SA and SArcmp (Eqs. (17)-(19)), on the singular values s_1 >= s_2 >= ...
 * of the matrix truncated. */
typedef enum {
    M2L_TRUNC_FROBENIUS = 0,  /* smallest r with sum_{i>r} s_i^2 <= eps^2 sum_i s_i^2,
                                 i.e. |K - K_r|_F <= eps |K|_F (the default: the paper's
                                 per-level SA and SArcmp costs of Sec. 5.2 follow from it) */
    M2L_TRUNC_SPECTRAL = 1    /* smallest r with s_{r+1} <= eps s_1, i.e. |K - K_r|_2 <= eps |K|_2 */
} m2l_truncation;
/* Under either criterion a cut never splits a cluster of equal singular
 * values (the truncation would not be unique): r grows while
 * s_r - s_{r+1} <= 1e-12 s_1. */

/* Arithmetic of the operator products (step 2 of Sec. 4.2.2).
 * Multipoles are double for M2L_FP64 and float otherwise. */
typedef enum {
    M2L_FP64 = 0,    /* FP64 SIMT products, FP64 accumulation */
    M2L_FP32 = 1,    /* FP32 SIMT products, FP32 accumulation */
    M2L_TF32 = 2,    /* tcgen05 kind::tf32 tensor-core products, FP32 accumulation in TMEM */
    M2L_BF16X3 = 3,  /* tcgen05 kind::f16 with bf16 hi/lo splits, three products
                        (hi*hi + hi*lo + lo*hi), FP32 accumulation in TMEM */
    M2L_TF32X3 = 4   /* tcgen05 kind::tf32 with tf32 hi/lo splits, three products */
} m2l_precision;

typedef struct m2l_ops m2l_ops;    /* opaque, library-owned */
typedef struct m2l_plan m2l_plan;  /* opaque, library-owned */

/* One octree level's interaction lists.  All pointers are device pointers
 * owned by the caller and must stay valid until the work that uses them has
 * run on the stream. */
typedef struct {
    int level;                   /* octree level, informational */
    double width;                /* cell width w of this level (> 0) */
    int ncells_tgt;              /* number of target cells (>= 0, < 2^26) */
    int ncells_src;              /* number of source cells (>= 0, < 2^26) */
    const int32_t *tgt_ijk;      /* device [ncells_tgt][3] integer coordinates of the targets */
    const int32_t *src_ijk;      /* device [ncells_src][3] integer coordinates of the sources */
    const int32_t *il_offsets;   /* device [ncells_tgt + 1] CSR row offsets over targets, il_offsets[0] = 0 */
    const int32_t *il_sources;   /* device [nnz] source indices in [0, ncells_src) */
    int nnz;                     /* number of list entries, equal to il_offsets[ncells_tgt] */
} m2l_level;

/* ---------------------------------------------------------------------
 * Precompute (Sec. 4.2.1 and Sec. 4.2): builds, on the current device,
 *  - the 16 unique operators K_p, t_p in T_sym = {t1 >= t2 >= t3 >= 0}
 *    (Eqs. (23)-(24)), in FP64, K_p[m(alpha)][n(beta)] = K(xbar_alpha, ybar_beta)
 *    (Eq. (15)).  Homogeneous kernels are assembled at unit width and scaled
 *    by w^degree at apply time (Sec. 3.2); 1/sqrt(r^2+c^2) is assembled at
 *    `width` and may only be applied to levels of that width;
 *  - the 48 permutation tables sigma_g (Eqs. (26)-(29)) and the 343-entry
 *    table t -> (p, g);
 *  - when eps > 0, a truncated SVD of each K_p, K_p ~ (U_p Sigma_p) V_p^T
 *    (Eq. (20)), at the rank the truncation criterion gives (M2L_TRUNC_FROBENIUS
 *    here; m2l_precompute_ex chooses).  The SVD runs on the device in FP64:
 *    Householder QR with column pivoting of K_p^T, then one-sided Jacobi on
 *    R^T (rotations of column pairs in round-robin order until every pair is
 *    orthogonal to 1e-12 relative to the columns' norms).
 * ell: Chebyshev order, 2 <= ell <= 8.  eps: 0 for full rank, else in (0, 1).
 * width: cell width for the non-homogeneous kernel (ignored otherwise).
 * out: receives a new m2l_ops; free with m2l_ops_free.
 * Synchronous (returns after the device work is done).  Errors: M2L_EINVAL
 * for out-of-range arguments, M2L_ENOMEM, M2L_ECUDA. */
m2l_status m2l_precompute(m2l_kernel kernel, int ell, double eps, double width, m2l_ops **out);

/* m2l_precompute with the low-rank factors (eps > 0) computed by adaptive
 * cross approximation followed by a truncated SVD (Sec. 4.1 and Sec. 5, the
 * cheaper precompute; Bebendorf's ACA with partial pivoting), on the device:
 * ACA of each K_p stopped at |u_k| |v_k| <= 0.01 eps |S_k|_F (pivot row 0
 * first; the column of the largest residual; the next row of the largest
 * |u_k| among unused rows; first index on ties), QR of both factor sets
 * (Gram-Schmidt with one re-orthogonalisation), one-sided Jacobi SVD of the
 * small core, truncation with the criterion of m2l_precompute.  The factors
 * have the layout of m2l_precompute's (U = U_K Sigma, V = V_K) and every apply
 * entry point uses them alike.  With eps = 0 it equals m2l_precompute.
 * Errors as m2l_precompute; M2L_ECUDA if a Jacobi SVD does not converge. */
m2l_status m2l_precompute_aca(m2l_kernel kernel, int ell, double eps, double width, m2l_ops **out);

/* m2l_precompute (aca = 0) or m2l_precompute_aca (aca = 1) with the truncation
 * criterion `trunc` (m2l_truncation) for the low-rank factors; SA objects made
 * from the ops (m2l_sa_create) use the same criterion.  M2L_EINVAL for an
 * unknown criterion or aca outside {0, 1}; other errors as m2l_precompute. */
m2l_status m2l_precompute_ex(m2l_kernel kernel, int ell, double eps, double width, int trunc, int aca,
                             m2l_ops **out);

/* The truncation criterion (m2l_truncation) the ops were built with. */
m2l_status m2l_ops_truncation(const m2l_ops *ops, int *trunc);

/* Jacobi sweeps of the SVD of each operator p (the full K_p for m2l_precompute,
 * the ACA core for m2l_precompute_aca); M2L_EINVAL for full-rank ops. */
m2l_status m2l_ops_svd_sweeps(const m2l_ops *ops, int32_t *sweeps16);

/* Per operator p: ACA terms before the recompression and Jacobi sweeps, for
 * ops from m2l_precompute_aca with eps > 0 (else M2L_EINVAL); NULL skips one. */
m2l_status m2l_ops_aca_info(const m2l_ops *ops, int32_t *aca_terms16, int32_t *jacobi_sweeps16);

/* Re-runs the device assembly of the full-rank operators and tables of
 * `ops` into its existing buffers (no allocation), stream-ordered.  Used to
 * time the precompute as part of a step.  M2L_EUNSUPPORTED for ops built with
 * eps > 0. */
m2l_status m2l_ops_rebuild(m2l_ops *ops, void *stream);

/* m2l_ops_rebuild in two parts, for a step that classifies its levels while
 * the operators are assembled: m2l_ops_rebuild_tables re-runs the tables of
 * Sec. 4.2.1 (sigma_g, the t -> (p, g) table, T_sym: all that classification
 * reads), m2l_ops_rebuild_operators the assembly of the 16 operators
 * (Eq. (15), which reads T_sym), so it must follow the tables in stream order.
 * Classification of a level may run on another stream once the tables are
 * done; an apply needs both parts (and m2l_ops_prepare) done.  Same rules and
 * errors as m2l_ops_rebuild. */
m2l_status m2l_ops_rebuild_tables(m2l_ops *ops, void *stream);
m2l_status m2l_ops_rebuild_operators(m2l_ops *ops, void *stream);

/* Host copies of the tables, for checking (Sec. 4.2.1).  Any output may be
 * NULL.  ranks16: [16] ranks r_p (ell^3 when full rank).  sigma48: [48][ell^3]
 * with sigma48[g][j] = m(pi_g(m^{-1}(j))), g = 8 * perm_id + flip_mask where
 * flip_mask bit i is set when t_i < 0 and perm_id indexes the axis order
 * (|t_i| >= |t_j| >= |t_k|, ties by lower axis first) among the six
 * permutations of (0,1,2) in lexicographic order.  lut343: at slot
 * (t1+3) + 7 (t2+3) + 49 (t3+3), p | (g << 8), with p the index of p(t) in
 * T_sym sorted lexicographically ascending, or 0xFFFF for |t|_inf <= 1.
 * Then K_t[a][b] = K_p[sigma_g(a)][sigma_g(b)]. */
m2l_status m2l_ops_query(const m2l_ops *ops, int *ranks16, int16_t *sigma48, uint16_t *lut343);

/* Host copy of the 16 FP64 operators as stored ([16][ell^3][ell^3], at unit
 * width for homogeneous kernels).  host_out must hold 16 * ell^6 doubles. */
m2l_status m2l_ops_copy_operators(const m2l_ops *ops, double *host_out);

/* Host copy of the low-rank factors of operator p: U (= U_p Sigma_p) and V,
 * both [ell^3][r_p] row-major.  M2L_EINVAL when ops is full rank. */
m2l_status m2l_ops_copy_lowrank(const m2l_ops *ops, int p, double *host_U, double *host_V);

/* Basic facts of an ops object; any output may be NULL. */
m2l_status m2l_ops_info(const m2l_ops *ops, int *ell, int *kernel_type, double *eps,
                        double *ref_width, int *homogeneity_degree);

void m2l_ops_free(m2l_ops *ops);

/* ---------------------------------------------------------------------
 * Apply (Eq. (7) through Eqs. (30)-(32) and Alg. 2):
 *   locals[X] += sum_{Y in list(X)} K_{t(X,Y)} multipoles[Y]
 * Step a3: every entry is classified by t -> (p, g) and bucketed per
 * operator p, ordered by target (stable).  Steps a4-a6 run in one fused
 * kernel per precision: gather and permute the source vectors into the
 * panel W_p (W_p[sigma_g(b)] = w[b]), product F_p = K_p W_p, un-permute
 * (f[a] += F_p[sigma_g(a)]), sum over the columns of one target, scaled by
 * w^degree for homogeneous kernels, and one atomic add per target and node.
 * multipoles: device [ncells_src][ell^3], double for M2L_FP64 else float.
 * locals:     device [ncells_tgt][ell^3], accumulated (+=); double when
 *             precision == M2L_FP64 or locals_fp64 != 0, else float.
 * The workspace of ops is used: two apply calls on one ops object must not
 * overlap on the GPU (use plans, below, for that).
 * Errors: M2L_EINVAL (bad sizes, mismatched width for the non-homogeneous
 * kernel), M2L_EUNSUPPORTED, M2L_ENOMEM, M2L_ECUDA; list errors found on the
 * device are reported by m2l_sync_status. */
m2l_status m2l_apply_level(const m2l_ops *ops, const m2l_level *level, const void *multipoles,
                           void *locals, int precision, int locals_fp64, void *stream);

/* Adjoint of m2l_apply_level: grad_multipoles[Y] += K_t^T grad_locals[X]
 * over the same pairs.  Since K_{-t} = K_t^T (the kernel is symmetric, and
 * -t is the transfer vector of the reversed pair, Sec. 3.1), this is the
 * forward translation on the transposed list, which the library builds on
 * the device.  grad_locals: [ncells_tgt][ell^3];
 * grad_multipoles: [ncells_src][ell^3], accumulated; types as for apply with
 * the roles of the two arrays exchanged. */
m2l_status m2l_apply_level_adjoint(const m2l_ops *ops, const m2l_level *level,
                                   const void *grad_locals, void *grad_multipoles,
                                   int precision, int grad_fp64, void *stream);

/* The two halves of m2l_apply_level, for callers that time or overlap them:
 * m2l_classify_level runs step a3 into the workspace of ops (growing it on
 * first use), m2l_apply_classified runs steps a4-a6 on the last
 * classification of ops (same argument meanings as m2l_apply_level; the
 * level's width is remembered).  Both are stream-ordered; the pair on one ops
 * object must not overlap another apply on that object. */
m2l_status m2l_classify_level(const m2l_ops *ops, const m2l_level *level, void *stream);
m2l_status m2l_apply_classified(const m2l_ops *ops, const void *multipoles, void *locals, int precision,
                                int locals_fp64, void *stream);

/* Plans: the classification (step a3) of one level's lists, kept in
 * plan-owned device memory so that repeated applies on unchanged lists skip
 * it.  The level's ijk/list arrays are read at creation only.  adjoint != 0
 * plans the transposed translation.  m2l_plan_apply allocates nothing and is
 * stream-ordered. */
m2l_status m2l_plan_create(const m2l_ops *ops, const m2l_level *level, int adjoint, void *stream,
                           m2l_plan **out);
m2l_status m2l_plan_apply(const m2l_plan *plan, const void *in_vectors, void *out_vectors,
                          int precision, int out_fp64, void *stream);
/* Host copy of a plan's per-operator counts n_p ([16]) and bucketed records
 * ([nvalid][3]: source index, target index, g, in execution order). */
m2l_status m2l_plan_query(const m2l_plan *plan, int64_t *counts16, int32_t *records, int64_t *nvalid);
void m2l_plan_free(m2l_plan *plan);
/* Which kernel the tensor-core applies of a plan take.  *dense = 1 when the
 * level was also classified for the target-stationary kernel (ell <= 5,
 * full-rank operators, at least 16384 target cells whose lists hold at least
 * half of the 189 far-field entries per cell of a full level, Sec. 3.2): its
 * targets are grouped by octant into at most *units units of *unit_width
 * columns.  *dense = 0: the operator-bucketed kernel.  Host-side only (no
 * synchronisation); any output pointer may be NULL. */
m2l_status m2l_plan_kernel_info(const m2l_plan *plan, int *dense, int *units, int *unit_width);
/* Re-classify a level into an existing plan (step a3 of Alg. 2, as in
 * m2l_plan_create), asynchronously on `stream`: no host synchronisation, and
 * no allocation once the plan's buffers have held a classification of at
 * least level->nnz entries (the first call after m2l_plan_create allocates its
 * scratch again).  The plan keeps its direction (adjoint or not) and takes
 * the level's width.  Plans of different levels may be re-classified and
 * applied concurrently on different streams; calls on one plan are ordered by
 * its stream.  Errors: M2L_EINVAL for a null plan or an invalid level (as
 * m2l_apply_level); bad list entries are reported by m2l_sync_status. */
m2l_status m2l_plan_classify(m2l_plan *plan, const m2l_level *level, void *stream);

/* Build, on `stream`, the kernel layouts of the operators for `precision`
 * (the step every first apply after m2l_precompute / m2l_ops_rebuild takes
 * otherwise): call it before applying one m2l_ops from several streams, so
 * that no apply builds them concurrently.  Stream-ordered; allocates on its
 * first call per precision only.  Errors: M2L_EINVAL (null ops, unknown
 * precision), M2L_EUNSUPPORTED (as the apply would return). */
m2l_status m2l_ops_prepare(const m2l_ops *ops, int precision, void *stream);

/* Batched apply: nbatch independent (ops, level) problems, classified (one
 * plan each) and then applied as an m2l_batch (m2l_batch_create/run/free
 * inside the call; the call synchronises `stream` and allocates its plans --
 * create an m2l_batch once for repeated or graph-captured use).  Tensor-core
 * precisions with FP64 locals, orders above 6 or low-rank operators apply the
 * problems one launch each.  in[i], out[i] follow the types of m2l_apply_level. */
m2l_status m2l_apply_batch(const m2l_ops *const *ops, const m2l_level *levels,
                           const void *const *multipoles, void *const *locals, int nbatch,
                           int precision, int locals_fp64, void *stream);

/* Persistent batches (the batched-trees workload): a fixed set of planned
 * translations -- any mix of trees, levels, orders and operator sets -- run
 * by persistent kernel launches over a global tile queue (the blocking of
 * Alg. 2 along many target cells, Sec. 4.2.3, extended across problems).
 *  - M2L_FP32, M2L_FP64: CUDA-core products, ONE launch over every problem
 *    (ell <= 7; out_fp64 selects double outputs for FP32);
 *  - M2L_TF32, M2L_BF16X3, M2L_TF32X3: tcgen05 products, ONE launch per
 *    vector length ell^3 over every problem of that order (ell <= 6), each
 *    class (problem, unique operator) with its operator image -- images built
 *    once per distinct operator set and scale; per order the problems' input
 *    vectors are gathered into one array by a kernel and the results added
 *    back by another (FP32 outputs only).
 * in[i], out[i]: device vectors of plan i (types as m2l_plan_apply).
 * Creation reads the plans' bucket sizes (synchronises `stream`), picks the
 * tile shape with a built-in autotuner -- each candidate timed on scratch
 * outputs: tile width 32 or 64 for the CUDA cores; for the tensor cores, tile
 * width 32 or 64 interactions and one or two epilogue groups wherever they fit
 * shared memory -- cached per precision, order and interaction count, and
 * uploads the descriptor tables.  m2l_batch_run allocates nothing and issues a
 * fixed sequence of launches, so it may be captured in a CUDA graph; the
 * plans and vectors must outlive the batch, and the batch copies the plans'
 * buckets at creation (re-classifying a plan does not change the batch).
 * List errors found on the device are reported to the status word of the
 * first plan's operators.  Full-rank operators only. */
typedef struct m2l_batch m2l_batch;
m2l_status m2l_batch_create(const m2l_plan *const *plans, int nbatch, const void *const *in, void *const *out,
                            int precision, int out_fp64, void *stream, m2l_batch **out_batch);
m2l_status m2l_batch_run(const m2l_batch *batch, void *stream);
/* tile_width: columns per tile chosen by the autotuner; tiles: tiles per run;
 * tuned_ms: the autotuner's best time (0 when taken from its cache). */
m2l_status m2l_batch_info(const m2l_batch *batch, int *tile_width, int64_t *tiles, double *tuned_ms);
/* Per launch group of a batch (host-side): ell3[i] the vector length of group
 * i (the padded order of the CUDA-core batch's single group), tile_width[i]
 * and epilogue_groups[i] the autotuner's choice (0 epilogue groups for the
 * CUDA cores); up to max_groups entries are written, *ngroups receives the
 * number of groups. */
m2l_status m2l_batch_groups(const m2l_batch *batch, int max_groups, int32_t *ell3, int32_t *tile_width,
                            int32_t *epilogue_groups, int32_t *ngroups);
void m2l_batch_free(m2l_batch *batch);

/* ---------------------------------------------------------------------
 * The bbFMM matvec around the M2L translation (Sec. 2.1.1, Eqs. (5)-(8)):
 * P2M at the leaves, M2M up to level 2, the symmetry-blocked M2L at every
 * level 2..leaf, L2L down to the leaves, then L2P plus the direct near field
 * over the <= 27 neighbour leaves (Eq. (1) restricted to them, exact
 * coincidences skipped).  Uniform-depth octree on [lo, lo + domain_width)^3
 * with empty cells pruned; particles are binned into half-open leaf cells
 * (top face clamped); the cells of a level are sorted by linear index (x
 * fastest), as are the lists of m2l_build_lists.  The paper leaves these
 * passes unchanged; they surround the path it optimises.
 *
 * m2l_fmm_create: ops[L - 2] are the operators of level L = 2..leaf_level
 *   (one m2l_ops for all levels when the kernel is homogeneous; a
 *   non-homogeneous kernel needs one set per level width); they must share
 *   kernel and order (ell <= 8).  xyz: device [n][3], double if fp64 != 0,
 *   else float.  Builds the tree, the kept cells of every level, their
 *   interaction lists and one M2L plan per level; synchronous; allocates
 *   everything it keeps.  leaf_level in [2, 8].
 * m2l_fmm_evaluate: charges (device [n]) -> potentials (device [n], written,
 *   input order), same type as xyz; precision M2L_FP64 for an fp64 FMM, one
 *   of the other precisions for an FP32 one.  Stream-ordered; no allocation.
 * m2l_fmm_query: host copies of level L's cell coordinates ([ncells][3]),
 *   multipoles W and locals F ([ncells][ell^3], the FMM's type; F includes
 *   the L2L of the parents) after an evaluate; NULL skips one.  Synchronous.
 * m2l_fmm_info: leaf level and, per level 0..8, kept cells and list entries.
 * Errors: M2L_EINVAL (bad arguments, precision not matching the FMM's type),
 * M2L_EUNSUPPORTED (ell > 8 or level width beyond the operators'), and those
 * of m2l_plan_create / m2l_plan_apply. */
typedef struct m2l_fmm m2l_fmm;
m2l_status m2l_fmm_create(const m2l_ops *const *ops, int n_particles, const void *xyz, int fp64,
                          int leaf_level, double lo, double domain_width, void *stream, m2l_fmm **out);
m2l_status m2l_fmm_evaluate(const m2l_fmm *fmm, const void *xyz, const void *charges, void *potentials,
                            int precision, void *stream);
m2l_status m2l_fmm_query(const m2l_fmm *fmm, int level, int32_t *host_ijk, void *host_W, void *host_F);
m2l_status m2l_fmm_info(const m2l_fmm *fmm, int *leaf_level, int64_t *ncells9, int64_t *nnz9);
void m2l_fmm_free(m2l_fmm *fmm);

/* ---------------------------------------------------------------------
 * SA and SArcmp (Sec. 4.1, Eqs. (17)-(19)): the alternative that compresses
 * all 316 operators of a level with ONE pair of bases instead of using their
 * symmetries.  The operators are joined as K_row = [K_t1 ... K_t316] and
 * K_col = [K_t1; ...; K_t316]; truncated SVDs K_row ~ U S V^T and
 * K_col ~ A G B^T give K_t ~ U C_t B^T with the r x r cores C_t = U^T K_t B
 * (Eq. (18)).  r is the larger of the two truncation ranks at accuracy eps
 * under the truncation criterion of ops (m2l_truncation; eps = 0 keeps all
 * n3 = ell^3 of them).  SArcmp (recompress != 0, Eq. (19)) replaces a core by
 * its truncated SVD X_t Y_t^T of rank r_t (same criterion, on C_t's own
 * singular values) when 2 r_t < r; otherwise C_t is kept.
 *
 * m2l_sa_create: builds the factors of the operators in ops (full rank, any
 *   eps of ops; only ops' 16 unique operators and their symmetries are
 *   read) in FP64 on the device, every SVD by one-sided Jacobi rotations
 *   (as m2l_precompute's); synchronous; allocates what it keeps.  eps in
 *   [0, 1).  r <= 128 (larger: M2L_EUNSUPPORTED).
 * m2l_sa_info: r, the number of recompressed cores and (host [343], may be
 *   NULL) r_t per t-slot (t + 3) . (1, 7, 49), 0 where C_t is kept whole or
 *   the slot is not a far-field transfer vector.
 * m2l_sa_copy_factors: host copies (FP64) of U^T [r][n3], B [n3][r], and the
 *   per-slot X [343][r][r] and Y [343][r][r]: X holds C_t where r_t = 0,
 *   else X_t in its first r_t columns with Y_t in Y's; NULL skips one.
 *   Synchronous.
 * m2l_sa_apply_level: locals[X] += scale U C_t B^T multipoles[Y] over the
 *   level's list, computed as compress (w^ = B^T w for every source cell),
 *   cores per transfer vector (f^[X] += C_t w^[Y]), decompress
 *   (F += scale U f^); scale as m2l_apply_level.  precision M2L_FP64 (double
 *   vectors) or M2L_FP32 (float multipoles; locals float, or double with
 *   locals_fp64 != 0) on the CUDA cores; M2L_TF32 / M2L_BF16X3 / M2L_TF32X3
 *   (float vectors as M2L_FP32) run the cores on the tcgen05 tensor cores,
 *   one class per transfer vector, with the dense C_t (X_t Y_t^T where SArcmp
 *   recompressed it); the first call in such a precision builds its operator
 *   images (synchronous, allocating).  Stream-ordered; allocates its
 *   workspace on first use or growth; list errors as m2l_apply_level
 *   (skipped entries, reported by m2l_sync_status on sa's ops).  Work on one
 *   m2l_sa object must be ordered on one stream.
 * Errors: M2L_EINVAL (null or bad arguments), M2L_EUNSUPPORTED (rank,
 *   precision), M2L_ECUDA / M2L_ENOMEM. */
typedef struct m2l_sa m2l_sa;
m2l_status m2l_sa_create(const m2l_ops *ops, double eps, int recompress, void *stream, m2l_sa **out);
m2l_status m2l_sa_info(const m2l_sa *sa, int *rank, int *n_recompressed, int32_t *host_rt343);
m2l_status m2l_sa_copy_factors(const m2l_sa *sa, double *host_Ut, double *host_B, double *host_X,
                               double *host_Y);
m2l_status m2l_sa_apply_level(const m2l_sa *sa, const m2l_level *level, const void *multipoles, void *locals,
                              int precision, int locals_fp64, void *stream);
void m2l_sa_free(m2l_sa *sa);

/* ---------------------------------------------------------------------
 * Directional FMM (dFMM) M2L for the Helmholtz kernel (Sec. 2.1.2):
 *   F^u_X += K_t W^u_Y,  (K_t)_{ab} = exp(i k r_ab) / r_ab,  r_ab = |xbar_a - ybar_b|
 * (Eq. (13); the 4 pi of Eq. (33) dropped like for the other kernels).  The
 * directional phases exp(+-i k u.x) belong to P2M and L2P (Eqs. (12), (14));
 * the M2L operator is the plain kernel, identical for every cone, and the 48
 * symmetries of Sec. 4.2.1 apply to any transfer vector.  Each cell of a
 * level holds one expansion per cone: multipoles and locals are complex,
 * interleaved (re, im), [ncells][n_cones][ell^3] (complex double for
 * M2L_FP64, complex float for M2L_FP32).
 *
 * Readings (the paper defers these to its reference on the dFMM):
 *  - a level of cell width w is high-frequency (hf) when k w >= 1;
 *  - a pair is admissible when |t|_inf >= 2 and, at an hf level, also
 *    |c_X - c_Y| > max(k w^2, 2 w), evaluated in FP64 as
 *    ((t.t) w) w > ((k w) w)^2 and t.t > 4;
 *  - cones: each face of the cube [-1, 1]^3 split into m x m squares, m the
 *    smallest power of two >= k w (m = 0, one cone, at an lf level); the cone
 *    of a pair is the square hit along c_X - c_Y: face axis f = the first axis
 *    of largest |t_i|, side s = (t_f < 0), on the other axes a < b the squares
 *    i = min(floor((t_a + |t_f|) m / (2 |t_f|)), m - 1); cone
 *    (2 f + s) m^2 + i_b m + i_a;
 *  - lists (Alg. 1 on a uniform-depth octree, per level): Y is in the list of
 *    (X, cone of X - Y) when the pair is admissible at this level and no pair
 *    of their ancestors at levels 0 .. level - 1 is.
 *
 * m2l_dfmm_build_lists: the lists of `level` (cell width domain_width /
 *   2^level, coordinates in [0, 2^level)^3, level <= 8, m <= 32).  CSR over
 *   target expansions e = x * n_cones + c: il_offsets device
 *   [ncells_tgt * n_cones + 1]; within an expansion the sources ascend in
 *   linear cell index (x fastest), i.e. in source index when the source
 *   cells are sorted that way (source cells must be distinct).  Three
 *   calls: with il_offsets == NULL it only writes *n_cones; with
 *   il_sources == NULL it writes *n_cones, the offsets and *nnz_out; then it
 *   fills il_sources (device [nnz]).  Synchronous.  The source expansion of
 *   an entry is y * n_cones + c.
 * m2l_dfmm_plan_create: classifies the level's entries (t -> p(t), g(t)),
 *   finds T_sym (the distinct p(t), lexicographic) and the class sizes n_p
 *   (Sec. 4.2.3: not known before the lists), assembles the complex K_p at
 *   the level's width in FP64 (and an FP32 copy) and buckets the entries.
 *   Synchronous; allocates what it keeps; the level's arrays may be freed
 *   afterwards.  Entries with |t|_inf < 2 or indices out of range:
 *   M2L_EINVAL.
 * m2l_dfmm_plan_info: |T_sym|, n_cones, nnz; host_tsym [nsym][3] and
 *   host_np [nsym] when not NULL.
 * m2l_dfmm_plan_apply: locals += M2L(multipoles), stream-ordered.
 *   M2L_FP64 / M2L_FP32: complex products on the CUDA cores (complex double /
 *   complex float vectors).  M2L_TF32 / M2L_BF16X3 / M2L_TF32X3 (ell <= 5,
 *   complex float vectors): the complex product as a real one of twice the
 *   size, [[Re K, -Im K], [Im K, Re K]] on the stacked (Re, Im) vector, on
 *   the tcgen05 tensor cores with FP32 accumulation.  Results are added with
 *   atomics, so the summation order of a target varies from run to run
 *   within rounding.  The first call in a tensor-core precision builds that
 *   precision's operator images as m2l_dfmm_plan_prepare does (synchronous,
 *   allocating); later calls allocate nothing.
 * m2l_dfmm_plan_prepare: builds the layout of one precision ahead of the
 *   first apply (synchronous).  M2L_EUNSUPPORTED for a tensor-core precision
 *   with ell > 5.
 * m2l_dfmm_plan_sync: synchronises `stream`, returns and clears the plan's
 *   device status word (M2L_ETIMEOUT when a bounded wait of the tensor-core
 *   kernel gave up). */
typedef struct {
    int level;                   /* octree level, informational */
    double width;                /* cell width w (> 0) */
    int ncells_tgt, ncells_src;  /* cells; ncells_tgt * n_cones < 2^26 */
    int n_cones;                 /* expansions per cell (>= 1) */
    const int32_t *tgt_ijk;      /* device [ncells_tgt][3] */
    const int32_t *src_ijk;      /* device [ncells_src][3] */
    const int32_t *il_offsets;   /* device [ncells_tgt * n_cones + 1], CSR over target expansions */
    const int32_t *il_sources;   /* device [nnz] source cells */
    int nnz;
} m2l_dlevel;
typedef struct m2l_dplan m2l_dplan;
m2l_status m2l_dfmm_build_lists(int level, double wavenumber, double domain_width, int ncells_tgt,
                                const int32_t *tgt_ijk, int ncells_src, const int32_t *src_ijk, int *n_cones,
                                int32_t *il_offsets, int32_t *il_sources, int64_t *nnz_out, void *stream);
m2l_status m2l_dfmm_plan_create(int ell, double wavenumber, const m2l_dlevel *level, void *stream,
                                m2l_dplan **out);
m2l_status m2l_dfmm_plan_info(const m2l_dplan *plan, int *nsym, int *n_cones, int64_t *nnz, int32_t *host_tsym,
                              int64_t *host_np);
m2l_status m2l_dfmm_plan_apply(const m2l_dplan *plan, const void *multipoles, void *locals, int precision,
                               void *stream);
m2l_status m2l_dfmm_plan_prepare(m2l_dplan *plan, int precision, void *stream);
m2l_status m2l_dfmm_plan_sync(const m2l_dplan *plan, void *stream);
void m2l_dfmm_plan_free(m2l_dplan *plan);

/* ---------------------------------------------------------------------
 * Interaction lists (Sec. 3.2, Alg. 1 for asymptotically smooth kernels):
 * Y is in the list of X when their parents are neighbours,
 * |floor(X/2) - floor(Y/2)|_inf <= 1, and |X - Y|_inf >= 2.  Sources of a
 * target are listed in ascending source index.  Two calls: with
 * il_sources == NULL, writes the row offsets (device [ncells_tgt + 1]) and
 * *nnz_out (host); then, with il_sources (device [nnz]), fills the lists.
 * Cells are looked up in a dense table of side 2^max_coord_bits (<= 256).
 * Synchronous. */
m2l_status m2l_build_lists(int ncells_tgt, const int32_t *tgt_ijk, int ncells_src,
                           const int32_t *src_ijk, int32_t *il_offsets, int32_t *il_sources,
                           int64_t *nnz_out, void *stream);

/* ---------------------------------------------------------------------
 * m2l_apply_level_noalloc: m2l_apply_level with M2L_FP32 products and float
 * locals, for callers that must not allocate device memory while they run --
 * code that executes between a framework's set-up and tear-down phases under
 * a fixed memory budget, inside a real-time loop, or where a cudaMalloc would
 * synchronise the device or deadlock against another allocator.  The paper
 * has no counterpart: it is an interface of this library only.
 * It calls no cudaMalloc, cudaFree or allocating library routine.  Its
 * scratch (interaction buckets and the FP32 operator layout) is one
 * file-scope device array of about 10.7 MB that every GPU which loads the
 * library holds until the process exits.  Limits: nnz <= 524288 list
 * entries, ell <= 6, full-rank ops (eps == 0); larger requests return
 * M2L_EINVAL (nnz) or M2L_EUNSUPPORTED (ell, low rank) before any work.
 * The first call on a device looks up the array's device address with
 * cudaGetSymbolAddress (once per device, with that device current): make
 * that first call before any stream capture.  All calls share the array and
 * each call rewrites what it reads, so calls whose GPU work overlaps (other
 * streams, other threads) race: order them on one stream.
 * Arguments and results as m2l_apply_level (locals accumulated, list errors
 * reported by m2l_sync_status). */
m2l_status m2l_apply_level_noalloc(const m2l_ops *ops, const m2l_level *level, const float *multipoles,
                                   float *locals, void *stream);

/* Test switches of an ops object (0 = none).  M2L_DEBUG_STALL_PRODUCER makes
 * every CTA of the tensor-core apply withhold its first stage signal: the
 * MMA warp's bounded wait (about two seconds) runs out, the CTA drains its
 * own asynchronous copies, frees its tensor memory and returns, and the next
 * m2l_sync_status reports M2L_ETIMEOUT.  Used to test failure detection
 * without faulting the GPU; the results of such a call are incomplete. */
#define M2L_DEBUG_STALL_PRODUCER 1
/* M2L_DEBUG_NO_DENSE makes the tensor-core precisions apply full levels with
 * the operator-bucketed kernel instead of the target-stationary one, so that
 * the two can be compared on the same plan (results agree to rounding). */
#define M2L_DEBUG_NO_DENSE 2
m2l_status m2l_ops_set_debug(m2l_ops *ops, int flags);

/* ---------------------------------------------------------------------
 * Synchronises `stream`, then returns and clears the device status word of
 * ops (M2L_OK, M2L_EINVAL for list entries that were skipped, M2L_ETIMEOUT). */
m2l_status m2l_sync_status(const m2l_ops *ops, void *stream);

/* Message of the last failing call on this thread ("" if none). */
const char *m2l_last_error(void);

/* Number of kernel launches the library has issued on this process (all
 * entry points), for launch accounting. */
int64_t m2l_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* M2L_H */
