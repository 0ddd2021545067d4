/*
 * Plain FP64 CPU loops of the M2L oracle.  TEST INFRASTRUCTURE ONLY: nothing
 * in the product path may link or call this file; only tests, the smoke check
 * and the CPU-baseline leg of the benchmark do.
 *
 * Every routine is a literal transcription of a definition of the paper
 * (Messner, Bramas, Coulaud, Darve, "Optimized M2L kernels for the Chebyshev
 * interpolation based fast multipole method"), with no blocking, no symmetry
 * and no reordering of sums beyond the definition's own order.
 *
 * Build: gcc -O2 -ffp-contract=off -shared -fPIC m2l_oracle.c -o libm2l_oracle.so -lm
 * (-ffp-contract=off keeps every product rounded before it is added, on x86
 * and on Arm alike.)
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>

/* Kernel functions (Sec. 1 and Eq. (33); the configs use 1/r without 4*pi):
 * kind 0: 1/r, kind 1: 1/r^4, kind 2: 1/sqrt(r^2 + c^2). */
static double kernel_of_r(int kind, double c, double r)
{
    if (kind == 0) return 1.0 / r;
    if (kind == 1) { double r2 = r * r; return 1.0 / (r2 * r2); }
    return 1.0 / sqrt(r * r + c * c);
}

static double kernel_xy(int kind, double c, const double *x, const double *y)
{
    double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
    double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    return kernel_of_r(kind, c, r);
}

/*
 * M2L operator of one cell pair, Eq. (15): (K_t)_{m(alpha) n(beta)} =
 * K(xbar_alpha, ybar_beta).  xnodes, ynodes: [n3][3] absolute node
 * coordinates of the target and source cell, already in m()/n() order.
 * out: row-major [n3][n3].
 */
void oracle_assemble_pair(int kind, double c, int n3, const double *xnodes,
                          const double *ynodes, double *out)
{
    for (int a = 0; a < n3; ++a)
        for (int b = 0; b < n3; ++b)
            out[(size_t)a * n3 + b] = kernel_xy(kind, c, xnodes + 3 * a, ynodes + 3 * b);
}

/*
 * Cell-by-cell M2L, Eq. (7): for every target X (in array order) and every
 * source Y of its interaction list (in list order), f_X += K_{t(X,Y)} w_Y,
 * with t = (c_X - c_Y)/w (Sec. 3.1) taken from integer cell coordinates.
 *
 * ops: [343][n3][n3], the operator of transfer vector t stored at slot
 * (t1+3) + 7 (t2+3) + 49 (t3+3); the caller fills the slots it needs.
 * scale multiplies every product sum (1.0 for plain use).
 * Returns 0, or -1 - e for the first list entry e whose t is outside
 * [-3,3]^3 or inside the near field (|t|_inf <= 1).
 */
long oracle_m2l_apply(int n3, const double *ops, int ntgt, const int32_t *tgt_ijk,
                      const int32_t *src_ijk, const int32_t *offsets, const int32_t *sources,
                      const double *multipoles, double *locals)
{
    for (int x = 0; x < ntgt; ++x) {
        double *f = locals + (size_t)x * n3;
        for (int e = offsets[x]; e < offsets[x + 1]; ++e) {
            int y = sources[e];
            int t1 = tgt_ijk[3 * x + 0] - src_ijk[3 * y + 0];
            int t2 = tgt_ijk[3 * x + 1] - src_ijk[3 * y + 1];
            int t3 = tgt_ijk[3 * x + 2] - src_ijk[3 * y + 2];
            int m = abs(t1) > abs(t2) ? abs(t1) : abs(t2);
            m = m > abs(t3) ? m : abs(t3);
            if (m < 2 || m > 3) return -1 - (long)e;
            const double *K = ops + (size_t)((t1 + 3) + 7 * (t2 + 3) + 49 * (t3 + 3)) * n3 * n3;
            const double *w = multipoles + (size_t)y * n3;
            for (int a = 0; a < n3; ++a) {
                double s = 0.0;
                for (int b = 0; b < n3; ++b) s += K[(size_t)a * n3 + b] * w[b];
                f[a] += s;
            }
        }
    }
    return 0;
}

/*
 * Adjoint of the map above: g_Y += K_{t(X,Y)}^T g_X over the same pairs
 * (the transpose of Eq. (7) as a linear map from all w to all f).
 */
long oracle_m2l_apply_adjoint(int n3, const double *ops, int ntgt, const int32_t *tgt_ijk,
                              const int32_t *src_ijk, const int32_t *offsets,
                              const int32_t *sources, const double *grad_locals,
                              double *grad_multipoles)
{
    for (int x = 0; x < ntgt; ++x) {
        const double *gx = grad_locals + (size_t)x * n3;
        for (int e = offsets[x]; e < offsets[x + 1]; ++e) {
            int y = sources[e];
            int t1 = tgt_ijk[3 * x + 0] - src_ijk[3 * y + 0];
            int t2 = tgt_ijk[3 * x + 1] - src_ijk[3 * y + 1];
            int t3 = tgt_ijk[3 * x + 2] - src_ijk[3 * y + 2];
            int m = abs(t1) > abs(t2) ? abs(t1) : abs(t2);
            m = m > abs(t3) ? m : abs(t3);
            if (m < 2 || m > 3) return -1 - (long)e;
            const double *K = ops + (size_t)((t1 + 3) + 7 * (t2 + 3) + 49 * (t3 + 3)) * n3 * n3;
            double *gy = grad_multipoles + (size_t)y * n3;
            for (int b = 0; b < n3; ++b) {
                double s = 0.0;
                for (int a = 0; a < n3; ++a) s += K[(size_t)a * n3 + b] * gx[a];
                gy[b] += s;
            }
        }
    }
    return 0;
}

/*
 * Direct sum, Eq. (1): f_i = sum_j K(x_i, y_j) w_j, skipping exact
 * coincidences x_i == y_j (the singular self-interaction).
 */
void oracle_direct_sum(int kind, double c, long ntgt, const double *x, long nsrc,
                       const double *y, const double *w, double *f)
{
    for (long i = 0; i < ntgt; ++i) {
        double s = 0.0;
        for (long j = 0; j < nsrc; ++j) {
            if (x[3 * i] == y[3 * j] && x[3 * i + 1] == y[3 * j + 1] && x[3 * i + 2] == y[3 * j + 2])
                continue;
            s += kernel_xy(kind, c, x + 3 * i, y + 3 * j) * w[j];
        }
        f[i] = s;
    }
}
