// Singular value decompositions of the precompute, on the device, in FP64:
// one-sided Jacobi rotations (Hestenes' method), batched over matrices.
//
// For a column-major m x n matrix A (m >= n) the method applies plane
// rotations to pairs of columns until every pair is orthogonal to working
// accuracy: A V = W Sigma with V orthogonal, the columns of W Sigma mutually
// orthogonal, sigma_j = |a_j|.  So A = W Sigma V^T: the columns of the
// rotated A are the left singular vectors scaled by the singular values (what
// the low-rank factors U_t = U_r Sigma_r of Eq. (20) store), V holds the right
// singular vectors.  Rotations are computed from the columns themselves
// (not from a Gram matrix), so small singular values keep an absolute error of
// a few units of roundoff of |A|: the truncation criteria below act on values
// down to eps |A| with eps >= 1e-12.
//
// Order of the pairs: the round-robin (circle) method: n - 1 rounds of n / 2
// disjoint pairs each (n rounded up to even; the extra index is a dummy), so
// all pairs of a round rotate concurrently.  One launch per round; one warp
// per (matrix, pair) when the columns are short, one 256-thread block when
// they are long.  A sweep ends without rotations, and the matrix has
// converged, when every pair satisfies |a_i . a_j| <= tol |a_i| |a_j|
// (Demmel and Veselic's stopping rule) with tol = 1e-12: safely above the
// rounding noise of the dot products, and far below what changes a singular
// value the truncation sees (a pair orthogonal to tol perturbs the column
// norms by O(tol^2)).  The smooth kernels' operators have strongly graded
// spectra and nearly parallel columns: taken as they are they need 25-50
// sweeps (ell 4-8), so the sweep limit is 100; step a1 hands over the R factor
// of a pivoted QR instead, which converges in 7-11.
#include <math.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "m2l_internal.cuh"

namespace m2l {
namespace {

constexpr int kSvdThreads = 256;
constexpr int kSvdMaxSweeps = 100;
constexpr int kLongColumn = 4096;   // columns longer than this get a whole block per pair
constexpr double kSvdTol = 1e-12;   // relative orthogonality of converged column pairs
constexpr double kClusterGap = 1e-12;   // singular values closer than this times s_1 form one cluster

__device__ __forceinline__ double warp_sum_d(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// The two column indices of pair `pr` in round `step` of the circle method over
// kk (even) indices: kk - 1 stays fixed, the others rotate.
__device__ __forceinline__ void round_pair(int kk, int step, int pr, int &a, int &b)
{
    if (pr == 0) {
        a = kk - 1;
        b = step;
    } else {
        a = (step + pr) % (kk - 1);
        b = (step - pr + (kk - 1)) % (kk - 1);
    }
    if (a > b) {
        const int t = a;
        a = b;
        b = t;
    }
}

// Rotation (c, s) that makes c a - s b and s a + c b orthogonal, from
// alpha = |a|^2, beta = |b|^2, gamma = a . b: the smaller root t of
// t^2 + 2 zeta t - 1 = 0, zeta = (beta - alpha) / (2 gamma) (Rutishauser).
__device__ __forceinline__ void rotation(double al, double be, double ga, double &c, double &s)
{
    const double zeta = (be - al) / (2.0 * ga);
    double t;
    if (fabs(zeta) > 1e150)
        t = 0.5 / zeta;
    else
        t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
    c = 1.0 / sqrt(1.0 + t * t);
    s = c * t;
}

// One round for every (matrix, pair); G threads per pair (32: a warp, or
// kSvdThreads: the block).  A [nb][n][m] column-major, V [nb][n][n] or null.
template <int G>
__global__ void __launch_bounds__(kSvdThreads)
jacobi_round_kernel(double *__restrict__ A, double *__restrict__ V, int m, int n, int kk, int step, int nb,
                    double tol, const int *__restrict__ done, int *__restrict__ rotated)
{
    constexpr int kPerBlock = kSvdThreads / G;
    const int sub = threadIdx.x / G, lane = threadIdx.x % G;
    const long item = (long)blockIdx.x * kPerBlock + sub;
    const int npair = kk / 2;
    if (item >= (long)nb * npair) return;   // uniform per pair group
    const int mat = (int)(item / npair), pr = (int)(item % npair);
    if (done[mat]) return;
    int a, b;
    round_pair(kk, step, pr, a, b);
    if (b >= n) return;   // the dummy index of an odd n
    double *ca = A + ((size_t)mat * n + a) * m, *cb = A + ((size_t)mat * n + b) * m;
    double al = 0.0, be = 0.0, ga = 0.0;
    for (int q = lane; q < m; q += G) {
        const double x = ca[q], y = cb[q];
        al += x * x;
        be += y * y;
        ga += x * y;
    }
    al = warp_sum_d(al);
    be = warp_sum_d(be);
    ga = warp_sum_d(ga);
    if (G > 32) {
        __shared__ double red[kSvdThreads / 32][3];
        const int w = threadIdx.x >> 5;
        if ((threadIdx.x & 31) == 0) {
            red[w][0] = al;
            red[w][1] = be;
            red[w][2] = ga;
        }
        __syncthreads();
        al = be = ga = 0.0;
        for (int q = 0; q < kSvdThreads / 32; ++q) {
            al += red[q][0];
            be += red[q][1];
            ga += red[q][2];
        }
    }
    if (ga == 0.0 || fabs(ga) <= tol * sqrt(al) * sqrt(be)) return;
    double c, s;
    rotation(al, be, ga, c, s);
    for (int q = lane; q < m; q += G) {
        const double x = ca[q], y = cb[q];
        ca[q] = c * x - s * y;
        cb[q] = s * x + c * y;
    }
    if (V) {
        double *va = V + ((size_t)mat * n + a) * n, *vb = V + ((size_t)mat * n + b) * n;
        for (int q = lane; q < n; q += G) {
            const double x = va[q], y = vb[q];
            va[q] = c * x - s * y;
            vb[q] = s * x + c * y;
        }
    }
    if (lane == 0) rotated[mat] = 1;
}

__global__ void identity_kernel(double *__restrict__ V, int n, int nb)
{
    const long total = (long)nb * n * n;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        const long r = i % ((long)n * n);
        V[i] = (r / n == r % n) ? 1.0 : 0.0;
    }
}

// sigma[mat][j] = |a_j|, one warp per column.
__global__ void column_norms_kernel(const double *__restrict__ A, int m, int n, int nb, double *__restrict__ sigma)
{
    const long col = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (col >= (long)nb * n) return;
    const double *c = A + (size_t)col * m;
    double s = 0.0;
    for (int q = lane; q < m; q += 32) s += c[q] * c[q];
    s = warp_sum_d(s);
    if (lane == 0) sigma[col] = sqrt(s);
}

int grid_of(long n, int threads)
{
    const long b = (n + threads - 1) / threads;
    return (int)std::min<long>(std::max<long>(b, 1), 1L << 20);
}

}  // namespace

m2l_status jacobi_svd(double *A, int m, int n, int nb, double *V, double *sigma, int *sweeps, cudaStream_t s)
{
    if (m < n || n < 1 || nb < 1) {
        set_error("jacobi_svd: need m >= n >= 1 and at least one matrix");
        return M2L_EINVAL;
    }
    DevBuf dflags;
    ScratchGuard guard{&dflags};
    m2l_status st = dflags.ensure(2 * (size_t)nb * sizeof(int));
    if (st != M2L_OK) return st;
    int *done = dflags.as<int>(), *rotated = dflags.as<int>() + nb;
    M2L_CUDA(cudaMemsetAsync(done, 0, (size_t)nb * sizeof(int), s));
    if (V) {
        identity_kernel<<<grid_of((long)nb * n * n, 256), 256, 0, s>>>(V, n, nb);
        M2L_LAUNCH_CHECK("identity_kernel");
    }
    const int kk = n + (n & 1);
    const double tol = kSvdTol;
    const long items = (long)nb * (kk / 2);
    const bool long_cols = m > kLongColumn;
    std::vector<int> hrot(nb), hdone(nb, 0);
    std::vector<int> hsweeps(nb, kSvdMaxSweeps + 1);
    int left = nb;
    for (int sweep = 0; sweep < kSvdMaxSweeps && left > 0 && n > 1; ++sweep) {
        M2L_CUDA(cudaMemsetAsync(rotated, 0, (size_t)nb * sizeof(int), s));
        for (int step = 0; step < kk - 1; ++step) {
            if (long_cols)
                jacobi_round_kernel<kSvdThreads><<<(unsigned)items, kSvdThreads, 0, s>>>(A, V, m, n, kk, step, nb,
                                                                                       tol, done, rotated);
            else
                jacobi_round_kernel<32><<<grid_of(items, kSvdThreads / 32), kSvdThreads, 0, s>>>(
                    A, V, m, n, kk, step, nb, tol, done, rotated);
            M2L_LAUNCH_CHECK("jacobi_round_kernel");
        }
        M2L_CUDA(cudaMemcpyAsync(hrot.data(), rotated, (size_t)nb * sizeof(int), cudaMemcpyDeviceToHost, s));
        M2L_CUDA(cudaStreamSynchronize(s));
        for (int i = 0; i < nb; ++i)
            if (!hdone[i] && !hrot[i]) {
                hdone[i] = 1;
                hsweeps[i] = sweep + 1;
                --left;
            }
        M2L_CUDA(cudaMemcpyAsync(done, hdone.data(), (size_t)nb * sizeof(int), cudaMemcpyHostToDevice, s));
    }
    if (n == 1) {
        left = 0;
        std::fill(hsweeps.begin(), hsweeps.end(), 0);
    }
    column_norms_kernel<<<grid_of((long)nb * n * 32, 256), 256, 0, s>>>(A, m, n, nb, sigma);
    M2L_LAUNCH_CHECK("column_norms_kernel");
    M2L_CUDA(cudaStreamSynchronize(s));
    if (sweeps) std::copy(hsweeps.begin(), hsweeps.end(), sweeps);
    if (left > 0) {
        set_error("Jacobi SVD: %d of %d matrices did not converge in %d sweeps", left, nb, kSvdMaxSweeps);
        return M2L_ECUDA;
    }
    return M2L_OK;
}

void order_descending(const double *sig, int n, int *order)
{
    std::iota(order, order + n, 0);
    std::stable_sort(order, order + n, [&](int a, int b) { return sig[a] > sig[b]; });
}

int truncation_rank(const double *s, int n, double eps, int trunc)
{
    if (eps <= 0.0 || n <= 0) return n;
    int r = n;
    if (trunc == M2L_TRUNC_SPECTRAL) {
        r = 0;
        while (r < n && s[r] > eps * s[0]) ++r;
    } else {
        // Frobenius tail: tail[r] = sum_{i >= r} s_i^2, accumulated from the smallest up
        std::vector<double> tail(n + 1, 0.0);
        for (int i = n - 1; i >= 0; --i) tail[i] = tail[i + 1] + s[i] * s[i];
        const double bound = eps * eps * tail[0];
        for (int k = 0; k <= n; ++k)
            if (tail[k] <= bound) {
                r = k;
                break;
            }
    }
    // the truncated SVD is unique only when s_r > s_{r+1}: a cut inside a cluster
    // of equal values (an operator's symmetry makes pairs) moves past the cluster
    while (r > 0 && r < n && s[r - 1] - s[r] <= kClusterGap * s[0]) ++r;
    return r;
}

}  // namespace m2l
