// Low-rank factors of the 16 unique operators by ACA followed by a truncated
// SVD (Sec. 4.1 and Sec. 5, after Bebendorf's partially pivoted adaptive cross
// approximation): the cheaper route to the factors K_p ~ U_p V_p^T of
// Eq. (20), with the same truncation criterion.  Everything runs on the
// device, one thread block per operator and step:
//
//  1. ACA: K ~ sum_k u_k v_k^T, stopped at |u_k| |v_k| <= eps_ACA |S_k|_F with
//     eps_ACA = 0.01 eps (pivot row 0 first; column of the largest residual;
//     next row of the largest |u_k| among unused rows; first index on ties).
//  2. QR of both factor sets by Gram-Schmidt with one re-orthogonalisation
//     pass (CGS2): U = Q_u R_u, V = Q_v R_v.
//  3. The k x k core C = R_u R_v^T.
//  4. Its SVD by one-sided Jacobi rotations (Hestenes' method; pairs in
//     round-robin order, one warp per pair): C Z = A with orthogonal columns,
//     C = W Sigma Z^T, sigma_j = |a_j|, W Sigma = A.
//  5. Truncation with the ops' criterion (Frobenius tail or spectral, as the
//     SVD path); the factors U_p = Q_u A_r (= U_K Sigma), V_p = Q_v Z_r, in the
//     layout of the SVD path.
#include <math.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "m2l_internal.cuh"

namespace m2l {
namespace {

constexpr int kAcaThreads = 256;
constexpr int kAcaWarps = kAcaThreads / 32;
constexpr double kAcaEpsFactor = 0.01;
constexpr int kJacobiSweeps = 60;

struct ArgMax {
    double v;
    int i;
};

// Largest value, first index on ties; every thread gets the result.
__device__ ArgMax block_argmax(double v, int i, ArgMax *red)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, v, o);
        const int oi = __shfl_down_sync(0xffffffffu, i, o);
        if (ov > v || (ov == v && oi < i)) {
            v = ov;
            i = oi;
        }
    }
    __syncthreads();
    if (lane == 0) red[w] = ArgMax{v, i};
    __syncthreads();
    ArgMax best = red[0];
    for (int q = 1; q < kAcaWarps; ++q)
        if (red[q].v > best.v || (red[q].v == best.v && red[q].i < best.i)) best = red[q];
    return best;
}

__device__ double block_sum(double v, double *red)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    for (int q = 0; q < kAcaWarps; ++q) s += red[q];
    return s;
}

__device__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// 1. ACA of K_p (row-major n x n); U[p][k][n], V[p][k][n] (term k contiguous).
__global__ void __launch_bounds__(kAcaThreads)
aca_kernel(int n, double eps_aca, const double *__restrict__ K64, double *__restrict__ U, double *__restrict__ V,
           int *__restrict__ kout)
{
    extern __shared__ double aca_sm[];
    double *r = aca_sm;                                        // [n] residual row
    double *dots = r + n;                                      // [2][n] u_l.u, v_l.v
    unsigned char *used = reinterpret_cast<unsigned char *>(dots + 2 * n);
    __shared__ ArgMax red_a[kAcaWarps];
    const int p = blockIdx.x;
    const double *K = K64 + (size_t)p * n * n;
    double *Up = U + (size_t)p * n * n;
    double *Vp = V + (size_t)p * n * n;
    for (int j = threadIdx.x; j < n; j += blockDim.x) used[j] = 0;
    __syncthreads();
    int i = 0, k = 0;
    double norm2 = 0.0;
    for (int it = 0; it < 2 * n && k < n; ++it) {
        if (threadIdx.x == 0) used[i] = 1;
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            double acc = K[(size_t)i * n + j];
            for (int l = 0; l < k; ++l) acc -= Up[(size_t)l * n + i] * Vp[(size_t)l * n + j];
            r[j] = acc;
        }
        __syncthreads();
        double best = -1.0;
        int bj = n;
        for (int j = threadIdx.x; j < n; j += blockDim.x)
            if (fabs(r[j]) > best) {
                best = fabs(r[j]);
                bj = j;
            }
        const ArgMax piv = block_argmax(best, bj, red_a);
        const int jp = piv.i;
        const double delta = r[jp];
        if (delta == 0.0) {   // exhausted row: the first unused row, no new term
            int first = n;
            for (int j = threadIdx.x; j < n; j += blockDim.x)
                if (!used[j] && j < first) first = j;
            const ArgMax f = block_argmax(-(double)first, first, red_a);
            if (f.i >= n) break;
            i = f.i;
            __syncthreads();
            continue;
        }
        double *uk = Up + (size_t)k * n;
        double *vk = Vp + (size_t)k * n;
        for (int j = threadIdx.x; j < n; j += blockDim.x) vk[j] = r[j] / delta;
        for (int q = threadIdx.x; q < n; q += blockDim.x) {
            double acc = K[(size_t)q * n + jp];
            for (int l = 0; l < k; ++l) acc -= Vp[(size_t)l * n + jp] * Up[(size_t)l * n + q];
            uk[q] = acc;
        }
        __syncthreads();
        // u_l.u_k and v_l.v_k, one warp per l
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int l = warp; l <= k; l += kAcaWarps) {
            double su = 0.0, sv = 0.0;
            for (int q = lane; q < n; q += 32) {
                su += Up[(size_t)l * n + q] * uk[q];
                sv += Vp[(size_t)l * n + q] * vk[q];
            }
            su = warp_sum(su);
            sv = warp_sum(sv);
            if (lane == 0) {
                dots[l] = su;
                dots[n + l] = sv;
            }
        }
        __syncthreads();
        double cross = 0.0;
        for (int l = 0; l < k; ++l) cross += dots[l] * dots[n + l];
        const double uu = dots[k], vv = dots[n + k];
        norm2 += 2.0 * cross + uu * vv;
        ++k;
        if (sqrt(uu * vv) <= eps_aca * sqrt(norm2)) break;
        double bu = -1.0;
        int bi = n;
        for (int q = threadIdx.x; q < n; q += blockDim.x)
            if (!used[q] && fabs(uk[q]) > bu) {
                bu = fabs(uk[q]);
                bi = q;
            }
        const ArgMax nx = block_argmax(bu, bi, red_a);
        if (nx.i >= n) break;
        i = nx.i;
        __syncthreads();
    }
    if (threadIdx.x == 0) kout[p] = k;
}

// 2. CGS2 QR in place of the k columns A[j][n] (j < k); R [k][k] row-major
//    (R[l][j], l <= j).  Block b: operator b / 2, factor b % 2 (U, V).
__global__ void __launch_bounds__(kAcaThreads)
cgs2_kernel(int n, int kmax, const int *__restrict__ kin, double *__restrict__ U, double *__restrict__ V,
            double *__restrict__ R)
{
    extern __shared__ double cg_sm[];   // [kmax] coefficients
    __shared__ double red_s[kAcaWarps];
    const int p = blockIdx.x >> 1, which = blockIdx.x & 1;
    const int k = kin[p];
    double *A = (which ? V : U) + (size_t)p * n * n;
    double *Rp = R + ((size_t)p * 2 + which) * kmax * kmax;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int idx = threadIdx.x; idx < kmax * kmax; idx += blockDim.x) Rp[idx] = 0.0;
    __syncthreads();
    for (int j = 0; j < k; ++j) {
        double *a = A + (size_t)j * n;
        for (int pass = 0; pass < 2; ++pass) {
            for (int l = warp; l < j; l += kAcaWarps) {
                double s = 0.0;
                for (int q = lane; q < n; q += 32) s += A[(size_t)l * n + q] * a[q];
                s = warp_sum(s);
                if (lane == 0) cg_sm[l] = s;
            }
            __syncthreads();
            for (int q = threadIdx.x; q < n; q += blockDim.x) {
                double acc = a[q];
                for (int l = 0; l < j; ++l) acc -= cg_sm[l] * A[(size_t)l * n + q];
                a[q] = acc;
            }
            if (threadIdx.x < j) Rp[(size_t)threadIdx.x * kmax + j] += cg_sm[threadIdx.x];
            for (int l = threadIdx.x + blockDim.x; l < j; l += blockDim.x) Rp[(size_t)l * kmax + j] += cg_sm[l];
            __syncthreads();
        }
        double s = 0.0;
        for (int q = threadIdx.x; q < n; q += blockDim.x) s += a[q] * a[q];
        const double nrm = sqrt(block_sum(s, red_s));
        for (int q = threadIdx.x; q < n; q += blockDim.x) a[q] = nrm > 0.0 ? a[q] / nrm : 0.0;
        if (threadIdx.x == 0) Rp[(size_t)j * kmax + j] = nrm;
        __syncthreads();
    }
}

// 3. C = R_u R_v^T, column-major [k][k] (column j at C + j * kmax); Z = I.
__global__ void core_kernel(int kmax, const int *__restrict__ kin, const double *__restrict__ R,
                            double *__restrict__ C, double *__restrict__ Z)
{
    const int p = blockIdx.y, k = kin[p];
    const double *Ru = R + (size_t)p * 2 * kmax * kmax;
    const double *Rv = Ru + (size_t)kmax * kmax;
    double *Cp = C + (size_t)p * kmax * kmax;
    double *Zp = Z + (size_t)p * kmax * kmax;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < kmax * kmax; idx += gridDim.x * blockDim.x) {
        const int j = idx / kmax, a = idx % kmax;   // column j, row a
        double s = 0.0;
        if (a < k && j < k)
            for (int l = 0; l < k; ++l) s += Ru[(size_t)a * kmax + l] * Rv[(size_t)j * kmax + l];
        Cp[idx] = s;
        Zp[idx] = (a == j) ? 1.0 : 0.0;
    }
}

// 4. One-sided Jacobi SVD of C (k x k, column-major), accumulating Z.  Sweeps
//    over all pairs in round-robin order (circle method: index kk - 1 fixed,
//    the others rotate), one warp per pair, until a sweep rotates nothing or
//    kJacobiSweeps sweeps have run.
__global__ void __launch_bounds__(kAcaThreads)
jacobi_kernel(int kmax, const int *__restrict__ kin, double *__restrict__ C, double *__restrict__ Z,
              int *__restrict__ sweeps_out)
{
    __shared__ int rotated;
    const int p = blockIdx.x, k = kin[p];
    double *Cp = C + (size_t)p * kmax * kmax;
    double *Zp = Z + (size_t)p * kmax * kmax;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kk = k + (k & 1);   // even count; index k is a dummy when k is odd
    int sweep = 0;
    for (; sweep < kJacobiSweeps && k > 1; ++sweep) {
        if (threadIdx.x == 0) rotated = 0;
        __syncthreads();
        for (int step = 0; step < kk - 1; ++step) {
            for (int pr = warp; pr < kk / 2; pr += kAcaWarps) {
                int a, b;
                if (pr == 0) {
                    a = kk - 1;
                    b = step;
                } else {
                    a = (step + pr) % (kk - 1);
                    b = (step - pr + (kk - 1)) % (kk - 1);
                }
                if (a >= k || b >= k) continue;
                if (a > b) {
                    const int tmp = a;
                    a = b;
                    b = tmp;
                }
                double *ca = Cp + (size_t)a * kmax, *cb = Cp + (size_t)b * kmax;
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int q = lane; q < k; q += 32) {
                    al += ca[q] * ca[q];
                    be += cb[q] * cb[q];
                    ga += ca[q] * cb[q];
                }
                al = warp_sum(al);
                be = warp_sum(be);
                ga = warp_sum(ga);
                if (fabs(ga) <= 1e-15 * sqrt(al * be) || ga == 0.0) continue;
                const double zeta = (be - al) / (2.0 * ga);
                const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
                double *za = Zp + (size_t)a * kmax, *zb = Zp + (size_t)b * kmax;
                for (int q = lane; q < k; q += 32) {
                    const double x = ca[q], y = cb[q];
                    ca[q] = c * x - s * y;
                    cb[q] = s * x + c * y;
                    const double zx = za[q], zy = zb[q];
                    za[q] = c * zx - s * zy;
                    zb[q] = s * zx + c * zy;
                }
                if (lane == 0) rotated = 1;
            }
            __syncthreads();
        }
        const int any = rotated;
        __syncthreads();
        if (!any) break;
    }
    if (threadIdx.x == 0) sweeps_out[p] = sweep;
}

__global__ void colnorm_kernel(int kmax, const int *__restrict__ kin, const double *__restrict__ C,
                               double *__restrict__ sig)
{
    const int p = blockIdx.x, k = kin[p];
    for (int j = threadIdx.x; j < kmax; j += blockDim.x) {
        double s = 0.0;
        if (j < k)
            for (int q = 0; q < k; ++q) s += C[(size_t)p * kmax * kmax + (size_t)j * kmax + q] *
                                             C[(size_t)p * kmax * kmax + (size_t)j * kmax + q];
        sig[(size_t)p * kmax + j] = sqrt(s);
    }
}

// 5. U64[p][row][q] = sum_l Q_u[l][row] A[order_q][l], V64[p][row][q] = sum_l Q_v[l][row] Z[order_q][l].
__global__ void aca_factors_kernel(int n, int kmax, int rmax, const int *__restrict__ kin,
                                   const int *__restrict__ ranks, const int *__restrict__ order,
                                   const double *__restrict__ Qu, const double *__restrict__ Qv,
                                   const double *__restrict__ C, const double *__restrict__ Z,
                                   double *__restrict__ U64, double *__restrict__ V64)
{
    const int p = blockIdx.y, k = kin[p], r = ranks[p];
    const double *qu = Qu + (size_t)p * n * n, *qv = Qv + (size_t)p * n * n;
    const double *Cp = C + (size_t)p * kmax * kmax, *Zp = Z + (size_t)p * kmax * kmax;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n * rmax; idx += gridDim.x * blockDim.x) {
        const int row = idx / rmax, q = idx % rmax;
        double u = 0.0, v = 0.0;
        if (q < r) {
            const int j = order[(size_t)p * kmax + q];
            for (int l = 0; l < k; ++l) {
                u += qu[(size_t)l * n + row] * Cp[(size_t)j * kmax + l];
                v += qv[(size_t)l * n + row] * Zp[(size_t)j * kmax + l];
            }
        }
        U64[((size_t)p * n + row) * rmax + q] = u;
        V64[((size_t)p * n + row) * rmax + q] = v;
    }
}

}  // namespace

m2l_status lowrank_factors_aca(m2l_ops *ops, int *aca_terms, int *jacobi_sweeps)
{
    const int n = ops->n3;
    const size_t nn = (size_t)n * n;
    DevBuf U, V, kd, R, C, Z, sw, sig, ord, dranks;
    ScratchGuard guard{&U, &V, &kd, &R, &C, &Z, &sw, &sig, &ord, &dranks};
    m2l_status st;
    if ((st = U.ensure(16 * nn * sizeof(double))) != M2L_OK) return st;
    if ((st = V.ensure(16 * nn * sizeof(double))) != M2L_OK) return st;
    if ((st = kd.ensure(16 * sizeof(int))) != M2L_OK) return st;
    if ((st = sw.ensure(16 * sizeof(int))) != M2L_OK) return st;
    const size_t smem = (size_t)3 * n * sizeof(double) + n;
    M2L_CUDA(cudaFuncSetAttribute(aca_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    aca_kernel<<<16, kAcaThreads, smem>>>(n, kAcaEpsFactor * ops->eps, ops->K64.as<double>(), U.as<double>(),
                                          V.as<double>(), kd.as<int>());
    M2L_LAUNCH_CHECK("aca_kernel");
    int hk[16];
    M2L_CUDA(cudaMemcpy(hk, kd.p, sizeof(hk), cudaMemcpyDeviceToHost));
    int kmax = 1;
    for (int p = 0; p < 16; ++p) kmax = std::max(kmax, hk[p]);
    if ((st = R.ensure((size_t)16 * 2 * kmax * kmax * sizeof(double))) != M2L_OK) return st;
    if ((st = C.ensure((size_t)16 * kmax * kmax * sizeof(double))) != M2L_OK) return st;
    if ((st = Z.ensure((size_t)16 * kmax * kmax * sizeof(double))) != M2L_OK) return st;
    if ((st = sig.ensure((size_t)16 * kmax * sizeof(double))) != M2L_OK) return st;
    if ((st = ord.ensure((size_t)16 * kmax * sizeof(int))) != M2L_OK) return st;
    if ((st = dranks.ensure(16 * sizeof(int))) != M2L_OK) return st;
    cgs2_kernel<<<32, kAcaThreads, (size_t)kmax * sizeof(double)>>>(n, kmax, kd.as<int>(), U.as<double>(),
                                                                     V.as<double>(), R.as<double>());
    M2L_LAUNCH_CHECK("cgs2_kernel");
    core_kernel<<<dim3((kmax * kmax + 255) / 256, 16), 256>>>(kmax, kd.as<int>(), R.as<double>(), C.as<double>(),
                                                             Z.as<double>());
    M2L_LAUNCH_CHECK("core_kernel");
    jacobi_kernel<<<16, kAcaThreads>>>(kmax, kd.as<int>(), C.as<double>(), Z.as<double>(), sw.as<int>());
    M2L_LAUNCH_CHECK("jacobi_kernel");
    colnorm_kernel<<<16, 256>>>(kmax, kd.as<int>(), C.as<double>(), sig.as<double>());
    M2L_LAUNCH_CHECK("colnorm_kernel");
    std::vector<double> hs((size_t)16 * kmax);
    int hsw[16];
    M2L_CUDA(cudaMemcpy(hs.data(), sig.p, hs.size() * sizeof(double), cudaMemcpyDeviceToHost));
    M2L_CUDA(cudaMemcpy(hsw, sw.p, sizeof(hsw), cudaMemcpyDeviceToHost));
    // truncation (the criterion of Eq. (20)) on the singular values in descending order
    std::vector<int> horder((size_t)16 * kmax, 0);
    int rmax = 1;
    for (int p = 0; p < 16; ++p) {
        if (hsw[p] >= kJacobiSweeps) {
            set_error("Jacobi SVD of operator %d did not converge in %d sweeps", p, kJacobiSweeps);
            return M2L_ECUDA;
        }
        const int k = hk[p];
        int *o = horder.data() + (size_t)p * kmax;
        std::iota(o, o + k, 0);
        const double *s = hs.data() + (size_t)p * kmax;
        std::stable_sort(o, o + k, [&](int a, int b) { return s[a] > s[b]; });
        std::vector<double> sorted(k);
        for (int i = 0; i < k; ++i) sorted[i] = s[o[i]];
        int r = truncation_rank(sorted.data(), k, ops->eps, ops->trunc);
        if (r < 1) r = 1;
        ops->ranks[p] = r;
        rmax = std::max(rmax, r);
        if (aca_terms) aca_terms[p] = k;
        if (jacobi_sweeps) jacobi_sweeps[p] = hsw[p];
    }
    ops->rmax = rmax;
    M2L_CUDA(cudaMemcpy(ord.p, horder.data(), horder.size() * sizeof(int), cudaMemcpyHostToDevice));
    M2L_CUDA(cudaMemcpy(dranks.p, ops->ranks, 16 * sizeof(int), cudaMemcpyHostToDevice));
    if ((st = ops->U64.ensure(16 * (size_t)n * rmax * sizeof(double))) != M2L_OK) return st;
    if ((st = ops->V64.ensure(16 * (size_t)n * rmax * sizeof(double))) != M2L_OK) return st;
    aca_factors_kernel<<<dim3((n * rmax + 255) / 256, 16), 256>>>(n, kmax, rmax, kd.as<int>(), dranks.as<int>(),
                                                                  ord.as<int>(), U.as<double>(), V.as<double>(),
                                                                  C.as<double>(), Z.as<double>(),
                                                                  ops->U64.as<double>(), ops->V64.as<double>());
    M2L_LAUNCH_CHECK("aca_factors_kernel");
    M2L_CUDA(cudaDeviceSynchronize());
    return M2L_OK;
}

}  // namespace m2l
