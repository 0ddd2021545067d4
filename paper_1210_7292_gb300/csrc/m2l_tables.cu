// Precompute of the 16 unique M2L operators and of the symmetry tables
// (steps a1 and a2), all on the device.
//
//  * T_sym = {t in T : t1 >= t2 >= t3 >= 0} (Eqs. (23)-(24)), 16 vectors for
//    the bbFMM, indexed in lexicographic ascending order.
//  * K_p[m(alpha)][n(beta)] = K(xbar_alpha - ybar_beta) (Eq. (15)) with
//    xbar_alpha - ybar_beta = w (t_p + (xi_alpha - xi_beta) / 2) for a pair of
//    cells of width w whose centres differ by w t_p.
//  * sigma_g(j) = m(pi(m^{-1}(j))), pi = pi^D o pi^A (Eqs. (26)-(29)), one
//    table per signed axis permutation g = 8 * perm_id + flip_mask.
//  * t -> (p(t), g(t)) for the 343 vectors of [-3, 3]^3.
#include <algorithm>
#include <vector>

#include "m2l_internal.cuh"

namespace m2l {
namespace {

// The six axis orders in lexicographic order.
__device__ __constant__ int c_perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

__global__ void tables_kernel(int ell, int16_t *__restrict__ sigma, uint16_t *__restrict__ lut,
                              int *__restrict__ tsym)
{
    __shared__ int s_tsym[16][3];
    if (threadIdx.x == 0) {
        int n = 0;
        for (int t1 = 2; t1 <= 3; ++t1)
            for (int t2 = 0; t2 <= t1; ++t2)
                for (int t3 = 0; t3 <= t2; ++t3) {
                    s_tsym[n][0] = t1;
                    s_tsym[n][1] = t2;
                    s_tsym[n][2] = t3;
                    ++n;
                }
    }
    __syncthreads();
    if (threadIdx.x < 48) tsym[threadIdx.x] = (&s_tsym[0][0])[threadIdx.x];

    const int n3 = ell * ell * ell;
    for (int idx = threadIdx.x; idx < 48 * n3; idx += blockDim.x) {
        const int g = idx / n3, j = idx % n3;
        const int flip = g & 7;
        const int *ord = c_perm[g >> 3];
        int a[3] = {j % ell, (j / ell) % ell, j / (ell * ell)};
        for (int i = 0; i < 3; ++i)
            if ((flip >> i) & 1) a[i] = ell - 1 - a[i];              // pi^A, Eq. (26)
        sigma[idx] = (int16_t)(a[ord[0]] + ell * a[ord[1]] + ell * ell * a[ord[2]]);  // pi^D, Eq. (27)
    }
    for (int s = threadIdx.x; s < 343; s += blockDim.x) {
        const int t[3] = {s % 7 - 3, (s / 7) % 7 - 3, s / 49 - 3};
        const int at[3] = {abs(t[0]), abs(t[1]), abs(t[2])};
        const int mx = max(at[0], max(at[1], at[2]));
        if (mx <= 1) {
            lut[s] = 0xFFFF;
            continue;
        }
        int flip = 0;
        for (int i = 0; i < 3; ++i)
            if (t[i] < 0) flip |= 1 << i;
        // axis order by |t_i| descending, stable (lower axis first on ties)
        int o[3] = {0, 1, 2};
        for (int i = 1; i < 3; ++i)
            for (int k = i; k > 0 && at[o[k]] > at[o[k - 1]]; --k) {
                int tmp = o[k];
                o[k] = o[k - 1];
                o[k - 1] = tmp;
            }
        const int perm_id = 2 * o[0] + (o[1] > o[2] ? 1 : 0);
        const int tp[3] = {at[o[0]], at[o[1]], at[o[2]]};
        int p = -1;
        for (int q = 0; q < 16; ++q)
            if (s_tsym[q][0] == tp[0] && s_tsym[q][1] == tp[1] && s_tsym[q][2] == tp[2]) p = q;
        lut[s] = (uint16_t)(p | ((8 * perm_id + flip) << 8));
    }
}

__device__ __forceinline__ double kernel_r(int kind, double c, double r)
{
    if (kind == 0) return 1.0 / r;
    if (kind == 1) {
        const double r2 = r * r;
        return 1.0 / (r2 * r2);
    }
    return 1.0 / sqrt(r * r + c * c);
}

__global__ void assemble_kernel(int ell, int kind, double c, double w, const int *__restrict__ tsym,
                                double *__restrict__ K)
{
    // Chebyshev roots ascending, -cos((2k+1) pi / (2 ell)), once per block
    __shared__ double xi[kMaxEll];
    if (threadIdx.x < ell) xi[threadIdx.x] = -cospi((2.0 * threadIdx.x + 1.0) / (2.0 * ell));
    __syncthreads();
    const int n3 = ell * ell * ell;
    const long total = 16L * n3 * n3;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total;
         idx += (long)gridDim.x * blockDim.x) {
        const int p = (int)(idx / ((long)n3 * n3));
        const int rem = (int)(idx % ((long)n3 * n3));
        const int a = rem / n3, b = rem % n3;
        const int ai[3] = {a % ell, (a / ell) % ell, a / (ell * ell)};
        const int bi[3] = {b % ell, (b / ell) % ell, b / (ell * ell)};
        double r2 = 0.0;
        for (int i = 0; i < 3; ++i) {
            const double d = w * ((double)tsym[3 * p + i] + 0.5 * (xi[ai[i]] - xi[bi[i]]));
            r2 += d * d;
        }
        K[idx] = kernel_r(kind, c, sqrt(r2));
    }
}

// U_p = U_K Sigma (first r_p columns), V_p = V_K, both [n3][rmax] row-major,
// from the column-major SVD M = U_M S V_M^T of M = K_p^T (so U_K = V_M, V_K = U_M).
// ---------------------------------------------------------------- step a1's SVD
// The truncated SVD of each K_p (Eq. (20)) as a QR-preconditioned one-sided
// Jacobi SVD (Drmac and Veselic): M = K_p^T (the row-major K_p read column-major)
// is factored M P = Q R by Householder QR with column pivoting, R^T by
// one-sided Jacobi, R^T V_J = W Sigma.  Then K_p = P R^T Q^T = (P W Sigma)(Q V_J)^T:
// U_p = (P W Sigma)_r, V_p = (Q V_J)_r.  The pivoting concentrates the norms on
// R's leading rows, so Jacobi on R^T converges in a handful of sweeps instead
// of the dozens it takes on K_p itself.
constexpr int kQrThreads = 512;
constexpr int kQrWarps = kQrThreads / 32;

__device__ __forceinline__ double qr_warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One block per matrix: A [p] column-major n x n (in place: R on and above the
// diagonal, the Householder vectors' tails below it), vhead [p][n] their first
// entries, beta [p][n] = 2 / (v^T v) (0 for a zero column), perm [p][n]: column k
// of M P is column perm[k] of M.
__global__ void __launch_bounds__(kQrThreads)
qrcp_kernel(int n, double *__restrict__ A, double *__restrict__ vhead, double *__restrict__ beta,
            int *__restrict__ perm)
{
    extern __shared__ double qr_smem[];
    double *cn = qr_smem;                              // [n] column norms^2 of the trailing block
    __shared__ double s_val[kQrWarps];
    __shared__ int s_idx[kQrWarps];
    __shared__ double s_alpha, s_v0, s_beta;
    __shared__ int s_piv;
    const int p = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *M = A + (size_t)p * n * n;
    int *pm = perm + (size_t)p * n;
    for (int j = threadIdx.x; j < n; j += blockDim.x) pm[j] = j;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        // 1. norms^2 of columns k..n-1 over rows k..n-1
        for (int j = k + warp; j < n; j += kQrWarps) {
            const double *c = M + (size_t)j * n;
            double s2 = 0.0;
            for (int i = k + lane; i < n; i += 32) s2 += c[i] * c[i];
            s2 = qr_warp_sum(s2);
            if (lane == 0) cn[j] = s2;
        }
        __syncthreads();
        // 2. the pivot: the largest norm, the first column on ties
        double bv = -1.0;
        int bi = n;
        for (int j = k + threadIdx.x; j < n; j += blockDim.x)
            if (cn[j] > bv) {
                bv = cn[j];
                bi = j;
            }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_down_sync(0xffffffffu, bv, o);
            const int oi = __shfl_down_sync(0xffffffffu, bi, o);
            if (ov > bv || (ov == bv && oi < bi)) {
                bv = ov;
                bi = oi;
            }
        }
        if (lane == 0) {
            s_val[warp] = bv;
            s_idx[warp] = bi;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double v = s_val[0];
            int ix = s_idx[0];
            for (int w = 1; w < kQrWarps; ++w)
                if (s_val[w] > v || (s_val[w] == v && s_idx[w] < ix)) {
                    v = s_val[w];
                    ix = s_idx[w];
                }
            s_piv = ix < n ? ix : k;
        }
        __syncthreads();
        const int piv = s_piv;
        // 3. swap columns k and piv (all rows: the rows above k hold R)
        if (piv != k) {
            double *ck = M + (size_t)k * n, *cp = M + (size_t)piv * n;
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const double t = ck[i];
                ck[i] = cp[i];
                cp[i] = t;
            }
            if (threadIdx.x == 0) {
                const int t = pm[k];
                pm[k] = pm[piv];
                pm[piv] = t;
                const double tn = cn[k];
                cn[k] = cn[piv];
                cn[piv] = tn;
            }
        }
        __syncthreads();
        // 4. the Householder reflector of column k: H x = alpha e_k
        if (threadIdx.x == 0) {
            const double x0 = M[(size_t)k * n + k];
            const double nx = sqrt(cn[k]);
            const double alpha = x0 >= 0.0 ? -nx : nx;
            const double v0 = x0 - alpha;
            const double vtv = cn[k] - x0 * x0 + v0 * v0;
            s_alpha = alpha;
            s_v0 = v0;
            s_beta = vtv > 0.0 ? 2.0 / vtv : 0.0;
        }
        __syncthreads();
        const double v0 = s_v0, bk = s_beta;
        const double *vk = M + (size_t)k * n;   // tail entries vk[i], i > k
        // 5. apply it to the columns k+1..n-1
        for (int j = k + 1 + warp; j < n; j += kQrWarps) {
            double *c = M + (size_t)j * n;
            double d = 0.0;
            for (int i = k + 1 + lane; i < n; i += 32) d += vk[i] * c[i];
            d = qr_warp_sum(d) + v0 * c[k];
            const double w = bk * d;
            __syncwarp();   // every lane has read c[k]
            if (lane == 0) c[k] -= w * v0;
            for (int i = k + 1 + lane; i < n; i += 32) c[i] -= w * vk[i];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            M[(size_t)k * n + k] = s_alpha;
            vhead[(size_t)p * n + k] = v0;
            beta[(size_t)p * n + k] = bk;
        }
        __syncthreads();
    }
}

// B [p] column-major = R^T: column j holds row j of R (R(j, i), i >= j), zeros above.
__global__ void r_transpose_kernel(int n, const double *__restrict__ A, double *__restrict__ B)
{
    const long nn = (long)n * n, total = 16 * nn;
    for (long x = blockIdx.x * (long)blockDim.x + threadIdx.x; x < total; x += (long)gridDim.x * blockDim.x) {
        const long p = x / nn, r = x % nn, j = r / n, i = r % n;
        B[x] = i >= j ? A[p * nn + i * n + j] : 0.0;
    }
}

// U[p][perm[k]][q] = (W Sigma)(k, order_q) for q < r_p, zero beyond.
__global__ void extract_u_kernel(int n3, int rmax, const int *__restrict__ ranks, const int *__restrict__ order,
                                 const int *__restrict__ perm, const double *__restrict__ B, double *__restrict__ U)
{
    const int p = blockIdx.y;
    const int r = ranks[p];
    const long nn = (long)n3 * n3;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n3 * rmax; idx += gridDim.x * blockDim.x) {
        const int k = idx / rmax, q = idx % rmax;
        const double u = q < r ? B[p * nn + (long)order[p * n3 + q] * n3 + k] : 0.0;
        U[((long)p * n3 + perm[p * n3 + k]) * rmax + q] = u;
    }
}

// V[p][:, q] = Q V_J[:, order_q] = H_0 H_1 ... H_{n-1} V_J[:, order_q] for q < r_p, zero
// beyond; one warp per column, the column in shared memory.
constexpr int kQWarps = 8;
__global__ void __launch_bounds__(kQWarps * 32)
apply_q_kernel(int n, int rmax, const int *__restrict__ ranks, const int *__restrict__ order,
               const double *__restrict__ A, const double *__restrict__ vhead, const double *__restrict__ beta,
               const double *__restrict__ VJ, double *__restrict__ V)
{
    extern __shared__ double q_smem[];
    const int p = blockIdx.y, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = blockIdx.x * kQWarps + warp;
    if (q >= rmax) return;
    const long nn = (long)n * n;
    double *x = q_smem + (size_t)warp * n;
    if (q >= ranks[p]) {
        for (int i = lane; i < n; i += 32) V[((long)p * n + i) * rmax + q] = 0.0;
        return;
    }
    const double *src = VJ + p * nn + (long)order[p * n + q] * n;
    for (int i = lane; i < n; i += 32) x[i] = src[i];
    __syncwarp();
    const double *M = A + p * nn;
    for (int k = n - 1; k >= 0; --k) {
        const double bk = beta[(long)p * n + k];
        if (bk == 0.0) continue;
        const double v0 = vhead[(long)p * n + k];
        const double *vk = M + (long)k * n;
        double d = 0.0;
        for (int i = k + 1 + lane; i < n; i += 32) d += vk[i] * x[i];
        d = qr_warp_sum(d) + v0 * x[k];
        const double w = bk * d;
        __syncwarp();
        if (lane == 0) x[k] -= w * v0;
        for (int i = k + 1 + lane; i < n; i += 32) x[i] -= w * vk[i];
        __syncwarp();
    }
    for (int i = lane; i < n; i += 32) V[((long)p * n + i) * rmax + q] = x[i];
}

template <typename T>
__global__ void transpose_pad_kernel(int n3, int kpad, int mpad, const double *__restrict__ K,
                                     T *__restrict__ KT)
{
    // KT[p][k][a] = K[p][a][k], zero outside [0, n3)^2
    const long per = (long)kpad * mpad;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < 16 * per;
         idx += (long)gridDim.x * blockDim.x) {
        const int p = (int)(idx / per);
        const int rem = (int)(idx % per);
        const int k = rem / mpad, a = rem % mpad;
        double v = 0.0;
        if (k < n3 && a < n3) v = K[(long)p * n3 * n3 + (long)a * n3 + k];
        KT[idx] = (T)v;
    }
}

// Low-rank SIMT layouts: VT[p][k][r] (k < kpad, r < rpad): the columns of V as
// rows over the node index; UT[p][r][a] (r < rpad, a < mpad).
template <typename T>
__global__ void lowrank_layout_kernel(int n3, int rmax, int kpad, int mpad, int rpad,
                                      const double *__restrict__ U, const double *__restrict__ V,
                                      T *__restrict__ VT, T *__restrict__ UT)
{
    const int p = blockIdx.y;
    const long nv = (long)kpad * rpad, nu = (long)rpad * mpad;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < nv + nu;
         idx += (long)gridDim.x * blockDim.x) {
        if (idx < nv) {
            const int k = (int)(idx / rpad), r = (int)(idx % rpad);
            double v = (k < n3 && r < rmax) ? V[((long)p * n3 + k) * rmax + r] : 0.0;
            VT[p * nv + idx] = (T)v;
        } else {
            const long j = idx - nv;
            const int r = (int)(j / mpad), a = (int)(j % mpad);
            double u = (a < n3 && r < rmax) ? U[((long)p * n3 + a) * rmax + r] : 0.0;
            UT[p * nu + j] = (T)u;
        }
    }
}

}  // namespace

m2l_status build_tables(m2l_ops *ops, cudaStream_t s)
{
    tables_kernel<<<1, 256, 0, s>>>(ops->ell, ops->sigma.as<int16_t>(), ops->lut.as<uint16_t>(),
                                    ops->tsym.as<int>());
    M2L_LAUNCH_CHECK("tables_kernel");
    return M2L_OK;
}

m2l_status assemble_operators(m2l_ops *ops, cudaStream_t s)
{
    const long total = 16L * ops->n3 * ops->n3;
    const int threads = 256;
    const int blocks = (int)((total + threads - 1) / threads);
    assemble_kernel<<<blocks, threads, 0, s>>>(ops->ell, ops->kind, ops->c, ops->ref_width,
                                               ops->tsym.as<int>(), ops->K64.as<double>());
    M2L_LAUNCH_CHECK("assemble_kernel");
    return M2L_OK;
}

// Step a1's truncated SVD of the 16 operators (Eq. (20)), QR-preconditioned
// one-sided Jacobi on the device; ranks by the ops' truncation criterion.
m2l_status lowrank_factors(m2l_ops *ops)
{
    const int n = ops->n3;
    const size_t nn = (size_t)n * n;
    DevBuf A, B, S, VJ, vh, bt, pm, dord, dranks;
    ScratchGuard guard{&A, &B, &S, &VJ, &vh, &bt, &pm, &dord, &dranks};
    m2l_status st;
    if ((st = A.ensure(16 * nn * sizeof(double))) != M2L_OK) return st;
    if ((st = B.ensure(16 * nn * sizeof(double))) != M2L_OK) return st;
    if ((st = VJ.ensure(16 * nn * sizeof(double))) != M2L_OK) return st;
    if ((st = S.ensure(16 * (size_t)n * sizeof(double))) != M2L_OK) return st;
    if ((st = vh.ensure(16 * (size_t)n * sizeof(double))) != M2L_OK) return st;
    if ((st = bt.ensure(16 * (size_t)n * sizeof(double))) != M2L_OK) return st;
    if ((st = pm.ensure(16 * (size_t)n * sizeof(int))) != M2L_OK) return st;
    if ((st = dord.ensure(16 * (size_t)n * sizeof(int))) != M2L_OK) return st;
    if ((st = dranks.ensure(16 * sizeof(int))) != M2L_OK) return st;
    // M = K_p^T column-major is K_p's row-major memory
    M2L_CUDA(cudaMemcpy(A.p, ops->K64.p, 16 * nn * sizeof(double), cudaMemcpyDeviceToDevice));
    qrcp_kernel<<<16, kQrThreads, (size_t)n * sizeof(double)>>>(n, A.as<double>(), vh.as<double>(), bt.as<double>(),
                                                                pm.as<int>());
    M2L_LAUNCH_CHECK("qrcp_kernel");
    r_transpose_kernel<<<(int)std::min<size_t>((16 * nn + 255) / 256, 65535), 256>>>(n, A.as<double>(),
                                                                                    B.as<double>());
    M2L_LAUNCH_CHECK("r_transpose_kernel");
    if ((st = jacobi_svd(B.as<double>(), n, n, 16, VJ.as<double>(), S.as<double>(), ops->jacobi_sweeps, 0)) != M2L_OK)
        return st;
    std::vector<double> hS(16 * (size_t)n), sorted(n);
    std::vector<int> hord(16 * (size_t)n);
    M2L_CUDA(cudaMemcpy(hS.data(), S.p, hS.size() * sizeof(double), cudaMemcpyDeviceToHost));
    int rmax = 1;
    for (int p = 0; p < 16; ++p) {
        int *o = hord.data() + (size_t)p * n;
        order_descending(hS.data() + (size_t)p * n, n, o);
        for (int i = 0; i < n; ++i) sorted[i] = hS[(size_t)p * n + o[i]];
        int r = truncation_rank(sorted.data(), n, ops->eps, ops->trunc);
        if (r < 1) r = 1;
        ops->ranks[p] = r;
        if (r > rmax) rmax = r;
    }
    ops->rmax = rmax;
    if ((st = ops->U64.ensure(16 * (size_t)n * rmax * sizeof(double))) != M2L_OK) return st;
    if ((st = ops->V64.ensure(16 * (size_t)n * rmax * sizeof(double))) != M2L_OK) return st;
    M2L_CUDA(cudaMemcpy(dranks.p, ops->ranks, 16 * sizeof(int), cudaMemcpyHostToDevice));
    M2L_CUDA(cudaMemcpy(dord.p, hord.data(), hord.size() * sizeof(int), cudaMemcpyHostToDevice));
    extract_u_kernel<<<dim3((n * rmax + 255) / 256, 16), 256>>>(n, rmax, dranks.as<int>(), dord.as<int>(),
                                                                  pm.as<int>(), B.as<double>(), ops->U64.as<double>());
    M2L_LAUNCH_CHECK("extract_u_kernel");
    apply_q_kernel<<<dim3((rmax + kQWarps - 1) / kQWarps, 16), kQWarps * 32, (size_t)kQWarps * n * sizeof(double)>>>(
        n, rmax, dranks.as<int>(), dord.as<int>(), A.as<double>(), vh.as<double>(), bt.as<double>(),
        VJ.as<double>(), ops->V64.as<double>());
    M2L_LAUNCH_CHECK("apply_q_kernel");
    M2L_CUDA(cudaDeviceSynchronize());
    return M2L_OK;
}

// Padded sizes shared with the SIMT kernels.
int simt_kpad(int n3) { return (n3 + 31) / 32 * 32; }
int simt_mpad(int n3) { return (n3 + 127) / 128 * 128; }
int simt_rpad(int r) { return (r + 31) / 32 * 32; }

m2l_status prepare_simt_layout(const m2l_ops *ops, int fp64, cudaStream_t s)
{
    m2l_ops *o = const_cast<m2l_ops *>(ops);
    Layout &L = fp64 ? (ops->eps > 0 ? o->lr64 : o->simt64) : (ops->eps > 0 ? o->lr32 : o->simt32);
    if (L.ready) return M2L_OK;
    const int n3 = ops->n3, kpad = simt_kpad(n3), mpad = simt_mpad(n3);
    const size_t esz = fp64 ? sizeof(double) : sizeof(float);
    m2l_status st;
    if (ops->eps <= 0) {
        const size_t total = 16 * (size_t)kpad * mpad;
        if ((st = L.a.ensure(total * esz)) != M2L_OK) return st;
        const int blocks = (int)((total + 255) / 256);
        if (fp64)
            transpose_pad_kernel<double><<<blocks, 256, 0, s>>>(n3, kpad, mpad, ops->K64.as<double>(),
                                                                L.a.as<double>());
        else
            transpose_pad_kernel<float><<<blocks, 256, 0, s>>>(n3, kpad, mpad, ops->K64.as<double>(),
                                                               L.a.as<float>());
        M2L_LAUNCH_CHECK("transpose_pad_kernel");
    } else {
        const int rpad = simt_rpad(ops->rmax);
        const size_t nv = (size_t)kpad * rpad, nu = (size_t)rpad * mpad;
        if ((st = L.a.ensure(16 * nv * esz)) != M2L_OK) return st;
        if ((st = L.b.ensure(16 * nu * esz)) != M2L_OK) return st;
        dim3 grid((unsigned)((nv + nu + 255) / 256), 16);
        if (fp64)
            lowrank_layout_kernel<double><<<grid, 256, 0, s>>>(n3, ops->rmax, kpad, mpad, rpad,
                                                               ops->U64.as<double>(), ops->V64.as<double>(),
                                                               L.a.as<double>(), L.b.as<double>());
        else
            lowrank_layout_kernel<float><<<grid, 256, 0, s>>>(n3, ops->rmax, kpad, mpad, rpad,
                                                              ops->U64.as<double>(), ops->V64.as<double>(),
                                                              L.a.as<float>(), L.b.as<float>());
        M2L_LAUNCH_CHECK("lowrank_layout_kernel");
    }
    L.ready = true;
    return M2L_OK;
}

}  // namespace m2l

namespace m2l {

// FP32 transposed, zero-padded operator layout of the SIMT kernel written
// into caller-provided memory KT [16][kpad][mpad] (no allocation).
m2l_status launch_transpose_pad_f32(const m2l_ops *ops, float *KT, int kpad, int mpad, cudaStream_t s)
{
    const size_t total = 16 * (size_t)kpad * mpad;
    transpose_pad_kernel<float><<<(int)((total + 255) / 256), 256, 0, s>>>(ops->n3, kpad, mpad,
                                                                         ops->K64.as<double>(), KT);
    M2L_LAUNCH_CHECK("transpose_pad_kernel");
    return M2L_OK;
}

}  // namespace m2l
