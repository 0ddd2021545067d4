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
// A[p] = K_p^T stored row-major, i.e. K_p column-major: column j of K_p contiguous.
__global__ void to_column_major_kernel(int n3, const double *__restrict__ K, double *__restrict__ A)
{
    const long nn = (long)n3 * n3, total = 16 * nn;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        const long p = i / nn, r = i % nn, col = r / n3, row = r % n3;
        A[i] = K[p * nn + row * n3 + col];
    }
}

// After the one-sided Jacobi SVD K_p V = W Sigma (A holds W Sigma column-major):
// U[p][row][q] = (W Sigma)(row, order_q), V[p][row][q] = V(row, order_q) for
// q < r_p, zero beyond (the [16][n3][rmax] layout of the factors).
__global__ void extract_lowrank_kernel(int n3, int rmax, const int *__restrict__ ranks, const int *__restrict__ order,
                                       const double *__restrict__ A, const double *__restrict__ Vr,
                                       double *__restrict__ U, double *__restrict__ V)
{
    const int p = blockIdx.y;
    const int r = ranks[p];
    const long nn = (long)n3 * n3;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n3 * rmax; idx += gridDim.x * blockDim.x) {
        const int row = idx / rmax, k = idx % rmax;
        double u = 0.0, v = 0.0;
        if (k < r) {
            const long col = order[p * n3 + k];
            u = A[p * nn + col * n3 + row];
            v = Vr[p * nn + col * n3 + row];
        }
        U[(long)p * n3 * rmax + idx] = u;
        V[(long)p * n3 * rmax + idx] = v;
    }
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

// Step a1's truncated SVD of the 16 operators (Eq. (20)), by one-sided Jacobi
// on the device; ranks by the ops' truncation criterion.
m2l_status lowrank_factors(m2l_ops *ops)
{
    const int n = ops->n3;
    const size_t nn = (size_t)n * n;
    DevBuf A, S, VR, dord, dranks;
    ScratchGuard guard{&A, &S, &VR, &dord, &dranks};
    m2l_status st;
    if ((st = A.ensure(16 * nn * sizeof(double))) != M2L_OK) return st;
    if ((st = S.ensure(16 * (size_t)n * sizeof(double))) != M2L_OK) return st;
    if ((st = VR.ensure(16 * nn * sizeof(double))) != M2L_OK) return st;
    if ((st = dord.ensure(16 * (size_t)n * sizeof(int))) != M2L_OK) return st;
    if ((st = dranks.ensure(16 * sizeof(int))) != M2L_OK) return st;
    to_column_major_kernel<<<(int)std::min<size_t>((16 * nn + 255) / 256, 65535), 256>>>(n, ops->K64.as<double>(),
                                                                                         A.as<double>());
    M2L_LAUNCH_CHECK("to_column_major_kernel");
    if ((st = jacobi_svd(A.as<double>(), n, n, 16, VR.as<double>(), S.as<double>(), ops->jacobi_sweeps, 0)) != M2L_OK)
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
    dim3 grid((n * rmax + 255) / 256, 16);
    extract_lowrank_kernel<<<grid, 256>>>(n, rmax, dranks.as<int>(), dord.as<int>(), A.as<double>(), VR.as<double>(),
                                          ops->U64.as<double>(), ops->V64.as<double>());
    M2L_LAUNCH_CHECK("extract_lowrank_kernel");
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
