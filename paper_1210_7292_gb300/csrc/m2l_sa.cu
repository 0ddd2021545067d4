// The SA variant of the M2L translation and its recompression SArcmp
// (Sec. 4.1, Eqs. (17)-(19)): one low-rank basis for all operators of a level,
// K_t ~ U C_t B^* with C_t = U^* K_t B of size r x r, optionally
// C_t ~ Xbar_t Ybar_t^* of rank r_t < r / 2.  A second apply path beside the
// symmetry-blocked one, for comparison (the paper's Tables for SA/SArcmp).
//
// Set-up (synchronous): the 316 operators are expanded on the device from the
// 16 unique ones (K_t[a][b] = K_p[sigma(a)][sigma(b)]); one-sided Jacobi gives
// the two big SVDs; C_t = U^T (K_t B) by batched products; SArcmp by one small
// Jacobi SVD per t, all t in one batch.
// Apply: compress every source, w^ = B^T w (one GEMM); per transfer vector t,
// tiles of its interactions: gather w^, multiply by C_t (or by its two factors),
// add into f^ of the targets; decompress, f += scale U f^ (one GEMM).
#include <math.h>

#include <algorithm>
#include <vector>

#include "m2l_internal.cuh"

namespace m2l {
namespace {

constexpr int kSaTile = 32;        // interactions per core tile
constexpr int kSaMaxRank = 128;
constexpr int kSaThreads = 256;

// ---------------------------------------------------------------- products
// C[z] (+)= alpha A[z] B[z], row-major, A m x k, B k x n; 64 x 64 output tiles,
// 16-deep K slices in shared memory, 4 x 4 outputs per thread.
template <typename T, typename TO, bool ACC>
__global__ void __launch_bounds__(256)
gemm_rm_kernel(int m, int n, int k, const T *__restrict__ A, int lda, long long sA, const T *__restrict__ B, int ldb,
               long long sB, TO *__restrict__ C, int ldc, long long sC, double alpha)
{
    __shared__ T As[16][65];
    __shared__ T Bs[16][65];
    const int z = blockIdx.z;
    A += (size_t)z * sA;
    B += (size_t)z * sB;
    C += (size_t)z * sC;
    const int row0 = blockIdx.x * 64, col0 = blockIdx.y * 64;
    const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    for (int k0 = 0; k0 < k; k0 += 16) {
        for (int idx = threadIdx.x; idx < 16 * 64; idx += 256) {
            const int kk = idx / 64, rr = idx % 64;
            const int ar = row0 + rr, ak = k0 + kk;
            As[kk][rr] = (ar < m && ak < k) ? A[(size_t)ar * lda + ak] : T(0);
            const int bc = col0 + rr;
            Bs[kk][rr] = (ak < k && bc < n) ? B[(size_t)ak * ldb + bc] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            T a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][tr + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tc + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = row0 + tr + 16 * i;
        if (r >= m) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = col0 + tc + 16 * j;
            if (c >= n) continue;
            const TO v = (TO)(alpha * (double)acc[i][j]);
            if (ACC) C[(size_t)r * ldc + c] += v;
            else C[(size_t)r * ldc + c] = v;
        }
    }
}

template <typename T, typename TO, bool ACC>
void gemm_rm(int m, int n, int k, const T *A, int lda, long long sA, const T *B, int ldb, long long sB, TO *C,
             int ldc, long long sC, int batch, double alpha, cudaStream_t s)
{
    dim3 grid((m + 63) / 64, (n + 63) / 64, batch);
    gemm_rm_kernel<T, TO, ACC><<<grid, 256, 0, s>>>(m, n, k, A, lda, sA, B, ldb, sB, C, ldc, sC, alpha);
}

// ---------------------------------------------------------------- set-up
// The 316 operators from the 16 unique ones: row-major [nt][n3][n3], and the
// column-major K_col (m x n3) and K_row^T (m x n3), m = nt n3, for gesvd.
__global__ void sa_expand_kernel(int n3, int nt, const int *__restrict__ slots, const uint16_t *__restrict__ lut,
                                 const int16_t *__restrict__ sigma, const double *__restrict__ K64,
                                 double *__restrict__ Krm, double *__restrict__ Kcol, double *__restrict__ KrowT)
{
    const long long total = (long long)nt * n3 * n3, m = (long long)nt * n3;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int ti = (int)(idx / ((long long)n3 * n3));
        const int a = (int)((idx / n3) % n3), b = (int)(idx % n3);
        const uint16_t code = lut[slots[ti]];
        const int p = code & 0xFF, g = code >> 8;
        const double v = K64[((size_t)p * n3 + sigma[g * n3 + a]) * n3 + sigma[g * n3 + b]];
        Krm[idx] = v;
        Kcol[((long long)ti * n3 + a) + (long long)b * m] = v;
        KrowT[((long long)ti * n3 + b) + (long long)a * m] = v;
    }
}

// B [n3][r] and U^T [r][n3] from the right singular vectors of K_col and of
// K_row^T (Jacobi's V, column-major n3 x n3, vector ord[q] is the q-th largest).
__global__ void sa_basis_kernel(int n3, int r, const int *__restrict__ ord_col, const double *__restrict__ v_col,
                                const int *__restrict__ ord_row, const double *__restrict__ v_row,
                                double *__restrict__ B, double *__restrict__ Ut)
{
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n3 * r; idx += gridDim.x * blockDim.x) {
        const int j = idx / r, q = idx % r;
        B[(size_t)j * r + q] = v_col[(size_t)ord_col[q] * n3 + j];
        Ut[(size_t)q * n3 + j] = v_row[(size_t)ord_row[q] * n3 + j];
    }
}

// Column-major copies of the row-major r x r cores, for their Jacobi SVDs.
__global__ void sa_cores_colmajor_kernel(int r, int nt, const double *__restrict__ C, double *__restrict__ Ccm)
{
    const long rr = (long)r * r, total = (long)nt * rr;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        const long t = i / rr, e = i % rr, col = e / r, row = e % r;
        Ccm[i] = C[t * rr + row * r + col];
    }
}

template <typename TD, typename TS>
__global__ void convert_kernel(long long n, const TS *__restrict__ in, TD *__restrict__ out)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (TD)in[i];
}

// ---------------------------------------------------------------- bucketing
// Slot of every list entry (warp per target) and block-level slot counts.
__global__ void sa_slot_kernel(int ntgt, int nnz, const int32_t *__restrict__ offsets,
                               const int32_t *__restrict__ sources, const int32_t *__restrict__ tgt_ijk,
                               const int32_t *__restrict__ src_ijk, int nsrc, const uint16_t *__restrict__ lut,
                               int16_t *__restrict__ slot, int32_t *__restrict__ cnt, int *__restrict__ status)
{
    __shared__ int hist[343];
    for (int i = threadIdx.x; i < 343; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp < ntgt) {
        const int o0 = offsets[warp], o1 = offsets[warp + 1];
        if (o0 < 0 || o1 < o0 || o1 > nnz) {
            if (lane == 0) atomicOr(status, ST_BAD_INDEX);
        } else {
            for (int e = o0 + lane; e < o1; e += 32) {
                const int y = sources[e];
                int sl = -1;
                if (y >= 0 && y < nsrc) {
                    const int t0 = tgt_ijk[3 * warp] - src_ijk[3 * y];
                    const int t1 = tgt_ijk[3 * warp + 1] - src_ijk[3 * y + 1];
                    const int t2 = tgt_ijk[3 * warp + 2] - src_ijk[3 * y + 2];
                    if (abs(t0) <= 3 && abs(t1) <= 3 && abs(t2) <= 3) {
                        const int s = (t0 + 3) + 7 * (t1 + 3) + 49 * (t2 + 3);
                        if (lut[s] != 0xFFFF) sl = s;
                    }
                }
                if (sl < 0) atomicOr(status, y < 0 || y >= nsrc ? ST_BAD_INDEX : ST_BAD_PAIR);
                else atomicAdd(&hist[sl], 1);
                slot[e] = (int16_t)sl;
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 343; i += blockDim.x)
        if (hist[i]) atomicAdd(cnt + i, hist[i]);
}

// Records {source, target} in slot buckets (order inside a bucket is free: every
// target appears at most once per transfer vector).
__global__ void sa_scatter_kernel(int ntgt, const int32_t *__restrict__ offsets, const int32_t *__restrict__ sources,
                                  const int16_t *__restrict__ slot, const int32_t *__restrict__ start,
                                  int32_t *__restrict__ cursor, int2 *__restrict__ rec)
{
    __shared__ int hist[343], base[343];
    for (int i = threadIdx.x; i < 343; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const bool have = warp < ntgt;
    const int o0 = have ? offsets[warp] : 0, o1 = have ? offsets[warp + 1] : 0;
    for (int e = o0 + lane; e < o1; e += 32)
        if (slot[e] >= 0) atomicAdd(&hist[slot[e]], 1);
    __syncthreads();
    for (int i = threadIdx.x; i < 343; i += blockDim.x) {
        base[i] = hist[i] ? start[i] + atomicAdd(cursor + i, hist[i]) : 0;
        hist[i] = 0;
    }
    __syncthreads();
    for (int e = o0 + lane; e < o1; e += 32) {
        const int sl = slot[e];
        if (sl < 0) continue;
        rec[base[sl] + atomicAdd(&hist[sl], 1)] = make_int2(sources[e], warp);
    }
}

// ---------------------------------------------------------------- core
// Tiles of kSaTile interactions of one transfer vector: f^[X] += C_t w^[Y],
// C_t = X_t Y_t^T of rank k_t (SArcmp) or X_t = C_t whole (k_t = 0).
// Xt holds X_t transposed, Xt[j][a] (row stride r), Y holds Y_t as Y[q][j]
// (row stride r).  With STAGE the factors of the current transfer vector are
// copied to shared memory, else they are read from global memory (L2).
template <typename T, bool STAGE>
__global__ void __launch_bounds__(kSaThreads)
sa_core_kernel(int r, const int32_t *__restrict__ start, const int2 *__restrict__ rec, const T *__restrict__ Xt,
               const T *__restrict__ Yf, const int *__restrict__ kt, const T *__restrict__ what, T *__restrict__ fhat)
{
    extern __shared__ __align__(16) unsigned char sa_smem[];
    T *sW = reinterpret_cast<T *>(sa_smem);   // kSaTile x r gathered w^
    T *sZ = sW + kSaTile * r;                 // kSaTile x r (Y_t^T w^ in the first k columns)
    T *sX = sZ + kSaTile * r;                 // r x r, X_t^T   (STAGE only)
    T *sY = sX + r * r;                       // r x k, Y_t     (STAGE only)
    __shared__ int s_tile[344];
    __shared__ int2 s_rec[kSaTile];
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int sl = 0; sl < 343; ++sl) {
            s_tile[sl] = acc;
            acc += (start[sl + 1] - start[sl] + kSaTile - 1) / kSaTile;
        }
        s_tile[343] = acc;
    }
    __syncthreads();
    const int ntiles = s_tile[343];
    int sl = 0, cur_sl = -1, k = 0;
    const T *Mt = nullptr, *My = nullptr;
    int ldy = r;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        while (sl < 342 && tile >= s_tile[sl + 1]) ++sl;
        const int c0 = start[sl] + (tile - s_tile[sl]) * kSaTile;
        const int nc = min(kSaTile, start[sl + 1] - c0);
        __syncthreads();   // previous tile's readers are done with sW, sZ, sX, sY
        if (sl != cur_sl) {
            k = kt[sl];
            const size_t fo = (size_t)sl * r * r;
            if (STAGE) {
                for (int i = threadIdx.x; i < r * r; i += blockDim.x) sX[i] = Xt[fo + i];
                for (int i = threadIdx.x; i < r * k; i += blockDim.x) sY[i] = Yf[fo + (i / k) * r + (i % k)];
                Mt = sX;
                My = sY;
                ldy = k;
            } else {
                Mt = Xt + fo;
                My = Yf + fo;
                ldy = r;
            }
            cur_sl = sl;
        }
        if (threadIdx.x < kSaTile) s_rec[threadIdx.x] = threadIdx.x < nc ? rec[c0 + threadIdx.x] : make_int2(0, -1);
        __syncthreads();
        for (int i = threadIdx.x; i < kSaTile * r; i += blockDim.x) {
            const int c = i / r, q = i % r;
            sW[i] = c < nc ? what[(size_t)s_rec[c].x * r + q] : T(0);
        }
        __syncthreads();
        const T *src = sW;
        int kin = r;
        if (k > 0) {
            // z = Y_t^T w^  (kSaTile x k)
            for (int i = threadIdx.x; i < kSaTile * k; i += blockDim.x) {
                const int c = i / k, j = i % k;
                T sum = T(0);
                for (int q = 0; q < r; ++q) sum += My[q * ldy + j] * sW[c * r + q];
                sZ[c * r + j] = sum;
            }
            __syncthreads();
            src = sZ;
            kin = k;
        }
        // y = X_t z  (or C_t w^): output a of column c, X_t(a, j) at Mt[j * r + a]
        for (int i = threadIdx.x; i < kSaTile * r; i += blockDim.x) {
            const int c = i / r, a = i % r;
            if (c >= nc) continue;
            T sum = T(0);
            for (int j = 0; j < kin; ++j) sum += Mt[j * r + a] * src[c * r + j];
            atomicAdd(fhat + (size_t)s_rec[c].y * r + a, sum);
        }
    }
}

__global__ void sa_transpose_kernel(int r, const double *__restrict__ X, double *__restrict__ Xt)
{
    const long long total = 343LL * r * r;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long z = idx / ((long long)r * r);
        const int a = (int)((idx / r) % r), j = (int)(idx % r);
        Xt[z * r * r + (long long)j * r + a] = X[idx];
    }
}

// Dense cores for the tensor-core apply: C_t itself, or X_t Y_t^T where SArcmp
// recompressed it (the rank saving does not pay on the tensor cores).
__global__ void sa_dense_kernel(int r, const int *__restrict__ kt, const double *__restrict__ X,
                                const double *__restrict__ Y, double *__restrict__ Cd)
{
    const long long total = 343LL * r * r;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int sl = (int)(idx / ((long long)r * r));
        const int a = (int)((idx / r) % r), b = (int)(idx % r);
        const int k = kt[sl];
        const double *Xs = X + (size_t)sl * r * r, *Ys = Y + (size_t)sl * r * r;
        double v;
        if (k == 0) {
            v = Xs[(size_t)a * r + b];
        } else {
            v = 0.0;
            for (int q = 0; q < k; ++q) v += Xs[(size_t)a * r + q] * Ys[(size_t)b * r + q];
        }
        Cd[idx] = v;
    }
}

// Identity gather tables (no symmetry in SA): row k of the panel reads node k.
__global__ void sa_identity_kernel(int r, int kpad, int16_t *__restrict__ tinv)
{
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < 48 * kpad; idx += gridDim.x * blockDim.x) {
        const int k = idx % kpad;
        tinv[idx] = (int16_t)(k < r ? k : 0);
    }
}

// Tile offsets of the slot buckets for tiles of tcols interactions.
__global__ void sa_tiles_kernel(const int32_t *__restrict__ start, int tcols, int32_t *__restrict__ tstart)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int acc = 0;
    for (int sl = 0; sl < 343; ++sl) {
        tstart[sl] = acc;
        acc += (start[sl + 1] - start[sl] + tcols - 1) / tcols;
    }
    tstart[343] = acc;
}

int sa_grid(long n)
{
    long b = (n + 255) / 256;
    return (int)(b > 4096 ? 4096 : (b < 1 ? 1 : b));
}

}  // namespace
}  // namespace m2l

using namespace m2l;

struct m2l_sa {
    const m2l_ops *ops = nullptr;
    int r = 0, n3 = 0, recompress = 0, n_recompressed = 0;
    double eps = 0.0;
    std::vector<int> kt;              // per slot: k_t (0: C_t kept whole)
    m2l::DevBuf U64t, B64, X64, Y64;  // U^T [r][n3], B [n3][r], X, Y [343][r][r] (double)
    m2l::DevBuf Xt64;                 // X transposed per slot (kernel layout)
    m2l::DevBuf U32t, B32, Xt32, Y32; // float copies for the FP32 apply
    m2l::DevBuf dkt, start, cursor, slot, rec, what, fhat, cnt;
    struct Tc {                        // tensor-core images of the dense cores (built on first use)
        m2l::DevBuf img, tinv;
        int tcols = 0;
        bool ready = false;
    } tc[3];                           // M2L_TF32, M2L_BF16X3, M2L_TF32X3
    m2l::DevBuf tstart;                // tile offsets per slot [344]
};

namespace {

void sa_release(m2l_sa *a)
{
    if (!a) return;
    cudaDeviceSynchronize();
    m2l::DevBuf *bs[] = {&a->U64t,     &a->B64,       &a->X64,       &a->Y64,       &a->Xt64,      &a->U32t,
                         &a->B32,      &a->Xt32,      &a->Y32,       &a->dkt,       &a->start,     &a->cursor,
                         &a->slot,     &a->rec,       &a->what,      &a->fhat,      &a->cnt,       &a->tc[0].img,
                         &a->tc[0].tinv, &a->tc[1].img, &a->tc[1].tinv, &a->tc[2].img, &a->tc[2].tinv, &a->tstart};
    for (m2l::DevBuf *b : bs) b->release();
    delete a;
}

// Scratch of the set-up, released on every return.
struct SaScratch {
    DevBuf dslots, Krm, Kcol, KrowT, S1, S2, V1, V2, ord1, ord2, T1, Cfull, Ccm, Vc, sc;
    ~SaScratch()
    {
        cudaDeviceSynchronize();
        DevBuf *bs[] = {&dslots, &Krm, &Kcol, &KrowT, &S1, &S2, &V1, &V2, &ord1, &ord2, &T1, &Cfull, &Ccm, &Vc, &sc};
        for (DevBuf *b : bs) b->release();
    }
};

#define SA_TRY(x) do { m2l_status st_ = (x); if (st_ != M2L_OK) return st_; } while (0)

// Order (descending) and truncation rank of one set of Jacobi singular values.
int sa_rank(const std::vector<double> &sv, int n, double eps, int trunc, std::vector<int> &order)
{
    order.resize(n);
    order_descending(sv.data(), n, order.data());
    std::vector<double> sorted(n);
    for (int i = 0; i < n; ++i) sorted[i] = sv[order[i]];
    const int r = truncation_rank(sorted.data(), n, eps, trunc);
    return r < 1 ? 1 : r;
}

m2l_status sa_build(m2l_sa *a, cudaStream_t s)
{
    const m2l_ops *ops = a->ops;
    const int n3 = ops->n3;
    a->n3 = n3;
    SaScratch w;
    // the 316 far-field transfer vectors, in slot order
    std::vector<uint16_t> hlut(343);
    M2L_CUDA(cudaMemcpy(hlut.data(), ops->lut.p, 343 * sizeof(uint16_t), cudaMemcpyDeviceToHost));
    std::vector<int> slots;
    for (int i = 0; i < 343; ++i)
        if (hlut[i] != 0xFFFF) slots.push_back(i);
    const int nt = (int)slots.size();
    const long long m = (long long)nt * n3;
    SA_TRY(w.dslots.ensure(nt * sizeof(int)));
    SA_TRY(w.Krm.ensure((size_t)m * n3 * sizeof(double)));
    SA_TRY(w.Kcol.ensure((size_t)m * n3 * sizeof(double)));
    SA_TRY(w.KrowT.ensure((size_t)m * n3 * sizeof(double)));
    SA_TRY(w.S1.ensure(n3 * sizeof(double)));
    SA_TRY(w.S2.ensure(n3 * sizeof(double)));
    SA_TRY(w.V1.ensure((size_t)n3 * n3 * sizeof(double)));
    SA_TRY(w.V2.ensure((size_t)n3 * n3 * sizeof(double)));
    SA_TRY(w.ord1.ensure(n3 * sizeof(int)));
    SA_TRY(w.ord2.ensure(n3 * sizeof(int)));
    M2L_CUDA(cudaMemcpy(w.dslots.p, slots.data(), nt * sizeof(int), cudaMemcpyHostToDevice));
    sa_expand_kernel<<<sa_grid((long)m * n3), 256, 0, s>>>(n3, nt, w.dslots.as<int>(), ops->lut.as<uint16_t>(),
                                                             ops->sigma.as<int16_t>(), ops->K64.as<double>(),
                                                             w.Krm.as<double>(), w.Kcol.as<double>(),
                                                             w.KrowT.as<double>());
    M2L_LAUNCH_CHECK("sa_expand_kernel");
    M2L_CUDA(cudaStreamSynchronize(s));
    // the two SVDs of Eq. (17) by one-sided Jacobi; only the right singular
    // vectors (the accumulated rotations) are kept
    SA_TRY(jacobi_svd(w.Kcol.as<double>(), (int)m, n3, 1, w.V1.as<double>(), w.S1.as<double>(), nullptr, s));
    SA_TRY(jacobi_svd(w.KrowT.as<double>(), (int)m, n3, 1, w.V2.as<double>(), w.S2.as<double>(), nullptr, s));
    std::vector<double> s1(n3), s2(n3);
    std::vector<int> o1, o2;
    M2L_CUDA(cudaMemcpy(s1.data(), w.S1.p, n3 * sizeof(double), cudaMemcpyDeviceToHost));
    M2L_CUDA(cudaMemcpy(s2.data(), w.S2.p, n3 * sizeof(double), cudaMemcpyDeviceToHost));
    const int trunc = a->ops->trunc;
    const int r = std::max(sa_rank(s2, n3, a->eps, trunc, o2), sa_rank(s1, n3, a->eps, trunc, o1));
    if (r > kSaMaxRank) {
        set_error("SA rank %d exceeds %d", r, kSaMaxRank);
        return M2L_EUNSUPPORTED;
    }
    a->r = r;
    SA_TRY(a->B64.ensure((size_t)n3 * r * sizeof(double)));
    SA_TRY(a->U64t.ensure((size_t)r * n3 * sizeof(double)));
    M2L_CUDA(cudaMemcpy(w.ord1.p, o1.data(), n3 * sizeof(int), cudaMemcpyHostToDevice));
    M2L_CUDA(cudaMemcpy(w.ord2.p, o2.data(), n3 * sizeof(int), cudaMemcpyHostToDevice));
    sa_basis_kernel<<<sa_grid((long)n3 * r), 256, 0, s>>>(n3, r, w.ord1.as<int>(), w.V1.as<double>(),
                                                          w.ord2.as<int>(), w.V2.as<double>(),
                                                          a->B64.as<double>(), a->U64t.as<double>());
    M2L_LAUNCH_CHECK("sa_basis_kernel");
    // C_t = U^T (K_t B), Eq. (18), for the 316 transfer vectors
    SA_TRY(w.T1.ensure((size_t)nt * n3 * r * sizeof(double)));
    SA_TRY(w.Cfull.ensure((size_t)nt * r * r * sizeof(double)));
    gemm_rm<double, double, false>(n3, r, n3, w.Krm.as<double>(), n3, (long long)n3 * n3, a->B64.as<double>(), r, 0,
                                   w.T1.as<double>(), r, (long long)n3 * r, nt, 1.0, s);
    M2L_LAUNCH_CHECK("gemm(K_t B)");
    gemm_rm<double, double, false>(r, r, n3, a->U64t.as<double>(), n3, 0, w.T1.as<double>(), r, (long long)n3 * r,
                                   w.Cfull.as<double>(), r, (long long)r * r, nt, 1.0, s);
    M2L_LAUNCH_CHECK("gemm(U^T K_t B)");
    // factors per slot: X [r][r] holds C_t, or X_t in its first k_t columns; Y [r][r] Y_t likewise
    const size_t rr = (size_t)r * r;
    SA_TRY(a->X64.ensure(343 * rr * sizeof(double)));
    SA_TRY(a->Y64.ensure(343 * rr * sizeof(double)));
    M2L_CUDA(cudaMemsetAsync(a->X64.p, 0, 343 * rr * sizeof(double), s));
    M2L_CUDA(cudaMemsetAsync(a->Y64.p, 0, 343 * rr * sizeof(double), s));
    a->kt.assign(343, 0);
    // SArcmp, Eq. (19): one-sided Jacobi SVD of every core, C_t V = W Sigma, so
    // C_t ~ X_t Y_t^T with X_t = (W Sigma)_k (column-major Jacobi output) and
    // Y_t = V_k, the k = r_t largest; kept only when 2 r_t < r.
    std::vector<double> hW, hV, hs;
    std::vector<int> ord;
    if (a->recompress) {
        SA_TRY(w.Ccm.ensure((size_t)nt * rr * sizeof(double)));
        SA_TRY(w.Vc.ensure((size_t)nt * rr * sizeof(double)));
        SA_TRY(w.sc.ensure((size_t)nt * r * sizeof(double)));
        sa_cores_colmajor_kernel<<<sa_grid((long)nt * rr), 256, 0, s>>>(r, nt, w.Cfull.as<double>(),
                                                                        w.Ccm.as<double>());
        M2L_LAUNCH_CHECK("sa_cores_colmajor_kernel");
        SA_TRY(jacobi_svd(w.Ccm.as<double>(), r, r, nt, w.Vc.as<double>(), w.sc.as<double>(), nullptr, s));
        hW.resize((size_t)nt * rr);
        hV.resize((size_t)nt * rr);
        hs.resize((size_t)nt * r);
        M2L_CUDA(cudaMemcpy(hW.data(), w.Ccm.p, hW.size() * sizeof(double), cudaMemcpyDeviceToHost));
        M2L_CUDA(cudaMemcpy(hV.data(), w.Vc.p, hV.size() * sizeof(double), cudaMemcpyDeviceToHost));
        M2L_CUDA(cudaMemcpy(hs.data(), w.sc.p, hs.size() * sizeof(double), cudaMemcpyDeviceToHost));
    }
    std::vector<double> cs(r), hX(rr), hY(rr);
    for (int i = 0; i < nt; ++i) {
        const int sl = slots[i];
        double *Cd = w.Cfull.as<double>() + (size_t)i * rr;
        double *Xd = a->X64.as<double>() + (size_t)sl * rr;
        double *Yd = a->Y64.as<double>() + (size_t)sl * rr;
        int k = 0;
        if (a->recompress) {
            std::copy(hs.begin() + (size_t)i * r, hs.begin() + (size_t)(i + 1) * r, cs.begin());
            const int rt = sa_rank(cs, r, a->eps, trunc, ord);
            if (2 * rt < r) {
                k = rt;
                const double *Wt = hW.data() + (size_t)i * rr, *Vt = hV.data() + (size_t)i * rr;
                std::fill(hX.begin(), hX.end(), 0.0);
                std::fill(hY.begin(), hY.end(), 0.0);
                for (int q = 0; q < k; ++q) {
                    const size_t col = (size_t)ord[q] * r;
                    for (int row = 0; row < r; ++row) {
                        hX[(size_t)row * r + q] = Wt[col + row];   // (W Sigma)(row, q-th)
                        hY[(size_t)row * r + q] = Vt[col + row];   // V(row, q-th)
                    }
                }
                M2L_CUDA(cudaMemcpy(Xd, hX.data(), rr * sizeof(double), cudaMemcpyHostToDevice));
                M2L_CUDA(cudaMemcpy(Yd, hY.data(), rr * sizeof(double), cudaMemcpyHostToDevice));
                a->n_recompressed++;
            }
        }
        if (k == 0) M2L_CUDA(cudaMemcpyAsync(Xd, Cd, rr * sizeof(double), cudaMemcpyDeviceToDevice, s));
        a->kt[sl] = k;
    }
    // kernel layouts: X transposed per slot, and float copies
    SA_TRY(a->Xt64.ensure(343 * rr * sizeof(double)));
    sa_transpose_kernel<<<sa_grid(343L * r * r), 256, 0, s>>>(r, a->X64.as<double>(), a->Xt64.as<double>());
    M2L_LAUNCH_CHECK("sa_transpose_kernel");
    SA_TRY(a->U32t.ensure((size_t)r * n3 * sizeof(float)));
    SA_TRY(a->B32.ensure((size_t)n3 * r * sizeof(float)));
    SA_TRY(a->Xt32.ensure(343 * rr * sizeof(float)));
    SA_TRY(a->Y32.ensure(343 * rr * sizeof(float)));
    convert_kernel<float, double><<<sa_grid((long)r * n3), 256, 0, s>>>((long long)r * n3, a->U64t.as<double>(),
                                                                       a->U32t.as<float>());
    convert_kernel<float, double><<<sa_grid((long)r * n3), 256, 0, s>>>((long long)r * n3, a->B64.as<double>(),
                                                                       a->B32.as<float>());
    convert_kernel<float, double><<<sa_grid(343L * r * r), 256, 0, s>>>(343LL * r * r, a->Xt64.as<double>(),
                                                                       a->Xt32.as<float>());
    convert_kernel<float, double><<<sa_grid(343L * r * r), 256, 0, s>>>(343LL * r * r, a->Y64.as<double>(),
                                                                       a->Y32.as<float>());
    M2L_LAUNCH_CHECK("convert_kernel");
    SA_TRY(a->dkt.ensure(343 * sizeof(int)));
    SA_TRY(a->start.ensure(344 * sizeof(int32_t)));
    SA_TRY(a->cursor.ensure(343 * sizeof(int32_t)));
    SA_TRY(a->cnt.ensure(344 * sizeof(int32_t)));
    M2L_CUDA(cudaMemcpy(a->dkt.p, a->kt.data(), 343 * sizeof(int), cudaMemcpyHostToDevice));
    M2L_CUDA(cudaStreamSynchronize(s));
    return M2L_OK;
}

// Shared memory of the core kernel: gathered w^ and z always, the factors when staged.
size_t sa_core_smem(int r, size_t esz, bool stage)
{
    return (size_t)(2 * kSaTile * r + (stage ? r * r + r * (r / 2) : 0)) * esz;
}

m2l_status sa_prepare_tc(m2l_sa *a, int precision, cudaStream_t s)
{
    const int ti = precision == M2L_TF32 ? 0 : precision == M2L_BF16X3 ? 1 : 2;
    m2l_sa::Tc &L = a->tc[ti];
    if (L.ready) return M2L_OK;
    const int r = a->r;
    int kpad = 0, tcols = 0;
    size_t per_op = 0;
    if (!tc_general_config(precision, r, &kpad, &per_op, &tcols)) {
        set_error("no tensor-core configuration for SA rank %d", r);
        return M2L_EUNSUPPORTED;
    }
    DevBuf Cd;
    ScratchGuard guard{&Cd};
    SA_TRY(Cd.ensure(343ULL * r * r * sizeof(double)));
    SA_TRY(L.img.ensure(343ULL * per_op));
    SA_TRY(L.tinv.ensure((size_t)48 * kpad * sizeof(int16_t)));
    SA_TRY(a->tstart.ensure(344 * sizeof(int32_t)));
    sa_dense_kernel<<<sa_grid(343L * r * r), 256, 0, s>>>(r, a->dkt.as<int>(), a->X64.as<double>(), a->Y64.as<double>(),
                                                          Cd.as<double>());
    M2L_LAUNCH_CHECK("sa_dense_kernel");
    SA_TRY(tc_general_images(precision, r, 343, Cd.as<double>(), L.img.as<uint8_t>(), s));
    sa_identity_kernel<<<sa_grid(48L * kpad), 256, 0, s>>>(r, kpad, L.tinv.as<int16_t>());
    M2L_LAUNCH_CHECK("sa_identity_kernel");
    M2L_CUDA(cudaStreamSynchronize(s));
    L.tcols = tcols;
    L.ready = true;
    return M2L_OK;
}

template <typename T, typename TO>
m2l_status sa_apply(m2l_sa *a, const m2l_level *lv, const T *w, TO *loc, double scale, cudaStream_t s,
                    int tc_precision = -1)
{
    const int r = a->r, n3 = a->n3, nnz = lv->nnz;
    const int ntgt = lv->ncells_tgt, nsrc = lv->ncells_src;
    if (nnz == 0 || ntgt == 0) return M2L_OK;
    SA_TRY(a->slot.ensure((size_t)nnz * sizeof(int16_t)));
    SA_TRY(a->rec.ensure((size_t)nnz * sizeof(int2)));
    SA_TRY(a->what.ensure((size_t)(nsrc > 0 ? nsrc : 1) * r * sizeof(T)));
    SA_TRY(a->fhat.ensure((size_t)ntgt * r * sizeof(T)));
    // bucketing by transfer vector
    M2L_CUDA(cudaMemsetAsync(a->cnt.p, 0, 344 * sizeof(int32_t), s));
    M2L_CUDA(cudaMemsetAsync(a->cursor.p, 0, 343 * sizeof(int32_t), s));
    const int wblocks = (int)(((long)ntgt * 32 + 255) / 256);
    sa_slot_kernel<<<wblocks, 256, 0, s>>>(ntgt, nnz, lv->il_offsets, lv->il_sources, lv->tgt_ijk, lv->src_ijk, nsrc,
                                           a->ops->lut.as<uint16_t>(), a->slot.as<int16_t>(), a->cnt.as<int32_t>(),
                                           a->ops->d_status);
    M2L_LAUNCH_CHECK("sa_slot_kernel");
    SA_TRY(launch_exclusive_scan(a->cnt.as<int32_t>(), a->start.as<int32_t>(), 343, s));
    sa_scatter_kernel<<<wblocks, 256, 0, s>>>(ntgt, lv->il_offsets, lv->il_sources, a->slot.as<int16_t>(),
                                              a->start.as<int32_t>(), a->cursor.as<int32_t>(), a->rec.as<int2>());
    M2L_LAUNCH_CHECK("sa_scatter_kernel");
    const bool f64 = sizeof(T) == 8;
    const T *Bm = static_cast<const T *>(f64 ? a->B64.p : a->B32.p);
    const T *Ut = static_cast<const T *>(f64 ? a->U64t.p : a->U32t.p);
    const T *Xt = static_cast<const T *>(f64 ? a->Xt64.p : a->Xt32.p);
    const T *Yf = static_cast<const T *>(f64 ? a->Y64.p : a->Y32.p);
    // compress: w^ = w B  (nsrc x r)
    if (nsrc > 0) {
        gemm_rm<T, T, false>(nsrc, r, n3, w, n3, 0, Bm, r, 0, a->what.as<T>(), r, 0, 1, 1.0, s);
        M2L_LAUNCH_CHECK("gemm(compress)");
    }
    // core: f^[X] += C_t w^[Y]
    M2L_CUDA(cudaMemsetAsync(a->fhat.p, 0, (size_t)ntgt * r * sizeof(T), s));
    if constexpr (sizeof(T) == 4) {
        if (tc_precision >= 0) {   // on the tensor cores, one class per transfer vector
            const m2l_sa::Tc &L = a->tc[tc_precision == M2L_TF32 ? 0 : tc_precision == M2L_BF16X3 ? 1 : 2];
            sa_tiles_kernel<<<1, 32, 0, s>>>(a->start.as<int32_t>(), L.tcols, a->tstart.as<int32_t>());
            M2L_LAUNCH_CHECK("sa_tiles_kernel");
            SA_TRY(tc_general_apply(tc_precision, r, 343, a->tstart.as<int>(), a->rec.as<int2>(), a->start.as<int>(),
                                    L.img.as<uint8_t>(), L.tinv.as<int16_t>(), nnz, a->what.as<float>(),
                                    a->fhat.as<float>(), a->ops->d_status, s));
            gemm_rm<T, TO, true>(ntgt, n3, r, a->fhat.as<T>(), r, 0, Ut, n3, 0, loc, n3, 0, 1, scale, s);
            M2L_LAUNCH_CHECK("gemm(decompress)");
            return M2L_OK;
        }
    }
    const bool stage = (int)sa_core_smem(r, sizeof(T), true) + 4096 <= max_smem_optin();
    const size_t smem = sa_core_smem(r, sizeof(T), stage);
    const long tiles_bound = (long)nnz / kSaTile + 343;
    const int grid = (int)std::min<long>((long)num_sms() * 4, tiles_bound);
    if (stage) {
        M2L_CUDA(cudaFuncSetAttribute(sa_core_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        sa_core_kernel<T, true><<<grid, kSaThreads, smem, s>>>(r, a->start.as<int32_t>(), a->rec.as<int2>(), Xt, Yf,
                                                                a->dkt.as<int>(), a->what.as<T>(), a->fhat.as<T>());
    } else {
        M2L_CUDA(cudaFuncSetAttribute(sa_core_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        sa_core_kernel<T, false><<<grid, kSaThreads, smem, s>>>(r, a->start.as<int32_t>(), a->rec.as<int2>(), Xt, Yf,
                                                                 a->dkt.as<int>(), a->what.as<T>(), a->fhat.as<T>());
    }
    M2L_LAUNCH_CHECK("sa_core_kernel");
    // decompress: f += scale f^ U^T  (ntgt x n3)
    gemm_rm<T, TO, true>(ntgt, n3, r, a->fhat.as<T>(), r, 0, Ut, n3, 0, loc, n3, 0, 1, scale, s);
    M2L_LAUNCH_CHECK("gemm(decompress)");
    return M2L_OK;
}

}  // namespace

extern "C" {

m2l_status m2l_sa_create(const m2l_ops *ops, double eps, int recompress, void *stream, m2l_sa **out)
{
    if (!ops || !out || !(eps >= 0.0) || eps >= 1.0) { set_error("bad SA arguments"); return M2L_EINVAL; }
    *out = nullptr;
    m2l_sa *a = new m2l_sa();
    a->ops = ops;
    a->eps = eps;
    a->recompress = recompress ? 1 : 0;
    m2l_status st = sa_build(a, (cudaStream_t)stream);
    if (st != M2L_OK) { sa_release(a); return st; }
    *out = a;
    return M2L_OK;
}

m2l_status m2l_sa_info(const m2l_sa *sa, int *rank, int *n_recompressed, int32_t *kt343)
{
    if (!sa) { set_error("null SA"); return M2L_EINVAL; }
    if (rank) *rank = sa->r;
    if (n_recompressed) *n_recompressed = sa->n_recompressed;
    if (kt343)
        for (int i = 0; i < 343; ++i) kt343[i] = sa->kt[i];
    return M2L_OK;
}

m2l_status m2l_sa_copy_factors(const m2l_sa *sa, double *host_Ut, double *host_B, double *host_X, double *host_Y)
{
    if (!sa) { set_error("null SA"); return M2L_EINVAL; }
    M2L_CUDA(cudaDeviceSynchronize());
    const size_t r = sa->r, n3 = sa->n3;
    if (host_Ut) M2L_CUDA(cudaMemcpy(host_Ut, sa->U64t.p, r * n3 * sizeof(double), cudaMemcpyDeviceToHost));
    if (host_B) M2L_CUDA(cudaMemcpy(host_B, sa->B64.p, n3 * r * sizeof(double), cudaMemcpyDeviceToHost));
    if (host_X) M2L_CUDA(cudaMemcpy(host_X, sa->X64.p, 343 * r * r * sizeof(double), cudaMemcpyDeviceToHost));
    if (host_Y) M2L_CUDA(cudaMemcpy(host_Y, sa->Y64.p, 343 * r * r * sizeof(double), cudaMemcpyDeviceToHost));
    return M2L_OK;
}

m2l_status m2l_sa_apply_level(const m2l_sa *sa_c, const m2l_level *level, const void *multipoles, void *locals,
                              int precision, int locals_fp64, void *stream)
{
    m2l_sa *sa = const_cast<m2l_sa *>(sa_c);
    if (!sa || !level) { set_error("null SA or level"); return M2L_EINVAL; }
    const m2l_ops *ops = sa->ops;
    if (m2l_status st = check_device(ops)) return st;
    if (level->ncells_tgt < 0 || level->ncells_src < 0 || level->nnz < 0 ||
        (level->nnz > 0 && (!level->il_sources || !level->il_offsets || !level->tgt_ijk || !level->src_ijk ||
                            !multipoles || !locals))) {
        set_error("bad level for the SA apply");
        return M2L_EINVAL;
    }
    double scale = 1.0;
    if (ops->homogeneous) scale = pow(level->width / ops->ref_width, (double)ops->hom_degree);
    else if (fabs(level->width - ops->ref_width) > 1e-12 * ops->ref_width) {
        set_error("level width differs from the operators' (kernel not homogeneous)");
        return M2L_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == M2L_FP64) return sa_apply<double, double>(sa, level, (const double *)multipoles, (double *)locals, scale, s);
    if (precision == M2L_FP32) {
        if (locals_fp64) return sa_apply<float, double>(sa, level, (const float *)multipoles, (double *)locals, scale, s);
        return sa_apply<float, float>(sa, level, (const float *)multipoles, (float *)locals, scale, s);
    }
    if (precision == M2L_TF32 || precision == M2L_BF16X3 || precision == M2L_TF32X3) {
        m2l_status st = sa_prepare_tc(sa, precision, s);
        if (st != M2L_OK) return st;
        if (locals_fp64)
            return sa_apply<float, double>(sa, level, (const float *)multipoles, (double *)locals, scale, s, precision);
        return sa_apply<float, float>(sa, level, (const float *)multipoles, (float *)locals, scale, s, precision);
    }
    set_error("unknown precision %d", precision);
    return M2L_EINVAL;
}

void m2l_sa_free(m2l_sa *sa) { sa_release(sa); }

}  // extern "C"
