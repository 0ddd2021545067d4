// Steps a4-a6 on the CUDA cores (FP64 and FP32): one fused kernel per
// precision that, for a tile of NT bucketed interactions of operator p,
//   a4  gathers the source multipoles and permutes them into the panel,
//       W_p[sigma_g(b)][c] = w_Y[b]                            (Eq. (30))
//   a5  multiplies F_p = K_p W_p                                (Eq. (31)),
//       or U_p (V_p^T W_p) for the low-rank operators           (Eq. (20))
//   a6  un-permutes f[a] = F_p[sigma_g(a)][c], sums the consecutive columns
//       of one target and adds the sum to the target's local     (Eq. (32))
// with one atomic add per (target, node) and tile (Alg. 2, third loop).
// The panel and the product never leave shared memory.
#include "m2l_internal.cuh"

namespace m2l {

int simt_kpad(int n3);
int simt_mpad(int n3);
int simt_rpad(int r);
m2l_status prepare_simt_layout(const m2l_ops *ops, int fp64, cudaStream_t s);

namespace {

constexpr int kThreads = 256;   // 8 warps x 16 rows = 128 rows per M chunk
constexpr int kRowsPerWarp = 16;

template <typename T> struct VecOf;
template <> struct VecOf<float> { using type = float4; static constexpr int n = 4; };
template <> struct VecOf<double> { using type = double2; static constexpr int n = 2; };

template <typename T> constexpr int kc_of() { return sizeof(T) == 8 ? 16 : 32; }

// out_mode 0: Out[c * ldo + m]  (column-major, for the un-permute epilogue)
// out_mode 1: Out[m * ldo + c]  (row-major over m, a B operand for the next product)
template <typename T, int NT, int OUT_MODE>
__device__ __forceinline__ void gemm_chunked(const T *__restrict__ A, int ldA, int K, int M,
                                             const T *__restrict__ Bs, T *__restrict__ As,
                                             T *__restrict__ Out, int ldo)
{
    constexpr int KC = kc_of<T>();
    constexpr int CPL = NT / 32;   // columns per lane
    using V = typename VecOf<T>::type;
    constexpr int VN = VecOf<T>::n;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int mc = 0; mc < M; mc += 128) {
        const int mrows = min(128, M - mc);
        const bool active = kRowsPerWarp * warp < mrows;
        T acc[kRowsPerWarp][CPL];
#pragma unroll
        for (int i = 0; i < kRowsPerWarp; ++i)
#pragma unroll
            for (int j = 0; j < CPL; ++j) acc[i][j] = T(0);
        for (int kc = 0; kc < K; kc += KC) {
            __syncthreads();
            for (int idx = threadIdx.x; idx < KC * 128; idx += kThreads) {
                const int kk = idx >> 7, m = idx & 127;
                As[idx] = (m < mrows) ? A[(size_t)(kc + kk) * ldA + mc + m] : T(0);
            }
            __syncthreads();
            if (active) {
#pragma unroll 4
                for (int kk = 0; kk < KC; ++kk) {
                    T a[kRowsPerWarp];
                    const V *ap = reinterpret_cast<const V *>(As + kk * 128 + kRowsPerWarp * warp);
#pragma unroll
                    for (int v = 0; v < kRowsPerWarp / VN; ++v) {
                        const V x = ap[v];
                        if constexpr (VN == 4) {
                            a[4 * v] = x.x; a[4 * v + 1] = x.y; a[4 * v + 2] = x.z; a[4 * v + 3] = x.w;
                        } else {
                            a[2 * v] = x.x; a[2 * v + 1] = x.y;
                        }
                    }
                    T b[CPL];
#pragma unroll
                    for (int j = 0; j < CPL; ++j) b[j] = Bs[(kc + kk) * (NT + 1) + lane + 32 * j];
#pragma unroll
                    for (int i = 0; i < kRowsPerWarp; ++i)
#pragma unroll
                        for (int j = 0; j < CPL; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
                }
            }
        }
        if (active) {
#pragma unroll
            for (int i = 0; i < kRowsPerWarp; ++i) {
                const int m = mc + kRowsPerWarp * warp + i;
                if (m < M) {
#pragma unroll
                    for (int j = 0; j < CPL; ++j) {
                        const int c = lane + 32 * j;
                        if (OUT_MODE == 0) Out[c * ldo + m] = acc[i][j];
                        else Out[m * ldo + c] = acc[i][j];
                    }
                }
            }
        }
    }
    __syncthreads();
}

template <typename TO, typename T>
__device__ __forceinline__ void atomic_add_out(TO *addr, T v);
template <> __device__ __forceinline__ void atomic_add_out<float, float>(float *a, float v) { atomicAdd(a, v); }
template <> __device__ __forceinline__ void atomic_add_out<double, float>(double *a, float v) { atomicAdd(a, (double)v); }
template <> __device__ __forceinline__ void atomic_add_out<double, double>(double *a, double v) { atomicAdd(a, v); }

// LOWRANK = false: A1 = K_p^T layout [kpad][mpad].
// LOWRANK = true:  A1 = V_p layout [kpad][rpad], A2 = (U_p Sigma_p)^T layout [rpad][mpad].
template <typename T, typename TO, int NT, bool LOWRANK>
__global__ void __launch_bounds__(kThreads)
simt_apply_kernel(const int2 *__restrict__ rec, const int *__restrict__ class_off,
                  const T *__restrict__ A1, const T *__restrict__ A2, const int16_t *__restrict__ sigma,
                  const T *__restrict__ mp, TO *__restrict__ out, int n3, int kpad, int mpad, int rpad,
                  double scale)
{
    constexpr int KC = kc_of<T>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *As = reinterpret_cast<T *>(smem_raw);                   // [KC][128]
    T *Bs = As + KC * 128;                                     // [kpad][NT + 1]
    const size_t bs_elems = (size_t)kpad * (NT + 1);
    const size_t cs_elems = (size_t)NT * (mpad + 1);
    T *Cs = LOWRANK ? Bs : Bs + bs_elems;                      // [NT][mpad + 1]
    T *Zs = LOWRANK ? Bs + (bs_elems > cs_elems ? bs_elems : cs_elems) : nullptr;  // [rpad][NT + 1]
    int2 *recs = reinterpret_cast<int2 *>(LOWRANK ? Zs + (size_t)rpad * (NT + 1) : Cs + cs_elems);
    __shared__ int tile_start[17];

    if (threadIdx.x == 0) {
        int acc = 0;
        for (int p = 0; p < 16; ++p) {
            tile_start[p] = acc;
            acc += (class_off[p + 1] - class_off[p] + NT - 1) / NT;
        }
        tile_start[16] = acc;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    const int ntiles = tile_start[16];

    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        int p = 0;
        while (p < 15 && tile >= tile_start[p + 1]) ++p;
        const int col0 = class_off[p] + (tile - tile_start[p]) * NT;
        const int nc = min(NT, class_off[p + 1] - col0);
        for (int c = threadIdx.x; c < NT; c += kThreads) recs[c] = (c < nc) ? rec[col0 + c] : make_int2(0, 0);
        // rows n3..kpad-1 of the panel stay zero
        for (int idx = threadIdx.x; idx < (kpad - n3) * (NT + 1); idx += kThreads) Bs[n3 * (NT + 1) + idx] = T(0);
        __syncthreads();
        // a4: gather + permute, one warp per column
        for (int c = warp; c < NT; c += kThreads / 32) {
            if (c < nc) {
                const int2 r = recs[c];
                const int g = rec_g(r.y);
                const T *w = mp + (size_t)r.x * n3;
                const int16_t *sg = sigma + g * n3;
                for (int b = lane; b < n3; b += 32) Bs[sg[b] * (NT + 1) + c] = w[b];
            } else {
                for (int b = lane; b < n3; b += 32) Bs[b * (NT + 1) + c] = T(0);
            }
        }
        __syncthreads();
        // a5: the operator product(s)
        if (!LOWRANK) {
            gemm_chunked<T, NT, 0>(A1 + (size_t)p * kpad * mpad, mpad, kpad, n3, Bs, As, Cs, mpad + 1);
        } else {
            gemm_chunked<T, NT, 1>(A1 + (size_t)p * kpad * rpad, rpad, kpad, rpad, Bs, As, Zs, NT + 1);
            gemm_chunked<T, NT, 0>(A2 + (size_t)p * rpad * mpad, mpad, rpad, n3, Zs, As, Cs, mpad + 1);
        }
        // a6: un-permute, segmented sum over the columns of one target, atomic add
        for (int a = threadIdx.x; a < n3; a += kThreads) {
            T acc = T(0);
            int cur = rec_tgt(recs[0].y);
            for (int c = 0; c < nc; ++c) {
                const int2 r = recs[c];
                const int tgt = rec_tgt(r.y);
                const int g = rec_g(r.y);
                if (tgt != cur) {
                    atomic_add_out<TO, T>(out + (size_t)cur * n3 + a, (T)(acc * (T)scale));
                    acc = T(0);
                    cur = tgt;
                }
                acc += Cs[c * (mpad + 1) + sigma[g * n3 + a]];
            }
            atomic_add_out<TO, T>(out + (size_t)cur * n3 + a, (T)(acc * (T)scale));
        }
        __syncthreads();
    }
}

// Shared memory of one launch configuration (must match the kernel's carve-up).
template <typename T, int NT, bool LOWRANK>
size_t simt_smem(const m2l_ops *ops)
{
    const int n3 = ops->n3, kpad = simt_kpad(n3), mpad = simt_mpad(n3);
    const int rpad = LOWRANK ? simt_rpad(ops->rmax) : 0;
    const size_t bs = (size_t)kpad * (NT + 1), cs = (size_t)NT * (mpad + 1);
    size_t elems = (size_t)kc_of<T>() * 128;
    if (LOWRANK) elems += (bs > cs ? bs : cs) + (size_t)rpad * (NT + 1);
    else elems += bs + cs;
    return elems * sizeof(T) + NT * sizeof(int2);
}

template <typename T, typename TO, int NT, bool LOWRANK>
m2l_status launch_one(const m2l_ops *ops, const Buckets &b, const T *A1, const T *A2, const T *in, TO *out,
                      double scale, cudaStream_t s)
{
    const int n3 = ops->n3, kpad = simt_kpad(n3), mpad = simt_mpad(n3);
    const int rpad = LOWRANK ? simt_rpad(ops->rmax) : 0;
    const size_t smem = simt_smem<T, NT, LOWRANK>(ops);
    if ((int)smem > max_smem_optin()) {
        set_error("order %d needs %zu bytes of shared memory in the SIMT kernel", ops->ell, smem);
        return M2L_EUNSUPPORTED;
    }
    auto kern = simt_apply_kernel<T, TO, NT, LOWRANK>;
    M2L_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    M2L_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
    if (per_sm < 1) per_sm = 1;
    const long tiles_bound = (long)(b.nnz + NT - 1) / NT + 16;
    long grid = (long)num_sms() * per_sm;
    if (grid > tiles_bound) grid = tiles_bound;
    if (grid < 1) grid = 1;
    kern<<<(int)grid, kThreads, smem, s>>>(b.rec.as<int2>(), b.class_off.as<int>(), A1, A2,
                                           ops->sigma.as<int16_t>(), in, out, n3, kpad, mpad, rpad, scale);
    M2L_LAUNCH_CHECK("simt_apply_kernel");
    return M2L_OK;
}

}  // namespace

template <typename TO, bool LOWRANK>
static m2l_status launch_f32(const m2l_ops *ops, const Buckets &b, const Layout &L, const void *in, void *out,
                             double scale, cudaStream_t s)
{
    // 64 columns per tile when the panel and the product fit, else 32
    if ((int)simt_smem<float, 64, LOWRANK>(ops) <= max_smem_optin())
        return launch_one<float, TO, 64, LOWRANK>(ops, b, L.a.as<float>(), L.b.as<float>(), (const float *)in,
                                                  (TO *)out, scale, s);
    return launch_one<float, TO, 32, LOWRANK>(ops, b, L.a.as<float>(), L.b.as<float>(), (const float *)in,
                                              (TO *)out, scale, s);
}

m2l_status launch_simt(const m2l_ops *ops, const Buckets &b, const void *in, void *out, int precision,
                       int out_fp64, double scale, cudaStream_t s)
{
    const bool fp64 = (precision == M2L_FP64);
    m2l_status st = prepare_simt_layout(ops, fp64 ? 1 : 0, s);
    if (st != M2L_OK) return st;
    if (b.nnz == 0) return M2L_OK;
    const bool lr = ops->eps > 0;
    if (fp64) {
        const Layout &L = lr ? ops->lr64 : ops->simt64;
        if (lr)
            return launch_one<double, double, 32, true>(ops, b, L.a.as<double>(), L.b.as<double>(),
                                                        (const double *)in, (double *)out, scale, s);
        return launch_one<double, double, 32, false>(ops, b, L.a.as<double>(), nullptr, (const double *)in,
                                                     (double *)out, scale, s);
    }
    const Layout &L = lr ? ops->lr32 : ops->simt32;
    if (out_fp64)
        return lr ? launch_f32<double, true>(ops, b, L, in, out, scale, s)
                  : launch_f32<double, false>(ops, b, L, in, out, scale, s);
    return lr ? launch_f32<float, true>(ops, b, L, in, out, scale, s)
              : launch_f32<float, false>(ops, b, L, in, out, scale, s);
}

}  // namespace m2l

namespace m2l {

// The FP32 full-rank SIMT kernel on caller-provided buckets and operator
// layout (no allocation).  Only the 64-column configuration is offered.
m2l_status launch_simt_f32_raw(const m2l_ops *ops, const int2 *rec, const int *class_off, int nnz, const float *KT,
                               const float *in, float *out, double scale, cudaStream_t s)
{
    if (nnz == 0) return M2L_OK;
    const int n3 = ops->n3, kpad = simt_kpad(n3), mpad = simt_mpad(n3);
    const size_t smem = simt_smem<float, 64, false>(ops);
    if ((int)smem > max_smem_optin()) {
        set_error("order %d needs %zu bytes of shared memory in the SIMT kernel", ops->ell, smem);
        return M2L_EUNSUPPORTED;
    }
    auto kern = simt_apply_kernel<float, float, 64, false>;
    M2L_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    M2L_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
    if (per_sm < 1) per_sm = 1;
    long grid = (long)num_sms() * per_sm;
    const long tiles_bound = (long)(nnz + 63) / 64 + 16;
    if (grid > tiles_bound) grid = tiles_bound;
    kern<<<(int)grid, kThreads, smem, s>>>(rec, class_off, KT, nullptr, ops->sigma.as<int16_t>(), in, out, n3, kpad,
                                           mpad, 0, scale);
    M2L_LAUNCH_CHECK("simt_apply_kernel");
    return M2L_OK;
}

}  // namespace m2l

// ---------------------------------------------------------------------------
// Batched apply: many (operator set, level) problems in one persistent launch.
namespace m2l {


namespace {

template <typename T, int NT>
__global__ void __launch_bounds__(kThreads)
simt_batch_kernel(const BatchDesc *__restrict__ descs, int nprob, int total_tiles)
{
    constexpr int KC = kc_of<T>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_base[1025];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool base_in_smem = nprob <= 1024;
    if (base_in_smem)
        for (int i = threadIdx.x; i < nprob; i += kThreads) s_base[i] = descs[i].tile_base;
    __syncthreads();
    for (int tile = blockIdx.x; tile < total_tiles; tile += gridDim.x) {
        // problem owning the tile: last problem whose tile_base <= tile
        int lo = 0, hi = nprob - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            const int b = base_in_smem ? s_base[mid] : descs[mid].tile_base;
            if (b <= tile) lo = mid; else hi = mid - 1;
        }
        const BatchDesc &d = descs[lo];
        const int lt = tile - d.tile_base;
        int p = 0;
        while (p < 15 && lt >= d.tile_start[p + 1]) ++p;
        const int col0 = d.class_off[p] + (lt - d.tile_start[p]) * NT;
        const int nc = min(NT, d.class_off[p + 1] - col0);
        const int n3 = d.n3, kpad = d.kpad, mpad = d.mpad;
        T *As = reinterpret_cast<T *>(smem_raw);                   // [KC][128]
        T *Bs = As + KC * 128;                                     // [kpad][NT + 1]
        T *Cs = Bs + (size_t)kpad * (NT + 1);                      // [NT][mpad + 1]
        int2 *recs = reinterpret_cast<int2 *>(Cs + (size_t)NT * (mpad + 1));
        const T *mp = static_cast<const T *>(d.in);
        for (int c = threadIdx.x; c < NT; c += kThreads) recs[c] = (c < nc) ? d.rec[col0 + c] : make_int2(0, 0);
        for (int idx = threadIdx.x; idx < (kpad - n3) * (NT + 1); idx += kThreads) Bs[n3 * (NT + 1) + idx] = T(0);
        __syncthreads();
        for (int c = warp; c < NT; c += kThreads / 32) {
            if (c < nc) {
                const int2 r = recs[c];
                const T *w = mp + (size_t)r.x * n3;
                const int16_t *sg = d.sigma + rec_g(r.y) * n3;
                for (int b = lane; b < n3; b += 32) Bs[sg[b] * (NT + 1) + c] = w[b];
            } else {
                for (int b = lane; b < n3; b += 32) Bs[b * (NT + 1) + c] = T(0);
            }
        }
        __syncthreads();
        gemm_chunked<T, NT, 0>(static_cast<const T *>(d.A) + (size_t)p * kpad * mpad, mpad, kpad, n3, Bs, As, Cs,
                               mpad + 1);
        for (int a = threadIdx.x; a < n3; a += kThreads) {
            T acc = T(0);
            int cur = rec_tgt(recs[0].y);
            for (int c = 0; c < nc; ++c) {
                const int2 r = recs[c];
                const int tgt = rec_tgt(r.y);
                if (tgt != cur) {
                    if (d.out_fp64) atomicAdd(static_cast<double *>(d.out) + (size_t)cur * n3 + a, (double)acc * d.scale);
                    else atomicAdd(static_cast<float *>(d.out) + (size_t)cur * n3 + a, (float)(acc * (T)d.scale));
                    acc = T(0);
                    cur = tgt;
                }
                acc += Cs[c * (mpad + 1) + d.sigma[rec_g(r.y) * n3 + a]];
            }
            if (d.out_fp64) atomicAdd(static_cast<double *>(d.out) + (size_t)cur * n3 + a, (double)acc * d.scale);
            else atomicAdd(static_cast<float *>(d.out) + (size_t)cur * n3 + a, (float)(acc * (T)d.scale));
        }
        __syncthreads();
    }
}

}  // namespace

size_t batch_smem_bytes(int fp64, int nt, int kpad_max, int mpad_max)
{
    const size_t esz = fp64 ? sizeof(double) : sizeof(float);
    const size_t kc = fp64 ? 16 : 32;
    return (kc * 128 + (size_t)kpad_max * (nt + 1) + (size_t)nt * (mpad_max + 1)) * esz + nt * sizeof(int2);
}

// One persistent launch over all problems of the table.
m2l_status launch_simt_batch(const BatchDesc *descs, int nprob, int total_tiles, int fp64, int nt, int kpad_max,
                             int mpad_max, cudaStream_t s)
{
    if (total_tiles == 0) return M2L_OK;
    const size_t smem = batch_smem_bytes(fp64, nt, kpad_max, mpad_max);
    if ((int)smem > max_smem_optin()) {
        set_error("batched SIMT kernel needs %zu bytes of shared memory", smem);
        return M2L_EUNSUPPORTED;
    }
    void (*kern)(const BatchDesc *, int, int);
    if (fp64) kern = simt_batch_kernel<double, 32>;
    else if (nt == 64) kern = simt_batch_kernel<float, 64>;
    else kern = simt_batch_kernel<float, 32>;
    M2L_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    M2L_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
    if (per_sm < 1) per_sm = 1;
    long grid = (long)num_sms() * per_sm;
    if (grid > total_tiles) grid = total_tiles;
    kern<<<(int)grid, kThreads, smem, s>>>(descs, nprob, total_tiles);
    M2L_LAUNCH_CHECK("simt_batch_kernel");
    return M2L_OK;
}

}  // namespace m2l
