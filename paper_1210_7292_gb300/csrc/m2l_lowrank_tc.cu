// Step a5 with the per-operator low-rank factors (Eq. (20), K_p ~ U_p Sigma_p
// V_p^T, the IA variant of Sec. 4.2 blocked by Alg. 2) on the tcgen05 tensor
// cores: two passes of the large-order kernel over the same operator buckets.
//
//   pass 1: Z = V_p^T W_p   -- gather and permute the source vectors exactly as
//           the full-rank product (Eq. (30)); the product (rank rows, padded to
//           128) of every record is stored unpermuted, one row of Z per record;
//   pass 2: F = (U_p Sigma_p) Z -- the panel is Z's rows of the tile's records
//           (gathered through an identity table), K = the padded rank; then the
//           un-permutation f[a] += F[sigma_g(a)] (Eq. (32)), the sum over a
//           target's consecutive records and one atomic add per (target, node)
//           and run, as the full-rank kernel does.
//
// Per 64-record tile each pass streams 6 operator blocks of 128 x 128 bytes
// (for ell = 7 in BF16x3: V_p^T is one M tile x 6 K columns, U_p Sigma_p three
// M tiles x 2 K columns), a third of the 18 blocks of the full-rank operator
// per 32 records: the large-order kernel is bound by that operator stream.
// The ranks r_p <= 128 are padded to 128 with zero rows (pass 1) and columns
// (pass 2) of the factor images.
#include "m2l_tc_big.cuh"

namespace m2l {
namespace {

// Factor images in the (M tile, K column) block layout of the large-order
// kernel: for operator p, A[row][k] = src[p][k][row] (transpose = 1, the
// V_p^T of pass 1, src = V [16][n3][ld]) or src[p][row][k] (transpose = 0,
// U_p Sigma_p of pass 2, src = U [16][n3][ld]); zero outside rows x cols.
template <int KIND>
__global__ void lr_image_kernel(int rows, int cols, int ld, int n3, int MT, int KA, int transpose,
                                const double *__restrict__ src, uint8_t *__restrict__ img)
{
    using Tr = TcTraits<KIND>;
    constexpr int E = 128 / Tr::esz;
    const int block_bytes = 128 * 128 * Tr::nparts;
    const int p = blockIdx.y;
    const long per_op = (long)MT * 128 * KA * E;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < per_op; idx += (long)gridDim.x * blockDim.x) {
        const int rowg = (int)(idx / (KA * E)), kk = (int)(idx % (KA * E));
        const int mt = rowg / 128, row = rowg % 128, ka = kk / E, e = kk % E;
        double x = 0.0;
        if (rowg < rows && kk < cols)
            x = transpose ? src[((size_t)p * n3 + kk) * ld + rowg] : src[((size_t)p * n3 + rowg) * ld + kk];
        const int chunk = e / (16 / Tr::esz), within = e % (16 / Tr::esz);
        uint8_t *blk = img + ((size_t)(p * MT + mt) * KA + ka) * block_bytes;
        const uint32_t off = swz_off(row, chunk) + (uint32_t)(within * Tr::esz);
        if constexpr (KIND == TC_BF16X3) {
            const __nv_bfloat16 h = __double2bfloat16(x);
            const __nv_bfloat16 l = __double2bfloat16(x - (double)__bfloat162float(h));
            *reinterpret_cast<__nv_bfloat16 *>(blk + off) = h;
            *reinterpret_cast<__nv_bfloat16 *>(blk + 128 * 128 + off) = l;
        } else if constexpr (KIND == TC_TF32) {
            *reinterpret_cast<float *>(blk + off) = tf32_rna((float)x);
        } else {
            const float h = tf32_rna((float)x);
            const float l = tf32_rna((float)(x - (double)h));
            *reinterpret_cast<float *>(blk + off) = h;
            *reinterpret_cast<float *>(blk + 128 * 128 + off) = l;
        }
    }
}

// inv[g][b'] for the un-permutation of pass 2 (rows padded to `stride`), and
// the identity table [48][kpad] of its gather.
__global__ void lr_tables_kernel(int n3, int stride, int kpad, const int16_t *__restrict__ sigma,
                                 int16_t *__restrict__ inv, int16_t *__restrict__ ident)
{
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < 48 * n3; idx += gridDim.x * blockDim.x) {
        const int g = idx / n3, b = idx % n3;
        inv[g * stride + sigma[idx]] = (int16_t)b;
    }
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < 48 * kpad; idx += gridDim.x * blockDim.x)
        ident[idx] = (int16_t)(idx % kpad);
}

// Shapes per order: pass 1 (M tiles 1, K columns over ell^3), pass 2 (M tiles
// over ell^3, K columns over the padded rank).
template <int KIND, int ELL3>
struct LrShape {
    static constexpr int E = 128 / TcTraits<KIND>::esz;
    static constexpr int KA1 = (ELL3 + E - 1) / E;
    static constexpr int MT2 = (ELL3 + 127) / 128;
    static constexpr int KA2 = kLrRankPad / E;
};

template <int KIND, int MT, int KA, int MODE>
constexpr int lr_nt()
{
    return BigCfg<KIND, MT, KA, 64, MODE == 1 ? 1 : 2>::SMEM <= 225 * 1024 ? 64 : 32;
}

template <int KIND, int MT, int KA, int MODE>
m2l_status launch_pass(const m2l_ops *ops, const Buckets &b, const uint8_t *img, const int16_t *sinv,
                       const int16_t *sinv_prod, const float *in, float *out_f32, double *out_f64, int n_out, int n_in,
                       double scale, cudaStream_t s)
{
    constexpr int NT = lr_nt<KIND, MT, KA, MODE>();
    constexpr int EG = MODE == 1 ? 1 : 2;
    using C = BigCfg<KIND, MT, KA, NT, EG>;
    if (C::SMEM > max_smem_optin()) {
        set_error("low-rank tensor-core pass needs %d bytes of shared memory", C::SMEM);
        return M2L_EUNSUPPORTED;
    }
    auto kern = tc_big_kernel<KIND, MT, KA, NT, EG, MODE>;
    M2L_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    long grid = num_sms();
    const long tiles_bound = (long)(b.nnz + NT - 1) / NT + 16;
    if (grid > tiles_bound) grid = tiles_bound;
    kern<<<(int)grid, big_threads(EG), C::SMEM, s>>>(b.rec.as<int2>(), b.class_off.as<int>(), img, sinv, in, out_f32,
                                                     out_f64, n_out, (float)scale, ops->d_status,
                                                     (ops->debug_flags & M2L_DEBUG_STALL_PRODUCER) ? 1 : 0, kNumSym,
                                                     nullptr, nullptr, n_in, sinv_prod);
    M2L_LAUNCH_CHECK("tc_big_kernel");
    return M2L_OK;
}

template <int KIND>
Layout &lr_layout(const m2l_ops *ops)
{
    m2l_ops *o = const_cast<m2l_ops *>(ops);
    return KIND == TC_TF32 ? o->lrtc_tf32 : KIND == TC_BF16X3 ? o->lrtc_bf16x3 : o->lrtc_tf32x3;
}

template <int KIND, int ELL3>
m2l_status launch_lr(const m2l_ops *ops, const Buckets &b, const float *in, void *out, int out_fp64, double scale,
                     cudaStream_t s)
{
    using Tr = TcTraits<KIND>;
    using S = LrShape<KIND, ELL3>;
    constexpr int E = S::E;
    const int n3 = ops->n3;
    const size_t blk = (size_t)128 * 128 * Tr::nparts;
    const size_t img1 = (size_t)16 * 1 * S::KA1 * blk, img2 = (size_t)16 * S::MT2 * S::KA2 * blk;
    const int kpad1 = S::KA1 * E, stride2 = S::MT2 * 128, kpad2 = S::KA2 * E;
    Layout &L = lr_layout<KIND>(ops);
    m2l_status st;
    if (!L.ready) {
        if ((st = L.a.ensure(img1 + img2)) != M2L_OK) return st;
        if ((st = L.b.ensure((size_t)48 * (kpad1 + stride2 + kpad2) * sizeof(int16_t))) != M2L_OK) return st;
        M2L_CUDA(cudaMemsetAsync(L.b.p, 0, (size_t)48 * (kpad1 + stride2 + kpad2) * sizeof(int16_t), s));
        const int rmax = ops->rmax;
        dim3 g1((unsigned)((128L * S::KA1 * E + 255) / 256), 16), g2((unsigned)((S::MT2 * 128L * S::KA2 * E + 255) / 256), 16);
        lr_image_kernel<KIND><<<g1, 256, 0, s>>>(rmax, n3, rmax, n3, 1, S::KA1, 1, ops->V64.as<double>(),
                                                 L.a.as<uint8_t>());
        M2L_LAUNCH_CHECK("lr_image_kernel");
        lr_image_kernel<KIND><<<g2, 256, 0, s>>>(n3, rmax, rmax, n3, S::MT2, S::KA2, 0, ops->U64.as<double>(),
                                                 L.a.as<uint8_t>() + img1);
        M2L_LAUNCH_CHECK("lr_image_kernel");
        int16_t *t1 = L.b.as<int16_t>(), *t2 = t1 + 48 * kpad1, *t3 = t2 + 48 * stride2;
        sigma_inverse_padded_kernel<<<(48 * n3 + 255) / 256, 256, 0, s>>>(n3, kpad1, ops->sigma.as<int16_t>(), t1);
        M2L_LAUNCH_CHECK("sigma_inverse_padded_kernel");
        lr_tables_kernel<<<(48 * (n3 > kpad2 ? n3 : kpad2) + 255) / 256, 256, 0, s>>>(n3, stride2, kpad2,
                                                                                  ops->sigma.as<int16_t>(), t2, t3);
        M2L_LAUNCH_CHECK("lr_tables_kernel");
        L.ready = true;
    }
    if (b.nnz == 0) return M2L_OK;
    if (b.lrz.bytes < (size_t)b.nnz * kLrRankPad * sizeof(float)) {
        set_error("plan classified before its operators were low rank: no first-pass buffer");
        return M2L_EINVAL;
    }
    const int16_t *t1 = L.b.as<int16_t>(), *t2 = t1 + 48 * kpad1, *t3 = t2 + 48 * stride2;
    float *z = b.lrz.as<float>();
    st = launch_pass<KIND, 1, S::KA1, 1>(ops, b, L.a.as<uint8_t>(), t1, nullptr, in, z, nullptr, kLrRankPad, n3, 1.0,
                                         s);
    if (st != M2L_OK) return st;
    return launch_pass<KIND, S::MT2, S::KA2, 2>(ops, b, L.a.as<uint8_t>() + img1, t2, t3, z,
                                                out_fp64 ? nullptr : (float *)out, out_fp64 ? (double *)out : nullptr,
                                                n3, kLrRankPad, scale, s);
}

template <int KIND>
m2l_status launch_lr_kind(const m2l_ops *ops, const Buckets &b, const float *in, void *out, int out_fp64, double scale,
                          cudaStream_t s)
{
    switch (ops->ell) {
    case 5: return launch_lr<KIND, 125>(ops, b, in, out, out_fp64, scale, s);
    case 6: return launch_lr<KIND, 216>(ops, b, in, out, out_fp64, scale, s);
    case 7: return launch_lr<KIND, 343>(ops, b, in, out, out_fp64, scale, s);
    default:
        set_error("tensor-core low-rank products take ell 5-7, got %d", ops->ell);
        return M2L_EUNSUPPORTED;
    }
}

}  // namespace

m2l_status launch_tc_lowrank(const m2l_ops *ops, const Buckets &b, int precision, const float *in, void *out,
                             int out_fp64, double scale, cudaStream_t s)
{
    if (ops->rmax > kLrRankPad) {
        set_error("tensor-core low-rank products take ranks <= %d, got %d", kLrRankPad, ops->rmax);
        return M2L_EUNSUPPORTED;
    }
    switch (precision) {
    case M2L_TF32: return launch_lr_kind<TC_TF32>(ops, b, in, out, out_fp64, scale, s);
    case M2L_BF16X3: return launch_lr_kind<TC_BF16X3>(ops, b, in, out, out_fp64, scale, s);
    case M2L_TF32X3: return launch_lr_kind<TC_TF32X3>(ops, b, in, out, out_fp64, scale, s);
    default:
        set_error("not a tensor-core precision: %d", precision);
        return M2L_EINVAL;
    }
}

}  // namespace m2l
