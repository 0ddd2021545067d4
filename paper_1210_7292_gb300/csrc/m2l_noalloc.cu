// m2l_apply_level_noalloc: the FP32 level translation without any device
// allocation.  Its scratch memory (the interaction buckets of step a3 and the
// FP32 operator layout) lives in one file-scope device array instead of
// library-grown buffers.
#include <math.h>

#include <mutex>

#include "m2l_internal.cuh"

namespace m2l {

m2l_status bucket_raw(const m2l_ops *ops, int ntgt, int nsrc, int nnz, const int32_t *tgt_ijk,
                      const int32_t *src_ijk, const int32_t *offsets, const int32_t *sources, int2 *rec,
                      int32_t *tgt_of, uint16_t *code, int32_t *seg, int32_t *class_off, cudaStream_t s);
m2l_status launch_transpose_pad_f32(const m2l_ops *ops, float *KT, int kpad, int mpad, cudaStream_t s);
m2l_status launch_simt_f32_raw(const m2l_ops *ops, const int2 *rec, const int *class_off, int nnz, const float *KT,
                               const float *in, float *out, double scale, cudaStream_t s);

namespace {

constexpr size_t kNoallocMaxNnz = (size_t)1 << 19;   // 524,288 list entries
constexpr int kNoallocMaxEll = 6;
constexpr size_t kMaxSeg = (kNoallocMaxNnz + kSegEntries - 1) / kSegEntries;
constexpr size_t kKpadMax = 224, kMpadMax = 256;     // simt_kpad/simt_mpad of ell = 6 (216 nodes)

constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t kOffRec = 0;
constexpr size_t kOffTgt = align256(kOffRec + kNoallocMaxNnz * sizeof(int2));
constexpr size_t kOffCode = align256(kOffTgt + kNoallocMaxNnz * sizeof(int32_t));
constexpr size_t kOffSeg = align256(kOffCode + kNoallocMaxNnz * sizeof(uint16_t));
constexpr size_t kOffClass = align256(kOffSeg + 2 * (17 * kMaxSeg + 1) * sizeof(int32_t));
constexpr size_t kOffKT = align256(kOffClass + 18 * sizeof(int32_t));
constexpr size_t kScratchBytes = align256(kOffKT + 16 * kKpadMax * kMpadMax * sizeof(float));

// The scratch of every call on this device (about 10.7 MB).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device; looked up once
// per device (the host-side symbol is not a device address).
m2l_status scratch_address(unsigned char **out)
{
    int dev = 0;
    M2L_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device index %d beyond %d", dev, kMaxDevices);
        return M2L_EUNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_scratch_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_ptr[dev];
    return M2L_OK;
}

}  // namespace
}  // namespace m2l

using namespace m2l;

extern "C" m2l_status m2l_apply_level_noalloc(const m2l_ops *ops, const m2l_level *lv, const float *multipoles,
                                              float *locals, void *stream)
{
    if (!ops || !lv) { set_error("null ops or level"); return M2L_EINVAL; }
    // the scratch array is looked up on the current device, and the kernels read
    // the operators and tables of the device that built ops: the two must agree
    if (m2l_status st = check_device(ops)) return st;
    if (ops->ell > kNoallocMaxEll) {
        set_error("m2l_apply_level_noalloc supports ell <= %d, got %d", kNoallocMaxEll, ops->ell);
        return M2L_EUNSUPPORTED;
    }
    if (ops->eps > 0) { set_error("m2l_apply_level_noalloc takes full-rank operators only"); return M2L_EUNSUPPORTED; }
    if (lv->nnz < 0 || lv->ncells_tgt < 0 || lv->ncells_src < 0) { set_error("negative size"); return M2L_EINVAL; }
    if ((size_t)lv->nnz > kNoallocMaxNnz) {
        set_error("m2l_apply_level_noalloc takes at most %zu list entries, got %d", kNoallocMaxNnz, lv->nnz);
        return M2L_EINVAL;
    }
    if (lv->ncells_tgt >= (1 << kTgtBits) || lv->ncells_src >= (1 << kTgtBits)) {
        set_error("more than 2^26 cells in one level");
        return M2L_EUNSUPPORTED;
    }
    if (!(lv->width > 0.0) || !isfinite(lv->width)) { set_error("level width must be positive"); return M2L_EINVAL; }
    if (lv->nnz > 0 && (!lv->tgt_ijk || !lv->src_ijk || !lv->il_offsets || !lv->il_sources || !multipoles ||
                        !locals || lv->ncells_tgt == 0)) {
        set_error("null pointer with nnz > 0");
        return M2L_EINVAL;
    }
    double scale = 1.0;
    if (ops->homogeneous) {
        scale = pow(lv->width / ops->ref_width, (double)ops->hom_degree);
    } else if (fabs(lv->width - ops->ref_width) > 1e-12 * ops->ref_width) {
        set_error("level width differs from the operators' width (kernel is not homogeneous)");
        return M2L_EINVAL;
    }
    unsigned char *base = nullptr;
    m2l_status st = scratch_address(&base);
    if (st != M2L_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    int2 *rec = reinterpret_cast<int2 *>(base + kOffRec);
    int32_t *tgt_of = reinterpret_cast<int32_t *>(base + kOffTgt);
    uint16_t *code = reinterpret_cast<uint16_t *>(base + kOffCode);
    int32_t *seg = reinterpret_cast<int32_t *>(base + kOffSeg);
    int32_t *class_off = reinterpret_cast<int32_t *>(base + kOffClass);
    float *KT = reinterpret_cast<float *>(base + kOffKT);
    const int kpad = simt_kpad(ops->n3), mpad = simt_mpad(ops->n3);
    // every call rewrites the operator layout and the buckets it reads
    st = launch_transpose_pad_f32(ops, KT, kpad, mpad, s);
    if (st != M2L_OK) return st;
    st = bucket_raw(ops, lv->ncells_tgt, lv->ncells_src, lv->nnz, lv->tgt_ijk, lv->src_ijk, lv->il_offsets,
                    lv->il_sources, rec, tgt_of, code, seg, class_off, s);
    if (st != M2L_OK) return st;
    return launch_simt_f32_raw(ops, rec, class_off, lv->nnz, KT, multipoles, locals, scale, s);
}
