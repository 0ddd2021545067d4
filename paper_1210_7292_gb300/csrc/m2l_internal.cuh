// Internal declarations of the M2L library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <initializer_list>
#include <string>

#include "../../include/m2l.h"

struct m2l_ops;

namespace m2l {

// Device status word bits, set by kernels with atomicOr.
enum : int {
    ST_BAD_PAIR = 1,      // a list entry whose t is not a far-field transfer vector
    ST_BAD_INDEX = 2,     // a source/target index or CSR offset out of range
    ST_TIMEOUT = 4,       // a bounded wait gave up
    ST_BAD_TABLE = 8      // a table lookup outside its range
};

constexpr int kMaxEll = 8;
constexpr int kNumSym = 16;     // |T_sym| for the bbFMM (Sec. 4.2.1)
constexpr int kNumPerm = 48;    // signed axis permutations
constexpr int kTgtBits = 26;    // record packing: tgt | g << 26
constexpr int kSegEntries = 2048;  // entries per block segment of the stable bucketing

// Bucketed record .y field: target index in the low 26 bits, permutation
// index g (< 48) in the high 6 bits.  Unpacked with unsigned shifts: g >= 32
// sets the sign bit of the int.
__host__ __device__ __forceinline__ int rec_pack(int tgt, int g)
{
    return (int)((unsigned)tgt | ((unsigned)g << kTgtBits));
}
__host__ __device__ __forceinline__ int rec_tgt(int y) { return (int)((unsigned)y & ((1u << kTgtBits) - 1u)); }
__host__ __device__ __forceinline__ int rec_g(int y)
{
    const int g = (int)((unsigned)y >> kTgtBits);
    return g < kNumPerm ? g : kNumPerm - 1;   // never taken for records written by the classifier
}

void set_error(const char *fmt, ...);
// M2L_EINVAL unless the calling thread's current device is the one that built ops
m2l_status check_device(const m2l_ops *ops);
m2l_status cuda_fail(cudaError_t e, const char *what);
void count_launch(int n = 1);

#define M2L_CUDA(call)                                                   \
    do {                                                                 \
        cudaError_t e_ = (call);                                         \
        if (e_ != cudaSuccess) return ::m2l::cuda_fail(e_, #call);       \
    } while (0)

#define M2L_LAUNCH_CHECK(what)                                           \
    do {                                                                 \
        ::m2l::count_launch();                                           \
        cudaError_t e_ = cudaGetLastError();                             \
        if (e_ != cudaSuccess) return ::m2l::cuda_fail(e_, what);        \
    } while (0)

// A device buffer that only grows.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    m2l_status ensure(size_t need);
    void release();
    template <typename T> T *as() const { return static_cast<T *>(p); }
};

// Releases scratch buffers on every return path of the scope that declares it
// (cudaFree synchronises with the device, so work using them has finished).
struct ScratchGuard {
    DevBuf *bufs[24];
    int n = 0;
    ScratchGuard(std::initializer_list<DevBuf *> l)
    {
        for (DevBuf *b : l)
            if (n < 24) bufs[n++] = b;
    }
    ~ScratchGuard()
    {
        for (int i = 0; i < n; ++i) bufs[i]->release();
    }
    ScratchGuard(const ScratchGuard &) = delete;
    ScratchGuard &operator=(const ScratchGuard &) = delete;
};

// Output of the dense classification (step a3 for full levels, used by the
// target-stationary tensor-core kernel): targets grouped by the octant of
// their cell into units of at most nu columns; per unit and transfer-vector
// slot (the 343-entry index of t), the source of every column.
struct DenseBuckets {
    DevBuf unit_tgt;   // int32 [umax][nu]: target index of each column, -1 for padding
    DevBuf tab;        // int32 [umax][343][nu]: source index + 1 of each column and slot, 0 = none
    DevBuf slots;      // uint16 [umax][344]: [0] number of active slots, then the slots ascending
    DevBuf meta;       // int32 [64]: [0] = number of units; per octant counts, starts, unit offsets
    DevBuf work;       // int32 scratch: per-target ranks and (unit, column), block counts, slot flags
    DevBuf bsplit;     // split multipoles [nsrc + 1][parts][kpad] of the last apply (row nsrc = 0)
    int umax = 0, nu = 0, ntgt = 0, nsrc = 0, nnz = 0;
    bool valid = false;
    void release()
    {
        unit_tgt.release(); tab.release(); slots.release(); meta.release(); work.release(); bsplit.release();
        valid = false;
    }
};

// Output of the classification and bucketing (step a3).
struct Buckets {
    DevBuf rec;        // int2 [nnz]: .x = source index, .y = target | g << 26, bucketed
    DevBuf tgt_of;     // int32 [nnz] target of each list entry (scratch)
    DevBuf code;       // uint16 [nnz] p | g << 8, or 0xFFFF for a rejected entry (scratch)
    DevBuf seg;        // int32 [17][nseg] per-segment counts, then positions (scratch)
    DevBuf class_off;  // int32 [18]: start of bucket p at [p], [16] = valid total, [17] = nnz
    // adjoint: transposed list (scratch)
    DevBuf t_off, t_src, t_cursor;
    DevBuf lrz;           // float [nnz][128]: first-pass products of the tensor-core low-rank apply
    DenseBuckets dense;   // filled instead of the buckets for full levels that the dense kernel serves
    mutable bool have_rec = true;   // rec/class_off hold the buckets (else derived from dense on demand)
    int nnz = 0;
    int ntgt = 0;
    int nsrc = 0;
};

// Operand layouts prepared for one precision (built on first use).
struct Layout {
    DevBuf a;      // operator matrices in the kernel's layout
    DevBuf b;      // second operand set (low rank V, or lo parts)
    bool ready = false;
};

}  // namespace m2l

struct m2l_ops {
    int kind = 0;
    double c = 0.0;
    int ell = 0, n3 = 0;
    double eps = 0.0;
    double ref_width = 1.0;
    int hom_degree = 0;       // 0 when not homogeneous
    int homogeneous = 0;
    int device = 0;
    int ranks[16] = {0};
    int rmax = 0;
    m2l::DevBuf K64;          // double [16][n3][n3]
    m2l::DevBuf sigma;        // int16 [48][n3]
    m2l::DevBuf lut;          // uint16 [343]
    m2l::DevBuf tsym;         // int32 [16][3]
    m2l::DevBuf U64, V64;     // double [16][n3][rmax] (low rank; zero-padded columns)
    m2l::Layout simt64, simt32, lr64, lr32, tc_tf32, tc_bf16x3, tc_tf32x3;
    m2l::Layout tcd_tf32, tcd_bf16x3, tcd_tf32x3;   // per-slot operator images of the dense kernel
    m2l::Layout lrtc_tf32, lrtc_bf16x3, lrtc_tf32x3; // low-rank factor images of the tensor-core apply
    mutable m2l::Buckets ws;  // workspace of m2l_apply_level
    mutable double ws_scale = 1.0;  // scale of the level last classified into ws
    int trunc = M2L_TRUNC_FROBENIUS;  // truncation criterion (m2l_truncation)
    int lowrank_method = 0;   // 0: truncated SVD, 1: ACA + truncated SVD
    int aca_terms[16] = {0};  // ACA terms before the recompression (method 1)
    int jacobi_sweeps[16] = {0};  // sweeps of each operator's (method 0) or core's (method 1) SVD
    int *d_status = nullptr;  // device status word
    int debug_flags = 0;      // M2L_DEBUG_* test switches
};

struct m2l_plan {
    const m2l_ops *ops = nullptr;
    int adjoint = 0;
    double width = 0.0;
    int n_out = 0, n_in = 0;
    m2l::Buckets b;
};

namespace m2l {

// One-sided Jacobi SVD of nb column-major m x n matrices (m >= n), in place
// (m2l_svd.cu): A <- A V with orthogonal columns, V [nb][n][n] (column-major,
// may be null) the accumulated rotations, sigma [nb][n] the column norms
// (unsorted), sweeps [nb] (host, may be null).  Synchronises the stream.
m2l_status jacobi_svd(double *A, int m, int n, int nb, double *V, double *sigma, int *sweeps, cudaStream_t s);
// order[0..n) = indices of sig by descending value (stable).
void order_descending(const double *sig, int n, int *order);
// Truncation rank of s (descending, length n) at accuracy eps under the
// m2l_truncation criterion trunc; n for eps <= 0.
int truncation_rank(const double *s, int n, double eps, int trunc);

// Precompute (m2l_tables.cu)
m2l_status build_tables(m2l_ops *ops, cudaStream_t s);
m2l_status assemble_operators(m2l_ops *ops, cudaStream_t s);
m2l_status lowrank_factors(m2l_ops *ops);
m2l_status lowrank_factors_aca(m2l_ops *ops, int *aca_terms, int *jacobi_sweeps);
m2l_status prepare_simt_layout(const m2l_ops *ops, int fp64, cudaStream_t s);
int simt_kpad(int n3);
int simt_mpad(int n3);
int simt_rpad(int r);

// Classification (m2l_classify.cu)
m2l_status classify(const m2l_ops *ops, const m2l_level *lv, int adjoint, Buckets &b, cudaStream_t s);
m2l_status launch_exclusive_scan(const int32_t *in, int32_t *out, int n, cudaStream_t s);

// Apply kernels
m2l_status launch_simt(const m2l_ops *ops, const Buckets &b, const void *in, void *out, int precision,
                       int out_fp64, double scale, cudaStream_t s);
m2l_status launch_tc(const m2l_ops *ops, const Buckets &b, const void *in, void *out, int precision,
                     int out_fp64, double scale, cudaStream_t s);

int num_sms();
int max_smem_optin();

// Dense classification and the target-stationary tensor-core apply (m2l_dense.cu).
bool dense_eligible(const m2l_ops *ops, int ntgt, int nnz);
m2l_status dense_classify(const m2l_ops *ops, int ntgt, int nsrc, int nnz, const int32_t *tgt_ijk,
                          const int32_t *src_ijk, const int32_t *offsets, const int32_t *sources, DenseBuckets &d,
                          cudaStream_t s);
m2l_status dense_prepare(const m2l_ops *ops, int precision, cudaStream_t s);
m2l_status launch_tc_dense(const m2l_ops *ops, const DenseBuckets &d, int precision, const float *in, void *out,
                           int out_fp64, double scale, cudaStream_t s);
// Low-rank products on the tensor cores (m2l_lowrank_tc.cu), two passes of the
// large-order kernel; eps > 0, ell 5-7, ranks <= 128.
constexpr int kLrRankPad = 128;
m2l_status launch_tc_lowrank(const m2l_ops *ops, const Buckets &b, int precision, const float *in, void *out,
                             int out_fp64, double scale, cudaStream_t s);

// Fill b.rec / b.class_off from the dense classification if they are not built
// (stream-ordered, no allocation).
m2l_status ensure_records(const m2l_ops *ops, const Buckets &b, cudaStream_t s);

// General tensor-core apply (the large-order kernel over ncls operator images
// of vector length N <= 256; used by the directional M2L).  tc_general_config
// gives the padded K length of the inverse-permutation tables, the image bytes
// per operator and the interactions per tile; tc_general_images builds the images from row-major FP64
// operators [ncls][N][N]; tc_general_apply adds into out.
bool tc_general_config(int precision, int N, int *kpad, size_t *img_bytes_per_op, int *tile_cols);
m2l_status tc_general_images(int precision, int N, int ncls, const double *K, uint8_t *img, cudaStream_t s);
m2l_status tc_general_apply(int precision, int N, int ncls, const int *tile_start, const int2 *rec,
                            const int *class_off, const uint8_t *img, const int16_t *tinv, int nnz, const float *in,
                            float *out, int *status, cudaStream_t s);

// Persistent batches on the tensor cores (m2l_batch_tc.cu): per vector length one
// launch of the large-order kernel over all problems' (problem, operator) classes.
struct TcBatch;
m2l_status tc_batch_create(const m2l_plan *const *plans, int nbatch, const void *const *in, void *const *out,
                           int precision, cudaStream_t s, TcBatch **out_batch);
m2l_status tc_batch_run(const TcBatch *b, cudaStream_t s);
void tc_batch_info(const TcBatch *b, int *tile_width, int64_t *tiles, double *tuned_ms, int *epilogue_groups,
                   int *launches);
int tc_batch_groups(const TcBatch *b, int max, int *n3, int *tile_width, int *epilogue_groups);
void tc_batch_free(TcBatch *b);

// One problem of a batched persistent launch (host-built, copied to the device).
struct BatchDesc {
    const int2 *rec;          // bucketed records of the problem
    const void *A;            // transposed operator layout [16][kpad][mpad] (float or double)
    const int16_t *sigma;     // permutation tables [48][n3]
    const void *in;           // input vectors [n_in][n3]
    void *out;                // output vectors [n_out][n3] (accumulated)
    double scale;             // w^degree for homogeneous kernels, else 1
    int n3, kpad, mpad, out_fp64;
    int class_off[17];        // bucket offsets (from the plan)
    int tile_start[17];       // first tile of each bucket within the problem
    int tile_base;            // first global tile of the problem
    int pad_;
};

}  // namespace m2l
