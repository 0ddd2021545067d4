// The C ABI of include/m2l.h: argument checking, ownership, dispatch.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <vector>

#include "m2l_internal.cuh"

namespace m2l {

static thread_local char g_err[1024] = "";
static std::atomic<long long> g_launches{0};

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

m2l_status cuda_fail(cudaError_t e, const char *what)
{
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? M2L_ENOMEM : M2L_ECUDA;
}

void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

m2l_status DevBuf::ensure(size_t need)
{
    if (need <= bytes && p) return M2L_OK;
    release();
    if (need == 0) need = 16;
    cudaError_t e = cudaMalloc(&p, need);
    if (e != cudaSuccess) {
        p = nullptr;
        bytes = 0;
        return cuda_fail(e, "cudaMalloc");
    }
    bytes = need;
    return M2L_OK;
}

void DevBuf::release()
{
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
}

int num_sms()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

int max_smem_optin()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return n;
}

static bool is_homogeneous(int kind, int *degree)
{
    if (kind == M2L_K_INV_R) { *degree = -1; return true; }
    if (kind == M2L_K_INV_R4) { *degree = -4; return true; }
    *degree = 0;
    return false;
}

m2l_status check_device(const m2l_ops *ops)
{
    int dev = -1;
    M2L_CUDA(cudaGetDevice(&dev));
    if (dev != ops->device) {
        set_error("the current device is %d, but the operators live on device %d", dev, ops->device);
        return M2L_EINVAL;
    }
    return M2L_OK;
}

static m2l_status check_level(const m2l_ops *ops, const m2l_level *lv, double *scale)
{
    if (!ops || !lv) { set_error("null ops or level"); return M2L_EINVAL; }
    if (m2l_status st = check_device(ops)) return st;
    if (!(lv->width > 0.0) || !isfinite(lv->width)) { set_error("level width must be positive"); return M2L_EINVAL; }
    if (lv->ncells_tgt < 0 || lv->ncells_src < 0 || lv->nnz < 0) { set_error("negative size"); return M2L_EINVAL; }
    if (lv->ncells_tgt >= (1 << kTgtBits) || lv->ncells_src >= (1 << kTgtBits)) {
        set_error("more than 2^26 cells in one level");
        return M2L_EUNSUPPORTED;
    }
    if (lv->nnz > 0 && (!lv->il_sources || !lv->tgt_ijk || !lv->src_ijk || !lv->il_offsets || lv->ncells_tgt == 0)) {
        set_error("null list pointer with nnz > 0");
        return M2L_EINVAL;
    }
    if (ops->homogeneous) {
        *scale = pow(lv->width / ops->ref_width, (double)ops->hom_degree);
    } else {
        if (fabs(lv->width - ops->ref_width) > 1e-12 * ops->ref_width) {
            set_error("level width %.17g differs from the operators' width %.17g (kernel is not homogeneous)",
                      lv->width, ops->ref_width);
            return M2L_EINVAL;
        }
        *scale = 1.0;
    }
    return M2L_OK;
}

static m2l_status dispatch(const m2l_ops *ops, const Buckets &b, const void *in, void *out, int precision,
                           int out_fp64, double scale, cudaStream_t s)
{
    if (b.nnz > 0 && (!in || !out)) { set_error("null vector pointer"); return M2L_EINVAL; }
    if (m2l_status st = check_device(ops)) return st;
    const bool tc = precision == M2L_TF32 || precision == M2L_BF16X3 || precision == M2L_TF32X3;
    const bool dense = tc && b.dense.valid && !(ops->debug_flags & M2L_DEBUG_NO_DENSE);
    if (b.nnz > 0 && !dense)
        if (m2l_status st = ensure_records(ops, b, s)) return st;
    switch (precision) {
    case M2L_FP64:
    case M2L_FP32:
        return launch_simt(ops, b, in, out, precision, out_fp64, scale, s);
    case M2L_TF32:
    case M2L_BF16X3:
    case M2L_TF32X3:
        return launch_tc(ops, b, in, out, precision, out_fp64, scale, s);
    default:
        set_error("unknown precision %d", precision);
        return M2L_EINVAL;
    }
}

}  // namespace m2l

using namespace m2l;

namespace {
m2l_status precompute_impl(m2l_kernel kernel, int ell, double eps, double width, int aca, int trunc, m2l_ops **out);
}

extern "C" {

const char *m2l_last_error(void) { return g_err; }

int64_t m2l_launch_count(void) { return (int64_t)g_launches.load(); }

m2l_status m2l_precompute(m2l_kernel kernel, int ell, double eps, double width, m2l_ops **out)
{
    return precompute_impl(kernel, ell, eps, width, 0, M2L_TRUNC_FROBENIUS, out);
}

m2l_status m2l_precompute_aca(m2l_kernel kernel, int ell, double eps, double width, m2l_ops **out)
{
    return precompute_impl(kernel, ell, eps, width, 1, M2L_TRUNC_FROBENIUS, out);
}

m2l_status m2l_precompute_ex(m2l_kernel kernel, int ell, double eps, double width, int trunc, int aca,
                             m2l_ops **out)
{
    if (out) *out = nullptr;
    if (trunc != M2L_TRUNC_FROBENIUS && trunc != M2L_TRUNC_SPECTRAL) {
        set_error("unknown truncation criterion %d", trunc);
        return M2L_EINVAL;
    }
    if (aca != 0 && aca != 1) {
        set_error("aca must be 0 or 1, got %d", aca);
        return M2L_EINVAL;
    }
    return precompute_impl(kernel, ell, eps, width, aca, trunc, out);
}

m2l_status m2l_ops_truncation(const m2l_ops *ops, int *trunc)
{
    if (!ops || !trunc) { set_error("null argument"); return M2L_EINVAL; }
    *trunc = ops->trunc;
    return M2L_OK;
}

m2l_status m2l_ops_svd_sweeps(const m2l_ops *ops, int32_t *sweeps16)
{
    if (!ops || !sweeps16) { set_error("null argument"); return M2L_EINVAL; }
    if (ops->eps <= 0) { set_error("operators are full rank"); return M2L_EINVAL; }
    for (int p = 0; p < 16; ++p) sweeps16[p] = ops->jacobi_sweeps[p];
    return M2L_OK;
}

m2l_status m2l_ops_aca_info(const m2l_ops *ops, int32_t *aca_terms16, int32_t *jacobi_sweeps16)
{
    if (!ops) { set_error("null ops"); return M2L_EINVAL; }
    if (ops->lowrank_method != 1) { set_error("ops not built by m2l_precompute_aca with eps > 0"); return M2L_EINVAL; }
    for (int p = 0; p < 16; ++p) {
        if (aca_terms16) aca_terms16[p] = ops->aca_terms[p];
        if (jacobi_sweeps16) jacobi_sweeps16[p] = ops->jacobi_sweeps[p];
    }
    return M2L_OK;
}

}  // extern "C"

namespace {
m2l_status precompute_impl(m2l_kernel kernel, int ell, double eps, double width, int aca, int trunc, m2l_ops **out)
{
    g_err[0] = 0;
    if (!out) { set_error("null output pointer"); return M2L_EINVAL; }
    *out = nullptr;
    if (ell < 2 || ell > kMaxEll) { set_error("ell must be in [2, %d], got %d", kMaxEll, ell); return M2L_EINVAL; }
    if (kernel.type < 0 || kernel.type > 2) { set_error("unknown kernel type %d", kernel.type); return M2L_EINVAL; }
    if (!(eps >= 0.0 && eps < 1.0)) { set_error("eps must be in [0, 1)"); return M2L_EINVAL; }
    if (kernel.type == M2L_K_INV_SQRT_R2C2 && (!(width > 0.0) || !isfinite(width) || !(kernel.c >= 0.0))) {
        set_error("the non-homogeneous kernel needs width > 0 and c >= 0");
        return M2L_EINVAL;
    }
    m2l_ops *ops = new m2l_ops();
    ops->kind = kernel.type;
    ops->c = kernel.c;
    ops->ell = ell;
    ops->n3 = ell * ell * ell;
    ops->eps = eps;
    ops->trunc = trunc;
    ops->homogeneous = is_homogeneous(kernel.type, &ops->hom_degree) ? 1 : 0;
    ops->ref_width = ops->homogeneous ? 1.0 : width;
    cudaGetDevice(&ops->device);
    m2l_status st = M2L_OK;
    const int n3 = ops->n3;
    if (st == M2L_OK) st = ops->K64.ensure(16 * (size_t)n3 * n3 * sizeof(double));
    if (st == M2L_OK) st = ops->sigma.ensure(48 * (size_t)n3 * sizeof(int16_t));
    if (st == M2L_OK) st = ops->lut.ensure(343 * sizeof(uint16_t));
    if (st == M2L_OK) st = ops->tsym.ensure(48 * sizeof(int));
    if (st == M2L_OK) {
        cudaError_t e = cudaMalloc(&ops->d_status, sizeof(int));
        if (e != cudaSuccess) st = cuda_fail(e, "cudaMalloc(status)");
        else if ((e = cudaMemset(ops->d_status, 0, sizeof(int))) != cudaSuccess) st = cuda_fail(e, "cudaMemset");
    }
    if (st == M2L_OK) st = build_tables(ops, 0);
    if (st == M2L_OK) st = assemble_operators(ops, 0);
    if (st == M2L_OK) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) st = cuda_fail(e, "precompute");
    }
    for (int p = 0; p < 16; ++p) ops->ranks[p] = n3;
    ops->rmax = n3;
    if (st == M2L_OK && eps > 0.0) {
        ops->lowrank_method = aca ? 1 : 0;
        st = aca ? lowrank_factors_aca(ops, ops->aca_terms, ops->jacobi_sweeps) : lowrank_factors(ops);
    }
    if (st != M2L_OK) {
        m2l_ops_free(ops);
        return st;
    }
    *out = ops;
    return M2L_OK;
}
}  // namespace

extern "C" {

namespace {
m2l_status rebuild_part(m2l_ops *ops, void *stream, bool tables, bool operators)
{
    if (!ops) { set_error("null ops"); return M2L_EINVAL; }
    if (ops->eps > 0) { set_error("rebuild of low-rank operators is not supported"); return M2L_EUNSUPPORTED; }
    m2l_status st = check_device(ops);
    if (st != M2L_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (tables) st = build_tables(ops, s);
    if (st == M2L_OK && operators) st = assemble_operators(ops, s);
    // derived layouts are rebuilt from the new masters on their next use
    ops->simt64.ready = ops->simt32.ready = false;
    ops->tc_tf32.ready = ops->tc_bf16x3.ready = ops->tc_tf32x3.ready = false;
    ops->tcd_tf32.ready = ops->tcd_bf16x3.ready = ops->tcd_tf32x3.ready = false;
    return st;
}
}  // namespace

m2l_status m2l_ops_rebuild(m2l_ops *ops, void *stream) { return rebuild_part(ops, stream, true, true); }

m2l_status m2l_ops_rebuild_tables(m2l_ops *ops, void *stream) { return rebuild_part(ops, stream, true, false); }

m2l_status m2l_ops_rebuild_operators(m2l_ops *ops, void *stream) { return rebuild_part(ops, stream, false, true); }

m2l_status m2l_ops_query(const m2l_ops *ops, int *ranks16, int16_t *sigma48, uint16_t *lut343)
{
    if (!ops) { set_error("null ops"); return M2L_EINVAL; }
    M2L_CUDA(cudaDeviceSynchronize());
    if (ranks16) memcpy(ranks16, ops->ranks, 16 * sizeof(int));
    if (sigma48) M2L_CUDA(cudaMemcpy(sigma48, ops->sigma.p, 48 * (size_t)ops->n3 * sizeof(int16_t), cudaMemcpyDeviceToHost));
    if (lut343) M2L_CUDA(cudaMemcpy(lut343, ops->lut.p, 343 * sizeof(uint16_t), cudaMemcpyDeviceToHost));
    return M2L_OK;
}

m2l_status m2l_ops_copy_operators(const m2l_ops *ops, double *host_out)
{
    if (!ops || !host_out) { set_error("null argument"); return M2L_EINVAL; }
    M2L_CUDA(cudaDeviceSynchronize());
    M2L_CUDA(cudaMemcpy(host_out, ops->K64.p, 16 * (size_t)ops->n3 * ops->n3 * sizeof(double), cudaMemcpyDeviceToHost));
    return M2L_OK;
}

m2l_status m2l_ops_copy_lowrank(const m2l_ops *ops, int p, double *host_U, double *host_V)
{
    if (!ops || p < 0 || p >= 16) { set_error("bad ops or operator index"); return M2L_EINVAL; }
    if (ops->eps <= 0) { set_error("operators are full rank"); return M2L_EINVAL; }
    M2L_CUDA(cudaDeviceSynchronize());
    const int n3 = ops->n3, r = ops->ranks[p], rmax = ops->rmax;
    // the device stores [n3][rmax]; copy the first r columns
    for (int row = 0; row < n3; ++row) {
        if (host_U)
            M2L_CUDA(cudaMemcpy(host_U + (size_t)row * r, ops->U64.as<double>() + ((size_t)p * n3 + row) * rmax,
                                r * sizeof(double), cudaMemcpyDeviceToHost));
        if (host_V)
            M2L_CUDA(cudaMemcpy(host_V + (size_t)row * r, ops->V64.as<double>() + ((size_t)p * n3 + row) * rmax,
                                r * sizeof(double), cudaMemcpyDeviceToHost));
    }
    return M2L_OK;
}

m2l_status m2l_ops_info(const m2l_ops *ops, int *ell, int *kernel_type, double *eps, double *ref_width,
                        int *homogeneity_degree)
{
    if (!ops) { set_error("null ops"); return M2L_EINVAL; }
    if (ell) *ell = ops->ell;
    if (kernel_type) *kernel_type = ops->kind;
    if (eps) *eps = ops->eps;
    if (ref_width) *ref_width = ops->ref_width;
    if (homogeneity_degree) *homogeneity_degree = ops->hom_degree;
    return M2L_OK;
}

void m2l_ops_free(m2l_ops *ops)
{
    if (!ops) return;
    cudaDeviceSynchronize();
    ops->K64.release(); ops->sigma.release(); ops->lut.release(); ops->tsym.release();
    ops->U64.release(); ops->V64.release();
    Layout *ls[] = {&ops->simt64, &ops->simt32, &ops->lr64, &ops->lr32, &ops->tc_tf32, &ops->tc_bf16x3, &ops->tc_tf32x3,
                    &ops->tcd_tf32, &ops->tcd_bf16x3, &ops->tcd_tf32x3, &ops->lrtc_tf32, &ops->lrtc_bf16x3,
                    &ops->lrtc_tf32x3};
    for (Layout *l : ls) { l->a.release(); l->b.release(); }
    Buckets &b = ops->ws;
    b.rec.release(); b.tgt_of.release(); b.code.release(); b.seg.release(); b.class_off.release();
    b.t_off.release(); b.t_src.release(); b.t_cursor.release(); b.dense.release(); b.lrz.release();
    if (ops->d_status) cudaFree(ops->d_status);
    delete ops;
}

m2l_status m2l_apply_level(const m2l_ops *ops, const m2l_level *level, const void *multipoles, void *locals,
                           int precision, int locals_fp64, void *stream)
{
    double scale = 1.0;
    m2l_status st = check_level(ops, level, &scale);
    if (st != M2L_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    st = classify(ops, level, 0, ops->ws, s);
    if (st != M2L_OK) return st;
    return dispatch(ops, ops->ws, multipoles, locals, precision, locals_fp64, scale, s);
}

m2l_status m2l_classify_level(const m2l_ops *ops, const m2l_level *level, void *stream)
{
    double scale = 1.0;
    m2l_status st = check_level(ops, level, &scale);
    if (st != M2L_OK) return st;
    st = classify(ops, level, 0, ops->ws, (cudaStream_t)stream);
    if (st == M2L_OK) ops->ws_scale = scale;
    return st;
}

m2l_status m2l_apply_classified(const m2l_ops *ops, const void *multipoles, void *locals, int precision,
                                int locals_fp64, void *stream)
{
    if (!ops) { set_error("null ops"); return M2L_EINVAL; }
    return dispatch(ops, ops->ws, multipoles, locals, precision, locals_fp64, ops->ws_scale, (cudaStream_t)stream);
}

m2l_status m2l_apply_level_adjoint(const m2l_ops *ops, const m2l_level *level, const void *grad_locals,
                                   void *grad_multipoles, int precision, int grad_fp64, void *stream)
{
    double scale = 1.0;
    m2l_status st = check_level(ops, level, &scale);
    if (st != M2L_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    st = classify(ops, level, 1, ops->ws, s);
    if (st != M2L_OK) return st;
    return dispatch(ops, ops->ws, grad_locals, grad_multipoles, precision, grad_fp64, scale, s);
}

m2l_status m2l_plan_create(const m2l_ops *ops, const m2l_level *level, int adjoint, void *stream, m2l_plan **out)
{
    if (!out) { set_error("null output pointer"); return M2L_EINVAL; }
    *out = nullptr;
    double scale = 1.0;
    m2l_status st = check_level(ops, level, &scale);
    if (st != M2L_OK) return st;
    m2l_plan *plan = new m2l_plan();
    plan->ops = ops;
    plan->adjoint = adjoint ? 1 : 0;
    plan->width = level->width;
    plan->n_out = adjoint ? level->ncells_src : level->ncells_tgt;
    plan->n_in = adjoint ? level->ncells_tgt : level->ncells_src;
    st = classify(ops, level, plan->adjoint, plan->b, (cudaStream_t)stream);
    if (st == M2L_OK) {
        cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
        if (e != cudaSuccess) st = cuda_fail(e, "plan classification");
    }
    // transposition scratch is not needed after creation
    plan->b.t_off.release(); plan->b.t_src.release(); plan->b.t_cursor.release();
    plan->b.tgt_of.release(); plan->b.code.release(); plan->b.seg.release();
    if (st != M2L_OK) {
        m2l_plan_free(plan);
        return st;
    }
    *out = plan;
    return M2L_OK;
}

m2l_status m2l_plan_apply(const m2l_plan *plan, const void *in_vectors, void *out_vectors, int precision,
                          int out_fp64, void *stream)
{
    if (!plan) { set_error("null plan"); return M2L_EINVAL; }
    const m2l_ops *ops = plan->ops;
    double scale = ops->homogeneous ? pow(plan->width / ops->ref_width, (double)ops->hom_degree) : 1.0;
    return dispatch(ops, plan->b, in_vectors, out_vectors, precision, out_fp64, scale, (cudaStream_t)stream);
}

m2l_status m2l_plan_classify(m2l_plan *plan, const m2l_level *level, void *stream)
{
    if (!plan) { set_error("null plan"); return M2L_EINVAL; }
    double scale = 1.0;
    m2l_status st = check_level(plan->ops, level, &scale);
    if (st != M2L_OK) return st;
    st = classify(plan->ops, level, plan->adjoint, plan->b, (cudaStream_t)stream);
    if (st != M2L_OK) return st;
    plan->width = level->width;
    plan->n_out = plan->adjoint ? level->ncells_src : level->ncells_tgt;
    plan->n_in = plan->adjoint ? level->ncells_tgt : level->ncells_src;
    return M2L_OK;
}

m2l_status m2l_ops_prepare(const m2l_ops *ops, int precision, void *stream)
{
    if (!ops) { set_error("null ops"); return M2L_EINVAL; }
    // an apply over no interactions builds the layouts and launches nothing else;
    // the tensor-core precisions also get the per-slot images of the dense kernel
    Buckets empty;
    m2l_status st = dispatch(ops, empty, nullptr, nullptr, precision, 0, 1.0, (cudaStream_t)stream);
    if (st != M2L_OK) return st;
    return dense_prepare(ops, precision, (cudaStream_t)stream);
}

m2l_status m2l_plan_query(const m2l_plan *plan, int64_t *counts16, int32_t *records, int64_t *nvalid)
{
    if (!plan) { set_error("null plan"); return M2L_EINVAL; }
    M2L_CUDA(cudaDeviceSynchronize());
    if (m2l_status st = ensure_records(plan->ops, plan->b, 0)) return st;
    M2L_CUDA(cudaDeviceSynchronize());
    int32_t off[18] = {0};
    if (plan->b.nnz > 0) M2L_CUDA(cudaMemcpy(off, plan->b.class_off.p, sizeof(off), cudaMemcpyDeviceToHost));
    if (counts16)
        for (int p = 0; p < 16; ++p) counts16[p] = off[p + 1] - off[p];
    if (nvalid) *nvalid = off[16];
    if (records && off[16] > 0) {
        const int n = off[16];
        int2 *tmp = (int2 *)malloc((size_t)n * sizeof(int2));
        if (!tmp) { set_error("host allocation failed"); return M2L_ENOMEM; }
        cudaError_t e = cudaMemcpy(tmp, plan->b.rec.p, (size_t)n * sizeof(int2), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) { free(tmp); return cuda_fail(e, "plan records"); }
        for (int i = 0; i < n; ++i) {
            records[3 * i] = tmp[i].x;
            records[3 * i + 1] = rec_tgt(tmp[i].y);
            records[3 * i + 2] = (int)((unsigned)tmp[i].y >> kTgtBits);
        }
        free(tmp);
    }
    return M2L_OK;
}

m2l_status m2l_plan_kernel_info(const m2l_plan *plan, int *dense, int *units, int *unit_width)
{
    if (!plan) { set_error("null plan"); return M2L_EINVAL; }
    const DenseBuckets &d = plan->b.dense;
    if (dense) *dense = d.valid ? 1 : 0;
    if (units) *units = d.valid ? d.umax : 0;
    if (unit_width) *unit_width = d.valid ? d.nu : 0;
    return M2L_OK;
}

void m2l_plan_free(m2l_plan *plan)
{
    if (!plan) return;
    cudaDeviceSynchronize();
    Buckets &b = plan->b;
    b.rec.release(); b.tgt_of.release(); b.code.release(); b.seg.release(); b.class_off.release();
    b.t_off.release(); b.t_src.release(); b.t_cursor.release(); b.dense.release(); b.lrz.release();
    delete plan;
}

m2l_status m2l_apply_batch(const m2l_ops *const *ops, const m2l_level *levels, const void *const *multipoles,
                           void *const *locals, int nbatch, int precision, int locals_fp64, void *stream)
{
    if (nbatch < 0 || (nbatch > 0 && (!ops || !levels || !multipoles || !locals))) {
        set_error("bad batch arguments");
        return M2L_EINVAL;
    }
    bool loop = precision != M2L_FP32 && precision != M2L_FP64 && locals_fp64 != 0;
    for (int i = 0; i < nbatch && !loop; ++i)
        if (precision != M2L_FP32 && precision != M2L_FP64 && (!ops[i] || ops[i]->n3 > 256 || ops[i]->eps > 0))
            loop = true;
    if (loop) {
        // FP64 outputs, orders above 6 or low-rank operators on the tensor cores: one apply per problem
        for (int i = 0; i < nbatch; ++i) {
            m2l_status st = m2l_apply_level(ops[i], &levels[i], multipoles[i], locals[i], precision, locals_fp64, stream);
            if (st != M2L_OK) return st;
        }
        return M2L_OK;
    }
    std::vector<m2l_plan *> plans(nbatch, nullptr);
    m2l_status st = M2L_OK;
    for (int i = 0; i < nbatch && st == M2L_OK; ++i) st = m2l_plan_create(ops[i], &levels[i], 0, stream, &plans[i]);
    m2l_batch *b = nullptr;
    if (st == M2L_OK) st = m2l_batch_create(plans.data(), nbatch, multipoles, locals, precision, locals_fp64, stream, &b);
    if (st == M2L_OK) st = m2l_batch_run(b, stream);
    if (st == M2L_OK) {
        cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
        if (e != cudaSuccess) st = cuda_fail(e, "batched apply");
    }
    m2l_batch_free(b);
    for (m2l_plan *p : plans) m2l_plan_free(p);
    return st;
}

m2l_status m2l_ops_set_debug(m2l_ops *ops, int flags)
{
    if (!ops) { set_error("null ops"); return M2L_EINVAL; }
    ops->debug_flags = flags;
    return M2L_OK;
}

m2l_status m2l_sync_status(const m2l_ops *ops, void *stream)
{
    if (!ops) { set_error("null ops"); return M2L_EINVAL; }
    M2L_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    int st = 0;
    M2L_CUDA(cudaMemcpy(&st, ops->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    M2L_CUDA(cudaMemset(ops->d_status, 0, sizeof(int)));
    if (st & ST_TIMEOUT) { set_error("a bounded device wait timed out"); return M2L_ETIMEOUT; }
    if (st & (ST_BAD_PAIR | ST_BAD_INDEX | ST_BAD_TABLE)) {
        set_error("interaction list rejected on the device (status bits 0x%x): %s%s", st,
                  (st & ST_BAD_PAIR) ? "entries that are not far-field pairs; " : "",
                  (st & ST_BAD_INDEX) ? "indices or offsets out of range" : "");
        return M2L_EINVAL;
    }
    return M2L_OK;
}

}  // extern "C"
