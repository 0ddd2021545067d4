// Batched apply (many uneven trees and levels in one persistent launch) and
// the autotuner of its tile width.
#include <math.h>
#include <string.h>

#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "m2l_internal.cuh"

namespace m2l {


m2l_status launch_simt_batch(const BatchDesc *descs, int nprob, int total_tiles, int fp64, int nt, int kpad_max,
                             int mpad_max, cudaStream_t s);
size_t batch_smem_bytes(int fp64, int nt, int kpad_max, int mpad_max);

namespace {

// Autotuner cache: (fp64, kpad_max, mpad_max, log2 of the interaction count) -> tile width.
std::mutex g_tune_mutex;
std::map<std::tuple<int, int, int, int>, std::pair<int, double>> g_tune_cache;

int log2_bucket(long long n)
{
    int b = 0;
    while (n > 1) { n >>= 1; ++b; }
    return b;
}

// Tile tables of every problem for tile width nt; returns the total tile count.
int fill_tiles(std::vector<BatchDesc> &d, int nt)
{
    int base = 0;
    for (auto &x : d) {
        x.tile_base = base;
        int acc = 0;
        for (int p = 0; p < 16; ++p) {
            x.tile_start[p] = acc;
            acc += (x.class_off[p + 1] - x.class_off[p] + nt - 1) / nt;
        }
        x.tile_start[16] = acc;
        base += acc;
    }
    return base;
}

}  // namespace
}  // namespace m2l

struct m2l_batch {
    int fp64 = 0, nprob = 0, total_tiles = 0, nt = 32, kpad_max = 0, mpad_max = 0;
    double tuned_ms = 0.0;
    long long nnz = 0;
    m2l::DevBuf descs;
    m2l::TcBatch *tc = nullptr;   // tensor-core precisions
};

using namespace m2l;

extern "C" m2l_status m2l_batch_create(const m2l_plan *const *plans, int nbatch, const void *const *in,
                                       void *const *out, int precision, int out_fp64, void *stream,
                                       m2l_batch **out_batch)
{
    if (!out_batch || nbatch < 0 || (nbatch > 0 && (!plans || !in || !out))) {
        set_error("bad batch arguments");
        return M2L_EINVAL;
    }
    *out_batch = nullptr;
    if (precision == M2L_TF32 || precision == M2L_BF16X3 || precision == M2L_TF32X3) {
        if (out_fp64) { set_error("the tensor-core batch writes FP32 outputs"); return M2L_EUNSUPPORTED; }
        for (int i = 0; i < nbatch; ++i)
            if (!plans[i] || !in[i] || !out[i]) { set_error("null plan or vector in batch entry %d", i); return M2L_EINVAL; }
        TcBatch *tc = nullptr;
        m2l_status st = tc_batch_create(plans, nbatch, in, out, precision, (cudaStream_t)stream, &tc);
        if (st != M2L_OK) return st;
        m2l_batch *b = new m2l_batch();
        b->nprob = nbatch;
        b->tc = tc;
        *out_batch = b;
        return M2L_OK;
    }
    if (precision != M2L_FP32 && precision != M2L_FP64) {
        set_error("unknown precision %d", precision);
        return M2L_EINVAL;
    }
    const int fp64 = precision == M2L_FP64;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<BatchDesc> d(nbatch);
    int kpad_max = 32, mpad_max = 128;
    long long nnz = 0;
    for (int i = 0; i < nbatch; ++i) {
        const m2l_plan *pl = plans[i];
        if (!pl || !in[i] || !out[i]) { set_error("null plan or vector in batch entry %d", i); return M2L_EINVAL; }
        const m2l_ops *ops = pl->ops;
        if (m2l_status st = check_device(ops)) return st;
        if (ops->eps > 0) { set_error("the persistent batch takes full-rank operators"); return M2L_EUNSUPPORTED; }
        m2l_status st = prepare_simt_layout(ops, fp64, s);
        if (st == M2L_OK && pl->b.nnz > 0) st = ensure_records(ops, pl->b, s);
        if (st != M2L_OK) return st;
        int32_t off[18] = {0};
        if (pl->b.nnz > 0) {
            M2L_CUDA(cudaStreamSynchronize(s));
            M2L_CUDA(cudaMemcpy(off, pl->b.class_off.p, sizeof(off), cudaMemcpyDeviceToHost));
        }
        BatchDesc &x = d[i];
        memset(&x, 0, sizeof(x));
        x.rec = pl->b.rec.as<int2>();
        const Layout &L = fp64 ? ops->simt64 : ops->simt32;
        x.A = L.a.p;
        x.sigma = ops->sigma.as<int16_t>();
        x.in = in[i];
        x.out = out[i];
        x.scale = ops->homogeneous ? pow(pl->width / ops->ref_width, (double)ops->hom_degree) : 1.0;
        x.n3 = ops->n3;
        x.kpad = simt_kpad(ops->n3);
        x.mpad = simt_mpad(ops->n3);
        x.out_fp64 = (fp64 || out_fp64) ? 1 : 0;
        for (int p = 0; p < 17; ++p) x.class_off[p] = off[p];
        if (x.kpad > kpad_max) kpad_max = x.kpad;
        if (x.mpad > mpad_max) mpad_max = x.mpad;
        nnz += off[16];
    }
    m2l_batch *b = new m2l_batch();
    b->fp64 = fp64;
    b->nprob = nbatch;
    b->kpad_max = kpad_max;
    b->mpad_max = mpad_max;
    b->nnz = nnz;
    m2l_status st = b->descs.ensure((size_t)(nbatch > 0 ? nbatch : 1) * sizeof(BatchDesc));
    if (st != M2L_OK) { delete b; return st; }

    // Autotuner: the tile width (columns per tile) of the persistent kernel, timed on
    // scratch outputs and cached per (precision, padded sizes, log2 interactions).
    std::vector<int> cands;
    if (fp64) cands = {32};
    else cands = {32, 64};
    for (auto it = cands.begin(); it != cands.end();)
        it = ((int)batch_smem_bytes(fp64, *it, kpad_max, mpad_max) > max_smem_optin()) ? cands.erase(it) : it + 1;
    if (cands.empty()) { delete b; set_error("no batched configuration fits shared memory"); return M2L_EUNSUPPORTED; }
    const auto key = std::make_tuple(fp64, kpad_max, mpad_max, log2_bucket(nnz));
    int best = cands.front();
    double best_ms = 0.0;
    bool cached = false;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) { best = it->second.first; best_ms = it->second.second; cached = true; }
    }
    if (!cached && cands.size() > 1 && nnz > 0) {
        // scratch copies of the outputs, so the caller's vectors are untouched
        std::vector<BatchDesc> dt = d;
        size_t total = 0;
        std::vector<size_t> offs(nbatch);
        for (int i = 0; i < nbatch; ++i) {
            offs[i] = total;
            const size_t esz = dt[i].out_fp64 ? sizeof(double) : sizeof(float);
            // upper bound of the output rows: the largest target index + 1 is not known on
            // the host, so the scratch region covers the caller's whole output extent
            total += (size_t)plans[i]->n_out * dt[i].n3 * esz;
            total = (total + 255) / 256 * 256;
        }
        DevBuf scratch, tdesc;
        st = scratch.ensure(total);
        if (st == M2L_OK) st = tdesc.ensure((size_t)nbatch * sizeof(BatchDesc));
        for (int i = 0; i < nbatch && st == M2L_OK; ++i) dt[i].out = scratch.as<char>() + offs[i];
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (st == M2L_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) {
            set_error("cudaEventCreate failed");
            st = M2L_ECUDA;
        }
        double best_t = 1e30;
        for (int nt : cands) {
            if (st != M2L_OK) break;
            const int tiles = fill_tiles(dt, nt);
            if (cudaMemcpyAsync(tdesc.p, dt.data(), (size_t)nbatch * sizeof(BatchDesc), cudaMemcpyHostToDevice, s) !=
                cudaSuccess) { st = M2L_ECUDA; break; }
            float tmin = 1e30f;
            for (int rep = 0; rep < 4 && st == M2L_OK; ++rep) {
                cudaEventRecord(e0, s);
                st = launch_simt_batch(tdesc.as<BatchDesc>(), nbatch, tiles, fp64, nt, kpad_max, mpad_max, s);
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0 && ms < tmin) tmin = ms;   // first launch is a warm-up
            }
            if (tmin < best_t) { best_t = tmin; best = nt; }
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaStreamSynchronize(s);
        scratch.release();
        tdesc.release();
        if (st != M2L_OK) { delete b; return st; }
        best_ms = best_t;
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune_cache[key] = std::make_pair(best, best_ms);
    }
    b->nt = best;
    b->tuned_ms = best_ms;
    b->total_tiles = fill_tiles(d, best);
    if (nbatch > 0) {
        cudaError_t e = cudaMemcpyAsync(b->descs.p, d.data(), (size_t)nbatch * sizeof(BatchDesc),
                                        cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { delete b; return cuda_fail(e, "batch descriptors"); }
    }
    *out_batch = b;
    return M2L_OK;
}

extern "C" m2l_status m2l_batch_run(const m2l_batch *b, void *stream)
{
    if (!b) { set_error("null batch"); return M2L_EINVAL; }
    if (b->tc) return tc_batch_run(b->tc, (cudaStream_t)stream);
    return launch_simt_batch(b->descs.as<BatchDesc>(), b->nprob, b->total_tiles, b->fp64, b->nt, b->kpad_max,
                             b->mpad_max, (cudaStream_t)stream);
}

extern "C" m2l_status m2l_batch_info(const m2l_batch *b, int *tile_width, int64_t *tiles, double *tuned_ms)
{
    if (!b) { set_error("null batch"); return M2L_EINVAL; }
    if (b->tc) {
        tc_batch_info(b->tc, tile_width, tiles, tuned_ms, nullptr, nullptr);
        return M2L_OK;
    }
    if (tile_width) *tile_width = b->nt;
    if (tiles) *tiles = b->total_tiles;
    if (tuned_ms) *tuned_ms = b->tuned_ms;
    return M2L_OK;
}

extern "C" void m2l_batch_free(m2l_batch *b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    b->descs.release();
    if (b->tc) tc_batch_free(b->tc);
    delete b;
}

extern "C" m2l_status m2l_batch_groups(const m2l_batch *b, int max_groups, int32_t *ell3, int32_t *tile_width,
                                       int32_t *epilogue_groups, int32_t *ngroups)
{
    if (!b || max_groups < 0 || (max_groups > 0 && (!ell3 || !tile_width || !epilogue_groups))) {
        set_error("bad batch or output arrays");
        return M2L_EINVAL;
    }
    if (!b->tc) {
        // the CUDA-core batch is one launch over every problem
        if (max_groups > 0) {
            ell3[0] = b->mpad_max;
            tile_width[0] = b->nt;
            epilogue_groups[0] = 0;
        }
        if (ngroups) *ngroups = 1;
        return M2L_OK;
    }
    std::vector<int> n3(max_groups > 0 ? max_groups : 1), nt(n3.size()), eg(n3.size());
    const int n = tc_batch_groups(b->tc, max_groups, n3.data(), nt.data(), eg.data());
    for (int i = 0; i < n && i < max_groups; ++i) {
        ell3[i] = n3[i];
        tile_width[i] = nt[i];
        epilogue_groups[i] = eg[i];
    }
    if (ngroups) *ngroups = n;
    return M2L_OK;
}
