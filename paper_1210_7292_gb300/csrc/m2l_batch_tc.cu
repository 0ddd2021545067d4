// Persistent batches on the tensor cores: many planned translations (trees x
// levels, mixed orders, per-level operator sets) in one launch per vector
// length.
//
// A batch groups its problems by ell^3.  A group becomes one bucketed problem
// of the large-order tcgen05 kernel (the blocking of Alg. 2 over many target
// cells, Sec. 4.2.3, across trees as well): its classes are the pairs
// (problem, unique operator p), in problem order, each class's bucket the
// plan's bucket with source and target indices offset into the group's
// concatenated vectors; the operator images are built once per distinct
// (operator set, scale) and shared by classes through a class -> image map.
// A run is, per group: gather the problems' input vectors into the group's
// input rows, zero the group's output rows, one persistent launch, add the
// output rows into the problems' outputs.
//
// Tile shapes (interactions per tile, epilogue groups; the stage and ring
// depths follow from shared memory) are picked by timing every candidate that
// fits on scratch outputs, cached per (precision, vector length, log2 of the
// interaction count).
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "m2l_tc_big.cuh"

namespace m2l {

struct CatDesc {
    const float *in;    // problem input vectors [in_rows][n3]
    float *out;         // problem output vectors [out_rows][n3]
    long long in_rows, out_rows, in_off, out_off;
};

struct TcGroup {
    int n3 = 0, ncls = 0, nprob = 0, kpad = 0, nimg = 0;
    long long nnz = 0, in_rows = 0, out_rows = 0;
    int nt = 0, eg = 0;                    // chosen tile width and epilogue groups
    int tiles32 = 0, tiles64 = 0;
    double tuned_ms = 0.0;
    DevBuf img, img_of, tinv, ts32, ts64, class_off, rec, in_cat, out_cat, descs;
};

namespace {

// Problem i's input rows into the group's rows [in_off, in_off + in_rows).
__global__ void cat_gather_kernel(const CatDesc *__restrict__ d, int n3, float *__restrict__ in_cat)
{
    const CatDesc c = d[blockIdx.y];
    const long long n = c.in_rows * n3;
    float *dst = in_cat + c.in_off * n3;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        dst[k] = c.in[k];
}

// out += the group's rows [out_off, out_off + out_rows) of problem i.
__global__ void cat_scatter_kernel(const CatDesc *__restrict__ d, int n3, const float *__restrict__ out_cat)
{
    const CatDesc c = d[blockIdx.y];
    const long long n = c.out_rows * n3;
    const float *src = out_cat + c.out_off * n3;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        c.out[k] += src[k];
}

// A plan's bucketed records with source and target indices moved into the group.
__global__ void cat_records_kernel(int n, const int2 *__restrict__ rec, int sbase, int tbase, int2 *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int2 r = rec[i];
    out[i] = make_int2(r.x + sbase, rec_pack(rec_tgt(r.y) + tbase, rec_g(r.y)));
}

__global__ void scale_copy_kernel(long long n, const double *__restrict__ K, double scale, double *__restrict__ out)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        out[k] = K[k] * scale;
}

constexpr int kCandNt[2] = {32, 64};
constexpr int kCandEg[2] = {1, 2};

std::mutex g_tc_tune_mutex;
std::map<std::tuple<int, int, int>, std::tuple<int, int, double>> g_tc_tune_cache;

template <int KIND, int MT, int KA, int NT, int EG>
m2l_status launch_group_cfg(const TcGroup &g, int *status, cudaStream_t s)
{
    using C = BigCfg<KIND, MT, KA, NT, EG>;
    if (C::SMEM > max_smem_optin()) {
        set_error("tile shape (%d columns, %d epilogue groups) does not fit shared memory", NT, EG);
        return M2L_EUNSUPPORTED;
    }
    auto kern = tc_big_kernel<KIND, MT, KA, NT, EG>;
    M2L_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    const int tiles = NT == 32 ? g.tiles32 : g.tiles64;
    int grid = num_sms();
    if (grid > tiles) grid = tiles;
    if (grid < 1) return M2L_OK;
    kern<<<grid, big_threads(EG), C::SMEM, s>>>(g.rec.as<int2>(), g.class_off.as<int>(), g.img.as<uint8_t>(),
                                                g.tinv.as<int16_t>(), g.in_cat.as<float>(), g.out_cat.as<float>(),
                                                nullptr, g.n3, 1.0f, status, 0, g.ncls,
                                                NT == 32 ? g.ts32.as<int>() : g.ts64.as<int>(), g.img_of.as<int>(),
                                                g.n3, nullptr);
    M2L_LAUNCH_CHECK("tc_big_kernel");
    return M2L_OK;
}

template <int KIND, int MT, int KA>
m2l_status launch_group_shape(const TcGroup &g, int nt, int eg, int *status, cudaStream_t s)
{
    if (nt == 32 && eg == 1) return launch_group_cfg<KIND, MT, KA, 32, 1>(g, status, s);
    if (nt == 32 && eg == 2) return launch_group_cfg<KIND, MT, KA, 32, 2>(g, status, s);
    if (nt == 64 && eg == 1) return launch_group_cfg<KIND, MT, KA, 64, 1>(g, status, s);
    if (nt == 64 && eg == 2) return launch_group_cfg<KIND, MT, KA, 64, 2>(g, status, s);
    set_error("no tile shape (%d, %d)", nt, eg);
    return M2L_EINVAL;
}

template <int KIND, int MT, int KA>
bool shape_fits(int nt, int eg)
{
    int smem = 0;
    if (nt == 32) smem = eg == 1 ? BigCfg<KIND, MT, KA, 32, 1>::SMEM : BigCfg<KIND, MT, KA, 32, 2>::SMEM;
    else smem = eg == 1 ? BigCfg<KIND, MT, KA, 64, 1>::SMEM : BigCfg<KIND, MT, KA, 64, 2>::SMEM;
    return smem <= max_smem_optin();
}

// One persistent launch of group g in tile shape (nt, eg).
m2l_status launch_group(int precision, const TcGroup &g, int nt, int eg, int *status, cudaStream_t s)
{
    const bool two = g.n3 > 128;
    switch (precision) {
    case M2L_BF16X3:
        return two ? launch_group_shape<TC_BF16X3, 2, 4>(g, nt, eg, status, s)
                   : launch_group_shape<TC_BF16X3, 1, 2>(g, nt, eg, status, s);
    case M2L_TF32X3:
        return two ? launch_group_shape<TC_TF32X3, 2, 8>(g, nt, eg, status, s)
                   : launch_group_shape<TC_TF32X3, 1, 4>(g, nt, eg, status, s);
    case M2L_TF32:
        return two ? launch_group_shape<TC_TF32, 2, 8>(g, nt, eg, status, s)
                   : launch_group_shape<TC_TF32, 1, 4>(g, nt, eg, status, s);
    default:
        set_error("not a tensor-core precision: %d", precision);
        return M2L_EINVAL;
    }
}

bool fits(int precision, int n3, int nt, int eg)
{
    const bool two = n3 > 128;
    switch (precision) {
    case M2L_BF16X3: return two ? shape_fits<TC_BF16X3, 2, 4>(nt, eg) : shape_fits<TC_BF16X3, 1, 2>(nt, eg);
    case M2L_TF32X3: return two ? shape_fits<TC_TF32X3, 2, 8>(nt, eg) : shape_fits<TC_TF32X3, 1, 4>(nt, eg);
    case M2L_TF32: return two ? shape_fits<TC_TF32, 2, 8>(nt, eg) : shape_fits<TC_TF32, 1, 4>(nt, eg);
    default: return false;
    }
}

int log2_bucket_ll(long long n)
{
    int b = 0;
    while (n > 1) { n >>= 1; ++b; }
    return b;
}

}  // namespace

// A batch of planned translations on the tensor cores: one group per vector length.
struct TcBatch {
    int precision = 0;
    int *status = nullptr;       // status word the launches report to (first problem's operators)
    std::vector<TcGroup *> groups;
    ~TcBatch()
    {
        for (TcGroup *g : groups) {
            DevBuf *bufs[] = {&g->img, &g->img_of, &g->tinv, &g->ts32, &g->ts64, &g->class_off, &g->rec,
                              &g->in_cat, &g->out_cat, &g->descs};
            for (DevBuf *b : bufs) b->release();
            delete g;
        }
    }
};

namespace {

// The pieces of one group after its bucket sizes are known on the host.
struct ProbInfo {
    const m2l_plan *plan;
    const float *in;
    float *out;
    int32_t off[18];
    double scale;
};

m2l_status build_group(int precision, const std::vector<ProbInfo> &pr, TcGroup &g, cudaStream_t s)
{
    m2l_status st;
    const m2l_ops *ops0 = pr[0].plan->ops;
    const int n3 = ops0->n3;
    int kpad = 0, tcols = 0;
    size_t per_op = 0;
    if (!tc_general_config(precision, n3, &kpad, &per_op, &tcols)) {
        set_error("no tensor-core batch configuration for vectors of %d values", n3);
        return M2L_EUNSUPPORTED;
    }
    g.n3 = n3;
    g.kpad = kpad;
    g.nprob = (int)pr.size();
    g.ncls = 16 * g.nprob;
    // classes (problem, p) in problem order; images per distinct (operator set, scale)
    std::vector<int32_t> cls_off(g.ncls + 1), img_of(g.ncls);
    std::vector<std::pair<const m2l_ops *, double>> imgs;
    std::vector<CatDesc> cat(g.nprob);
    long long base = 0, in_rows = 0, out_rows = 0;
    for (int j = 0; j < g.nprob; ++j) {
        const ProbInfo &p = pr[j];
        int k = 0;
        while (k < (int)imgs.size() && !(imgs[k].first == p.plan->ops && imgs[k].second == p.scale)) ++k;
        if (k == (int)imgs.size()) imgs.push_back({p.plan->ops, p.scale});
        for (int q = 0; q < 16; ++q) {
            cls_off[16 * j + q] = (int32_t)(base + p.off[q]);
            img_of[16 * j + q] = 16 * k + q;
        }
        base += p.off[16];
        cat[j] = CatDesc{p.in, p.out, (long long)p.plan->n_in, (long long)p.plan->n_out, in_rows, out_rows};
        in_rows += p.plan->n_in;
        out_rows += p.plan->n_out;
    }
    cls_off[g.ncls] = (int32_t)base;
    if (base >= (1LL << 31) || out_rows >= (1LL << kTgtBits) || in_rows >= (1LL << 31)) {
        set_error("tensor-core batch too large for one group");
        return M2L_EUNSUPPORTED;
    }
    g.nnz = base;
    g.in_rows = in_rows;
    g.out_rows = out_rows;
    g.nimg = (int)imgs.size();
    std::vector<int32_t> ts32(g.ncls + 1, 0), ts64(g.ncls + 1, 0);
    for (int c = 0; c < g.ncls; ++c) {
        const int n = cls_off[c + 1] - cls_off[c];
        ts32[c + 1] = ts32[c] + (n + 31) / 32;
        ts64[c + 1] = ts64[c] + (n + 63) / 64;
    }
    g.tiles32 = ts32[g.ncls];
    g.tiles64 = ts64[g.ncls];
    if ((st = g.img.ensure((size_t)g.nimg * 16 * per_op)) != M2L_OK) return st;
    if ((st = g.img_of.ensure((size_t)g.ncls * sizeof(int32_t))) != M2L_OK) return st;
    if ((st = g.tinv.ensure((size_t)48 * kpad * sizeof(int16_t))) != M2L_OK) return st;
    if ((st = g.ts32.ensure((size_t)(g.ncls + 1) * sizeof(int32_t))) != M2L_OK) return st;
    if ((st = g.ts64.ensure((size_t)(g.ncls + 1) * sizeof(int32_t))) != M2L_OK) return st;
    if ((st = g.class_off.ensure((size_t)(g.ncls + 1) * sizeof(int32_t))) != M2L_OK) return st;
    if ((st = g.rec.ensure((size_t)(base > 0 ? base : 1) * sizeof(int2))) != M2L_OK) return st;
    if ((st = g.in_cat.ensure((size_t)(in_rows > 0 ? in_rows : 1) * n3 * sizeof(float))) != M2L_OK) return st;
    if ((st = g.out_cat.ensure((size_t)(out_rows > 0 ? out_rows : 1) * n3 * sizeof(float))) != M2L_OK) return st;
    if ((st = g.descs.ensure((size_t)g.nprob * sizeof(CatDesc))) != M2L_OK) return st;
    M2L_CUDA(cudaMemcpyAsync(g.img_of.p, img_of.data(), img_of.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    M2L_CUDA(cudaMemcpyAsync(g.ts32.p, ts32.data(), ts32.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    M2L_CUDA(cudaMemcpyAsync(g.ts64.p, ts64.data(), ts64.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    M2L_CUDA(cudaMemcpyAsync(g.class_off.p, cls_off.data(), cls_off.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                             s));
    M2L_CUDA(cudaMemcpyAsync(g.descs.p, cat.data(), cat.size() * sizeof(CatDesc), cudaMemcpyHostToDevice, s));
    // operator images: the FP64 masters times the problem's scale (w^degree for
    // homogeneous kernels), 16 per distinct set
    DevBuf tmp;
    ScratchGuard guard{&tmp};
    if ((st = tmp.ensure((size_t)16 * n3 * n3 * sizeof(double))) != M2L_OK) return st;
    for (int k = 0; k < g.nimg; ++k) {
        const long long n = 16LL * n3 * n3;
        scale_copy_kernel<<<(int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096), 256, 0, s>>>(
            n, imgs[k].first->K64.as<double>(), imgs[k].second, tmp.as<double>());
        M2L_LAUNCH_CHECK("scale_copy_kernel");
        if ((st = tc_general_images(precision, n3, 16, tmp.as<double>(), g.img.as<uint8_t>() + (size_t)k * 16 * per_op,
                                    s)) != M2L_OK)
            return st;
        // tmp is rewritten by the next set only after these images are built (same stream)
    }
    M2L_CUDA(cudaMemsetAsync(g.tinv.p, 0, (size_t)48 * kpad * sizeof(int16_t), s));
    sigma_inverse_padded_kernel<<<(48 * n3 + 255) / 256, 256, 0, s>>>(n3, kpad, ops0->sigma.as<int16_t>(),
                                                                    g.tinv.as<int16_t>());
    M2L_LAUNCH_CHECK("sigma_inverse_padded_kernel");
    for (int j = 0; j < g.nprob; ++j) {
        const int n = pr[j].off[16];
        if (n == 0) continue;
        cat_records_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, pr[j].plan->b.rec.as<int2>(), (int)cat[j].in_off,
                                                           (int)cat[j].out_off, g.rec.as<int2>() + cls_off[16 * j]);
        M2L_LAUNCH_CHECK("cat_records_kernel");
    }
    M2L_CUDA(cudaStreamSynchronize(s));   // tmp is released at return
    return M2L_OK;
}

m2l_status run_group(int precision, const TcGroup &g, int nt, int eg, int *status, cudaStream_t s, bool scatter)
{
    if (g.nnz == 0) return M2L_OK;
    const long long in_n = g.in_rows * g.n3;
    const int gx = (int)((in_n / g.nprob + 255) / 256 < 1024 ? (in_n / g.nprob + 255) / 256 + 1 : 1024);
    cat_gather_kernel<<<dim3(gx, g.nprob), 256, 0, s>>>(g.descs.as<CatDesc>(), g.n3, g.in_cat.as<float>());
    M2L_LAUNCH_CHECK("cat_gather_kernel");
    M2L_CUDA(cudaMemsetAsync(g.out_cat.p, 0, (size_t)g.out_rows * g.n3 * sizeof(float), s));
    m2l_status st = launch_group(precision, g, nt, eg, status, s);
    if (st != M2L_OK || !scatter) return st;
    const long long out_n = g.out_rows * g.n3;
    const int sx = (int)((out_n / g.nprob + 255) / 256 < 1024 ? (out_n / g.nprob + 255) / 256 + 1 : 1024);
    cat_scatter_kernel<<<dim3(sx, g.nprob), 256, 0, s>>>(g.descs.as<CatDesc>(), g.n3, g.out_cat.as<float>());
    M2L_LAUNCH_CHECK("cat_scatter_kernel");
    return M2L_OK;
}

// Times every fitting tile shape on the group's scratch rows (the problems'
// outputs are not touched) and keeps the fastest; cached per
// (precision, vector length, log2 of the interaction count).
m2l_status tune_group(int precision, TcGroup &g, int *status, cudaStream_t s)
{
    const auto key = std::make_tuple(precision, g.n3, log2_bucket_ll(g.nnz));
    {
        std::lock_guard<std::mutex> lock(g_tc_tune_mutex);
        auto it = g_tc_tune_cache.find(key);
        if (it != g_tc_tune_cache.end()) {
            g.nt = std::get<0>(it->second);
            g.eg = std::get<1>(it->second);
            g.tuned_ms = std::get<2>(it->second);
            return M2L_OK;
        }
    }
    std::vector<std::pair<int, int>> cands;
    for (int nt : kCandNt)
        for (int eg : kCandEg)
            if (fits(precision, g.n3, nt, eg)) cands.push_back({nt, eg});
    if (cands.empty()) {
        set_error("no tensor-core tile shape fits shared memory for vectors of %d values", g.n3);
        return M2L_EUNSUPPORTED;
    }
    g.nt = cands[0].first;
    g.eg = cands[0].second;
    if (cands.size() == 1 || g.nnz == 0) return M2L_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        set_error("cudaEventCreate failed");
        return M2L_ECUDA;
    }
    m2l_status st = M2L_OK;
    double best = 1e30;
    for (const auto &c : cands) {
        float tmin = 1e30f;
        for (int rep = 0; rep < 4 && st == M2L_OK; ++rep) {
            cudaEventRecord(e0, s);
            st = run_group(precision, g, c.first, c.second, status, s, false);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms < tmin) tmin = ms;   // the first run is a warm-up
        }
        if (st != M2L_OK) break;
        if (tmin < best) {
            best = tmin;
            g.nt = c.first;
            g.eg = c.second;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != M2L_OK) return st;
    g.tuned_ms = best;
    std::lock_guard<std::mutex> lock(g_tc_tune_mutex);
    g_tc_tune_cache[key] = std::make_tuple(g.nt, g.eg, best);
    return M2L_OK;
}

}  // namespace

m2l_status tc_batch_create(const m2l_plan *const *plans, int nbatch, const void *const *in, void *const *out,
                           int precision, cudaStream_t s, TcBatch **out_batch)
{
    *out_batch = nullptr;
    std::map<int, std::vector<ProbInfo>> by_n3;
    for (int i = 0; i < nbatch; ++i) {
        const m2l_plan *pl = plans[i];
        const m2l_ops *ops = pl->ops;
        if (m2l_status st = check_device(ops)) return st;
        if (ops->eps > 0) { set_error("the tensor-core batch takes full-rank operators"); return M2L_EUNSUPPORTED; }
        if (ops->n3 > 256) {
            set_error("the tensor-core batch takes ell <= 6, got ell = %d", ops->ell);
            return M2L_EUNSUPPORTED;
        }
        if (pl->b.nnz > 0)
            if (m2l_status st = ensure_records(ops, pl->b, s)) return st;
        ProbInfo p;
        p.plan = pl;
        p.in = static_cast<const float *>(in[i]);
        p.out = static_cast<float *>(out[i]);
        memset(p.off, 0, sizeof(p.off));
        if (pl->b.nnz > 0) {
            M2L_CUDA(cudaStreamSynchronize(s));
            M2L_CUDA(cudaMemcpy(p.off, pl->b.class_off.p, sizeof(p.off), cudaMemcpyDeviceToHost));
        }
        p.scale = ops->homogeneous ? pow(pl->width / ops->ref_width, (double)ops->hom_degree) : 1.0;
        by_n3[ops->n3].push_back(p);
    }
    TcBatch *b = new TcBatch();
    b->precision = precision;
    b->status = nbatch > 0 ? plans[0]->ops->d_status : nullptr;
    m2l_status st = M2L_OK;
    for (auto &kv : by_n3) {
        TcGroup *g = new TcGroup();
        b->groups.push_back(g);
        if ((st = build_group(precision, kv.second, *g, s)) != M2L_OK) break;
        if ((st = tune_group(precision, *g, b->status, s)) != M2L_OK) break;
    }
    if (st == M2L_OK) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "tensor-core batch set-up");
    }
    if (st != M2L_OK) {
        delete b;
        return st;
    }
    *out_batch = b;
    return M2L_OK;
}

m2l_status tc_batch_run(const TcBatch *b, cudaStream_t s)
{
    for (const TcGroup *g : b->groups)
        if (m2l_status st = run_group(b->precision, *g, g->nt, g->eg, b->status, s, true)) return st;
    return M2L_OK;
}

void tc_batch_info(const TcBatch *b, int *tile_width, int64_t *tiles, double *tuned_ms, int *epilogue_groups,
                   int *launches)
{
    int nt = 0, eg = 0;
    int64_t t = 0;
    double ms = 0.0;
    for (const TcGroup *g : b->groups) {
        if (g->nt > nt) nt = g->nt;
        if (g->eg > eg) eg = g->eg;
        t += g->nt == 32 ? g->tiles32 : g->tiles64;
        ms += g->tuned_ms;
    }
    if (tile_width) *tile_width = nt;
    if (tiles) *tiles = t;
    if (tuned_ms) *tuned_ms = ms;
    if (epilogue_groups) *epilogue_groups = eg;
    if (launches) *launches = (int)b->groups.size();
}

int tc_batch_groups(const TcBatch *b, int max, int *n3, int *tile_width, int *epilogue_groups)
{
    const int n = (int)b->groups.size();
    for (int i = 0; i < n && i < max; ++i) {
        n3[i] = b->groups[i]->n3;
        tile_width[i] = b->groups[i]->nt;
        epilogue_groups[i] = b->groups[i]->eg;
    }
    return n;
}

void tc_batch_free(TcBatch *b) { delete b; }

}  // namespace m2l
