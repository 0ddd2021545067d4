// Interaction lists of one level (Sec. 3.2; Alg. 1 for asymptotically
// smooth kernels): Y is in the list of X when the parents are neighbours and
// X, Y are not, |X - Y|_inf >= 2.  The candidates of X are the 8 children of
// each of the 27 neighbours of its parent (6^3 = 216 cells, Sec. 3.2).
#include "m2l_internal.cuh"

namespace m2l {
namespace {

__global__ void extent_kernel(int n, const int32_t *__restrict__ ijk, int *__restrict__ ext)
{
    int mx = 0, mn = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 3 * n; i += gridDim.x * blockDim.x) {
        mx = max(mx, ijk[i]);
        mn = min(mn, ijk[i]);
    }
    atomicMax(ext, mx);
    atomicMin(ext + 1, mn);
}

__global__ void scatter_cells_kernel(int n, const int32_t *__restrict__ ijk, int side, int *__restrict__ table,
                                     int *__restrict__ dup)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const long key = ijk[3 * i] + (long)side * (ijk[3 * i + 1] + (long)side * ijk[3 * i + 2]);
        if (atomicCAS(table + key, -1, i) != -1) atomicOr(dup, 1);
    }
}

__device__ __forceinline__ int candidate(int idx, const int *x, int side, const int *__restrict__ table)
{
    const int d = idx >> 3, ch = idx & 7;
    const int dd[3] = {d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1};
    int y[3];
    for (int i = 0; i < 3; ++i) {
        y[i] = 2 * ((x[i] >> 1) + dd[i]) + ((ch >> i) & 1);
        if (y[i] < 0 || y[i] >= side) return -1;
    }
    const int m = max(abs(x[0] - y[0]), max(abs(x[1] - y[1]), abs(x[2] - y[2])));
    if (m < 2) return -1;
    return table[y[0] + (long)side * (y[1] + (long)side * y[2])];
}

// one warp per target: count (fill == 0) or write the sorted list (fill == 1)
__global__ void lists_kernel(int ntgt, const int32_t *__restrict__ tgt_ijk, int side,
                             const int *__restrict__ table, int32_t *__restrict__ counts,
                             const int32_t *__restrict__ offsets, int32_t *__restrict__ sources, int fill)
{
    __shared__ int buf[8][216];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = blockIdx.x * 8 + wib;
    if (t >= ntgt) return;
    int x[3] = {tgt_ijk[3 * t], tgt_ijk[3 * t + 1], tgt_ijk[3 * t + 2]};
    bool in_range = x[0] >= 0 && x[1] >= 0 && x[2] >= 0 && x[0] < side && x[1] < side && x[2] < side;
    int n = 0;
    for (int base = 0; base < 216; base += 32) {
        const int idx = base + lane;
        const int y = (in_range && idx < 216) ? candidate(idx, x, side, table) : -1;
        const unsigned m = __ballot_sync(0xffffffffu, y >= 0);
        if (y >= 0) buf[wib][n + __popc(m & ((1u << lane) - 1u))] = y;
        n += __popc(m);
    }
    __syncwarp();
    if (!fill) {
        if (lane == 0) counts[t] = n;
        return;
    }
    const int o = offsets[t];
    for (int i = lane; i < n; i += 32) {
        const int v = buf[wib][i];
        int r = 0;
        for (int j = 0; j < n; ++j) r += buf[wib][j] < v;
        sources[o + r] = v;
    }
}

}  // namespace
}  // namespace m2l

using namespace m2l;

extern "C" m2l_status m2l_build_lists(int ncells_tgt, const int32_t *tgt_ijk, int ncells_src, const int32_t *src_ijk,
                                      int32_t *il_offsets, int32_t *il_sources, int64_t *nnz_out, void *stream)
{
    if (ncells_tgt < 0 || ncells_src < 0 || !il_offsets || !nnz_out ||
        (ncells_tgt > 0 && !tgt_ijk) || (ncells_src > 0 && !src_ijk)) {
        set_error("bad list-builder arguments");
        return M2L_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    DevBuf ext, table, cnt, dup;
    ScratchGuard guard{&ext, &table, &cnt, &dup};
    m2l_status st;
    if ((st = ext.ensure(2 * sizeof(int))) != M2L_OK) return st;
    if ((st = dup.ensure(sizeof(int))) != M2L_OK) return st;
    M2L_CUDA(cudaMemsetAsync(ext.p, 0, 2 * sizeof(int), s));
    M2L_CUDA(cudaMemsetAsync(dup.p, 0, sizeof(int), s));
    if (ncells_src > 0) {
        extent_kernel<<<64, 256, 0, s>>>(ncells_src, src_ijk, ext.as<int>());
        M2L_LAUNCH_CHECK("extent_kernel");
    }
    if (ncells_tgt > 0) {
        extent_kernel<<<64, 256, 0, s>>>(ncells_tgt, tgt_ijk, ext.as<int>());
        M2L_LAUNCH_CHECK("extent_kernel");
    }
    int hext[2];
    M2L_CUDA(cudaMemcpyAsync(hext, ext.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    M2L_CUDA(cudaStreamSynchronize(s));
    if (hext[1] < 0) { set_error("negative cell coordinate"); return M2L_EINVAL; }
    int side = 1;
    while (side <= hext[0]) side <<= 1;
    if (side > 256) { set_error("cell coordinates beyond 255 (level > 8)"); return M2L_EUNSUPPORTED; }
    const size_t cells = (size_t)side * side * side;
    if ((st = table.ensure(cells * sizeof(int))) != M2L_OK) return st;
    if ((st = cnt.ensure((size_t)(ncells_tgt + 1) * sizeof(int))) != M2L_OK) return st;
    M2L_CUDA(cudaMemsetAsync(table.p, 0xFF, cells * sizeof(int), s));
    if (ncells_src > 0) {
        scatter_cells_kernel<<<(ncells_src + 255) / 256, 256, 0, s>>>(ncells_src, src_ijk, side, table.as<int>(),
                                                                     dup.as<int>());
        M2L_LAUNCH_CHECK("scatter_cells_kernel");
    }
    M2L_CUDA(cudaMemsetAsync(cnt.p, 0, (size_t)(ncells_tgt + 1) * sizeof(int), s));
    const int blocks = (ncells_tgt + 7) / 8;
    if (ncells_tgt > 0) {
        lists_kernel<<<blocks, 256, 0, s>>>(ncells_tgt, tgt_ijk, side, table.as<int>(), cnt.as<int32_t>(), nullptr,
                                            nullptr, 0);
        M2L_LAUNCH_CHECK("lists_kernel(count)");
    }
    if ((st = launch_exclusive_scan(cnt.as<int32_t>(), il_offsets, ncells_tgt, s)) != M2L_OK) return st;
    int total = 0, hdup = 0;
    M2L_CUDA(cudaMemcpyAsync(&total, il_offsets + ncells_tgt, sizeof(int), cudaMemcpyDeviceToHost, s));
    M2L_CUDA(cudaMemcpyAsync(&hdup, dup.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    M2L_CUDA(cudaStreamSynchronize(s));
    if (hdup) { set_error("duplicate source cell coordinates"); return M2L_EINVAL; }
    *nnz_out = total;
    if (il_sources && ncells_tgt > 0) {
        lists_kernel<<<blocks, 256, 0, s>>>(ncells_tgt, tgt_ijk, side, table.as<int>(), nullptr, il_offsets,
                                            il_sources, 1);
        M2L_LAUNCH_CHECK("lists_kernel(fill)");
        M2L_CUDA(cudaStreamSynchronize(s));
    }
    return M2L_OK;
}
