// Step a3: classification of every interaction by its transfer vector and
// stable bucketing per unique operator (the first loop of Alg. 2, blocked
// along many target cells as in Sec. 4.2.3, "Blocking along multiple target
// cells").
//
// For list entry e = (X, Y): t = X - Y (Sec. 3.1), (p, g) = lut(t).  Entries
// are counting-sorted by p, keeping list order inside a bucket, so that each
// bucket is ordered by target and the epilogue can sum the columns of one
// target before its atomic add.  Output record: {Y, X | g << 26}.
#include "m2l_internal.cuh"

namespace m2l {
namespace {

constexpr int kScanThreads = 1024;

// Target of every list entry; validates the CSR offsets.
__global__ void tgt_of_kernel(int ntgt, int nnz, const int32_t *__restrict__ offsets,
                              int32_t *__restrict__ tgt_of, int *__restrict__ status)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= ntgt) return;
    const int o0 = offsets[warp], o1 = offsets[warp + 1];
    bool ok = (o0 >= 0) && (o1 >= o0) && (o1 <= nnz);
    if (warp == 0 && o0 != 0) ok = false;
    if (warp == ntgt - 1 && o1 != nnz) ok = false;
    if (!ok) {
        if (lane == 0) atomicOr(status, ST_BAD_INDEX);
        return;
    }
    for (int e = o0 + lane; e < o1; e += 32) tgt_of[e] = warp;
}

__device__ __forceinline__ uint16_t classify_entry(int e, const int32_t *__restrict__ tgt_of,
                                                   const int32_t *__restrict__ sources,
                                                   const int32_t *__restrict__ tgt_ijk,
                                                   const int32_t *__restrict__ src_ijk, int nsrc,
                                                   const uint16_t *__restrict__ lut, int *status)
{
    const int x = tgt_of[e];
    const int y = sources[e];
    if (x < 0 || y < 0 || y >= nsrc) {
        atomicOr(status, ST_BAD_INDEX);
        return 0xFFFF;
    }
    const int t0 = tgt_ijk[3 * x] - src_ijk[3 * y];
    const int t1 = tgt_ijk[3 * x + 1] - src_ijk[3 * y + 1];
    const int t2 = tgt_ijk[3 * x + 2] - src_ijk[3 * y + 2];
    if (abs(t0) > 3 || abs(t1) > 3 || abs(t2) > 3) {
        atomicOr(status, ST_BAD_PAIR);
        return 0xFFFF;
    }
    const uint16_t c = lut[(t0 + 3) + 7 * (t1 + 3) + 49 * (t2 + 3)];
    if (c == 0xFFFF) atomicOr(status, ST_BAD_PAIR);
    return c;
}

constexpr int kSegWarps = kSegEntries / 256;   // warps per segment block (one round of 8 x 32 each)

// One block per segment of kSegEntries entries, warp w taking entries
// [w 256, (w+1) 256) of it: the class code of every entry (written for the
// scatter) and the per-class counts of the segment.
__global__ void __launch_bounds__(kSegWarps * 32)
classify_count_kernel(int nnz, int nseg, const int32_t *__restrict__ tgt_of, const int32_t *__restrict__ sources,
                      const int32_t *__restrict__ tgt_ijk, const int32_t *__restrict__ src_ijk, int nsrc,
                      const uint16_t *__restrict__ lut, uint16_t *__restrict__ code, int32_t *__restrict__ seg_counts,
                      int *__restrict__ status)
{
    __shared__ int cnt[kSegWarps][17];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int seg = blockIdx.x;
    for (int i = threadIdx.x; i < kSegWarps * 17; i += blockDim.x) cnt[i / 17][i % 17] = 0;
    __syncthreads();
    const int e0 = seg * kSegEntries + w * 256;
    const int e1 = min(nnz, seg * kSegEntries + kSegEntries);
    int cls[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int e = e0 + 32 * u + lane;
        cls[u] = 17;
        if (e < e1) {
            const uint16_t c = classify_entry(e, tgt_of, sources, tgt_ijk, src_ijk, nsrc, lut, status);
            code[e] = c;
            cls[u] = (c == 0xFFFF) ? 16 : (c & 0xFF);
        }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const unsigned peers = __match_any_sync(0xffffffffu, cls[u]);
        if (cls[u] < 17 && lane == __ffs(peers) - 1) cnt[w][cls[u]] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    if (threadIdx.x < 17) {
        int sum = 0;
#pragma unroll
        for (int k = 0; k < kSegWarps; ++k) sum += cnt[k][threadIdx.x];
        seg_counts[(size_t)threadIdx.x * nseg + seg] = sum;
    }
}

// Exclusive scan of n ints by one block of kScanThreads threads; returns the
// total to every thread.  Each round covers 8 kScanThreads elements, eight
// consecutive ones per thread.
__device__ int block_exclusive_scan(const int32_t *__restrict__ in, int32_t *__restrict__ out, int n)
{
    __shared__ int warp_sums[kScanThreads / 32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int base = 0; base < n; base += 8 * kScanThreads) {
        const int i0 = base + 8 * threadIdx.x;
        int v[8];
        int tsum = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            v[k] = (i0 + k < n) ? in[i0 + k] : 0;
            tsum += v[k];
        }
        int incl = tsum;
        for (int d = 1; d < 32; d <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += u;
        }
        if (lane == 31) warp_sums[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int s = warp_sums[lane];
            for (int d = 1; d < 32; d <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, s, d);
                if (lane >= d) s += u;
            }
            warp_sums[lane] = s;   // inclusive over warps
        }
        __syncthreads();
        int run = carry + (wid > 0 ? warp_sums[wid - 1] : 0) + incl - tsum;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (i0 + k < n) out[i0 + k] = run;
            run += v[k];
        }
        __syncthreads();
        if (threadIdx.x == kScanThreads - 1) carry = run;
        __syncthreads();
    }
    return carry;
}

// Single-block exclusive scan of n ints; out[n] = total.
__global__ void __launch_bounds__(kScanThreads) exclusive_scan_kernel(const int32_t *__restrict__ in,
                                                                      int32_t *__restrict__ out, int n)
{
    const int total = block_exclusive_scan(in, out, n);
    if (threadIdx.x == 0) out[n] = total;
}

// Per-class positions of the segments: block c scans row c of counts [17][nseg]
// into pos, then stores the row total in counts[c nseg] (the row is read by now).
__global__ void __launch_bounds__(kScanThreads) row_scan_kernel(int32_t *__restrict__ counts,
                                                                int32_t *__restrict__ pos, int nseg)
{
    const int c = blockIdx.x;
    const int total = block_exclusive_scan(counts + (size_t)c * nseg, pos + (size_t)c * nseg, nseg);
    if (threadIdx.x == 0) counts[(size_t)c * nseg] = total;
}

// Bucket starts from the class totals left by row_scan_kernel in counts[c nseg].
__global__ void class_offsets_kernel(int nseg, int nnz, const int32_t *__restrict__ counts,
                                     int32_t *__restrict__ class_off)
{
    if (threadIdx.x != 0) return;
    int run = 0;
    for (int c = 0; c < 17; ++c) {
        class_off[c] = run;
        run += counts[(size_t)c * nseg];
    }
    class_off[17] = nnz;
}

// One block per segment, warp w taking entries [w 256, (w+1) 256) of it, in
// order: the counts of each warp, then stable positions inside each bucket
// from the segment's position and the counts of the warps before.
__global__ void __launch_bounds__(kSegWarps * 32)
scatter_kernel(int nnz, int nseg, const uint16_t *__restrict__ code, const int32_t *__restrict__ tgt_of,
               const int32_t *__restrict__ sources, const int32_t *__restrict__ seg_pos,
               const int32_t *__restrict__ class_off, int2 *__restrict__ rec)
{
    __shared__ int cnt[kSegWarps][17];
    __shared__ int base[kSegWarps][17];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int seg = blockIdx.x;
    for (int i = threadIdx.x; i < kSegWarps * 17; i += blockDim.x) cnt[i / 17][i % 17] = 0;
    __syncthreads();
    const int e0 = seg * kSegEntries + w * 256;
    const int e1 = min(nnz, seg * kSegEntries + kSegEntries);
    const unsigned lt = (1u << lane) - 1u;
    int cls[8], src[8], tgt[8];
    uint16_t cc[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int e = e0 + 32 * u + lane;
        cls[u] = 17;
        cc[u] = 0xFFFF;
        src[u] = 0;
        tgt[u] = 0;
        if (e < e1) {
            cc[u] = code[e];
            cls[u] = (cc[u] == 0xFFFF) ? 16 : (cc[u] & 0xFF);
            src[u] = sources[e];
            tgt[u] = tgt_of[e];
        }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const unsigned peers = __match_any_sync(0xffffffffu, cls[u]);
        if (cls[u] < 17 && lane == __ffs(peers) - 1) cnt[w][cls[u]] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    if (threadIdx.x < 17) {
        int run = class_off[threadIdx.x] + seg_pos[(size_t)threadIdx.x * nseg + seg];
#pragma unroll
        for (int k = 0; k < kSegWarps; ++k) {
            base[k][threadIdx.x] = run;
            run += cnt[k][threadIdx.x];
        }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const unsigned peers = __match_any_sync(0xffffffffu, cls[u]);
        int pos = 0;
        if (cls[u] < 17) pos = base[w][cls[u]] + __popc(peers & lt);
        __syncwarp();
        if (cls[u] < 17 && lane == __ffs(peers) - 1) base[w][cls[u]] += __popc(peers);
        __syncwarp();
        if (cls[u] < 16) rec[pos] = make_int2(src[u], rec_pack(tgt[u], (int)(cc[u] >> 8)));
    }
}

// ---- list transposition for the adjoint ----
__global__ void count_sources_kernel(int nnz, int nsrc, const int32_t *__restrict__ tgt_of,
                                     const int32_t *__restrict__ sources, int32_t *__restrict__ cnt,
                                     int *__restrict__ status)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += gridDim.x * blockDim.x) {
        const int y = sources[e];
        if (y < 0 || y >= nsrc || tgt_of[e] < 0) {
            atomicOr(status, ST_BAD_INDEX);
            continue;
        }
        atomicAdd(cnt + y, 1);
    }
}

__global__ void fill_transposed_kernel(int nnz, int nsrc, const int32_t *__restrict__ tgt_of,
                                       const int32_t *__restrict__ sources, int32_t *__restrict__ cursor,
                                       int32_t *__restrict__ t_src)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += gridDim.x * blockDim.x) {
        const int y = sources[e];
        const int x = tgt_of[e];
        if (y < 0 || y >= nsrc || x < 0) continue;
        const int pos = atomicAdd(cursor + y, 1);
        t_src[pos] = x;
    }
}

// One warp per transposed row: sort ascending by rank counting, so the
// transposed list is independent of the atomic fill order.
__global__ void sort_rows_kernel(int nrows, const int32_t *__restrict__ off, int32_t *__restrict__ vals,
                                 int32_t *__restrict__ scratch)
{
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= nrows) return;
    const int o0 = off[row], o1 = off[row + 1];
    for (int i = o0 + lane; i < o1; i += 32) {
        const int v = vals[i];
        int r = 0;
        for (int j = o0; j < o1; ++j) {
            const int u = vals[j];
            r += (u < v) || (u == v && j < i);
        }
        scratch[o0 + r] = v;
    }
    __syncwarp();
    for (int i = o0 + lane; i < o1; i += 32) vals[i] = scratch[i];
}

}  // namespace

m2l_status launch_exclusive_scan(const int32_t *in, int32_t *out, int n, cudaStream_t s)
{
    exclusive_scan_kernel<<<1, kScanThreads, 0, s>>>(in, out, n);
    M2L_LAUNCH_CHECK("exclusive_scan_kernel");
    return M2L_OK;
}

static m2l_status bucket(const m2l_ops *ops, int ntgt, int nsrc, int nnz, const int32_t *tgt_ijk,
                         const int32_t *src_ijk, const int32_t *offsets, const int32_t *sources, Buckets &b,
                         cudaStream_t s)
{
    m2l_status st;
    b.dense.valid = false;
    b.have_rec = true;
    const int nseg = (nnz + kSegEntries - 1) / kSegEntries;
    if ((st = b.rec.ensure((size_t)(nnz > 0 ? nnz : 1) * sizeof(int2))) != M2L_OK) return st;
    // low-rank operators: the first-pass products of the tensor-core apply, one row per record
    if (ops->eps > 0 && nnz > 0)
        if ((st = b.lrz.ensure((size_t)nnz * kLrRankPad * sizeof(float))) != M2L_OK) return st;
    if (nnz > 0 && dense_eligible(ops, ntgt, nnz)) {
        // full level: the dense classification only; the operator buckets are derived
        // from it if a bucketed kernel is asked for (their buffers are allocated now)
        if ((st = b.class_off.ensure(18 * sizeof(int32_t))) != M2L_OK) return st;
        b.nnz = nnz;
        b.ntgt = ntgt;
        b.nsrc = nsrc;
        st = dense_classify(ops, ntgt, nsrc, nnz, tgt_ijk, src_ijk, offsets, sources, b.dense, s);
        if (st == M2L_OK) b.have_rec = false;
        return st;
    }
    if ((st = b.tgt_of.ensure((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t))) != M2L_OK) return st;
    if ((st = b.code.ensure((size_t)(nnz > 0 ? nnz : 1) * sizeof(uint16_t))) != M2L_OK) return st;
    if ((st = b.seg.ensure((size_t)(17 * (size_t)nseg + 1) * 2 * sizeof(int32_t))) != M2L_OK) return st;
    if ((st = b.class_off.ensure(18 * sizeof(int32_t))) != M2L_OK) return st;
    b.nnz = nnz;
    b.ntgt = ntgt;
    b.nsrc = nsrc;
    if (nnz == 0) {
        M2L_CUDA(cudaMemsetAsync(b.class_off.p, 0, 18 * sizeof(int32_t), s));
        return M2L_OK;
    }
    M2L_CUDA(cudaMemsetAsync(b.tgt_of.p, 0xFF, (size_t)nnz * sizeof(int32_t), s));
    if (ntgt > 0) {
        const int threads = 256;
        const int blocks = (int)(((long)ntgt * 32 + threads - 1) / threads);
        tgt_of_kernel<<<blocks, threads, 0, s>>>(ntgt, nnz, offsets, b.tgt_of.as<int32_t>(), ops->d_status);
        M2L_LAUNCH_CHECK("tgt_of_kernel");
    }
    int32_t *counts = b.seg.as<int32_t>();
    int32_t *pos = counts + 17 * (size_t)nseg + 1;
    classify_count_kernel<<<nseg, kSegWarps * 32, 0, s>>>(nnz, nseg, b.tgt_of.as<int32_t>(), sources, tgt_ijk,
                                                           src_ijk, nsrc, ops->lut.as<uint16_t>(),
                                                           b.code.as<uint16_t>(), counts, ops->d_status);
    M2L_LAUNCH_CHECK("classify_count_kernel");
    row_scan_kernel<<<17, kScanThreads, 0, s>>>(counts, pos, nseg);
    M2L_LAUNCH_CHECK("row_scan_kernel");
    class_offsets_kernel<<<1, 32, 0, s>>>(nseg, nnz, counts, b.class_off.as<int32_t>());
    M2L_LAUNCH_CHECK("class_offsets_kernel");
    scatter_kernel<<<nseg, kSegWarps * 32, 0, s>>>(nnz, nseg, b.code.as<uint16_t>(), b.tgt_of.as<int32_t>(), sources,
                                                    pos, b.class_off.as<int32_t>(), b.rec.as<int2>());
    M2L_LAUNCH_CHECK("scatter_kernel");
    return M2L_OK;
}

m2l_status classify(const m2l_ops *ops, const m2l_level *lv, int adjoint, Buckets &b, cudaStream_t s)
{
    if (!adjoint)
        return bucket(ops, lv->ncells_tgt, lv->ncells_src, lv->nnz, lv->tgt_ijk, lv->src_ijk, lv->il_offsets,
                      lv->il_sources, b, s);
    // Adjoint: transpose the list (rows over sources), then bucket it with the
    // roles of the two cell sets exchanged; t becomes -t, whose operator is K_t^T.
    const int nnz = lv->nnz, ntgt = lv->ncells_tgt, nsrc = lv->ncells_src;
    m2l_status st;
    if ((st = b.tgt_of.ensure((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t))) != M2L_OK) return st;
    if ((st = b.t_off.ensure((size_t)(nsrc + 2) * 2 * sizeof(int32_t))) != M2L_OK) return st;
    if ((st = b.t_src.ensure((size_t)(nnz > 0 ? nnz : 1) * 2 * sizeof(int32_t))) != M2L_OK) return st;
    if ((st = b.t_cursor.ensure((size_t)(nsrc + 1) * sizeof(int32_t))) != M2L_OK) return st;
    int32_t *cnt = b.t_off.as<int32_t>();
    int32_t *toff = cnt + nsrc + 1;
    int32_t *tsrc = b.t_src.as<int32_t>();
    int32_t *scratch = tsrc + (nnz > 0 ? nnz : 1);
    M2L_CUDA(cudaMemsetAsync(cnt, 0, (size_t)(nsrc + 1) * sizeof(int32_t), s));
    if (nnz > 0) {
        M2L_CUDA(cudaMemsetAsync(b.tgt_of.p, 0xFF, (size_t)nnz * sizeof(int32_t), s));
        if (ntgt > 0) {
            const int blocks = (int)(((long)ntgt * 32 + 255) / 256);
            tgt_of_kernel<<<blocks, 256, 0, s>>>(ntgt, nnz, lv->il_offsets, b.tgt_of.as<int32_t>(), ops->d_status);
            M2L_LAUNCH_CHECK("tgt_of_kernel");
        }
        const int eb = (nnz + 255) / 256 < 4096 ? (nnz + 255) / 256 : 4096;
        count_sources_kernel<<<eb, 256, 0, s>>>(nnz, nsrc, b.tgt_of.as<int32_t>(), lv->il_sources, cnt,
                                               ops->d_status);
        M2L_LAUNCH_CHECK("count_sources_kernel");
    }
    exclusive_scan_kernel<<<1, kScanThreads, 0, s>>>(cnt, toff, nsrc);
    M2L_LAUNCH_CHECK("exclusive_scan_kernel");
    if (nnz > 0) {
        M2L_CUDA(cudaMemcpyAsync(b.t_cursor.p, toff, (size_t)nsrc * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        const int eb = (nnz + 255) / 256 < 4096 ? (nnz + 255) / 256 : 4096;
        fill_transposed_kernel<<<eb, 256, 0, s>>>(nnz, nsrc, b.tgt_of.as<int32_t>(), lv->il_sources,
                                                 b.t_cursor.as<int32_t>(), tsrc);
        M2L_LAUNCH_CHECK("fill_transposed_kernel");
        if (nsrc > 0) {
            const int blocks = (int)(((long)nsrc * 32 + 255) / 256);
            sort_rows_kernel<<<blocks, 256, 0, s>>>(nsrc, toff, tsrc, scratch);
            M2L_LAUNCH_CHECK("sort_rows_kernel");
        }
    }
    // entries rejected while counting are absent from the transposed list, so
    // its length is toff[nsrc], which only the device knows: bucket all nnz
    // slots; the tail beyond toff[nsrc] is marked invalid by tgt_of = -1.
    return bucket(ops, nsrc, ntgt, nnz, lv->src_ijk, lv->tgt_ijk, toff, tsrc, b, s);
}

}  // namespace m2l

namespace m2l {

// Bucketing into caller-provided device buffers (no allocation): the same
// kernels as bucket(), with rec [nnz], tgt_of [nnz], code [nnz],
// seg [2 * (17 * nseg + 1)] and class_off [18] supplied by the caller.
m2l_status bucket_raw(const m2l_ops *ops, int ntgt, int nsrc, int nnz, const int32_t *tgt_ijk,
                      const int32_t *src_ijk, const int32_t *offsets, const int32_t *sources, int2 *rec,
                      int32_t *tgt_of, uint16_t *code, int32_t *seg, int32_t *class_off, cudaStream_t s)
{
    if (nnz == 0) {
        M2L_CUDA(cudaMemsetAsync(class_off, 0, 18 * sizeof(int32_t), s));
        return M2L_OK;
    }
    const int nseg = (nnz + kSegEntries - 1) / kSegEntries;
    M2L_CUDA(cudaMemsetAsync(tgt_of, 0xFF, (size_t)nnz * sizeof(int32_t), s));
    if (ntgt > 0) {
        const int blocks = (int)(((long)ntgt * 32 + 255) / 256);
        tgt_of_kernel<<<blocks, 256, 0, s>>>(ntgt, nnz, offsets, tgt_of, ops->d_status);
        M2L_LAUNCH_CHECK("tgt_of_kernel");
    }
    int32_t *counts = seg;
    int32_t *pos = seg + 17 * (size_t)nseg + 1;
    classify_count_kernel<<<nseg, kSegWarps * 32, 0, s>>>(nnz, nseg, tgt_of, sources, tgt_ijk, src_ijk, nsrc,
                                                           ops->lut.as<uint16_t>(), code, counts, ops->d_status);
    M2L_LAUNCH_CHECK("classify_count_kernel");
    row_scan_kernel<<<17, kScanThreads, 0, s>>>(counts, pos, nseg);
    M2L_LAUNCH_CHECK("row_scan_kernel");
    class_offsets_kernel<<<1, 32, 0, s>>>(nseg, nnz, counts, class_off);
    M2L_LAUNCH_CHECK("class_offsets_kernel");
    scatter_kernel<<<nseg, kSegWarps * 32, 0, s>>>(nnz, nseg, code, tgt_of, sources, pos, class_off, rec);
    M2L_LAUNCH_CHECK("scatter_kernel");
    return M2L_OK;
}

}  // namespace m2l
