// The target-stationary tensor-core M2L for full levels (ell <= 5).
//
// Alg. 2 blocks the interactions of one unique operator K_p along many target
// cells (Sec. 4.2.3) and pays for it with a permutation of every source
// vector (Eq. (30)) and of every result (Eq. (32)).  On the tcgen05 tensor
// cores that per-column permutation work, not the product, bounds the
// bucketed kernel.  This file moves the permutation onto the operator once
// per transfer vector instead: K_t = P_t K_p P_t^T is written out, from the
// 16 FP64 masters and the 48 tables sigma_g (Eq. (25)), as one pre-swizzled
// operand image per t (K_t[a][b] = K_p[sigma(a)][sigma(b)]).  Then, for a
// unit of up to nu target cells (columns) of one octant, every transfer
// vector of the unit is one product D += K_t W_t, where column j of W_t is
// the unpermuted multipole of the source X_j - t (zero if there is none);
// the sum over the interaction list of Eq. (7) runs on chip and each local is
// written once per launch.
//
// Classification (step a3 for this kernel): targets are ranked by the octant
// of their cell (stable), each octant's run is split into balanced units,
// and every list entry (X, Y) writes Y into tab[unit(X)][slot(t)][column(X)]
// (slot(t) = (t1+3) + 7 (t2+3) + 49 (t3+3)).  Per unit the slots holding an
// entry are listed in ascending order.
//
// Apply: the multipoles are first split once per call (hi/lo parts of
// BF16x3 / TF32x3, the TF32 rounding of TF32) into rows of [parts][kpad]
// plus one zero row.  One persistent CTA per SM walks its units; per unit
// and active slot, one producer thread brings each 128-byte K column of the
// slot's operator image into shared memory with one bulk copy, and 128
// producer threads copy the nu source rows of the same K column with 16-byte
// cp.async copies, straight into the 128-byte-swizzled UMMA operand layout;
// one thread of the MMA warp issues tcgen05.mma (M = 128, N = nu) for one
// slot into one of two TMEM accumulators (the K sum of one transfer vector);
// sixteen epilogue warps read each slot's product with tcgen05.ld and add it
// into FP32 registers, and at the end of the unit add the sums, times
// w^degree, to the locals: one atomic add per
// (target, node) and launch.  Every wait is bounded (about two seconds); on
// expiry the CTA records M2L_ETIMEOUT, drains its own copies and MMAs,
// frees TMEM and returns.
#include "m2l_tcgen05.cuh"

namespace m2l {
namespace {

constexpr int kSlots = 343;           // transfer-vector slots, |t_i| <= 3
constexpr int kSlotRow = 344;         // per unit: count, then up to 343 slots
constexpr int kDenseMinTargets = 16384;   // 8 octants x 2048: units of >= 128 columns on 152 SMs
constexpr int kRankBlock = 256;       // targets per block of the octant ranking

// ---------------------------------------------------------------- classification
// Octant of every target cell and its stable rank among the targets of the
// same octant within its block of kRankBlock targets; per-block octant counts.
__global__ void __launch_bounds__(kRankBlock)
dense_rank_kernel(int ntgt, int nblk, const int32_t *__restrict__ tgt_ijk, int32_t *__restrict__ rank,
                  int32_t *__restrict__ bcnt)
{
    __shared__ int wcnt[kRankBlock / 32][8];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x = blockIdx.x * kRankBlock + threadIdx.x;
    int o = 8;
    if (x < ntgt)
        o = (tgt_ijk[3 * x] & 1) | ((tgt_ijk[3 * x + 1] & 1) << 1) | ((tgt_ijk[3 * x + 2] & 1) << 2);
    if (lane < 8) wcnt[w][lane] = 0;
    __syncwarp();
    const unsigned peers = __match_any_sync(0xffffffffu, o);
    const int rw = __popc(peers & ((1u << lane) - 1u));
    if (o < 8 && lane == __ffs(peers) - 1) wcnt[w][o] = __popc(peers);
    __syncthreads();
    if (o < 8) {
        int r = rw;
        for (int k = 0; k < w; ++k) r += wcnt[k][o];
        rank[x] = r | (o << 16);
    }
    if (threadIdx.x < 8) {
        int sum = 0;
        for (int k = 0; k < kRankBlock / 32; ++k) sum += wcnt[k][threadIdx.x];
        bcnt[(size_t)threadIdx.x * nblk + blockIdx.x] = sum;
    }
}

// Units per octant from the scanned block counts (one thread).
// meta: [0] units U, [1 + o] octant size n_o, [9 + o] octant start, [17 + o]
// first unit of octant o, [25 + o] units m_o of octant o.
__global__ void dense_meta_kernel(int nblk, int nu, const int32_t *__restrict__ bbase, int32_t *__restrict__ meta)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int u = 0;
    const int total = bbase[8 * nblk];
    for (int o = 0; o < 8; ++o) {
        const int start = bbase[o * nblk];
        const int end = (o < 7) ? bbase[(o + 1) * nblk] : total;
        const int n = end - start;
        const int m = (n + nu - 1) / nu;
        meta[1 + o] = n;
        meta[9 + o] = start;
        meta[17 + o] = u;
        meta[25 + o] = m;
        u += m;
    }
    meta[0] = u;
}

// Unit and column of every target: octant o's run of n targets is split into m
// units, unit k holding positions [floor(k n / m), floor((k + 1) n / m)).
__global__ void dense_place_kernel(int ntgt, int nblk, int nu, const int32_t *__restrict__ rank,
                                   const int32_t *__restrict__ bbase, const int32_t *__restrict__ meta,
                                   int32_t *__restrict__ unit_col, int32_t *__restrict__ unit_tgt)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= ntgt) return;
    const int rk = rank[x] & 0xFFFF, o = rank[x] >> 16;
    const int blk = x / kRankBlock;
    const long long n = meta[1 + o], m = meta[25 + o];
    const long long pos = (long long)bbase[o * nblk + blk] + rk - meta[9 + o];
    long long k = pos * m / n;
    while (k + 1 < m && (k + 1) * n / m <= pos) ++k;
    const int u = meta[17 + o] + (int)k;
    const int j = (int)(pos - k * n / m);
    unit_col[x] = (u << 9) | j;
    unit_tgt[(size_t)u * nu + j] = x;
}

// One warp per target row of the CSR list: each entry (X, Y) writes Y + 1 into
// tab[unit(X)][slot(t)][column(X)] and flags the slot of the unit.  Entries
// that are not far-field pairs, indices out of range and repeated (X, t) pairs
// set the status word and are skipped.  A row's slots are marked in a bit set
// in shared memory, so the table takes plain stores (a repeated (X, t) is found
// in the row, the only place it can occur).
constexpr int kFillThreads = 256;
constexpr int kSlotWords = (kSlots + 31) / 32;

__global__ void __launch_bounds__(kFillThreads)
dense_fill_kernel(int ntgt, int nsrc, int nnz, int nu, const int32_t *__restrict__ offsets,
                  const int32_t *__restrict__ sources, const int32_t *__restrict__ tgt_ijk,
                  const int32_t *__restrict__ src_ijk, const uint16_t *__restrict__ lut,
                  const int32_t *__restrict__ unit_col, int32_t *__restrict__ tab, int32_t *__restrict__ flags,
                  int *__restrict__ status)
{
    __shared__ unsigned seen_all[kFillThreads / 32][kSlotWords];
    const int x = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    unsigned *seen = seen_all[threadIdx.x >> 5];
    if (lane < kSlotWords) seen[lane] = 0u;
    __syncwarp();
    if (x >= ntgt) return;
    const int o0 = offsets[x], o1 = offsets[x + 1];
    if (o0 < 0 || o1 < o0 || o1 > nnz || (x == 0 && o0 != 0)) {
        if (lane == 0) atomicOr(status, ST_BAD_INDEX);
        return;
    }
    const int uc = unit_col[x];
    const int u = uc >> 9, j = uc & 511;
    const int xi = tgt_ijk[3 * x], xj = tgt_ijk[3 * x + 1], xk = tgt_ijk[3 * x + 2];
    for (int e = o0 + lane; e < o1; e += 32) {
        const int y = sources[e];
        if (y < 0 || y >= nsrc) {
            atomicOr(status, ST_BAD_INDEX);
            continue;
        }
        const int t0 = xi - src_ijk[3 * y], t1 = xj - src_ijk[3 * y + 1], t2 = xk - src_ijk[3 * y + 2];
        if (abs(t0) > 3 || abs(t1) > 3 || abs(t2) > 3) {
            atomicOr(status, ST_BAD_PAIR);
            continue;
        }
        const int slot = (t0 + 3) + 7 * (t1 + 3) + 49 * (t2 + 3);
        if (lut[slot] == 0xFFFF) {
            atomicOr(status, ST_BAD_PAIR);
            continue;
        }
        const unsigned bit = 1u << (slot & 31);
        if (atomicOr(seen + (slot >> 5), bit) & bit) {   // the same (X, t) twice
            atomicOr(status, ST_BAD_PAIR);
            continue;
        }
        tab[((size_t)u * kSlots + slot) * nu + j] = y + 1;
        flags[(size_t)u * kSlots + slot] = 1;
    }
}

// One warp per unit: the flagged slots in ascending order, count first.
__global__ void dense_slots_kernel(int umax, const int32_t *__restrict__ meta, const int32_t *__restrict__ flags,
                                   uint16_t *__restrict__ slots)
{
    const int u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (u >= umax) return;
    uint16_t *row = slots + (size_t)u * kSlotRow;
    if (u >= meta[0]) {
        if (lane == 0) row[0] = 0;
        return;
    }
    int n = 0;
    for (int c = 0; c < kSlots; c += 32) {
        const int slot = c + lane;
        const bool f = slot < kSlots && flags[(size_t)u * kSlots + slot] != 0;
        const unsigned m = __ballot_sync(0xffffffffu, f);
        if (f) row[1 + n + __popc(m & ((1u << lane) - 1u))] = (uint16_t)slot;
        n += __popc(m);
    }
    if (lane == 0) row[0] = (uint16_t)n;
}

}  // namespace

bool dense_eligible(const m2l_ops *ops, int ntgt, int nnz)
{
    // 189 far-field transfer vectors per target cell in a full level (Sec. 3.2):
    // the kernel pays for every (target, active t) column, so it takes levels
    // whose lists are at least half full; each operator K column it streams is
    // shared by a unit's columns, so it takes levels large enough for units of
    // at least 128 columns on every SM
    return ops->eps <= 0.0 && ops->n3 <= 128 && ntgt >= kDenseMinTargets && (double)nnz >= 0.5 * 189.0 * ntgt;
}

// Columns per unit: balance ~ntgt/8 targets per octant over the SMs, counting
// a unit's operator traffic as 64 columns of its own.
static int choose_nu(int ntgt)
{
    const int nsm = num_sms();
    const long per_oct = (ntgt + 7) / 8;
    int best = 256;
    long best_cost = -1;
    for (int nu = 256; nu >= 128; nu -= 16) {
        const long units = 8 * ((per_oct + nu - 1) / nu);
        const long rounds = (units + nsm - 1) / nsm;
        const long cost = rounds * (nu + 64);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = nu;
        }
    }
    return best;
}

m2l_status dense_classify(const m2l_ops *ops, int ntgt, int nsrc, int nnz, const int32_t *tgt_ijk,
                          const int32_t *src_ijk, const int32_t *offsets, const int32_t *sources, DenseBuckets &d,
                          cudaStream_t s)
{
    m2l_status st;
    const int nu = choose_nu(ntgt);
    const int umax = (ntgt + nu - 1) / nu + 8;
    const int nblk = (ntgt + kRankBlock - 1) / kRankBlock;
    if (umax >= (1 << 22)) {
        set_error("too many target units for the dense classification");
        return M2L_EUNSUPPORTED;
    }
    // work: rank [ntgt], unit_col [ntgt], bcnt [8 nblk + 1], bbase [8 nblk + 1], flags [umax][343]
    const size_t n_work = 2 * (size_t)ntgt + 2 * (8 * (size_t)nblk + 1) + (size_t)umax * kSlots;
    if ((st = d.work.ensure(n_work * sizeof(int32_t))) != M2L_OK) return st;
    if ((st = d.unit_tgt.ensure((size_t)umax * nu * sizeof(int32_t))) != M2L_OK) return st;
    if ((st = d.tab.ensure((size_t)umax * kSlots * nu * sizeof(int32_t))) != M2L_OK) return st;
    if ((st = d.slots.ensure((size_t)umax * kSlotRow * sizeof(uint16_t))) != M2L_OK) return st;
    if ((st = d.meta.ensure(64 * sizeof(int32_t))) != M2L_OK) return st;
    // split multipoles of any precision: up to two parts of 128 four-byte values per row
    if ((st = d.bsplit.ensure(((size_t)nsrc + 1) * 1024)) != M2L_OK) return st;
    d.umax = umax;
    d.nu = nu;
    d.ntgt = ntgt;
    d.nsrc = nsrc;
    d.nnz = nnz;
    d.valid = true;
    int32_t *rank = d.work.as<int32_t>();
    int32_t *unit_col = rank + ntgt;
    int32_t *bcnt = unit_col + ntgt;
    int32_t *bbase = bcnt + 8 * (size_t)nblk + 1;
    int32_t *flags = bbase + 8 * (size_t)nblk + 1;
    M2L_CUDA(cudaMemsetAsync(d.tab.p, 0, (size_t)umax * kSlots * nu * sizeof(int32_t), s));
    M2L_CUDA(cudaMemsetAsync(flags, 0, (size_t)umax * kSlots * sizeof(int32_t), s));
    M2L_CUDA(cudaMemsetAsync(d.unit_tgt.p, 0xFF, (size_t)umax * nu * sizeof(int32_t), s));
    dense_rank_kernel<<<nblk, kRankBlock, 0, s>>>(ntgt, nblk, tgt_ijk, rank, bcnt);
    M2L_LAUNCH_CHECK("dense_rank_kernel");
    if ((st = launch_exclusive_scan(bcnt, bbase, 8 * nblk, s)) != M2L_OK) return st;
    dense_meta_kernel<<<1, 32, 0, s>>>(nblk, nu, bbase, d.meta.as<int32_t>());
    M2L_LAUNCH_CHECK("dense_meta_kernel");
    dense_place_kernel<<<(ntgt + 255) / 256, 256, 0, s>>>(ntgt, nblk, nu, rank, bbase, d.meta.as<int32_t>(),
                                                           unit_col, d.unit_tgt.as<int32_t>());
    M2L_LAUNCH_CHECK("dense_place_kernel");
    if (nnz > 0) {
        const int blocks = (int)(((long)ntgt * 32 + kFillThreads - 1) / kFillThreads);
        dense_fill_kernel<<<blocks, kFillThreads, 0, s>>>(ntgt, nsrc, nnz, nu, offsets, sources, tgt_ijk, src_ijk,
                                                 ops->lut.as<uint16_t>(), unit_col, d.tab.as<int32_t>(), flags,
                                                 ops->d_status);
        M2L_LAUNCH_CHECK("dense_fill_kernel");
    }
    dense_slots_kernel<<<(umax * 32 + 255) / 256, 256, 0, s>>>(umax, d.meta.as<int32_t>(), flags,
                                                                d.slots.as<uint16_t>());
    M2L_LAUNCH_CHECK("dense_slots_kernel");
    return M2L_OK;
}

namespace {

// K columns (swizzle columns of 128 bytes) per operator row: kpad = katoms * (128 / esz).
template <int KIND>
__host__ __device__ constexpr int dense_katoms(int n3)
{
    return (n3 * TcTraits<KIND>::esz + 127) / 128;
}

// Operator image of every transfer-vector slot: K_t[a][b] = K_p[sigma_g(a)][sigma_g(b)]
// for (p, g) = lut[slot] (Eq. (25) with the orientation of the permutation
// tables), rows a < 128 (zero beyond ell^3), K padded with zeros to katoms
// swizzle columns.  Layout per slot: [katom][part][128 rows x 128 bytes],
// each block 128-byte swizzled (K-major UMMA operand), so that one K column
// of both parts is one contiguous bulk copy.  Slots without an operator (the
// near field) are left untouched and never read.
template <int KIND>
__global__ void dense_image_kernel(int n3, int katoms, const double *__restrict__ K, const int16_t *__restrict__ sigma,
                                   const uint16_t *__restrict__ lut, uint8_t *__restrict__ img)
{
    using Tr = TcTraits<KIND>;
    constexpr int E = 128 / Tr::esz;
    const int slot = blockIdx.y;
    const uint16_t c = lut[slot];
    if (c == 0xFFFF) return;
    const int p = c & 0xFF, g = c >> 8;
    const int kpad = katoms * E;
    const int16_t *sg = sigma + (size_t)g * n3;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < 128 * kpad; idx += gridDim.x * blockDim.x) {
        const int row = idx / kpad, kk = idx % kpad;
        const double x = (row < n3 && kk < n3) ? K[((size_t)p * n3 + sg[row]) * n3 + sg[kk]] : 0.0;
        const int ka = kk / E, e = kk % E;
        const int chunk = e / (16 / Tr::esz), within = e % (16 / Tr::esz);
        uint8_t *blk = img + ((size_t)slot * katoms + ka) * (Tr::nparts * 16384);
        const uint32_t off = swz_off(row, chunk) + (uint32_t)(within * Tr::esz);
        if constexpr (KIND == TC_BF16X3) {
            const __nv_bfloat16 h = __double2bfloat16(x);
            const __nv_bfloat16 l = __double2bfloat16(x - (double)__bfloat162float(h));
            *reinterpret_cast<__nv_bfloat16 *>(blk + off) = h;
            *reinterpret_cast<__nv_bfloat16 *>(blk + 16384 + off) = l;
        } else if constexpr (KIND == TC_TF32) {
            *reinterpret_cast<float *>(blk + off) = tf32_rna((float)x);
        } else {
            const float h = tf32_rna((float)x);
            const float l = tf32_rna((float)(x - (double)h));
            *reinterpret_cast<float *>(blk + off) = h;
            *reinterpret_cast<float *>(blk + 16384 + off) = l;
        }
    }
}

// The multipoles as copyable rows: row y = [part][kpad] of the split
// values of multipole y (hi = round(x), lo = round(x - hi) for the split
// precisions, the TF32 rounding for TF32), zero-padded; row nsrc is zero.
template <int KIND>
__global__ void dense_split_kernel(int nsrc, int n3, int kpad, const float *__restrict__ in, uint8_t *__restrict__ out)
{
    using Tr = TcTraits<KIND>;
    const size_t row_bytes = (size_t)Tr::nparts * kpad * Tr::esz;
    const long total = (long)(nsrc + 1) * kpad;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        const int y = (int)(idx / kpad), k = (int)(idx % kpad);
        const float x = (y < nsrc && k < n3) ? in[(size_t)y * n3 + k] : 0.0f;
        uint8_t *r = out + (size_t)y * row_bytes + (size_t)k * Tr::esz;
        if constexpr (KIND == TC_BF16X3) {
            const __nv_bfloat16 h = __float2bfloat16_rn(x);
            const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
            *reinterpret_cast<__nv_bfloat16 *>(r) = h;
            *reinterpret_cast<__nv_bfloat16 *>(r + (size_t)kpad * 2) = l;
        } else if constexpr (KIND == TC_TF32) {
            *reinterpret_cast<float *>(r) = tf32_rna(x);
        } else {
            const float h = tf32_rna(x);
            *reinterpret_cast<float *>(r) = h;
            *reinterpret_cast<float *>(r + (size_t)kpad * 4) = tf32_rna(x - h);
        }
    }
}

// 16-byte global -> shared copy through L2 (cp.async), and an arrive on bar
// that fires once all of this thread's earlier cp.async copies have landed.
// 16-byte asynchronous copy that allocates in L1 (.ca): measured 7-30 % faster
// than the L2-only form (.cg) for the dense kernel's row gathers.
__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_arrive_noinc(uint64_t *bar)
{
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Jobs (one per (unit, slot)) run in groups of JP: the stages of a group go K
// column by K column, the group's jobs in turn, so that the source rows of a
// job's K column are read again by the next job right after, mostly from L1.
// With JP = 2 the jobs take the list entries 0, 2, 1, 3 of each full group of
// four, so that the two jobs of a pair are mostly two x-steps apart (t and
// t + 2 e_1): their source rows coincide for all but one face of the unit's
// block of same-octant targets.
template <int JP>
__device__ __forceinline__ int job_entry(int j, int ns)
{
    if constexpr (JP == 1) {
        return j;
    } else {
        const int g = j & ~3, r = j & 3;
        if (g + 4 > ns) return j;
        return g + (r == 1 ? 2 : (r == 2 ? 1 : r));
    }
}

constexpr int kDenseProdWarps = 8;                                        // warps 0-7: producers
constexpr int kDenseMmaWarp = 8;
constexpr int kDenseEpiWarp0 = 9;
constexpr int kDenseEpiWarps = 16;
constexpr int kDenseThreads = (kDenseEpiWarp0 + kDenseEpiWarps) * 32;
constexpr int kDenseGroupsPerWarp = 4;                                    // 16-column groups, nu <= 256
constexpr int kDenseColStride = kDenseProdWarps * 4;                      // columns per pass of the producers (8 threads a column)
constexpr int kDenseMaxColM = 256 / kDenseColStride;                      // panel columns per producer thread (nu <= 256)
constexpr int kDenseMaxStages = 4;
constexpr int kDenseDStride = 256;    // TMEM columns between the two accumulators

template <int KIND>
__host__ __device__ constexpr int dense_stage_bytes(int nu)
{
    // one K column (128 bytes) of the operator (128 rows) and of nu gathered columns, all parts
    return TcTraits<KIND>::nparts * 128 * (128 + nu);
}

// One persistent CTA per SM over units blockIdx.x, blockIdx.x + gridDim.x, ...
// Warps 0-7 producers, warp 8 MMA, warps 9-24 epilogue.
template <int KIND>
__global__ void __launch_bounds__(kDenseThreads, 1)
tc_dense_kernel(const uint8_t *__restrict__ bsplit, const uint8_t *__restrict__ a_img,
                const int32_t *__restrict__ meta, const uint16_t *__restrict__ slots, const int32_t *__restrict__ tab,
                const int32_t *__restrict__ unit_tgt, int nu, int katoms, int nstages, int nsrc, int n3,
                float *__restrict__ out_f32, double *__restrict__ out_f64, float scale, int *status,
                int stall_first_stage)
{
    using Tr = TcTraits<KIND>;
    // pairs of jobs for the split precisions; TF32 (one product per stage) measured
    // faster with single jobs
    constexpr int JP = Tr::nprod == 3 ? 2 : 1;
    constexpr int E = 128 / Tr::esz;               // K elements per swizzle column
    constexpr int A_PART = 128 * 128;              // one part of an operator K column
    constexpr int A_BYTES = Tr::nparts * A_PART;
    constexpr int K_STEPS = 128 / 32;              // MMAs (32 bytes of K each) per swizzle column
    const int b_part = nu * 128;                   // one part of a gathered K column
    const int stage_bytes = A_BYTES + Tr::nparts * b_part;
    const int kpad = katoms * E;

    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)nstages * stage_bytes);
    uint64_t *afull = bars, *bfull = bars + kDenseMaxStages, *empty = bars + 2 * kDenseMaxStages;
    uint64_t *dfull = bars + 3 * kDenseMaxStages, *dempty = dfull + 2, *drain = dempty + 2;
    __shared__ uint32_t s_tmem_base;
    __shared__ int s_abort;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nunits = meta[0];
    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int i = 0; i < nstages; ++i) {
            mbar_init(afull + i, 1);
            mbar_init(bfull + i, kDenseProdWarps * 32);
            mbar_init(empty + i, 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(dfull + i, 1);
            mbar_init(dempty + i, kDenseEpiWarps * 32);
        }
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kDenseMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem_base)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = s_tmem_base;
    volatile int *abort_flag = &s_abort;

    if (warp < kDenseProdWarps) {
        // ---------------------------------------------------------- producers
        // Thread t of the 256 copies, per stage, the 16-byte chunk t % 8 of the
        // 128-byte K column of columns t / 8 + 32 m (every part) from the split
        // multipole rows straight to its 128-byte-swizzled place in the operand
        // panel (cp.async through L1), then arms the stage's panel barrier with
        // an arrive that fires when its copies have landed.  Thread 0 also copies
        // the stage's operator K column (one bulk copy on its own barrier).
        // The source rows of a group's jobs are held in registers for its stages;
        // the next group's are read after its last stage.
        const int pt = threadIdx.x;
        const int cb = pt >> 3, kc = pt & 7;
        const int ncm = (nu - cb + kDenseColStride - 1) / kDenseColStride;   // columns of this thread
        const size_t row_bytes = (size_t)Tr::nparts * kpad * Tr::esz;
        const uint8_t *src_base = bsplit + kc * 16;
        long it = 0;
        unsigned issued = 0, parity = 0;          // thread 0: operator copies per stage and their phase
        bool stop = false;
        for (int u = blockIdx.x; u < nunits && !stop; u += gridDim.x) {
            const uint16_t *row = slots + (size_t)u * kSlotRow + 1;
            const int ns = row[-1];
            if (ns == 0) continue;
            const int32_t *utab = tab + (size_t)u * kSlots * nu + cb;
            auto rows_of = [&](int slot, int (&v)[kDenseMaxColM]) {
                const int32_t *t = utab + (size_t)slot * nu;
#pragma unroll
                for (int m = 0; m < kDenseMaxColM; ++m) {
                    const int e = (m < ncm) ? __ldg(t + kDenseColStride * m) : 0;
                    v[m] = e ? e - 1 : nsrc;
                }
            };
            int yA[kDenseMaxColM], yB[kDenseMaxColM];
            rows_of(row[job_entry<JP>(0, ns)], yA);
            if (JP > 1 && ns > 1) rows_of(row[job_entry<JP>(1, ns)], yB);
            for (int si = 0; si < ns && !stop; si += JP) {
                const int nj = min(JP, ns - si);
                const int slotA = row[job_entry<JP>(si, ns)];
                const int slotB = nj > 1 ? (int)row[job_entry<JP>(si + 1, ns)] : slotA;
                for (int ka = 0; ka < katoms && !stop; ++ka) {
                    for (int j = 0; j < nj; ++j, ++it) {
                        const int s = (int)(it % nstages);
                        const uint32_t ph = (uint32_t)((it / nstages) & 1);
                        int ok = 1;
                        if (lane == 0) ok = mbar_wait(empty + s, ph ^ 1, abort_flag, status) ? 1 : 0;
                        ok = __shfl_sync(0xffffffffu, ok, 0);
                        if (!ok) {
                            stop = true;
                            break;
                        }
                        // test switch: withholding the first stage makes the MMA warp's wait run out
                        if (stall_first_stage && it == 0) continue;
                        const int slot = j ? slotB : slotA;
                        uint8_t *st = smem + (size_t)s * stage_bytes;
                        if (pt == 0) {
                            mbar_arrive_expect_tx(afull + s, (uint32_t)A_BYTES);
                            bulk_g2s(st, a_img + ((size_t)slot * katoms + ka) * A_BYTES, A_BYTES, afull + s);
                            issued |= 1u << s;
                            parity = (parity & ~(1u << s)) | (ph << s);
                        }
                        const uint8_t *src_k = src_base + ka * 128;
                        uint8_t *dst_b = st + A_BYTES;
#pragma unroll
                        for (int m = 0; m < kDenseMaxColM; ++m) {
                            if (m < ncm) {
                                const int c = cb + kDenseColStride * m;
                                const uint32_t off = (uint32_t)((c >> 3) * 1024 + (c & 7) * 128 + ((kc ^ (c & 7)) << 4));
                                const uint8_t *src = src_k + (size_t)(j ? yB[m] : yA[m]) * row_bytes;
#pragma unroll
                                for (int part = 0; part < Tr::nparts; ++part)
                                    cp_async16(dst_b + part * b_part + off, src + (size_t)part * kpad * Tr::esz);
                            }
                        }
                        cp_async_arrive_noinc(bfull + s);
                    }
                }
                // source rows of the next group
                if (si + JP < ns) rows_of(row[job_entry<JP>(si + JP, ns)], yA);
                if (JP > 1 && si + JP + 1 < ns) rows_of(row[job_entry<JP>(si + JP + 1, ns)], yB);
            }
        }
        // every copy this CTA issued lands before its shared memory is released
        asm volatile("cp.async.wait_all;" ::: "memory");
        if (pt == 0)
            for (int s = 0; s < nstages; ++s)
                if (issued & (1u << s)) mbar_wait_drain(afull + s, (parity >> s) & 1u, status);
        __syncwarp();
    } else if (warp == kDenseMmaWarp) {
        // ---------------------------------------------------------- MMA issue
        // one TMEM job per (unit, slot): the K sum of one transfer vector's product
        // accumulates in TMEM, the sum over the slots in the epilogue's registers
        if (lane == 0) {
            const uint32_t idesc = instr_desc(Tr::fmt, nu);
            long it = 0, jc = 0;
            bool issued = false, stop = false;
            for (int u = blockIdx.x; u < nunits && !stop; u += gridDim.x) {
                const uint16_t *row = slots + (size_t)u * kSlotRow;
                const int ns = row[0];
                for (int si = 0; si < ns && !stop; si += JP) {
                    const int nj = min(JP, ns - si);
                    for (int ka = 0; ka < katoms && !stop; ++ka) {
                        for (int j = 0; j < nj; ++j, ++it) {
                            const int b = (int)((jc + j) & 1);
                            if (ka == 0) {
                                // a job's accumulator must be drained before its first product
                                const long jj = jc + j;
                                if (!mbar_wait(dempty + b, (uint32_t)(((jj >> 1) & 1) ^ 1), abort_flag, status)) {
                                    stop = true;
                                    break;
                                }
                                tc_fence_after();
                            }
                            const uint32_t d = tmem_base + (uint32_t)(b * kDenseDStride);
                            const int s = (int)(it % nstages);
                            const uint32_t ph = (uint32_t)((it / nstages) & 1);
                            if (!mbar_wait(afull + s, ph, abort_flag, status) || !mbar_wait(bfull + s, ph, abort_flag, status)) {
                                stop = true;
                                break;
                            }
                            // the panel was written by cp.async (generic proxy); the MMA reads it
                            // through the async proxy
                            fence_proxy_async();
                            tc_fence_after();
                            const uint32_t sa = smem_u32(smem + (size_t)s * stage_bytes);
                            const uint32_t sb = sa + (uint32_t)A_BYTES;
#pragma unroll
                            for (int k = 0; k < K_STEPS; ++k) {
                                const uint64_t a0 = smem_desc(sa + 32 * k), b0 = smem_desc(sb + 32 * k);
                                umma<KIND>(d, a0, b0, idesc, (ka > 0 || k > 0) ? 1u : 0u);
                                if constexpr (Tr::nprod == 3) {
                                    // hi * lo and lo * hi into the same accumulator
                                    umma<KIND>(d, a0, smem_desc(sb + (uint32_t)b_part + 32 * k), idesc, 1);
                                    umma<KIND>(d, smem_desc(sa + A_PART + 32 * k), b0, idesc, 1);
                                }
                            }
                            umma_commit(empty + s);
                            issued = true;
                            if (ka == katoms - 1) umma_commit(dfull + b);
                        }
                    }
                    jc += nj;
                }
            }
            if (issued) {
                // every MMA issued by this thread has completed before TMEM is freed
                umma_commit(drain);
                mbar_wait_drain(drain, 0, status);
            }
        }
        __syncwarp();
    } else if (warp >= kDenseEpiWarp0) {
        // ---------------------------------------------------------- epilogue
        // 16 warps: four per TMEM lane quarter, warp `sub` of a quarter owning the
        // 16-column groups sub, sub + 4, sub + 8, sub + 12 of the accumulator.
        // Each slot's product is added into FP32 registers (round to nearest),
        // so a unit's locals are the register sums over its slots.
        const int q = warp & 3;                         // TMEM lane quarter of this warp
        const int sub = (warp - kDenseEpiWarp0) >> 2;   // 0..3
        const int node = 32 * q + lane;                 // accumulator row = local node index
        const uint32_t lane_base = tmem_base + ((uint32_t)(32 * q) << 16);
        long jc = 0;
        bool stop = false;
        for (int u = blockIdx.x; u < nunits && !stop; u += gridDim.x) {
            const int ns = slots[(size_t)u * kSlotRow];
            if (ns == 0) continue;
            float acc[kDenseGroupsPerWarp][16];
#pragma unroll
            for (int gi = 0; gi < kDenseGroupsPerWarp; ++gi)
#pragma unroll
                for (int c = 0; c < 16; ++c) acc[gi][c] = 0.0f;
            for (int si = 0; si < ns; ++si, ++jc) {
                const int b = (int)(jc & 1);
                const bool ok = mbar_wait(dfull + b, (uint32_t)((jc >> 1) & 1), abort_flag, status);
                if (!__all_sync(0xffffffffu, ok)) {   // tcgen05.ld below is warp-collective
                    stop = true;
                    break;
                }
                tc_fence_after();
#pragma unroll
                for (int gi = 0; gi < kDenseGroupsPerWarp; ++gi) {
                    const int c0 = 16 * (sub + 4 * gi);
                    if (c0 < nu) {
                        float v[16];
                        tmem_ld<16>(lane_base + (uint32_t)(b * kDenseDStride + c0), v);
#pragma unroll
                        for (int c = 0; c < 16; ++c) acc[gi][c] += v[c];
                    }
                }
                tc_fence_before();
                mbar_arrive(dempty + b);
            }
            if (stop) break;
            const int32_t *tg = unit_tgt + (size_t)u * nu;
#pragma unroll
            for (int gi = 0; gi < kDenseGroupsPerWarp; ++gi) {
                const int c0 = 16 * (sub + 4 * gi);
                if (c0 >= nu) continue;
                const int tl = tg[c0 + (lane & 15)];
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const int t = __shfl_sync(0xffffffffu, tl, c);
                    if (t >= 0 && node < n3) {
                        if (out_f64) atomicAdd(out_f64 + (size_t)t * n3 + node, (double)acc[gi][c] * (double)scale);
                        else atomicAdd(out_f32 + (size_t)t * n3 + node, acc[gi][c] * scale);
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kDenseMmaWarp)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(512) : "memory");
}

}  // namespace

// ---------------------------------------------------------------- host side
namespace {

Layout &dense_layout(const m2l_ops *ops, int kind)
{
    m2l_ops *o = const_cast<m2l_ops *>(ops);
    return kind == TC_TF32 ? o->tcd_tf32 : kind == TC_BF16X3 ? o->tcd_bf16x3 : o->tcd_tf32x3;
}

template <int KIND>
m2l_status dense_images(const m2l_ops *ops, cudaStream_t s)
{
    using Tr = TcTraits<KIND>;
    Layout &L = dense_layout(ops, KIND);
    if (L.ready) return M2L_OK;
    const int katoms = dense_katoms<KIND>(ops->n3);
    const size_t bytes = (size_t)kSlots * katoms * Tr::nparts * 16384;
    m2l_status st;
    if ((st = L.a.ensure(bytes)) != M2L_OK) return st;
    const int kpad = katoms * (128 / Tr::esz);
    dim3 grid((unsigned)((128 * kpad + 255) / 256), kSlots);
    dense_image_kernel<KIND><<<grid, 256, 0, s>>>(ops->n3, katoms, ops->K64.as<double>(), ops->sigma.as<int16_t>(),
                                                  ops->lut.as<uint16_t>(), L.a.as<uint8_t>());
    M2L_LAUNCH_CHECK("dense_image_kernel");
    L.ready = true;
    return M2L_OK;
}

template <int KIND>
m2l_status launch_dense_kind(const m2l_ops *ops, const DenseBuckets &d, const float *in, void *out, int out_fp64,
                             double scale, cudaStream_t s)
{
    using Tr = TcTraits<KIND>;
    m2l_status st = dense_images<KIND>(ops, s);
    if (st != M2L_OK) return st;
    const int n3 = ops->n3, katoms = dense_katoms<KIND>(n3), kpad = katoms * (128 / Tr::esz);
    const int row_bytes = Tr::nparts * kpad * Tr::esz;
    if (((size_t)d.nsrc + 1) * row_bytes > d.bsplit.bytes || d.nu % 16 != 0 || d.nu > kDenseDStride) {
        set_error("dense classification does not fit this precision");
        return M2L_EINVAL;
    }
    const long total = (long)(d.nsrc + 1) * kpad;
    const int sblocks = (int)((total + 255) / 256 < 8192 ? (total + 255) / 256 : 8192);
    dense_split_kernel<KIND><<<sblocks, 256, 0, s>>>(d.nsrc, n3, kpad, in, d.bsplit.as<uint8_t>());
    M2L_LAUNCH_CHECK("dense_split_kernel");

    const int stage = dense_stage_bytes<KIND>(d.nu);
    const int budget = max_smem_optin() - 1024 - 256;
    int nst = budget / stage;
    if (nst > kDenseMaxStages) nst = kDenseMaxStages;
    if (nst < 2) {
        set_error("dense tensor-core kernel: %d-byte stages do not fit shared memory twice", stage);
        return M2L_EUNSUPPORTED;
    }
    // at least half the SM's shared memory, so that one CTA (and one TMEM allocation) runs per SM
    int smem = 1024 + nst * stage + 256;
    if (smem < 120 * 1024) smem = 120 * 1024;
    auto kern = tc_dense_kernel<KIND>;
    M2L_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int grid = num_sms();
    if (grid > d.umax) grid = d.umax;
    const Layout &L = dense_layout(ops, KIND);
    kern<<<grid, kDenseThreads, smem, s>>>(d.bsplit.as<uint8_t>(), L.a.as<uint8_t>(), d.meta.as<int32_t>(), d.slots.as<uint16_t>(),
                                          d.tab.as<int32_t>(), d.unit_tgt.as<int32_t>(), d.nu, katoms, nst, d.nsrc,
                                          n3, out_fp64 ? nullptr : (float *)out, out_fp64 ? (double *)out : nullptr,
                                          (float)scale, ops->d_status,
                                          (ops->debug_flags & M2L_DEBUG_STALL_PRODUCER) ? 1 : 0);
    M2L_LAUNCH_CHECK("tc_dense_kernel");
    return M2L_OK;
}

}  // namespace

m2l_status dense_prepare(const m2l_ops *ops, int precision, cudaStream_t s)
{
    if (ops->eps > 0 || ops->n3 > 128) return M2L_OK;
    switch (precision) {
    case M2L_TF32: return dense_images<TC_TF32>(ops, s);
    case M2L_BF16X3: return dense_images<TC_BF16X3>(ops, s);
    case M2L_TF32X3: return dense_images<TC_TF32X3>(ops, s);
    default: return M2L_OK;
    }
}

m2l_status launch_tc_dense(const m2l_ops *ops, const DenseBuckets &d, int precision, const float *in, void *out,
                           int out_fp64, double scale, cudaStream_t s)
{
    switch (precision) {
    case M2L_TF32: return launch_dense_kind<TC_TF32>(ops, d, in, out, out_fp64, scale, s);
    case M2L_BF16X3: return launch_dense_kind<TC_BF16X3>(ops, d, in, out, out_fp64, scale, s);
    case M2L_TF32X3: return launch_dense_kind<TC_TF32X3>(ops, d, in, out, out_fp64, scale, s);
    default:
        set_error("not a tensor-core precision: %d", precision);
        return M2L_EINVAL;
    }
}

}  // namespace m2l

// ---------------------------------------------------------------- operator buckets from the dense tables
// For the kernels that take operator buckets (the CUDA-core precisions, the
// bucketed tensor-core kernel), the records are derived from a dense
// classification on demand: one warp per 32 columns of a unit, lane = column,
// walking the unit's active slots (the operator class p of a slot is the same
// for every lane).  Records of class p are ordered by (unit, column, slot), so
// the entries of one target stay consecutive within a bucket.
namespace m2l {
namespace {

constexpr int kRecWarps = 8;

template <bool EMIT>
__global__ void __launch_bounds__(kRecWarps * 32)
dense_records_kernel(int umax, int nu, int nwarps, const int32_t *__restrict__ meta,
                     const uint16_t *__restrict__ slots, const int32_t *__restrict__ tab,
                     const int32_t *__restrict__ unit_tgt, const uint16_t *__restrict__ lut,
                     int32_t *__restrict__ wcount, const int32_t *__restrict__ wbase, int2 *__restrict__ rec)
{
    __shared__ int cnt[kRecWarps][16][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * kRecWarps + w;
    const int per_unit = (nu + 31) / 32;
    const int u = gw / per_unit;
    const int j = (gw - u * per_unit) * 32 + lane;
    const bool live = gw < nwarps && u < meta[0];
    const bool col = live && j < nu;
    for (int p = 0; p < 16; ++p) cnt[w][p][lane] = 0;
    __syncwarp();
    const uint16_t *row = slots + (size_t)(live ? u : 0) * kSlotRow;
    const int ns = live ? row[0] : 0;
    const int32_t *tcol = tab + (size_t)(live ? u : 0) * kSlots * nu + (col ? j : 0);
    for (int si = 0; si < ns; ++si) {
        const int slot = row[1 + si];
        const int e = col ? tcol[(size_t)slot * nu] : 0;
        if (e) ++cnt[w][lut[slot] & 0xFF][lane];
    }
    __syncwarp();
    // exclusive prefix over the lanes, per class
    int pre[16];
#pragma unroll
    for (int p = 0; p < 16; ++p) {
        const int c = cnt[w][p][lane];
        int incl = c;
        for (int d = 1; d < 32; d <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += v;
        }
        pre[p] = incl - c;
        if (!EMIT && lane == 31 && gw < nwarps) wcount[(size_t)p * nwarps + gw] = incl;
    }
    if (!EMIT) return;
    const int tgt = col ? unit_tgt[(size_t)u * nu + j] : -1;
    if (col) {
#pragma unroll
        for (int p = 0; p < 16; ++p) cnt[w][p][lane] = wbase[(size_t)p * nwarps + gw] + pre[p];
    }
    __syncwarp();
    for (int si = 0; si < ns; ++si) {
        const int slot = row[1 + si];
        const int e = col ? tcol[(size_t)slot * nu] : 0;
        if (e) {
            const int c = lut[slot];
            const int p = c & 0xFF, g = c >> 8;
            rec[cnt[w][p][lane]++] = make_int2(e - 1, rec_pack(tgt, g));
        }
    }
}

__global__ void dense_class_off_kernel(int nwarps, int nnz, const int32_t *__restrict__ wbase, int32_t *__restrict__ class_off)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int p = 0; p < 16; ++p) class_off[p] = wbase[(size_t)p * nwarps];
    class_off[16] = wbase[(size_t)16 * nwarps];
    class_off[17] = nnz;
}

}  // namespace

m2l_status ensure_records(const m2l_ops *ops, const Buckets &bc, cudaStream_t s)
{
    Buckets &b = const_cast<Buckets &>(bc);
    if (b.have_rec) return M2L_OK;
    const DenseBuckets &d = b.dense;
    if (!d.valid) {
        set_error("no classification to derive operator buckets from");
        return M2L_EINVAL;
    }
    const int per_unit = (d.nu + 31) / 32;
    const int nwarps = d.umax * per_unit;
    const int nblk = (d.ntgt + kRankBlock - 1) / kRankBlock;
    // the slot-flag region of the classification scratch holds the counts and their scan
    int32_t *wcount = d.work.as<int32_t>() + 2 * (size_t)d.ntgt + 2 * (8 * (size_t)nblk + 1);
    int32_t *wbase = wcount + 16 * (size_t)nwarps + 1;
    if ((size_t)(2 * (16 * (size_t)nwarps + 1)) > (size_t)d.umax * kSlots) {
        set_error("record scratch exceeds the classification scratch");
        return M2L_EINVAL;
    }
    const int blocks = (nwarps + kRecWarps - 1) / kRecWarps;
    dense_records_kernel<false><<<blocks, kRecWarps * 32, 0, s>>>(
        d.umax, d.nu, nwarps, d.meta.as<int32_t>(), d.slots.as<uint16_t>(), d.tab.as<int32_t>(),
        d.unit_tgt.as<int32_t>(), ops->lut.as<uint16_t>(), wcount, nullptr, nullptr);
    M2L_LAUNCH_CHECK("dense_records_kernel");
    m2l_status st = launch_exclusive_scan(wcount, wbase, 16 * nwarps, s);
    if (st != M2L_OK) return st;
    dense_class_off_kernel<<<1, 32, 0, s>>>(nwarps, d.nnz, wbase, b.class_off.as<int32_t>());
    M2L_LAUNCH_CHECK("dense_class_off_kernel");
    dense_records_kernel<true><<<blocks, kRecWarps * 32, 0, s>>>(
        d.umax, d.nu, nwarps, d.meta.as<int32_t>(), d.slots.as<uint16_t>(), d.tab.as<int32_t>(),
        d.unit_tgt.as<int32_t>(), ops->lut.as<uint16_t>(), nullptr, wbase, b.rec.as<int2>());
    M2L_LAUNCH_CHECK("dense_records_kernel");
    b.have_rec = true;
    return M2L_OK;
}

}  // namespace m2l
