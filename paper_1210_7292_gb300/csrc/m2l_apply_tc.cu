// Steps a4-a6 on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// One persistent CTA per SM walks a contiguous range of tiles; a tile is NT
// bucketed interactions of one unique operator K_p (Alg. 2, blocked along many
// target cells as in Sec. 4.2.3).  Warp roles:
//   warps 0-3  producers: per tile, gather the NT source multipoles and
//              permute them (W_p[sigma_g(b)][c] = w[b], Eq. (30)) straight into
//              a 128-byte-swizzled K-major shared-memory panel (the UMMA B
//              operand), rounded to TF32 or split into BF16/TF32 hi + lo;
//              when the operator changes, one thread copies its pre-swizzled
//              image (the UMMA A operand) with cp.async.bulk.
//   warp 4     allocates TMEM and issues tcgen05.mma (one thread):
//              F_p = K_p W_p (Eq. (31)) into a double-buffered TMEM accumulator,
//              three products hi*hi + hi*lo + lo*hi for the split precisions.
//   warps 5-8  epilogue: tcgen05.ld of the accumulator, un-permutation
//              f[a] += F_p[sigma_g(a)] (Eq. (32)) through a shared-memory
//              transpose, sum over the consecutive columns of one target,
//              one atomic add per (target, node) and run (Alg. 2, third loop).
// Shared-memory stages and TMEM buffers are handed over with mbarriers; every
// wait is bounded (about two seconds), after which the CTA records
// M2L_ETIMEOUT in the status word, drains its asynchronous work and returns.
#include <cuda_bf16.h>

#include "m2l_internal.cuh"

namespace m2l {
namespace {

constexpr int kProducerWarps = 4;
constexpr int kMmaWarp = 4;
constexpr int kEpiWarp0 = 5;
constexpr int kThreadsTC = 9 * 32;
constexpr long long kWaitCycles = 4000000000LL;   // ~2 s at 2 GHz

enum TcKind : int { TC_TF32 = 0, TC_BF16X3 = 1, TC_TF32X3 = 2 };

template <int KIND> struct TcTraits;
template <> struct TcTraits<TC_TF32> {
    static constexpr int esz = 4, nparts = 1, nprod = 1, NT = 128;
    static constexpr uint32_t fmt = 2;  // TF32 in the kind::tf32 instruction descriptor
};
template <> struct TcTraits<TC_BF16X3> {
    static constexpr int esz = 2, nparts = 2, nprod = 3, NT = 128;
    static constexpr uint32_t fmt = 1;  // BF16 in the kind::f16 instruction descriptor
};
template <> struct TcTraits<TC_TF32X3> {
    static constexpr int esz = 4, nparts = 2, nprod = 3, NT = 32;
    static constexpr uint32_t fmt = 2;
};

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: false when the CTA is aborting or the wait timed out (which
// starts the abort and records the timeout).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag, int *status)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (clock64() - t0 > kWaitCycles) {
            *abort_flag = 1;
            atomicOr(status, ST_TIMEOUT);
            return false;
        }
    }
}

// Bounded wait that ignores the abort flag: used to let this CTA's own
// asynchronous copies and MMAs land before it frees their resources.
__device__ __forceinline__ bool mbar_wait_drain(uint64_t *bar, uint32_t parity, int *status)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > kWaitCycles) {
            atomicOr(status, ST_TIMEOUT);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void named_bar_sync(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Named barrier that also ORs a predicate over the participating threads.
__device__ __forceinline__ int named_bar_or(int id, int nthreads, int pred)
{
    int r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.s32 p, %3, 0;\n\t"
        "bar.red.or.pred q, %1, %2, p;\n\tselp.s32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"(id), "r"(nthreads), "r"(pred)
        : "memory");
    return r;
}

// UMMA shared-memory descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);        // start address
    d |= (uint64_t)1 << 16;                         // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;               // stride byte offset
    d |= (uint64_t)1 << 46;                         // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;                         // 128-byte swizzle
    return d;
}

// Instruction descriptor: F32 accumulator, K-major A and B, M = 128, N = n.
__device__ __forceinline__ uint32_t instr_desc(uint32_t fmt, int n)
{
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

template <int KIND>
__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    if constexpr (KIND == TC_BF16X3) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
            : "memory");
    }
}

__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float tf32_rna(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Byte offset of 16-byte chunk `chunk` (of the 8 in a 128-byte row) of row
// `row` inside one swizzle column of `rows` rows: 8-row groups of 1024 B, the
// chunk index XOR-ed with the row inside its group.
__device__ __forceinline__ uint32_t swz_off(int row, int chunk)
{
    return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((chunk ^ (row & 7)) << 4));
}

struct TileSched {
    int first, last;   // [first, last) tile indices of this CTA
};

// Tile t -> (operator p, first bucketed column, column count).
__device__ __forceinline__ void tile_info(int t, const int *tile_start, const int *class_off, int NT, int &p,
                                          int &col0, int &nc)
{
    p = 0;
    while (p < 15 && t >= tile_start[p + 1]) ++p;
    col0 = class_off[p] + (t - tile_start[p]) * NT;
    nc = min(NT, class_off[p + 1] - col0);
}

template <int KIND>
__global__ void __launch_bounds__(kThreadsTC, 1)
tc_apply_kernel(const int2 *__restrict__ rec, const int *__restrict__ class_off,
                const uint8_t *__restrict__ a_img, int a_bytes, const int16_t *__restrict__ sigma,
                const int16_t *__restrict__ sigma_inv, const float *__restrict__ mp, float *__restrict__ out_f32,
                double *__restrict__ out_f64, int n3, int katoms, float scale, int *status)
{
    using Tr = TcTraits<KIND>;
    constexpr int NT = Tr::NT;
    constexpr int ELEMS_PER_ATOM = 128 / Tr::esz;          // K elements per 128-byte row
    constexpr int K_PER_MMA = 32 / Tr::esz;                 // 8 (tf32) or 16 (bf16)
    constexpr int MMAS_PER_ATOM = ELEMS_PER_ATOM / K_PER_MMA;  // 4
    const int a_part_bytes = katoms * 128 * 128;            // one operand part of A (128 rows)
    const int b_part_bytes = katoms * NT * 128;             // one operand part of a B stage
    const int b_stage_bytes = b_part_bytes * Tr::nparts;

    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = smem;                                      // a_bytes
    uint8_t *sB = sA + a_bytes;                              // 2 stages
    float *sF = reinterpret_cast<float *>(sB + 2 * b_stage_bytes);   // [32][129] epilogue transpose
    uint64_t *bars = reinterpret_cast<uint64_t *>(sF + 32 * 129);
    uint64_t *full = bars, *empty = bars + 2, *tfull = bars + 4, *tempty = bars + 6, *afull = bars + 8,
             *drain = bars + 9;
    __shared__ uint32_t s_tmem_base;
    __shared__ int s_abort;
    __shared__ int s_tile_start[17];
    __shared__ TileSched s_sched;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int TMEM_COLS = 2 * NT;

    if (threadIdx.x == 0) {
        int acc = 0;
        for (int p = 0; p < 16; ++p) {
            s_tile_start[p] = acc;
            acc += (class_off[p + 1] - class_off[p] + NT - 1) / NT;
        }
        s_tile_start[16] = acc;
        const int per = (acc + gridDim.x - 1) / gridDim.x;
        s_sched.first = min(acc, (int)blockIdx.x * per);
        s_sched.last = min(acc, s_sched.first + per);
        s_abort = 0;
        for (int i = 0; i < 2; ++i) {
            mbar_init(full + i, kProducerWarps * 32);
            mbar_init(empty + i, 1);
            mbar_init(tfull + i, 1);
            mbar_init(tempty + i, 4 * 32);
        }
        mbar_init(afull, 1);
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = s_tmem_base;
    const int first = s_sched.first, last = s_sched.last;
    volatile int *abort_flag = &s_abort;

    if (warp < kProducerWarps) {
        // ------------------------------------------------------------ producers
        const int ptid = threadIdx.x;   // 0..127
        int prev_p = -1;
        uint32_t a_loads = 0;
        for (int t = first; t < last; ++t) {
            const int i = t - first, s = i & 1, k = i >> 1;
            int p, col0, nc;
            tile_info(t, s_tile_start, class_off, NT, p, col0, nc);
            if (p != prev_p) {
                if (ptid == 0) {
                    bool ok = true;
                    if (i > 0) ok = mbar_wait(empty + ((i - 1) & 1), ((i - 1) >> 1) & 1, abort_flag, status);
                    if (ok) {
                        mbar_arrive_expect_tx(afull, (uint32_t)a_bytes);
                        bulk_g2s(sA, a_img + (size_t)p * a_bytes, (uint32_t)a_bytes, afull);
                        ++a_loads;
                    }
                }
                prev_p = p;
            }
            if (!mbar_wait(empty + s, (k & 1) ^ 1, abort_flag, status)) break;
            uint8_t *stage = sB + s * b_stage_bytes;
            if constexpr (KIND == TC_BF16X3) {
                // 8 bf16 per 16-byte chunk; half a warp per column
                const int nchunks = katoms * 8;
                for (int c = (ptid >> 4); c < NT; c += 8) {
                    const int2 r = (c < nc) ? rec[col0 + c] : make_int2(0, 0);
                    const int g = rec_g(r.y);
                    const float *w = mp + (size_t)r.x * n3;
                    const int16_t *si = sigma_inv + g * n3;
                    for (int j = (ptid & 15); j < nchunks; j += 16) {
                        uint32_t hi[4], lo[4];
#pragma unroll
                        for (int e = 0; e < 8; e += 2) {
                            float v[2];
#pragma unroll
                            for (int q = 0; q < 2; ++q) {
                                const int kk = 8 * j + e + q;
                                v[q] = (c < nc && kk < n3) ? __ldg(w + si[kk]) : 0.0f;
                            }
                            const __nv_bfloat16 h0 = __float2bfloat16_rn(v[0]);
                            const __nv_bfloat16 h1 = __float2bfloat16_rn(v[1]);
                            const __nv_bfloat16 l0 = __float2bfloat16_rn(v[0] - __bfloat162float(h0));
                            const __nv_bfloat16 l1 = __float2bfloat16_rn(v[1] - __bfloat162float(h1));
                            hi[e / 2] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
                            lo[e / 2] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
                        }
                        const uint32_t off = (uint32_t)(j >> 3) * (uint32_t)(NT * 128) + swz_off(c, j & 7);
                        *reinterpret_cast<uint4 *>(stage + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                        *reinterpret_cast<uint4 *>(stage + b_part_bytes + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
                    }
                }
            } else {
                // 4 fp32 per 16-byte chunk; one warp per column
                const int nchunks = katoms * 8;
                for (int c = warp; c < NT; c += kProducerWarps) {
                    const int2 r = (c < nc) ? rec[col0 + c] : make_int2(0, 0);
                    const int g = rec_g(r.y);
                    const float *w = mp + (size_t)r.x * n3;
                    const int16_t *si = sigma_inv + g * n3;
                    for (int j = lane; j < nchunks; j += 32) {
                        float v[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int kk = 4 * j + e;
                            v[e] = (c < nc && kk < n3) ? __ldg(w + si[kk]) : 0.0f;
                        }
                        const uint32_t off = (uint32_t)(j >> 3) * (uint32_t)(NT * 128) + swz_off(c, j & 7);
                        if constexpr (KIND == TC_TF32) {
                            *reinterpret_cast<float4 *>(stage + off) =
                                make_float4(tf32_rna(v[0]), tf32_rna(v[1]), tf32_rna(v[2]), tf32_rna(v[3]));
                        } else {
                            float h[4], l[4];
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                h[e] = tf32_rna(v[e]);
                                l[e] = tf32_rna(v[e] - h[e]);
                            }
                            *reinterpret_cast<float4 *>(stage + off) = make_float4(h[0], h[1], h[2], h[3]);
                            *reinterpret_cast<float4 *>(stage + b_part_bytes + off) = make_float4(l[0], l[1], l[2], l[3]);
                        }
                    }
                }
            }
            fence_proxy_async();
            mbar_arrive(full + s);
        }
        // an operator image still in flight must land before the CTA exits
        if (ptid == 0 && a_loads > 0) mbar_wait_drain(afull, (a_loads - 1) & 1, status);
    } else if (warp == kMmaWarp) {
        // ------------------------------------------------------------ MMA issue
        if (lane == 0) {
            const uint32_t idesc = instr_desc(Tr::fmt, NT);
            const uint32_t a_base = smem_u32(sA), b_base = smem_u32(sB);
            int prev_p = -1;
            uint32_t a_loads = 0;
            bool issued = false;
            for (int t = first; t < last; ++t) {
                const int i = t - first, s = i & 1, k = i >> 1;
                int p, col0, nc;
                tile_info(t, s_tile_start, class_off, NT, p, col0, nc);
                if (!mbar_wait(full + s, k & 1, abort_flag, status)) break;
                if (p != prev_p) {
                    if (!mbar_wait(afull, a_loads & 1, abort_flag, status)) break;
                    ++a_loads;
                    prev_p = p;
                }
                if (!mbar_wait(tempty + s, (k & 1) ^ 1, abort_flag, status)) break;
                tc_fence_after();
                const uint32_t d = tmem_base + (uint32_t)(s * NT);
                const uint32_t bst = b_base + (uint32_t)(s * b_stage_bytes);
                uint32_t accum = 0;
                for (int ka = 0; ka < katoms; ++ka) {
                    for (int m = 0; m < MMAS_PER_ATOM; ++m) {
                        const uint32_t koff = (uint32_t)(m * 32);
                        const uint32_t a0 = a_base + (uint32_t)(ka * 128 * 128) + koff;
                        const uint32_t b0 = bst + (uint32_t)(ka * NT * 128) + koff;
                        umma<KIND>(d, smem_desc(a0), smem_desc(b0), idesc, accum);
                        accum = 1;
                        if constexpr (Tr::nprod == 3) {
                            // hi*lo and lo*hi into the same accumulator
                            umma<KIND>(d, smem_desc(a0), smem_desc(b0 + (uint32_t)b_part_bytes), idesc, 1);
                            umma<KIND>(d, smem_desc(a0 + (uint32_t)a_part_bytes), smem_desc(b0), idesc, 1);
                        }
                    }
                }
                umma_commit(empty + s);
                umma_commit(tfull + s);
                issued = true;
            }
            if (issued) {
                // every MMA issued by this thread has completed before TMEM is freed
                umma_commit(drain);
                mbar_wait_drain(drain, 0, status);
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ epilogue
        const int q = warp & 3;               // TMEM lane quarter this warp may read
        const int row = 32 * q + lane;        // accumulator row (permuted node a')
        const int a = threadIdx.x - kEpiWarp0 * 32;   // output node handled in the reduction
        const int16_t *sg_base = sigma;
        int cur = -1;
        float acc = 0.0f;
        for (int t = first; t < last; ++t) {
            const int i = t - first, s = i & 1, k = i >> 1;
            int p, col0, nc;
            tile_info(t, s_tile_start, class_off, NT, p, col0, nc);
            // all four epilogue warps leave together if any of them gave up
            const bool ok = mbar_wait(tfull + s, k & 1, abort_flag, status);
            if (named_bar_or(1, 128, ok ? 0 : 1)) break;
            tc_fence_after();
            for (int ch = 0; ch < NT / 32; ++ch) {
                float v[32];
                tmem_ld32(tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(s * NT + 32 * ch), v);
                if (ch == NT / 32 - 1) {
                    tc_fence_before();
                    mbar_arrive(tempty + s);
                }
#pragma unroll
                for (int j = 0; j < 32; ++j) sF[j * 129 + row] = v[j];
                named_bar_sync(1, 128);
                if (a < n3) {
                    const int cend = min(32, nc - 32 * ch);
                    for (int j = 0; j < cend; ++j) {
                        const int2 r = __ldg(rec + col0 + 32 * ch + j);
                        const int tgt = rec_tgt(r.y);
                        const int g = rec_g(r.y);
                        if (tgt != cur) {
                            if (cur >= 0) {
                                if (out_f64) atomicAdd(out_f64 + (size_t)cur * n3 + a, (double)acc * (double)scale);
                                else atomicAdd(out_f32 + (size_t)cur * n3 + a, acc * scale);
                            }
                            acc = 0.0f;
                            cur = tgt;
                        }
                        acc += sF[j * 129 + __ldg(sg_base + g * n3 + a)];
                    }
                }
                named_bar_sync(1, 128);
            }
        }
        if (a < n3 && cur >= 0) {
            if (out_f64) atomicAdd(out_f64 + (size_t)cur * n3 + a, (double)acc * (double)scale);
            else atomicAdd(out_f32 + (size_t)cur * n3 + a, acc * scale);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kMmaWarp)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                     : "memory");
}

// ---------------------------------------------------------------- layouts
__global__ void sigma_inverse_kernel(int n3, const int16_t *__restrict__ sigma, int16_t *__restrict__ inv)
{
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < 48 * n3; idx += gridDim.x * blockDim.x) {
        const int g = idx / n3, b = idx % n3;
        inv[g * n3 + sigma[idx]] = (int16_t)b;
    }
}

// Pre-swizzled A images: per operator p, nparts x katoms swizzle columns of
// 128 rows x 128 bytes; row a = output node (zero beyond n3), K = source node.
template <int KIND>
__global__ void a_image_kernel(int n3, int katoms, const double *__restrict__ K, uint8_t *__restrict__ img)
{
    using Tr = TcTraits<KIND>;
    constexpr int E = 128 / Tr::esz;
    const int part_bytes = katoms * 128 * 128;
    const int p = blockIdx.y;
    uint8_t *base = img + (size_t)p * part_bytes * Tr::nparts;
    const int kpad = katoms * E;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < 128 * kpad; idx += gridDim.x * blockDim.x) {
        const int row = idx / kpad, kk = idx % kpad;
        const double x = (row < n3 && kk < n3) ? K[((size_t)p * n3 + row) * n3 + kk] : 0.0;
        const int ka = kk / E, e = kk % E;
        const int chunk = e / (16 / Tr::esz), within = e % (16 / Tr::esz);
        const uint32_t off = (uint32_t)ka * 16384u +
                             (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + (((chunk ^ (row & 7))) << 4)) +
                             (uint32_t)(within * Tr::esz);
        if constexpr (KIND == TC_BF16X3) {
            const __nv_bfloat16 h = __double2bfloat16(x);
            const __nv_bfloat16 l = __double2bfloat16(x - (double)__bfloat162float(h));
            *reinterpret_cast<__nv_bfloat16 *>(base + off) = h;
            *reinterpret_cast<__nv_bfloat16 *>(base + part_bytes + off) = l;
        } else if constexpr (KIND == TC_TF32) {
            *reinterpret_cast<float *>(base + off) = tf32_rna((float)x);
        } else {
            const float h = tf32_rna((float)x);
            const float l = tf32_rna((float)(x - (double)h));
            *reinterpret_cast<float *>(base + off) = h;
            *reinterpret_cast<float *>(base + part_bytes + off) = l;
        }
    }
}

template <int KIND>
int tc_katoms(int n3)
{
    constexpr int E = 128 / TcTraits<KIND>::esz;
    return (n3 + E - 1) / E;
}

template <int KIND>
size_t tc_smem_bytes(int katoms)
{
    using Tr = TcTraits<KIND>;
    const size_t a = (size_t)katoms * 128 * 128 * Tr::nparts;
    const size_t b = 2 * (size_t)katoms * Tr::NT * 128 * Tr::nparts;
    return 1024 + a + b + 32 * 129 * sizeof(float) + 16 * sizeof(uint64_t);
}

template <int KIND>
m2l_status launch_kind(const m2l_ops *ops, const Buckets &b, Layout &L, const float *in, void *out, int out_fp64,
                       double scale, cudaStream_t s)
{
    using Tr = TcTraits<KIND>;
    const int n3 = ops->n3;
    if (n3 > 128) {
        set_error("tensor-core precisions support ell <= 5 (ell^3 <= 128); got ell = %d", ops->ell);
        return M2L_EUNSUPPORTED;
    }
    if (ops->eps > 0) {
        set_error("tensor-core precisions take full-rank operators");
        return M2L_EUNSUPPORTED;
    }
    const int katoms = tc_katoms<KIND>(n3);
    const int a_bytes = katoms * 128 * 128 * Tr::nparts;
    m2l_status st;
    if (!L.ready) {
        if ((st = L.a.ensure((size_t)16 * a_bytes)) != M2L_OK) return st;
        if ((st = L.b.ensure((size_t)48 * n3 * sizeof(int16_t))) != M2L_OK) return st;
        M2L_CUDA(cudaMemsetAsync(L.a.p, 0, (size_t)16 * a_bytes, s));
        dim3 grid((128 * katoms * (128 / Tr::esz) + 255) / 256, 16);
        a_image_kernel<KIND><<<grid, 256, 0, s>>>(n3, katoms, ops->K64.as<double>(), L.a.as<uint8_t>());
        M2L_LAUNCH_CHECK("a_image_kernel");
        sigma_inverse_kernel<<<(48 * n3 + 255) / 256, 256, 0, s>>>(n3, ops->sigma.as<int16_t>(), L.b.as<int16_t>());
        M2L_LAUNCH_CHECK("sigma_inverse_kernel");
        L.ready = true;
    }
    if (b.nnz == 0) return M2L_OK;
    const size_t smem = tc_smem_bytes<KIND>(katoms);
    if ((int)smem > max_smem_optin()) {
        set_error("tensor-core kernel needs %zu bytes of shared memory", smem);
        return M2L_EUNSUPPORTED;
    }
    auto kern = tc_apply_kernel<KIND>;
    M2L_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    long grid = num_sms();
    const long tiles_bound = (long)(b.nnz + Tr::NT - 1) / Tr::NT + 16;
    if (grid > tiles_bound) grid = tiles_bound;
    kern<<<(int)grid, kThreadsTC, smem, s>>>(b.rec.as<int2>(), b.class_off.as<int>(), L.a.as<uint8_t>(), a_bytes,
                                             ops->sigma.as<int16_t>(), L.b.as<int16_t>(), in,
                                             out_fp64 ? nullptr : (float *)out, out_fp64 ? (double *)out : nullptr,
                                             n3, katoms, (float)scale, ops->d_status);
    M2L_LAUNCH_CHECK("tc_apply_kernel");
    return M2L_OK;
}

}  // namespace

m2l_status launch_tc(const m2l_ops *ops, const Buckets &b, const void *in, void *out, int precision, int out_fp64,
                     double scale, cudaStream_t s)
{
    m2l_ops *o = const_cast<m2l_ops *>(ops);
    switch (precision) {
    case M2L_TF32:
        return launch_kind<TC_TF32>(ops, b, o->tc_tf32, (const float *)in, out, out_fp64, scale, s);
    case M2L_BF16X3:
        return launch_kind<TC_BF16X3>(ops, b, o->tc_bf16x3, (const float *)in, out, out_fp64, scale, s);
    case M2L_TF32X3:
        return launch_kind<TC_TF32X3>(ops, b, o->tc_tf32x3, (const float *)in, out, out_fp64, scale, s);
    default:
        set_error("not a tensor-core precision: %d", precision);
        return M2L_EINVAL;
    }
}

}  // namespace m2l
