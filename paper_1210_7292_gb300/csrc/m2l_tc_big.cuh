// The operator-bucketed tcgen05 kernel for vectors longer than 128 values
// (orders 6-8, the directional M2L's complex embedding, batches of trees),
// shared by the translation units that launch it (internal linkage), with the
// image builder of its streamed operator blocks and its tile bookkeeping.
#pragma once

#include "m2l_tcgen05.cuh"

namespace m2l {
namespace {

constexpr int kProducerWarps = 8;
constexpr int kMmaWarp = 8;

struct TileSched {
    int first, last;   // [first, last) tile indices of this CTA
};

// Tile t -> (operator p, first bucketed column, column count).  p is a cursor:
// it starts at 0 and each caller asks for non-decreasing t, so the search
// moves only at operator boundaries.
__device__ __forceinline__ void tile_info(int t, const int *tile_start, const int *class_off, int NT, int &p,
                                          int &col0, int &nc, int last_cls = kNumSym - 1)
{
    while (p < last_cls && t >= tile_start[p + 1]) ++p;
    col0 = class_off[p] + (t - tile_start[p]) * NT;
    nc = min(NT, class_off[p + 1] - col0);
}

// ---------------------------------------------------------------- orders 6..8
// For ell^3 > 128 the operator spans MT = ceil(ell^3 / 128) M tiles and does not
// fit in shared memory: it is streamed per tile as (M tile, swizzle column)
// blocks of 128 rows x 128 bytes through a ring of RS slots by a loader warp
// (cp.async.bulk), while the panel of NT = 32 columns is resident in NB stages;
// the MT accumulators of a tile live side by side in TMEM.  Roles: warps 0-7
// producers, warp 8 MMA, warp 9 operator loader, warps 10-13 epilogue.
constexpr int kBigNT = 32;
constexpr int kBigLoaderWarp = 9;
constexpr int kBigEpiWarp0 = 10;

template <int KIND, int MT, int KA, int NT_ = kBigNT, int EG_ = 1>
struct BigCfg {
    using Tr = TcTraits<KIND>;
    static constexpr int E = 128 / Tr::esz;                  // K elements per swizzle column
    static constexpr int KPAD = KA * E;
    static constexpr int A_BLOCK = 128 * 128 * Tr::nparts;   // one (M tile, K column) block, all parts
    static constexpr int A_PART = 128 * 128;
    static constexpr int B_PART = KA * NT_ * 128;
    static constexpr int B_STAGE = B_PART * Tr::nparts;
    static constexpr int FS = MT * 128 + 4;                   // epilogue transpose column stride (floats)
    static constexpr int FIXED = 1024 + EG_ * 16 * FS * 4 + 2 * NT_ * 8 + EG_ * 2 * NT_ * 4 + 32 * 8;
    static constexpr int BUDGET = 225 * 1024;
    static constexpr int NB = (FIXED + 2 * B_STAGE + 3 * A_BLOCK <= BUDGET) ? 2 : 1;
    static constexpr int RS = (FIXED + NB * B_STAGE + 4 * A_BLOCK <= BUDGET) ? 4
                              : ((FIXED + NB * B_STAGE + 3 * A_BLOCK <= BUDGET) ? 3 : 2);
    static constexpr int SMEM = FIXED + NB * B_STAGE + RS * A_BLOCK;
    static constexpr int TMEM_COLS = (2 * MT * NT_ <= 128) ? 128 : ((2 * MT * NT_ <= 256) ? 256 : 512);
};

// EG_ epilogue groups of four warps: with two, group g drains TMEM buffer g
// (every other tile), each with its own transpose buffer and named barrier.
constexpr int big_threads(int eg) { return (kBigEpiWarp0 + 4 * eg) * 32; }

// MODE 0: the M2L of Alg. 2 (gather + permute, product, un-permute + scatter-add).
// MODE 1: first low-rank pass, Z = V_p^T W_p (Eq. (20)): gather + permute as in
//         mode 0, the product's columns stored unpermuted to out_f32 at the
//         record's position (n3 values per record, no accumulation).
// MODE 2: second low-rank pass, F = (U_p Sigma_p) Z: the column of a record is
//         row col0 + c of mp (n_in values, gathered through sinv_prod, an
//         identity table), un-permute + scatter-add as in mode 0.
template <int KIND, int MT, int KA, int NT_ = kBigNT, int EG_ = 1, int MODE = 0>
__global__ void __launch_bounds__(big_threads(EG_), 1)
tc_big_kernel(const int2 *__restrict__ rec, const int *__restrict__ class_off, const uint8_t *__restrict__ a_img,
              const int16_t *__restrict__ sinv_pad, const float *__restrict__ mp, float *__restrict__ out_f32,
              double *__restrict__ out_f64, int n3, float scale, int *status, int stall_first_stage, int ncls,
              const int *__restrict__ tile_start_g, const int *__restrict__ img_of_class, int n_in,
              const int16_t *__restrict__ sinv_prod)
{
    // n3 is the vector length; with tile_start_g (device, ncls + 1 tile offsets)
    // the classes are ncls operators of a_img, else the 16 of the symmetry method.
    // img_of_class (device, optional) maps a class to its image in a_img, so that
    // classes with the same operator share one image.
    using Tr = TcTraits<KIND>;
    using C = BigCfg<KIND, MT, KA, NT_, EG_>;
    constexpr int NT = NT_;
    constexpr int EG = EG_;
    constexpr int EPC = 16 / Tr::esz;
    constexpr int CPC = KA * 8;                      // 16-byte chunks per column and part
    constexpr int NPT = kProducerWarps * 32;
    constexpr int ITEMS = (NT * CPC + NPT - 1) / NPT;
    constexpr int MMAS_PER_ATOM = 4;
    constexpr int NB = C::NB, RS = C::RS, FS = C::FS;

    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint8_t *sRing = smem;                                        // RS operator blocks
    uint8_t *sB = sRing + RS * C::A_BLOCK;                        // NB panel stages
    float *sF_all = reinterpret_cast<float *>(sB + NB * C::B_STAGE);   // [EG][16][FS]
    int2 *s_prec = reinterpret_cast<int2 *>(sF_all + EG * 16 * FS);    // [NB][NT]
    int *e_goff_all = reinterpret_cast<int *>(s_prec + 2 * NT);        // [EG][NT]
    int *e_tgt_all = e_goff_all + EG * NT;                             // [EG][NT]
    uint64_t *bars = reinterpret_cast<uint64_t *>(e_tgt_all + EG * NT);
    uint64_t *full = bars, *empty = bars + 2, *afull = bars + 4, *aempty = bars + 8, *tfull = bars + 12,
             *tempty = bars + 14, *drain = bars + 16;
    __shared__ uint32_t s_tmem_base;
    __shared__ int s_abort;
    __shared__ int s_tile_start[17];
    __shared__ TileSched s_sched;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        int acc = 0;
        if (tile_start_g) {
            acc = tile_start_g[ncls];
        } else {
            for (int p = 0; p < 16; ++p) {
                s_tile_start[p] = acc;
                acc += (class_off[p + 1] - class_off[p] + NT - 1) / NT;
            }
            s_tile_start[16] = acc;
        }
        const int per = (acc + gridDim.x - 1) / gridDim.x;
        s_sched.first = min(acc, (int)blockIdx.x * per);
        s_sched.last = min(acc, s_sched.first + per);
        s_abort = 0;
        for (int i = 0; i < NB; ++i) {
            mbar_init(full + i, NPT);
            mbar_init(empty + i, 1);
        }
        for (int i = 0; i < RS; ++i) {
            mbar_init(afull + i, 1);
            mbar_init(aempty + i, 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(tfull + i, 1);
            mbar_init(tempty + i, 4 * 32);
        }
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem_base)),
                     "r"(C::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = s_tmem_base;
    const int first = s_sched.first, last = s_sched.last;
    volatile int *abort_flag = &s_abort;
    const int *ts = tile_start_g ? tile_start_g : s_tile_start;
    const int lastc = (tile_start_g ? ncls : 16) - 1;

    if (warp < kProducerWarps) {
        // ------------------------------------------------------------ panel producers
        const int ptid = threadIdx.x;
        int p = 0;   // operator cursor (tile_info)
        for (int t = first; t < last; ++t) {
            const int i = t - first, s = i % NB, ks = i / NB;
            int col0, nc;
            tile_info(t, ts, class_off, NT, p, col0, nc, lastc);
            int2 *prec = s_prec + s * NT;
            if (ptid < NT) prec[ptid] = (ptid < nc) ? __ldg(rec + col0 + ptid) : make_int2(0, 0);
            named_bar_sync(2, NPT);
            float v[ITEMS][EPC];
#pragma unroll
            for (int u = 0; u < ITEMS; ++u) {
                const int it = ptid + u * NPT;
                const int c = it / CPC, j = it % CPC;
                const bool live = (it < NT * CPC) && (c < nc);
                const int2 r = live ? prec[c] : make_int2(0, 0);
                const float *w = mp + (size_t)(MODE == 2 ? col0 + c : r.x) * n_in;
                const int16_t *si = (sinv_prod ? sinv_prod : sinv_pad) + rec_g(r.y) * C::KPAD + EPC * j;
                int16_t idx[EPC];
                if (live) {
                    if constexpr (EPC == 4) {
                        const uint2 qv = __ldg(reinterpret_cast<const uint2 *>(si));
                        idx[0] = (int16_t)(qv.x & 0xFFFF); idx[1] = (int16_t)(qv.x >> 16);
                        idx[2] = (int16_t)(qv.y & 0xFFFF); idx[3] = (int16_t)(qv.y >> 16);
                    } else {
                        const uint4 qv = __ldg(reinterpret_cast<const uint4 *>(si));
                        const uint32_t qq[4] = {qv.x, qv.y, qv.z, qv.w};
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            idx[2 * e] = (int16_t)(qq[e] & 0xFFFF);
                            idx[2 * e + 1] = (int16_t)(qq[e] >> 16);
                        }
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < EPC; ++e) idx[e] = 0;
                }
#pragma unroll
                for (int e = 0; e < EPC; ++e) v[u][e] = live ? __ldg(w + idx[e]) : 0.0f;
            }
            const bool ok = mbar_wait(empty + s, (ks & 1) ^ 1, abort_flag, status);
            if (named_bar_or(2, NPT, ok ? 0 : 1)) break;
            uint8_t *stage = sB + s * C::B_STAGE;
#pragma unroll
            for (int u = 0; u < ITEMS; ++u) {
                const int it = ptid + u * NPT;
                if (it >= NT * CPC) break;
                const int c = it / CPC, j = it % CPC;
                const uint32_t off = (uint32_t)(j >> 3) * (uint32_t)(NT * 128) + swz_off(c, j & 7);
                if constexpr (KIND == TC_BF16X3) {
                    uint32_t hi[4], lo[4];
#pragma unroll
                    for (int e = 0; e < 8; e += 2) {
                        const __nv_bfloat16 h0 = __float2bfloat16_rn(v[u][e]);
                        const __nv_bfloat16 h1 = __float2bfloat16_rn(v[u][e + 1]);
                        const __nv_bfloat16 l0 = __float2bfloat16_rn(v[u][e] - __bfloat162float(h0));
                        const __nv_bfloat16 l1 = __float2bfloat16_rn(v[u][e + 1] - __bfloat162float(h1));
                        hi[e / 2] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
                        lo[e / 2] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
                    }
                    *reinterpret_cast<uint4 *>(stage + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                    *reinterpret_cast<uint4 *>(stage + C::B_PART + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
                } else if constexpr (KIND == TC_TF32) {
                    *reinterpret_cast<float4 *>(stage + off) =
                        make_float4(tf32_rna(v[u][0]), tf32_rna(v[u][1]), tf32_rna(v[u][2]), tf32_rna(v[u][3]));
                } else {
                    float h[4], l[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        h[e] = tf32_rna(v[u][e]);
                        l[e] = tf32_rna(v[u][e] - h[e]);
                    }
                    *reinterpret_cast<float4 *>(stage + off) = make_float4(h[0], h[1], h[2], h[3]);
                    *reinterpret_cast<float4 *>(stage + C::B_PART + off) = make_float4(l[0], l[1], l[2], l[3]);
                }
            }
            fence_proxy_async();
            if (!(stall_first_stage && i == 0)) mbar_arrive(full + s);
        }
    } else if (warp == kMmaWarp) {
        // ------------------------------------------------------------ MMA issue
        if (lane == 0) {
            const uint32_t idesc = instr_desc(Tr::fmt, NT);
            const uint32_t ring = smem_u32(sRing), b_base = smem_u32(sB);
            bool issued = false;
            for (int t = first; t < last; ++t) {
                const int i = t - first, s = i % NB, ks = i / NB, buf = i & 1, kb = i >> 1;
                if (!mbar_wait(full + s, ks & 1, abort_flag, status)) break;
                if (!mbar_wait(tempty + buf, (kb & 1) ^ 1, abort_flag, status)) break;
                tc_fence_after();
                const uint32_t bst = b_base + (uint32_t)(s * C::B_STAGE);
                bool ok = true;
                for (int mt = 0; mt < MT && ok; ++mt) {
                    const uint32_t d = tmem_base + (uint32_t)((buf * MT + mt) * NT);
                    for (int ka = 0; ka < KA; ++ka) {
                        const int gblk = (i * MT + mt) * KA + ka;
                        const int q = gblk % RS, u = gblk / RS;
                        if (!mbar_wait(afull + q, u & 1, abort_flag, status)) { ok = false; break; }
                        tc_fence_after();
                        const uint32_t ab = ring + (uint32_t)(q * C::A_BLOCK);
#pragma unroll
                        for (int m = 0; m < MMAS_PER_ATOM; ++m) {
                            const uint32_t koff = (uint32_t)(m * 32);
                            const uint32_t a0 = ab + koff;
                            const uint32_t b0 = bst + (uint32_t)(ka * NT * 128) + koff;
                            umma<KIND>(d, smem_desc(a0), smem_desc(b0), idesc, (ka > 0 || m > 0) ? 1u : 0u);
                            if constexpr (Tr::nprod == 3) {
                                umma<KIND>(d, smem_desc(a0), smem_desc(b0 + (uint32_t)C::B_PART), idesc, 1);
                                umma<KIND>(d, smem_desc(a0 + (uint32_t)C::A_PART), smem_desc(b0), idesc, 1);
                            }
                        }
                        umma_commit(aempty + q);   // ring slot free once these products are done
                        issued = true;
                    }
                }
                if (!ok) break;
                umma_commit(empty + s);
                umma_commit(tfull + buf);
            }
            if (issued) {
                umma_commit(drain);
                mbar_wait_drain(drain, 0, status);
            }
        }
        __syncwarp();
    } else if (warp == kBigLoaderWarp) {
        // ------------------------------------------------------------ operator blocks
        if (lane == 0) {
            int last_u[4] = {-1, -1, -1, -1};
            int p = 0;   // operator cursor (tile_info)
            for (int t = first; t < last; ++t) {
                const int i = t - first;
                int col0, nc;
                tile_info(t, ts, class_off, NT, p, col0, nc, lastc);
                bool ok = true;
                for (int mt = 0; mt < MT && ok; ++mt)
                    for (int ka = 0; ka < KA; ++ka) {
                        const int gblk = (i * MT + mt) * KA + ka;
                        const int q = gblk % RS, u = gblk / RS;
                        if (!mbar_wait(aempty + q, (u & 1) ^ 1, abort_flag, status)) { ok = false; break; }
                        mbar_arrive_expect_tx(afull + q, (uint32_t)C::A_BLOCK);
                        const int pi = img_of_class ? __ldg(img_of_class + p) : p;
                        bulk_g2s(sRing + q * C::A_BLOCK, a_img + ((size_t)(pi * MT + mt) * KA + ka) * C::A_BLOCK,
                                 (uint32_t)C::A_BLOCK, afull + q);
                        last_u[q] = u;
                    }
                if (!ok) break;
            }
            // operator blocks still in flight land before the CTA exits
            for (int q = 0; q < RS; ++q)
                if (last_u[q] >= 0) mbar_wait_drain(afull + q, last_u[q] & 1, status);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ epilogue
        const int grp = (threadIdx.x - kBigEpiWarp0 * 32) / 128;
        const int a = threadIdx.x - kBigEpiWarp0 * 32 - 128 * grp;   // 0..127 within the group
        const int q = warp & 3;
        const int bar_id = grp == 0 ? 1 : 3;
        float *sF = sF_all + grp * 16 * FS;
        int *e_goff = e_goff_all + grp * NT;
        int *e_tgt = e_tgt_all + grp * NT;
        int cur = -1;
        float acc[MT];
#pragma unroll
        for (int k = 0; k < MT; ++k) acc[k] = 0.0f;
        int p = 0;   // operator cursor (tile_info)
        for (int t = first; t < last; ++t) {
            const int i = t - first, buf = i & 1, kb = i >> 1;
            int col0, nc;
            tile_info(t, ts, class_off, NT, p, col0, nc, lastc);
            if (EG == 2 && buf != grp) continue;
            if (a < NT) {
                const int2 r = (a < nc) ? __ldg(rec + col0 + a) : make_int2(0, 0);
                // un-permutation table rows: K-padded for the M2L, row-padded (MT tiles)
                // for the second low-rank pass, whose K is the rank
                e_goff[a] = rec_g(r.y) * (MODE == 2 ? MT * 128 : C::KPAD);
                e_tgt[a] = (a < nc) ? rec_tgt(r.y) : -1;
            }
            const bool ok = mbar_wait(tfull + buf, kb & 1, abort_flag, status);
            if (named_bar_or(bar_id, 128, ok ? 0 : 1)) break;
            tc_fence_after();
#pragma unroll 1
            for (int ch = 0; ch < NT / 16; ++ch) {
                // the chunk's table offsets in registers: read from shared memory inside
                // the scatter below, each would wait for the previous store to sF
                int go[16];
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) go[jj] = e_goff[16 * ch + jj];
#pragma unroll 1
                for (int mt = 0; mt < MT; ++mt) {
                    float v[16];
                    tmem_ld<16>(tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)((buf * MT + mt) * NT + 16 * ch), v);
                    if (ch == NT / 16 - 1 && mt == MT - 1) {
                        tc_fence_before();
                        mbar_arrive(tempty + buf);
                    }
                    const int row = mt * 128 + 32 * q + lane;
                    if constexpr (MODE == 1) {
                        // Z column of the record, unpermuted, no accumulation
                        if (row < n3) {
#pragma unroll
                            for (int jj = 0; jj < 16; ++jj)
                                if (16 * ch + jj < nc) out_f32[(size_t)(col0 + 16 * ch + jj) * n3 + row] = v[jj];
                        }
                        continue;
                    }
                    if (row < n3) {
#pragma unroll
                        for (int jj = 0; jj < 16; ++jj)
                            sF[jj * FS + __ldg(sinv_pad + go[jj] + row)] = v[jj];
                    }
                }
                if constexpr (MODE == 1) continue;
                named_bar_sync(bar_id, 128);
                int tg[16];
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) tg[jj] = e_tgt[16 * ch + jj];
                unsigned bm = 0u;
                int prev = cur;
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) {
                    bm |= ((tg[jj] >= 0 && tg[jj] != prev) ? 1u : 0u) << jj;
                    prev = tg[jj] >= 0 ? tg[jj] : prev;
                }
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) {
                    if (bm & (1u << jj)) {
                        if (cur >= 0) {
#pragma unroll
                            for (int k = 0; k < MT; ++k) {
                                const int node = a + 128 * k;
                                if (node < n3) {
                                    if (out_f64) atomicAdd(out_f64 + (size_t)cur * n3 + node, (double)acc[k] * (double)scale);
                                    else atomicAdd(out_f32 + (size_t)cur * n3 + node, acc[k] * scale);
                                }
                            }
                        }
#pragma unroll
                        for (int k = 0; k < MT; ++k) acc[k] = 0.0f;
                        cur = tg[jj];
                    }
#pragma unroll
                    for (int k = 0; k < MT; ++k) {
                        const int node = a + 128 * k;
                        if (node < n3) acc[k] += sF[jj * FS + node];
                    }
                }
                named_bar_sync(bar_id, 128);
            }
        }
        if (cur >= 0) {
#pragma unroll
            for (int k = 0; k < MT; ++k) {
                const int node = a + 128 * k;
                if (node < n3) {
                    if (out_f64) atomicAdd(out_f64 + (size_t)cur * n3 + node, (double)acc[k] * (double)scale);
                    else atomicAdd(out_f32 + (size_t)cur * n3 + node, acc[k] * scale);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kMmaWarp)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(C::TMEM_COLS)
                     : "memory");
}


// Inverse permutations padded to KPAD entries per row (padding -> index 0).
__global__ void sigma_inverse_padded_kernel(int n3, int kpad, const int16_t *__restrict__ sigma,
                                            int16_t *__restrict__ inv)
{
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < 48 * n3; idx += gridDim.x * blockDim.x) {
        const int g = idx / n3, b = idx % n3;
        inv[g * kpad + sigma[idx]] = (int16_t)b;
    }
}

// Operator images in (M tile, swizzle column) blocks: per operator p, MT x KA
// blocks of nparts x 128 rows x 128 bytes, each 128-byte swizzled.
template <int KIND>
__global__ void a_block_image_kernel(int n3, int MT, int KA, const double *__restrict__ K, uint8_t *__restrict__ img)
{
    using Tr = TcTraits<KIND>;
    constexpr int E = 128 / Tr::esz;
    const int block_bytes = 128 * 128 * Tr::nparts;
    const int p = blockIdx.y;
    const long per_op = (long)MT * 128 * KA * E;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < per_op; idx += (long)gridDim.x * blockDim.x) {
        const int rowg = (int)(idx / (KA * E)), kk = (int)(idx % (KA * E));
        const int mt = rowg / 128, row = rowg % 128, ka = kk / E, e = kk % E;
        const double x = (rowg < n3 && kk < n3) ? K[((size_t)p * n3 + rowg) * n3 + kk] : 0.0;
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

// Two epilogue groups where their shared memory fits, else one.
template <int KIND, int MT, int KA>
constexpr int real_eg()
{
    return BigCfg<KIND, MT, KA, kBigNT, 2>::SMEM <= 227 * 1024 - 256 ? 2 : 1;
}

// Tile shape of the M2L for orders 6-8: the widest tile whose panel, ring and
// epilogue fit, preferring two epilogue groups.  Each operator block streamed
// from L2 and read by the tensor core then serves NT columns, so the A-operand
// traffic per interaction falls as 1 / NT; a second epilogue group drains every
// other tile.  Measured on GB300 at the 1/r^4 workload's level 6 (232 230
// interactions): ell 7 BF16x3 0.54 -> 0.37 ms (64 x 2), TF32 0.51 -> 0.38 ms
// (64 x 2), TF32x3 0.87 -> 0.63 ms (48 x 1); ell 8 BF16x3 0.88 -> 0.65 ms (48 x 1).
template <int KIND, int MT, int KA, int NT, int EG>
constexpr bool big_fits()
{
    return BigCfg<KIND, MT, KA, NT, EG>::SMEM <= 227 * 1024 - 256 && 2 * MT * NT <= 512;
}

template <int KIND, int MT, int KA>
constexpr int big_nt()
{
    return big_fits<KIND, MT, KA, 64, 2>() ? 64
         : (big_fits<KIND, MT, KA, 48, 2>() || big_fits<KIND, MT, KA, 48, 1>()) ? 48 : kBigNT;
}

template <int KIND, int MT, int KA>
constexpr int big_eg()
{
    return big_fits<KIND, MT, KA, 64, 2>() ? 2
         : big_fits<KIND, MT, KA, 48, 2>() ? 2
         : big_fits<KIND, MT, KA, 48, 1>() ? 1 : real_eg<KIND, MT, KA>();
}

// The general form of the large-order kernel: ncls operator images of vector
// length N <= 256 (one or two M tiles), tile offsets given on the device.
// Tiles hold 64 interactions where that fits shared memory (each operator block
// streamed from L2 then serves twice the columns), else 32.
constexpr int kGeneralEG = 2;

template <int KIND, int MT, int KA>
constexpr int general_nt()
{
    return BigCfg<KIND, MT, KA, 64, kGeneralEG>::SMEM <= 227 * 1024 ? 64 : kBigNT;
}

template <int KIND>
bool general_shape(int N, int &mt, int &ka)
{
    constexpr int E = 128 / TcTraits<KIND>::esz;
    if (N <= 0 || N > 256) return false;
    mt = N <= 128 ? 1 : 2;
    ka = (mt * 128) / E;   // K padded to the M tiles
    return true;
}

}  // namespace
}  // namespace m2l
