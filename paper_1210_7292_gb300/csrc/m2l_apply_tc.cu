// Steps a4-a6 on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// One persistent CTA per SM walks a contiguous range of tiles; a tile is NT
// bucketed interactions of one unique operator K_p (Alg. 2, blocked along many
// target cells as in Sec. 4.2.3).  Warp roles:
//   warps 0-7  producers: per tile, gather the NT source multipoles (one
//              column per warp at a time, lane l taking K elements
//              [EPL l, EPL (l+1)), so a warp-wide load reads one vector) and
//              permute them (W_p[sigma_g(b)][c] = w[b], Eq. (30)) straight into
//              a 128-byte-swizzled K-major shared-memory panel (the UMMA B
//              operand), rounded to TF32 or split into BF16/TF32 hi + lo;
//              when the operator changes, warps 0-3 (one per TMEM lane
//              quarter) write its rows into TMEM with tcgen05.st: the UMMA A
//              operand lives in TMEM, next to the accumulators.
//   warp 8     allocates TMEM and issues tcgen05.mma (one thread):
//              F_p = K_p W_p (Eq. (31)) into one of three or four TMEM
//              accumulators, three products hi*hi + hi*lo + lo*hi for the
//              split precisions.
//   warps 9-24 epilogue (four groups of four, each owning a quarter of the
//              columns of every tile): tcgen05.ld of the accumulator, un-permutation
//              f[a] += F_p[sigma_g(a)] (Eq. (32)) through a shared-memory
//              transpose, sum over the consecutive columns of one target,
//              one atomic add per (target, node) and run (Alg. 2, third loop).
// Shared-memory stages and TMEM buffers are handed over with mbarriers; every
// wait is bounded (about two seconds), after which the CTA records
// M2L_ETIMEOUT in the status word, drains its asynchronous work and returns.
#include "m2l_tc_big.cuh"

namespace m2l {
namespace {

constexpr int kEpiWarp0 = 9;
constexpr int kEpiGroups = 4;                        // epilogue groups of four warps
constexpr int kEpiWarps = 4 * kEpiGroups;
constexpr int kThreadsTC = (kProducerWarps + 1 + kEpiWarps) * 32;

// TMEM columns of one operand part of A for KATOMS swizzle columns of K.
template <int KIND>
__host__ __device__ constexpr int tc_a_cols_part(int katoms)
{
    return katoms * (128 / TcTraits<KIND>::esz) * TcTraits<KIND>::esz / 4;
}

template <int KIND, int KATOMS>
__global__ void __launch_bounds__(kThreadsTC, 1)
tc_apply_kernel(const int2 *__restrict__ rec, const int *__restrict__ class_off,
                const uint32_t *__restrict__ a_img, const int16_t *__restrict__ sigma_inv,
                const float *__restrict__ mp, float *__restrict__ out_f32, double *__restrict__ out_f64, int ell,
                int n3, float scale, int *status, int stall_first_stage)
{
    using Tr = TcTraits<KIND>;
    constexpr int NT = Tr::NT;
    constexpr int ELEMS_PER_ATOM = 128 / Tr::esz;           // K elements per 128-byte row
    constexpr int K_PER_MMA = 32 / Tr::esz;                  // 8 (tf32) or 16 (bf16)
    constexpr int MMAS_PER_ATOM = ELEMS_PER_ATOM / K_PER_MMA;  // 4
    constexpr int KPAD = KATOMS * ELEMS_PER_ATOM;            // padded K (source nodes)
    constexpr int NPT = kProducerWarps * 32;                 // producer threads
    constexpr int EPL = KPAD / 32;                           // K elements per lane and column
    constexpr int CPW = NT / kProducerWarps;                 // columns per producer warp
    constexpr int NPASS = CPW >= 16 ? 2 : 1;                 // gather passes per tile (register budget)
    constexpr int CPP = CPW / NPASS;                         // columns per warp and pass
    constexpr int NWL = EPL * Tr::esz / 4;                   // 32-bit words per lane, column and part
    constexpr int A_COLS_PART = tc_a_cols_part<KIND>(KATOMS);  // TMEM columns of one part of A
    constexpr int B_PART = KATOMS * NT * 128;                // one operand part of a B stage
    constexpr int B_STAGE = B_PART * Tr::nparts;
    constexpr int ECOLS = NT / kEpiGroups;                   // columns per epilogue group and tile
    constexpr int ECH = ECOLS < 16 ? ECOLS : 16;             // columns per TMEM load
    static_assert(KPAD % 32 == 0 && NT % kProducerWarps == 0 && NWL >= 1, "producer mapping");
    static_assert(ECOLS % ECH == 0 && (ECH == 16 || ECH == 8), "epilogue chunking");

    extern __shared__ uint8_t smem_raw[];
    // 1024-byte alignment by offsetting the __shared__ array itself, so that every
    // access below stays a shared-memory access (an integer round trip would
    // turn them into generic ones)
    uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint8_t *sB = smem;                                               // 2 stages
    float *sF = reinterpret_cast<float *>(sB + 2 * B_STAGE);          // [groups][2 buffers][ECH][129]
    int16_t *s_sinv = reinterpret_cast<int16_t *>(sF + 2 * kEpiGroups * ECH * 129);  // [48][KPAD] inverse perms
    int2 *s_prec = reinterpret_cast<int2 *>(s_sinv + 48 * KPAD);      // [2][NT] producer records
    int2 *s_erec = s_prec + 2 * NT;                                   // [2][NT] writer + [2][NT] int target tables
    int2 *s_gaff = s_erec + 3 * NT;                                   // [48] affine form of sigma_g^{-1}
    uint64_t *bars = reinterpret_cast<uint64_t *>(s_gaff + 48);
    uint64_t *full = bars, *empty = bars + 2, *tfull = bars + 4, *tempty = bars + 8, *a_ready = bars + 12,
             *drain = bars + 13;
    __shared__ uint32_t s_tmem_base;
    __shared__ int s_abort;
    __shared__ int s_tile_start[17];
    __shared__ TileSched s_sched;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // TMEM: NACC accumulators of NT columns, then the operator (nparts x A_COLS_PART columns)
    constexpr int NACC = (4 * NT + Tr::nparts * A_COLS_PART <= 512) ? 4 : 3;
    constexpr int A_COL0 = NACC * NT;
    constexpr int TMEM_COLS = tmem_alloc_cols(A_COL0 + Tr::nparts * A_COLS_PART);
    static_assert(A_COL0 + Tr::nparts * A_COLS_PART <= 512 && A_COLS_PART % 32 == 0, "TMEM budget");

    // inverse permutation tables sigma_g^{-1}, rows padded to KPAD with index 0
    // (padded K rows of the panel meet zero operator columns)
    for (int idx = threadIdx.x; idx < 48 * KPAD; idx += blockDim.x) {
        const int g = idx / KPAD, kk = idx % KPAD;
        s_sinv[idx] = (kk < n3) ? sigma_inv[g * n3 + kk] : (int16_t)0;
    }
    // sigma_g^{-1} is a signed axis permutation of the node digits, hence affine in
    // them: sigma_g^{-1}(a') = C + sum_e M_e d_e(a'), with C = sigma_g^{-1}(0) and
    // M_e = sigma_g^{-1}(ell^e) - C.  Kept as the byte multipliers 4 M_e (a dp4a
    // operand, |4 M_e| <= 4 ell^2 <= 100 for ell <= 5) and 4 C.
    if (threadIdx.x < 48) {
        const int g = threadIdx.x;
        const int c0 = sigma_inv[g * n3];
        uint32_t m = 0;
        for (int e = 0, pw = 1; e < 3; ++e, pw *= ell)
            m |= ((uint32_t)(4 * (sigma_inv[g * n3 + pw] - c0)) & 0xFFu) << (8 * e);
        s_gaff[g] = make_int2((int)m, 4 * c0);
    }
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
            mbar_init(full + i, NPT);
            mbar_init(empty + i, 1);
        }
        for (int i = 0; i < NACC; ++i) {
            mbar_init(tfull + i, 1);
            mbar_init(tempty + i, kEpiWarps * 32);
        }
        mbar_init(a_ready, 128);
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
        // warp w fills columns w, w + 8, ...; lane l the K elements [EPL l, EPL (l + 1)) of
        // each, so that one warp-wide gather reads a single source vector
        const int ptid = threadIdx.x;
        const int kbyte = EPL * lane * Tr::esz;                       // byte position along K
        const uint32_t lane_off = (uint32_t)(kbyte >> 7) * (uint32_t)(NT * 128);  // swizzle column
        const int lane_chunk = (kbyte & 127) >> 4, lane_within = kbyte & 15;
        int prev_p = -1;
        int p = 0, p1 = 0;                   // operator cursors of this tile and of the next
        // records are fetched one tile ahead, into a register of thread c < NT
        int2 nxt = make_int2(0, 0);
        if (first < last && ptid < NT) {
            int c00, nc0;
            tile_info(first, s_tile_start, class_off, NT, p1, c00, nc0);
            if (ptid < nc0) nxt = __ldg(rec + c00 + ptid);
        }
        for (int t = first; t < last; ++t) {
            const int i = t - first, s = i & 1, k = i >> 1;
            int col0, nc;
            tile_info(t, s_tile_start, class_off, NT, p, col0, nc);
            if (p != prev_p) {
                // the operator changes: once the MMAs of the previous tile (the last readers
                // of the old operator) are complete, warps 0-3 write the rows of K_p into
                // TMEM, each warp its own lane quarter, thread ptid row ptid
                if (ptid < 128) {
                    bool ok = true;
                    if (i > 0) ok = mbar_wait(empty + ((i - 1) & 1), ((i - 1) >> 1) & 1, abort_flag, status);
                    // tcgen05.st is warp-collective: the whole warp writes or none of it
                    if (__all_sync(0xffffffffu, ok)) {
                        tc_fence_after();
#pragma unroll 1
                        for (int part = 0; part < Tr::nparts; ++part) {
                            const uint4 *src = reinterpret_cast<const uint4 *>(
                                a_img + (((size_t)p * Tr::nparts + part) * 128 + ptid) * A_COLS_PART);
#pragma unroll 1
                            for (int c0 = 0; c0 < A_COLS_PART; c0 += 32) {
                                uint32_t r[32];
#pragma unroll
                                for (int v = 0; v < 8; ++v) {
                                    const uint4 x = __ldg(src + c0 / 4 + v);
                                    r[4 * v] = x.x; r[4 * v + 1] = x.y; r[4 * v + 2] = x.z; r[4 * v + 3] = x.w;
                                }
                                tmem_st32(tmem_base + ((uint32_t)(32 * warp) << 16) +
                                              (uint32_t)(A_COL0 + part * A_COLS_PART + c0), r);
                            }
                        }
                        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                        tc_fence_before();
                        mbar_arrive(a_ready);
                    }
                }
                prev_p = p;
            }
            // records of this tile; the previous tile with this stage is fully consumed
            int2 *prec = s_prec + s * NT;
            if (ptid < NT) {
                prec[ptid] = nxt;
                nxt = make_int2(0, 0);
                if (t + 1 < last) {
                    int c01, nc1;
                    tile_info(t + 1, s_tile_start, class_off, NT, p1, c01, nc1);
                    if (ptid < nc1) nxt = __ldg(rec + c01 + ptid);
                }
            }
            named_bar_sync(2, NPT);
            uint8_t *stage = sB + s * B_STAGE;
            bool stop = false;
#pragma unroll
            for (int pass = 0; pass < NPASS; ++pass) {
                // issue every gather of this pass before the stores (the first pass also
                // before waiting for the stage)
                float v[CPP][EPL];
#pragma unroll
                for (int uu = 0; uu < CPP; ++uu) {
                    const int c = warp + (pass * CPP + uu) * kProducerWarps;
                    const bool live = (c < nc);
                    const int2 r = live ? prec[c] : make_int2(0, 0);
                    const float *w = mp + (size_t)r.x * n3;
                    const int16_t *si = s_sinv + rec_g(r.y) * KPAD + EPL * lane;
                    int idx[EPL];
                    if constexpr (EPL == 4) {
                        const uint2 q = *reinterpret_cast<const uint2 *>(si);
                        idx[0] = (int16_t)(q.x & 0xFFFF); idx[1] = (int16_t)(q.x >> 16);
                        idx[2] = (int16_t)(q.y & 0xFFFF); idx[3] = (int16_t)(q.y >> 16);
                    } else if constexpr (EPL == 2) {
                        const uint32_t q = *reinterpret_cast<const uint32_t *>(si);
                        idx[0] = (int16_t)(q & 0xFFFF); idx[1] = (int16_t)(q >> 16);
                    } else {
                        idx[0] = si[0];
                    }
#pragma unroll
                    for (int e = 0; e < EPL; ++e) v[uu][e] = live ? __ldg(w + idx[e]) : 0.0f;
                }
                if (pass == 0) {
                    const bool ok = mbar_wait(empty + s, (k & 1) ^ 1, abort_flag, status);
                    if (named_bar_or(2, NPT, ok ? 0 : 1)) {
                        stop = true;
                        break;
                    }
                }
#pragma unroll
                for (int uu = 0; uu < CPP; ++uu) {
                    const int c = warp + (pass * CPP + uu) * kProducerWarps;
                    uint8_t *dst = stage + lane_off + swz_off(c, lane_chunk) + lane_within;
                    uint32_t hi[NWL], lo[NWL];
                    if constexpr (KIND == TC_BF16X3) {
#pragma unroll
                        for (int e = 0; e < EPL; e += 2) {
                            // two values per conversion, the even K index in the low half
                            const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[uu][e], v[uu][e + 1]);
                            const uint32_t hu = *reinterpret_cast<const uint32_t *>(&h2);
                            const __nv_bfloat162 l2 = __floats2bfloat162_rn(
                                v[uu][e] - __uint_as_float(hu << 16), v[uu][e + 1] - __uint_as_float(hu & 0xFFFF0000u));
                            hi[e / 2] = hu;
                            lo[e / 2] = *reinterpret_cast<const uint32_t *>(&l2);
                        }
                    } else {
#pragma unroll
                        for (int e = 0; e < EPL; ++e) {
                            const float h = tf32_rna(v[uu][e]);
                            hi[e] = __float_as_uint(h);
                            lo[e] = __float_as_uint(tf32_rna(v[uu][e] - h));
                        }
                    }
                    st_shared_words<NWL>(dst, hi);
                    if constexpr (Tr::nparts == 2) st_shared_words<NWL>(dst + B_PART, lo);
                }
            }
            if (stop) break;
            fence_proxy_async();
            // stall_first_stage (a test switch) withholds the first stage's signal, so the
            // MMA warp's bounded wait runs out and the CTA takes its abort path
            if (!(stall_first_stage && i == 0)) mbar_arrive(full + s);
        }
    } else if (warp == kMmaWarp) {
        // ------------------------------------------------------------ MMA issue
        if (lane == 0) {
            const uint32_t idesc = instr_desc(Tr::fmt, NT);
            const uint32_t a_base = tmem_base + (uint32_t)A_COL0, b_base = smem_u32(sB);
            int prev_p = -1, p = 0;
            uint32_t a_loads = 0;
            bool issued = false;
            for (int t = first; t < last; ++t) {
                const int i = t - first, s = i & 1, k = i >> 1;
                int col0, nc;
                tile_info(t, s_tile_start, class_off, NT, p, col0, nc);
                if (!mbar_wait(full + s, k & 1, abort_flag, status)) break;
                if (p != prev_p) {
                    if (!mbar_wait(a_ready, a_loads & 1, abort_flag, status)) break;
                    tc_fence_after();
                    ++a_loads;
                    prev_p = p;
                }
                const int ab = i % NACC, ak = i / NACC;
                if (!mbar_wait(tempty + ab, (ak & 1) ^ 1, abort_flag, status)) break;
                tc_fence_after();
                const uint32_t d = tmem_base + (uint32_t)(ab * NT);
                const uint32_t bst = b_base + (uint32_t)(s * B_STAGE);
                uint32_t accum = 0;
#pragma unroll
                for (int ka = 0; ka < KATOMS; ++ka) {
#pragma unroll
                    for (int m = 0; m < MMAS_PER_ATOM; ++m) {
                        // 32 bytes of K per MMA: 8 TMEM columns of A, 32 bytes into the swizzled B row
                        const uint32_t a0 = a_base + (uint32_t)(ka * 32 + m * 8);
                        const uint32_t b0 = bst + (uint32_t)(ka * NT * 128) + (uint32_t)(m * 32);
                        umma_ta<KIND>(d, a0, smem_desc(b0), idesc, accum);
                        accum = 1;
                        if constexpr (Tr::nprod == 3) {
                            // hi*lo and lo*hi into the same accumulator
                            umma_ta<KIND>(d, a0, smem_desc(b0 + (uint32_t)B_PART), idesc, 1);
                            umma_ta<KIND>(d, a0 + (uint32_t)A_COLS_PART, smem_desc(b0), idesc, 1);
                        }
                    }
                }
                umma_commit(empty + s);
                umma_commit(tfull + ab);
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
        // four groups of four warps; group G owns columns [G*ECOLS, (G+1)*ECOLS) of every tile
        const int et = threadIdx.x - kEpiWarp0 * 32;   // 0..255
        const int G = et >> 7;
        const int a = et & 127;                        // output node handled in the reduction
        const int q = warp & 3;                        // TMEM lane quarter this warp may read
        const int row = 32 * q + lane;                 // accumulator row (permuted node a')
        const int bar_id = G == 0 ? 1 : 2 + G;         // named barriers 1, 3, 4, 5 (2: producers)
        // two transpose buffers per group: chunk c (counted across tiles) uses buffer c & 1,
        // so one barrier per chunk separates its writes from its reads
        float *sFg = sF + 2 * G * ECH * 129;
        constexpr int NCHG = ECOLS / ECH;                 // chunks per group and tile
        // per column of this group, double-buffered by tile: the dp4a multipliers of its sigma
        // and the byte address of node 0 of its transpose column; and its target (-1: dead)
        int2 *e_wt0 = s_erec + G * 2 * ECOLS;
        int *e_tgt0 = reinterpret_cast<int *>(s_erec + 2 * NT) + G * 2 * ECOLS;
        // digits of a' in signed bytes, the other dp4a operand
        const int xd = (row % ell) | ((row / ell % ell) << 8) | ((row / (ell * ell)) << 16);
        const int col_addr = (int)smem_u32(sFg) + (a % ECH) * 129 * 4;   // used by threads a < ECOLS
        int cur = -1;
        float acc = 0.0f;
        const int gc0 = G * ECOLS;                        // first tile column of this group
        // records are fetched one tile ahead, into a register of thread a < ECOLS (y = -1: dead column)
        int nxt = -1;
        int p1 = 0;                                       // operator cursor of the next tile
        if (first < last && a < ECOLS) {
            int c00, nc0;
            tile_info(first, s_tile_start, class_off, NT, p1, c00, nc0);
            if (a < nc0 - gc0) nxt = __ldg(rec + c00 + gc0 + a).y;
        }
        for (int t = first; t < last; ++t) {
            const int i = t - first, ab = i % NACC, ak = i / NACC;
            int2 *e_wt = e_wt0 + (i & 1) * ECOLS;
            int *e_tgt = e_tgt0 + (i & 1) * ECOLS;
            if (a < ECOLS) {
                const int2 ga = s_gaff[nxt == -1 ? 0 : rec_g(nxt)];
                const int bsel = ((i * NCHG + a / ECH) & 1) * (ECH * 129 * 4);
                e_wt[a] = make_int2(ga.x, ga.y + col_addr + bsel);
                e_tgt[a] = (nxt == -1) ? -1 : rec_tgt(nxt);
                nxt = -1;
                if (t + 1 < last) {
                    int c01, nc1;
                    tile_info(t + 1, s_tile_start, class_off, NT, p1, c01, nc1);
                    if (a < nc1 - gc0) nxt = __ldg(rec + c01 + gc0 + a).y;
                }
            }
            // all four warps of the group leave together if any of them gave up
            const bool ok = mbar_wait(tfull + ab, ak & 1, abort_flag, status);
            if (named_bar_or(bar_id, 128, ok ? 0 : 1)) break;
            tc_fence_after();
#pragma unroll 1
            for (int ch = 0; ch < ECOLS / ECH; ++ch) {
                float v[ECH];
                tmem_ld<ECH>(tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(ab * NT + gc0 + ECH * ch), v);
                if (ch == ECOLS / ECH - 1) {
                    tc_fence_before();
                    mbar_arrive(tempty + ab);
                }
                // un-permute on the write: row a' of column jj lands at node sigma_g^{-1}(a')
                if (row < n3) {
                    const int2 *wt = e_wt + ECH * ch;
#pragma unroll
                    for (int jj = 0; jj < ECH; ++jj) {
                        const int2 e = wt[jj];
                        const uint32_t addr = (uint32_t)__dp4a(xd, e.x, e.y);
                        asm volatile("st.shared.f32 [%0], %1;" ::"r"(addr), "f"(v[jj]) : "memory");
                    }
                }
                named_bar_sync(bar_id, 128);
                // run starts of this chunk as one warp ballot: lane jj tests column jj, live and
                // with a target other than its predecessor's (the dead columns of a ragged tile
                // come last, so the predecessor of a live column is live or the open run)
                unsigned bm;
                {
                    const int jl = lane < ECH ? lane : ECH - 1;
                    const int tj = e_tgt[ECH * ch + jl];
                    const int tp = (jl > 0) ? e_tgt[ECH * ch + jl - 1] : (ch > 0 ? e_tgt[ECH * ch - 1] : cur);
                    bm = __ballot_sync(0xffffffffu, lane < ECH && tj >= 0 && tj != tp);
                }
                // rows a >= n3 of the transpose are never written: read (in bounds) and never added
                const float *fb = sFg + ((i * NCHG + ch) & 1) * (ECH * 129);
                float x[ECH];
#pragma unroll
                for (int jj = 0; jj < ECH; ++jj) x[jj] = fb[jj * 129 + a];
#pragma unroll
                for (int h = 0; h < ECH; h += 8) {
                    if (((bm >> h) & 0xFFu) == 0u) {
                        // no run starts in these eight columns: one tree sum
                        acc += ((x[h] + x[h + 1]) + (x[h + 2] + x[h + 3])) + ((x[h + 4] + x[h + 5]) + (x[h + 6] + x[h + 7]));
                        continue;
                    }
#pragma unroll
                    for (int jj = h; jj < h + 8; ++jj) {
                        if (bm & (1u << jj)) {
                            if (cur >= 0 && a < n3) {
                                if (out_f64) atomicAdd(out_f64 + (size_t)cur * n3 + a, (double)acc * (double)scale);
                                else atomicAdd(out_f32 + (size_t)cur * n3 + a, acc * scale);
                            }
                            acc = 0.0f;
                            cur = e_tgt[ECH * ch + jj];
                        }
                        acc += x[jj];
                    }
                }
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

// Operator images for TMEM: per operator p and operand part, 128 rows of
// tc_a_cols_part 32-bit columns (row a = output node, zero beyond n3; column j
// = source node j for TF32, source nodes 2j and 2j + 1 for BF16, the even one in
// the low half), the split precisions storing hi and lo as two parts.
template <int KIND>
__global__ void a_tmem_image_kernel(int n3, int cols_part, const double *__restrict__ K, uint32_t *__restrict__ img)
{
    using Tr = TcTraits<KIND>;
    const int p = blockIdx.y;
    uint32_t *base = img + (size_t)p * Tr::nparts * 128 * cols_part;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < 128 * cols_part; idx += gridDim.x * blockDim.x) {
        const int row = idx / cols_part, col = idx % cols_part;
        if constexpr (KIND == TC_BF16X3) {
            uint32_t hi = 0, lo = 0;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int kk = 2 * col + h;
                const double x = (row < n3 && kk < n3) ? K[((size_t)p * n3 + row) * n3 + kk] : 0.0;
                const __nv_bfloat16 bh = __double2bfloat16(x);
                const __nv_bfloat16 bl = __double2bfloat16(x - (double)__bfloat162float(bh));
                hi |= (uint32_t)__bfloat16_as_ushort(bh) << (16 * h);
                lo |= (uint32_t)__bfloat16_as_ushort(bl) << (16 * h);
            }
            base[idx] = hi;
            base[128 * cols_part + idx] = lo;
        } else {
            const double x = (row < n3 && col < n3) ? K[((size_t)p * n3 + row) * n3 + col] : 0.0;
            const float h = tf32_rna((float)x);
            base[idx] = __float_as_uint(h);
            if constexpr (KIND == TC_TF32X3) base[128 * cols_part + idx] = __float_as_uint(tf32_rna((float)(x - (double)h)));
        }
    }
}

template <int KIND>
int tc_katoms(int n3)
{
    constexpr int E = 128 / TcTraits<KIND>::esz;
    int k = (n3 + E - 1) / E;
    return k == 3 ? 4 : k;   // instantiated for 1, 2 and 4 swizzle columns
}

template <int KIND>
size_t tc_smem_bytes(int katoms)
{
    using Tr = TcTraits<KIND>;
    constexpr int ECOLS = Tr::NT / kEpiGroups;
    constexpr int ECH = ECOLS < 16 ? ECOLS : 16;
    const size_t b = 2 * (size_t)katoms * Tr::NT * 128 * Tr::nparts;
    const size_t kpad = (size_t)katoms * (128 / Tr::esz);
    return 1024 + b + 2 * kEpiGroups * ECH * 129 * sizeof(float) + 48 * kpad * sizeof(int16_t) +
           (5 * Tr::NT + 48) * sizeof(int2) + 16 * sizeof(uint64_t);
}

template <int KIND, int KATOMS>
m2l_status launch_atoms(const m2l_ops *ops, const Buckets &b, Layout &L, const float *in, void *out,
                        int out_fp64, double scale, cudaStream_t s)
{
    using Tr = TcTraits<KIND>;
    const size_t smem = tc_smem_bytes<KIND>(KATOMS);
    if ((int)smem > max_smem_optin()) {
        set_error("tensor-core kernel needs %zu bytes of shared memory", smem);
        return M2L_EUNSUPPORTED;
    }
    auto kern = tc_apply_kernel<KIND, KATOMS>;
    M2L_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    long grid = num_sms();
    const long tiles_bound = (long)(b.nnz + Tr::NT - 1) / Tr::NT + 16;
    if (grid > tiles_bound) grid = tiles_bound;
    kern<<<(int)grid, kThreadsTC, smem, s>>>(b.rec.as<int2>(), b.class_off.as<int>(), L.a.as<uint32_t>(),
                                             L.b.as<int16_t>(), in, out_fp64 ? nullptr : (float *)out,
                                             out_fp64 ? (double *)out : nullptr, ops->ell, ops->n3, (float)scale,
                                             ops->d_status, (ops->debug_flags & M2L_DEBUG_STALL_PRODUCER) ? 1 : 0);
    M2L_LAUNCH_CHECK("tc_apply_kernel");
    return M2L_OK;
}

template <int KIND>
m2l_status launch_big_ell(const m2l_ops *ops, const Buckets &b, Layout &L, const float *in, void *out, int out_fp64,
                          double scale, cudaStream_t s);

template <int KIND>
m2l_status launch_kind(const m2l_ops *ops, const Buckets &b, Layout &L, const float *in, void *out, int out_fp64,
                       double scale, cudaStream_t s)
{
    using Tr = TcTraits<KIND>;
    constexpr int prec = KIND == TC_TF32 ? M2L_TF32 : KIND == TC_BF16X3 ? M2L_BF16X3 : M2L_TF32X3;
    const int n3 = ops->n3;
    // per-operator low-rank factors: two passes of the large-order kernel
    if (ops->eps > 0) return launch_tc_lowrank(ops, b, prec, in, out, out_fp64, scale, s);
    if (n3 > 128) return launch_big_ell<KIND>(ops, b, L, in, out, out_fp64, scale, s);
    if (b.nnz > 0 && b.dense.valid && !(ops->debug_flags & M2L_DEBUG_NO_DENSE))
        return launch_tc_dense(ops, b.dense, prec, in, out, out_fp64, scale, s);
    const int katoms = tc_katoms<KIND>(n3);
    const int cols_part = tc_a_cols_part<KIND>(katoms);
    const size_t a_bytes = (size_t)Tr::nparts * 128 * cols_part * sizeof(uint32_t);
    m2l_status st;
    if (!L.ready) {
        if ((st = L.a.ensure((size_t)16 * a_bytes)) != M2L_OK) return st;
        if ((st = L.b.ensure((size_t)48 * n3 * sizeof(int16_t))) != M2L_OK) return st;
        dim3 grid((128 * cols_part + 255) / 256, 16);
        a_tmem_image_kernel<KIND><<<grid, 256, 0, s>>>(n3, cols_part, ops->K64.as<double>(), L.a.as<uint32_t>());
        M2L_LAUNCH_CHECK("a_tmem_image_kernel");
        sigma_inverse_kernel<<<(48 * n3 + 255) / 256, 256, 0, s>>>(n3, ops->sigma.as<int16_t>(), L.b.as<int16_t>());
        M2L_LAUNCH_CHECK("sigma_inverse_kernel");
        L.ready = true;
    }
    if (b.nnz == 0) return M2L_OK;
    if (katoms == 1) return launch_atoms<KIND, 1>(ops, b, L, in, out, out_fp64, scale, s);
    if (katoms == 2) return launch_atoms<KIND, 2>(ops, b, L, in, out, out_fp64, scale, s);
    if constexpr (KIND != TC_BF16X3)   // bf16 rows hold 64 nodes: ell <= 5 needs at most two columns
        return launch_atoms<KIND, 4>(ops, b, L, in, out, out_fp64, scale, s);
    set_error("no tensor-core configuration for %d swizzle columns", katoms);
    return M2L_EUNSUPPORTED;
}


template <int KIND, int MT, int KA>
m2l_status launch_big(const m2l_ops *ops, const Buckets &b, Layout &L, const float *in, void *out, int out_fp64,
                      double scale, cudaStream_t s)
{
    using Tr = TcTraits<KIND>;
    constexpr int NT = big_nt<KIND, MT, KA>();
    constexpr int EG = big_eg<KIND, MT, KA>();
    using C = BigCfg<KIND, MT, KA, NT, EG>;
    const int n3 = ops->n3;
    const size_t img_bytes = (size_t)16 * MT * KA * C::A_BLOCK;
    m2l_status st;
    if (!L.ready) {
        if ((st = L.a.ensure(img_bytes)) != M2L_OK) return st;
        if ((st = L.b.ensure((size_t)48 * C::KPAD * sizeof(int16_t))) != M2L_OK) return st;
        M2L_CUDA(cudaMemsetAsync(L.a.p, 0, img_bytes, s));
        M2L_CUDA(cudaMemsetAsync(L.b.p, 0, (size_t)48 * C::KPAD * sizeof(int16_t), s));
        dim3 grid((unsigned)((MT * 128L * KA * C::E + 255) / 256), 16);
        a_block_image_kernel<KIND><<<grid, 256, 0, s>>>(n3, MT, KA, ops->K64.as<double>(), L.a.as<uint8_t>());
        M2L_LAUNCH_CHECK("a_block_image_kernel");
        sigma_inverse_padded_kernel<<<(48 * n3 + 255) / 256, 256, 0, s>>>(n3, C::KPAD, ops->sigma.as<int16_t>(),
                                                                        L.b.as<int16_t>());
        M2L_LAUNCH_CHECK("sigma_inverse_padded_kernel");
        L.ready = true;
    }
    if (b.nnz == 0) return M2L_OK;
    if (C::SMEM > max_smem_optin()) {
        set_error("tensor-core kernel for ell = %d needs %d bytes of shared memory", ops->ell, C::SMEM);
        return M2L_EUNSUPPORTED;
    }
    auto kern = tc_big_kernel<KIND, MT, KA, NT, EG>;
    M2L_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    long grid = num_sms();
    const long tiles_bound = (long)(b.nnz + NT - 1) / NT + 16;
    if (grid > tiles_bound) grid = tiles_bound;
    kern<<<(int)grid, big_threads(EG), C::SMEM, s>>>(b.rec.as<int2>(), b.class_off.as<int>(), L.a.as<uint8_t>(),
                                                 L.b.as<int16_t>(), in, out_fp64 ? nullptr : (float *)out,
                                                 out_fp64 ? (double *)out : nullptr, n3, (float)scale, ops->d_status,
                                                 (ops->debug_flags & M2L_DEBUG_STALL_PRODUCER) ? 1 : 0, kNumSym,
                                                 nullptr, nullptr, n3, nullptr);
    M2L_LAUNCH_CHECK("tc_big_kernel");
    return M2L_OK;
}

template <int KIND>
m2l_status launch_big_ell(const m2l_ops *ops, const Buckets &b, Layout &L, const float *in, void *out, int out_fp64,
                          double scale, cudaStream_t s)
{
    constexpr bool BF = (KIND == TC_BF16X3);
    switch (ops->ell) {
    case 6: return BF ? launch_big<KIND, 2, 4>(ops, b, L, in, out, out_fp64, scale, s)
                      : launch_big<KIND, 2, 7>(ops, b, L, in, out, out_fp64, scale, s);
    case 7: return BF ? launch_big<KIND, 3, 6>(ops, b, L, in, out, out_fp64, scale, s)
                      : launch_big<KIND, 3, 11>(ops, b, L, in, out, out_fp64, scale, s);
    case 8: return BF ? launch_big<KIND, 4, 8>(ops, b, L, in, out, out_fp64, scale, s)
                      : launch_big<KIND, 4, 16>(ops, b, L, in, out, out_fp64, scale, s);
    default:
        set_error("no tensor-core configuration for ell = %d", ops->ell);
        return M2L_EUNSUPPORTED;
    }
}

template <int KIND, int MT, int KA>
m2l_status launch_big_general(int N, int ncls, const int *tile_start, const int2 *rec, const int *class_off,
                              const uint8_t *img, const int16_t *tinv, int nnz, const float *in, float *out,
                              int *status, cudaStream_t s)
{
    constexpr int NT = general_nt<KIND, MT, KA>();
    using C = BigCfg<KIND, MT, KA, NT, kGeneralEG>;
    if (C::SMEM > max_smem_optin()) {
        set_error("tensor-core kernel for vector length %d needs %d bytes of shared memory", N, C::SMEM);
        return M2L_EUNSUPPORTED;
    }
    auto kern = tc_big_kernel<KIND, MT, KA, NT, kGeneralEG>;
    M2L_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    long grid = num_sms();
    const long tiles_bound = (long)(nnz + NT - 1) / NT + ncls;
    if (grid > tiles_bound) grid = tiles_bound;
    kern<<<(int)grid, big_threads(kGeneralEG), C::SMEM, s>>>(rec, class_off, img, tinv, in, out, nullptr, N, 1.0f,
                                                             status, 0, ncls, tile_start, nullptr, N, nullptr);
    M2L_LAUNCH_CHECK("tc_big_kernel");
    return M2L_OK;
}


}  // namespace

bool tc_general_config(int precision, int N, int *kpad, size_t *img_bytes_per_op, int *tile_cols)
{
    int mt = 0, ka = 0, esz = 0, nparts = 0, nt = 0;
    const bool two = N > 128;
    switch (precision) {
    case M2L_TF32:
        if (!general_shape<TC_TF32>(N, mt, ka)) return false;
        esz = 4; nparts = 1;
        nt = two ? general_nt<TC_TF32, 2, 8>() : general_nt<TC_TF32, 1, 4>();
        break;
    case M2L_BF16X3:
        if (!general_shape<TC_BF16X3>(N, mt, ka)) return false;
        esz = 2; nparts = 2;
        nt = two ? general_nt<TC_BF16X3, 2, 4>() : general_nt<TC_BF16X3, 1, 2>();
        break;
    case M2L_TF32X3:
        if (!general_shape<TC_TF32X3>(N, mt, ka)) return false;
        esz = 4; nparts = 2;
        nt = two ? general_nt<TC_TF32X3, 2, 8>() : general_nt<TC_TF32X3, 1, 4>();
        break;
    default: return false;
    }
    if (tile_cols) *tile_cols = nt;
    if (kpad) *kpad = ka * (128 / esz);
    if (img_bytes_per_op) *img_bytes_per_op = (size_t)mt * ka * 128 * 128 * nparts;
    return true;
}

m2l_status tc_general_images(int precision, int N, int ncls, const double *K, uint8_t *img, cudaStream_t s)
{
    int mt = 0, ka = 0;
    dim3 grid(1, ncls);
    switch (precision) {
    case M2L_TF32:
        general_shape<TC_TF32>(N, mt, ka);
        grid.x = (unsigned)((mt * 128L * ka * 32 + 255) / 256);
        a_block_image_kernel<TC_TF32><<<grid, 256, 0, s>>>(N, mt, ka, K, img);
        break;
    case M2L_BF16X3:
        general_shape<TC_BF16X3>(N, mt, ka);
        grid.x = (unsigned)((mt * 128L * ka * 64 + 255) / 256);
        a_block_image_kernel<TC_BF16X3><<<grid, 256, 0, s>>>(N, mt, ka, K, img);
        break;
    case M2L_TF32X3:
        general_shape<TC_TF32X3>(N, mt, ka);
        grid.x = (unsigned)((mt * 128L * ka * 32 + 255) / 256);
        a_block_image_kernel<TC_TF32X3><<<grid, 256, 0, s>>>(N, mt, ka, K, img);
        break;
    default:
        set_error("not a tensor-core precision: %d", precision);
        return M2L_EINVAL;
    }
    M2L_LAUNCH_CHECK("a_block_image_kernel");
    return M2L_OK;
}

m2l_status tc_general_apply(int precision, int N, int ncls, const int *tile_start, const int2 *rec,
                            const int *class_off, const uint8_t *img, const int16_t *tinv, int nnz, const float *in,
                            float *out, int *status, cudaStream_t s)
{
    const bool two = N > 128;
    switch (precision) {
    case M2L_TF32:
        return two ? launch_big_general<TC_TF32, 2, 8>(N, ncls, tile_start, rec, class_off, img, tinv, nnz, in, out, status, s)
                   : launch_big_general<TC_TF32, 1, 4>(N, ncls, tile_start, rec, class_off, img, tinv, nnz, in, out, status, s);
    case M2L_BF16X3:
        return two ? launch_big_general<TC_BF16X3, 2, 4>(N, ncls, tile_start, rec, class_off, img, tinv, nnz, in, out, status, s)
                   : launch_big_general<TC_BF16X3, 1, 2>(N, ncls, tile_start, rec, class_off, img, tinv, nnz, in, out, status, s);
    case M2L_TF32X3:
        return two ? launch_big_general<TC_TF32X3, 2, 8>(N, ncls, tile_start, rec, class_off, img, tinv, nnz, in, out, status, s)
                   : launch_big_general<TC_TF32X3, 1, 4>(N, ncls, tile_start, rec, class_off, img, tinv, nnz, in, out, status, s);
    default:
        set_error("not a tensor-core precision: %d", precision);
        return M2L_EINVAL;
    }
}

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
