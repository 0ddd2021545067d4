// The M2L of the directional FMM for the Helmholtz kernel (Sec. 2.1.2,
// Eq. (13)): F^u_X += K_t W^u_Y, K_t[a][b] = K(xbar_a, ybar_b) with
// K(x, y) = exp(i k |x - y|) / |x - y|, for every pair of a level's
// directional far field, one expansion per (cell, cone).  The phases of the
// directional kernel live in P2M and L2P; the operator is the plain kernel,
// so the symmetries of Sec. 4.2.1 hold for any transfer vector and the
// blocking of Alg. 2 applies with the classes found from the lists
// (|T_sym| and n_p are not known before the lists exist, Sec. 4.2.3).
//
//  * lists: Alg. 1 on a uniform-depth octree, written per level: Y is in the
//    far field of X at level L when the pair is admissible at L and no pair of
//    their ancestors is.  Admissibility: |t|_inf >= 2, and at a high-frequency
//    level (k w >= 1) also |c_X - c_Y| > max(k w^2, 2 w).  Cones: the faces of the cube
//    split into m x m squares, m the smallest power of two >= k w; the cone of
//    a pair is the square hit along c_X - c_Y.
//  * plan: classification t -> (p(t), g(t)) over the entries, T_sym in
//    lexicographic order, the complex operators K_p, buckets by p.
//  * apply: tiles of one class; the permuted multipoles of a tile are
//    gathered once into shared memory (row sigma_g(b) of column j holds
//    W_j[b]), the complex product runs over 64-row blocks of K_p, and each
//    result row i is added to the target's node sigma_g^-1(i).
#include <math.h>

#include <algorithm>
#include <vector>

#include "m2l_internal.cuh"

namespace m2l {
namespace {

constexpr int kDMaxM = 32;           // squares per face edge (6 * 32^2 cones)
constexpr int kDListWarps = 4;
constexpr int kDThreads = 256;

// ---------------------------------------------------------------- readings
__host__ __device__ __forceinline__ double d_width(double dw, int level) { return dw / (double)(1 << level); }

__host__ __device__ __forceinline__ int d_cone_m(double k, double w)
{
    if (!(k * w >= 1.0)) return 0;
    int m = 1;
    while ((double)m < k * w) m *= 2;
    return m;
}

// Separated pair at a level of width w (products rounded one by one, as written).
__device__ __forceinline__ bool d_admissible(double k, double w, int t0, int t1, int t2)
{
    const int tinf = max(abs(t0), max(abs(t1), abs(t2)));
    if (tinf < 2) return false;
    if (!(k * w >= 1.0)) return true;
    const double tt = (double)(t0 * t0 + t1 * t1 + t2 * t2);
    const double kww = __dmul_rn(__dmul_rn(k, w), w);
    return __dmul_rn(__dmul_rn(tt, w), w) > __dmul_rn(kww, kww) && tt > 4.0;
}

// Cone of the direction t (integer arithmetic): face axis f (first largest
// |t_i|), side s = (t_f < 0), squares along the other two axes a < b.
__device__ __forceinline__ int d_cone_index(int m, int t0, int t1, int t2)
{
    if (m == 0) return 0;
    const int t[3] = {t0, t1, t2};
    const int at[3] = {abs(t0), abs(t1), abs(t2)};
    int f = 0;
    if (at[1] > at[f]) f = 1;
    if (at[2] > at[f]) f = 2;
    const int s = t[f] < 0 ? 1 : 0;
    const int a = f == 0 ? 1 : 0, b = f == 2 ? 1 : 2;
    const int T = at[f];
    const int ia = min((t[a] + T) * m / (2 * T), m - 1);
    const int ib = min((t[b] + T) * m / (2 * T), m - 1);
    return (2 * f + s) * m * m + ib * m + ia;
}

// ---------------------------------------------------------------- lists
__global__ void d_scatter_cells_kernel(int n, const int32_t *__restrict__ ijk, int side, int32_t *__restrict__ table,
                                       int *__restrict__ bad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int x = ijk[3 * i], y = ijk[3 * i + 1], z = ijk[3 * i + 2];
    if (x < 0 || y < 0 || z < 0 || x >= side || y >= side || z >= side) {
        atomicOr(bad, 1);
        return;
    }
    if (atomicExch(table + x + side * (y + side * z), i) != -1) atomicOr(bad, 2);
}

__global__ void d_check_cells_kernel(int n, const int32_t *__restrict__ ijk, int side, int *__restrict__ bad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int x = ijk[3 * i], y = ijk[3 * i + 1], z = ijk[3 * i + 2];
    if (x < 0 || y < 0 || z < 0 || x >= side || y >= side || z >= side) atomicOr(bad, 1);
}

// One warp per target cell.  The candidates t run over the box [-R, R]^3
// clipped to the grid, from +R down (x fastest), so that Y = X - t ascends
// in linear index and thus in source index.  Count pass: entries per cone;
// fill pass: sources written in that order within each (target, cone).
template <bool FILL>
__global__ void __launch_bounds__(kDListWarps * 32)
d_lists_kernel(int level, double k, double dw, int R, int C, int m, int ntgt, const int32_t *__restrict__ tgt_ijk,
               int side, const int32_t *__restrict__ table, int32_t *__restrict__ counts,
               const int32_t *__restrict__ offsets, int32_t *__restrict__ sources)
{
    extern __shared__ int d_cursor[];   // [kDListWarps][C]
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *my = d_cursor + wib * C;
    const int x = blockIdx.x * kDListWarps + wib;
    for (int c = lane; c < C; c += 32) my[c] = (FILL && x < ntgt) ? offsets[(size_t)x * C + c] : 0;
    __syncwarp();
    if (x < ntgt) {
        const int X[3] = {tgt_ijk[3 * x], tgt_ijk[3 * x + 1], tgt_ijk[3 * x + 2]};
        int hi[3], S[3];
        for (int i = 0; i < 3; ++i) {
            hi[i] = min(R, X[i]);                          // Y_i = X_i - t_i >= 0
            const int lo = max(-R, X[i] - (side - 1));     // Y_i <= side - 1
            S[i] = max(0, hi[i] - lo + 1);
        }
        const long long B = (long long)S[0] * S[1] * S[2];
        const double w = d_width(dw, level);
        for (long long j0 = 0; j0 < B; j0 += 32) {
            const long long j = j0 + lane;
            bool ok = false;
            int y = -1, c = 0;
            if (j < B) {
                const int t0 = hi[0] - (int)(j % S[0]);
                const int t1 = hi[1] - (int)((j / S[0]) % S[1]);
                const int t2 = hi[2] - (int)(j / ((long long)S[0] * S[1]));
                const int Y0 = X[0] - t0, Y1 = X[1] - t1, Y2 = X[2] - t2;
                y = table[Y0 + side * (Y1 + side * Y2)];
                if (y >= 0 && d_admissible(k, w, t0, t1, t2)) {
                    ok = true;
                    for (int l = 0; l < level && ok; ++l) {
                        const int sh = level - l;
                        if (d_admissible(k, d_width(dw, l), (X[0] >> sh) - (Y0 >> sh), (X[1] >> sh) - (Y1 >> sh),
                                         (X[2] >> sh) - (Y2 >> sh)))
                            ok = false;
                    }
                    if (ok) c = d_cone_index(m, t0, t1, t2);
                }
            }
            if (!__any_sync(0xffffffffu, ok)) continue;
            if (!FILL) {
                if (ok) atomicAdd(&my[c], 1);
            } else {
                const unsigned peers = __match_any_sync(0xffffffffu, ok ? c : -1);
                int base = 0;
                if (ok) base = my[c];
                __syncwarp();
                if (ok) {
                    sources[base + __popc(peers & ((1u << lane) - 1u))] = y;
                    if (lane == __ffs(peers) - 1) my[c] = base + __popc(peers);
                }
                __syncwarp();
            }
        }
    }
    __syncwarp();
    if (!FILL && x < ntgt)
        for (int c = lane; c < C; c += 32) counts[(size_t)x * C + c] = my[c];
}

// ---------------------------------------------------------------- plan
// Target expansion of every entry, and a validation of the CSR rows.
__global__ void d_tgt_of_kernel(int nrows, int nnz, int nsrc, const int32_t *__restrict__ offsets,
                                const int32_t *__restrict__ sources, int32_t *__restrict__ row_of,
                                int *__restrict__ status)
{
    const int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (e >= nrows) return;
    const int o0 = offsets[e], o1 = offsets[e + 1];
    if (o0 < 0 || o1 < o0 || o1 > nnz || (e == 0 && o0 != 0) || (e == nrows - 1 && o1 != nnz)) {
        if (lane == 0) atomicOr(status, ST_BAD_INDEX);
        return;
    }
    for (int i = o0 + lane; i < o1; i += 32) {
        row_of[i] = e;
        const int y = sources[i];
        if (y < 0 || y >= nsrc) atomicOr(status, ST_BAD_INDEX);
    }
}

struct DEntry {
    int t[3];
    bool ok;
};

__device__ __forceinline__ DEntry d_entry(int i, int C, const int32_t *__restrict__ row_of,
                                          const int32_t *__restrict__ sources, const int32_t *__restrict__ tgt_ijk,
                                          const int32_t *__restrict__ src_ijk, int nsrc)
{
    DEntry d;
    const int e = row_of[i], y = sources[i];
    d.ok = e >= 0 && y >= 0 && y < nsrc;
    if (!d.ok) return d;
    const int x = e / C;
    for (int a = 0; a < 3; ++a) d.t[a] = tgt_ijk[3 * x + a] - src_ijk[3 * y + a];
    d.ok = max(abs(d.t[0]), max(abs(d.t[1]), abs(d.t[2]))) >= 2;
    return d;
}

// p(t) (|t| sorted descending) and g(t) = 8 perm_id + flip (Eqs. (26)-(27)).
__device__ __forceinline__ void d_canonical(const int t[3], int tp[3], int &g)
{
    const int at[3] = {abs(t[0]), abs(t[1]), abs(t[2])};
    int flip = 0;
    for (int i = 0; i < 3; ++i)
        if (t[i] < 0) flip |= 1 << i;
    int o[3] = {0, 1, 2};
    for (int i = 1; i < 3; ++i)
        for (int q = i; q > 0 && at[o[q]] > at[o[q - 1]]; --q) {
            const int tmp = o[q];
            o[q] = o[q - 1];
            o[q - 1] = tmp;
        }
    const int perm_id = 2 * o[0] + (o[1] > o[2] ? 1 : 0);
    for (int i = 0; i < 3; ++i) tp[i] = at[o[i]];
    g = 8 * perm_id + flip;
}

__global__ void d_tmax_kernel(int nnz, int C, const int32_t *__restrict__ row_of, const int32_t *__restrict__ sources,
                              const int32_t *__restrict__ tgt_ijk, const int32_t *__restrict__ src_ijk, int nsrc,
                              int *__restrict__ tmax, int *__restrict__ status)
{
    int local = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += gridDim.x * blockDim.x) {
        const DEntry d = d_entry(i, C, row_of, sources, tgt_ijk, src_ijk, nsrc);
        if (!d.ok) {
            atomicOr(status, ST_BAD_PAIR);
            continue;
        }
        local = max(local, max(abs(d.t[0]), max(abs(d.t[1]), abs(d.t[2]))));
    }
    for (int o = 16; o > 0; o >>= 1) local = max(local, __shfl_xor_sync(0xffffffffu, local, o));
    if ((threadIdx.x & 31) == 0 && local > 0) atomicMax(tmax, local);
}

__global__ void d_flag_kernel(int nnz, int C, int M, const int32_t *__restrict__ row_of,
                              const int32_t *__restrict__ sources, const int32_t *__restrict__ tgt_ijk,
                              const int32_t *__restrict__ src_ijk, int nsrc, int32_t *__restrict__ flags)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += gridDim.x * blockDim.x) {
        const DEntry d = d_entry(i, C, row_of, sources, tgt_ijk, src_ijk, nsrc);
        if (!d.ok) continue;
        int tp[3], g;
        d_canonical(d.t, tp, g);
        flags[(tp[0] * (M + 1) + tp[1]) * (M + 1) + tp[2]] = 1;
    }
}

__global__ void d_tsym_kernel(int M, const int32_t *__restrict__ flags, const int32_t *__restrict__ pidx,
                              int32_t *__restrict__ tsym)
{
    const int n = (M + 1) * (M + 1) * (M + 1);
    for (int key = blockIdx.x * blockDim.x + threadIdx.x; key < n; key += gridDim.x * blockDim.x) {
        if (!flags[key]) continue;
        const int p = pidx[key];
        tsym[3 * p] = key / ((M + 1) * (M + 1));
        tsym[3 * p + 1] = (key / (M + 1)) % (M + 1);
        tsym[3 * p + 2] = key % (M + 1);
    }
}

// Class of every entry; class histogram.
__global__ void d_classify_kernel(int nnz, int C, int M, const int32_t *__restrict__ row_of,
                                  const int32_t *__restrict__ sources, const int32_t *__restrict__ tgt_ijk,
                                  const int32_t *__restrict__ src_ijk, int nsrc, const int32_t *__restrict__ pidx,
                                  int32_t *__restrict__ code, int32_t *__restrict__ cnt)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += gridDim.x * blockDim.x) {
        const DEntry d = d_entry(i, C, row_of, sources, tgt_ijk, src_ijk, nsrc);
        if (!d.ok) {
            code[i] = -1;
            continue;
        }
        int tp[3], g;
        d_canonical(d.t, tp, g);
        const int p = pidx[(tp[0] * (M + 1) + tp[1]) * (M + 1) + tp[2]];
        code[i] = p | (g << 24);
        atomicAdd(cnt + p, 1);
    }
}

// Buckets by class: {source expansion, target expansion | g << 26}.
__global__ void d_bucket_kernel(int nnz, int C, const int32_t *__restrict__ row_of,
                                const int32_t *__restrict__ sources, const int32_t *__restrict__ code,
                                const int32_t *__restrict__ class_off, int32_t *__restrict__ cursor,
                                int2 *__restrict__ rec)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += gridDim.x * blockDim.x) {
        const int cd = code[i];
        if (cd < 0) continue;
        const int p = cd & 0xFFFFFF, g = cd >> 24;
        const int e = row_of[i];
        const int pos = class_off[p] + atomicAdd(cursor + p, 1);
        rec[pos] = make_int2(sources[i] * C + e % C, rec_pack(e, g));
    }
}

// sigma_g and its inverse, [48][n3] (Eqs. (26)-(29)).
__global__ void d_sigma_kernel(int ell, int16_t *__restrict__ sigma, int16_t *__restrict__ sinv)
{
    const int n3 = ell * ell * ell;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < 48 * n3; idx += gridDim.x * blockDim.x) {
        const int g = idx / n3, j = idx % n3;
        const int flip = g & 7, pid = g >> 3;
        const int ord[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
        int a[3] = {j % ell, (j / ell) % ell, j / (ell * ell)};
        for (int i = 0; i < 3; ++i)
            if ((flip >> i) & 1) a[i] = ell - 1 - a[i];
        const int s = a[ord[pid][0]] + ell * a[ord[pid][1]] + ell * ell * a[ord[pid][2]];
        sigma[idx] = (int16_t)s;
        sinv[g * n3 + s] = (int16_t)j;
    }
}

// K_p[a][b] = exp(i k r) / r, r = |w (t_p + (xi_a - xi_b) / 2)| (Eq. (15)).
__global__ void d_assemble_kernel(int ell, int nsym, double k, double w, const int32_t *__restrict__ tsym,
                                  double2 *__restrict__ K64, float2 *__restrict__ K32)
{
    __shared__ double xi[kMaxEll];
    if (threadIdx.x < ell) xi[threadIdx.x] = -cospi((2.0 * threadIdx.x + 1.0) / (2.0 * ell));
    __syncthreads();
    const int n3 = ell * ell * ell;
    const long long total = (long long)nsym * n3 * n3;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int p = (int)(idx / ((long long)n3 * n3));
        const int rem = (int)(idx % ((long long)n3 * n3));
        const int a = rem / n3, b = rem % n3;
        const int ai[3] = {a % ell, (a / ell) % ell, a / (ell * ell)};
        const int bi[3] = {b % ell, (b / ell) % ell, b / (ell * ell)};
        double r2 = 0.0;
        for (int i = 0; i < 3; ++i) {
            const double d = w * ((double)tsym[3 * p + i] + 0.5 * (xi[ai[i]] - xi[bi[i]]));
            r2 += d * d;
        }
        const double r = sqrt(r2);
        double sn, cs;
        sincos(k * r, &sn, &cs);
        const double2 v = make_double2(cs / r, sn / r);
        K64[idx] = v;
        K32[idx] = make_float2((float)v.x, (float)v.y);
    }
}

// ---------------------------------------------------------------- apply
template <typename T> struct CT;
template <> struct CT<float> { using V = float2; };
template <> struct CT<double> { using V = double2; };

// Tiles of NT interactions of one class: Bs [kpad][NT + 1] gathered multipoles
// (zero rows from n3 to kpad), As [16][MR + 1] a slice of MR = 64 operator
// rows (padded: the slice is written along k), Cs [MR][NT + 1] results.
// (A single 128-row pass for n3 <= 128 was slower: its register footprint
// halves the resident blocks.)
constexpr int kDRows = 64;

__host__ __device__ __forceinline__ int d_kpad(int n3) { return (n3 + 15) / 16 * 16; }

template <typename T>
size_t d_apply_smem(int n3, int NT)
{
    const size_t b = (size_t)d_kpad(n3) * (NT + 1), a = (size_t)16 * (kDRows + 1), c = (size_t)kDRows * (NT + 1);
    return (b + a + c) * sizeof(typename CT<T>::V);
}

template <typename T, int NT>
__global__ void __launch_bounds__(kDThreads)
d_apply_kernel(int n3, int ntiles, const int4 *__restrict__ tiles, const int2 *__restrict__ rec,
               const typename CT<T>::V *__restrict__ K, const int16_t *__restrict__ sigma,
               const int16_t *__restrict__ sinv, const typename CT<T>::V *__restrict__ W, T *__restrict__ F)
{
    using V = typename CT<T>::V;
    constexpr int MR = kDRows;
    constexpr int NJ = NT / 16, NI = MR / 16;
    constexpr int LD = NT + 1, LDA = MR + 1;
    extern __shared__ __align__(16) unsigned char d_smem[];
    const int kpad = d_kpad(n3);
    V *Bs = reinterpret_cast<V *>(d_smem);
    V *As = Bs + (size_t)kpad * LD;
    V *Cs = As + 16 * LDA;
    __shared__ int2 s_rec[NT];
    const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int4 ti = tiles[tile];   // class, first record, count
        __syncthreads();
        if (threadIdx.x < NT) s_rec[threadIdx.x] = threadIdx.x < ti.z ? rec[ti.y + threadIdx.x] : make_int2(0, 0);
        __syncthreads();
        // gather: node b of column j goes to row sigma_g(b)
        for (int idx = threadIdx.x; idx < NT * n3; idx += blockDim.x) {
            const int j = idx / n3, b = idx % n3;
            V v;
            v.x = T(0);
            v.y = T(0);
            int row = b;
            if (j < ti.z) {
                const int2 r = s_rec[j];
                row = sigma[rec_g(r.y) * n3 + b];
                v = W[(size_t)r.x * n3 + b];
            }
            Bs[row * LD + j] = v;
        }
        for (int idx = threadIdx.x; idx < (kpad - n3) * NT; idx += blockDim.x) {
            V z;
            z.x = T(0);
            z.y = T(0);
            Bs[(n3 + idx / NT) * LD + idx % NT] = z;
        }
        __syncthreads();
        const V *Kp = K + (size_t)ti.x * n3 * n3;
        for (int r0 = 0; r0 < n3; r0 += MR) {
            T acc_re[NI][NJ], acc_im[NI][NJ];
#pragma unroll
            for (int i = 0; i < NI; ++i)
#pragma unroll
                for (int q = 0; q < NJ; ++q) acc_re[i][q] = acc_im[i][q] = T(0);
            // the MR x 16 operator slice, MR / 16 elements per thread; the next slice
            // is loaded into registers while the current one is multiplied
            constexpr int kPer = MR * 16 / kDThreads;
            V pre[kPer];
            auto load_slice = [&](int k0) {
#pragma unroll
                for (int u = 0; u < kPer; ++u) {
                    const int idx = threadIdx.x + u * kDThreads;
                    const int i = idx / 16, kk = idx % 16;
                    pre[u].x = T(0);
                    pre[u].y = T(0);
                    if (r0 + i < n3 && k0 + kk < n3) pre[u] = Kp[(size_t)(r0 + i) * n3 + k0 + kk];
                }
            };
            load_slice(0);
            for (int k0 = 0; k0 < n3; k0 += 16) {
#pragma unroll
                for (int u = 0; u < kPer; ++u) {
                    const int idx = threadIdx.x + u * kDThreads;
                    As[(idx % 16) * LDA + idx / 16] = pre[u];
                }
                __syncthreads();
                if (k0 + 16 < n3) load_slice(k0 + 16);
#pragma unroll
                for (int kk = 0; kk < 16; ++kk) {   // rows k0 + kk >= n3 of Bs hold zeros
                    V a[NI], b[NJ];
#pragma unroll
                    for (int i = 0; i < NI; ++i) a[i] = As[kk * LDA + tr + 16 * i];
#pragma unroll
                    for (int q = 0; q < NJ; ++q) b[q] = Bs[(k0 + kk) * LD + tc + 16 * q];
#pragma unroll
                    for (int i = 0; i < NI; ++i)
#pragma unroll
                        for (int q = 0; q < NJ; ++q) {
                            acc_re[i][q] += a[i].x * b[q].x - a[i].y * b[q].y;
                            acc_im[i][q] += a[i].x * b[q].y + a[i].y * b[q].x;
                        }
                }
                __syncthreads();
            }
#pragma unroll
            for (int i = 0; i < NI; ++i)
#pragma unroll
                for (int q = 0; q < NJ; ++q) {
                    V v;
                    v.x = acc_re[i][q];
                    v.y = acc_im[i][q];
                    Cs[(tr + 16 * i) * LD + tc + 16 * q] = v;
                }
            __syncthreads();
            // row i of the class product is node sigma_g^-1(i) of the target
            for (int idx = threadIdx.x; idx < MR * NT; idx += blockDim.x) {
                const int j = idx / MR, i = idx % MR;
                if (j < ti.z && r0 + i < n3) {
                    const int2 r = s_rec[j];
                    const int a = sinv[rec_g(r.y) * n3 + r0 + i];
                    T *dst = F + 2 * ((size_t)rec_tgt(r.y) * n3 + a);
                    const V v = Cs[i * LD + j];
                    atomicAdd(dst, v.x);
                    atomicAdd(dst + 1, v.y);
                }
            }
            __syncthreads();
        }
    }
}

// The complex product as a real one of twice the size: rows and columns
// [0, n3) hold real parts, [n3, 2 n3) imaginary parts,
// Kr = [[Re K, -Im K], [Im K, Re K]] (row-major [nsym][2 n3][2 n3]).
__global__ void d_embed_kernel(int n3, int nsym, const double2 *__restrict__ K, double *__restrict__ Kr)
{
    const int N = 2 * n3;
    const long long total = (long long)nsym * N * N;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int p = (int)(idx / ((long long)N * N));
        const int i = (int)((idx / N) % N), j = (int)(idx % N);
        const double2 v = K[((size_t)p * n3 + i % n3) * n3 + j % n3];
        double x;
        if ((i < n3) == (j < n3)) x = v.x;
        else x = (i < n3) ? -v.y : v.y;
        Kr[idx] = x;
    }
}

// tau_g^-1 over the stacked real vector, as indices into the interleaved complex
// one: row k < n3 reads Re w[sigma_g^-1(k)] (2 s), row n3 + k reads its Im
// (2 s + 1); padding rows read element 0 (their operator columns are zero).
__global__ void d_tinv_kernel(int n3, int kpad, const int16_t *__restrict__ sinv, int16_t *__restrict__ tinv)
{
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < 48 * kpad; idx += gridDim.x * blockDim.x) {
        const int g = idx / kpad, k = idx % kpad;
        int v = 0;
        if (k < n3) v = 2 * sinv[g * n3 + k];
        else if (k < 2 * n3) v = 2 * sinv[g * n3 + k - n3] + 1;
        tinv[idx] = (int16_t)v;
    }
}

int d_grid(long n)
{
    long b = (n + 255) / 256;
    return (int)(b > 4096 ? 4096 : (b < 1 ? 1 : b));
}

}  // namespace
}  // namespace m2l

using namespace m2l;

struct m2l_dplan {
    int ell = 0, n3 = 0, C = 0, ntgt = 0, nsrc = 0, nnz = 0, nsym = 0, level = 0;
    double k = 0.0, w = 0.0;
    std::vector<int32_t> tsym;       // [nsym][3], lexicographic
    std::vector<int64_t> np;         // interactions per class
    m2l::DevBuf K64, K32, sigma, sinv, rec, tiles32, tiles64, status, class_off;
    int ntiles32 = 0, ntiles64 = 0, nt32 = 64, nt64 = 32;
    struct Tc {                      // tensor-core layout of one precision (built on first use)
        m2l::DevBuf img, tinv, tstart;
        bool ready = false;
    } tc[3];                         // M2L_TF32, M2L_BF16X3, M2L_TF32X3
};

namespace {

void dplan_release(m2l_dplan *p)
{
    if (!p) return;
    cudaDeviceSynchronize();
    DevBuf *bs[] = {&p->K64,     &p->K32,        &p->sigma,      &p->sinv,      &p->rec,       &p->tiles32,
                    &p->tiles64, &p->status,     &p->class_off,  &p->tc[0].img, &p->tc[0].tinv, &p->tc[0].tstart,
                    &p->tc[1].img, &p->tc[1].tinv, &p->tc[1].tstart, &p->tc[2].img, &p->tc[2].tinv,
                    &p->tc[2].tstart};
    for (DevBuf *b : bs) b->release();
    delete p;
}

// Widest tile that fits shared memory.
int pick_nt(int n3, size_t esz2)
{
    for (int nt : {64, 32, 16}) {
        const size_t smem = ((size_t)d_kpad(n3) * (nt + 1) + 16 * (kDRows + 1) + kDRows * (nt + 1)) * esz2;
        if ((int)smem + 1024 <= max_smem_optin()) return nt;   // + the static tile records
    }
    return 0;
}

std::vector<int4> make_tiles(const std::vector<int64_t> &np, int nt)
{
    std::vector<int4> t;
    int64_t start = 0;
    for (size_t p = 0; p < np.size(); ++p) {
        for (int64_t s = 0; s < np[p]; s += nt)
            t.push_back(make_int4((int)p, (int)(start + s), (int)std::min<int64_t>(nt, np[p] - s), 0));
        start += np[p];
    }
    return t;
}

template <typename T, int NT>
m2l_status d_launch(const m2l_dplan *p, const DevBuf &tiles, int ntiles, const void *W, void *F, cudaStream_t s)
{
    using V = typename CT<T>::V;
    const size_t smem = d_apply_smem<T>(p->n3, NT);
    auto kern = d_apply_kernel<T, NT>;
    M2L_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    M2L_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kDThreads, smem));
    if (per_sm < 1) per_sm = 1;
    const int grid = (int)std::min<long>((long)num_sms() * per_sm, ntiles);
    const V *K = static_cast<const V *>(sizeof(T) == 8 ? p->K64.p : p->K32.p);
    kern<<<grid, kDThreads, smem, s>>>(p->n3, ntiles, tiles.as<int4>(), p->rec.as<int2>(), K, p->sigma.as<int16_t>(),
                                       p->sinv.as<int16_t>(), static_cast<const V *>(W), static_cast<T *>(F));
    M2L_LAUNCH_CHECK("d_apply_kernel");
    return M2L_OK;
}

template <typename T>
m2l_status d_dispatch(const m2l_dplan *p, int nt, const DevBuf &tiles, int ntiles, const void *W, void *F,
                      cudaStream_t s)
{
    if (nt == 64) return d_launch<T, 64>(p, tiles, ntiles, W, F, s);
    if (nt == 32) return d_launch<T, 32>(p, tiles, ntiles, W, F, s);
    if (nt == 16) return d_launch<T, 16>(p, tiles, ntiles, W, F, s);
    set_error("order %d does not fit the directional apply's shared memory", p->ell);
    return M2L_EUNSUPPORTED;
}

}  // namespace

extern "C" {

m2l_status m2l_dfmm_build_lists(int level, double wavenumber, double domain_width, int ncells_tgt,
                                const int32_t *tgt_ijk, int ncells_src, const int32_t *src_ijk, int *n_cones,
                                int32_t *il_offsets, int32_t *il_sources, int64_t *nnz_out, void *stream)
{
    if (level < 0 || level > 8 || !(wavenumber >= 0.0) || !(domain_width > 0.0) || ncells_tgt < 0 ||
        ncells_src < 0 || !n_cones || !nnz_out || (ncells_tgt > 0 && !tgt_ijk) || (ncells_src > 0 && !src_ijk)) {
        set_error("bad directional list-builder arguments");
        return M2L_EINVAL;
    }
    const double w = d_width(domain_width, level);
    const int m = d_cone_m(wavenumber, w);
    if (m > kDMaxM) {
        set_error("k w = %g needs %d squares per cone face edge (at most %d)", wavenumber * w, m, kDMaxM);
        return M2L_EUNSUPPORTED;
    }
    const int C = m ? 6 * m * m : 1;
    *n_cones = C;
    *nnz_out = 0;
    if (!il_offsets) return M2L_OK;   // sizing call
    const int R = 2 * (int)ceil(std::max(2.0, 2.0 * wavenumber * w)) + 1;
    const int side = 1 << level;
    cudaStream_t s = (cudaStream_t)stream;
    DevBuf table, cnt, bad;
    ScratchGuard guard{&table, &cnt, &bad};
    m2l_status st;
    const size_t cells = (size_t)side * side * side;
    const size_t rows = (size_t)ncells_tgt * C;
    if ((st = table.ensure(cells * sizeof(int32_t))) != M2L_OK) return st;
    if ((st = cnt.ensure((rows + 1) * sizeof(int32_t))) != M2L_OK) return st;
    if ((st = bad.ensure(sizeof(int))) != M2L_OK) return st;
    M2L_CUDA(cudaMemsetAsync(table.p, 0xFF, cells * sizeof(int32_t), s));
    M2L_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), s));
    if (ncells_src > 0) {
        d_scatter_cells_kernel<<<(ncells_src + 255) / 256, 256, 0, s>>>(ncells_src, src_ijk, side, table.as<int32_t>(),
                                                                       bad.as<int>());
        M2L_LAUNCH_CHECK("d_scatter_cells_kernel");
    }
    if (ncells_tgt > 0) {
        d_check_cells_kernel<<<(ncells_tgt + 255) / 256, 256, 0, s>>>(ncells_tgt, tgt_ijk, side, bad.as<int>());
        M2L_LAUNCH_CHECK("d_check_cells_kernel");
    }
    int hbad = 0;
    M2L_CUDA(cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    M2L_CUDA(cudaStreamSynchronize(s));
    if (hbad) {
        set_error(hbad & 1 ? "cell coordinates outside the level's grid" : "duplicate source cells");
        return M2L_EINVAL;
    }
    if (ncells_tgt == 0) {
        M2L_CUDA(cudaMemsetAsync(il_offsets, 0, sizeof(int32_t), s));
        M2L_CUDA(cudaStreamSynchronize(s));
        return M2L_OK;
    }
    const size_t smem = (size_t)kDListWarps * C * sizeof(int);
    const int blocks = (ncells_tgt + kDListWarps - 1) / kDListWarps;
    if (smem > 48 * 1024) {
        M2L_CUDA(cudaFuncSetAttribute(d_lists_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        M2L_CUDA(cudaFuncSetAttribute(d_lists_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    d_lists_kernel<false><<<blocks, kDListWarps * 32, smem, s>>>(level, wavenumber, domain_width, R, C, m, ncells_tgt,
                                                                 tgt_ijk, side, table.as<int32_t>(), cnt.as<int32_t>(),
                                                                 nullptr, nullptr);
    M2L_LAUNCH_CHECK("d_lists_kernel(count)");
    if ((st = launch_exclusive_scan(cnt.as<int32_t>(), il_offsets, (int)rows, s)) != M2L_OK) return st;
    int total = 0;
    M2L_CUDA(cudaMemcpyAsync(&total, il_offsets + rows, sizeof(int), cudaMemcpyDeviceToHost, s));
    M2L_CUDA(cudaStreamSynchronize(s));
    *nnz_out = total;
    if (il_sources && total > 0) {
        d_lists_kernel<true><<<blocks, kDListWarps * 32, smem, s>>>(level, wavenumber, domain_width, R, C, m,
                                                                    ncells_tgt, tgt_ijk, side, table.as<int32_t>(),
                                                                    nullptr, il_offsets, il_sources);
        M2L_LAUNCH_CHECK("d_lists_kernel(fill)");
        M2L_CUDA(cudaStreamSynchronize(s));
    }
    return M2L_OK;
}

m2l_status m2l_dfmm_plan_create(int ell, double wavenumber, const m2l_dlevel *lv, void *stream, m2l_dplan **out)
{
    if (!out || !lv || ell < 2 || ell > kMaxEll || !(wavenumber >= 0.0) || !(lv->width > 0.0) ||
        lv->ncells_tgt < 0 || lv->ncells_src < 0 || lv->n_cones < 1 || lv->nnz < 0 ||
        (long long)lv->ncells_tgt * lv->n_cones >= (1LL << kTgtBits) ||
        (long long)lv->ncells_src * lv->n_cones >= (1LL << 31) ||
        (lv->ncells_tgt > 0 && (!lv->tgt_ijk || !lv->il_offsets)) ||
        (lv->nnz > 0 && (!lv->il_sources || !lv->src_ijk))) {
        set_error("bad directional plan arguments");
        return M2L_EINVAL;
    }
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    m2l_dplan *p = new m2l_dplan();
    p->ell = ell;
    p->n3 = ell * ell * ell;
    p->C = lv->n_cones;
    p->ntgt = lv->ncells_tgt;
    p->nsrc = lv->ncells_src;
    p->nnz = lv->nnz;
    p->level = lv->level;
    p->k = wavenumber;
    p->w = lv->width;
    DevBuf row_of, tmax, flags, pidx, code, cnt, cursor, tsym;
    ScratchGuard guard{&row_of, &tmax, &flags, &pidx, &code, &cnt, &cursor, &tsym};
    DevBuf &coff = p->class_off;
    m2l_status st = M2L_OK;
    auto fail = [&](m2l_status e) { dplan_release(p); return e; };
    const int nnz = lv->nnz, C = p->C, n3 = p->n3;
    const int nrows = p->ntgt * C;
    if ((st = p->status.ensure(sizeof(int))) != M2L_OK) return fail(st);
    if (cudaMemsetAsync(p->status.p, 0, sizeof(int), s) != cudaSuccess) return fail(cuda_fail(cudaGetLastError(), "memset"));
    int M = 0;
    if (nnz > 0 && nrows == 0) {
        set_error("list entries without target expansions");
        return fail(M2L_EINVAL);
    }
    if (nnz > 0) {
        if ((st = row_of.ensure((size_t)nnz * sizeof(int32_t))) != M2L_OK) return fail(st);
        if ((st = tmax.ensure(sizeof(int))) != M2L_OK) return fail(st);
        if (cudaMemsetAsync(row_of.p, 0xFF, (size_t)nnz * sizeof(int32_t), s) != cudaSuccess ||
            cudaMemsetAsync(tmax.p, 0, sizeof(int), s) != cudaSuccess)
            return fail(cuda_fail(cudaGetLastError(), "memset"));
        d_tgt_of_kernel<<<(int)(((long)nrows * 32 + 255) / 256), 256, 0, s>>>(nrows, nnz, p->nsrc, lv->il_offsets,
                                                                           lv->il_sources, row_of.as<int32_t>(),
                                                                           p->status.as<int>());
        d_tmax_kernel<<<d_grid(nnz), 256, 0, s>>>(nnz, C, row_of.as<int32_t>(), lv->il_sources, lv->tgt_ijk,
                                                 lv->src_ijk, p->nsrc, tmax.as<int>(), p->status.as<int>());
        count_launch(2);
        int hst = 0;
        if (cudaMemcpyAsync(&M, tmax.p, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(&hst, p->status.p, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return fail(cuda_fail(cudaGetLastError(), "directional classification"));
        if (hst) {
            set_error("directional list rejected (status 0x%x): %s", hst,
                      (hst & ST_BAD_INDEX) ? "offsets or indices out of range" : "entries with |t|_inf < 2");
            return fail(M2L_EINVAL);
        }
        const size_t nkey = (size_t)(M + 1) * (M + 1) * (M + 1);
        if ((st = flags.ensure((nkey + 1) * sizeof(int32_t))) != M2L_OK) return fail(st);
        if ((st = pidx.ensure((nkey + 1) * sizeof(int32_t))) != M2L_OK) return fail(st);
        if (cudaMemsetAsync(flags.p, 0, (nkey + 1) * sizeof(int32_t), s) != cudaSuccess)
            return fail(cuda_fail(cudaGetLastError(), "memset"));
        d_flag_kernel<<<d_grid(nnz), 256, 0, s>>>(nnz, C, M, row_of.as<int32_t>(), lv->il_sources, lv->tgt_ijk,
                                                 lv->src_ijk, p->nsrc, flags.as<int32_t>());
        count_launch();
        if ((st = launch_exclusive_scan(flags.as<int32_t>(), pidx.as<int32_t>(), (int)nkey, s)) != M2L_OK)
            return fail(st);
        int nsym = 0;
        if (cudaMemcpyAsync(&nsym, pidx.as<int32_t>() + nkey, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return fail(cuda_fail(cudaGetLastError(), "T_sym"));
        p->nsym = nsym;
        if ((st = tsym.ensure((size_t)3 * nsym * sizeof(int32_t))) != M2L_OK) return fail(st);
        if ((st = code.ensure((size_t)nnz * sizeof(int32_t))) != M2L_OK) return fail(st);
        if ((st = cnt.ensure((size_t)nsym * sizeof(int32_t))) != M2L_OK) return fail(st);
        if ((st = cursor.ensure((size_t)nsym * sizeof(int32_t))) != M2L_OK) return fail(st);
        if ((st = coff.ensure((size_t)(nsym + 1) * sizeof(int32_t))) != M2L_OK) return fail(st);
        if ((st = p->rec.ensure((size_t)nnz * sizeof(int2))) != M2L_OK) return fail(st);
        if (cudaMemsetAsync(cnt.p, 0, (size_t)nsym * sizeof(int32_t), s) != cudaSuccess ||
            cudaMemsetAsync(cursor.p, 0, (size_t)nsym * sizeof(int32_t), s) != cudaSuccess)
            return fail(cuda_fail(cudaGetLastError(), "memset"));
        d_tsym_kernel<<<d_grid((long)nkey), 256, 0, s>>>(M, flags.as<int32_t>(), pidx.as<int32_t>(), tsym.as<int32_t>());
        d_classify_kernel<<<d_grid(nnz), 256, 0, s>>>(nnz, C, M, row_of.as<int32_t>(), lv->il_sources, lv->tgt_ijk,
                                                     lv->src_ijk, p->nsrc, pidx.as<int32_t>(), code.as<int32_t>(),
                                                     cnt.as<int32_t>());
        count_launch(2);
        std::vector<int32_t> hcnt(nsym);
        p->tsym.resize((size_t)3 * nsym);
        if (cudaMemcpyAsync(hcnt.data(), cnt.p, (size_t)nsym * sizeof(int32_t), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaMemcpyAsync(p->tsym.data(), tsym.p, (size_t)3 * nsym * sizeof(int32_t), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return fail(cuda_fail(cudaGetLastError(), "class counts"));
        std::vector<int32_t> hoff(nsym + 1, 0);
        p->np.assign(nsym, 0);
        for (int q = 0; q < nsym; ++q) {
            hoff[q + 1] = hoff[q] + hcnt[q];
            p->np[q] = hcnt[q];
        }
        if (cudaMemcpyAsync(coff.p, hoff.data(), (size_t)(nsym + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
            return fail(cuda_fail(cudaGetLastError(), "class offsets"));
        d_bucket_kernel<<<d_grid(nnz), 256, 0, s>>>(nnz, C, row_of.as<int32_t>(), lv->il_sources, code.as<int32_t>(),
                                                   coff.as<int32_t>(), cursor.as<int32_t>(), p->rec.as<int2>());
        count_launch();
    }
    // tables and operators
    if ((st = p->sigma.ensure((size_t)48 * n3 * sizeof(int16_t))) != M2L_OK) return fail(st);
    if ((st = p->sinv.ensure((size_t)48 * n3 * sizeof(int16_t))) != M2L_OK) return fail(st);
    d_sigma_kernel<<<d_grid(48L * n3), 256, 0, s>>>(ell, p->sigma.as<int16_t>(), p->sinv.as<int16_t>());
    count_launch();
    const size_t nk = (size_t)std::max(p->nsym, 1) * n3 * n3;
    if ((st = p->K64.ensure(nk * sizeof(double2))) != M2L_OK) return fail(st);
    if ((st = p->K32.ensure(nk * sizeof(float2))) != M2L_OK) return fail(st);
    if (p->nsym > 0) {
        d_assemble_kernel<<<d_grid((long)(p->nsym) * n3 * n3), 256, 0, s>>>(ell, p->nsym, wavenumber, lv->width,
                                                                            tsym.as<int32_t>(), p->K64.as<double2>(),
                                                                            p->K32.as<float2>());
        count_launch();
    }
    // tiles for the two element sizes
    p->nt32 = pick_nt(n3, sizeof(float2));
    p->nt64 = pick_nt(n3, sizeof(double2));
    for (int fp64 = 0; fp64 < 2; ++fp64) {
        const int nt = fp64 ? p->nt64 : p->nt32;
        std::vector<int4> t = nt ? make_tiles(p->np, nt) : std::vector<int4>();
        DevBuf &tb = fp64 ? p->tiles64 : p->tiles32;
        (fp64 ? p->ntiles64 : p->ntiles32) = (int)t.size();
        if ((st = tb.ensure(std::max<size_t>(t.size(), 1) * sizeof(int4))) != M2L_OK) return fail(st);
        if (!t.empty() &&
            cudaMemcpyAsync(tb.p, t.data(), t.size() * sizeof(int4), cudaMemcpyHostToDevice, s) != cudaSuccess)
            return fail(cuda_fail(cudaGetLastError(), "tiles"));
    }
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return fail(cuda_fail(cudaGetLastError(), "directional plan"));
    *out = p;
    return M2L_OK;
}

m2l_status m2l_dfmm_plan_info(const m2l_dplan *p, int *nsym, int *n_cones, int64_t *nnz, int32_t *host_tsym,
                              int64_t *host_np)
{
    if (!p) { set_error("null directional plan"); return M2L_EINVAL; }
    if (nsym) *nsym = p->nsym;
    if (n_cones) *n_cones = p->C;
    if (nnz) *nnz = p->nnz;
    if (host_tsym) std::copy(p->tsym.begin(), p->tsym.end(), host_tsym);
    if (host_np) std::copy(p->np.begin(), p->np.end(), host_np);
    return M2L_OK;
}

m2l_status m2l_dfmm_plan_prepare(m2l_dplan *p, int precision, void *stream)
{
    if (!p) { set_error("null directional plan"); return M2L_EINVAL; }
    if (precision == M2L_FP64 || precision == M2L_FP32) return M2L_OK;
    const int ti = precision == M2L_TF32 ? 0 : precision == M2L_BF16X3 ? 1 : precision == M2L_TF32X3 ? 2 : -1;
    if (ti < 0) { set_error("unknown precision %d", precision); return M2L_EINVAL; }
    m2l_dplan::Tc &L = p->tc[ti];
    if (L.ready) return M2L_OK;
    const int n3 = p->n3, N = 2 * n3, nsym = std::max(p->nsym, 1);
    int kpad = 0, tcols = 0;
    size_t per_op = 0;
    if (!tc_general_config(precision, N, &kpad, &per_op, &tcols)) {
        set_error("the directional tensor-core apply takes ell <= 5 (ell = %d)", p->ell);
        return M2L_EUNSUPPORTED;
    }
    cudaStream_t s = (cudaStream_t)stream;
    DevBuf Kr;
    ScratchGuard guard{&Kr};
    m2l_status st;
    if ((st = Kr.ensure((size_t)nsym * N * N * sizeof(double))) != M2L_OK) return st;
    if ((st = L.img.ensure((size_t)nsym * per_op)) != M2L_OK) return st;
    if ((st = L.tinv.ensure((size_t)48 * kpad * sizeof(int16_t))) != M2L_OK) return st;
    if ((st = L.tstart.ensure((size_t)(nsym + 1) * sizeof(int32_t))) != M2L_OK) return st;
    if (p->nsym > 0) {
        d_embed_kernel<<<d_grid((long)p->nsym * N * N), 256, 0, s>>>(n3, p->nsym, p->K64.as<double2>(), Kr.as<double>());
        M2L_LAUNCH_CHECK("d_embed_kernel");
        if ((st = tc_general_images(precision, N, p->nsym, Kr.as<double>(), L.img.as<uint8_t>(), s)) != M2L_OK)
            return st;
    }
    d_tinv_kernel<<<d_grid(48L * kpad), 256, 0, s>>>(n3, kpad, p->sinv.as<int16_t>(), L.tinv.as<int16_t>());
    M2L_LAUNCH_CHECK("d_tinv_kernel");
    std::vector<int32_t> ts(p->nsym + 1, 0);   // tiles of tcols interactions per class
    for (int q = 0; q < p->nsym; ++q) ts[q + 1] = ts[q] + (int)((p->np[q] + tcols - 1) / tcols);
    M2L_CUDA(cudaMemcpyAsync(L.tstart.p, ts.data(), ts.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    M2L_CUDA(cudaStreamSynchronize(s));
    L.ready = true;
    return M2L_OK;
}

m2l_status m2l_dfmm_plan_sync(const m2l_dplan *p, void *stream)
{
    if (!p) { set_error("null directional plan"); return M2L_EINVAL; }
    M2L_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    int st = 0;
    M2L_CUDA(cudaMemcpy(&st, p->status.p, sizeof(int), cudaMemcpyDeviceToHost));
    M2L_CUDA(cudaMemset(p->status.p, 0, sizeof(int)));
    if (st & ST_TIMEOUT) { set_error("a bounded device wait timed out"); return M2L_ETIMEOUT; }
    if (st) { set_error("directional apply status 0x%x", st); return M2L_EINVAL; }
    return M2L_OK;
}

m2l_status m2l_dfmm_plan_apply(const m2l_dplan *p, const void *multipoles, void *locals, int precision,
                               void *stream)
{
    if (!p) { set_error("null directional plan"); return M2L_EINVAL; }
    if (p->nnz == 0) return M2L_OK;
    if (!multipoles || !locals) { set_error("null multipoles or locals"); return M2L_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == M2L_FP64) return d_dispatch<double>(p, p->nt64, p->tiles64, p->ntiles64, multipoles, locals, s);
    if (precision == M2L_FP32) return d_dispatch<float>(p, p->nt32, p->tiles32, p->ntiles32, multipoles, locals, s);
    if (precision == M2L_TF32 || precision == M2L_BF16X3 || precision == M2L_TF32X3) {
        m2l_status st = m2l_dfmm_plan_prepare(const_cast<m2l_dplan *>(p), precision, stream);
        if (st != M2L_OK) return st;
        const m2l_dplan::Tc &L = p->tc[precision == M2L_TF32 ? 0 : precision == M2L_BF16X3 ? 1 : 2];
        return tc_general_apply(precision, 2 * p->n3, p->nsym, L.tstart.as<int>(), p->rec.as<int2>(),
                                p->class_off.as<int>(), L.img.as<uint8_t>(), L.tinv.as<int16_t>(), p->nnz,
                                static_cast<const float *>(multipoles), static_cast<float *>(locals),
                                p->status.as<int>(), s);
    }
    set_error("unknown precision %d", precision);
    return M2L_EINVAL;
}

void m2l_dfmm_plan_free(m2l_dplan *p) { dplan_release(p); }

}  // extern "C"
