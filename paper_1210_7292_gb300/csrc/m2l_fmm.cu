// The bbFMM matvec around the M2L translation (Sec. 2.1.1, Eqs. (5)-(8)):
// P2M at the leaves, M2M up to level 2, the symmetry-blocked M2L at every
// level (through per-level plans), L2L down to the leaves, then L2P plus the
// direct near field over the <= 27 neighbour leaves (Sec. 3.2).
//
// Uniform-depth octree on [lo, lo + width)^3 with empty cells pruned; the
// cells of every level are kept sorted by linear index (x fastest), with a
// dense lookup table per level.  Interpolation (Eq. (3)) uses the Lagrange
// basis on the ell Chebyshev roots; the child-parent transfers of M2M and L2L
// are tensor products of two ell x ell one-dimensional matrices (one per
// child side) and are applied as three one-axis contractions per child.
#include <math.h>

#include <vector>

#include "m2l_internal.cuh"

namespace m2l {
namespace {

constexpr int kFmmThreads = 128;
constexpr int kMaxN3 = 512;   // ell <= 8

// Lagrange basis of the ell roots at reference coordinate x.
template <typename T>
__device__ __forceinline__ void lagrange(int ell, T x, const T *__restrict__ xi, const T *__restrict__ inv_den, T *L)
{
    for (int k = 0; k < ell; ++k) {
        T v = inv_den[k];
        for (int j = 0; j < ell; ++j)
            if (j != k) v *= (x - xi[j]);
        L[k] = v;
    }
}

template <typename T>
__device__ __forceinline__ T kernel_of_r2(int kind, T c, T r2)
{
    if (kind == M2L_K_INV_R) return T(1) / sqrt(r2);
    if (kind == M2L_K_INV_R4) return T(1) / (r2 * r2);
    return T(1) / sqrt(r2 + c * c);
}

// FP32: the hardware reciprocal square root (within a few ulp, far below the
// FMM's own error) instead of a division by a square root.
template <>
__device__ __forceinline__ float kernel_of_r2<float>(int kind, float c, float r2)
{
    if (kind == M2L_K_INV_R) return rsqrtf(r2);
    if (kind == M2L_K_INV_R4) {
        const float r = rsqrtf(r2);
        const float r2i = r * r;
        return r2i * r2i;
    }
    return rsqrtf(r2 + c * c);
}

constexpr int kP2PThreads = 64;     // targets per pass of a near-field block
constexpr int kP2PChunk = 512;      // sources staged per chunk

// Leaf cell of every particle (binned in double, as the cells are half-open
// with the top face clamped) and the particle count per dense leaf cell.
template <typename T>
__global__ void bin_count_kernel(int n, const T *__restrict__ xyz, double lo, double w, int side,
                                 int32_t *__restrict__ lin, int32_t *__restrict__ cnt)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int c[3];
        for (int d = 0; d < 3; ++d) {
            const int v = (int)floor(((double)xyz[3 * i + d] - lo) / w);
            c[d] = min(max(v, 0), side - 1);
        }
        const int l = c[0] + side * (c[1] + side * c[2]);
        lin[i] = l;
        atomicAdd(cnt + l, 1);
    }
}

__global__ void bin_scatter_kernel(int n, const int32_t *__restrict__ lin, const int32_t *__restrict__ start,
                                   int32_t *__restrict__ cursor, int32_t *__restrict__ perm)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int l = lin[i];
        perm[start[l] + atomicAdd(cursor + l, 1)] = i;
    }
}

__global__ void leaf_flags_kernel(int ncells, const int32_t *__restrict__ cnt, int32_t *__restrict__ flag)
{
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < ncells; l += gridDim.x * blockDim.x)
        flag[l] = cnt[l] > 0 ? 1 : 0;
}

// A parent is kept when one of its children is.
__global__ void parent_flags_kernel(int child_side, const int32_t *__restrict__ child_flag,
                                    int32_t *__restrict__ parent_flag)
{
    const int ncells = child_side * child_side * child_side, ps = child_side / 2;
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < ncells; l += gridDim.x * blockDim.x) {
        if (!child_flag[l]) continue;
        const int i = l % child_side, j = (l / child_side) % child_side, k = l / (child_side * child_side);
        parent_flag[(i >> 1) + ps * ((j >> 1) + ps * (k >> 1))] = 1;
    }
}

// Kept cells in linear order: coordinates and the dense lookup table.
__global__ void compact_kernel(int side, const int32_t *__restrict__ flag, const int32_t *__restrict__ pos,
                               int32_t *__restrict__ ijk, int32_t *__restrict__ lookup)
{
    const int ncells = side * side * side;
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < ncells; l += gridDim.x * blockDim.x) {
        if (flag[l]) {
            const int id = pos[l];
            ijk[3 * id] = l % side;
            ijk[3 * id + 1] = (l / side) % side;
            ijk[3 * id + 2] = l / (side * side);
            lookup[l] = id;
        } else {
            lookup[l] = -1;
        }
    }
}

// P2M, Eq. (6): W_beta = sum_j S(y_j, ybar_beta) q_j, one block per leaf.
template <typename T>
__global__ void __launch_bounds__(kFmmThreads)
p2m_kernel(int ell, int ncells, const int32_t *__restrict__ ijk, int side, const int32_t *__restrict__ start,
           const int32_t *__restrict__ perm, const T *__restrict__ xyz, const T *__restrict__ q, double lo, double w,
           const T *__restrict__ xi, const T *__restrict__ inv_den, T *__restrict__ W)
{
    __shared__ T sL[32][3][8];
    __shared__ T sq[32];
    const int cid = blockIdx.x;
    if (cid >= ncells) return;
    const int n3 = ell * ell * ell;
    const int ci = ijk[3 * cid], cj = ijk[3 * cid + 1], ck = ijk[3 * cid + 2];
    const int l = ci + side * (cj + side * ck);
    const int j0 = start[l], j1 = start[l + 1];
    const T ctr[3] = {T(lo + w * (ci + 0.5)), T(lo + w * (cj + 0.5)), T(lo + w * (ck + 0.5))};
    const T half = T(0.5 * w);
    T acc[kMaxN3 / kFmmThreads];
#pragma unroll
    for (int r = 0; r < kMaxN3 / kFmmThreads; ++r) acc[r] = T(0);
    for (int base = j0; base < j1; base += 32) {
        __syncthreads();
        if (threadIdx.x < 32) {
            const int jj = base + threadIdx.x;
            if (jj < j1) {
                const int p = perm[jj];
                for (int d = 0; d < 3; ++d) lagrange(ell, (xyz[3 * p + d] - ctr[d]) / half, xi, inv_den, sL[threadIdx.x][d]);
                sq[threadIdx.x] = q[p];
            } else {
                sq[threadIdx.x] = T(0);
                for (int d = 0; d < 3; ++d)
                    for (int k = 0; k < ell; ++k) sL[threadIdx.x][d][k] = T(0);
            }
        }
        __syncthreads();
        const int nj = min(32, j1 - base);
#pragma unroll
        for (int r = 0; r < kMaxN3 / kFmmThreads; ++r) {
            const int b = threadIdx.x + kFmmThreads * r;
            if (b >= n3) break;
            const int b0 = b % ell, b1 = (b / ell) % ell, b2 = b / (ell * ell);
            T s = acc[r];
            for (int jj = 0; jj < nj; ++jj) s += sL[jj][0][b0] * sL[jj][1][b1] * sL[jj][2][b2] * sq[jj];
            acc[r] = s;
        }
    }
#pragma unroll
    for (int r = 0; r < kMaxN3 / kFmmThreads; ++r) {
        const int b = threadIdx.x + kFmmThreads * r;
        if (b < n3) W[(size_t)cid * n3 + b] = acc[r];
    }
}

// One axis of a child-parent transfer on a tensor in shared memory:
// out[.., a_axis, ..] = sum_k in[.., k, ..] * M[k][a_axis] (up = true, M2M)
// or sum_k in[.., k, ..] * M[a_axis][k] (up = false, L2L).
template <typename T>
__device__ __forceinline__ void contract_axis(int ell, int axis, const T *in, T *out, const T *M, bool up)
{
    const int n3 = ell * ell * ell;
    const int stride = axis == 0 ? 1 : (axis == 1 ? ell : ell * ell);
    for (int idx = threadIdx.x; idx < n3; idx += blockDim.x) {
        const int a = (idx / stride) % ell;
        const int base = idx - a * stride;
        T s = T(0);
        for (int k = 0; k < ell; ++k) s += in[base + k * stride] * (up ? M[k * ell + a] : M[a * ell + k]);
        out[idx] = s;
    }
}

// M2M, Eq. (6) with the children's nodes as the particles: one block per parent.
template <typename T>
__global__ void __launch_bounds__(kFmmThreads)
m2m_kernel(int ell, int ncells, const int32_t *__restrict__ ijk, int child_side, const int32_t *__restrict__ child_lookup,
           const T *__restrict__ Wc, const T *__restrict__ M2, T *__restrict__ Wp)
{
    __shared__ T sW[kMaxN3], sA[kMaxN3], sB[kMaxN3], sOut[kMaxN3];
    __shared__ T sM[2][64];
    const int pid = blockIdx.x;
    if (pid >= ncells) return;
    const int n3 = ell * ell * ell;
    for (int i = threadIdx.x; i < 2 * ell * ell; i += blockDim.x) sM[i / (ell * ell)][i % (ell * ell)] = M2[i];
    for (int i = threadIdx.x; i < n3; i += blockDim.x) sOut[i] = T(0);
    const int pi = ijk[3 * pid], pj = ijk[3 * pid + 1], pk = ijk[3 * pid + 2];
    for (int o = 0; o < 8; ++o) {
        const int s0 = o & 1, s1 = (o >> 1) & 1, s2 = (o >> 2) & 1;
        const int cl = (2 * pi + s0) + child_side * ((2 * pj + s1) + child_side * (2 * pk + s2));
        const int cid = child_lookup[cl];
        if (cid < 0) continue;   // uniform over the block
        __syncthreads();
        for (int i = threadIdx.x; i < n3; i += blockDim.x) sW[i] = Wc[(size_t)cid * n3 + i];
        __syncthreads();
        contract_axis(ell, 0, sW, sA, sM[s0], true);
        __syncthreads();
        contract_axis(ell, 1, sA, sB, sM[s1], true);
        __syncthreads();
        contract_axis(ell, 2, sB, sA, sM[s2], true);
        __syncthreads();
        for (int i = threadIdx.x; i < n3; i += blockDim.x) sOut[i] += sA[i];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n3; i += blockDim.x) Wp[(size_t)pid * n3 + i] = sOut[i];
}

// L2L, Eq. (8): the child's nodes receive the parent's interpolant (added to the
// child's own M2L local).  One block per child cell.
template <typename T>
__global__ void __launch_bounds__(kFmmThreads)
l2l_kernel(int ell, int ncells, const int32_t *__restrict__ ijk, int parent_side,
           const int32_t *__restrict__ parent_lookup, const T *__restrict__ Fp, const T *__restrict__ M2,
           T *__restrict__ Fc)
{
    __shared__ T sF[kMaxN3], sA[kMaxN3], sB[kMaxN3];
    __shared__ T sM[2][64];
    const int cid = blockIdx.x;
    if (cid >= ncells) return;
    const int n3 = ell * ell * ell;
    for (int i = threadIdx.x; i < 2 * ell * ell; i += blockDim.x) sM[i / (ell * ell)][i % (ell * ell)] = M2[i];
    const int ci = ijk[3 * cid], cj = ijk[3 * cid + 1], ck = ijk[3 * cid + 2];
    const int pid = parent_lookup[(ci >> 1) + parent_side * ((cj >> 1) + parent_side * (ck >> 1))];
    if (pid < 0) return;   // cannot happen: a kept cell's parent is kept
    for (int i = threadIdx.x; i < n3; i += blockDim.x) sF[i] = Fp[(size_t)pid * n3 + i];
    __syncthreads();
    contract_axis(ell, 0, sF, sA, sM[ci & 1], false);
    __syncthreads();
    contract_axis(ell, 1, sA, sB, sM[cj & 1], false);
    __syncthreads();
    contract_axis(ell, 2, sB, sA, sM[ck & 1], false);
    __syncthreads();
    for (int i = threadIdx.x; i < n3; i += blockDim.x) Fc[(size_t)cid * n3 + i] += sA[i];
}

// L2P (Eq. (8)) plus the direct near field over the <= 27 neighbour leaves (Eq. (1)
// restricted to them, exact coincidences skipped): one block per leaf, one thread
// per target particle; the sources of all neighbours, concatenated, are staged in
// shared memory in chunks.  Potentials are written in the particles' input order.
template <typename T, int KIND>
__global__ void __launch_bounds__(kP2PThreads)
l2p_p2p_kernel(int ell, double c, int ncells, const int32_t *__restrict__ ijk, int side,
               const int32_t *__restrict__ start, const int32_t *__restrict__ perm, const T *__restrict__ xyz,
               const T *__restrict__ q, double lo, double w, const T *__restrict__ xi, const T *__restrict__ inv_den,
               const T *__restrict__ F, T *__restrict__ phi)
{
    __shared__ T sF[kMaxN3];
    __shared__ T sx[kP2PChunk][4];
    __shared__ int nb_start[27], nb_pre[28];
    const int cid = blockIdx.x;
    if (cid >= ncells) return;
    const int n3 = ell * ell * ell;
    const int ci = ijk[3 * cid], cj = ijk[3 * cid + 1], ck = ijk[3 * cid + 2];
    const int l = ci + side * (cj + side * ck);
    const int j0 = start[l], j1 = start[l + 1];
    for (int i = threadIdx.x; i < n3; i += blockDim.x) sF[i] = F[(size_t)cid * n3 + i];
    if (threadIdx.x == 0) {
        // the neighbour leaves' particle ranges, as one concatenated source list
        int run = 0, k = 0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx, ++k) {
                    const int ni = ci + dx, nj = cj + dy, nk = ck + dz;
                    int s0 = 0, n = 0;
                    if (ni >= 0 && nj >= 0 && nk >= 0 && ni < side && nj < side && nk < side) {
                        const int nl = ni + side * (nj + side * nk);
                        s0 = start[nl];
                        n = start[nl + 1] - s0;
                    }
                    nb_start[k] = s0;
                    nb_pre[k] = run;
                    run += n;
                }
        nb_pre[27] = run;
    }
    __syncthreads();
    const int nsrc = nb_pre[27];
    const T ctr[3] = {T(lo + w * (ci + 0.5)), T(lo + w * (cj + 0.5)), T(lo + w * (ck + 0.5))};
    const T half = T(0.5 * w);
    const T cc = T(c);
    // two targets per thread and pass (up to 2 kP2PThreads per leaf in one sweep of the sources)
    for (int tb = j0; tb < j1; tb += 2 * kP2PThreads) {
        int p[2];
        bool live[2];
        T x[2][3], f[2], near[2];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int it = tb + r * kP2PThreads + threadIdx.x;
            live[r] = it < j1;
            p[r] = live[r] ? perm[it] : 0;
            for (int d = 0; d < 3; ++d) x[r][d] = live[r] ? xyz[3 * p[r] + d] : T(0);
            f[r] = T(0);
            near[r] = T(0);
            if (live[r]) {
                T L0[8], L1[8], L2[8];
                lagrange(ell, (x[r][0] - ctr[0]) / half, xi, inv_den, L0);
                lagrange(ell, (x[r][1] - ctr[1]) / half, xi, inv_den, L1);
                lagrange(ell, (x[r][2] - ctr[2]) / half, xi, inv_den, L2);
                for (int a2 = 0; a2 < ell; ++a2) {
                    T s1 = T(0);
                    for (int a1 = 0; a1 < ell; ++a1) {
                        T s0 = T(0);
                        for (int a0 = 0; a0 < ell; ++a0) s0 += L0[a0] * sF[a0 + ell * (a1 + ell * a2)];
                        s1 += L1[a1] * s0;
                    }
                    f[r] += L2[a2] * s1;
                }
            }
        }
        const bool any1 = tb + kP2PThreads < j1;   // block-uniform: a second target per thread exists
        for (int cb = 0; cb < nsrc; cb += kP2PChunk) {
            __syncthreads();
            const int cn = min(kP2PChunk, nsrc - cb);
            for (int u = threadIdx.x; u < cn; u += kP2PThreads) {
                const int g = cb + u;
                int k = 0;
                while (nb_pre[k + 1] <= g) ++k;
                const int ps = perm[nb_start[k] + (g - nb_pre[k])];
                sx[u][0] = xyz[3 * ps];
                sx[u][1] = xyz[3 * ps + 1];
                sx[u][2] = xyz[3 * ps + 2];
                sx[u][3] = q[ps];
            }
            __syncthreads();
            if (any1) {
                if (live[0]) {
#pragma unroll 4
                    for (int jj = 0; jj < cn; ++jj) {
                        const T sq = sx[jj][3];
#pragma unroll
                        for (int r = 0; r < 2; ++r) {
                            const T d0 = x[r][0] - sx[jj][0], d1 = x[r][1] - sx[jj][1], d2 = x[r][2] - sx[jj][2];
                            const T r2 = d0 * d0 + d1 * d1 + d2 * d2;
                            // exact coincidences (the target itself) contribute nothing
                            const T k = kernel_of_r2(KIND, cc, r2 > T(0) ? r2 : T(1));
                            near[r] += (r2 > T(0) ? k : T(0)) * sq;
                        }
                    }
                }
            } else if (live[0]) {
#pragma unroll 4
                for (int jj = 0; jj < cn; ++jj) {
                    const T d0 = x[0][0] - sx[jj][0], d1 = x[0][1] - sx[jj][1], d2 = x[0][2] - sx[jj][2];
                    const T r2 = d0 * d0 + d1 * d1 + d2 * d2;
                    const T k = kernel_of_r2(KIND, cc, r2 > T(0) ? r2 : T(1));
                    near[0] += (r2 > T(0) ? k : T(0)) * sx[jj][3];
                }
            }
        }
#pragma unroll
        for (int r = 0; r < 2; ++r)
            if (live[r]) phi[p[r]] = f[r] + near[r];
    }
}

int grid_for(long n, int threads)
{
    long b = (n + threads - 1) / threads;
    if (b > 4096) b = 4096;
    return b < 1 ? 1 : (int)b;
}

}  // namespace
}  // namespace m2l

using namespace m2l;

struct m2l_fmm {
    int fp64 = 0, n = 0, leaf = 0, ell = 0, n3 = 0, kind = 0;
    double c = 0.0, lo = 0.0, dw = 0.0;
    DevBuf perm, start, xi, inv_den, M2;
    struct Lvl {
        int ncells = 0, side = 0;
        int64_t nnz = 0;
        DevBuf ijk, lookup, W, F, off, src;
        m2l_level lv{};
        m2l_plan *plan = nullptr;
    };
    std::vector<Lvl> lv;   // index = level
};

namespace {

void fmm_release(m2l_fmm *f)
{
    if (!f) return;
    cudaDeviceSynchronize();
    f->perm.release(); f->start.release(); f->xi.release(); f->inv_den.release(); f->M2.release();
    for (auto &L : f->lv) {
        L.ijk.release(); L.lookup.release(); L.W.release(); L.F.release(); L.off.release(); L.src.release();
        if (L.plan) m2l_plan_free(L.plan);
        L.plan = nullptr;
    }
    delete f;
}

template <typename T>
m2l_status upload_constants(m2l_fmm *f, cudaStream_t s)
{
    const int ell = f->ell;
    // Chebyshev roots in ascending order and the Lagrange denominators
    std::vector<double> xi(ell), den(ell), M(2 * ell * ell);
    for (int k = 0; k < ell; ++k) xi[k] = -cos((2.0 * k + 1.0) * M_PI / (2.0 * ell));
    for (int k = 0; k < ell; ++k) {
        double d = 1.0;
        for (int j = 0; j < ell; ++j)
            if (j != k) d *= (xi[k] - xi[j]);
        den[k] = 1.0 / d;
    }
    // M[s][i][k] = L_k(s - 1/2 + xi_i / 2): parent basis k at child node i of side s
    for (int side = 0; side < 2; ++side)
        for (int i = 0; i < ell; ++i) {
            const double x = side - 0.5 + 0.5 * xi[i];
            for (int k = 0; k < ell; ++k) {
                double v = den[k];
                for (int j = 0; j < ell; ++j)
                    if (j != k) v *= (x - xi[j]);
                M[(side * ell + i) * ell + k] = v;
            }
        }
    std::vector<T> hxi(xi.begin(), xi.end()), hden(den.begin(), den.end()), hM(M.begin(), M.end());
    m2l_status st;
    if ((st = f->xi.ensure(ell * sizeof(T))) != M2L_OK) return st;
    if ((st = f->inv_den.ensure(ell * sizeof(T))) != M2L_OK) return st;
    if ((st = f->M2.ensure(2 * ell * ell * sizeof(T))) != M2L_OK) return st;
    M2L_CUDA(cudaMemcpyAsync(f->xi.p, hxi.data(), ell * sizeof(T), cudaMemcpyHostToDevice, s));
    M2L_CUDA(cudaMemcpyAsync(f->inv_den.p, hden.data(), ell * sizeof(T), cudaMemcpyHostToDevice, s));
    M2L_CUDA(cudaMemcpyAsync(f->M2.p, hM.data(), 2 * ell * ell * sizeof(T), cudaMemcpyHostToDevice, s));
    M2L_CUDA(cudaStreamSynchronize(s));
    return M2L_OK;
}

template <typename T>
m2l_status fmm_build(m2l_fmm *f, const m2l_ops *const *ops, const T *xyz, cudaStream_t s)
{
    m2l_status st;
    const int n = f->n, leaf = f->leaf;
    const int side = 1 << leaf;
    const size_t dense = (size_t)side * side * side;
    DevBuf lin, cnt, cursor, flag, pflag, pos;
    ScratchGuard guard{&lin, &cnt, &cursor, &flag, &pflag, &pos};
    auto cleanup = [&]() { lin.release(); cnt.release(); cursor.release(); flag.release(); pflag.release(); pos.release(); };
    if ((st = f->perm.ensure((size_t)(n > 0 ? n : 1) * sizeof(int32_t))) != M2L_OK) return st;
    if ((st = f->start.ensure((dense + 1) * sizeof(int32_t))) != M2L_OK) return st;
    if ((st = lin.ensure((size_t)(n > 0 ? n : 1) * sizeof(int32_t))) != M2L_OK) { cleanup(); return st; }
    if ((st = cnt.ensure((dense + 1) * sizeof(int32_t))) != M2L_OK) { cleanup(); return st; }
    if ((st = cursor.ensure(dense * sizeof(int32_t))) != M2L_OK) { cleanup(); return st; }
    if ((st = flag.ensure((dense + 1) * sizeof(int32_t))) != M2L_OK) { cleanup(); return st; }
    if ((st = pflag.ensure((dense / 8 + 1) * sizeof(int32_t))) != M2L_OK) { cleanup(); return st; }
    if ((st = pos.ensure((dense + 1) * sizeof(int32_t))) != M2L_OK) { cleanup(); return st; }
    const double wl = f->dw / side;
    M2L_CUDA(cudaMemsetAsync(cnt.p, 0, (dense + 1) * sizeof(int32_t), s));
    M2L_CUDA(cudaMemsetAsync(cursor.p, 0, dense * sizeof(int32_t), s));
    if (n > 0) {
        bin_count_kernel<T><<<grid_for(n, 256), 256, 0, s>>>(n, xyz, f->lo, wl, side, lin.as<int32_t>(),
                                                            cnt.as<int32_t>());
        M2L_LAUNCH_CHECK("bin_count_kernel");
    }
    if ((st = launch_exclusive_scan(cnt.as<int32_t>(), f->start.as<int32_t>(), (int)dense, s)) != M2L_OK) {
        cleanup();
        return st;
    }
    if (n > 0) {
        bin_scatter_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, lin.as<int32_t>(), f->start.as<int32_t>(),
                                                            cursor.as<int32_t>(), f->perm.as<int32_t>());
        M2L_LAUNCH_CHECK("bin_scatter_kernel");
    }
    leaf_flags_kernel<<<grid_for((long)dense, 256), 256, 0, s>>>((int)dense, cnt.as<int32_t>(), flag.as<int32_t>());
    M2L_LAUNCH_CHECK("leaf_flags_kernel");
    f->lv.assign(leaf + 1, m2l_fmm::Lvl());
    for (int L = leaf; L >= 2; --L) {
        const int sd = 1 << L;
        const size_t dn = (size_t)sd * sd * sd;
        if (L < leaf) {
            // flags of level L from those of level L + 1 (kept in `flag`)
            M2L_CUDA(cudaMemsetAsync(pflag.p, 0, dn * sizeof(int32_t), s));
            parent_flags_kernel<<<grid_for((long)dn * 8, 256), 256, 0, s>>>(2 * sd, flag.as<int32_t>(),
                                                                              pflag.as<int32_t>());
            M2L_LAUNCH_CHECK("parent_flags_kernel");
            M2L_CUDA(cudaMemcpyAsync(flag.p, pflag.p, dn * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        }
        if ((st = launch_exclusive_scan(flag.as<int32_t>(), pos.as<int32_t>(), (int)dn, s)) != M2L_OK) {
            cleanup();
            return st;
        }
        int count = 0;
        M2L_CUDA(cudaMemcpyAsync(&count, pos.as<int32_t>() + dn, sizeof(int), cudaMemcpyDeviceToHost, s));
        M2L_CUDA(cudaStreamSynchronize(s));
        m2l_fmm::Lvl &V = f->lv[L];
        V.ncells = count;
        V.side = sd;
        const size_t nc = (size_t)(count > 0 ? count : 1);
        if ((st = V.ijk.ensure(nc * 3 * sizeof(int32_t))) != M2L_OK) { cleanup(); return st; }
        if ((st = V.lookup.ensure(dn * sizeof(int32_t))) != M2L_OK) { cleanup(); return st; }
        if ((st = V.W.ensure(nc * f->n3 * sizeof(T))) != M2L_OK) { cleanup(); return st; }
        if ((st = V.F.ensure(nc * f->n3 * sizeof(T))) != M2L_OK) { cleanup(); return st; }
        if ((st = V.off.ensure((nc + 1) * sizeof(int32_t))) != M2L_OK) { cleanup(); return st; }
        compact_kernel<<<grid_for((long)dn, 256), 256, 0, s>>>(sd, flag.as<int32_t>(), pos.as<int32_t>(),
                                                               V.ijk.as<int32_t>(), V.lookup.as<int32_t>());
        M2L_LAUNCH_CHECK("compact_kernel");
        // interaction lists (Sec. 3.2) and the level's M2L plan
        int64_t nnz = 0;
        if ((st = m2l_build_lists(count, V.ijk.as<int32_t>(), count, V.ijk.as<int32_t>(), V.off.as<int32_t>(),
                                  nullptr, &nnz, s)) != M2L_OK) { cleanup(); return st; }
        if ((st = V.src.ensure((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t))) != M2L_OK) { cleanup(); return st; }
        if (nnz > 0 && (st = m2l_build_lists(count, V.ijk.as<int32_t>(), count, V.ijk.as<int32_t>(),
                                             V.off.as<int32_t>(), V.src.as<int32_t>(), &nnz, s)) != M2L_OK) {
            cleanup();
            return st;
        }
        V.nnz = nnz;
        V.lv.level = L;
        V.lv.width = f->dw / sd;
        V.lv.ncells_tgt = V.lv.ncells_src = count;
        V.lv.tgt_ijk = V.lv.src_ijk = V.ijk.as<int32_t>();
        V.lv.il_offsets = V.off.as<int32_t>();
        V.lv.il_sources = V.src.as<int32_t>();
        V.lv.nnz = (int)nnz;
        if ((st = m2l_plan_create(ops[L - 2], &V.lv, 0, s, &V.plan)) != M2L_OK) { cleanup(); return st; }
    }
    cleanup();
    return upload_constants<T>(f, s);
}

template <typename T>
m2l_status fmm_eval(const m2l_fmm *f, const T *xyz, const T *q, T *phi, int precision, cudaStream_t s)
{
    m2l_status st;
    const int leaf = f->leaf, ell = f->ell, n3 = f->n3;
    const auto &V = f->lv;
    const double wl = f->dw / (1 << leaf);
    if (V[leaf].ncells > 0) {
        p2m_kernel<T><<<V[leaf].ncells, kFmmThreads, 0, s>>>(ell, V[leaf].ncells, V[leaf].ijk.as<int32_t>(),
                                                             V[leaf].side, f->start.as<int32_t>(),
                                                             f->perm.as<int32_t>(), xyz, q, f->lo, wl,
                                                             f->xi.as<T>(), f->inv_den.as<T>(), V[leaf].W.as<T>());
        M2L_LAUNCH_CHECK("p2m_kernel");
    }
    for (int L = leaf - 1; L >= 2; --L) {
        if (V[L].ncells == 0) continue;
        m2m_kernel<T><<<V[L].ncells, kFmmThreads, 0, s>>>(ell, V[L].ncells, V[L].ijk.as<int32_t>(), V[L + 1].side,
                                                          V[L + 1].lookup.as<int32_t>(), V[L + 1].W.as<T>(),
                                                          f->M2.as<T>(), V[L].W.as<T>());
        M2L_LAUNCH_CHECK("m2m_kernel");
    }
    for (int L = 2; L <= leaf; ++L) {
        if (V[L].ncells == 0) continue;
        M2L_CUDA(cudaMemsetAsync(V[L].F.p, 0, (size_t)V[L].ncells * n3 * sizeof(T), s));
        if ((st = m2l_plan_apply(V[L].plan, V[L].W.p, V[L].F.p, precision, f->fp64, s)) != M2L_OK) return st;
    }
    for (int L = 3; L <= leaf; ++L) {
        if (V[L].ncells == 0) continue;
        l2l_kernel<T><<<V[L].ncells, kFmmThreads, 0, s>>>(ell, V[L].ncells, V[L].ijk.as<int32_t>(), V[L - 1].side,
                                                          V[L - 1].lookup.as<int32_t>(), V[L - 1].F.as<T>(),
                                                          f->M2.as<T>(), V[L].F.as<T>());
        M2L_LAUNCH_CHECK("l2l_kernel");
    }
    if (V[leaf].ncells > 0) {
        auto kern = f->kind == M2L_K_INV_R ? l2p_p2p_kernel<T, M2L_K_INV_R>
                    : f->kind == M2L_K_INV_R4 ? l2p_p2p_kernel<T, M2L_K_INV_R4>
                                               : l2p_p2p_kernel<T, M2L_K_INV_SQRT_R2C2>;
        kern<<<V[leaf].ncells, kP2PThreads, 0, s>>>(ell, f->c, V[leaf].ncells, V[leaf].ijk.as<int32_t>(), V[leaf].side,
                                                    f->start.as<int32_t>(), f->perm.as<int32_t>(), xyz, q, f->lo, wl,
                                                    f->xi.as<T>(), f->inv_den.as<T>(), V[leaf].F.as<T>(), phi);
        M2L_LAUNCH_CHECK("l2p_p2p_kernel");
    }
    return M2L_OK;
}

}  // namespace

extern "C" {

m2l_status m2l_fmm_create(const m2l_ops *const *ops, int n_particles, const void *xyz, int fp64, int leaf_level,
                          double lo, double domain_width, void *stream, m2l_fmm **out)
{
    if (!out || !ops || n_particles < 0 || (n_particles > 0 && !xyz) || leaf_level < 2 || leaf_level > 8 ||
        !(domain_width > 0.0) || !isfinite(lo)) {
        set_error("bad FMM arguments (leaf level must be in [2, 8])");
        return M2L_EINVAL;
    }
    *out = nullptr;
    const m2l_ops *leaf_ops = ops[leaf_level - 2];
    for (int L = 2; L <= leaf_level; ++L) {
        const m2l_ops *o = ops[L - 2];
        if (!o) { set_error("null operators for level %d", L); return M2L_EINVAL; }
        if (m2l_status st = check_device(o)) return st;
        if (o->ell != leaf_ops->ell || o->kind != leaf_ops->kind || o->c != leaf_ops->c) {
            set_error("the operators of all levels must share kernel and order");
            return M2L_EINVAL;
        }
    }
    if (leaf_ops->ell > 8) { set_error("ell <= 8"); return M2L_EUNSUPPORTED; }
    m2l_fmm *f = new m2l_fmm();
    f->fp64 = fp64 ? 1 : 0;
    f->n = n_particles;
    f->leaf = leaf_level;
    f->ell = leaf_ops->ell;
    f->n3 = leaf_ops->n3;
    f->kind = leaf_ops->kind;
    f->c = leaf_ops->c;
    f->lo = lo;
    f->dw = domain_width;
    cudaStream_t s = (cudaStream_t)stream;
    m2l_status st = fp64 ? fmm_build<double>(f, ops, (const double *)xyz, s) : fmm_build<float>(f, ops, (const float *)xyz, s);
    if (st == M2L_OK) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "FMM set-up");
    }
    if (st != M2L_OK) {
        fmm_release(f);
        return st;
    }
    *out = f;
    return M2L_OK;
}

m2l_status m2l_fmm_evaluate(const m2l_fmm *fmm, const void *xyz, const void *charges, void *potentials,
                            int precision, void *stream)
{
    if (!fmm || (fmm->n > 0 && (!xyz || !charges || !potentials))) { set_error("bad FMM evaluate arguments"); return M2L_EINVAL; }
    if ((precision == M2L_FP64) != (fmm->fp64 == 1)) {
        set_error("M2L_FP64 goes with an FP64 FMM, the other precisions with an FP32 one");
        return M2L_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    return fmm->fp64 ? fmm_eval<double>(fmm, (const double *)xyz, (const double *)charges, (double *)potentials, precision, s)
                     : fmm_eval<float>(fmm, (const float *)xyz, (const float *)charges, (float *)potentials, precision, s);
}

m2l_status m2l_fmm_query(const m2l_fmm *fmm, int level, int32_t *host_ijk, void *host_W, void *host_F)
{
    if (!fmm || level < 2 || level > fmm->leaf) { set_error("bad FMM level"); return M2L_EINVAL; }
    M2L_CUDA(cudaDeviceSynchronize());
    const auto &V = fmm->lv[level];
    const size_t esz = fmm->fp64 ? sizeof(double) : sizeof(float);
    if (V.ncells > 0) {
        if (host_ijk) M2L_CUDA(cudaMemcpy(host_ijk, V.ijk.p, (size_t)V.ncells * 3 * sizeof(int32_t), cudaMemcpyDeviceToHost));
        if (host_W) M2L_CUDA(cudaMemcpy(host_W, V.W.p, (size_t)V.ncells * fmm->n3 * esz, cudaMemcpyDeviceToHost));
        if (host_F) M2L_CUDA(cudaMemcpy(host_F, V.F.p, (size_t)V.ncells * fmm->n3 * esz, cudaMemcpyDeviceToHost));
    }
    return M2L_OK;
}

m2l_status m2l_fmm_info(const m2l_fmm *fmm, int *leaf_level, int64_t *ncells9, int64_t *nnz9)
{
    if (!fmm) { set_error("null FMM"); return M2L_EINVAL; }
    if (leaf_level) *leaf_level = fmm->leaf;
    for (int L = 0; L <= 8; ++L) {
        const bool have = L >= 2 && L <= fmm->leaf;
        if (ncells9) ncells9[L] = have ? fmm->lv[L].ncells : 0;
        if (nnz9) nnz9[L] = have ? fmm->lv[L].nnz : 0;
    }
    return M2L_OK;
}

void m2l_fmm_free(m2l_fmm *fmm) { fmm_release(fmm); }

}  // extern "C"
