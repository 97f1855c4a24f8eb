// Leaf self-block inverses (arxiv 2307.03968 eq. 12, [Z~_N]^{-1} read as the
// block-diagonal D^{-1} of the leaf self blocks).
//
// The complex128 block is inverted in place by Gauss-Jordan elimination with
// partial (row) pivoting, all arithmetic in FP64; row exchanges are undone on the
// columns in reverse order at the end.  Leaves of up to SMEM_LEAF unknowns: one
// CTA per leaf holds the block in shared memory (k_factor_gj).  Larger leaves
// (the paper's leaves run to about a thousand unknowns): the blocks of all of
// them sit in a device workspace and each pivot step is two launches over all of
// them, k_gj_pivot (pivot search, row exchange and scaling of the pivot row, one
// CTA per leaf) and k_gj_eliminate (the update of every other row, spread over
// the whole GPU), then k_gj_finish undoes the exchanges and writes the outputs.
// Launch boundaries order the steps: no CTA waits for another.  The inverse is written column-major (np x np, np = padded
// leaf length, zero padding) as complex64, and as complex128 when the operator
// keeps an FP64 copy; the complex64 copy of D itself (same layout) is written
// too, for FP64-accumulated residuals.  A zero pivot records HM_ERR_SINGULAR.
#include "hm_internal.h"

#include <algorithm>
#include <cstdint>
#include <vector>

namespace hm {
namespace {

__device__ __forceinline__ double2 zmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zinv(double2 a)
{
    // 1/a with scaling by the larger component (Smith's method)
    if (fabs(a.x) >= fabs(a.y)) {
        const double r = a.y / a.x, d = a.x + a.y * r;
        return make_double2(1.0 / d, -r / d);
    }
    const double r = a.x / a.y, d = a.y + a.x * r;
    return make_double2(r / d, -1.0 / d);
}

constexpr int SMEM_LEAF = 112;    // largest leaf held whole in shared memory (FP64 complex: 200 KB)
constexpr int MAX_LEAF = 1536;    // largest leaf of the workspace variant

__global__ void __launch_bounds__(256)
k_factor_gj(const int32_t *__restrict__ pleaf_off, const int64_t *__restrict__ leaf_n,
            const int64_t *__restrict__ self_off, const double2 *__restrict__ self64,
            const int64_t *__restrict__ dinv_off, float2 *__restrict__ dinv32, double2 *__restrict__ dinv64,
            float2 *__restrict__ self32, int *status, int *bad_leaf)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int leaf = blockIdx.x;
    const int n = (int)leaf_n[leaf];
    if (n > SMEM_LEAF) return;                              // the workspace variant takes it
    const int np = pleaf_off[leaf + 1] - pleaf_off[leaf];
    double2 *A = reinterpret_cast<double2 *>(smem_raw);    // n x n row-major
    double2 *colk = A + n * n;                              // [n]
    int *piv = reinterpret_cast<int *>(colk + n);           // [n]
    __shared__ int s_p;
    __shared__ double2 s_inv;
    __shared__ int s_singular;
    const int tid = threadIdx.x, nt = blockDim.x;
    const double2 *S = self64 + self_off[leaf];
    const int64_t doff = dinv_off[leaf];
    for (int e = tid; e < np * np; e += nt) {
        const int j = e / np, i = e - j * np;   // column-major target (i row, j col)
        double2 v = make_double2(0.0, 0.0);
        if (i < n && j < n) v = S[(int64_t)i * n + j];
        self32[doff + e] = make_float2((float)v.x, (float)v.y);
    }
    for (int e = tid; e < n * n; e += nt) A[e] = S[e];
    if (tid == 0) s_singular = 0;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (tid < 32) {
            double best = -1.0;
            int bi = k;
            for (int i = k + tid; i < n; i += 32) {
                const double2 a = A[i * n + k];
                const double mag = a.x * a.x + a.y * a.y;
                if (mag > best) { best = mag; bi = i; }
            }
            for (int s = 16; s >= 1; s >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, s);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, s);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (tid == 0) {
                s_p = bi;
                if (!(best > 0.0)) s_singular = 1;
            }
        }
        __syncthreads();
        if (s_singular) break;
        const int p = s_p;
        if (p != k)
            for (int j = tid; j < n; j += nt) {
                const double2 t = A[k * n + j];
                A[k * n + j] = A[p * n + j];
                A[p * n + j] = t;
            }
        if (tid == 0) piv[k] = p;
        __syncthreads();
        if (tid == 0) s_inv = zinv(A[k * n + k]);
        __syncthreads();
        const double2 inv = s_inv;
        for (int j = tid; j < n; j += nt) {
            const double2 v = (j == k) ? make_double2(1.0, 0.0) : A[k * n + j];
            A[k * n + j] = zmul(v, inv);
        }
        for (int i = tid; i < n; i += nt) colk[i] = (i == k) ? make_double2(0.0, 0.0) : A[i * n + k];
        __syncthreads();
        for (int e = tid; e < n * n; e += nt) {
            const int i = e / n, j = e - i * n;
            if (i == k) continue;
            const double2 f = colk[i];
            const double2 base = (j == k) ? make_double2(0.0, 0.0) : A[e];
            const double2 r = A[k * n + j];
            A[e] = make_double2(base.x - (f.x * r.x - f.y * r.y), base.y - (f.x * r.y + f.y * r.x));
        }
        __syncthreads();
    }
    if (s_singular) {
        if (tid == 0) {
            if (atomicCAS(status, 0, (int)HM_ERR_SINGULAR) == 0) *bad_leaf = leaf;
        }
        return;
    }
    for (int k = n - 1; k >= 0; --k) {
        const int p = piv[k];
        if (p != k)
            for (int i = tid; i < n; i += nt) {
                const double2 t = A[i * n + k];
                A[i * n + k] = A[i * n + p];
                A[i * n + p] = t;
            }
        __syncthreads();
    }
    for (int e = tid; e < np * np; e += nt) {
        const int j = e / np, i = e - j * np;
        double2 v = make_double2(0.0, 0.0);
        if (i < n && j < n) v = A[i * n + j];
        dinv32[doff + e] = make_float2((float)v.x, (float)v.y);
        if (dinv64) dinv64[doff + e] = v;
    }
}

// ---- the workspace variant: large leaf b (leaf index big[b], n = leaf_n) has its
// block at W + woff[b] (row-major n x n), its pivots at piv + poff[b], its column k at
// colk + poff[b]; bad[b] marks a zero pivot (the leaf's later steps are skipped)

// copy the blocks in and the complex64 copy of D out (column-major, zero padded)
__global__ void __launch_bounds__(256)
k_gj_load(const int32_t *__restrict__ big, const int64_t *__restrict__ woff, const int32_t *__restrict__ pleaf_off,
          const int64_t *__restrict__ leaf_n, const int64_t *__restrict__ self_off, const double2 *__restrict__ self64,
          const int64_t *__restrict__ dinv_off, float2 *__restrict__ self32, double2 *__restrict__ W, int *bad)
{
    const int b = blockIdx.x, leaf = big[b];
    const int n = (int)leaf_n[leaf], np = pleaf_off[leaf + 1] - pleaf_off[leaf];
    const double2 *S = self64 + self_off[leaf];
    double2 *A = W + woff[b];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
    for (int64_t e = tid; e < (int64_t)n * n; e += blockDim.x) A[e] = S[e];
    for (int j = w; j < np; j += nw)
        for (int i = lane; i < np; i += 32) {
            double2 v = make_double2(0.0, 0.0);
            if (i < n && j < n) v = S[(int64_t)i * n + j];
            self32[dinv_off[leaf] + (int64_t)j * np + i] = make_float2((float)v.x, (float)v.y);
        }
    if (tid == 0) bad[b] = 0;
}

// step k, one CTA per large leaf: pivot search in column k (rows k..n-1), row
// exchange, scaling of the pivot row (A[k][k] = 1 / pivot), column k kept in colk
__global__ void __launch_bounds__(256)
k_gj_pivot(int k, const int32_t *__restrict__ big, const int64_t *__restrict__ woff, const int64_t *__restrict__ poff,
           const int64_t *__restrict__ leaf_n, double2 *__restrict__ W, double2 *__restrict__ colk,
           int *__restrict__ piv, int *__restrict__ bad)
{
    __shared__ int s_p;
    __shared__ double2 s_inv;
    const int b = blockIdx.x, leaf = big[b];
    const int n = (int)leaf_n[leaf];
    if (k >= n || bad[b]) return;
    double2 *A = W + woff[b];
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid < 32) {
        double best = -1.0;
        int bi = k;
        for (int i = k + tid; i < n; i += 32) {
            const double2 a = A[(int64_t)i * n + k];
            const double mag = a.x * a.x + a.y * a.y;
            if (mag > best) { best = mag; bi = i; }
        }
        for (int sh = 16; sh >= 1; sh >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, sh);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, sh);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (tid == 0) {
            s_p = best > 0.0 ? bi : -1;
            if (!(best > 0.0)) bad[b] = 1;
        }
    }
    __syncthreads();
    const int p = s_p;
    if (p < 0) return;
    if (p != k)
        for (int j = tid; j < n; j += nt) {
            const double2 t = A[(int64_t)k * n + j];
            A[(int64_t)k * n + j] = A[(int64_t)p * n + j];
            A[(int64_t)p * n + j] = t;
        }
    if (tid == 0) piv[poff[b] + k] = p;
    __syncthreads();
    if (tid == 0) s_inv = zinv(A[(int64_t)k * n + k]);
    __syncthreads();
    const double2 inv = s_inv;
    for (int i = tid; i < n; i += nt) colk[poff[b] + i] = (i == k) ? make_double2(0.0, 0.0) : A[(int64_t)i * n + k];
    for (int j = tid; j < n; j += nt) {
        const double2 v = (j == k) ? make_double2(1.0, 0.0) : A[(int64_t)k * n + j];
        A[(int64_t)k * n + j] = zmul(v, inv);
    }
}

// step k, every row i != k of every large leaf: A[i][j] -= colk[i] * A[k][j] (the
// pivot row already scaled; at j = k this leaves -colk[i] * A[k][k]); blockIdx.y
// = leaf, each warp one row
constexpr int GJ_ROWS = 8;
__global__ void __launch_bounds__(GJ_ROWS * 32)
k_gj_eliminate(int k, const int32_t *__restrict__ big, const int64_t *__restrict__ woff,
               const int64_t *__restrict__ poff, const int64_t *__restrict__ leaf_n, double2 *__restrict__ W,
               const double2 *__restrict__ colk, const int *__restrict__ bad)
{
    const int b = blockIdx.y, leaf = big[b];
    const int n = (int)leaf_n[leaf];
    const int i = blockIdx.x * GJ_ROWS + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (k >= n || bad[b] || i >= n || i == k) return;
    double2 *A = W + woff[b];
    const double2 f = colk[poff[b] + i];
    const double2 *R = A + (int64_t)k * n;
    double2 *Ai = A + (int64_t)i * n;
    for (int j = lane; j < n; j += 32) {
        const double2 base = (j == k) ? make_double2(0.0, 0.0) : Ai[j];
        const double2 r = R[j];
        Ai[j] = make_double2(base.x - (f.x * r.x - f.y * r.y), base.y - (f.x * r.y + f.y * r.x));
    }
}

// undo the row exchanges on the columns (reverse order) and write the inverse
// (complex64, and complex128 if kept), column-major zero padded; a zero pivot
// records HM_ERR_SINGULAR
__global__ void __launch_bounds__(256)
k_gj_finish(const int32_t *__restrict__ big, const int64_t *__restrict__ woff, const int64_t *__restrict__ poff,
            const int32_t *__restrict__ pleaf_off, const int64_t *__restrict__ leaf_n,
            const int64_t *__restrict__ dinv_off, double2 *__restrict__ W, const int *__restrict__ piv,
            const int *__restrict__ bad, float2 *__restrict__ dinv32, double2 *__restrict__ dinv64, int *status,
            int *bad_leaf)
{
    const int b = blockIdx.x, leaf = big[b];
    const int n = (int)leaf_n[leaf], np = pleaf_off[leaf + 1] - pleaf_off[leaf];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
    if (bad[b]) {
        if (tid == 0 && atomicCAS(status, 0, (int)HM_ERR_SINGULAR) == 0) *bad_leaf = leaf;
        return;
    }
    double2 *A = W + woff[b];
    const int *pv = piv + poff[b];
    for (int k = n - 1; k >= 0; --k) {
        const int p = pv[k];
        if (p != k)
            for (int i = tid; i < n; i += blockDim.x) {
                const double2 t = A[(int64_t)i * n + k];
                A[(int64_t)i * n + k] = A[(int64_t)i * n + p];
                A[(int64_t)i * n + p] = t;
            }
        __syncthreads();
    }
    const int64_t doff = dinv_off[leaf];
    for (int j = w; j < np; j += nw)
        for (int i = lane; i < np; i += 32) {
            double2 v = make_double2(0.0, 0.0);
            if (i < n && j < n) v = A[(int64_t)i * n + j];
            dinv32[doff + (int64_t)j * np + i] = make_float2((float)v.x, (float)v.y);
            if (dinv64) dinv64[doff + (int64_t)j * np + i] = v;
        }
}

} // namespace

int factor_max_leaf() { return MAX_LEAF; }

hm_status launch_factor(hm_matrix h, cudaStream_t s)
{
    int64_t maxsmall = 0, maxbig = 0;
    std::vector<int32_t> big;
    std::vector<int64_t> woff, poff;
    int64_t wtot = 0, ptot = 0;
    for (int64_t i = 0; i < h->n_leaves; ++i) {
        const int64_t n = h->leaf_off[i + 1] - h->leaf_off[i];
        if (n > MAX_LEAF) return fail(HM_ERR_ARG, "leaf larger than the factorisation supports");
        if (n > SMEM_LEAF) {
            big.push_back((int32_t)i);
            woff.push_back(wtot);
            poff.push_back(ptot);
            wtot += n * n;
            ptot += n;
            maxbig = std::max(maxbig, n);
        } else {
            maxsmall = std::max(maxsmall, n);
        }
    }
    if (maxsmall > 0) {
        const size_t smem = maxsmall * maxsmall * sizeof(double2) + maxsmall * sizeof(double2) + maxsmall * sizeof(int) + 16;
        cudaFuncSetAttribute(k_factor_gj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_factor_gj<<<(unsigned)h->n_leaves, 256, smem, s>>>(h->d_pleaf_off, h->d_leaf_n, h->d_self_off, h->d_self64,
                                                           h->d_dinv_off, h->d_dinv32, h->d_dinv64, h->d_self32,
                                                           h->d_status, h->d_bad_leaf);
    }
    if (big.empty()) return HM_OK;
    // large leaves: blocks, pivots, pivot columns and flags in a workspace held for this call
    const int nb = (int)big.size();
    const size_t bytes = sizeof(double2) * (size_t)(wtot + ptot) + sizeof(int) * (size_t)(ptot + nb) +
                         sizeof(int32_t) * nb + 2 * sizeof(int64_t) * nb + 256;
    unsigned char *ws = nullptr;
    HM_CUDA(cudaMalloc((void **)&ws, bytes));
    double2 *W = (double2 *)ws, *colk = W + wtot;
    int *piv = (int *)(colk + ptot), *bad = piv + ptot;
    int32_t *d_big = (int32_t *)(bad + nb);
    int64_t *d_woff = (int64_t *)(((uintptr_t)(d_big + nb) + 7) & ~(uintptr_t)7), *d_poff = d_woff + nb;
    cudaError_t e = cudaMemcpyAsync(d_big, big.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_woff, woff.data(), sizeof(int64_t) * nb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_poff, poff.data(), sizeof(int64_t) * nb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        k_gj_load<<<nb, 256, 0, s>>>(d_big, d_woff, h->d_pleaf_off, h->d_leaf_n, h->d_self_off, h->d_self64,
                                     h->d_dinv_off, h->d_self32, W, bad);
        const dim3 eg((unsigned)((maxbig + GJ_ROWS - 1) / GJ_ROWS), (unsigned)nb);
        for (int k = 0; k < (int)maxbig; ++k) {
            k_gj_pivot<<<nb, 256, 0, s>>>(k, d_big, d_woff, d_poff, h->d_leaf_n, W, colk, piv, bad);
            k_gj_eliminate<<<eg, GJ_ROWS * 32, 0, s>>>(k, d_big, d_woff, d_poff, h->d_leaf_n, W, colk, bad);
        }
        k_gj_finish<<<nb, 256, 0, s>>>(d_big, d_woff, d_poff, h->d_pleaf_off, h->d_leaf_n, h->d_dinv_off, W, piv, bad,
                                       h->d_dinv32, h->d_dinv64, h->d_status, h->d_bad_leaf);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    cudaFree(ws);
    if (e != cudaSuccess) return cuda_fail(e, "large-leaf factorisation");
    return HM_OK;
}

} // namespace hm
