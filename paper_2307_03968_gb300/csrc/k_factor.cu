// Leaf self-block inverses (arxiv 2307.03968 eq. 12, [Z~_N]^{-1} read as the
// block-diagonal D^{-1} of the leaf self blocks).
//
// One CTA per leaf: the complex128 block is loaded into shared memory and
// inverted in place by Gauss-Jordan elimination with partial (row) pivoting,
// all arithmetic in FP64; row exchanges are undone on the columns in reverse
// order at the end.  The inverse is written column-major (np x np, np = padded
// leaf length, zero padding) as complex64, and as complex128 when the operator
// keeps an FP64 copy; the complex64 copy of D itself (same layout) is written
// too, for FP64-accumulated residuals.  A zero pivot records HM_ERR_SINGULAR.
#include "hm_internal.h"

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

__global__ void __launch_bounds__(256)
k_factor_gj(const int32_t *__restrict__ pleaf_off, const int64_t *__restrict__ leaf_n,
            const int64_t *__restrict__ self_off, const double2 *__restrict__ self64,
            const int64_t *__restrict__ dinv_off, float2 *__restrict__ dinv32, double2 *__restrict__ dinv64,
            float2 *__restrict__ self32, int *status, int *bad_leaf)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int leaf = blockIdx.x;
    const int n = (int)leaf_n[leaf];
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

} // namespace

int factor_max_leaf() { return 112; }

void launch_factor(hm_matrix h, cudaStream_t s)
{
    int64_t maxn = 0;
    for (int64_t i = 0; i < h->n_leaves; ++i) maxn = std::max<int64_t>(maxn, h->leaf_off[i + 1] - h->leaf_off[i]);
    const size_t smem = maxn * maxn * sizeof(double2) + maxn * sizeof(double2) + maxn * sizeof(int) + 16;
    cudaFuncSetAttribute(k_factor_gj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_factor_gj<<<(unsigned)h->n_leaves, 256, smem, s>>>(h->d_pleaf_off, h->d_leaf_n, h->d_self_off, h->d_self64,
                                                       h->d_dinv_off, h->d_dinv32, h->d_dinv64, h->d_self32,
                                                       h->d_status, h->d_bad_leaf);
}

} // namespace hm
