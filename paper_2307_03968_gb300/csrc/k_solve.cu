// Device kernels of the power-series solve (arxiv 2307.03968 §IV, eqs. 12-22).
//
//  (the block product is in k_product.cu, the FP64-class residual in k_residual.cu)
//  k_leaf_update   per leaf: out = y - D_i^{-1} z_i (the series accumulate of
//                  x_j = y - D^{-1} M x_{j-1}), or out = D_i^{-1} z_i; clears z.
//  helpers         permutation in/out, residual, finiteness check.
#include "k_solve_dev.cuh"

#include <cuda_runtime.h>

namespace hm {
namespace {

using namespace kc;

// Per leaf (blockIdx.x) and right-hand side (blockIdx.y): leaf_update_leaf.
template <class T>
__global__ void __launch_bounds__(256)
k_leaf_update(const int32_t *__restrict__ pleaf_off, const int64_t *__restrict__ dinv_off,
              const typename CT<T>::C *__restrict__ dinv, const typename CT<T>::C *y,
              typename CT<T>::C *zin, typename CT<T>::C *out, int64_t ld, int zero_in)
{
    using C = typename CT<T>::C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ C part[8][64];
    leaf_update_leaf<T>(blockIdx.x, blockIdx.y, pleaf_off, dinv_off, dinv, y, zin, out, ld, zero_in,
                        reinterpret_cast<C *>(smem_raw), part);
}

// acc += D x for the complex64 self blocks (column-major, like D^{-1}), with
// accumulation in precision A (float or double)
template <class A>
__global__ void __launch_bounds__(256)
k_apply_self(const int32_t *__restrict__ pleaf_off, const int64_t *__restrict__ off,
             const float2 *__restrict__ self, const float2 *__restrict__ x, typename CT<A>::C *acc, int64_t ld)
{
    using CA = typename CT<A>::C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CA *xs = reinterpret_cast<CA *>(smem_raw);
    __shared__ CA part[8][64];
    const int leaf = blockIdx.x, r = blockIdx.y;
    const int o = pleaf_off[leaf], np = pleaf_off[leaf + 1] - o;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (int j = tid; j < np; j += blockDim.x) xs[j] = conv<CA>(x[r * ld + o + j]);
    __syncthreads();
    const float2 *S = self + off[leaf];
    for (int rc = 0; rc < np; rc += 64) {
        const int i = rc + 2 * lane;
        CA a0 = czero(CA()), a1 = czero(CA());
        if (i < np)
            for (int j = w; j < np; j += 8) {
                Pair<float> d = ld_stream(S + (int64_t)j * np + i);
                cfma(a0, conv<CA>(d.a), xs[j]);
                cfma(a1, conv<CA>(d.b), xs[j]);
            }
        part[w][2 * lane] = a0;
        part[w][2 * lane + 1] = a1;
        __syncthreads();
        if (tid < 64 && rc + tid < np) {
            CA s = part[0][tid];
#pragma unroll
            for (int q = 1; q < 8; ++q) s = cadd(s, part[q][tid]);
            const int64_t g = r * ld + o + rc + tid;
            acc[g] = cadd(acc[g], s);
        }
        __syncthreads();
    }
}

template <class C>
__global__ void k_permute_in(const C *__restrict__ b, int64_t ldb, C *__restrict__ xt, int64_t pN,
                             const int32_t *__restrict__ pperm, int nrhs)
{
    const int64_t total = pN * nrhs;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / pN, p = t - r * pN;
        const int32_t src = pperm[p];
        xt[t] = src >= 0 ? b[r * ldb + src] : czero(C());
    }
}

// Per leaf (blockIdx.x) and right-hand side (blockIdx.y), complex64: the leaf's rows
// of bt = P b (0 at pads), then y = D_i^{-1} bt_i (the first step of the series, eq. 12
// applied to the permuted right-hand side) in the same CTA.
__global__ void __launch_bounds__(256)
k_permute_leaf(const int32_t *__restrict__ pleaf_off, const int64_t *__restrict__ dinv_off,
               const float2 *__restrict__ dinv, const int32_t *__restrict__ pperm, const float2 *__restrict__ b,
               int64_t ldb, float2 *bt, float2 *y, int64_t pN)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ float2 part[8][64];
    const int leaf = blockIdx.x, r = blockIdx.y;
    const int o = pleaf_off[leaf], np = pleaf_off[leaf + 1] - o;
    for (int j = threadIdx.x; j < np; j += blockDim.x) {
        const int32_t src = pperm[o + j];
        bt[r * pN + o + j] = src >= 0 ? b[r * ldb + src] : make_float2(0.f, 0.f);
    }
    __syncthreads();                                       // this CTA's writes of bt_i, read back below
    leaf_update_leaf<float>(leaf, r, pleaf_off, dinv_off, dinv, nullptr, bt, y, pN, 0,
                            reinterpret_cast<float2 *>(smem_raw), part);
}

template <class C>
__global__ void k_permute_out(const C *__restrict__ xt, int64_t pN, C *__restrict__ x, int64_t ldx,
                              const int32_t *__restrict__ pperm, int nrhs)
{
    const int64_t total = pN * nrhs;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / pN, p = t - r * pN;
        const int32_t dst = pperm[p];
        if (dst >= 0) x[r * ldx + dst] = xt[t];
    }
}

template <class C>
__global__ void k_sub(const C *y, const C *w, C *out, int64_t n)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        out[t] = csub(y[t], w[t]);
}

template <class C>
__global__ void k_add(C *x, const C *dx, int64_t n)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        x[t] = cadd(x[t], dx[t]);
}

template <class C>
__global__ void k_check_finite(const C *x, int64_t n, int *status)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const C v = x[t];
        if (!isfinite(v.x) || !isfinite(v.y)) {
            atomicCAS(status, 0, (int)HM_ERR_DIVERGED);
            return;
        }
    }
}

// the end of a complex64 solve in one pass: v = xt (+ dx), non-finite v -> HM_ERR_DIVERGED,
// x[r * ldx + pperm[p]] = v (the refinement's add, the check and the un-permutation)
__global__ void k_finish(const float2 *__restrict__ xt, const float2 *__restrict__ dx, int64_t pN, float2 *__restrict__ x,
                         int64_t ldx, const int32_t *__restrict__ pperm, int nrhs, int *status)
{
    const int64_t total = pN * nrhs;
    bool bad = false;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        float2 v = xt[t];
        if (dx) v = cadd(v, dx[t]);
        bad |= !isfinite(v.x) || !isfinite(v.y);
        const int64_t r = t / pN, p = t - r * pN;
        const int32_t dst = pperm[p];
        if (dst >= 0) x[r * ldx + dst] = v;
    }
    if (bad) atomicCAS(status, 0, (int)HM_ERR_DIVERGED);
}

// The last series step of a complex64 solve and the end of the solve, per leaf
// (blockIdx.x) and right-hand side (blockIdx.y): out_i = y_i - D_i^{-1} z_i (z_i cleared),
// then v = (base ? base_i + out_i : out_i), non-finite v -> HM_ERR_DIVERGED, and
// x[r * ldx + pperm[p]] = v (k_leaf_update followed by k_finish, in one CTA).
__global__ void __launch_bounds__(256)
k_leaf_finish(const int32_t *__restrict__ pleaf_off, const int64_t *__restrict__ dinv_off,
              const float2 *__restrict__ dinv, const float2 *y, float2 *z, float2 *out, const float2 *base,
              int64_t pN, float2 *__restrict__ x, int64_t ldx, const int32_t *__restrict__ pperm, int *status)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ float2 part[8][64];
    const int leaf = blockIdx.x, r = blockIdx.y;
    leaf_update_leaf<float>(leaf, r, pleaf_off, dinv_off, dinv, y, z, out, pN, 1,
                            reinterpret_cast<float2 *>(smem_raw), part);
    __syncthreads();                                       // this CTA's writes of out_i, read back below
    const int o = pleaf_off[leaf], np = pleaf_off[leaf + 1] - o;
    bool bad = false;
    for (int j = threadIdx.x; j < np; j += blockDim.x) {
        const int64_t g = r * pN + o + j;
        float2 v = out[g];
        if (base) v = cadd(v, base[g]);
        bad |= !isfinite(v.x) || !isfinite(v.y);
        const int32_t dst = pperm[o + j];
        if (dst >= 0) x[r * ldx + dst] = v;
    }
    if (bad) atomicCAS(status, 0, (int)HM_ERR_DIVERGED);
}

__global__ void k_f32_to_f64(const float2 *a, double2 *b, int64_t n)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        b[t] = make_double2(a[t].x, a[t].y);
}

__global__ void k_f64_to_f32(const double2 *a, float2 *b, int64_t n)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        b[t] = make_float2((float)a[t].x, (float)a[t].y);
}

int grid_for(int64_t n, int block = 256)
{
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > 4096) g = 4096;
    return (int)g;
}

} // namespace

void launch_permute_in(const void *b, int64_t ldb, void *xt, int64_t pN, const int32_t *pperm, int nrhs,
                       bool fp64, cudaStream_t s)
{
    const int g = grid_for(pN * nrhs);
    if (fp64)
        k_permute_in<double2><<<g, 256, 0, s>>>((const double2 *)b, ldb, (double2 *)xt, pN, pperm, nrhs);
    else
        k_permute_in<float2><<<g, 256, 0, s>>>((const float2 *)b, ldb, (float2 *)xt, pN, pperm, nrhs);
}

void launch_permute_out(const void *xt, int64_t pN, void *x, int64_t ldx, const int32_t *pperm, int nrhs,
                        bool fp64, cudaStream_t s)
{
    const int g = grid_for(pN * nrhs);
    if (fp64)
        k_permute_out<double2><<<g, 256, 0, s>>>((const double2 *)xt, pN, (double2 *)x, ldx, pperm, nrhs);
    else
        k_permute_out<float2><<<g, 256, 0, s>>>((const float2 *)xt, pN, (float2 *)x, ldx, pperm, nrhs);
}

void launch_zero(void *p, size_t bytes, cudaStream_t s) { cudaMemsetAsync(p, 0, bytes, s); }

static int64_t max_padded_leaf(hm_matrix h)
{
    int64_t maxnp = 0;
    for (int64_t i = 0; i < h->n_leaves; ++i) maxnp = std::max<int64_t>(maxnp, h->pleaf_off[i + 1] - h->pleaf_off[i]);
    return maxnp;
}

void launch_apply_self_f32(hm_matrix h, const float2 *x, float2 *acc, int nrhs, cudaStream_t s)
{
    dim3 grid((unsigned)h->n_leaves, (unsigned)nrhs);
    k_apply_self<float><<<grid, 256, max_padded_leaf(h) * sizeof(float2), s>>>(h->d_pleaf_off, h->d_dinv_off,
                                                                              h->d_self32, x, acc, h->pN);
}

void launch_permute_leaf(hm_matrix h, const float2 *b, int64_t ldb, float2 *bt, float2 *y, int nrhs, cudaStream_t s)
{
    dim3 grid((unsigned)h->n_leaves, (unsigned)nrhs);
    k_permute_leaf<<<grid, 256, max_padded_leaf(h) * sizeof(float2), s>>>(h->d_pleaf_off, h->d_dinv_off, h->d_dinv32,
                                                                          h->d_pperm, b, ldb, bt, y, h->pN);
}

void launch_leaf_update(hm_matrix h, const void *y, void *zin, void *out, int nrhs, bool zero_in, bool fp64,
                        cudaStream_t s)
{
    const int64_t maxnp = max_padded_leaf(h);
    dim3 grid((unsigned)h->n_leaves, (unsigned)nrhs);
    if (fp64)
        k_leaf_update<double><<<grid, 256, maxnp * sizeof(double2), s>>>(
            h->d_pleaf_off, h->d_dinv_off, h->d_dinv64, (const double2 *)y, (double2 *)zin, (double2 *)out, h->pN,
            zero_in ? 1 : 0);
    else
        k_leaf_update<float><<<grid, 256, maxnp * sizeof(float2), s>>>(
            h->d_pleaf_off, h->d_dinv_off, h->d_dinv32, (const float2 *)y, (float2 *)zin, (float2 *)out, h->pN,
            zero_in ? 1 : 0);
}

void launch_sub(const void *y, const void *w, void *out, int64_t n, bool fp64, cudaStream_t s)
{
    const int g = grid_for(n);
    if (fp64) k_sub<double2><<<g, 256, 0, s>>>((const double2 *)y, (const double2 *)w, (double2 *)out, n);
    else k_sub<float2><<<g, 256, 0, s>>>((const float2 *)y, (const float2 *)w, (float2 *)out, n);
}

void launch_add_inplace(void *x, const void *dx, int64_t n, bool fp64, cudaStream_t s)
{
    const int g = grid_for(n);
    if (fp64) k_add<double2><<<g, 256, 0, s>>>((double2 *)x, (const double2 *)dx, n);
    else k_add<float2><<<g, 256, 0, s>>>((float2 *)x, (const float2 *)dx, n);
}

void launch_check_finite(const void *x, int64_t n, bool fp64, int *status, cudaStream_t s)
{
    const int g = grid_for(n);
    if (fp64) k_check_finite<double2><<<g, 256, 0, s>>>((const double2 *)x, n, status);
    else k_check_finite<float2><<<g, 256, 0, s>>>((const float2 *)x, n, status);
}

void launch_leaf_finish(hm_matrix h, const float2 *y, float2 *z, float2 *out, const float2 *base, float2 *x,
                        int64_t ldx, int nrhs, cudaStream_t s)
{
    dim3 grid((unsigned)h->n_leaves, (unsigned)nrhs);
    k_leaf_finish<<<grid, 256, max_padded_leaf(h) * sizeof(float2), s>>>(h->d_pleaf_off, h->d_dinv_off, h->d_dinv32, y,
                                                                         z, out, base, h->pN, x, ldx, h->d_pperm,
                                                                         h->d_status);
}

void launch_finish(const float2 *xt, const float2 *dx, int64_t pN, float2 *x, int64_t ldx, const int32_t *pperm,
                   int nrhs, int *status, cudaStream_t s)
{
    k_finish<<<grid_for(pN * nrhs), 256, 0, s>>>(xt, dx, pN, x, ldx, pperm, nrhs, status);
}

void launch_convert_f32_to_f64(const float2 *a, double2 *b, int64_t n, cudaStream_t s)
{
    k_f32_to_f64<<<grid_for(n), 256, 0, s>>>(a, b, n);
}

void launch_convert_f64_to_f32(const double2 *a, float2 *b, int64_t n, cudaStream_t s)
{
    k_f64_to_f32<<<grid_for(n), 256, 0, s>>>(a, b, n);
}

} // namespace hm
