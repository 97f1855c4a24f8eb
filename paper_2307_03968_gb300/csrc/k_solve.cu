// Device kernels of the power-series solve (arxiv 2307.03968 §IV, eqs. 12-22).
//
//  k_apply_items   z += M x over a list of stored blocks (half storage, §III):
//                  every block is read once and acts on both of its clusters,
//                    dense  B (I,J):  z_I += B x_J,            z_J += B^T x_I
//                    low rank U V:    z_I += U (V x_J),        z_J += V^T (U^T x_I)
//                  One warp per block; a lane owns two adjacent columns, so the
//                  column-side product accumulates in registers and the row-side
//                  product is a transpose reduction over the warp (shuffles).
//                  Results go to z with vector atomics (order-free sums).
//  k_leaf_update   per leaf: out = y - D_i^{-1} z_i (the series accumulate of
//                  x_j = y - D^{-1} M x_{j-1}), or out = D_i^{-1} z_i; clears z.
//  helpers         permutation in/out, residual, finiteness check.
#include "hm_internal.h"

#include <cuda_runtime.h>

namespace hm {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int APPLY_WARPS = 8;   // warps per CTA of the product kernel

template <class T> struct CT;
template <> struct CT<float> { using C = float2; };
template <> struct CT<double> { using C = double2; };

template <class T> struct Pair { typename CT<T>::C a, b; };

__device__ __forceinline__ float2 czero(float2) { return make_float2(0.f, 0.f); }
__device__ __forceinline__ double2 czero(double2) { return make_double2(0.0, 0.0); }

template <class CA, class CB> __device__ __forceinline__ CA conv(CB v);
template <> __device__ __forceinline__ float2 conv<float2, float2>(float2 v) { return v; }
template <> __device__ __forceinline__ double2 conv<double2, double2>(double2 v) { return v; }
template <> __device__ __forceinline__ double2 conv<double2, float2>(float2 v) { return make_double2(v.x, v.y); }

// acc += a * b (complex)
__device__ __forceinline__ void cfma(float2 &acc, float2 a, float2 b)
{
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}
__device__ __forceinline__ void cfma(double2 &acc, double2 a, double2 b)
{
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

__device__ __forceinline__ float2 shfl_xor(float2 v, int s)
{
    return make_float2(__shfl_xor_sync(FULL, v.x, s), __shfl_xor_sync(FULL, v.y, s));
}
__device__ __forceinline__ double2 shfl_xor(double2 v, int s)
{
    return make_double2(__shfl_xor_sync(FULL, v.x, s), __shfl_xor_sync(FULL, v.y, s));
}
__device__ __forceinline__ float2 shfl_idx(float2 v, int l)
{
    return make_float2(__shfl_sync(FULL, v.x, l), __shfl_sync(FULL, v.y, l));
}
__device__ __forceinline__ double2 shfl_idx(double2 v, int l)
{
    return make_double2(__shfl_sync(FULL, v.x, l), __shfl_sync(FULL, v.y, l));
}

// streaming load of two adjacent complex values (16-byte aligned for complex64)
__device__ __forceinline__ Pair<float> ld_stream(const float2 *p)
{
    float4 v = __ldcs(reinterpret_cast<const float4 *>(p));
    return {make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
__device__ __forceinline__ Pair<double> ld_stream(const double2 *p) { return {__ldcs(p), __ldcs(p + 1)}; }
// cached load (data read twice by the same warp)
__device__ __forceinline__ Pair<float> ld_cached(const float2 *p)
{
    float4 v = __ldg(reinterpret_cast<const float4 *>(p));
    return {make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
__device__ __forceinline__ Pair<double> ld_cached(const double2 *p) { return {__ldg(p), __ldg(p + 1)}; }
__device__ __forceinline__ Pair<float> ld_vec(const float2 *p)
{
    float4 v = *reinterpret_cast<const float4 *>(p);
    return {make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
__device__ __forceinline__ Pair<double> ld_vec(const double2 *p) { return {p[0], p[1]}; }

// z[0] += a, z[1] += b (one 16-byte vector reduction for complex64)
__device__ __forceinline__ void red2(float2 *z, float2 a, float2 b)
{
    atomicAdd(reinterpret_cast<float4 *>(z), make_float4(a.x, a.y, b.x, b.y));
}
__device__ __forceinline__ void red2(double2 *z, double2 a, double2 b)
{
    atomicAdd(&z[0].x, a.x); atomicAdd(&z[0].y, a.y);
    atomicAdd(&z[1].x, b.x); atomicAdd(&z[1].y, b.y);
}
__device__ __forceinline__ void red1(float2 *z, float2 a) { atomicAdd(z, a); }
__device__ __forceinline__ void red1(double2 *z, double2 a) { atomicAdd(&z->x, a.x); atomicAdd(&z->y, a.y); }

__device__ __forceinline__ int even_d(int v) { return (v + 1) & ~1; }

// Transpose reduction: on entry every lane holds v[0..31]; on exit lane l holds
// in v[0] the sum over all lanes of v[l].  31 shuffles per component.
template <class CA>
__device__ __forceinline__ void transpose_reduce32(CA (&v)[32], int lane)
{
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const bool up = (lane & s) != 0;
#pragma unroll
        for (int j = 0; j < s; ++j) {
            CA send = up ? v[j] : v[j + s];
            CA keep = up ? v[j + s] : v[j];
            v[j] = cadd(keep, shfl_xor(send, s));
        }
    }
}

// On entry every lane holds v[0..7]; on exit every lane l holds in v[0] the sum
// over all 32 lanes of v[l & 7].
template <class CA>
__device__ __forceinline__ void reduce8(CA (&v)[8], int lane)
{
#pragma unroll
    for (int s = 4; s >= 1; s >>= 1) {
        const bool up = (lane & s) != 0;
#pragma unroll
        for (int j = 0; j < s; ++j) {
            CA send = up ? v[j] : v[j + s];
            CA keep = up ? v[j + s] : v[j];
            v[j] = cadd(keep, shfl_xor(send, s));
        }
    }
    v[0] = cadd(v[0], shfl_xor(v[0], 8));
    v[0] = cadd(v[0], shfl_xor(v[0], 16));
}

// Dense near block B (m x n, row-major, stride even(n)) between leaves I (rows)
// and J (columns):  z_I += B x_J,  z_J += B^T x_I.
template <class T, class A>
__device__ __forceinline__ void dense_item(const Item &it, const typename CT<T>::C *__restrict__ pool,
                                           const typename CT<T>::C *__restrict__ x,
                                           typename CT<A>::C *__restrict__ z, typename CT<T>::C *xs, int lane)
{
    using CTy = typename CT<T>::C;
    using CA = typename CT<A>::C;
    const CTy *B = pool + it.off;
    const int m = it.m, n = it.n, ld = even_d(n);
    const CA zero = czero(CA());
    for (int c0 = 0; c0 < n; c0 += 64) {
        const int j = c0 + 2 * lane;
        const bool jv = j < n;
        CA xj0 = zero, xj1 = zero;
        if (jv) {
            xj0 = conv<CA>(x[it.col0 + j]);
            if (j + 1 < n) xj1 = conv<CA>(x[it.col0 + j + 1]);
        }
        CA cs0 = zero, cs1 = zero;
        for (int r0 = 0; r0 < m; r0 += 32) {
            __syncwarp();
            xs[lane] = (r0 + lane < m) ? x[it.row0 + r0 + lane] : czero(CTy());
            __syncwarp();
            CA rp[32];
#pragma unroll
            for (int rr = 0; rr < 32; ++rr) {
                const int i = r0 + rr;
                Pair<T> b{czero(CTy()), czero(CTy())};
                if (jv && i < m) b = ld_stream(B + (int64_t)i * ld + j);
                const CA xi = conv<CA>(xs[rr]);
                const CA ba = conv<CA>(b.a), bb = conv<CA>(b.b);
                cfma(cs0, ba, xi);
                cfma(cs1, bb, xi);
                CA t = zero;
                cfma(t, ba, xj0);
                cfma(t, bb, xj1);
                rp[rr] = t;
            }
            transpose_reduce32<CA>(rp, lane);
            if (r0 + lane < m) red1(z + it.row0 + r0 + lane, rp[0]);
        }
        if (jv) {
            if (j + 1 < n) red2(z + it.col0 + j, cs0, cs1);
            else red1(z + it.col0 + j, cs0);
        }
    }
}

// Low-rank far block U V with U^T (k x m) and V (k x n) row-major, m and n the
// padded (even) cluster lengths:  z_I += U (V x_J),  z_J += V^T (U^T x_I).
template <class T, class A>
__device__ __forceinline__ void lowrank_item(const Item &it, const typename CT<T>::C *__restrict__ pool,
                                             const typename CT<T>::C *__restrict__ x,
                                             typename CT<A>::C *__restrict__ z, int lane)
{
    using CTy = typename CT<T>::C;
    using CA = typename CT<A>::C;
    const int m = it.m, n = it.n, k = it.k;
    const CTy *UT = pool + it.off;
    const CTy *V = UT + (int64_t)k * m;
    const CA zero = czero(CA());
    if (m <= 64 && n <= 64) {
        // registers hold a chunk of 8 rank rows of both panels
        const int i = 2 * lane;
        const bool iv = i < m, jv = i < n;
        CA xi0 = zero, xi1 = zero, xj0 = zero, xj1 = zero;
        if (iv) { Pair<T> p = ld_vec(x + it.row0 + i); xi0 = conv<CA>(p.a); xi1 = conv<CA>(p.b); }
        if (jv) { Pair<T> p = ld_vec(x + it.col0 + i); xj0 = conv<CA>(p.a); xj1 = conv<CA>(p.b); }
        CA oi0 = zero, oi1 = zero, oj0 = zero, oj1 = zero;
        for (int l0 = 0; l0 < k; l0 += 8) {
            Pair<T> u[8], v[8];
#pragma unroll
            for (int l = 0; l < 8; ++l) {
                u[l] = {czero(CTy()), czero(CTy())};
                v[l] = u[l];
                if (l0 + l < k) {
                    if (iv) u[l] = ld_stream(UT + (int64_t)(l0 + l) * m + i);
                    if (jv) v[l] = ld_stream(V + (int64_t)(l0 + l) * n + i);
                }
            }
            CA tp[8], t[8];
#pragma unroll
            for (int l = 0; l < 8; ++l) {
                tp[l] = zero;
                cfma(tp[l], conv<CA>(u[l].a), xi0);
                cfma(tp[l], conv<CA>(u[l].b), xi1);
                t[l] = zero;
                cfma(t[l], conv<CA>(v[l].a), xj0);
                cfma(t[l], conv<CA>(v[l].b), xj1);
            }
            reduce8<CA>(tp, lane);
            reduce8<CA>(t, lane);
#pragma unroll
            for (int l = 0; l < 8; ++l) {
                const CA tl = shfl_idx(t[0], l);     // (V x_J)_l
                const CA tpl = shfl_idx(tp[0], l);   // (U^T x_I)_l
                cfma(oi0, conv<CA>(u[l].a), tl);
                cfma(oi1, conv<CA>(u[l].b), tl);
                cfma(oj0, conv<CA>(v[l].a), tpl);
                cfma(oj1, conv<CA>(v[l].b), tpl);
            }
        }
        if (iv) red2(z + it.row0 + i, oi0, oi1);
        if (jv) red2(z + it.col0 + i, oj0, oj1);
        return;
    }
    // general sizes: 64-column chunks; the panels are read twice (second read cached)
    for (int l0 = 0; l0 < k; l0 += 8) {
        CA tp[8], t[8];
#pragma unroll
        for (int l = 0; l < 8; ++l) { tp[l] = zero; t[l] = zero; }
        for (int c0 = 0; c0 < m; c0 += 64) {
            const int i = c0 + 2 * lane;
            if (i < m) {
                Pair<T> p = ld_vec(x + it.row0 + i);
                const CA a0 = conv<CA>(p.a), a1 = conv<CA>(p.b);
#pragma unroll
                for (int l = 0; l < 8; ++l)
                    if (l0 + l < k) {
                        Pair<T> u = ld_cached(UT + (int64_t)(l0 + l) * m + i);
                        cfma(tp[l], conv<CA>(u.a), a0);
                        cfma(tp[l], conv<CA>(u.b), a1);
                    }
            }
        }
        for (int c0 = 0; c0 < n; c0 += 64) {
            const int j = c0 + 2 * lane;
            if (j < n) {
                Pair<T> p = ld_vec(x + it.col0 + j);
                const CA a0 = conv<CA>(p.a), a1 = conv<CA>(p.b);
#pragma unroll
                for (int l = 0; l < 8; ++l)
                    if (l0 + l < k) {
                        Pair<T> v = ld_cached(V + (int64_t)(l0 + l) * n + j);
                        cfma(t[l], conv<CA>(v.a), a0);
                        cfma(t[l], conv<CA>(v.b), a1);
                    }
            }
        }
        reduce8<CA>(tp, lane);
        reduce8<CA>(t, lane);
        CA tb[8], tpb[8];
#pragma unroll
        for (int l = 0; l < 8; ++l) { tb[l] = shfl_idx(t[0], l); tpb[l] = shfl_idx(tp[0], l); }
        for (int c0 = 0; c0 < m; c0 += 64) {
            const int i = c0 + 2 * lane;
            if (i < m) {
                CA o0 = zero, o1 = zero;
#pragma unroll
                for (int l = 0; l < 8; ++l)
                    if (l0 + l < k) {
                        Pair<T> u = ld_cached(UT + (int64_t)(l0 + l) * m + i);
                        cfma(o0, conv<CA>(u.a), tb[l]);
                        cfma(o1, conv<CA>(u.b), tb[l]);
                    }
                red2(z + it.row0 + i, o0, o1);
            }
        }
        for (int c0 = 0; c0 < n; c0 += 64) {
            const int j = c0 + 2 * lane;
            if (j < n) {
                CA o0 = zero, o1 = zero;
#pragma unroll
                for (int l = 0; l < 8; ++l)
                    if (l0 + l < k) {
                        Pair<T> v = ld_cached(V + (int64_t)(l0 + l) * n + j);
                        cfma(o0, conv<CA>(v.a), tpb[l]);
                        cfma(o1, conv<CA>(v.b), tpb[l]);
                    }
                red2(z + it.col0 + j, o0, o1);
            }
        }
    }
}

template <class T, class A>
__global__ void __launch_bounds__(APPLY_WARPS * 32)
k_apply_items(const Item *__restrict__ items, int64_t n_items, const typename CT<T>::C *__restrict__ pool,
              const typename CT<T>::C *__restrict__ x, int64_t ldx, typename CT<A>::C *__restrict__ z,
              int64_t ldz, int nrhs)
{
    using CTy = typename CT<T>::C;
    __shared__ CTy xs_all[APPLY_WARPS][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t nw = (int64_t)gridDim.x * APPLY_WARPS;
    for (int64_t t = (int64_t)blockIdx.x * APPLY_WARPS + w; t < n_items; t += nw) {
        const Item it = items[t];
        for (int r = 0; r < nrhs; ++r) {
            if (it.k == 0)
                dense_item<T, A>(it, pool, x + r * ldx, z + r * ldz, xs_all[w], lane);
            else
                lowrank_item<T, A>(it, pool, x + r * ldx, z + r * ldz, lane);
        }
    }
}

// Per leaf (blockIdx.x) and right-hand side (blockIdx.y):
//   w = D_i^{-1} zin_i ;  out_i = y ? y_i - w : w ;  zin_i = 0 if zero_in.
// D_i^{-1} is column-major np x np (np = padded leaf length), zero padded.
template <class T>
__global__ void __launch_bounds__(256)
k_leaf_update(const int32_t *__restrict__ pleaf_off, const int64_t *__restrict__ dinv_off,
              const typename CT<T>::C *__restrict__ dinv, const typename CT<T>::C *y,
              typename CT<T>::C *zin, typename CT<T>::C *out, int64_t ld, int zero_in)
{
    using C = typename CT<T>::C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *zs = reinterpret_cast<C *>(smem_raw);          // [np]
    __shared__ C part[8][64];
    const int leaf = blockIdx.x, r = blockIdx.y;
    const int o = pleaf_off[leaf], np = pleaf_off[leaf + 1] - o;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    C *zr = zin + r * ld + o;
    for (int j = tid; j < np; j += blockDim.x) zs[j] = zr[j];
    __syncthreads();
    if (zero_in)
        for (int j = tid; j < np; j += blockDim.x) zr[j] = czero(C());
    const C *Di = dinv + dinv_off[leaf];
    for (int rc = 0; rc < np; rc += 64) {
        const int i = rc + 2 * lane;
        C a0 = czero(C()), a1 = czero(C());
        if (i < np)
            for (int j = w; j < np; j += 8) {
                Pair<T> d = ld_stream(Di + (int64_t)j * np + i);
                const C zj = zs[j];
                cfma(a0, d.a, zj);
                cfma(a1, d.b, zj);
            }
        part[w][2 * lane] = a0;
        part[w][2 * lane + 1] = a1;
        __syncthreads();
        if (tid < 64 && rc + tid < np) {
            C s = part[0][tid];
#pragma unroll
            for (int q = 1; q < 8; ++q) s = cadd(s, part[q][tid]);
            const int64_t g = r * ld + o + rc + tid;
            out[g] = y ? csub(y[g], s) : s;
        }
        __syncthreads();
    }
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

__global__ void k_residual(const float2 *__restrict__ b, const double2 *__restrict__ acc, float2 *__restrict__ r,
                           double *norms, int64_t pN, int nrhs)
{
    const int64_t total = pN * nrhs;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t col = t / pN;
        const double2 bb = conv<double2>(b[t]);
        const double2 rr = csub(bb, acc[t]);
        r[t] = make_float2((float)rr.x, (float)rr.y);
        atomicAdd(&norms[2 * col], rr.x * rr.x + rr.y * rr.y);
        atomicAdd(&norms[2 * col + 1], bb.x * bb.x + bb.y * bb.y);
    }
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

template <class T, class A>
int apply_grid(hm_matrix h)
{
    static int per_sm = -1;
    if (per_sm < 0) {
        int v = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_apply_items<T, A>, APPLY_WARPS * 32, 0);
        per_sm = v > 0 ? v : 1;
    }
    return per_sm * (h->num_sms > 0 ? h->num_sms : 1);
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

void launch_apply_items(hm_matrix h, const LevelList &L, const void *x, void *z, int nrhs, bool fp64,
                        cudaStream_t s)
{
    const int64_t n = (int64_t)L.items.size();
    if (n == 0) return;
    if (fp64) {
        int g = apply_grid<double, double>(h);
        if ((int64_t)g * APPLY_WARPS > n) g = (int)((n + APPLY_WARPS - 1) / APPLY_WARPS);
        k_apply_items<double, double><<<g, APPLY_WARPS * 32, 0, s>>>(
            L.d_items, n, h->d_pool64, (const double2 *)x, h->pN, (double2 *)z, h->pN, nrhs);
    } else {
        int g = apply_grid<float, float>(h);
        if ((int64_t)g * APPLY_WARPS > n) g = (int)((n + APPLY_WARPS - 1) / APPLY_WARPS);
        k_apply_items<float, float><<<g, APPLY_WARPS * 32, 0, s>>>(
            L.d_items, n, h->d_pool32, (const float2 *)x, h->pN, (float2 *)z, h->pN, nrhs);
    }
}

void launch_apply_items_acc64(hm_matrix h, const LevelList &L, const float2 *x, double2 *acc, int nrhs,
                              cudaStream_t s)
{
    const int64_t n = (int64_t)L.items.size();
    if (n == 0) return;
    int g = apply_grid<float, double>(h);
    if ((int64_t)g * APPLY_WARPS > n) g = (int)((n + APPLY_WARPS - 1) / APPLY_WARPS);
    k_apply_items<float, double><<<g, APPLY_WARPS * 32, 0, s>>>(L.d_items, n, h->d_pool32, x, h->pN, acc,
                                                                  h->pN, nrhs);
}

static int64_t max_padded_leaf(hm_matrix h)
{
    int64_t maxnp = 0;
    for (int64_t i = 0; i < h->n_leaves; ++i) maxnp = std::max<int64_t>(maxnp, h->pleaf_off[i + 1] - h->pleaf_off[i]);
    return maxnp;
}

void launch_apply_self_acc64(hm_matrix h, const float2 *x, double2 *acc, int nrhs, cudaStream_t s)
{
    dim3 grid((unsigned)h->n_leaves, (unsigned)nrhs);
    k_apply_self<double><<<grid, 256, max_padded_leaf(h) * sizeof(double2), s>>>(h->d_pleaf_off, h->d_dinv_off,
                                                                                h->d_self32, x, acc, h->pN);
}

void launch_apply_self_f32(hm_matrix h, const float2 *x, float2 *acc, int nrhs, cudaStream_t s)
{
    dim3 grid((unsigned)h->n_leaves, (unsigned)nrhs);
    k_apply_self<float><<<grid, 256, max_padded_leaf(h) * sizeof(float2), s>>>(h->d_pleaf_off, h->d_dinv_off,
                                                                              h->d_self32, x, acc, h->pN);
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

void launch_residual(const float2 *b, const double2 *acc, float2 *r, double *norms, int64_t pN, int nrhs,
                     cudaStream_t s)
{
    k_residual<<<grid_for(pN * nrhs), 256, 0, s>>>(b, acc, r, norms, pN, nrhs);
}

void launch_check_finite(const void *x, int64_t n, bool fp64, int *status, cudaStream_t s)
{
    const int g = grid_for(n);
    if (fp64) k_check_finite<double2><<<g, 256, 0, s>>>((const double2 *)x, n, status);
    else k_check_finite<float2><<<g, 256, 0, s>>>((const float2 *)x, n, status);
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
