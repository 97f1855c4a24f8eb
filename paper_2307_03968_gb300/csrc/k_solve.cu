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

// On entry every lane holds v[0..15]; on exit lane l holds in v[0] the sum over
// all 32 lanes of v[l & 15].  16 shuffles per component.
template <class CA>
__device__ __forceinline__ void transpose_reduce16(CA (&v)[16], int lane)
{
#pragma unroll
    for (int s = 8; s >= 1; s >>= 1) {
        const bool up = (lane & s) != 0;
#pragma unroll
        for (int j = 0; j < s; ++j) {
            CA send = up ? v[j] : v[j + s];
            CA keep = up ? v[j + s] : v[j];
            v[j] = cadd(keep, shfl_xor(send, s));
        }
    }
    v[0] = cadd(v[0], shfl_xor(v[0], 16));
}

// On entry every lane holds v[0..3]; on exit lane l holds in v[0] the sum over
// all 32 lanes of v[l & 3].
template <class CA>
__device__ __forceinline__ void reduce4(CA (&v)[4], int lane)
{
#pragma unroll
    for (int s = 2; s >= 1; s >>= 1) {
        const bool up = (lane & s) != 0;
#pragma unroll
        for (int j = 0; j < s; ++j) {
            CA send = up ? v[j] : v[j + s];
            CA keep = up ? v[j + s] : v[j];
            v[j] = cadd(keep, shfl_xor(send, s));
        }
    }
    v[0] = cadd(v[0], shfl_xor(v[0], 4));
    v[0] = cadd(v[0], shfl_xor(v[0], 8));
    v[0] = cadd(v[0], shfl_xor(v[0], 16));
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
template <class T, class A, bool PART>
__device__ __forceinline__ void dense_item(const Item &it, const typename CT<T>::C *__restrict__ pool,
                                           const typename CT<T>::C *__restrict__ x,
                                           typename CT<A>::C *__restrict__ z, typename CT<T>::C *xs, int lane)
{
    // PART: z is this right-hand side's partial buffer; the block's slot is
    // [it.pad, it.pad + even(m)) for the row side and the next even(n) for the
    // column side, written with plain stores (every slot entry is written).
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
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int rb = r0 + 16 * half;
                if (rb >= m) break;
                CA rp[16];
#pragma unroll
                for (int rr = 0; rr < 16; ++rr) {
                    const int i = rb + rr;
                    Pair<T> b{czero(CTy()), czero(CTy())};
                    if (jv && i < m) b = ld_stream(B + (int64_t)i * ld + j);
                    const CA xi = conv<CA>(xs[16 * half + rr]);
                    const CA ba = conv<CA>(b.a), bb = conv<CA>(b.b);
                    cfma(cs0, ba, xi);
                    cfma(cs1, bb, xi);
                    CA t = zero;
                    cfma(t, ba, xj0);
                    cfma(t, bb, xj1);
                    rp[rr] = t;
                }
                transpose_reduce16<CA>(rp, lane);
                const int row = rb + lane;
                if (lane < 16) {
                    if (PART) {
                        if (row < even_d(m)) z[it.pad + row] = rp[0];
                    } else if (row < m) {
                        red1(z + it.row0 + row, rp[0]);
                    }
                }
            }
        }
        if (jv) {
            if (PART) {
                z[it.pad + even_d(m) + j] = cs0;
                z[it.pad + even_d(m) + j + 1] = cs1;
            } else if (j + 1 < n) {
                red2(z + it.col0 + j, cs0, cs1);
            } else {
                red1(z + it.col0 + j, cs0);
            }
        }
    }
}

// Low-rank far block U V with U^T (k x m) and V (k x n) row-major, m and n the
// padded (even) cluster lengths:  z_I += U (V x_J),  z_J += V^T (U^T x_I).
template <class T, class A, bool PART>
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
        for (int l0 = 0; l0 < k; l0 += 4) {
            Pair<T> u[4], v[4];
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                u[l] = {czero(CTy()), czero(CTy())};
                v[l] = u[l];
                if (l0 + l < k) {
                    if (iv) u[l] = ld_stream(UT + (int64_t)(l0 + l) * m + i);
                    if (jv) v[l] = ld_stream(V + (int64_t)(l0 + l) * n + i);
                }
            }
            CA tp[4], t[4];
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                tp[l] = zero;
                cfma(tp[l], conv<CA>(u[l].a), xi0);
                cfma(tp[l], conv<CA>(u[l].b), xi1);
                t[l] = zero;
                cfma(t[l], conv<CA>(v[l].a), xj0);
                cfma(t[l], conv<CA>(v[l].b), xj1);
            }
            reduce4<CA>(tp, lane);
            reduce4<CA>(t, lane);
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                if (l0 + l >= k) break;
                const CA tl = shfl_idx(t[0], l);     // (V x_J)_l
                const CA tpl = shfl_idx(tp[0], l);   // (U^T x_I)_l
                cfma(oi0, conv<CA>(u[l].a), tl);
                cfma(oi1, conv<CA>(u[l].b), tl);
                cfma(oj0, conv<CA>(v[l].a), tpl);
                cfma(oj1, conv<CA>(v[l].b), tpl);
            }
        }
        if (PART) {
            if (iv) { z[it.pad + i] = oi0; z[it.pad + i + 1] = oi1; }
            if (jv) { z[it.pad + m + i] = oj0; z[it.pad + m + i + 1] = oj1; }
        } else {
            if (iv) red2(z + it.row0 + i, oi0, oi1);
            if (jv) red2(z + it.col0 + i, oj0, oj1);
        }
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
                if (PART) {
                    // slots accumulate over rank chunks: first chunk stores, later chunks add
                    if (l0 == 0) { z[it.pad + i] = o0; z[it.pad + i + 1] = o1; }
                    else { z[it.pad + i] = cadd(z[it.pad + i], o0); z[it.pad + i + 1] = cadd(z[it.pad + i + 1], o1); }
                } else {
                    red2(z + it.row0 + i, o0, o1);
                }
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
                if (PART) {
                    CA *q = z + it.pad + m + j;
                    if (l0 == 0) { q[0] = o0; q[1] = o1; }
                    else { q[0] = cadd(q[0], o0); q[1] = cadd(q[1], o1); }
                } else {
                    red2(z + it.col0 + j, o0, o1);
                }
            }
        }
    }
}

template <class T, class A, bool PART>
__global__ void __launch_bounds__(APPLY_WARPS * 32, 2)
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
                dense_item<T, A, PART>(it, pool, x + r * ldx, z + r * ldz, xs_all[w], lane);
            else
                lowrank_item<T, A, PART>(it, pool, x + r * ldx, z + r * ldz, lane);
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

// ---------------------------------------------------------------------------
// FP64-class products for the refinement residual (complex64 data).
//
// GB300 runs FP64 at a small fraction of its FP32 rate, so a full-operator pass
// in FP64 arithmetic costs many times its HBM time.  The residual products
// therefore use error-free transformations in FP32 (Ogita, Rump & Oishi,
// "Accurate sum and dot product", SIAM J. Sci. Comput. 2005, algorithm Dot2):
// every product a*b is split exactly into p + e with e = fma(a, b, -p), and
// every sum is compensated (Knuth's TwoSum), so each block's sums are as
// accurate as if computed in twice the working precision.  The per-block
// results are stored as FP64 partial slots and summed across blocks in FP64.
struct df { float hi, lo; };
struct cdf { df re, im; };

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// acc += a * b  (Dot2 step)
__device__ __forceinline__ void dot2(df &acc, float a, float b)
{
    const float p = a * b;
    const float ep = fmaf(a, b, -p);
    float s, q;
    two_sum(acc.hi, p, s, q);
    acc.hi = s;
    acc.lo += q + ep;
}
// acc += a * b for complex a (FP32) and b (FP32)
__device__ __forceinline__ void cdot2(cdf &acc, float2 a, float2 b)
{
    dot2(acc.re, a.x, b.x);
    dot2(acc.re, -a.y, b.y);
    dot2(acc.im, a.x, b.y);
    dot2(acc.im, a.y, b.x);
}
// acc += a * (bh + bl) for complex a and a double-float complex b
__device__ __forceinline__ void cdot2_df(cdf &acc, float2 a, const cdf &b)
{
    cdot2(acc, a, make_float2(b.re.hi, b.im.hi));
    acc.re.lo += a.x * b.re.lo - a.y * b.im.lo;
    acc.im.lo += a.x * b.im.lo + a.y * b.re.lo;
}
__device__ __forceinline__ df df_add(df a, df b)
{
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e += a.lo + b.lo;
    const float h = s + e;
    return {h, e - (h - s)};
}
__device__ __forceinline__ cdf cdf_add(const cdf &a, const cdf &b) { return {df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ cdf cdf_zero() { return {{0.f, 0.f}, {0.f, 0.f}}; }
__device__ __forceinline__ cdf shfl_xor(const cdf &v, int s)
{
    return {{__shfl_xor_sync(FULL, v.re.hi, s), __shfl_xor_sync(FULL, v.re.lo, s)},
            {__shfl_xor_sync(FULL, v.im.hi, s), __shfl_xor_sync(FULL, v.im.lo, s)}};
}
__device__ __forceinline__ cdf shfl_idx(const cdf &v, int l)
{
    return {{__shfl_sync(FULL, v.re.hi, l), __shfl_sync(FULL, v.re.lo, l)},
            {__shfl_sync(FULL, v.im.hi, l), __shfl_sync(FULL, v.im.lo, l)}};
}
__device__ __forceinline__ double2 to_d2(const cdf &v)
{
    return make_double2((double)v.re.hi + (double)v.re.lo, (double)v.im.hi + (double)v.im.lo);
}
// lane l ends with the sum over all lanes of v[l & (S-1)] in v[0] (S = 8 or 4)
template <int S>
__device__ __forceinline__ void reduce_cdf(cdf (&v)[S], int lane)
{
#pragma unroll
    for (int s = S / 2; s >= 1; s >>= 1) {
        const bool up = (lane & s) != 0;
#pragma unroll
        for (int j = 0; j < s; ++j) {
            const cdf send = up ? v[j] : v[j + s];
            const cdf keep = up ? v[j + s] : v[j];
            v[j] = cdf_add(keep, shfl_xor(send, s));
        }
    }
#pragma unroll
    for (int s = S; s < 32; s <<= 1) v[0] = cdf_add(v[0], shfl_xor(v[0], s));
}

// Dense block: slot rows (even(m)) = B x_J, slot columns (even(n)) = B^T x_I.
__device__ __forceinline__ void dense_item_c(const Item &it, const float2 *__restrict__ pool,
                                             const float2 *__restrict__ x, double2 *__restrict__ part, float2 *xs,
                                             int lane)
{
    const float2 *B = pool + it.off;
    const int m = it.m, n = it.n, ld = even_d(n), em = even_d(m);
    for (int c0 = 0; c0 < n; c0 += 64) {
        const int j = c0 + 2 * lane;
        const bool jv = j < n;
        float2 xj0 = make_float2(0.f, 0.f), xj1 = xj0;
        if (jv) {
            xj0 = x[it.col0 + j];
            if (j + 1 < n) xj1 = x[it.col0 + j + 1];
        }
        cdf cs0 = cdf_zero(), cs1 = cdf_zero();
        for (int r0 = 0; r0 < m; r0 += 32) {
            __syncwarp();
            xs[lane] = (r0 + lane < m) ? x[it.row0 + r0 + lane] : make_float2(0.f, 0.f);
            __syncwarp();
            for (int q = 0; q < 4; ++q) {
                const int rb = r0 + 8 * q;
                if (rb >= m) break;
                cdf rp[8];
#pragma unroll
                for (int rr = 0; rr < 8; ++rr) {
                    const int i = rb + rr;
                    Pair<float> b{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
                    if (jv && i < m) b = ld_stream(B + (int64_t)i * ld + j);
                    const float2 xi = xs[8 * q + rr];
                    cdot2(cs0, b.a, xi);
                    cdot2(cs1, b.b, xi);
                    rp[rr] = cdf_zero();
                    cdot2(rp[rr], b.a, xj0);
                    cdot2(rp[rr], b.b, xj1);
                }
                reduce_cdf<8>(rp, lane);
                const int row = rb + lane;
                if (lane < 8 && row < em) part[it.pad + row] = to_d2(rp[0]);
            }
        }
        if (jv) {
            part[it.pad + em + j] = to_d2(cs0);
            part[it.pad + em + j + 1] = to_d2(cs1);
        }
    }
}

// Low-rank block U V: slot rows (m) = U (V x_J), slot columns (n) = V^T (U^T x_I);
// the rank-k intermediates stay in double-float.
__device__ __forceinline__ void lowrank_item_c(const Item &it, const float2 *__restrict__ pool,
                                               const float2 *__restrict__ x, double2 *__restrict__ part, int lane)
{
    const int m = it.m, n = it.n, k = it.k;
    const float2 *UT = pool + it.off;
    const float2 *V = UT + (int64_t)k * m;
    for (int l0 = 0; l0 < k; l0 += 4) {
        cdf tp[4], t[4];
#pragma unroll
        for (int l = 0; l < 4; ++l) { tp[l] = cdf_zero(); t[l] = cdf_zero(); }
        for (int c0 = 0; c0 < m; c0 += 64) {
            const int i = c0 + 2 * lane;
            if (i >= m) continue;
            const Pair<float> xp = ld_vec(x + it.row0 + i);
#pragma unroll
            for (int l = 0; l < 4; ++l)
                if (l0 + l < k) {
                    const Pair<float> u = ld_cached(UT + (int64_t)(l0 + l) * m + i);
                    cdot2(tp[l], u.a, xp.a);
                    cdot2(tp[l], u.b, xp.b);
                }
        }
        for (int c0 = 0; c0 < n; c0 += 64) {
            const int j = c0 + 2 * lane;
            if (j >= n) continue;
            const Pair<float> xp = ld_vec(x + it.col0 + j);
#pragma unroll
            for (int l = 0; l < 4; ++l)
                if (l0 + l < k) {
                    const Pair<float> v = ld_cached(V + (int64_t)(l0 + l) * n + j);
                    cdot2(t[l], v.a, xp.a);
                    cdot2(t[l], v.b, xp.b);
                }
        }
        reduce_cdf<4>(tp, lane);
        reduce_cdf<4>(t, lane);
        cdf tb[4], tpb[4];
#pragma unroll
        for (int l = 0; l < 4; ++l) { tb[l] = shfl_idx(t[0], l); tpb[l] = shfl_idx(tp[0], l); }
        for (int c0 = 0; c0 < m; c0 += 64) {
            const int i = c0 + 2 * lane;
            if (i >= m) continue;
            cdf o0 = cdf_zero(), o1 = cdf_zero();
#pragma unroll
            for (int l = 0; l < 4; ++l)
                if (l0 + l < k) {
                    const Pair<float> u = ld_cached(UT + (int64_t)(l0 + l) * m + i);
                    cdot2_df(o0, u.a, tb[l]);
                    cdot2_df(o1, u.b, tb[l]);
                }
            double2 *q = part + it.pad + i;
            const double2 a0 = to_d2(o0), a1 = to_d2(o1);
            if (l0 == 0) { q[0] = a0; q[1] = a1; }
            else { q[0] = cadd(q[0], a0); q[1] = cadd(q[1], a1); }
        }
        for (int c0 = 0; c0 < n; c0 += 64) {
            const int j = c0 + 2 * lane;
            if (j >= n) continue;
            cdf o0 = cdf_zero(), o1 = cdf_zero();
#pragma unroll
            for (int l = 0; l < 4; ++l)
                if (l0 + l < k) {
                    const Pair<float> v = ld_cached(V + (int64_t)(l0 + l) * n + j);
                    cdot2_df(o0, v.a, tpb[l]);
                    cdot2_df(o1, v.b, tpb[l]);
                }
            double2 *q = part + it.pad + m + j;
            const double2 a0 = to_d2(o0), a1 = to_d2(o1);
            if (l0 == 0) { q[0] = a0; q[1] = a1; }
            else { q[0] = cadd(q[0], a0); q[1] = cadd(q[1], a1); }
        }
    }
}

__global__ void __launch_bounds__(APPLY_WARPS * 32)
k_residual_items(const Item *__restrict__ items, int64_t n_items, const float2 *__restrict__ pool,
                 const float2 *__restrict__ x, int64_t ldx, double2 *__restrict__ part, int64_t pstride, int nrhs)
{
    __shared__ float2 xs_all[APPLY_WARPS][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t nw = (int64_t)gridDim.x * APPLY_WARPS;
    for (int64_t t = (int64_t)blockIdx.x * APPLY_WARPS + w; t < n_items; t += nw) {
        const Item it = items[t];
        for (int r = 0; r < nrhs; ++r) {
            if (it.k == 0) dense_item_c(it, pool, x + r * ldx, part + r * pstride, xs_all[w], lane);
            else lowrank_item_c(it, pool, x + r * ldx, part + r * pstride, lane);
        }
    }
}

// Per leaf (blockIdx.x) and right-hand side (blockIdx.y): acc = D_I x_I +
// sum of the leaf's partial slots of levels 1..m, in FP64 and in a fixed order
// (each of the 4 warps sums every 4th slot, lanes own row pairs; the warps are
// then added in warp order).  If b is given, out = b - acc (complex64) and
// |r|^2, |b|^2 go to norms; else out = acc (complex64).  No atomics on sums.
__global__ void __launch_bounds__(128)
k_gather_acc64(const int32_t *__restrict__ pleaf_off, const int64_t *__restrict__ dinv_off,
               const float2 *__restrict__ self32, const float2 *__restrict__ x, int64_t ld,
               const int64_t *__restrict__ csr_off, int csr_stride, int m, const int64_t *__restrict__ csr_idx,
               const double2 *__restrict__ part, int64_t pstride, const float2 *__restrict__ b,
               float2 *__restrict__ out, double *norms)
{
    constexpr int MAXR = 128;
    __shared__ double2 acc_s[4][MAXR];
    __shared__ double2 xs[MAXR];
    __shared__ double red[2][4];
    const int leaf = blockIdx.x, r = blockIdx.y;
    const int o = pleaf_off[leaf], np = pleaf_off[leaf + 1] - o;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (int j = tid; j < np; j += blockDim.x) xs[j] = conv<double2>(x[r * ld + o + j]);
    __syncthreads();
    const double2 *P = part + r * pstride;
    const int64_t e0 = csr_off[(int64_t)leaf * csr_stride], e1 = csr_off[(int64_t)leaf * csr_stride + m];
    for (int rc = 0; rc < np; rc += 64) {
        const int i = rc + 2 * lane;
        double2 a0 = make_double2(0, 0), a1 = make_double2(0, 0);
        if (i < np) {
            int64_t e = e0 + w;
            for (; e + 12 < e1; e += 16) {      // four slots in flight per warp
                const int64_t q0 = csr_idx[e], q1 = csr_idx[e + 4], q2 = csr_idx[e + 8], q3 = csr_idx[e + 12];
                const double2 v00 = P[q0 + i], v01 = P[q0 + i + 1], v10 = P[q1 + i], v11 = P[q1 + i + 1];
                const double2 v20 = P[q2 + i], v21 = P[q2 + i + 1], v30 = P[q3 + i], v31 = P[q3 + i + 1];
                a0 = cadd(a0, cadd(cadd(v00, v10), cadd(v20, v30)));
                a1 = cadd(a1, cadd(cadd(v01, v11), cadd(v21, v31)));
            }
            for (; e < e1; e += 4) {
                const int64_t q = csr_idx[e];
                a0 = cadd(a0, P[q + i]);
                a1 = cadd(a1, P[q + i + 1]);
            }
            if (w == 0) {   // the self block, FP64
                const float2 *S = self32 + dinv_off[leaf];   // column-major
                for (int j = 0; j < np; ++j) {
                    const Pair<float> d = ld_vec(S + (int64_t)j * np + i);
                    cfma(a0, conv<double2>(d.a), xs[j]);
                    cfma(a1, conv<double2>(d.b), xs[j]);
                }
            }
        }
        acc_s[w][2 * lane] = a0;
        acc_s[w][2 * lane + 1] = a1;
        __syncthreads();
        double rr = 0.0, bb = 0.0;
        if (tid < 64 && rc + tid < np) {
            double2 acc = acc_s[0][tid];
            for (int q = 1; q < 4; ++q) acc = cadd(acc, acc_s[q][tid]);
            const int64_t g = r * ld + o + rc + tid;
            if (b) {
                const double2 bv = conv<double2>(b[g]);
                const double2 rv = csub(bv, acc);
                out[g] = make_float2((float)rv.x, (float)rv.y);
                rr = rv.x * rv.x + rv.y * rv.y;
                bb = bv.x * bv.x + bv.y * bv.y;
            } else {
                out[g] = make_float2((float)acc.x, (float)acc.y);
            }
        }
        if (norms && tid < 64) {
            for (int s = 16; s >= 1; s >>= 1) {
                rr += __shfl_xor_sync(FULL, rr, s);
                bb += __shfl_xor_sync(FULL, bb, s);
            }
            if (lane == 0) {
                atomicAdd(&norms[2 * r], rr);
                atomicAdd(&norms[2 * r + 1], bb);
            }
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

template <class T, class A, bool PART>
int apply_grid(hm_matrix h)
{
    static int per_sm = -1;
    if (per_sm < 0) {
        int v = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_apply_items<T, A, PART>, APPLY_WARPS * 32, 0);
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
        int g = apply_grid<double, double, false>(h);
        if ((int64_t)g * APPLY_WARPS > n) g = (int)((n + APPLY_WARPS - 1) / APPLY_WARPS);
        k_apply_items<double, double, false><<<g, APPLY_WARPS * 32, 0, s>>>(
            L.d_items, n, h->d_pool64, (const double2 *)x, h->pN, (double2 *)z, h->pN, nrhs);
    } else {
        int g = apply_grid<float, float, false>(h);
        if ((int64_t)g * APPLY_WARPS > n) g = (int)((n + APPLY_WARPS - 1) / APPLY_WARPS);
        k_apply_items<float, float, false><<<g, APPLY_WARPS * 32, 0, s>>>(
            L.d_items, n, h->d_pool32, (const float2 *)x, h->pN, (float2 *)z, h->pN, nrhs);
    }
}

void launch_apply_items_partials(hm_matrix h, const LevelList &L, const float2 *x, double2 *part, int64_t pstride,
                                 int nrhs, cudaStream_t s)
{
    const int64_t n = (int64_t)L.items.size();
    if (n == 0) return;
    static int per_sm = -1;
    if (per_sm < 0) {
        int v = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_residual_items, APPLY_WARPS * 32, 0);
        per_sm = v > 0 ? v : 1;
    }
    int g = per_sm * (h->num_sms > 0 ? h->num_sms : 1);
    if ((int64_t)g * APPLY_WARPS > n) g = (int)((n + APPLY_WARPS - 1) / APPLY_WARPS);
    k_residual_items<<<g, APPLY_WARPS * 32, 0, s>>>(L.d_items, n, h->d_pool32, x, h->pN, part, pstride, nrhs);
}

void launch_gather_acc64(hm_matrix h, const float2 *x, int m, const double2 *part, int64_t pstride,
                         const float2 *b, float2 *out, double *norms, int nrhs, cudaStream_t s)
{
    dim3 grid((unsigned)h->n_leaves, (unsigned)nrhs);
    const int64_t maxnp = [&] {
        int64_t v = 0;
        for (int64_t i = 0; i < h->n_leaves; ++i) v = std::max<int64_t>(v, h->pleaf_off[i + 1] - h->pleaf_off[i]);
        return v;
    }();
    (void)maxnp;
    k_gather_acc64<<<grid, 128, 0, s>>>(h->d_pleaf_off, h->d_dinv_off, h->d_self32, x, h->pN,
                                                              h->d_csr_off, h->n_levels + 1, m, h->d_csr_idx, part,
                                                              pstride, b, out, norms);
}

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

void launch_convert_f32_to_f64(const float2 *a, double2 *b, int64_t n, cudaStream_t s)
{
    k_f32_to_f64<<<grid_for(n), 256, 0, s>>>(a, b, n);
}

void launch_convert_f64_to_f32(const double2 *a, float2 *b, int64_t n, cudaStream_t s)
{
    k_f64_to_f32<<<grid_for(n), 256, 0, s>>>(a, b, n);
}

} // namespace hm
