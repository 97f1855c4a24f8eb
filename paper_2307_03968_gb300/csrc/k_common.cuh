// Device helpers shared by the solve kernels: complex arithmetic on float2 /
// double2, 128-bit pair loads, vector reductions into z, and warp transpose
// reductions (a lane ends up holding the sum over the warp of one of the
// values every lane held).
#pragma once

#include "hm_internal.h"

namespace hm {
namespace kc {

constexpr unsigned FULL = 0xffffffffu;

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


} // namespace kc
} // namespace hm
