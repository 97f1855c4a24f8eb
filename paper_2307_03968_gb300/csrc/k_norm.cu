// Small kernels of the level-operator norm estimate (arxiv 2307.03968 §IV:
// the power series of (I + U)^{-1}, U = D^{-1} M_l, converges when the
// spectral radius of U is below one; the paper states its operating bound as a
// norm below 0.1).  The estimate itself (power iterations on U and on U^H U,
// driven from hm_api.cu with the product and leaf-inverse kernels) needs:
//  k_seed_vector   a deterministic start vector in padded tree order (zero pads)
//  k_norm2         |v|^2 accumulated in FP64 into one device double
//  k_conj_scale    dst = op(src) / sqrt(*nrm2), op = identity or conjugation
#include "k_common.cuh"

#include <cuda_runtime.h>

namespace hm {
namespace {

// counter-based hash of (seed, index) to a float in [-1, 1): the start vector of the
// power iterations only has to be generic (not orthogonal to the dominant vectors)
__device__ __forceinline__ float hash_unit(uint32_t seed, uint32_t i)
{
    uint32_t v = i * 0x9E3779B9u ^ (seed + 0x7F4A7C15u);
    v ^= v >> 16; v *= 0x85EBCA6Bu;
    v ^= v >> 13; v *= 0xC2B2AE35u;
    v ^= v >> 16;
    return (float)(v >> 8) * (2.0f / 16777216.0f) - 1.0f;
}

__global__ void k_seed_vector(float2 *v, const int32_t *__restrict__ pperm, int64_t pN, uint32_t seed)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < pN; t += (int64_t)gridDim.x * blockDim.x)
        v[t] = pperm[t] >= 0 ? make_float2(hash_unit(seed, (uint32_t)(2 * t)), hash_unit(seed, (uint32_t)(2 * t + 1)))
                             : make_float2(0.f, 0.f);
}

__global__ void __launch_bounds__(256) k_norm2(const float2 *__restrict__ v, int64_t n, double *out)
{
    double s = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const float2 a = v[t];
        s += (double)a.x * a.x + (double)a.y * a.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double ws[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) ws[w] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) b += ws[q];
        atomicAdd(out, b);
    }
}

__global__ void k_conj_scale(const float2 *src, float2 *dst, int64_t n, const double *nrm2, int conj)
{
    const double q = *nrm2;
    const float f = q > 0.0 ? (float)(1.0 / sqrt(q)) : 0.0f;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const float2 a = src[t];
        dst[t] = make_float2(a.x * f, conj ? -a.y * f : a.y * f);
    }
}

int grid_norm(int64_t n)
{
    int64_t g = (n + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 1024));
}

} // namespace

void launch_seed_vector(float2 *v, const int32_t *pperm, int64_t pN, uint32_t seed, cudaStream_t s)
{
    k_seed_vector<<<grid_norm(pN), 256, 0, s>>>(v, pperm, pN, seed);
}

void launch_norm2(const float2 *v, int64_t n, double *out, cudaStream_t s)
{
    cudaMemsetAsync(out, 0, sizeof(double), s);
    k_norm2<<<grid_norm(n), 256, 0, s>>>(v, n, out);
}

void launch_conj_scale(const float2 *src, float2 *dst, int64_t n, const double *nrm2, bool conj, cudaStream_t s)
{
    k_conj_scale<<<grid_norm(n), 256, 0, s>>>(src, dst, n, nrm2, conj ? 1 : 0);
}

} // namespace hm
