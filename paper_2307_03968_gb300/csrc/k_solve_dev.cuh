// Device body of the series accumulate (arxiv 2307.03968 eqs. 20-22: x_j = y -
// D^{-1} z) for one leaf, shared by the leaf-update kernel (k_solve.cu) and the
// one-launch solve (k_persist.cu).  Its vector pointers carry no __restrict__:
// in the one-launch solve they are written by other CTAs between phases.
#pragma once

#include "k_common.cuh"

namespace hm {
namespace {

using namespace kc;

// Per leaf and right-hand side, by a CTA of 256 threads (zs: np entries and part:
// shared-memory buffers of the caller):
//   w = D_i^{-1} zin_i ;  out_i = y ? y_i - w : w ;  zin_i = 0 if zero_in.
// D_i^{-1} is column-major np x np (np = padded leaf length), zero padded.
template <class T>
__device__ __forceinline__ void leaf_update_leaf(int leaf, int r, const int32_t *__restrict__ pleaf_off,
                                                 const int64_t *__restrict__ dinv_off,
                                                 const typename CT<T>::C *__restrict__ dinv,
                                                 const typename CT<T>::C *y, typename CT<T>::C *zin,
                                                 typename CT<T>::C *out, int64_t ld, int zero_in,
                                                 typename CT<T>::C *zs, typename CT<T>::C (*part)[64])
{
    using C = typename CT<T>::C;
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

} // namespace
} // namespace hm
