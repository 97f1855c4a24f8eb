// Device bodies of the block product z += M x for one stored block (arxiv
// 2307.03968 eq. 6 and eq. 8, with the half storage of §III: every stored
// block is read once and acts on both of its clusters), one warp per block:
//     dense  B (I,J):  z_I += B x_J,            z_J += B^T x_I
//     low rank U V:    z_I += U (V x_J),        z_J += V^T (U^T x_I)
// Used by the product kernel (k_product.cu) and by the one-launch solve
// (k_persist.cu).  HM_XR qualifies the vector pointers: __restrict__ in the
// product kernel; empty in the one-launch solve, whose vectors are written by
// other CTAs between its phases (no loads through the non-coherent path).
#pragma once

#include "k_common.cuh"

#ifndef HM_XR
#define HM_XR __restrict__
#endif

namespace hm {
namespace {

using namespace kc;

// Dense near block B (m x n, row-major, stride even(n)) between leaves I (rows)
// and J (columns):  z_I += B x_J,  z_J += B^T x_I.
template <class T, class A>
__device__ __forceinline__ void dense_item(const Item &it, const typename CT<T>::C *__restrict__ pool,
                                           const typename CT<T>::C *HM_XR x,
                                           typename CT<A>::C *HM_XR z, typename CT<T>::C *xs, int lane)
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
                if (lane < 16 && row < m) red1(z + it.row0 + row, rp[0]);
            }
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
                                             const typename CT<T>::C *HM_XR x,
                                             typename CT<A>::C *HM_XR z, int lane)
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

} // namespace
} // namespace hm
