// Device bodies of the FP64-class residual r = b - A_m x (the refinement step's
// residual, computed to FP64-class accuracy over complex64 blocks): the
// products of one stored block into its double-float partial slots (one warp
// per block), and the per-leaf gather of the slots with D_I x_I.  Used by the
// residual kernels (k_residual.cu) and by the one-launch solve (k_persist.cu).
// HM_XR qualifies the pointers of data written during a solve: __restrict__ in
// the residual kernels; empty in the one-launch solve, whose vectors and slots
// are written by other CTAs between its phases.
#pragma once

#include "k_dot2.cuh"

#ifndef HM_XR
#define HM_XR __restrict__
#endif

namespace hm {
namespace {

using namespace kc;
using namespace dot2;

// Dense block: slot rows (even(m)) = B x_J, slot columns (even(n)) = B^T x_I.
// A lane owns two adjacent columns.  Row side: per row, the lane's two terms form
// one short error-free chain, then the lanes' double-float sums are reduced.
// Column side: chains over four rows at a time, folded into a double-float sum.
__device__ __forceinline__ void dense_item_c(const Item &it, const float2 *__restrict__ pool,
                                             const float2 *HM_XR x, cdf *HM_XR part, float2 *xs,
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
        const float mxj = fmaxf(linf(xj0), linf(xj1));
        cdf cs0 = cdf_zero(), cs1 = cdf_zero();
        for (int r0 = 0; r0 < m; r0 += 32) {
            __syncwarp();
            xs[lane] = (r0 + lane < m) ? x[it.row0 + r0 + lane] : make_float2(0.f, 0.f);
            __syncwarp();
            for (int q = 0; q < 4; ++q) {
                const int rb = r0 + 8 * q;
                if (rb >= m) break;
                Pair<float> b[8];
#pragma unroll
                for (int rr = 0; rr < 8; ++rr) {
                    b[rr] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
                    if (jv && rb + rr < m) b[rr] = ld_stream(B + (int64_t)(rb + rr) * ld + j);
                }
                cdf rp[8];
#pragma unroll
                for (int rr = 0; rr < 8; ++rr) {
                    const float sg = chain_sigma(__fadd_rn(l1(b[rr].a), l1(b[rr].b)), mxj);
                    cxacc c;
                    cxfirst(c, sg, b[rr].a, xj0);
                    cxstep(c, b[rr].b, xj1);
                    rp[rr] = cxclose(c, sg);
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float2 xi[4];
                    float mxi = 0.f, sa0 = 0.f, sa1 = 0.f;
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        xi[u] = xs[8 * q + 4 * h + u];
                        mxi = fmaxf(mxi, linf(xi[u]));
                        sa0 = __fadd_rn(sa0, l1(b[4 * h + u].a));
                        sa1 = __fadd_rn(sa1, l1(b[4 * h + u].b));
                    }
                    const float s0 = chain_sigma(sa0, mxi), s1 = chain_sigma(sa1, mxi);
                    cxacc k0, k1;
                    cxfirst(k0, s0, b[4 * h].a, xi[0]);
                    cxfirst(k1, s1, b[4 * h].b, xi[0]);
#pragma unroll
                    for (int u = 1; u < 4; ++u) {
                        cxstep(k0, b[4 * h + u].a, xi[u]);
                        cxstep(k1, b[4 * h + u].b, xi[u]);
                    }
                    cs0 = cdf_add(cs0, cxclose(k0, s0));
                    cs1 = cdf_add(cs1, cxclose(k1, s1));
                }
                reduce_cdf<8>(rp, lane);
                const int row = rb + lane;
                // a block wider than 64 columns is swept in column chunks: the row slot
                // takes the first chunk's sums and then adds the next ones (same lane, in order)
                if (lane < 8 && row < em) part[it.pad + row] = c0 == 0 ? rp[0] : cdf_add(part[it.pad + row], rp[0]);
            }
        }
        if (jv) {
            part[it.pad + em + j] = cs0;
            part[it.pad + em + j + 1] = cs1;
        }
    }
}

// Low-rank block U V: slot rows (m) = U (V x_J), slot columns (n) = V^T (U^T x_I);
// the rank-k intermediates stay in double-float.  Blocks of up to 64 x 64 use the
// short biased chains, larger ones Dot2.
__device__ __forceinline__ void lowrank_item_c(const Item &it, const float2 *__restrict__ pool,
                                               const float2 *HM_XR x, cdf *HM_XR part, int lane)
{
    const int m = it.m, n = it.n, k = it.k;
    const float2 *UT = pool + it.off;
    const float2 *V = UT + (int64_t)k * m;
    if (m <= 64 && n <= 64) {
        // registers hold a chunk of 4 rank rows of both panels; outputs stay in
        // registers across chunks and are stored once
        const int i = 2 * lane;
        const bool iv = i < m, jv = i < n;
        Pair<float> xi{make_float2(0.f, 0.f), make_float2(0.f, 0.f)}, xj = xi;
        if (iv) xi = ld_vec(x + it.row0 + i);
        if (jv) xj = ld_vec(x + it.col0 + i);
        const float mxi = fmaxf(linf(xi.a), linf(xi.b)), mxj = fmaxf(linf(xj.a), linf(xj.b));
        cdf oi0 = cdf_zero(), oi1 = cdf_zero(), oj0 = cdf_zero(), oj1 = cdf_zero();
        for (int l0 = 0; l0 < k; l0 += 4) {
            Pair<float> u[4], v[4];
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                u[l] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
                v[l] = u[l];
                if (l0 + l < k) {
                    if (iv) u[l] = ld_stream(UT + (int64_t)(l0 + l) * m + i);
                    if (jv) v[l] = ld_stream(V + (int64_t)(l0 + l) * n + i);
                }
            }
            // stage 1: the lane's two terms of every rank row as one short chain,
            // then the lanes' double-float sums reduced (rank rows past k are zero)
            cdf tp[4], t[4];
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const float su = chain_sigma(__fadd_rn(l1(u[l].a), l1(u[l].b)), mxi);
                const float sv = chain_sigma(__fadd_rn(l1(v[l].a), l1(v[l].b)), mxj);
                cxacc cu, cv;
                cxfirst(cu, su, u[l].a, xi.a);
                cxstep(cu, u[l].b, xi.b);
                cxfirst(cv, sv, v[l].a, xj.a);
                cxstep(cv, v[l].b, xj.b);
                tp[l] = cxclose(cu, su);
                t[l] = cxclose(cv, sv);
            }
            reduce_cdf<4>(tp, lane);
            reduce_cdf<4>(t, lane);
            // stage 2: one chain over the chunk's rank rows per output, folded
            cdf tl[4], tpl[4];
            float mt = 0.f, mtp = 0.f, si0 = 0.f, si1 = 0.f, sj0 = 0.f, sj1 = 0.f;
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                tl[l] = shfl_idx(t[0], l);
                tpl[l] = shfl_idx(tp[0], l);
                mt = fmaxf(mt, fmaxf(fabsf(tl[l].re.hi), fabsf(tl[l].im.hi)));
                mtp = fmaxf(mtp, fmaxf(fabsf(tpl[l].re.hi), fabsf(tpl[l].im.hi)));
                si0 = __fadd_rn(si0, l1(u[l].a));
                si1 = __fadd_rn(si1, l1(u[l].b));
                sj0 = __fadd_rn(sj0, l1(v[l].a));
                sj1 = __fadd_rn(sj1, l1(v[l].b));
            }
            si0 = chain_sigma(si0, mt);
            si1 = chain_sigma(si1, mt);
            sj0 = chain_sigma(sj0, mtp);
            sj1 = chain_sigma(sj1, mtp);
            cxacc ci0, ci1, cj0, cj1;
            cxfirst_df(ci0, si0, u[0].a, tl[0]);
            cxfirst_df(ci1, si1, u[0].b, tl[0]);
            cxfirst_df(cj0, sj0, v[0].a, tpl[0]);
            cxfirst_df(cj1, sj1, v[0].b, tpl[0]);
#pragma unroll
            for (int l = 1; l < 4; ++l) {
                cxstep_df(ci0, u[l].a, tl[l]);
                cxstep_df(ci1, u[l].b, tl[l]);
                cxstep_df(cj0, v[l].a, tpl[l]);
                cxstep_df(cj1, v[l].b, tpl[l]);
            }
            oi0 = cdf_add(oi0, cxclose(ci0, si0));
            oi1 = cdf_add(oi1, cxclose(ci1, si1));
            oj0 = cdf_add(oj0, cxclose(cj0, sj0));
            oj1 = cdf_add(oj1, cxclose(cj1, sj1));
        }
        if (iv) { part[it.pad + i] = oi0; part[it.pad + i + 1] = oi1; }
        if (jv) { part[it.pad + m + i] = oj0; part[it.pad + m + i + 1] = oj1; }
        return;
    }
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
            cdf *q = part + it.pad + i;
            if (l0 == 0) { q[0] = o0; q[1] = o1; }
            else { q[0] = cdf_add(q[0], o0); q[1] = cdf_add(q[1], o1); }
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
            cdf *q = part + it.pad + m + j;
            if (l0 == 0) { q[0] = o0; q[1] = o1; }
            else { q[0] = cdf_add(q[0], o0); q[1] = cdf_add(q[1], o1); }
        }
    }
}

// Per leaf and right-hand side: acc = D_I x_I +
// sum of the leaf's partial slots of levels 1..m, in double-float arithmetic and
// in a fixed order (each of the GW warps sums every GW-th slot with compensated
// additions and takes every GW-th column of D_I x_I in Dot2; lanes own row pairs;
// the warps are then added in warp order).  If b is given, out = b - acc (in FP64,
// rounded to complex64) and |r|^2, |b|^2 go to norms; else out = acc (complex64).
// No atomics on sums.
// The body for one (leaf, right-hand side) pair, run by a CTA of GW warps;
// acc_s and xs (the leaf's x, np entries) are shared-memory buffers of the caller.
constexpr int GW = 8;   // warps per leaf
__device__ __forceinline__ void gather_leaf(int leaf, int r, const int32_t *__restrict__ pleaf_off,
                                            const int64_t *__restrict__ dinv_off, const float2 *__restrict__ self32,
                                            const float2 *HM_XR x, int64_t ld, const int64_t *__restrict__ csr_off,
                                            int csr_stride, int m, const int64_t *__restrict__ csr_idx,
                                            const cdf *HM_XR part, int64_t pstride, const float2 *HM_XR b,
                                            float2 *HM_XR out, double *norms, cdf (*acc_s)[64], float2 *xs)
{
    const int o = pleaf_off[leaf], np = pleaf_off[leaf + 1] - o;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (int j = tid; j < np; j += blockDim.x) xs[j] = x[r * ld + o + j];
    __syncthreads();
    const cdf *P = part + r * pstride;
    const int64_t e0 = csr_off[(int64_t)leaf * csr_stride], e1 = csr_off[(int64_t)leaf * csr_stride + m];
    const float2 *S = self32 + dinv_off[leaf];                      // column-major np x np
    for (int rc = 0; rc < np; rc += 64) {
        const int i = rc + 2 * lane;
        cdf a0 = cdf_zero(), a1 = cdf_zero();
        if (i < np) {
            int64_t e = e0 + w;
            for (; e + 3 * GW < e1; e += 4 * GW) {   // four slots in flight per warp
                const int64_t q0 = csr_idx[e], q1 = csr_idx[e + GW], q2 = csr_idx[e + 2 * GW], q3 = csr_idx[e + 3 * GW];
                const cdf v00 = P[q0 + i], v01 = P[q0 + i + 1], v10 = P[q1 + i], v11 = P[q1 + i + 1];
                const cdf v20 = P[q2 + i], v21 = P[q2 + i + 1], v30 = P[q3 + i], v31 = P[q3 + i + 1];
                a0 = cdf_add(a0, cdf_add(cdf_add(v00, v10), cdf_add(v20, v30)));
                a1 = cdf_add(a1, cdf_add(cdf_add(v01, v11), cdf_add(v21, v31)));
            }
            for (; e < e1; e += GW) {
                const int64_t q = csr_idx[e];
                a0 = cdf_add(a0, P[q + i]);
                a1 = cdf_add(a1, P[q + i + 1]);
            }
            for (int j = w; j < np; j += GW) {      // the self block, Dot2, every GW-th column
                const Pair<float> d = ld_vec(S + (int64_t)j * np + i);
                cdot2(a0, d.a, xs[j]);
                cdot2(a1, d.b, xs[j]);
            }
        }
        acc_s[w][2 * lane] = a0;
        acc_s[w][2 * lane + 1] = a1;
        __syncthreads();
        double rr = 0.0, bb = 0.0;
        if (tid < 64 && rc + tid < np) {
            cdf accf = acc_s[0][tid];
            for (int q = 1; q < GW; ++q) accf = cdf_add(accf, acc_s[q][tid]);
            const double2 acc = to_d2(accf);
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

} // namespace
} // namespace hm
