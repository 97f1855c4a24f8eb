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

// ---------------------------------------------------------------------------
// Blocks of up to 64 x 64 (dense, or low-rank of any rank) on common grids: every output sum of a
// block side takes one sigma from the block's precomputed bound (k_item_bounds:
// largest row / column 1-norm) and the largest input component, so the lanes'
// grid parts add exactly in plain FP32 (k_dot2.cuh).  The warp covers the block
// as 4 row groups x 8 column groups: lane (rg, cg) takes rows i = 4 s + rg and
// the column pairs (16 t + 2 cg, +1), t = 0..3, so that each row is summed over 8
// lanes and each column over 4 (instead of a 32-lane double-float reduction per
// row), and every load of a row quarter is one 128-byte segment.
constexpr int GRID_MAX = 64;

// one row quarter of a dense block: the lane's column pairs of row i (zero past the block)
__device__ __forceinline__ void grid_row_load(Pair<float> (&b)[4], const float2 *__restrict__ A, int i, int rows,
                                              int cols, int ld, int cg)
{
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        b[t] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        if (i < rows && 16 * t + 2 * cg < cols) b[t] = ld_stream(A + (int64_t)i * ld + 16 * t + 2 * cg);
    }
}

// One row of the dense common-grid pass: the row's sum over the lane's 8 columns
// (one chain), reduced over the row group's 8 lanes and written to rdst[i] (i < rlim),
// and the row's terms added to the lane's 8 column chains.
__device__ __forceinline__ void grid_row(const Pair<float> (&b)[4], int i, int rows, const float2 (&u)[4][2],
                                         float sR, cdf *rdst, int rlim, const float2 *v, cxacc (&acc)[4][2], int lane)
{
    const int cg = lane & 7;
    cxacc c;
    cx_start(c, sR);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        cxstep(c, b[t].a, u[t][0]);
        cxstep(c, b[t].b, u[t][1]);
    }
    if (i < rows) {
        const float2 vi = v[i];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            cxstep(acc[t][0], b[t].a, vi);
            cxstep(acc[t][1], b[t].b, vi);
        }
    }
    float rv[4] = {__fsub_rn(c.re.tau, sR), c.re.r, __fsub_rn(c.im.tau, sR), c.im.r};
    // value index bit 1 (re / im) by cg bit 2, bit 0 (grid part / remainder) by cg bit 1,
    // then the pair of lanes cg, cg ^ 1 adds its two partial sums
    xreduce_step<2>(rv, lane, 4);
    xreduce_step<1>(rv, lane, 2);
    rv[0] = __fadd_rn(rv[0], __shfl_xor_sync(FULL, rv[0], 1));
    if ((cg & 1) == 0 && i < rlim) reinterpret_cast<float *>(rdst + i)[2 * ((cg >> 2) & 1) + ((cg >> 1) & 1)] = rv[0];
}

// Dense block of at most 64 x 64 on common grids, one pass: rsum_i = sum_j A_ij u_j
// (grid sR, to rdst[i] for i < rlim) and csum_j = sum_i A_ij v_i (grid sC, to
// cdst[j], cdst[j + 1] for even j < cols).  A row-major, rows x cols, row stride ld;
// each row is loaded one row ahead of its arithmetic.
__device__ __forceinline__ void grid_pass(const float2 *__restrict__ A, int rows, int cols, int ld,
                                          const float2 (&u)[4][2], float sR, cdf *rdst, int rlim, const float2 *v,
                                          float sC, cdf *cdst, int lane)
{
    const int cg = lane & 7, rg = lane >> 3;
    cxacc acc[4][2];
#pragma unroll
    for (int t = 0; t < 4; ++t) { cx_start(acc[t][0], sC); cx_start(acc[t][1], sC); }
    const int ns = (rows + 3) >> 2;
    Pair<float> b0[4], b1[4];
    grid_row_load(b0, A, rg, rows, cols, ld, cg);
#pragma unroll 1
    for (int s = 0; s < ns; s += 2) {
        const int i = 4 * s + rg;
        grid_row_load(b1, A, i + 4, rows, cols, ld, cg);
        grid_row(b0, i, rows, u, sR, rdst, rlim, v, acc, lane);
        if (s + 1 < ns) {
            grid_row_load(b0, A, i + 8, rows, cols, ld, cg);
            grid_row(b1, i + 4, rows, u, sR, rdst, rlim, v, acc, lane);
        }
    }
    float w[32];
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            w[8 * t + 4 * e] = __fsub_rn(acc[t][e].re.tau, sC);
            w[8 * t + 4 * e + 1] = acc[t][e].re.r;
            w[8 * t + 4 * e + 2] = __fsub_rn(acc[t][e].im.tau, sC);
            w[8 * t + 4 * e + 3] = acc[t][e].im.r;
        }
    // over the column group's 4 lanes: index bit 4 (t bit 1) by rg bit 1, bit 3 (t bit 0)
    // by rg bit 0, so lane (rg, cg) ends with its pair of t = rg
    xreduce_step<16>(w, lane, 16);
    xreduce_step<8>(w, lane, 8);
    const int j = 16 * rg + 2 * cg;
    if (j < cols) {
        cdst[j] = {{w[0], w[1]}, {w[2], w[3]}};
        cdst[j + 1] = {{w[4], w[5]}, {w[6], w[7]}};
    }
}

// the lane's column-pair inputs x[16 t + 2 cg], x[... + 1] (pairs at j < len) and the
// largest input component over the warp
__device__ __forceinline__ float grid_inputs(const float2 *HM_XR x, int len, float2 (&u)[4][2], int lane)
{
    const int cg = lane & 7;
    float mx = 0.f;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int j = 16 * t + 2 * cg;
        u[t][0] = u[t][1] = make_float2(0.f, 0.f);
        if (j < len) {
            u[t][0] = x[j];
            if (j + 1 < len) u[t][1] = x[j + 1];
        }
        mx = fmaxf(mx, fmaxf(linf(u[t][0]), linf(u[t][1])));
    }
    return warp_max(mx);
}

// Dense block of at most 64 x 64: slot rows (even(m)) = B x_J, slot columns
// (even(n)) = B^T x_I.  bnd.x / bnd.y: largest row / column 1-norm of B.
__device__ __forceinline__ void dense_item_g(const Item &it, float4 bnd, const float2 *__restrict__ pool,
                                             const float2 *HM_XR x, cdf *HM_XR part, float2 *xs, int lane)
{
    const int m = it.m, n = it.n;
    float2 u[4][2];
    const float mxj = grid_inputs(x + it.col0, n, u, lane);
    __syncwarp();
    const float2 xa = 2 * lane < m ? x[it.row0 + 2 * lane] : make_float2(0.f, 0.f);
    const float2 xb = 2 * lane + 1 < m ? x[it.row0 + 2 * lane + 1] : make_float2(0.f, 0.f);
    xs[2 * lane] = xa;
    xs[2 * lane + 1] = xb;
    const float mxi = warp_max(fmaxf(linf(xa), linf(xb)));
    __syncwarp();
    grid_pass(pool + it.off, m, n, even_d(n), u, grid_sigma(bnd.x, mxj), part + it.pad, even_d(m), xs,
              grid_sigma(bnd.y, mxi), part + it.pad + even_d(m), lane);
}

// the lane's two columns (i, i + 1) of the rank rows l0, l0 + 1 of U^T and V (zero
// past the rank or the panel)
__device__ __forceinline__ void lr_load(Pair<float> (&u)[2], Pair<float> (&v)[2], const float2 *__restrict__ UT,
                                        const float2 *__restrict__ V, int l0, int k, int m, int n, int i, bool iv,
                                        bool jv)
{
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        u[l] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        v[l] = u[l];
        if (l0 + l < k) {
            if (iv) u[l] = ld_stream(UT + (int64_t)(l0 + l) * m + i);
            if (jv) v[l] = ld_stream(V + (int64_t)(l0 + l) * n + i);
        }
    }
}

// one pair of rank rows l0, l0 + 1 of a low-rank block (u: U^T, v: V, the lane's two
// columns each): stage 1 on the common grids s1u, s1v, reduced over the warp, then
// the pair's rank rows into the outputs' stage-2 chains
__device__ __forceinline__ void lr_pair(const Pair<float> (&u)[2], const Pair<float> (&v)[2], const Pair<float> &xi,
                                        const Pair<float> &xj, float s1u, float s1v, cxacc &ci0, cxacc &ci1,
                                        cxacc &cj0, cxacc &cj1, int lane)
{
    // value index 4 l + (grid re, rem re, grid im, rem im)
    float gu[8], gv[8];
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        cxacc cu, cv;
        cx_start(cu, s1u);
        cxstep(cu, u[l].a, xi.a);
        cxstep(cu, u[l].b, xi.b);
        cx_start(cv, s1v);
        cxstep(cv, v[l].a, xj.a);
        cxstep(cv, v[l].b, xj.b);
        gu[4 * l] = __fsub_rn(cu.re.tau, s1u);
        gu[4 * l + 1] = cu.re.r;
        gu[4 * l + 2] = __fsub_rn(cu.im.tau, s1u);
        gu[4 * l + 3] = cu.im.r;
        gv[4 * l] = __fsub_rn(cv.re.tau, s1v);
        gv[4 * l + 1] = cv.re.r;
        gv[4 * l + 2] = __fsub_rn(cv.im.tau, s1v);
        gv[4 * l + 3] = cv.im.r;
    }
    // over the warp: index bits 2..0 by lane bits 4..2, then the four lanes 4 q .. 4 q + 3
    // add their quarters: lane L ends with value L / 4 summed over all lanes
    xreduce_step<4>(gu, lane, 16);
    xreduce_step<4>(gv, lane, 16);
    xreduce_step<2>(gu, lane, 8);
    xreduce_step<2>(gv, lane, 8);
    xreduce_step<1>(gu, lane, 4);
    xreduce_step<1>(gv, lane, 4);
#pragma unroll
    for (int sh = 1; sh <= 2; sh <<= 1) {
        gu[0] = __fadd_rn(gu[0], __shfl_xor_sync(FULL, gu[0], sh));
        gv[0] = __fadd_rn(gv[0], __shfl_xor_sync(FULL, gv[0], sh));
    }
    // stage 2 (rank rows past k have zero factors and zero intermediates)
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        const cdf tl = {{__shfl_sync(FULL, gv[0], 16 * l), __shfl_sync(FULL, gv[0], 16 * l + 4)},
                        {__shfl_sync(FULL, gv[0], 16 * l + 8), __shfl_sync(FULL, gv[0], 16 * l + 12)}};
        const cdf tpl = {{__shfl_sync(FULL, gu[0], 16 * l), __shfl_sync(FULL, gu[0], 16 * l + 4)},
                         {__shfl_sync(FULL, gu[0], 16 * l + 8), __shfl_sync(FULL, gu[0], 16 * l + 12)}};
        cxstep_df(ci0, u[l].a, tl);
        cxstep_df(ci1, u[l].b, tl);
        cxstep_df(cj0, v[l].a, tpl);
        cxstep_df(cj1, v[l].b, tpl);
    }
}

// the last rank row of an odd rank (u, v: that row's two columns of U^T and V): as
// lr_pair for one row
__device__ __forceinline__ void lr_single(const Pair<float> &u, const Pair<float> &v, const Pair<float> &xi,
                                          const Pair<float> &xj, float s1u, float s1v, cxacc &ci0, cxacc &ci1,
                                          cxacc &cj0, cxacc &cj1, int lane)
{
    cxacc cu, cv;
    cx_start(cu, s1u);
    cxstep(cu, u.a, xi.a);
    cxstep(cu, u.b, xi.b);
    cx_start(cv, s1v);
    cxstep(cv, v.a, xj.a);
    cxstep(cv, v.b, xj.b);
    float gu[4] = {__fsub_rn(cu.re.tau, s1u), cu.re.r, __fsub_rn(cu.im.tau, s1u), cu.im.r};
    float gv[4] = {__fsub_rn(cv.re.tau, s1v), cv.re.r, __fsub_rn(cv.im.tau, s1v), cv.im.r};
    // index bits 1..0 by lane bits 4..3, then the eight lanes 8 c .. 8 c + 7 add their
    // eighths: lane L ends with value L / 8 summed over all lanes
    xreduce_step<2>(gu, lane, 16);
    xreduce_step<2>(gv, lane, 16);
    xreduce_step<1>(gu, lane, 8);
    xreduce_step<1>(gv, lane, 8);
#pragma unroll
    for (int sh = 1; sh <= 4; sh <<= 1) {
        gu[0] = __fadd_rn(gu[0], __shfl_xor_sync(FULL, gu[0], sh));
        gv[0] = __fadd_rn(gv[0], __shfl_xor_sync(FULL, gv[0], sh));
    }
    const cdf tl = {{__shfl_sync(FULL, gv[0], 0), __shfl_sync(FULL, gv[0], 8)},
                    {__shfl_sync(FULL, gv[0], 16), __shfl_sync(FULL, gv[0], 24)}};
    const cdf tpl = {{__shfl_sync(FULL, gu[0], 0), __shfl_sync(FULL, gu[0], 8)},
                     {__shfl_sync(FULL, gu[0], 16), __shfl_sync(FULL, gu[0], 24)}};
    cxstep_df(ci0, u.a, tl);
    cxstep_df(ci1, u.b, tl);
    cxstep_df(cj0, v.a, tpl);
    cxstep_df(cj1, v.b, tpl);
}

// Low-rank block U V of at most 64 x 64 (U^T k x m, V k x n, m, n padded even):
// slot rows (m) = U (V x_J), slot columns (n) = V^T (U^T x_I), one pass over pairs
// of rank rows (loaded one pair ahead).  A lane owns the rows / columns 2 lane,
// 2 lane + 1 of both panels.  Both stages run on common grids.  Stage 1 (the rank-k
// intermediates tp = U^T x_I, t = V x_J; bnd.x, bnd.y: largest rank-row 1-norms of
// U^T and V): the 32-lane reductions add the grid parts exactly in plain FP32.
// Stage 2 (the outputs; bnd.z, bnd.w: largest column 1-norms of U^T and V): the
// leading part of each intermediate is a grid sum, at most half its grid's sigma,
// which bounds the inputs, so each output is one chain over all rank rows.
__device__ __forceinline__ void lowrank_item_g(const Item &it, float4 bnd, const float2 *__restrict__ pool,
                                               const float2 *HM_XR x, cdf *HM_XR part, int lane)
{
    const int m = it.m, n = it.n, k = it.k;
    const float2 *UT = pool + it.off;
    const float2 *V = UT + (int64_t)k * m;
    const int i = 2 * lane;
    const bool iv = i < m, jv = i < n;
    Pair<float> u[2], v[2];
    lr_load(u, v, UT, V, 0, k, m, n, i, iv, jv);
    Pair<float> xi{make_float2(0.f, 0.f), make_float2(0.f, 0.f)}, xj = xi;
    if (iv) xi = ld_vec(x + it.row0 + i);
    if (jv) xj = ld_vec(x + it.col0 + i);
    const float s1u = grid_sigma(bnd.x, warp_max(fmaxf(linf(xi.a), linf(xi.b))));
    const float s1v = grid_sigma(bnd.y, warp_max(fmaxf(linf(xj.a), linf(xj.b))));
    const float s2i = grid_sigma(bnd.z, 0.5f * s1v), s2j = grid_sigma(bnd.w, 0.5f * s1u);
    cxacc ci0, ci1, cj0, cj1;
    cx_start(ci0, s2i);
    cx_start(ci1, s2i);
    cx_start(cj0, s2j);
    cx_start(cj1, s2j);
#pragma unroll 1
    for (int l0 = 0; l0 + 1 < k; l0 += 2) {
        Pair<float> un[2], vn[2];
        lr_load(un, vn, UT, V, l0 + 2, k, m, n, i, iv, jv);
        lr_pair(u, v, xi, xj, s1u, s1v, ci0, ci1, cj0, cj1, lane);
#pragma unroll
        for (int l = 0; l < 2; ++l) { u[l] = un[l]; v[l] = vn[l]; }
    }
    if (k & 1) lr_single(u[0], v[0], xi, xj, s1u, s1v, ci0, ci1, cj0, cj1, lane);   // row k - 1
    if (iv) { part[it.pad + i] = cxclose(ci0, s2i); part[it.pad + i + 1] = cxclose(ci1, s2i); }
    if (jv) { part[it.pad + m + i] = cxclose(cj0, s2j); part[it.pad + m + i + 1] = cxclose(cj1, s2j); }
}

// Low-rank block U V larger than 64 x 64: slot rows (m) = U (V x_J), slot columns
// (n) = V^T (U^T x_I), in Dot2; the rank-k intermediates stay in double-float.
__device__ __forceinline__ void lowrank_item_c(const Item &it, const float2 *__restrict__ pool,
                                               const float2 *HM_XR x, cdf *HM_XR part, int lane)
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

// The residual products of one block (item t of a list with bounds bnd): on the
// common grids where it fits (at most 64 x 64, rank <= 64), else the short-chain
// and Dot2 bodies above.  xs: GRID_MAX float2 of the warp's shared memory.
__device__ __forceinline__ void resid_item(const Item &it, const float4 *__restrict__ bnd, int64_t t,
                                           const float2 *__restrict__ pool, const float2 *HM_XR x,
                                           cdf *HM_XR part, float2 *xs, int lane)
{
    if (it.m <= GRID_MAX && it.n <= GRID_MAX) {
        // the whole block into L2 first: the row (chunk) loads after the first then hit L2
        const char *blk = reinterpret_cast<const char *>(pool + it.off);
        const int64_t bytes = item_elems(it) * (int64_t)sizeof(float2);
        for (int64_t o = (int64_t)lane * 128; o < bytes; o += 32 * 128)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(blk + o));
        const float4 bb = bnd[t];
        if (it.k == 0) dense_item_g(it, bb, pool, x, part, xs, lane);
        else lowrank_item_g(it, bb, pool, x, part, lane);
    } else if (it.k == 0) {
        dense_item_c(it, pool, x, part, xs, lane);
    } else {
        lowrank_item_c(it, pool, x, part, lane);
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
            // four slots in flight per warp; the next round's slot indices are loaded with this
            // round's slots, so that only the first round waits for its indices
            int64_t e = e0 + w;
            bool more = e + 3 * GW < e1;
            int64_t q0 = 0, q1 = 0, q2 = 0, q3 = 0;
            if (more) { q0 = csr_idx[e]; q1 = csr_idx[e + GW]; q2 = csr_idx[e + 2 * GW]; q3 = csr_idx[e + 3 * GW]; }
            while (more) {
                const cdf v00 = P[q0 + i], v01 = P[q0 + i + 1], v10 = P[q1 + i], v11 = P[q1 + i + 1];
                const cdf v20 = P[q2 + i], v21 = P[q2 + i + 1], v30 = P[q3 + i], v31 = P[q3 + i + 1];
                e += 4 * GW;
                more = e + 3 * GW < e1;
                if (more) { q0 = csr_idx[e]; q1 = csr_idx[e + GW]; q2 = csr_idx[e + 2 * GW]; q3 = csr_idx[e + 3 * GW]; }
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
