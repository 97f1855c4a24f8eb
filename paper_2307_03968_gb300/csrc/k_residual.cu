// FP64-class residual of the refinement step, r = b - A_m x, over complex64
// blocks (the precision rule of the solve: the final residual check runs at
// FP64-class accuracy).  k_residual_items writes every block's products into
// its double-float partial slots (no atomics), summing each block with short
// error-free chains (biased accumulator, k_dot2.cuh) folded into double-float
// sums; k_gather_acc64 sums each leaf's slots in a fixed order with compensated
// additions, adds D_I x_I (Dot2) and forms b - A x in FP64.
#include "k_dot2.cuh"

namespace hm {
namespace {

using namespace kc;
using namespace dot2;
constexpr int APPLY_WARPS = 8;

// Dense block: slot rows (even(m)) = B x_J, slot columns (even(n)) = B^T x_I.
// A lane owns two adjacent columns.  Row side: per row, the lane's two terms form
// one short error-free chain, then the lanes' double-float sums are reduced.
// Column side: chains over four rows at a time, folded into a double-float sum.
__device__ __forceinline__ void dense_item_c(const Item &it, const float2 *__restrict__ pool,
                                             const float2 *__restrict__ x, cdf *__restrict__ part, float2 *xs,
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
                                               const float2 *__restrict__ x, cdf *__restrict__ part, int lane)
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

__global__ void __launch_bounds__(APPLY_WARPS * 32, 2)
k_residual_items(const Item *__restrict__ items, int64_t n_items, const float2 *__restrict__ pool,
                 const float2 *__restrict__ x, int64_t ldx, cdf *__restrict__ part, int64_t pstride, int nrhs)
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
// sum of the leaf's partial slots of levels 1..m, in double-float arithmetic and
// in a fixed order (each of the GW warps sums every GW-th slot with compensated
// additions and takes every GW-th column of D_I x_I in Dot2; lanes own row pairs;
// the warps are then added in warp order).  If b is given, out = b - acc (in FP64,
// rounded to complex64) and |r|^2, |b|^2 go to norms; else out = acc (complex64).
// No atomics on sums.
constexpr int GW = 8;   // warps per leaf
__global__ void __launch_bounds__(GW * 32)
k_gather_acc64(const int32_t *__restrict__ pleaf_off, const int64_t *__restrict__ dinv_off,
               const float2 *__restrict__ self32, const float2 *__restrict__ x, int64_t ld,
               const int64_t *__restrict__ csr_off, int csr_stride, int m, const int64_t *__restrict__ csr_idx,
               const cdf *__restrict__ part, int64_t pstride, const float2 *__restrict__ b,
               float2 *__restrict__ out, double *norms)
{
    __shared__ cdf acc_s[GW][64];
    extern __shared__ __align__(16) unsigned char gsm[];
    float2 *xs = reinterpret_cast<float2 *>(gsm);                 // x of the leaf, np entries
    const int leaf = blockIdx.x, r = blockIdx.y;
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

void launch_apply_items_partials(hm_matrix h, const LevelList &L, const float2 *x, cdf *part, int64_t pstride,
                                 int nrhs, cudaStream_t s, int rb)
{
    const Item *list = L.d_items;
    int64_t n = (int64_t)L.items.size();
    if (rb < 0) rb = nrhs < MRHS_MIN_RHS ? 0 : nrhs <= 8 ? 8 : 16;
    if (rb > 0 && nrhs > 1 && L.n_small > 0) {
        // many right-hand sides: blocks that fit shared memory are read once per chunk
        launch_apply_items_partials_mrhs(h, L, x, part, pstride, nrhs, s, rb);
        list = L.d_big;
        n = L.n_big;
    }
    if (n == 0) return;
    static int per_sm = -1;
    if (per_sm < 0) {
        int v = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_residual_items, APPLY_WARPS * 32, 0);
        per_sm = v > 0 ? v : 1;
    }
    int g = per_sm * (h->num_sms > 0 ? h->num_sms : 1);
    if ((int64_t)g * APPLY_WARPS > n) g = (int)((n + APPLY_WARPS - 1) / APPLY_WARPS);
    k_residual_items<<<g, APPLY_WARPS * 32, 0, s>>>(list, n, h->d_pool32, x, h->pN, part, pstride, nrhs);
}

void launch_gather_acc64(hm_matrix h, const float2 *x, int m, const cdf *part, int64_t pstride,
                         const float2 *b, float2 *out, double *norms, int nrhs, cudaStream_t s)
{
    dim3 grid((unsigned)h->n_leaves, (unsigned)nrhs);
    const int64_t maxnp = [&] {
        int64_t v = 0;
        for (int64_t i = 0; i < h->n_leaves; ++i) v = std::max<int64_t>(v, h->pleaf_off[i + 1] - h->pleaf_off[i]);
        return v;
    }();
    k_gather_acc64<<<grid, GW * 32, sizeof(float2) * (size_t)std::max<int64_t>(maxnp, 1), s>>>(h->d_pleaf_off, h->d_dinv_off, h->d_self32, x, h->pN,
                                                              h->d_csr_off, h->n_levels + 1, m, h->d_csr_idx, part,
                                                              pstride, b, out, norms);
}

} // namespace hm
