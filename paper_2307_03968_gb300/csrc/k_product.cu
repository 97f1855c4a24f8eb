// Block product z += M x over a list of stored blocks (arxiv 2307.03968 eq. 6
// and eq. 8, with the half storage of §III: every stored block is read once and
// acts on both of its clusters):
//     dense  B (I,J):  z_I += B x_J,            z_J += B^T x_I
//     low rank U V:    z_I += U (V x_J),        z_J += V^T (U^T x_I)
// One warp per block, persistent grid (occupancy x SMs, 8 warps per CTA).  The
// complex64 instantiation is launched with three CTAs per SM (at most 80
// registers a thread), so that 24 warps per SM keep loads in flight.  A lane owns
// two adjacent columns, loaded as one 128-bit streaming load, so column-side sums
// accumulate in registers; row-side sums are warp transpose reductions.  Low-rank
// panels go in chunks of 8 rank rows held in registers, so U^T and V are read
// once.  Results go to z with vector atomics (order-free sums: reproducible to
// FP32 rounding, not bitwise).
#include "k_common.cuh"

namespace hm {
namespace {

using namespace kc;
constexpr int APPLY_WARPS = 8;   // warps per CTA of the product kernel

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

// MINB: CTAs per SM the register budget must allow (3 for complex64, so that 24
// warps per SM stream blocks; 1 for the FP64 comparator path, which needs more
// registers)
template <class T, class A, int MINB>
__global__ void __launch_bounds__(APPLY_WARPS * 32, MINB)
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

template <class T, class A, int MINB>
int apply_grid(hm_matrix h)
{
    static int per_sm = -1;
    if (per_sm < 0) {
        int v = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_apply_items<T, A, MINB>, APPLY_WARPS * 32, 0);
        per_sm = v > 0 ? v : 1;
    }
    return per_sm * (h->num_sms > 0 ? h->num_sms : 1);
}

} // namespace

void launch_apply_items(hm_matrix h, const LevelList &L, const void *x, void *z, int nrhs, bool fp64,
                        cudaStream_t s, int rb)
{
    const int64_t n = (int64_t)L.items.size();
    if (n == 0) return;
    if (fp64) {
        int g = apply_grid<double, double, 1>(h);
        if ((int64_t)g * APPLY_WARPS > n) g = (int)((n + APPLY_WARPS - 1) / APPLY_WARPS);
        k_apply_items<double, double, 1><<<g, APPLY_WARPS * 32, 0, s>>>(
            L.d_items, n, h->d_pool64, (const double2 *)x, h->pN, (double2 *)z, h->pN, nrhs);
    } else {
        const Item *list = L.d_items;
        int64_t cnt = n;
        if (rb < 0) rb = nrhs < MRHS_MIN_RHS ? 0 : nrhs <= 8 ? 8 : nrhs <= 16 ? 16 : 32;
        if (rb == RB_TC && nrhs > 1) {
            // the small blocks (dense and low-rank) on the tensor cores
            launch_apply_tc(h, L, (const float2 *)x, (float2 *)z, nrhs, s);
            list = L.d_big;
            cnt = L.n_big;
            if (cnt == 0) return;
        } else if (rb > 0 && nrhs > 1 && L.n_small > 0) {
            // many right-hand sides: blocks that fit shared memory are read once per RHS chunk
            launch_apply_items_mrhs(h, L, (const float2 *)x, (float2 *)z, nrhs, rb, s);
            list = L.d_big;
            cnt = L.n_big;
            if (cnt == 0) return;
        }
        int g = apply_grid<float, float, 3>(h);
        if ((int64_t)g * APPLY_WARPS > cnt) g = (int)((cnt + APPLY_WARPS - 1) / APPLY_WARPS);
        k_apply_items<float, float, 3><<<g, APPLY_WARPS * 32, 0, s>>>(
            list, cnt, h->d_pool32, (const float2 *)x, h->pN, (float2 *)z, h->pN, nrhs);
    }
}

} // namespace hm
