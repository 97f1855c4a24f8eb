// FP64-class residual of the refinement step, r = b - A_m x, over complex64
// blocks (the precision rule of the solve: the final residual check runs at
// FP64-class accuracy).  k_residual_items writes every block's products into
// its double-float partial slots (no atomics): blocks of up to 64 x 64 on
// common grids taken from per-block bounds (k_item_bounds, computed once when the
// item lists are uploaded), larger ones with short error-free chains folded into
// double-float sums (k_dot2.cuh, k_residual_dev.cuh); k_gather_acc64 sums each
// leaf's slots in a fixed order with compensated additions, adds D_I x_I (Dot2)
// and forms b - A x in FP64.
#include "k_residual_dev.cuh"
#include "k_solve_dev.cuh"

namespace hm {
namespace {

using namespace kc;
using namespace dot2;
constexpr int APPLY_WARPS = 8;

__global__ void __launch_bounds__(APPLY_WARPS * 32, 2)
k_residual_items(const Item *__restrict__ items, const float4 *__restrict__ bnd, int64_t n_items,
                 const float2 *__restrict__ pool, const float2 *__restrict__ x, int64_t ldx, cdf *__restrict__ part,
                 int64_t pstride, int nrhs)
{
    __shared__ __align__(16) float2 xs_all[APPLY_WARPS][GRID_MAX];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t nw = (int64_t)gridDim.x * APPLY_WARPS;
    for (int64_t t = (int64_t)blockIdx.x * APPLY_WARPS + w; t < n_items; t += nw) {
        const Item it = items[t];
        for (int r = 0; r < nrhs; ++r) resid_item(it, bnd, t, pool, x + r * ldx, part + r * pstride, xs_all[w], lane);
    }
}

// Per item, the bounds the common-grid residual products take their grids from
// (resid_item): dense B (m x n, read to column even(n) - 1): x = largest row
// 1-norm, y = largest column 1-norm; low-rank (U^T k x m, V k x n): x, z = largest
// row / column 1-norm of U^T, y, w = those of V.  Sums of |re| + |im| in FP64,
// rounded up to FP32 (each bound >= its exact value).  One warp per item.
__global__ void __launch_bounds__(256)
k_item_bounds(const Item *__restrict__ items, int64_t n_items, const float2 *__restrict__ pool,
              float4 *__restrict__ bnd)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < n_items; t += nw) {
        const Item it = items[t];
        const float2 *A = pool + it.off;
        double a, b, c = 0.0, d = 0.0;
        if (it.k == 0) {
            const int ld = even_d(it.n);
            l1_bounds(A, it.m, ld, ld, a, b, lane);
        } else {
            l1_bounds(A, it.k, it.m, it.m, a, c, lane);
            l1_bounds(A + (int64_t)it.k * it.m, it.k, it.n, it.n, b, d, lane);
        }
        if (lane == 0)
            bnd[t] = make_float4(__double2float_ru(a), __double2float_ru(b), __double2float_ru(c), __double2float_ru(d));
    }
}

// Per leaf (blockIdx.x) and right-hand side (blockIdx.y): acc = D_I x_I +
// sum of the leaf's partial slots of levels 1..m (gather_leaf).
__global__ void __launch_bounds__(GW * 32)
k_gather_acc64(const int32_t *__restrict__ pleaf_off, const int64_t *__restrict__ dinv_off,
               const float2 *__restrict__ self32, const float2 *__restrict__ x, int64_t ld,
               const int64_t *__restrict__ csr_off, int csr_stride, int m, const int64_t *__restrict__ csr_idx,
               const cdf *__restrict__ part, int64_t pstride, const float2 *__restrict__ b,
               float2 *__restrict__ out, double *norms)
{
    __shared__ cdf acc_s[GW][64];
    extern __shared__ __align__(16) unsigned char gsm[];
    gather_leaf(blockIdx.x, blockIdx.y, pleaf_off, dinv_off, self32, x, ld, csr_off, csr_stride, m, csr_idx, part,
                pstride, b, out, norms, acc_s, reinterpret_cast<float2 *>(gsm));
}

// The gather, then the next series step of the refinement in the same CTA: out = b - acc
// for the leaf (as k_gather_acc64), then y = D_i^{-1} out_i (the first step of the
// correction's series) from the out_i this CTA just wrote.
__global__ void __launch_bounds__(GW * 32)
k_gather_leaf_update(const int32_t *__restrict__ pleaf_off, const int64_t *__restrict__ dinv_off,
                     const float2 *__restrict__ self32, const float2 *__restrict__ dinv32, const float2 *__restrict__ x,
                     int64_t ld, const int64_t *__restrict__ csr_off, int csr_stride, int m,
                     const int64_t *__restrict__ csr_idx, const cdf *__restrict__ part, int64_t pstride,
                     const float2 *__restrict__ b, float2 *out, double *norms, float2 *y)
{
    __shared__ cdf acc_s[GW][64];
    __shared__ float2 lpart[8][64];
    extern __shared__ __align__(16) unsigned char gsm[];
    gather_leaf(blockIdx.x, blockIdx.y, pleaf_off, dinv_off, self32, x, ld, csr_off, csr_stride, m, csr_idx, part,
                pstride, b, out, norms, acc_s, reinterpret_cast<float2 *>(gsm));
    __syncthreads();                                       // this CTA's writes of out_i, read back below
    leaf_update_leaf<float>(blockIdx.x, blockIdx.y, pleaf_off, dinv_off, dinv32, nullptr, out, y, ld, 0,
                            reinterpret_cast<float2 *>(gsm), lpart);
}

} // namespace

void launch_gather_leaf_update(hm_matrix h, const float2 *x, int m, const cdf *part, int64_t pstride,
                               const float2 *b, float2 *out, double *norms, float2 *y, int nrhs, cudaStream_t s)
{
    dim3 grid((unsigned)h->n_leaves, (unsigned)nrhs);
    int64_t maxnp = 1;
    for (int64_t i = 0; i < h->n_leaves; ++i) maxnp = std::max<int64_t>(maxnp, h->pleaf_off[i + 1] - h->pleaf_off[i]);
    k_gather_leaf_update<<<grid, GW * 32, sizeof(float2) * (size_t)maxnp, s>>>(
        h->d_pleaf_off, h->d_dinv_off, h->d_self32, h->d_dinv32, x, h->pN, h->d_csr_off, h->n_levels + 1, m,
        h->d_csr_idx, part, pstride, b, out, norms, y);
}

int launch_apply_items_partials(hm_matrix h, const LevelList &L, const float2 *x, cdf *part, int64_t pstride,
                                int nrhs, cudaStream_t s, int rb)
{
    int launched = 0;
    const Item *list = L.d_res;
    const float4 *bnd = L.d_bnd;
    int64_t n = (int64_t)L.items.size();
    if (rb < 0) rb = nrhs < MRHS_MIN_RHS ? 0 : nrhs <= 8 ? 8 : 16;
    if (rb > 0 && nrhs > 1 && L.n_small > 0) {
        // many right-hand sides: blocks that fit shared memory are read once per chunk
        launch_apply_items_partials_mrhs(h, L, x, part, pstride, nrhs, s, rb);
        launched = 1;
        list = L.d_big;
        bnd = L.d_bnd_big;
        n = L.n_big;
    }
    if (n == 0) return launched;
    int g = (int)(residual_warps(h) / APPLY_WARPS);
    if ((int64_t)g * APPLY_WARPS > n) g = (int)((n + APPLY_WARPS - 1) / APPLY_WARPS);
    k_residual_items<<<g, APPLY_WARPS * 32, 0, s>>>(list, bnd, n, h->d_pool32, x, h->pN, part, pstride, nrhs);
    return launched + 1;
}

int64_t residual_warps(hm_matrix h)
{
    static int per_sm = -1;
    if (per_sm < 0) {
        int v = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_residual_items, APPLY_WARPS * 32, 0);
        per_sm = v > 0 ? v : 1;
    }
    if (h->num_sms <= 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
    }
    return (int64_t)per_sm * h->num_sms * APPLY_WARPS;
}

void launch_item_bounds(const Item *items, int64_t n, const float2 *pool, float4 *bnd, cudaStream_t s)
{
    if (n <= 0) return;
    const int g = (int)std::min<int64_t>((n + 7) / 8, 152 * 16);
    k_item_bounds<<<g, 256, 0, s>>>(items, n, pool, bnd);
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
