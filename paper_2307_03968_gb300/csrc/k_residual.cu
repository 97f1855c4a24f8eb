// FP64-class residual of the refinement step, r = b - A_m x, over complex64
// blocks (the precision rule of the solve: the final residual check runs at
// FP64-class accuracy).  k_residual_items writes every block's products into
// its double-float partial slots (no atomics), summing each block with short
// error-free chains (biased accumulator, k_dot2.cuh) folded into double-float
// sums; k_gather_acc64 sums each leaf's slots in a fixed order with compensated
// additions, adds D_I x_I (Dot2) and forms b - A x in FP64.
#include "k_residual_dev.cuh"

namespace hm {
namespace {

using namespace kc;
using namespace dot2;
constexpr int APPLY_WARPS = 8;

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
