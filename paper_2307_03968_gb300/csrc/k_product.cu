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
#include "k_product_dev.cuh"

namespace hm {
namespace {

using namespace kc;
constexpr int APPLY_WARPS = 8;   // warps per CTA of the product kernel


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

int64_t product_warps(hm_matrix h)
{
    if (h->num_sms <= 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
    }
    return (int64_t)apply_grid<float, float, 3>(h) * APPLY_WARPS;
}

int launch_apply_items(hm_matrix h, const LevelList &L, const void *x, void *z, int nrhs, bool fp64,
                       cudaStream_t s, int rb)
{
    const int64_t n = (int64_t)L.items.size();
    if (n == 0) return 0;
    if (fp64) {
        int g = apply_grid<double, double, 1>(h);
        if ((int64_t)g * APPLY_WARPS > n) g = (int)((n + APPLY_WARPS - 1) / APPLY_WARPS);
        k_apply_items<double, double, 1><<<g, APPLY_WARPS * 32, 0, s>>>(
            L.d_items, n, h->d_pool64, (const double2 *)x, h->pN, (double2 *)z, h->pN, nrhs);
        return 1;
    } else {
        int launched = 0;
        // tall dense blocks go as row panels (LevelList::d_prod), one warp each
        const Item *list = L.d_prod ? L.d_prod : L.d_items;
        int64_t cnt = L.d_prod ? L.n_prod : n;
        if (rb < 0) rb = nrhs < MRHS_MIN_RHS ? 0 : nrhs <= 8 ? 8 : nrhs <= 16 ? 16 : 32;
        if (rb == RB_TC && nrhs > 1) {
            // the small blocks (dense and low-rank) on the tensor cores
            launched += launch_apply_tc(h, L, (const float2 *)x, (float2 *)z, nrhs, s);
            list = L.d_prod ? L.d_prod_big : L.d_big;
            cnt = L.d_prod ? L.n_prod_big : L.n_big;
            if (cnt == 0) return launched;
        } else if (rb > 0 && nrhs > 1 && L.n_small > 0) {
            // many right-hand sides: blocks that fit shared memory are read once per RHS chunk
            launch_apply_items_mrhs(h, L, (const float2 *)x, (float2 *)z, nrhs, rb, s);
            launched += 1;
            list = L.d_prod ? L.d_prod_big : L.d_big;
            cnt = L.d_prod ? L.n_prod_big : L.n_big;
            if (cnt == 0) return launched;
        }
        int g = apply_grid<float, float, 3>(h);
        if ((int64_t)g * APPLY_WARPS > cnt) g = (int)((cnt + APPLY_WARPS - 1) / APPLY_WARPS);
        k_apply_items<float, float, 3><<<g, APPLY_WARPS * 32, 0, s>>>(
            list, cnt, h->d_pool32, (const float2 *)x, h->pN, (float2 *)z, h->pN, nrhs);
        return launched + 1;
    }
}

} // namespace hm
