// One-launch solve: the whole power-series solve (arxiv 2307.03968 §IV, eq. 19
// with the fixed-term series of eqs. 20-22, and the refinement step) as ONE
// cooperative kernel.  The host records the solve's kernel sequence as a list
// of phases (hm_api.cu); every CTA walks the list, doing its share of each
// phase with the same device bodies as the separate kernels (k_product_dev.cuh,
// k_residual_dev.cuh, k_solve_dev.cuh), and all CTAs meet at a grid-wide
// barrier between consecutive phases.  This removes the launch boundaries of
// the ~18-60 kernels of a solve, which dominate the time of small operators.
//
// The barrier is one word in global memory (reset by the host before every
// launch), which the arrivals flip as a whole; every CTA polls it a bounded
// number of times (the wait limit of the handle, default 2^24 polls), and a CTA
// that gives up records HM_ERR_TIMEOUT in the status word and leaves the kernel,
// so that every other CTA gives up at its next barrier too: no wait is unbounded.
// The launch is cooperative, so all CTAs are resident together.
//
// The vector pointers of the shared bodies are compiled without __restrict__
// here (HM_XR empty): the vectors and partial slots are written by other CTAs in
// earlier phases, so no load may go through the non-coherent path.
#define HM_XR
#include "k_product_dev.cuh"
#include "k_residual_dev.cuh"
#include "k_solve_dev.cuh"

namespace hm {
namespace {

using namespace kc;
using namespace dot2;

constexpr int PT = 256;                 // threads per CTA (8 warps, as the separate kernels)
constexpr int PW = PT / 32;
constexpr int PERSIST_MAX_NP = 128;     // largest padded leaf the shared-memory buffers hold
constexpr uint32_t BAR_POLLS = 1u << 24;

// Grid-wide barrier with a bounded wait; false if this CTA gave up (status set).
// One word: every CTA adds 1 except CTA 0, which adds 2^31 - (gridDim.x - 1), so
// the word's top bit flips exactly when the last CTA arrives and its low bits
// return to where they were (the same word serves every barrier of the launch).
// Each CTA polls for the flip of the bit it saw when it arrived.
__device__ __forceinline__ bool grid_barrier(const PersistCtx &c, int *give_up)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned inc = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1) : 1u;
        __threadfence();
        const unsigned old = atomicAdd(c.bar, inc);
        volatile unsigned *w = c.bar;
        uint32_t it = 0;
        while (((old ^ *w) & 0x80000000u) == 0) {
            if (++it > c.polls) {
                atomicCAS(c.status, 0, (int)HM_ERR_TIMEOUT);
                *give_up = 1;
                break;
            }
            if (it > 4096) __nanosleep(256);   // tight polls first, then back off
        }
        __threadfence();
    }
    __syncthreads();
    return *give_up == 0;
}

__device__ __forceinline__ int64_t gtid() { return (int64_t)blockIdx.x * PT + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return (int64_t)gridDim.x * PT; }

constexpr int PERSIST_SMEM = PW * 64 * sizeof(cdf) + PERSIST_MAX_NP * sizeof(float2);

// Every CTA runs the phases [0, n_phases) in order, with a grid barrier between
// consecutive phases.  sm: the CTA's shared-memory area (PERSIST_SMEM bytes),
// laid out per phase: the gather's double-float row sums (8 KB) and the leaf's x
// (1 KB) are the largest use.  Returns false if a barrier gave up.
// b_in / x_out, when given, replace the recorded right-hand-side and solution
// pointers of the permutation phases (the serving loop runs one recorded list
// for every slot's buffers).
__device__ bool run_phases(const Phase *phases, int n_phases, const PersistCtx &c, unsigned char *sm,
                           int *give_up, const void *b_in = nullptr, void *x_out = nullptr)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int p = 0; p < n_phases; ++p) {
        const Phase P = phases[p];
        switch (P.op) {
        case PH_PERMUTE_IN: {
            const float2 *b = (const float2 *)(b_in ? b_in : P.a);
            float2 *xt = (float2 *)P.c;
            for (int64_t t = gtid(); t < c.pN * P.nrhs; t += gstride()) {
                const int64_t r = t / c.pN, q = t - r * c.pN;
                const int32_t src = c.pperm[q];
                xt[t] = src >= 0 ? b[r * P.ld2 + src] : make_float2(0.f, 0.f);
            }
            break;
        }
        case PH_PERMUTE_OUT: {
            const float2 *xt = (const float2 *)P.a;
            float2 *x = (float2 *)(x_out ? x_out : P.c);
            for (int64_t t = gtid(); t < c.pN * P.nrhs; t += gstride()) {
                const int64_t r = t / c.pN, q = t - r * c.pN;
                const int32_t dst = c.pperm[q];
                if (dst >= 0) x[r * P.ld2 + dst] = xt[t];
            }
            break;
        }
        case PH_LEAF: {
            float2 *zs = reinterpret_cast<float2 *>(sm);
            float2(*part)[64] = reinterpret_cast<float2(*)[64]>(sm + PERSIST_MAX_NP * sizeof(float2));
            const int64_t nvb = c.n_leaves * P.nrhs;
            for (int64_t vb = blockIdx.x; vb < nvb; vb += gridDim.x) {
                const int leaf = (int)(vb % c.n_leaves), r = (int)(vb / c.n_leaves);
                leaf_update_leaf<float>(leaf, r, c.pleaf_off, c.dinv_off, c.dinv, (const float2 *)P.a,
                                        (float2 *)P.b, (float2 *)P.c, c.pN, P.m, zs, part);
            }
            break;
        }
        case PH_APPLY: {
            float2 *xs = reinterpret_cast<float2 *>(sm) + 32 * w;
            const float2 *x = (const float2 *)P.a;
            float2 *z = (float2 *)P.c;
            for (int64_t t = (int64_t)blockIdx.x * PW + w; t < P.n; t += (int64_t)gridDim.x * PW) {
                const Item it = P.items[t];
                for (int r = 0; r < P.nrhs; ++r) {
                    if (it.k == 0) dense_item<float, float>(it, c.pool, x + r * c.pN, z + r * c.pN, xs, lane);
                    else lowrank_item<float, float>(it, c.pool, x + r * c.pN, z + r * c.pN, lane);
                }
            }
            break;
        }
        case PH_RESID: {
            const float2 *x = (const float2 *)P.a;
            cdf *part = (cdf *)P.c;
            for (int64_t t = (int64_t)blockIdx.x * PW + w; t < P.n; t += (int64_t)gridDim.x * PW) {
                const Item it = P.items[t];
                for (int r = 0; r < P.nrhs; ++r)
                    resid_item(it, (const float4 *)P.d, t, c.pool, x + r * c.pN, part + r * P.ld,
                               reinterpret_cast<float2 *>(sm) + GRID_MAX * w, lane);
            }
            break;
        }
        case PH_GATHER: {
            cdf(*acc_s)[64] = reinterpret_cast<cdf(*)[64]>(sm);
            float2 *xs = reinterpret_cast<float2 *>(sm + PW * 64 * sizeof(cdf));
            const int64_t nvb = c.n_leaves * P.nrhs;
            for (int64_t vb = blockIdx.x; vb < nvb; vb += gridDim.x) {
                const int leaf = (int)(vb % c.n_leaves), r = (int)(vb / c.n_leaves);
                gather_leaf(leaf, r, c.pleaf_off, c.dinv_off, c.self32, (const float2 *)P.a, c.pN, c.csr_off,
                            c.csr_stride, P.m, c.csr_idx, (const cdf *)P.d, P.ld, (const float2 *)P.b,
                            (float2 *)P.c, P.norms, acc_s, xs);
            }
            break;
        }
        case PH_ZERO: {
            unsigned char *d = (unsigned char *)P.c;
            for (int64_t t = gtid(); t < P.n / 8; t += gstride()) reinterpret_cast<uint2 *>(d)[t] = make_uint2(0u, 0u);
            for (int64_t t = (P.n / 8) * 8 + gtid(); t < P.n; t += gstride()) d[t] = 0;
            break;
        }
        case PH_COPY: {
            const unsigned char *s = (const unsigned char *)P.a;
            unsigned char *d = (unsigned char *)P.c;
            for (int64_t t = gtid(); t < P.n / 8; t += gstride())
                reinterpret_cast<uint2 *>(d)[t] = reinterpret_cast<const uint2 *>(s)[t];
            for (int64_t t = (P.n / 8) * 8 + gtid(); t < P.n; t += gstride()) d[t] = s[t];
            break;
        }
        case PH_SUB: {
            const float2 *y = (const float2 *)P.a, *v = (const float2 *)P.b;
            float2 *o = (float2 *)P.c;
            for (int64_t t = gtid(); t < P.n; t += gstride()) o[t] = csub(y[t], v[t]);
            break;
        }
        case PH_ADD: {
            const float2 *dx = (const float2 *)P.a;
            float2 *x = (float2 *)P.c;
            for (int64_t t = gtid(); t < P.n; t += gstride()) x[t] = cadd(x[t], dx[t]);
            break;
        }
        case PH_CHECK: {
            const float2 *x = (const float2 *)P.a;
            for (int64_t t = gtid(); t < P.n; t += gstride()) {
                const float2 v = x[t];
                if (!isfinite(v.x) || !isfinite(v.y)) {
                    atomicCAS(c.status, 0, (int)HM_ERR_DIVERGED);
                    break;
                }
            }
            break;
        }
        default:
            break;
        }
        // P.pad: the next phase touches only what this thread wrote here (elementwise
        // phases over the same index space) or nothing this phase wrote: no barrier
        if (p + 1 < n_phases && !P.pad && !grid_barrier(c, give_up)) return false;
    }
    return true;
}

__global__ void __launch_bounds__(PT, 2) k_solve_persist(const Phase *__restrict__ phases, int n_phases, PersistCtx c)
{
    __shared__ __align__(16) unsigned char sm[PERSIST_SMEM];
    __shared__ int give_up;
    if (threadIdx.x == 0) give_up = 0;
    __syncthreads();
    run_phases(phases, n_phases, c, sm, &give_up);
}

// ---- the device-resident request loop ---------------------------------------------

__device__ __forceinline__ int ld_acquire_sys(const int32_t *p)
{
    int v;
    asm volatile("ld.acquire.sys.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_sys(int32_t *p, int v)
{
    asm volatile("st.release.sys.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// One cooperative kernel that serves solve requests from a ring in mapped host
// memory until it finds none for idle_polls polls (or a stop entry).  Per request:
// CTA 0 waits (bounded) for the ring entry at `head` to become ready, copies its
// phase list pointer and operator context into device memory, and all CTAs learn
// the decision at a grid barrier; they run the request's phases (the one-launch
// solve of that operator and right-hand-side count), meet at a barrier, and CTA 0
// marks the entry done (a system-scope release, which the host acquires before it
// copies the result out).  The right-hand sides and solutions are device buffers
// the host fills and drains with copies of its own.  Every wait is bounded; a
// barrier that gives up ends the loop with HM_ERR_TIMEOUT in *loop_status.
__global__ void __launch_bounds__(PT, 2) k_serve_loop(LoopEntry *ring, int ring_size, LoopCtl *ctl, LoopDev *dv,
                                                     unsigned *bar, int *loop_status, uint32_t idle_polls,
                                                     uint32_t bar_polls)
{
    __shared__ __align__(16) unsigned char sm[PERSIST_SMEM];
    __shared__ int give_up, go;
    if (threadIdx.x == 0) give_up = 0;
    __syncthreads();
    PersistCtx bc;
    memset(&bc, 0, sizeof(bc));
    bc.bar = bar;
    bc.status = loop_status;
    bc.polls = bar_polls;
    int64_t head = *(volatile int64_t *)&ctl->start;
    for (;;) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            LoopEntry *e = ring + head % ring_size;
            int st = -1;
            for (uint32_t it = 0; it <= idle_polls; ++it) {
                const int v = ld_acquire_sys(&e->state);
                if (v == LOOP_READY || v == LOOP_STOP) { st = v; break; }
                __nanosleep(1000);
            }
            if (st == LOOP_READY) {
                const volatile LoopEntry *ve = e;
                dv->cur_n = ve->n_phases;
                dv->cur_phases = ve->phases;
                dv->cur_b = ve->b;
                dv->cur_x = ve->x;
                const volatile uint64_t *src = reinterpret_cast<const volatile uint64_t *>(&e->ctx);
                uint64_t *dst = reinterpret_cast<uint64_t *>(&dv->cur_ctx);
                for (int q = 0; q < (int)(sizeof(PersistCtx) / 8); ++q) dst[q] = src[q];
                dv->decision = 1;
            } else {
                dv->decision = 0;
            }
        }
        if (!grid_barrier(bc, &give_up)) break;
        if (threadIdx.x == 0) go = *(volatile int *)&dv->decision;
        __syncthreads();
        if (!go) break;
        PersistCtx c = dv->cur_ctx;
        c.bar = bar;
        c.polls = bar_polls;
        if (!run_phases(dv->cur_phases, dv->cur_n, c, sm, &give_up, dv->cur_b, dv->cur_x)) break;
        if (!grid_barrier(bc, &give_up)) break;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            __threadfence_system();
            st_release_sys(&ring[head % ring_size].state, LOOP_DONE);
        }
        ++head;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *(volatile int64_t *)&ctl->head = head;
        __threadfence_system();
        st_release_sys(&ctl->exited, 1);
    }
}

} // namespace

void persist_ctx(hm_matrix h, PersistCtx *c)
{
    *c = PersistCtx{h->d_pperm, h->pN, h->n_leaves, h->d_pleaf_off, h->d_dinv_off, h->d_dinv32, h->d_self32,
                    h->d_pool32, h->d_csr_off, h->n_levels + 1, h->d_csr_idx, h->d_status, h->d_bar,
                    h->tc_wait_limit < 0 ? BAR_POLLS : (uint32_t)h->tc_wait_limit};
}

int serve_loop_grid(int num_sms)
{
    static int per_sm = -1;
    if (per_sm < 0) {
        int v = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_serve_loop, PT, 0);
        per_sm = v > 0 ? v : 1;
    }
    return per_sm * (num_sms > 0 ? num_sms : 1);
}

hm_status launch_serve_loop(LoopEntry *ring, int ring_size, LoopCtl *ctl, LoopDev *dv, unsigned *bar, int *loop_status,
                            int grid, uint32_t idle_polls, cudaStream_t s)
{
    HM_CUDA(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(PT);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    HM_CUDA(cudaLaunchKernelEx(&cfg, k_serve_loop, ring, ring_size, ctl, dv, bar, loop_status, idle_polls, BAR_POLLS));
    return HM_OK;
}

bool persist_supported(hm_matrix h)
{
    for (int64_t i = 0; i < h->n_leaves; ++i)
        if (h->pleaf_off[i + 1] - h->pleaf_off[i] > PERSIST_MAX_NP) return false;
    return h->d_pool32 && h->d_dinv32 && h->d_self32;
}

// One cooperative launch of the recorded phases.  The grid is the kernel's
// occupancy times the SM count, capped at the widest phase's work units, so
// that small operators barrier over fewer CTAs.
hm_status launch_persist(hm_matrix h, const Phase *d_phases, int n_phases, int units, cudaStream_t s)
{
    static int per_sm = -1;
    if (per_sm < 0) {
        int v = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_solve_persist, PT, 0);
        per_sm = v > 0 ? v : 1;
    }
    int g = per_sm * (h->num_sms > 0 ? h->num_sms : 1);
    if (units > 0 && units < g) g = units;
    PersistCtx c;
    persist_ctx(h, &c);
    HM_CUDA(cudaMemsetAsync(h->d_bar, 0, 2 * sizeof(unsigned), s));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)g);
    cfg.blockDim = dim3(PT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    HM_CUDA(cudaLaunchKernelEx(&cfg, k_solve_persist, d_phases, n_phases, c));
    return HM_OK;
}

} // namespace hm
