// hm_residual_noalloc: the refinement residual r = b - A_m x computed without
// allocating any memory.
//
// Who needs this: callers that are not allowed to allocate device memory once
// they are running.  A typical case is a serving process that reserves device
// memory up front, for example through a framework's caching allocator, and
// treats any later cudaMalloc as an error.  Such a cudaMalloc can fail
// although memory is free inside the reserved pools, and it can synchronise
// the device in the middle of a request.  Real-time loops have the same
// constraint.  hm_residual grows the handle's workspace on demand.  This
// variant never does: all of its temporary storage lives in one fixed array
// in device memory, defined below, which the library's device image carries.
//
// The array is g_noalloc_scratch, NOALLOC_SCRATCH_BYTES (32 MiB) per GPU.  It
// exists on every GPU that loads this library and is held until the process
// exits.  Its layout per call: permuted b, x and r (complex64, padded length
// times nrhs each), two FP64 norms per right-hand side, then the double-float
// partial slots of one right-hand side.  Calls whose sizes do not fit are rejected
// with HM_ERR_ARG before any device work.
#include "hm_internal.h"

#include <mutex>

namespace hm {
namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(32) << 20;

__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch, resolved once per device.  In host code
// the array's name is only a host-side stand-in, so the kernels receive this
// address instead.
constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void *g_addr[MAX_DEVICES] = {};

hm_status scratch_address(void **out)
{
    int dev = 0;
    HM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAX_DEVICES) return fail(HM_ERR_ARG, "device index out of range for the static scratch");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return HM_OK;
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

} // namespace
} // namespace hm

using namespace hm;

extern "C" hm_status hm_residual_noalloc(hm_matrix h, const void *b, int64_t ldb, const void *x, int64_t ldx,
                                         void *r, int64_t ldr, int nrhs, int n_levels, double *norms,
                                         void *stream)
{
    if (!h) return fail(HM_ERR_ARG, "null handle");
    if (nrhs < 0 || ldb < h->N || ldx < h->N || ldr < h->N) return fail(HM_ERR_ARG, "bad nrhs or leading dimension");
    if (nrhs == 0) return HM_OK;
    if (!b || !x || !r) return fail(HM_ERR_ARG, "null b, x or r");
    if (!h->factored) return fail(HM_ERR_STATE, "hm_factor_leaf has not completed (it also prepares D)");
    const size_t vec = align256(sizeof(float2) * (size_t)h->pN * nrhs);
    const size_t nrm = align256(2 * sizeof(double) * (size_t)nrhs);
    const size_t part = sizeof(dot2::cdf) * (size_t)std::max<int64_t>(h->partial_elems, 1);
    const size_t need = 3 * vec + nrm + part;
    if (need > NOALLOC_SCRATCH_BYTES)
        return fail(HM_ERR_ARG, "operator and nrhs need " + std::to_string(need) + " bytes of scratch; the static "
                                "scratch of hm_residual_noalloc holds " + std::to_string(NOALLOC_SCRATCH_BYTES));
    void *base = nullptr;
    hm_status st = scratch_address(&base);
    if (st != HM_OK) return st;
    unsigned char *p = (unsigned char *)base;
    float2 *bt = (float2 *)p, *xt = (float2 *)(p + vec), *rt = (float2 *)(p + 2 * vec);
    double *dn = (double *)(p + 3 * vec);
    dot2::cdf *dpart = (dot2::cdf *)(p + 3 * vec + nrm);
    cudaStream_t s = (cudaStream_t)stream;
    int m = (n_levels < 0 || n_levels > h->n_levels) ? h->n_levels : n_levels;
    if (m < 1) m = 1;
    // the array keeps the previous call's contents: the norms must start at zero;
    // the partial slots read by the gather are all rewritten below
    HM_CUDA(cudaMemsetAsync(dn, 0, 2 * sizeof(double) * nrhs, s));
    launch_permute_in(b, ldb, bt, h->pN, h->d_pperm, nrhs, false, s);
    launch_permute_in(x, ldx, xt, h->pN, h->d_pperm, nrhs, false, s);
    for (int j = 0; j < nrhs; ++j) {   // one right-hand side at a time through the partial slots
        const float2 *xj = xt + (int64_t)j * h->pN;
        for (int lev = 1; lev <= m; ++lev) {
            auto it = h->levels.find(lev);
            if (it == h->levels.end() || it->second.items.empty()) continue;
            launch_apply_items_partials(h, it->second, xj, dpart, h->partial_elems, 1, s);
        }
        launch_gather_acc64(h, xj, m, dpart, h->partial_elems, bt + (int64_t)j * h->pN, rt + (int64_t)j * h->pN,
                            dn + 2 * j, 1, s);
    }
    launch_permute_out(rt, h->pN, r, ldr, h->d_pperm, nrhs, false, s);
    HM_CUDA(cudaGetLastError());
    if (norms) {
        HM_CUDA(cudaMemcpyAsync(norms, dn, 2 * sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaStreamSynchronize(s));
    }
    return HM_OK;
}
