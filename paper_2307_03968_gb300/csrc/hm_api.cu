// C ABI of the hmps library: handle management, block import, leaf
// factorisation, the multi-level power-series solve (arxiv 2307.03968 §IV,
// eqs. 12-22) and the H-Matrix product.  The numerical work runs in the
// kernels of k_solve.cu / k_factor.cu / k_build.cu; this file only checks
// arguments, lays out device memory and enqueues kernels.
#include "hm_internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

namespace hm {

static thread_local std::string g_last_error;

hm_status fail(hm_status s, const std::string &msg)
{
    g_last_error = msg;
    return s;
}

hm_status cuda_fail(cudaError_t e, const char *what)
{
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? HM_ERR_OOM : HM_ERR_CUDA;
}

hm_status dev_alloc(hm_matrix h, void **p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    h->device_bytes += (int64_t)bytes;
    return HM_OK;
}

template <class T> static hm_status upload(hm_matrix h, T **dst, const std::vector<T> &src, cudaStream_t s)
{
    hm_status st = dev_alloc(h, (void **)dst, src.size() * sizeof(T));
    if (st != HM_OK) return st;
    if (!src.empty()) HM_CUDA(cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return HM_OK;
}

hm_status upload_item_lists(hm_matrix h, cudaStream_t s)
{
    hm_status st;
    for (auto &kv : h->levels) {
        LevelList &L = kv.second;
        std::vector<Item> small, big;
        L.small_dim = 2;
        L.small_rank = 0;
        for (const Item &it : L.items) {
            const bool fits = it.m <= MRHS_MAX_DIM && it.n <= MRHS_MAX_DIM && it.k <= MRHS_MAX_RANK;
            (fits ? small : big).push_back(it);
            if (fits) {
                L.small_dim = std::max<int>(L.small_dim, (int)std::max(even(it.m), even(it.n)));
                L.small_rank = std::max(L.small_rank, it.k);
            }
        }
        L.n_small = (int64_t)small.size();
        L.n_big = (int64_t)big.size();
        const std::map<int32_t, std::vector<TcProd>> by_out = directed_products(small);
        std::vector<TcUnit> rcu;
        std::vector<TcProd> rcp;
        build_owner_lists(by_out, rcu, rcp);
        TcLists tc;
        if (!build_tc_lists(by_out, tc)) return fail(HM_ERR_STATE, "tensor-core work lists out of their index bounds");
        L.n_rcu = (int64_t)rcu.size();
        if ((st = upload(h, &L.d_rcu, rcu, s)) != HM_OK) return st;
        if ((st = upload(h, &L.d_rcp, rcp, s)) != HM_OK) return st;
        if ((st = dev_alloc(h, (void **)&L.d_rcb, sizeof(float2) * rcp.size())) != HM_OK) return st;
        launch_prod_bounds(L.d_rcp, (int64_t)rcp.size(), h->d_pool32, L.d_rcb, s);
        L.n_tcu = (int64_t)tc.units.size();
        L.n_tco = (int64_t)tc.ops.size();
        L.n_xch = (int64_t)tc.xch.size();
        L.n_tcb = (int64_t)tc.batches.size();
        L.n_tcr = (int64_t)tc.rows.size();
        L.n_tchunk = tc.n_tchunk;
        h->tc_max_xch = std::max(h->tc_max_xch, L.n_xch);
        h->tc_max_tchunk = std::max(h->tc_max_tchunk, L.n_tchunk);
        if ((st = upload(h, &L.d_xch, tc.xch, s)) != HM_OK) return st;
        if ((st = upload(h, &L.d_items, L.items, s)) != HM_OK) return st;
        if ((st = upload(h, &L.d_small, small, s)) != HM_OK) return st;
        if ((st = upload(h, &L.d_big, big, s)) != HM_OK) return st;
        // the residual's own list (balanced for its round-robin warps) and the block bounds
        // of that list and of the big part
        const std::vector<Item> res = balanced_order(L.items, residual_warps(h), residual_cost);
        if ((st = upload(h, &L.d_res, res, s)) != HM_OK) return st;
        if ((st = dev_alloc(h, (void **)&L.d_bnd, sizeof(float4) * res.size())) != HM_OK) return st;
        if ((st = dev_alloc(h, (void **)&L.d_bnd_big, sizeof(float4) * big.size())) != HM_OK) return st;
        launch_item_bounds(L.d_res, (int64_t)res.size(), h->d_pool32, L.d_bnd, s);
        launch_item_bounds(L.d_big, L.n_big, h->d_pool32, L.d_bnd_big, s);
        HM_CUDA(cudaGetLastError());
        if ((st = upload(h, &L.d_tcu, tc.units, s)) != HM_OK) return st;
        if ((st = upload(h, &L.d_tco, tc.ops, s)) != HM_OK) return st;
        if ((st = upload(h, &L.d_tcb, tc.batches, s)) != HM_OK) return st;
        if ((st = upload(h, &L.d_tcr, tc.rows, s)) != HM_OK) return st;
        if ((st = upload(h, &L.d_tcc, tc.tchunks, s)) != HM_OK) return st;
        // the product's lists with tall dense blocks cut into row panels: a panel of rows
        // [r, r + mr) of a row-major block is itself a dense item with the same row stride
        auto panels = [](const std::vector<Item> &in, std::vector<Item> &out) {
            bool cut = false;
            for (const Item &it : in) {
                if (it.k != 0 || it.m <= PROD_PANEL) { out.push_back(it); continue; }
                cut = true;
                for (int32_t r = 0; r < it.m; r += PROD_PANEL) {
                    Item q = it;
                    q.off = it.off + (int64_t)r * even(it.n);
                    q.row0 = it.row0 + r;
                    q.m = std::min<int32_t>(PROD_PANEL, it.m - r);
                    out.push_back(q);
                }
            }
            return cut;
        };
        std::vector<Item> pa, pb;
        panels(L.items, pa);
        panels(big, pb);
        // the product kernel hands items to its warps round-robin: sorted by cost, largest
        // first, with every other round reversed, each warp gets an even share
        pa = balanced_order(pa, product_warps(h), product_cost);
        pb = balanced_order(pb, product_warps(h), product_cost);
        L.n_prod = (int64_t)pa.size();
        L.n_prod_big = (int64_t)pb.size();
        if ((st = upload(h, &L.d_prod, pa, s)) != HM_OK) return st;
        if ((st = upload(h, &L.d_prod_big, pb, s)) != HM_OK) return st;
    }
    return HM_OK;
}

static void clear_graphs(hm_matrix h)
{
    for (auto &kv : h->graphs) cudaGraphExecDestroy(kv.second);
    h->graphs.clear();
    // recorded one-launch phase lists hold workspace pointers too
    for (auto &kv : h->persist)
        if (kv.second.d) cudaFree(kv.second.d);
    h->persist.clear();
}

static void free_handle(hm_matrix h)
{
    if (!h) return;
    clear_graphs(h);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->d_bar) cudaFree(h->d_bar);
    for (cudaEvent_t e : h->prof_ev) cudaEventDestroy(e);
    void *geo[] = {h->d_qpd, h->d_vtx, h->d_ucell, h->d_ufree, h->d_ucoef, h->d_rhs_w};
    for (void *p : geo)
        if (p) cudaFree(p);
    void *ptrs[] = {h->d_pperm, h->d_pleaf_off, h->d_dinv_off, h->d_leaf_n, h->d_self_off, h->d_bad_leaf,
                    h->d_self64, h->d_self32, h->d_dinv32, h->d_dinv64, h->d_pool32, h->d_pool64, h->d_status,
                    h->ws.d_acc64, h->ws.d_io, h->ws.d_part, h->d_csr_off, h->d_csr_idx, h->ws.d_xpl, h->ws.d_tct,
                    h->ws.d_own};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (auto &kv : h->levels) {
        if (kv.second.d_items) cudaFree(kv.second.d_items);
        if (kv.second.d_prod) cudaFree(kv.second.d_prod);
        if (kv.second.d_prod_big) cudaFree(kv.second.d_prod_big);
        if (kv.second.d_small) cudaFree(kv.second.d_small);
        if (kv.second.d_big) cudaFree(kv.second.d_big);
        if (kv.second.d_res) cudaFree(kv.second.d_res);
        if (kv.second.d_bnd) cudaFree(kv.second.d_bnd);
        if (kv.second.d_bnd_big) cudaFree(kv.second.d_bnd_big);
        if (kv.second.d_tcu) cudaFree(kv.second.d_tcu);
        if (kv.second.d_tco) cudaFree(kv.second.d_tco);
        if (kv.second.d_tcb) cudaFree(kv.second.d_tcb);
        if (kv.second.d_tcr) cudaFree(kv.second.d_tcr);
        if (kv.second.d_tcc) cudaFree(kv.second.d_tcc);
        if (kv.second.d_xch) cudaFree(kv.second.d_xch);
        if (kv.second.d_rcu) cudaFree(kv.second.d_rcu);
        if (kv.second.d_rcp) cudaFree(kv.second.d_rcp);
        if (kv.second.d_rcb) cudaFree(kv.second.d_rcb);
    }
    for (void *p : h->ws.vec32) if (p) cudaFree(p);
    for (void *p : h->ws.vec64) if (p) cudaFree(p);
    if (h->h_status) cudaFreeHost(h->h_status);
    if (h->ws.h_pinned) cudaFreeHost(h->ws.h_pinned);
    delete h;
}

// Padded layout from perm / leaf_off; allocates the per-leaf arrays and the
// status word.  Called by every constructor once perm and leaf_off are set.
hm_status finalize_layout(hm_matrix h, cudaStream_t s)
{
    const int64_t L = h->n_leaves;
    h->pleaf_off.assign(L + 1, 0);
    for (int64_t i = 0; i < L; ++i) h->pleaf_off[i + 1] = h->pleaf_off[i] + even(h->leaf_off[i + 1] - h->leaf_off[i]);
    h->pN = h->pleaf_off[L];
    h->h_pperm.assign(h->pN, -1);
    for (int64_t i = 0; i < L; ++i)
        for (int64_t p = h->leaf_off[i]; p < h->leaf_off[i + 1]; ++p)
            h->h_pperm[h->pleaf_off[i] + (p - h->leaf_off[i])] = (int32_t)h->perm[p];
    h->dinv_off.assign(L, 0);
    h->self_off.assign(L, 0);
    int64_t doff = 0, soff = 0;
    std::vector<int64_t> leaf_n(L);
    for (int64_t i = 0; i < L; ++i) {
        const int64_t n = h->leaf_off[i + 1] - h->leaf_off[i], np = even(n);
        leaf_n[i] = n;
        h->dinv_off[i] = doff;
        h->self_off[i] = soff;
        doff += np * np;
        soff += n * n;
    }
    h->dinv_elems = doff;
    h->self_elems = soff;
    std::vector<int32_t> pl(h->pleaf_off.begin(), h->pleaf_off.end());
    hm_status st;
    if ((st = upload(h, &h->d_pperm, h->h_pperm, s)) != HM_OK) return st;
    if ((st = upload(h, &h->d_pleaf_off, pl, s)) != HM_OK) return st;
    if ((st = upload(h, &h->d_dinv_off, h->dinv_off, s)) != HM_OK) return st;
    if ((st = upload(h, &h->d_self_off, h->self_off, s)) != HM_OK) return st;
    if ((st = upload(h, &h->d_leaf_n, leaf_n, s)) != HM_OK) return st;
    if ((st = dev_alloc(h, (void **)&h->d_bad_leaf, sizeof(int))) != HM_OK) return st;
    if ((st = dev_alloc(h, (void **)&h->d_status, sizeof(int))) != HM_OK) return st;
    HM_CUDA(cudaMemsetAsync(h->d_status, 0, sizeof(int), s));
    HM_CUDA(cudaMemsetAsync(h->d_bad_leaf, 0xff, sizeof(int), s));
    HM_CUDA(cudaMallocHost((void **)&h->h_status, sizeof(int)));
    if ((st = dev_alloc(h, (void **)&h->d_dinv32, sizeof(float2) * h->dinv_elems)) != HM_OK) return st;
    if ((st = dev_alloc(h, (void **)&h->d_self32, sizeof(float2) * h->dinv_elems)) != HM_OK) return st;
    if (h->has_fp64)
        if ((st = dev_alloc(h, (void **)&h->d_dinv64, sizeof(double2) * h->dinv_elems)) != HM_OK) return st;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
    return HM_OK;
}

hm_status prepare_partials(hm_matrix h, cudaStream_t s)
{
    const int nl = std::max(h->n_levels, 1);
    std::vector<std::vector<int64_t>> lists((size_t)h->n_leaves * nl);
    auto leaf_of = [&](int64_t pp) {
        return (int64_t)(std::upper_bound(h->pleaf_off.begin(), h->pleaf_off.end(), pp) - h->pleaf_off.begin()) - 1;
    };
    int64_t off = 0;
    for (int lev = 1; lev <= nl; ++lev) {
        auto f = h->levels.find(lev);
        if (f == h->levels.end()) continue;
        for (Item &it : f->second.items) {
            const int64_t rl = even(it.m), cl = even(it.n);
            if (off > INT32_MAX - rl - cl) return fail(HM_ERR_ARG, "operator too large for the partial-slot index");
            it.pad = (int32_t)off;
            for (int64_t l = leaf_of(it.row0); l < h->n_leaves && h->pleaf_off[l] < it.row0 + rl; ++l)
                lists[l * nl + lev - 1].push_back(off + (h->pleaf_off[l] - it.row0));
            for (int64_t l = leaf_of(it.col0); l < h->n_leaves && h->pleaf_off[l] < it.col0 + cl; ++l)
                lists[l * nl + lev - 1].push_back(off + rl + (h->pleaf_off[l] - it.col0));
            off += rl + cl;
        }
    }
    h->partial_elems = off;
    std::vector<int64_t> csr_off((size_t)h->n_leaves * (nl + 1)), csr_idx;
    for (int64_t l = 0; l < h->n_leaves; ++l) {
        csr_off[l * (nl + 1)] = (int64_t)csr_idx.size();
        for (int lev = 1; lev <= nl; ++lev) {
            const auto &v = lists[l * nl + lev - 1];
            csr_idx.insert(csr_idx.end(), v.begin(), v.end());
            csr_off[l * (nl + 1) + lev] = (int64_t)csr_idx.size();
        }
    }
    hm_status st;
    if ((st = upload(h, &h->d_csr_off, csr_off, s)) != HM_OK) return st;
    if ((st = upload(h, &h->d_csr_idx, csr_idx, s)) != HM_OK) return st;
    return HM_OK;
}

// ---- solve orchestration ----------------------------------------------------------

struct SolveCtx {
    hm_matrix h;
    int nrhs, K, m;
    bool fp64;
    int prod_rb = -1, res_rb = -1;   // kernel choices (autotune), -1 = default
    cudaStream_t s;
    int64_t launches = 0;
    int64_t bytes = 0;
    size_t vbytes;   // bytes of one [nrhs][pN] vector
    std::vector<void *> Y, X, Z, W;  // per level 0..m
    // recording instead of launching (the one-launch solve): every step is appended as
    // a phase; units = the CTAs the widest phase can use (a leaf per CTA, a block per warp)
    std::vector<Phase> *rec = nullptr;
    int64_t units = 0;
    // a vector r whose first series step y = D^{-1} r (into Y[1]) a fused kernel has already
    // done (the permutation of b, the residual gather): the next P / Pflat on r skips it
    const void *y_ready = nullptr;
    // the end of the solve fused into the series step that writes fin_target (a leaf
    // update, launched): x = P^T (fin_base + fin_target) or P^T fin_target; fin_done when it ran
    const void *fin_target = nullptr;
    const float2 *fin_base = nullptr;
    float2 *fin_x = nullptr;
    int64_t fin_ldx = 0;
    bool fin_done = false;
};

static Phase phase(int op, int nrhs)
{
    Phase p;
    memset(&p, 0, sizeof(p));
    p.op = op;
    p.nrhs = nrhs;
    return p;
}

static void zero_vec(SolveCtx &c, void *p, size_t bytes)
{
    if (c.rec) {
        Phase q = phase(PH_ZERO, 1);
        q.c = p;
        q.n = (int64_t)bytes;
        c.rec->push_back(q);
        return;
    }
    cudaMemsetAsync(p, 0, bytes, c.s);
}

static void sub_vec(SolveCtx &c, const void *y, const void *w, void *out)
{
    c.launches++;
    if (c.rec) {
        Phase q = phase(PH_SUB, c.nrhs);
        q.a = y; q.b = w; q.c = out;
        q.n = c.h->pN * c.nrhs;
        c.rec->push_back(q);
        return;
    }
    launch_sub(y, w, out, c.h->pN * c.nrhs, c.fp64, c.s);
}

static size_t elem_size(bool fp64) { return fp64 ? sizeof(double2) : sizeof(float2); }

static hm_status ensure_workspace(hm_matrix h, int nrhs, int m)
{
    hm::Workspace &ws = h->ws;
    const size_t need_vecs = 4 * (size_t)(m + 1) + 8;
    if (ws.nrhs >= nrhs && ws.vec32.size() >= need_vecs && (!h->has_fp64 || ws.vec64.size() >= need_vecs))
        return HM_OK;
    clear_graphs(h);   // graphs hold the old workspace pointers
    for (void *p : ws.vec32) if (p) cudaFree(p);
    for (void *p : ws.vec64) if (p) cudaFree(p);
    if (ws.d_acc64) cudaFree(ws.d_acc64);
    if (ws.d_part) cudaFree(ws.d_part);
    ws.vec32.clear(); ws.vec64.clear(); ws.d_acc64 = nullptr; ws.d_part = nullptr;
    const int r = std::max(nrhs, ws.nrhs);
    const size_t n32 = sizeof(float2) * h->pN * r, n64 = sizeof(double2) * h->pN * r;
    ws.dev_bytes = (int64_t)(need_vecs * (n32 + (h->has_fp64 ? n64 : 0)) + 2 * sizeof(double) * r);
    for (size_t i = 0; i < need_vecs; ++i) {
        void *p = nullptr;
        HM_CUDA(cudaMalloc(&p, n32));
        HM_CUDA(cudaMemset(p, 0, n32));
        ws.vec32.push_back(p);
        if (h->has_fp64) {
            HM_CUDA(cudaMalloc(&p, n64));
            HM_CUDA(cudaMemset(p, 0, n64));
            ws.vec64.push_back(p);
        }
    }
    HM_CUDA(cudaMalloc((void **)&ws.d_acc64, 2 * sizeof(double) * r));
    if (ws.d_xpl) cudaFree(ws.d_xpl);
    ws.d_xpl = nullptr;
    ws.xpl_bytes = 0;
    if (ws.d_own) cudaFree(ws.d_own);   // owner sums: ensure_own
    ws.d_own = nullptr;
    ws.own_bytes = 0;
    if (ws.d_tct) cudaFree(ws.d_tct);   // stage-1 results of the tensor-core product: ensure_tct
    ws.d_tct = nullptr;
    ws.tct_bytes = 0;
    if (r >= MRHS_MIN_RHS && h->tc_max_xch > 0) {   // split x of the tensor-core product (it can be pinned from 4 RHS)
        ws.xpl_bytes = tc_xplane_bytes(h->tc_max_xch, r);
        HM_CUDA(cudaMalloc((void **)&ws.d_xpl, ws.xpl_bytes));
        ws.dev_bytes += (int64_t)ws.xpl_bytes;
    }
    ws.part_rhs = std::min(r, RESID_CHUNK);   // the partial slots themselves: ensure_partials
    ws.nrhs = r;
    return HM_OK;
}

// FP64 owner sums of the owner-computes residual ([level][RHS][pN] for the
// workspace's RHS count and m levels); allocated only by the calls that form a
// residual with that kernel, before any capture
static hm_status ensure_own(hm_matrix h, int m)
{
    hm::Workspace &ws = h->ws;
    const size_t bytes = sizeof(double2) * (size_t)std::max(m, 1) * (size_t)ws.nrhs * (size_t)h->pN;
    if (ws.d_own && ws.own_bytes >= bytes) return HM_OK;
    clear_graphs(h);   // graphs hold the old pointer
    if (ws.d_own) {
        cudaFree(ws.d_own);
        ws.dev_bytes -= (int64_t)ws.own_bytes;
    }
    ws.d_own = nullptr;
    ws.own_bytes = 0;
    HM_CUDA(cudaMalloc((void **)&ws.d_own, bytes));
    ws.own_bytes = bytes;
    ws.dev_bytes += (int64_t)bytes;
    return HM_OK;
}

// stage-1 results of the tensor-core product (T chunks of the largest level for the
// workspace's RHS tiles); allocated only by the calls that run that product, before
// any capture
static hm_status ensure_tct(hm_matrix h)
{
    hm::Workspace &ws = h->ws;
    const size_t bytes = tc_t_bytes(h->tc_max_tchunk, ws.nrhs);
    if (bytes == 0 || (ws.d_tct && ws.tct_bytes >= bytes)) return HM_OK;
    clear_graphs(h);   // graphs hold the old pointer
    if (ws.d_tct) {
        cudaFree(ws.d_tct);
        ws.dev_bytes -= (int64_t)ws.tct_bytes;
    }
    ws.d_tct = nullptr;
    ws.tct_bytes = 0;
    HM_CUDA(cudaMalloc((void **)&ws.d_tct, bytes));
    ws.tct_bytes = bytes;
    ws.dev_bytes += (int64_t)bytes;
    return HM_OK;
}

// the owner-computes residual applies when every level 1..m holds only items it takes
static bool own_applies(hm_matrix h, int m)
{
    bool any = false;
    for (int lev = 1; lev <= m; ++lev) {
        auto it = h->levels.find(lev);
        if (it == h->levels.end() || it->second.items.empty()) continue;
        if (it->second.n_big > 0) return false;
        any = true;
    }
    return any;
}

// Double-float partial slots of the residual products (ws.part_rhs right-hand sides at a
// time); allocated only by the calls that form a residual, before any capture
static hm_status ensure_partials(hm_matrix h)
{
    hm::Workspace &ws = h->ws;
    if (ws.d_part) return HM_OK;
    const size_t bytes = sizeof(dot2::cdf) * std::max<int64_t>(h->partial_elems, 1) * std::max(ws.part_rhs, 1);
    HM_CUDA(cudaMalloc((void **)&ws.d_part, bytes));
    ws.dev_bytes += (int64_t)bytes;
    return HM_OK;
}

static int64_t level_bytes(hm_matrix h, int lev, bool fp64)
{
    auto it = h->levels.find(lev);
    return it == h->levels.end() ? 0 : it->second.elems * (int64_t)elem_size(fp64);
}

// z (zeroed) += M_lev x
static void apply_level(SolveCtx &c, int lev, const void *x, void *z)
{
    auto it = c.h->levels.find(lev);
    if (it == c.h->levels.end() || it->second.items.empty()) return;
    hm_matrix h = c.h;
    if (c.rec) {
        Phase q = phase(PH_APPLY, c.nrhs);
        q.a = x; q.c = z;
        q.items = it->second.d_prod ? it->second.d_prod : it->second.d_items;
        q.n = it->second.d_prod ? it->second.n_prod : (int64_t)it->second.items.size();
        c.rec->push_back(q);
        c.units = std::max<int64_t>(c.units, (q.n + 7) / 8);   // a block per warp
        c.launches++;
        c.bytes += level_bytes(c.h, lev, c.fp64) * c.nrhs;
        return;
    }
    const bool timed = h->prof && !c.fp64;
    if (timed) {
        if (h->prof_used + 2 > h->prof_ev.size() && h->prof_ev.size() < 8192) {
            for (int q = 0; q < 256; ++q) {
                cudaEvent_t e;
                if (cudaEventCreate(&e) != cudaSuccess) break;
                h->prof_ev.push_back(e);
            }
        }
        if (h->prof_used + 2 <= h->prof_ev.size()) cudaEventRecord(h->prof_ev[h->prof_used], c.s);
    }
    const int launched = launch_apply_items(c.h, it->second, x, z, c.nrhs, c.fp64, c.s, c.prod_rb);
    if (timed && h->prof_used + 2 <= h->prof_ev.size()) {
        cudaEventRecord(h->prof_ev[h->prof_used + 1], c.s);
        h->prof_used += 2;
        h->prof_launches++;
        // algorithmic bytes: every stored block once, x read and z written once per right-hand side
        h->prof_bytes += it->second.alg_elems * 8 + 2 * 8 * h->N * (int64_t)c.nrhs;
    }
    c.launches += launched;
    c.bytes += level_bytes(c.h, lev, c.fp64) * c.nrhs;
}

// bytes a leaf update streams (D^{-1}, and the y / z / out vectors)
static int64_t leaf_update_bytes(const SolveCtx &c)
{
    return c.h->dinv_elems * (int64_t)elem_size(c.fp64) + 3 * (int64_t)c.vbytes;
}

static void leaf_update(SolveCtx &c, const void *y, void *zin, void *out, bool zero_in)
{
    if (c.rec) {
        Phase q = phase(PH_LEAF, c.nrhs);
        q.a = y; q.b = zin; q.c = out;
        q.m = zero_in ? 1 : 0;
        c.rec->push_back(q);
        c.units = std::max<int64_t>(c.units, c.h->n_leaves * c.nrhs);
    } else {
        launch_leaf_update(c.h, y, zin, out, c.nrhs, zero_in, c.fp64, c.s);
    }
    c.launches++;
    c.bytes += leaf_update_bytes(c);
}

static void copy_vec(SolveCtx &c, void *dst, const void *src)
{
    if (c.rec) {
        Phase q = phase(PH_COPY, 1);
        q.a = src; q.c = dst;
        q.n = (int64_t)c.vbytes;
        c.rec->push_back(q);
        return;
    }
    cudaMemcpyAsync(dst, src, c.vbytes, cudaMemcpyDeviceToDevice, c.s);
}

// x_j = y - D^{-1} z into dst (z cleared), fused with the end of the solve when dst is its target
static void last_leaf_update(SolveCtx &c, const void *Y, void *Z, void *dst)
{
    if (!c.rec && !c.fp64 && c.fin_target == dst) {
        launch_leaf_finish(c.h, (const float2 *)Y, (float2 *)Z, (float2 *)dst, c.fin_base, c.fin_x, c.fin_ldx, c.nrhs,
                           c.s);
        c.launches++;
        c.bytes += leaf_update_bytes(c);
        c.fin_done = true;
        return;
    }
    leaf_update(c, Y, Z, dst, true);
}

// P_level(r) -> out (eq. 19 nested recursion); out must not alias r.
// Invariant: Z[1] is all zero on entry and on exit.
static void P(SolveCtx &c, int level, const void *r, void *out)
{
    if (level == 0) {
        leaf_update(c, nullptr, const_cast<void *>(r), out, false);
        return;
    }
    if (level == 1) {
        void *Y = c.Y[1], *X = c.X[1], *Z = c.Z[1];
        if (c.y_ready == r) c.y_ready = nullptr;                       // y = D^{-1} r done with r
        else leaf_update(c, nullptr, const_cast<void *>(r), Y, false); // y = D^{-1} r
        const void *cur = Y;
        for (int j = 1; j <= c.K; ++j) {
            apply_level(c, 1, cur, Z);                                 // z = M_1 x_{j-1}
            void *dst = (j == c.K) ? out : X;
            last_leaf_update(c, Y, Z, dst);                            // x_j = y - D^{-1} z
            cur = dst;
        }
        if (c.K == 0) copy_vec(c, out, Y);
        return;
    }
    void *Y = c.Y[level], *X = c.X[level], *Z = c.Z[level], *W = c.W[level];
    P(c, level - 1, r, Y);                                              // y = P_{m-1}(r)
    const void *cur = Y;
    for (int j = 1; j <= c.K; ++j) {
        zero_vec(c, Z, c.vbytes);
        apply_level(c, level, cur, Z);                                  // z = M_m x
        P(c, level - 1, Z, W);                                          // w = P_{m-1}(z)
        void *dst = (j == c.K) ? out : X;
        sub_vec(c, Y, W, dst);                                          // x = y - w
        cur = dst;
    }
    if (c.K == 0) copy_vec(c, out, Y);
}

// Flat form: x = S_K(D^{-1}(A_m - D)) D^{-1} r
static void Pflat(SolveCtx &c, const void *r, void *out)
{
    void *Y = c.Y[1], *X = c.X[1], *Z = c.Z[1];
    if (c.y_ready == r) c.y_ready = nullptr;                           // y = D^{-1} r done with r
    else leaf_update(c, nullptr, const_cast<void *>(r), Y, false);
    const void *cur = Y;
    for (int j = 1; j <= c.K; ++j) {
        for (int lev = 1; lev <= c.m; ++lev) apply_level(c, lev, cur, Z);
        void *dst = (j == c.K) ? out : X;
        last_leaf_update(c, Y, Z, dst);
        cur = dst;
    }
    if (c.K == 0) copy_vec(c, out, Y);
}

// Estimates of the level operators U_l = D^{-1} M_l (§IV: the series of (I + U_l)^{-1}
// converges when the spectral radius of U_l is below one; the paper's operating bound is
// a norm below 0.1).  Per level with blocks, two power iterations of n_iter steps from
// deterministic start vectors, one right-hand side, complex64 vectors:
//  - on U: v <- U v / |U v|; rho_est = geometric mean of |U v| over the second half
//    of the steps (the growth rate of U^k v, which tends to the spectral radius when one
//    eigenvalue of largest modulus dominates);
//  - on U^H U: norm_est = |U v| for the final unit iterate v of (U^H U)^k v0, a lower
//    bound of ||U||_2 that rises to it (Rayleigh quotients of power iterates of a
//    positive semidefinite matrix do not decrease).  U^H y = conj(M D^{-1} conj(y))
//    because M and D are complex symmetric (the half storage of §III mirrors every
//    stored block by its transpose).
static hm_status estimate_norms(hm_matrix h, int n_iter, cudaStream_t s)
{
    SolveCtx c;
    c.h = h; c.nrhs = 1; c.K = 0; c.fp64 = false; c.s = s;
    c.m = std::max(h->n_levels, 1);
    c.vbytes = sizeof(float2) * h->pN;
    hm_status st = ensure_workspace(h, 1, c.m);
    if (st != HM_OK) return st;
    const bool prof = h->prof;
    h->prof = false;   // these products are not part of any timed solve
    float2 *v = (float2 *)h->ws.vec32[0], *t = (float2 *)h->ws.vec32[1], *z = (float2 *)h->ws.vec32[2],
           *u = (float2 *)h->ws.vec32[3];
    const int nl = std::min(c.m, 16);
    const size_t nrec = (size_t)nl * 2 * n_iter + 1;   // [level][rho | norm][step], then one scratch
    double *d = nullptr;
    HM_CUDA(cudaMalloc((void **)&d, nrec * sizeof(double)));
    HM_CUDA(cudaMemsetAsync(d, 0, nrec * sizeof(double), s));
    double *scratch = d + nrec - 1;
    const int64_t n = h->pN;
    std::vector<bool> has(nl + 1, false);
    for (int lev = 1; lev <= nl; ++lev) {
        auto it = h->levels.find(lev);
        if (it == h->levels.end() || it->second.items.empty()) continue;
        has[lev] = true;
        double *rec_rho = d + (size_t)(lev - 1) * 2 * n_iter, *rec_nrm = rec_rho + n_iter;
        cudaMemsetAsync(z, 0, c.vbytes, s);
        for (int pass = 0; pass < 2; ++pass) {
            launch_seed_vector(v, h->d_pperm, n, 0x5EED0000u + 16u * lev + pass, s);
            launch_norm2(v, n, scratch, s);
            launch_conj_scale(v, v, n, scratch, false, s);
            for (int k = 0; k < n_iter; ++k) {
                apply_level(c, lev, v, z);                     // z = M_l v
                leaf_update(c, nullptr, z, u, true);           // u = D^{-1} z = U v; z = 0
                if (pass == 0) {
                    launch_norm2(u, n, rec_rho + k, s);
                    launch_conj_scale(u, v, n, rec_rho + k, false, s);     // v = U v / |U v|
                } else {
                    launch_norm2(u, n, rec_nrm + k, s);
                    launch_conj_scale(u, v, n, rec_nrm + k, true, s);      // v = conj(U v) / |U v|
                    leaf_update(c, nullptr, v, t, false);
                    apply_level(c, lev, t, z);                             // z = conj(U^H U v) / |U v|
                    launch_norm2(z, n, scratch, s);
                    launch_conj_scale(z, v, n, scratch, true, s);          // v = U^H U v / |U^H U v|
                    cudaMemsetAsync(z, 0, c.vbytes, s);
                }
            }
        }
    }
    std::vector<double> hrec(nrec, 0.0);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(hrec.data(), d, nrec * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    h->prof = prof;
    if (e != cudaSuccess) return cuda_fail(e, "level-operator norm estimate");
    for (int l = 0; l < 16; ++l) h->norm_est[l] = h->rho_est[l] = 0.0;
    for (int lev = 1; lev <= nl; ++lev) {
        if (!has[lev]) continue;
        const double *rr = hrec.data() + (size_t)(lev - 1) * 2 * n_iter, *rn = rr + n_iter;
        double acc = 0.0;
        bool zero = false;
        for (int k = n_iter / 2; k < n_iter; ++k) {
            if (!(rr[k] > 0.0)) { zero = true; break; }
            acc += 0.5 * std::log(rr[k]);
        }
        h->rho_est[lev - 1] = zero ? 0.0 : std::exp(acc / (n_iter - n_iter / 2));
        h->norm_est[lev - 1] = std::sqrt(std::max(rn[n_iter - 1], 0.0));
    }
    h->norm_iters = n_iter;
    return HM_OK;
}

static int clamp_levels(hm_matrix h, int n_levels)
{
    int m = (n_levels < 0 || n_levels > h->n_levels) ? h->n_levels : n_levels;
    return std::max(m, 1);
}

// out = b - A_m x (with |r|^2, |b|^2 per column into norms) when b is given, else
// out = A_m x; complex64 blocks, FP64 products and sums, deterministic order:
// every block writes its double-float partial slots, then each leaf gathers its slots.
// y_next: when given, the series step that follows (y = D^{-1} out into Y[1]) is done in
// the gather's pass where that applies (one chunk of partial slots, launched), and
// c.y_ready tells the next P / Pflat so
static void residual64(SolveCtx &c, const float2 *xt, const float2 *bt, float2 *out, double *norms,
                       float2 *y_next = nullptr)
{
    hm_matrix h = c.h;
    if (!c.rec && c.res_rb == RB_OWN && h->ws.d_own &&
        h->ws.own_bytes >= sizeof(double2) * (size_t)c.m * (size_t)c.nrhs * (size_t)h->pN && own_applies(h, c.m)) {
        // owner-computes: each level's sums into its own FP64 [RHS][pN] array, then one gather
        const int64_t lstride = (int64_t)c.nrhs * h->pN;
        cudaMemsetAsync(h->ws.d_own, 0, sizeof(double2) * (size_t)c.m * (size_t)lstride, c.s);
        for (int lev = 1; lev <= c.m; ++lev) {
            auto it = h->levels.find(lev);
            if (it == h->levels.end() || it->second.items.empty()) continue;
            launch_resid_own(h, it->second, xt, h->ws.d_own + (int64_t)(lev - 1) * lstride, c.nrhs, c.s);
            c.launches++;
        }
        launch_gather_own(h, xt, c.m, h->ws.d_own, lstride, bt, out, norms, c.nrhs, c.s);
        c.launches += 2;
        return;
    }
    const int chunk = std::max(1, h->ws.part_rhs);
    for (int r0 = 0; r0 < c.nrhs; r0 += chunk) {
        const int nr = std::min(chunk, c.nrhs - r0);
        const float2 *x = xt + (int64_t)r0 * h->pN;
        if (c.rec) {   // one-launch solve: the one-RHS-at-a-time partial-slot products and the gather
            for (int lev = 1; lev <= c.m; ++lev) {
                auto it = h->levels.find(lev);
                if (it == h->levels.end() || it->second.items.empty()) continue;
                Phase q = phase(PH_RESID, nr);
                q.a = x; q.c = h->ws.d_part;
                q.ld = h->partial_elems;
                q.items = it->second.d_res;
                q.d = it->second.d_bnd;
                q.n = (int64_t)it->second.items.size();
                c.rec->push_back(q);
                c.units = std::max<int64_t>(c.units, (q.n + 7) / 8);   // a block per warp
                c.launches++;
            }
            Phase g = phase(PH_GATHER, nr);
            g.a = x;
            g.b = bt ? bt + (int64_t)r0 * h->pN : nullptr;
            g.c = out + (int64_t)r0 * h->pN;
            g.d = h->ws.d_part;
            g.ld = h->partial_elems;
            g.m = c.m;
            g.norms = norms ? norms + 2 * r0 : nullptr;
            c.rec->push_back(g);
            c.units = std::max<int64_t>(c.units, h->n_leaves * nr);
            c.launches++;
            continue;
        }
        for (int lev = 1; lev <= c.m; ++lev) {
            auto it = h->levels.find(lev);
            if (it == h->levels.end() || it->second.items.empty()) continue;
            c.launches += launch_apply_items_partials(h, it->second, x, h->ws.d_part, h->partial_elems, nr, c.s,
                                                      c.res_rb);
        }
        if (y_next && nr == c.nrhs) {
            launch_gather_leaf_update(h, x, c.m, h->ws.d_part, h->partial_elems, bt, out, norms, y_next, nr, c.s);
            c.bytes += leaf_update_bytes(c);
            c.y_ready = out;
        } else {
            launch_gather_acc64(h, x, c.m, h->ws.d_part, h->partial_elems, bt ? bt + (int64_t)r0 * h->pN : nullptr,
                                out + (int64_t)r0 * h->pN, norms ? norms + 2 * r0 : nullptr, nr, c.s);
        }
        c.launches++;
    }
}

// Autotuner of the many-right-hand-side kernels.  On the first complex64 solve,
// product or residual with a given right-hand-side count (>= MRHS_MIN_RHS), time
// on this operator, with CUDA events on the caller's stream, the leaf-level
// product with every candidate kernel (one right-hand side at a time; shared-
// memory chunks of 8, 16, 32) and the FP64-class residual products likewise (one
// at a time; chunks of 8, 16), and keep the fastest of each.  The candidates
// compute the same sums (up to the order of FP32 atomics), so the choice changes
// speed only.  It runs before any graph capture, so captured solves replay the
// chosen kernels.
// right-hand-side counts share a kernel choice per power-of-two bucket
static int tune_bucket(int nrhs)
{
    int b = MRHS_MIN_RHS;
    while (b < nrhs) b <<= 1;
    return b;
}

static hm_status autotune(hm_matrix h, int nrhs_req, int m, cudaStream_t s, bool residual)
{
    if (nrhs_req < MRHS_MIN_RHS) return HM_OK;
    const int nrhs = tune_bucket(nrhs_req);              // timed at the bucket's size
    auto have = h->tune.find(nrhs);
    if (have != h->tune.end() && (!residual || have->second.res_rb >= 0)) return HM_OK;
    auto it1 = h->levels.find(1);
    hm_matrix_s::Tune t;
    if (it1 == h->levels.end() || it1->second.items.empty() || it1->second.n_small == 0) {
        t.prod_rb = 0;
        t.res_rb = 0;
        h->tune[nrhs] = t;
        return HM_OK;
    }
    const bool do_prod = have == h->tune.end();
    if (!do_prod) t = have->second;
    const LevelList &L = it1->second;
    hm_status st = ensure_workspace(h, nrhs, m);
    if (st != HM_OK) return st;
    if (residual && (st = ensure_partials(h)) != HM_OK) return st;
    float2 *x = (float2 *)h->ws.vec32[0], *z = (float2 *)h->ws.vec32[1];
    HM_CUDA(cudaMemsetAsync(x, 0, sizeof(float2) * h->pN * nrhs, s));
    cudaEvent_t e0, e1;
    HM_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return fail(HM_ERR_CUDA, "cudaEventCreate"); }
    auto time_it = [&](auto &&launch, double &ms) -> hm_status {
        launch();                                       // warm-up (also sets kernel attributes)
        cudaEventRecord(e0, s);
        for (int r = 0; r < 3; ++r) launch();
        cudaEventRecord(e1, s);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "autotune");
        float f = 0.f;
        cudaEventElapsedTime(&f, e0, e1);
        ms = f / 3.0;
        return HM_OK;
    };
    double best = 1e30;
    const int prod_c[] = {0, 8, 16, 32, RB_TC};
    for (int rb : prod_c) {
        if (!do_prod) break;
        if (rb == RB_TC ? (nrhs < TC_MIN_RHS || L.n_tcu == 0) : (rb > 8 && rb / 2 >= nrhs))
            continue;   // a chunk of twice the RHS count or more only adds idle work; tensor tiles of 128 from 32 RHS
        double ms = 0;
        if (rb == RB_TC && (st = ensure_tct(h)) != HM_OK) break;
        if ((st = time_it([&] { launch_apply_items(h, L, x, z, nrhs, false, s, rb); }, ms)) != HM_OK) break;
        if (ms < best) { best = ms; t.prod_rb = rb; t.prod_ms = ms; }
    }
    // residual candidates, compared per right-hand side: the partial-slot kernels time a chunk of nr,
    // the owner-computes kernel all nrhs at once (when every level of the call takes it)
    const int nr = std::min(nrhs, std::max(1, h->ws.part_rhs));
    best = 1e30;
    const int res_c[] = {0, 8, 16, RB_OWN};
    for (int rb : res_c) {
        if (st != HM_OK || !residual) break;
        if (rb == RB_OWN) {
            if (!own_applies(h, m) || L.n_rcu == 0) continue;
            if ((st = ensure_own(h, m)) != HM_OK) break;
        } else if (rb > 8 && rb / 2 >= nr) {
            continue;
        }
        double ms = 0;
        if (rb == RB_OWN)
            st = time_it([&] { launch_resid_own(h, L, x, h->ws.d_own, nrhs, s); }, ms);
        else
            st = time_it([&] { launch_apply_items_partials(h, L, x, h->ws.d_part, h->partial_elems, nr, s, rb); }, ms);
        if (st != HM_OK) break;
        const double per_rhs = ms / (rb == RB_OWN ? nrhs : nr);
        if (per_rhs < best) { best = per_rhs; t.res_rb = rb; t.res_ms = ms; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != HM_OK) return st;
    h->tune[nrhs] = t;
    return HM_OK;
}

// the autotuner's (or hm_set_tuning's) kernel choices for the call, with the
// workspace the chosen product needs
static hm_status use_tuning(SolveCtx &c)
{
    if (c.nrhs < MRHS_MIN_RHS) return HM_OK;
    auto tn = c.h->tune.find(tune_bucket(c.nrhs));
    if (tn != c.h->tune.end()) {
        c.prod_rb = tn->second.prod_rb;
        c.res_rb = tn->second.res_rb;
    }
    return c.prod_rb == RB_TC ? ensure_tct(c.h) : HM_OK;
}

// permutations and vector updates of a solve, launched or recorded
static void permute_in_vec(SolveCtx &c, const void *b, int64_t ldb, void *bt)
{
    c.launches++;
    if (c.rec) {
        Phase q = phase(PH_PERMUTE_IN, c.nrhs);
        q.a = b; q.c = bt; q.ld2 = ldb;
        c.rec->push_back(q);
        return;
    }
    launch_permute_in(b, ldb, bt, c.h->pN, c.h->d_pperm, c.nrhs, c.fp64, c.s);
}

static void permute_out_vec(SolveCtx &c, const void *xt, void *x, int64_t ldx)
{
    c.launches++;
    if (c.rec) {
        Phase q = phase(PH_PERMUTE_OUT, c.nrhs);
        q.a = xt; q.c = x; q.ld2 = ldx;
        c.rec->push_back(q);
        return;
    }
    launch_permute_out(xt, c.h->pN, x, ldx, c.h->d_pperm, c.nrhs, c.fp64, c.s);
}

static void add_vec(SolveCtx &c, void *x, const void *dx)
{
    c.launches++;
    if (c.rec) {
        Phase q = phase(PH_ADD, c.nrhs);
        q.a = dx; q.c = x; q.n = c.h->pN * c.nrhs;
        c.rec->push_back(q);
        return;
    }
    launch_add_inplace(x, dx, c.h->pN * c.nrhs, false, c.s);
}

static void check_vec(SolveCtx &c, const void *x)
{
    c.launches++;
    if (c.rec) {
        Phase q = phase(PH_CHECK, c.nrhs);
        q.a = x; q.n = c.h->pN * c.nrhs;
        c.rec->push_back(q);
        return;
    }
    launch_check_finite(x, c.h->pN * c.nrhs, c.fp64, c.h->d_status, c.s);
}

// rec_out: record (or find) the one-launch phase list of this solve and return it
// without launching anything (the serving loop runs it)
static hm_status solve_device(hm_matrix h, const void *b, int64_t ldb, void *x, int64_t ldx, int nrhs,
                              const hm_solve_opts *o, cudaStream_t s, hm_solve_info *info,
                              const hm_matrix_s::PersistList **rec_out = nullptr)
{
    void *caller_stream = (void *)s;
    if (!h) return fail(HM_ERR_ARG, "null handle");
    if (!o) return fail(HM_ERR_ARG, "null opts");
    if (nrhs < 0) return fail(HM_ERR_ARG, "nrhs < 0");
    if (nrhs == 0) {
        if (info) { memset(info, 0, sizeof(*info)); info->levels_used = clamp_levels(h, o->n_levels); }
        return HM_OK;
    }
    if (!b || !x) return fail(HM_ERR_ARG, "null b or x");
    if (ldb < h->N || ldx < h->N) return fail(HM_ERR_ARG, "leading dimension < N");
    if (o->n_terms < 0 || o->n_terms > 64) return fail(HM_ERR_ARG, "n_terms out of range [0, 64]");
    if (!h->factored) return fail(HM_ERR_STATE, "hm_factor_leaf has not completed on this handle");
    if (o->fp64 && !h->has_fp64) return fail(HM_ERR_STATE, "fp64 solve needs an operator built with keep_fp64");
    if (o->fp64 && o->refine) return fail(HM_ERR_ARG, "refine applies to the complex64 path only");
    const size_t es = elem_size(o->fp64);
    {
        const char *bb = (const char *)b, *xx = (const char *)x;
        const size_t bl = es * (size_t)ldb * nrhs, xl = es * (size_t)ldx * nrhs;
        if (nrhs > 0 && bb < xx + xl && xx < bb + bl) return fail(HM_ERR_ARG, "b and x overlap");
    }
    SolveCtx c;
    c.h = h; c.nrhs = nrhs; c.K = o->n_terms; c.fp64 = o->fp64 != 0; c.s = s;
    c.m = clamp_levels(h, o->n_levels);
    c.vbytes = es * h->pN * nrhs;
    hm_status st = ensure_workspace(h, nrhs, c.m);
    if (st != HM_OK) return st;
    const bool resid = !o->fp64 && (o->refine || info);
    if (resid && (st = ensure_partials(h)) != HM_OK) return st;
    const bool persist = (o->persistent || rec_out) && !c.fp64 && persist_supported(h);
    if (rec_out && !persist) return fail(HM_ERR_ARG, "the operator does not fit the one-launch solve");
    if (!c.fp64 && !persist) {
        if ((st = autotune(h, nrhs, c.m, s, resid)) != HM_OK) return st;
        if ((st = use_tuning(c)) != HM_OK) return st;
        if (resid && c.res_rb == RB_OWN && own_applies(h, c.m) && (st = ensure_own(h, c.m)) != HM_OK) return st;
    }
    if (persist) {   // the one-launch solve runs the one-right-hand-side-at-a-time block bodies
        c.prod_rb = 0;
        c.res_rb = 0;
        if (!h->d_bar) HM_CUDA(cudaMalloc((void **)&h->d_bar, 2 * sizeof(unsigned)));
    }
    const bool use_graph = o->graph && !info && !h->prof && !rec_out;
    hm_matrix_s::GraphKey key{b, x, ldb, ldx, nrhs, c.K, c.m, o->nested, o->refine, o->fp64,
                              persist ? (info ? 2 : 1) : 0};
    if (use_graph) {
        auto g = h->graphs.find(key);
        if (g != h->graphs.end()) {
            HM_CUDA(cudaGraphLaunch(g->second, s));
            return HM_OK;
        }
    }
    std::vector<void *> &V = c.fp64 ? h->ws.vec64 : h->ws.vec32;
    size_t vi = 0;
    c.Y.assign(c.m + 1, nullptr); c.X = c.Y; c.Z = c.Y; c.W = c.Y;
    for (int l = 1; l <= c.m; ++l) { c.Y[l] = V[vi++]; c.X[l] = V[vi++]; c.Z[l] = V[vi++]; c.W[l] = V[vi++]; }
    void *bt = V[vi++], *xt = V[vi++], *rt = V[vi++], *dx = V[vi++];
    double *norms = o->refine ? h->ws.d_acc64 : nullptr;
    // the solve's steps, launched or recorded (the one-launch solve) through c
    auto steps = [&](SolveCtx &cc) {
        // complex64, launched: the permutation of b and the series' first step in one pass
        const bool fuse = !cc.rec && !cc.fp64;
        if (fuse) {
            launch_permute_leaf(h, (const float2 *)b, ldb, (float2 *)bt, (float2 *)cc.Y[1], nrhs, cc.s);
            cc.launches++;
            cc.bytes += leaf_update_bytes(cc);
            cc.y_ready = bt;
        } else {
            permute_in_vec(cc, b, ldb, bt);
        }
        // the end of the solve (add, check, un-permute) goes with the last leaf update where one
        // writes the solve's last vector (leaf-level nested, or flat), else as its own pass
        auto finish_with = [&](const void *target, const float2 *base) {
            if (!fuse || info) return;
            cc.fin_target = target;
            cc.fin_base = base;
            cc.fin_x = (float2 *)x;
            cc.fin_ldx = ldx;
            cc.fin_done = false;
        };
        if (!o->refine) finish_with(xt, nullptr);
        if (o->nested) P(cc, cc.m, bt, xt);
        else Pflat(cc, bt, xt);
        cc.fin_target = nullptr;
        if (o->refine) {
            zero_vec(cc, norms, 2 * sizeof(double) * nrhs);
            residual64(cc, (const float2 *)xt, (const float2 *)bt, (float2 *)rt, norms,
                       fuse ? (float2 *)cc.Y[1] : nullptr);
            finish_with(dx, (const float2 *)xt);
            if (o->nested) P(cc, cc.m, rt, dx);
            else Pflat(cc, rt, dx);
            cc.fin_target = nullptr;
            if (cc.fin_done) return;
            if (!cc.rec && !info) {   // add, check and un-permute in one kernel
                launch_finish((const float2 *)xt, (const float2 *)dx, h->pN, (float2 *)x, ldx, h->d_pperm, nrhs,
                              h->d_status, cc.s);
                cc.launches++;
                return;
            }
            add_vec(cc, xt, dx);
            if (info) {   // residual of the refined solution
                zero_vec(cc, norms, 2 * sizeof(double) * nrhs);
                residual64(cc, (const float2 *)xt, (const float2 *)bt, (float2 *)rt, norms);
            }
        } else if (!cc.rec && !cc.fp64) {
            if (cc.fin_done) return;
            launch_finish((const float2 *)xt, nullptr, h->pN, (float2 *)x, ldx, h->d_pperm, nrhs, h->d_status, cc.s);
            cc.launches++;
            return;
        }
        check_vec(cc, xt);
        permute_out_vec(cc, xt, x, ldx);
    };
    const hm_matrix_s::PersistList *pl = nullptr;
    if (persist) {
        auto it = h->persist.find(key);
        if (it == h->persist.end()) {
            std::vector<Phase> rec;
            SolveCtx r = c;
            r.rec = &rec;
            steps(r);
            // barriers that can go: zeroing the norms before the residual products (only the
            // gather, a barrier later, reads them); the elementwise tail add -> check ->
            // permute-out, where every thread reads only the elements it wrote itself
            for (size_t q = 0; q + 1 < rec.size(); ++q) {
                const int a = rec[q].op, nx = rec[q + 1].op;
                if (a == PH_ZERO && nx == PH_RESID && rec[q].c == (void *)norms) rec[q].pad = 1;
                if ((a == PH_ADD && (nx == PH_CHECK || nx == PH_PERMUTE_OUT)) ||
                    (a == PH_CHECK && nx == PH_PERMUTE_OUT))
                    rec[q].pad = 1;
            }
            hm_matrix_s::PersistList l;
            l.n = (int)rec.size();
            l.units = (int)std::min<int64_t>(r.units, 1 << 30);
            l.launches = r.launches;
            l.bytes = r.bytes;
            HM_CUDA(cudaMalloc((void **)&l.d, rec.size() * sizeof(Phase)));
            HM_CUDA(cudaMemcpy(l.d, rec.data(), rec.size() * sizeof(Phase), cudaMemcpyHostToDevice));
            it = h->persist.emplace(key, l).first;
        }
        pl = &it->second;
        if (rec_out) {
            *rec_out = pl;
            return HM_OK;
        }
    }
    if (use_graph) {
        if (!h->cap_stream) HM_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
        HM_CUDA(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
        c.s = h->cap_stream;
        s = h->cap_stream;
    }
    if (persist) {
        st = launch_persist(h, pl->d, pl->n, pl->units, s);
        c.launches = 1;            // one kernel (the recorded list replaces pl->launches launches)
        c.bytes = pl->bytes;
        if (st != HM_OK) {
            if (use_graph) {
                cudaGraph_t g = nullptr;
                cudaStreamEndCapture(h->cap_stream, &g);
                if (g) cudaGraphDestroy(g);
            }
            return st;
        }
    } else {
        steps(c);
    }
    if (use_graph) {
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(h->cap_stream, &graph);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
        h->graphs[key] = exec;
        HM_CUDA(cudaGraphLaunch(exec, (cudaStream_t)caller_stream));
        return HM_OK;
    }
    HM_CUDA(cudaGetLastError());
    if (info) {
        memset(info, 0, sizeof(*info));
        info->levels_used = c.m;
        info->kernel_launches = c.launches;
        info->bytes_streamed = c.bytes;
        info->convergent = h->norm_iters > 0 ? 1 : -1;
        for (int l = 0; l < std::min(c.m, 16); ++l) {
            info->norm_est[l] = h->norm_est[l];
            info->rho_est[l] = h->rho_est[l];
            if (h->norm_iters > 0 && h->rho_est[l] >= 1.0) info->convergent = 0;
        }
        HM_CUDA(cudaStreamSynchronize(s));
        if (norms) {
            std::vector<double> hn(2 * nrhs);
            HM_CUDA(cudaMemcpy(hn.data(), norms, hn.size() * sizeof(double), cudaMemcpyDeviceToHost));
            double worst = 0.0;
            for (int r = 0; r < nrhs; ++r)
                worst = std::max(worst, hn[2 * r + 1] > 0 ? std::sqrt(hn[2 * r] / hn[2 * r + 1]) : 0.0);
            info->rel_residual = worst;
        }
        int stv = 0;
        HM_CUDA(cudaMemcpy(&stv, h->d_status, sizeof(int), cudaMemcpyDeviceToHost));
        if (stv != 0) {
            cudaMemset(h->d_status, 0, sizeof(int));
            return fail((hm_status)stv, stv == HM_ERR_DIVERGED ? "device reported non-finite values in the solution"
                                        : "device status word reported an error during the solve");
        }
    }
    return HM_OK;
}

hm_status persist_phases(hm_matrix h, const void *b, void *x, int nrhs, const hm_solve_opts *o,
                         const Phase **phases, int *n_phases)
{
    const hm_matrix_s::PersistList *pl = nullptr;
    const hm_status st = solve_device(h, b, h->N, x, h->N, nrhs, o, nullptr, nullptr, &pl);
    if (st != HM_OK) return st;
    *phases = pl->d;
    *n_phases = pl->n;
    return HM_OK;
}

} // namespace hm

using namespace hm;

// ---- import of explicit blocks ---------------------------------------------------------

static hm_status import_blocks(const hm_blocks *B, cudaStream_t s, hm_matrix h)
{
    const int64_t N = B->n;
    h->N = N;
    h->perm.assign(B->perm, B->perm + N);
    {
        std::vector<char> seen(N, 0);
        for (int64_t p = 0; p < N; ++p) {
            const int64_t v = h->perm[p];
            if (v < 0 || v >= N || seen[v]) return fail(HM_ERR_ARG, "perm is not a permutation of 0..n-1");
            seen[v] = 1;
        }
    }
    if (B->n_leaves < 1) return fail(HM_ERR_ARG, "n_leaves < 1");
    h->n_leaves = B->n_leaves;
    h->leaf_off.assign(B->leaf_off, B->leaf_off + B->n_leaves + 1);
    if (h->leaf_off[0] != 0 || h->leaf_off[h->n_leaves] != N) return fail(HM_ERR_ARG, "leaf_off must run from 0 to n");
    for (int64_t i = 0; i < h->n_leaves; ++i) {
        const int64_t n = h->leaf_off[i + 1] - h->leaf_off[i];
        if (n < 1) return fail(HM_ERR_ARG, "empty leaf");
        if (n > factor_max_leaf()) return fail(HM_ERR_ARG, "leaf larger than the device factorisation supports");
    }
    h->has_fp64 = B->keep_fp64 != 0;
    hm_status st = finalize_layout(h, s);
    if (st != HM_OK) return st;
    // leaf index of each tree position, and leaf start lookup
    std::vector<int64_t> leaf_of(N);
    std::map<int64_t, int64_t> leaf_start, leaf_end;
    for (int64_t i = 0; i < h->n_leaves; ++i) {
        for (int64_t p = h->leaf_off[i]; p < h->leaf_off[i + 1]; ++p) leaf_of[p] = i;
        leaf_start[h->leaf_off[i]] = i;
        leaf_end[h->leaf_off[i + 1]] = i;
    }
    auto cluster = [&](int64_t r0, int64_t m, int64_t &pr0, int64_t &pm) -> bool {
        if (m < 1 || r0 < 0 || r0 + m > N) return false;
        auto a = leaf_start.find(r0);
        auto b = leaf_end.find(r0 + m);
        if (a == leaf_start.end() || b == leaf_end.end()) return false;
        pr0 = h->pleaf_off[a->second];
        pm = h->pleaf_off[b->second + 1] - pr0;
        return true;
    };
    auto ppos = [&](int64_t p) { const int64_t l = leaf_of[p]; return h->pleaf_off[l] + (p - h->leaf_off[l]); };

    // self blocks
    std::vector<double2> self64(h->self_elems);
    std::memcpy(self64.data(), B->self, sizeof(double2) * h->self_elems);
    if ((st = upload(h, &h->d_self64, self64, s)) != HM_OK) return st;

    // items and pool layout
    struct Pending { int level; Item it; int64_t src; int32_t tm, tn; int64_t trow0, tcol0; };
    std::vector<Pending> pend;
    int64_t pool = 0;
    int64_t nsrc = 0;
    for (int64_t b = 0; b < B->n_near; ++b) {
        const int64_t r0 = B->near_row0[b], c0 = B->near_col0[b];
        const int64_t m = B->near_m[b], n = B->near_n[b];
        if (r0 < 0 || c0 < 0 || r0 + m > N || c0 + n > N || m < 1 || n < 1)
            return fail(HM_ERR_ARG, "near block out of range");
        if (leaf_start.count(r0) == 0 || leaf_of[r0 + m - 1] != leaf_of[r0] || leaf_end.count(r0 + m) == 0 ||
            leaf_start.count(c0) == 0 || leaf_end.count(c0 + n) == 0 || leaf_of[c0 + n - 1] != leaf_of[c0])
            return fail(HM_ERR_ARG, "near blocks must couple two whole leaves");
        if (r0 + m > c0) return fail(HM_ERR_ARG, "near block rows must lie before its columns (half storage)");
        Item it{};
        it.off = pool; it.row0 = (int32_t)ppos(r0); it.col0 = (int32_t)ppos(c0);
        it.m = (int32_t)m; it.n = (int32_t)n; it.k = 0;
        pool += item_elems(it);
        pend.push_back({1, it, nsrc, (int32_t)m, (int32_t)n, r0, c0});
        nsrc += m * n;
    }
    int64_t usrc = 0;
    int max_level = 1, max_rank = 0;
    std::vector<int64_t> far_src(B->n_far);
    for (int64_t b = 0; b < B->n_far; ++b) {
        const int lev = B->far_level[b];
        const int64_t r0 = B->far_row0[b], c0 = B->far_col0[b];
        const int64_t m = B->far_m[b], n = B->far_n[b], k = B->far_rank[b];
        if (lev < 1 || lev > 16) return fail(HM_ERR_ARG, "far level out of range [1, 16]");
        if (k < 1 || k > 4096) return fail(HM_ERR_ARG, "far rank out of range");
        int64_t pr0, pm, pc0, pn;
        if (!cluster(r0, m, pr0, pm) || !cluster(c0, n, pc0, pn))
            return fail(HM_ERR_ARG, "far block rows/cols must be unions of whole leaves");
        if (r0 + m > c0) return fail(HM_ERR_ARG, "far block rows must lie before its columns (half storage)");
        Item it{};
        it.off = pool; it.row0 = (int32_t)pr0; it.col0 = (int32_t)pc0;
        it.m = (int32_t)pm; it.n = (int32_t)pn; it.k = (int32_t)k;
        pool += item_elems(it);
        far_src[b] = usrc;
        pend.push_back({lev, it, b, (int32_t)m, (int32_t)n, r0, c0});
        usrc += k * (m + n);
        max_level = std::max(max_level, lev);
        max_rank = std::max<int>(max_rank, (int)k);
    }
    h->pool_elems = pool;
    h->n_levels = max_level;
    h->max_rank = max_rank;
    // fill host pools
    std::vector<float2> p32(pool, make_float2(0.f, 0.f));
    std::vector<double2> p64;
    if (h->has_fp64) p64.assign(pool, make_double2(0.0, 0.0));
    const double2 *nv = reinterpret_cast<const double2 *>(B->near_vals);
    const double2 *fu = reinterpret_cast<const double2 *>(B->far_u);
    const double2 *fv = reinterpret_cast<const double2 *>(B->far_v);
    int64_t uo = 0, vo = 0;   // running offsets into far_u / far_v
    std::vector<int64_t> uoff(B->n_far), voff(B->n_far);
    for (int64_t b = 0; b < B->n_far; ++b) {
        uoff[b] = uo; voff[b] = vo;
        uo += (int64_t)B->far_m[b] * B->far_rank[b];
        vo += (int64_t)B->far_rank[b] * B->far_n[b];
    }
    auto put = [&](int64_t dst, double2 v) {
        p32[dst] = make_float2((float)v.x, (float)v.y);
        if (h->has_fp64) p64[dst] = v;
    };
    for (const Pending &pd : pend) {
        const Item &it = pd.it;
        if (it.k == 0) {
            const int64_t ld = even(it.n);
            for (int64_t i = 0; i < it.m; ++i)
                for (int64_t j = 0; j < it.n; ++j) put(it.off + i * ld + j, nv[pd.src + i * it.n + j]);
        } else {
            const int64_t b = pd.src, k = it.k;
            const int64_t m = pd.tm, n = pd.tn;
            const double2 *U = fu + uoff[b];     // m x k row-major
            const double2 *Vv = fv + voff[b];    // k x n row-major
            const int64_t vbase = it.off + k * it.m;
            for (int64_t i = 0; i < m; ++i) {
                const int64_t pi = ppos(pd.trow0 + i) - it.row0;
                for (int64_t l = 0; l < k; ++l) put(it.off + l * it.m + pi, U[i * k + l]);
            }
            for (int64_t j = 0; j < n; ++j) {
                const int64_t pj = ppos(pd.tcol0 + j) - it.col0;
                for (int64_t l = 0; l < k; ++l) put(vbase + l * it.n + pj, Vv[l * n + j]);
            }
        }
        LevelList &L = h->levels[pd.level];
        L.items.push_back(it);
        L.true_m.push_back(pd.tm);
        L.true_n.push_back(pd.tn);
        L.elems += item_elems(it);
        L.alg_elems += it.k == 0 ? (int64_t)pd.tm * pd.tn : (int64_t)it.k * (pd.tm + pd.tn);
        if (it.k == 0) L.n_dense++; else L.n_lowrank++;
    }
    (void)usrc;
    if ((st = upload(h, &h->d_pool32, p32, s)) != HM_OK) return st;
    if (h->has_fp64 && (st = upload(h, &h->d_pool64, p64, s)) != HM_OK) return st;
    if ((st = prepare_partials(h, s)) != HM_OK) return st;
    if ((st = upload_item_lists(h, s)) != HM_OK) return st;
    // tree depth is not given by the import; report the number of levels instead
    h->depth = max_level;
    HM_CUDA(cudaStreamSynchronize(s));
    return HM_OK;
}

extern "C" {

hm_status hm_build_from_blocks(const hm_blocks *blocks, void *stream, hm_matrix *out)
{
    if (!blocks || !out) return fail(HM_ERR_ARG, "null argument");
    *out = nullptr;
    const hm_blocks *B = blocks;
    if (B->n < 1 || !B->perm || !B->leaf_off || !B->self) return fail(HM_ERR_ARG, "missing n, perm, leaf_off or self");
    if (B->n > (int64_t)1 << 30) return fail(HM_ERR_ARG, "n too large");
    if (B->n_near < 0 || B->n_far < 0) return fail(HM_ERR_ARG, "negative block count");
    if (B->n_near > 0 && (!B->near_row0 || !B->near_col0 || !B->near_m || !B->near_n || !B->near_vals))
        return fail(HM_ERR_ARG, "missing near block arrays");
    if (B->n_far > 0 && (!B->far_level || !B->far_row0 || !B->far_col0 || !B->far_m || !B->far_n ||
                         !B->far_rank || !B->far_u || !B->far_v))
        return fail(HM_ERR_ARG, "missing far block arrays");
    hm_matrix h = new hm_matrix_s();
    hm_status st = import_blocks(B, (cudaStream_t)stream, h);
    if (st != HM_OK) {
        free_handle(h);
        return st;
    }
    *out = h;
    return HM_OK;
}

hm_status hm_build(const hm_mesh *mesh, const hm_build_opts *opts, void *stream, hm_matrix *out)
{
    if (!mesh || !opts || !out) return fail(HM_ERR_ARG, "null argument");
    *out = nullptr;
    return build_from_mesh(mesh, opts, (cudaStream_t)stream, out);
}

hm_status hm_factor_leaf(hm_matrix h, void *stream)
{
    if (!h) return fail(HM_ERR_ARG, "null handle");
    cudaStream_t s = (cudaStream_t)stream;
    HM_CUDA(cudaMemsetAsync(h->d_status, 0, sizeof(int), s));
    const hm_status fst = launch_factor(h, s);
    if (fst != HM_OK) return fst;
    HM_CUDA(cudaGetLastError());
    HM_CUDA(cudaStreamSynchronize(s));
    int stv = 0, bad = -1;
    HM_CUDA(cudaMemcpy(&stv, h->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    HM_CUDA(cudaMemcpy(&bad, h->d_bad_leaf, sizeof(int), cudaMemcpyDeviceToHost));
    if (stv != 0) {
        cudaMemset(h->d_status, 0, sizeof(int));
        h->factored = 0;
        return fail((hm_status)stv, "zero pivot in leaf self block " + std::to_string(bad));
    }
    h->factored = 1;
    return estimate_norms(h, HM_NORM_ITERS_DEFAULT, s);
}

hm_status hm_estimate_norms(hm_matrix h, int n_iter, void *stream)
{
    if (!h) return fail(HM_ERR_ARG, "null handle");
    if (n_iter < 2 || n_iter > 4096) return fail(HM_ERR_ARG, "n_iter out of range [2, 4096]");
    if (!h->factored) return fail(HM_ERR_STATE, "hm_factor_leaf has not completed on this handle");
    return estimate_norms(h, n_iter, (cudaStream_t)stream);
}

hm_status hm_powerseries_solve(hm_matrix h, const void *b, int64_t ldb, void *x, int64_t ldx, int nrhs,
                               const hm_solve_opts *opts, void *stream, hm_solve_info *info)
{
    return solve_device(h, b, ldb, x, ldx, nrhs, opts, (cudaStream_t)stream, info);
}

hm_status hm_powerseries_solve_host(hm_matrix h, const void *b, int64_t ldb, void *x, int64_t ldx, int nrhs,
                                    const hm_solve_opts *opts, void *stream)
{
    if (!h || !b || !x || !opts) return fail(HM_ERR_ARG, "null argument");
    if (nrhs < 0 || ldb < h->N || ldx < h->N) return fail(HM_ERR_ARG, "bad nrhs or leading dimension");
    if (nrhs == 0) return HM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t es = opts->fp64 ? sizeof(double2) : sizeof(float2);
    const size_t bytes = es * (size_t)h->N * nrhs;
    hm::Workspace &ws = h->ws;
    // page-locked caller buffers with leading dimension N are copied directly; pageable ones
    // (or strided) go through the handle's page-locked staging buffer
    auto pinned = [](const void *p) {
        cudaPointerAttributes a{};
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return a.type == cudaMemoryTypeHost;
    };
    const bool b_direct = ldb == h->N && pinned(b), x_direct = ldx == h->N && pinned(x);
    if (!(b_direct && x_direct) && ws.h_pinned_bytes < 2 * bytes) {
        if (ws.h_pinned) cudaFreeHost(ws.h_pinned);
        ws.h_pinned = nullptr;
        ws.h_pinned_bytes = 0;
        HM_CUDA(cudaMallocHost(&ws.h_pinned, 2 * bytes));
        ws.h_pinned_bytes = 2 * bytes;
    }
    if (ws.d_io_bytes < 2 * bytes) {
        if (ws.d_io) cudaFree(ws.d_io);
        ws.d_io = nullptr;
        ws.d_io_bytes = 0;
        HM_CUDA(cudaMalloc(&ws.d_io, 2 * bytes));
        ws.d_io_bytes = 2 * bytes;
    }
    char *hb = (char *)ws.h_pinned, *hx = hb ? hb + bytes : nullptr;
    char *db = (char *)ws.d_io, *dxp = db + bytes;
    if (b_direct) {
        HM_CUDA(cudaMemcpyAsync(db, b, bytes, cudaMemcpyHostToDevice, s));
    } else {
        for (int r = 0; r < nrhs; ++r)
            std::memcpy(hb + es * h->N * r, (const char *)b + es * (size_t)ldb * r, es * h->N);
        HM_CUDA(cudaMemcpyAsync(db, hb, bytes, cudaMemcpyHostToDevice, s));
    }
    hm_status st = solve_device(h, db, h->N, dxp, h->N, nrhs, opts, s, nullptr);
    if (st != HM_OK) return st;
    HM_CUDA(cudaMemcpyAsync(x_direct ? (char *)x : hx, dxp, bytes, cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaStreamSynchronize(s));
    if (!x_direct)
        for (int r = 0; r < nrhs; ++r)
            std::memcpy((char *)x + es * (size_t)ldx * r, hx + es * h->N * r, es * h->N);
    return HM_OK;
}

hm_status hm_apply(hm_matrix h, const void *x, int64_t ldx, void *y, int64_t ldy, int nrhs, int n_levels,
                   int fp64_accumulate, void *stream)
{
    if (!h || !x || !y) return fail(HM_ERR_ARG, "null argument");
    if (nrhs < 0 || ldx < h->N || ldy < h->N) return fail(HM_ERR_ARG, "bad nrhs or leading dimension");
    if (!h->factored) return fail(HM_ERR_STATE, "hm_factor_leaf has not completed (it also prepares D)");
    if (nrhs == 0) return HM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    SolveCtx c;
    c.h = h; c.nrhs = nrhs; c.K = 0; c.fp64 = false; c.s = s;
    c.m = clamp_levels(h, n_levels);
    c.vbytes = sizeof(float2) * h->pN * nrhs;
    hm_status st = ensure_workspace(h, nrhs, c.m);
    if (st != HM_OK) return st;
    if (fp64_accumulate && (st = ensure_partials(h)) != HM_OK) return st;
    if ((st = autotune(h, nrhs, c.m, s, fp64_accumulate != 0)) != HM_OK) return st;
    if ((st = use_tuning(c)) != HM_OK) return st;
    if (fp64_accumulate && c.res_rb == RB_OWN && own_applies(h, c.m) && (st = ensure_own(h, c.m)) != HM_OK)
        return st;
    void *xt = h->ws.vec32[0], *yt = h->ws.vec32[1];
    launch_permute_in(x, ldx, xt, h->pN, h->d_pperm, nrhs, false, s);
    if (fp64_accumulate) {
        residual64(c, (const float2 *)xt, nullptr, (float2 *)yt, nullptr);
    } else {
        HM_CUDA(cudaMemsetAsync(yt, 0, c.vbytes, s));
        launch_apply_self_f32(h, (const float2 *)xt, (float2 *)yt, nrhs, s);
        for (int lev = 1; lev <= c.m; ++lev) apply_level(c, lev, xt, yt);
    }
    launch_permute_out(yt, h->pN, y, ldy, h->d_pperm, nrhs, false, s);
    HM_CUDA(cudaGetLastError());
    return HM_OK;
}

hm_status hm_residual(hm_matrix h, const void *b, int64_t ldb, const void *x, int64_t ldx, void *r, int64_t ldr,
                      int nrhs, int n_levels, double *norms, void *stream)
{
    if (!h) return fail(HM_ERR_ARG, "null handle");
    if (nrhs < 0 || ldb < h->N || ldx < h->N || ldr < h->N) return fail(HM_ERR_ARG, "bad nrhs or leading dimension");
    if (nrhs == 0) return HM_OK;
    if (!b || !x || !r) return fail(HM_ERR_ARG, "null b, x or r");
    if (!h->factored) return fail(HM_ERR_STATE, "hm_factor_leaf has not completed (it also prepares D)");
    cudaStream_t s = (cudaStream_t)stream;
    SolveCtx c;
    c.h = h; c.nrhs = nrhs; c.K = 0; c.fp64 = false; c.s = s;
    c.m = clamp_levels(h, n_levels);
    c.vbytes = sizeof(float2) * h->pN * nrhs;
    hm_status st = ensure_workspace(h, nrhs, c.m);
    if (st != HM_OK) return st;
    if ((st = ensure_partials(h)) != HM_OK) return st;
    if ((st = autotune(h, nrhs, c.m, s, true)) != HM_OK) return st;
    if ((st = use_tuning(c)) != HM_OK) return st;
    if (c.res_rb == RB_OWN && own_applies(h, c.m) && (st = ensure_own(h, c.m)) != HM_OK) return st;
    void *bt = h->ws.vec32[0], *xt = h->ws.vec32[1], *rt = h->ws.vec32[3];
    launch_permute_in(b, ldb, bt, h->pN, h->d_pperm, nrhs, false, s);
    launch_permute_in(x, ldx, xt, h->pN, h->d_pperm, nrhs, false, s);
    double *dn = h->ws.d_acc64;
    HM_CUDA(cudaMemsetAsync(dn, 0, 2 * sizeof(double) * nrhs, s));
    residual64(c, (const float2 *)xt, (const float2 *)bt, (float2 *)rt, dn);
    launch_permute_out(rt, h->pN, r, ldr, h->d_pperm, nrhs, false, s);
    HM_CUDA(cudaGetLastError());
    if (norms) {
        HM_CUDA(cudaMemcpyAsync(norms, dn, 2 * sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaStreamSynchronize(s));
    }
    return HM_OK;
}

hm_status hm_rhs_plane_wave(hm_matrix h, const double *khat, const double *phat, int nrhs, void *b, int64_t ldb,
                            void *stream)
{
    if (!h || !khat || !phat || !b) return fail(HM_ERR_ARG, "null argument");
    if (!h->has_mesh) return fail(HM_ERR_STATE, "operator has no mesh (built from blocks)");
    if (nrhs < 0 || ldb < h->N) return fail(HM_ERR_ARG, "bad nrhs or leading dimension");
    if (nrhs == 0) return HM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<double> kp(6 * (size_t)nrhs);
    std::memcpy(kp.data(), khat, 3 * sizeof(double) * nrhs);
    std::memcpy(kp.data() + 3 * nrhs, phat, 3 * sizeof(double) * nrhs);
    double *d_kp = nullptr;
    HM_CUDA(cudaMalloc(&d_kp, kp.size() * sizeof(double)));
    cudaError_t e = cudaMemcpyAsync(d_kp, kp.data(), kp.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        launch_rhs_plane_wave(h, d_kp, d_kp + 3 * nrhs, nrhs, (float2 *)b, ldb, s);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_kp);
    if (e != cudaSuccess) return cuda_fail(e, "hm_rhs_plane_wave");
    return HM_OK;
}

hm_status hm_profile(hm_matrix h, int enable)
{
    if (!h) return fail(HM_ERR_ARG, "null handle");
    h->prof = enable != 0;
    if (enable) {
        h->prof_used = 0;
        h->prof_launches = 0;
        h->prof_bytes = 0;
    }
    return HM_OK;
}

hm_status hm_profile_read(hm_matrix h, double *product_ms, int64_t *launches, int64_t *bytes)
{
    if (!h || !product_ms || !launches || !bytes) return fail(HM_ERR_ARG, "null argument");
    double tot = 0.0;
    for (size_t q = 0; q + 1 < h->prof_used; q += 2) {
        HM_CUDA(cudaEventSynchronize(h->prof_ev[q + 1]));
        float ms = 0.f;
        HM_CUDA(cudaEventElapsedTime(&ms, h->prof_ev[q], h->prof_ev[q + 1]));
        tot += ms;
    }
    *product_ms = tot;
    *launches = h->prof_launches;
    *bytes = h->prof_bytes;
    return HM_OK;
}

hm_status hm_set_tuning(hm_matrix h, int nrhs, int prod_rb, int res_rb)
{
    if (!h) return fail(HM_ERR_ARG, "null handle");
    if (nrhs < MRHS_MIN_RHS) return fail(HM_ERR_ARG, "kernel choices apply from 4 right-hand sides on");
    const bool pok = prod_rb == 0 || prod_rb == 8 || prod_rb == 16 || prod_rb == 32 || prod_rb == RB_TC;
    const bool rok = res_rb == 0 || res_rb == 8 || res_rb == 16 || res_rb == RB_OWN;
    if (!pok || !rok) return fail(HM_ERR_ARG, "prod_rb must be 0, 8, 16, 32 or 1016 and res_rb 0, 8, 16 or 1017");
    hm_matrix_s::Tune t;
    t.prod_rb = prod_rb;
    t.res_rb = res_rb;
    h->tune[tune_bucket(nrhs)] = t;
    clear_graphs(h);   // captured solves hold the previous choice
    return HM_OK;
}

hm_status hm_set_wait_limit(hm_matrix h, int64_t polls)
{
    if (!h) return fail(HM_ERR_ARG, "null handle");
    if (polls > (int64_t)0xFFFFFFFF) return fail(HM_ERR_ARG, "polls above 2^32 - 1");
    h->tc_wait_limit = polls < 0 ? -1 : polls;
    clear_graphs(h);   // captured launches hold the previous limit
    return HM_OK;
}

hm_status hm_get_tuning(hm_matrix h, int nrhs, int *prod_rb, int *res_rb, double *prod_ms, double *res_ms)
{
    if (!h) return fail(HM_ERR_ARG, "null handle");
    auto it = nrhs < MRHS_MIN_RHS ? h->tune.end() : h->tune.find(tune_bucket(nrhs));
    if (it == h->tune.end()) return fail(HM_ERR_STATE, "no tuned kernel choice for this right-hand-side count");
    if (prod_rb) *prod_rb = it->second.prod_rb;
    if (res_rb) *res_rb = it->second.res_rb;
    if (prod_ms) *prod_ms = it->second.prod_ms;
    if (res_ms) *res_ms = it->second.res_ms;
    return HM_OK;
}

hm_status hm_get_info(hm_matrix h, hm_info *info)
{
    if (!h || !info) return fail(HM_ERR_ARG, "null argument");
    memset(info, 0, sizeof(*info));
    info->n = h->N;
    info->n_leaves = h->n_leaves;
    info->depth = h->depth;
    info->n_levels = h->n_levels;
    for (auto &kv : h->levels) {
        const int lev = kv.first;
        const LevelList &L = kv.second;
        if (lev == 1) {
            info->n_near = L.n_dense;
            for (size_t i = 0; i < L.items.size(); ++i)
                if (L.items[i].k == 0) info->near_elems += (int64_t)L.true_m[i] * L.true_n[i];
        }
        if (lev >= 1 && lev <= 16) {
            info->n_far[lev - 1] = L.n_lowrank;
            for (size_t i = 0; i < L.items.size(); ++i)
                if (L.items[i].k > 0) info->far_elems[lev - 1] += (int64_t)L.items[i].k * (L.true_m[i] + L.true_n[i]);
        }
    }
    for (int64_t i = 0; i < h->n_leaves; ++i) {
        const int64_t n = h->leaf_off[i + 1] - h->leaf_off[i];
        info->self_elems += n * n;
    }
    info->max_rank = h->max_rank;
    info->factored = h->factored;
    info->has_fp64 = h->has_fp64 ? 1 : 0;
    info->device_bytes = h->device_bytes + h->ws.dev_bytes + (int64_t)h->ws.d_io_bytes;
    for (int l = 0; l < 16; ++l) {
        info->norm_est[l] = h->norm_est[l];
        info->rho_est[l] = h->rho_est[l];
    }
    info->norm_iters = h->norm_iters;
    return HM_OK;
}

hm_status hm_get_perm(hm_matrix h, int64_t *perm)
{
    if (!h || !perm) return fail(HM_ERR_ARG, "null argument");
    std::copy(h->perm.begin(), h->perm.end(), perm);
    return HM_OK;
}

hm_status hm_get_leaves(hm_matrix h, int64_t *leaf_off)
{
    if (!h || !leaf_off) return fail(HM_ERR_ARG, "null argument");
    std::copy(h->leaf_off.begin(), h->leaf_off.end(), leaf_off);
    return HM_OK;
}

static int64_t tree_of_padded(hm_matrix h, int64_t pp)
{
    // padded position -> tree position (pp must not be a pad slot)
    auto it = std::upper_bound(h->pleaf_off.begin(), h->pleaf_off.end(), pp);
    const int64_t l = (it - h->pleaf_off.begin()) - 1;
    return h->leaf_off[l] + (pp - h->pleaf_off[l]);
}

hm_status hm_get_blocks(hm_matrix h, int level, int64_t *count, int64_t *row0, int64_t *col0, int32_t *m,
                        int32_t *n, int32_t *rank)
{
    if (!h || !count) return fail(HM_ERR_ARG, "null argument");
    auto f = h->levels.find(level);
    if (f == h->levels.end()) { *count = 0; return HM_OK; }
    const LevelList &L = f->second;
    *count = (int64_t)L.items.size();
    for (size_t i = 0; i < L.items.size(); ++i) {
        const Item &it = L.items[i];
        if (row0) row0[i] = tree_of_padded(h, it.row0);
        if (col0) col0[i] = tree_of_padded(h, it.col0);
        if (m) m[i] = L.true_m[i];
        if (n) n[i] = L.true_n[i];
        if (rank) rank[i] = it.k;
    }
    return HM_OK;
}

hm_status hm_get_block(hm_matrix h, int level, int64_t index, double *a, double *b)
{
    if (!h || !a) return fail(HM_ERR_ARG, "null argument");
    auto f = h->levels.find(level);
    if (f == h->levels.end() || index < 0 || index >= (int64_t)f->second.items.size())
        return fail(HM_ERR_ARG, "no such block");
    const LevelList &L = f->second;
    const Item it = L.items[index];
    const int64_t elems = item_elems(it);
    std::vector<double2> buf(elems);
    if (h->has_fp64) {
        HM_CUDA(cudaMemcpy(buf.data(), h->d_pool64 + it.off, elems * sizeof(double2), cudaMemcpyDeviceToHost));
    } else {
        std::vector<float2> t(elems);
        HM_CUDA(cudaMemcpy(t.data(), h->d_pool32 + it.off, elems * sizeof(float2), cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < elems; ++i) buf[i] = make_double2(t[i].x, t[i].y);
    }
    double2 *A = reinterpret_cast<double2 *>(a);
    const int64_t tm = L.true_m[index], tn = L.true_n[index];
    if (it.k == 0) {
        const int64_t ld = even(it.n);
        for (int64_t i = 0; i < tm; ++i)
            for (int64_t j = 0; j < tn; ++j) A[i * tn + j] = buf[i * ld + j];
        return HM_OK;
    }
    if (!b) return fail(HM_ERR_ARG, "low-rank block needs both a (U) and b (V)");
    double2 *Bv = reinterpret_cast<double2 *>(b);
    const int64_t k = it.k;
    int64_t ti = 0;
    for (int64_t pi = 0; pi < it.m; ++pi) {
        if (h->h_pperm[it.row0 + pi] < 0) continue;
        for (int64_t l = 0; l < k; ++l) A[ti * k + l] = buf[l * it.m + pi];
        ++ti;
    }
    int64_t tj = 0;
    for (int64_t pj = 0; pj < it.n; ++pj) {
        if (h->h_pperm[it.col0 + pj] < 0) continue;
        for (int64_t l = 0; l < k; ++l) Bv[l * tn + tj] = buf[k * it.m + l * it.n + pj];
        ++tj;
    }
    return HM_OK;
}

hm_status hm_sync_status(hm_matrix h, void *stream)
{
    if (!h) return fail(HM_ERR_ARG, "null handle");
    HM_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    int stv = 0;
    HM_CUDA(cudaMemcpy(&stv, h->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (stv != 0) {
        HM_CUDA(cudaMemset(h->d_status, 0, sizeof(int)));
        return fail((hm_status)stv, "device-side error recorded");
    }
    return HM_OK;
}

int64_t hm_size(hm_matrix h) { return h ? h->N : 0; }

void hm_destroy(hm_matrix h)
{
    if (!h) return;
    cudaDeviceSynchronize();
    free_handle(h);
}

const char *hm_last_error(void) { return g_last_error.c_str(); }

const char *hm_version(void) { return "hmps 0.1 (sm_103a)"; }

} // extern "C"
