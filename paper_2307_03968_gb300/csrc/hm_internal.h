// Internal declarations of the hmps library (not part of the C ABI).
//
// Data layout in HBM (one hm_matrix):
//  - "padded tree order": unknowns are permuted into tree order (leaves
//    contiguous, depth-first) and every leaf is padded to an even length, so
//    every leaf and every coarser cluster starts on a 16-byte boundary for
//    complex64 vectors.  pad slots hold zeros.  pN = padded length.
//  - vectors: column-major [nrhs][pN] complex.
//  - stored blocks (half storage, row cluster before column cluster) are
//    packed into one pool per precision, each block starting on an even
//    complex index:
//      dense  m x n   row-major, row stride ld = even(n)
//      low-rank       U^T (k x m', stride even(m')) then V (k x n', stride even(n')),
//                     m', n' = padded cluster lengths; the block is U V.
//  - leaf inverses D_i^{-1}: column-major n_i x n_i, column stride even(n_i).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>
#include <map>
#include <tuple>

#include "../../include/hmps.h"
#include "hm_lists.h"

namespace hm {

constexpr int MRHS_MIN_RHS = 4;     // from this many right-hand sides on, the multi-RHS kernels take the small blocks
constexpr int RESID_CHUNK = 16;     // right-hand sides per chunk of the FP64-class residual (partial slots held)
constexpr int RB_TC = 1016;         // product choice: tensor-core products of the small items, RHS tiles of 128
constexpr int TC_MIN_RHS = 32;      // the autotuner times the tensor-core product from this many RHS on
constexpr int RB_OWN = 1017;        // residual choice: owner-computes FP64-class products (levels of small items)

// Double-float numbers of the FP64-class residual (hi + lo, |lo| a few ulps of hi at
// most): a real one, and a complex one of 16 bytes, which is also the element of
// the residual's partial slots.
namespace dot2 {
struct df { float hi, lo; };
struct alignas(16) cdf { df re, im; };
} // namespace dot2


struct LevelList {
    int64_t alg_elems = 0;        // complex elements at unpadded sizes (algorithmic bytes / 8)
    std::vector<Item> items;      // host copy
    std::vector<int32_t> true_m, true_n;  // unpadded sizes (for export)
    Item *d_items = nullptr;      // device copy
    // the same items split for the multi-right-hand-side product: blocks of at
    // most MRHS_MAX_DIM x MRHS_MAX_DIM (and rank <= MRHS_MAX_RANK) staged whole
    // in shared memory, and the rest
    Item *d_small = nullptr, *d_big = nullptr;
    int64_t n_small = 0, n_big = 0;
    // the FP64-class residual's copy of the item list, in the order that balances its
    // round-robin warps, and per item of it / of d_big the block bounds of the
    // common-grid residual products (k_item_bounds: largest row and column 1-norms)
    Item *d_res = nullptr;
    float4 *d_bnd = nullptr, *d_bnd_big = nullptr;
    int small_dim = 0, small_rank = 0;   // largest (even) side and rank among the small items
    // the small items as directed products grouped into work units by output
    // cluster, for the tensor-core product (both mirrored halves of every block)
    TcOp *d_tco = nullptr;
    TcUnit *d_tcu = nullptr;          // units over d_tco
    int64_t n_tco = 0, n_tcu = 0;
    TcBatch *d_tcb = nullptr;         // stage-1 batches over the row table
    int64_t *d_tcr = nullptr;         // row table: W row offsets (-1 = zero row)
    int32_t *d_tcc = nullptr;         // chunk table: T chunk of each 8-row group
    int64_t n_tcb = 0, n_tcr = 0, n_tchunk = 0;   // batches, rows, T chunks per RHS tile
    // the same directed products with one unit per output cluster (the owner-computes
    // FP64-class residual: each output row summed by one CTA in a fixed order)
    TcProd *d_rcp = nullptr;
    TcUnit *d_rcu = nullptr;
    int64_t n_rcu = 0;
    float2 *d_rcb = nullptr;      // per product of d_rcp: its common-grid bounds (k_prod_bounds)
    // the input clusters' K chunks of 8 unknowns (padded-tree offset, valid length):
    // the tensor-core product splits x once per launch into these chunks
    XChunk *d_xch = nullptr;
    int64_t n_xch = 0;
    int64_t n_dense = 0, n_lowrank = 0;
    int64_t elems = 0;            // stored complex elements
    // the FP32 product's own copies of the item list and of its big part, with every dense
    // block of more than PROD_PANEL rows cut into row panels (the product kernel gives each
    // item to one warp: a leaf of ~1,000 unknowns would otherwise leave the GPU idle), in the
    // order that balances the kernel's round-robin warps (largest first, snake rounds)
    Item *d_prod = nullptr, *d_prod_big = nullptr;
    int64_t n_prod = 0, n_prod_big = 0;
};
constexpr int PROD_PANEL = 64;

// One phase of the one-launch solve (k_persist.cu): every kernel the solve would
// launch becomes a phase of one cooperative kernel, with a grid-wide barrier
// between consecutive phases.
enum PhaseOp : int32_t {
    PH_PERMUTE_IN = 1,   // c[r][p] = a[r * ld2 + pperm[p]] (0 at pads)
    PH_PERMUTE_OUT,      // c[r * ld2 + pperm[p]] = a[r][p]
    PH_LEAF,             // per leaf: c = (a ? a - Dinv b : Dinv b); b = 0 if m
    PH_APPLY,            // c += M a over items[0, n) (one RHS at a time per block)
    PH_RESID,            // FP64-class products of items[0, n) (block bounds d) into the partial slots c (stride ld)
    PH_GATHER,           // c = (b ? b - acc : acc), acc = D a + slots d of m levels; norms
    PH_ZERO,             // n bytes at c
    PH_COPY,             // n bytes a -> c
    PH_SUB,              // c = a - b, n complex
    PH_ADD,              // c += a, n complex
    PH_CHECK             // non-finite in a[0, n) -> HM_ERR_DIVERGED
};
struct Phase {
    int32_t op, nrhs;
    int64_t n;
    const void *a, *b;
    void *c;
    const void *d;
    const Item *items;
    int64_t ld, ld2;
    int32_t m;
    int32_t pad;         // 1 = no grid barrier after this phase (set by the recorder)
    double *norms;
};

// What the one-launch solve's phases read besides their own pointers: the
// operator's layout (one hm_matrix), its status word and the barrier words.
struct PersistCtx {
    const int32_t *pperm;
    int64_t pN;
    int64_t n_leaves;
    const int32_t *pleaf_off;
    const int64_t *dinv_off;
    const float2 *dinv;
    const float2 *self32;
    const float2 *pool;
    const int64_t *csr_off;
    int csr_stride;
    const int64_t *csr_idx;
    int *status;
    unsigned *bar;                      // the grid barrier's word (and a spare one)
    uint32_t polls;                     // barrier wait bound
};

// The device-resident request loop (k_serve_loop in k_persist.cu, driven by
// hm_server.cu): ring entries and the loop's control words live in pinned host
// memory mapped into the device's address space; LoopDev in device memory.
enum LoopState : int32_t { LOOP_FREE = 0, LOOP_READY = 1, LOOP_DONE = 2, LOOP_STOP = 3 };
struct LoopEntry {
    int32_t state;            // LoopState: ready / stop set by the host, done by the device
    int32_t n_phases;
    const Phase *phases;      // the request's one-launch phase list (device memory)
    const void *b;            // the batch's right-hand sides and solutions (device buffers of its slot):
    void *x;                  //   they replace the pointers the list was recorded with
    PersistCtx ctx;           // its operator's context (bar and polls are the loop's own)
};
struct LoopCtl {
    int64_t start;            // ring index the next launch starts at (host)
    int64_t head;             // ring index the loop had reached when it left (device)
    int32_t exited;           // 1 once the loop kernel has left (device)
    int32_t pad;
};
struct LoopDev {
    int32_t decision;         // 1 = serve the current entry, 0 = leave
    int32_t cur_n;
    const Phase *cur_phases;
    const void *cur_b;
    void *cur_x;
    PersistCtx cur_ctx;
};

struct Workspace {
    int nrhs = 0;
    // complex vectors [nrhs][pN], allocated for the current nrhs, per precision
    std::vector<void *> vec32, vec64;
    double *d_acc64 = nullptr;    // norms of the residual (2 doubles per right-hand side)
    dot2::cdf *d_part = nullptr;  // double-float partial slots for PART_RHS right-hand sides
    int part_rhs = 0;
    void *h_pinned = nullptr;     // pinned staging for host-buffer solves
    size_t h_pinned_bytes = 0;
    void *d_io = nullptr;         // device b / x for host-buffer solves
    size_t d_io_bytes = 0;
    int64_t dev_bytes = 0;        // device bytes held by the vectors, norms and partial slots
    float *d_xpl = nullptr;       // split x chunks of the tensor-core product (16 KB per chunk and RHS tile)
    size_t xpl_bytes = 0;
    float *d_tct = nullptr;       // stage-1 results T of the tensor-core product (TC_T_CHUNK floats per chunk and tile)
    size_t tct_bytes = 0;
    double2 *d_own = nullptr;     // FP64 owner sums of the residual, [level][RHS][pN]
    size_t own_bytes = 0;
};

} // namespace hm

struct hm_matrix_s {
    int64_t N = 0, pN = 0, n_leaves = 0;
    int depth = 0, n_levels = 0, max_rank = 0;
    std::vector<int64_t> perm;        // tree position -> original index
    std::vector<int64_t> leaf_off;    // tree positions
    std::vector<int64_t> pleaf_off;   // padded positions
    std::vector<int32_t> h_pperm;     // padded position -> original index or -1
    int32_t *d_pperm = nullptr;
    int32_t *d_pleaf_off = nullptr;   // [n_leaves+1]
    int64_t *d_dinv_off = nullptr;    // [n_leaves] complex offset of D_i^{-1} (and of the complex64 D_i)
    int64_t *d_leaf_n = nullptr;      // [n_leaves] true leaf sizes
    int64_t *d_self_off = nullptr;    // [n_leaves] complex offset of D_i in d_self64
    int *d_bad_leaf = nullptr;        // leaf index of the first zero pivot
    std::vector<int64_t> dinv_off;
    int64_t dinv_elems = 0;

    // leaf self blocks, complex128 row-major n_i x n_i (input of the factorisation)
    double2 *d_self64 = nullptr;
    float2 *d_self32 = nullptr;       // complex64 copy, column-major like D^{-1} (residual)
    std::vector<int64_t> self_off;    // complex offsets into d_self64 / d_self32
    int64_t self_elems = 0;
    float2 *d_dinv32 = nullptr;
    double2 *d_dinv64 = nullptr;
    int factored = 0;

    // block pools and per-level lists; level index 1 = leaf level
    float2 *d_pool32 = nullptr;
    double2 *d_pool64 = nullptr;
    int64_t pool_elems = 0;
    bool has_fp64 = false;
    std::map<int, hm::LevelList> levels;

    // partial slots of the deterministic FP64-class products: per leaf and level, the
    // list of slot positions holding contributions to that leaf's rows
    int64_t partial_elems = 0;
    int64_t *d_csr_off = nullptr;     // [n_leaves * (n_levels + 1)]
    int64_t *d_csr_idx = nullptr;

    int *d_status = nullptr;          // device status word (hm_status code, first error wins)
    int *h_status = nullptr;          // pinned mirror
    hm::Workspace ws;
    int64_t device_bytes = 0;
    int num_sms = 0;
    int64_t tc_max_xch = 0;           // largest split-x chunk count over the levels
    int64_t tc_max_tchunk = 0;        // largest T chunk count over the levels
    int64_t tc_wait_limit = -1;       // polls of each pipeline wait of the tensor-core product (-1 = default)

    // mesh geometry kept for excitation (operators made by hm_build):
    // b_m = sum over the two sides s of ucoef[m][s] * sum_q w_q (r_q - v) . p exp(-jk k . r_q)
    // on the side's cell (triangle or tetrahedron), v = the side's free vertex
    bool has_mesh = false;
    int basis = HM_RWG;
    int rhs_nq = 0;               // quadrature points per cell
    double *d_qpd = nullptr;      // n_cell x rhs_nq x 3 quadrature points
    double *d_rhs_w = nullptr;    // rhs_nq weights
    double *d_vtx = nullptr;      // nv x 3
    int32_t *d_ucell = nullptr, *d_ufree = nullptr;   // N x 2 (cell -1: no side)
    double *d_ucoef = nullptr;    // N x 2
    double wavenumber = 0.0;

    // CUDA graphs of whole solves, keyed by pointers, sizes and options
    struct GraphKey {
        const void *b; void *x; int64_t ldb, ldx; int nrhs, K, m, nested, refine, fp64, persist;
        bool operator<(const GraphKey &o) const
        {
            return std::tie(b, x, ldb, ldx, nrhs, K, m, nested, refine, fp64, persist) <
                   std::tie(o.b, o.x, o.ldb, o.ldx, o.nrhs, o.K, o.m, o.nested, o.refine, o.fp64, o.persist);
        }
    };
    std::map<GraphKey, cudaGraphExec_t> graphs;
    cudaStream_t cap_stream = nullptr;
    // phase lists of one-launch solves (device copies), keyed like the graphs; the
    // barrier words of the one-launch solve (count, generation)
    struct PersistList { hm::Phase *d = nullptr; int n = 0, units = 0; int64_t launches = 0, bytes = 0; };
    std::map<GraphKey, PersistList> persist;
    unsigned *d_bar = nullptr;

    // kernel choices measured on this operator per right-hand-side count (hm_api.cu autotune)
    struct Tune { int prod_rb = -1, res_rb = -1; double prod_ms = 0.0, res_ms = 0.0; };   // res_rb < 0: not tuned
    std::map<int, Tune> tune;

    // estimates of the level operators U_l = D^{-1} M_l (index l - 1), made by hm_factor_leaf /
    // hm_estimate_norms: ||U_l||_2 from power iterations on U^H U, the spectral radius from
    // the growth of power iterations on U; norm_iters = 0 when not estimated
    double norm_est[16] = {}, rho_est[16] = {};
    int norm_iters = 0;

    // opt-in event timing of the product kernel
    bool prof = false;
    std::vector<cudaEvent_t> prof_ev;     // pairs (start, end)
    size_t prof_used = 0;
    int64_t prof_launches = 0, prof_bytes = 0;
};

namespace hm {

// error helpers (hm_api.cu)
hm_status fail(hm_status s, const std::string &msg);
hm_status cuda_fail(cudaError_t e, const char *what);
#define HM_CUDA(call)                                                         \
    do {                                                                      \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) return ::hm::cuda_fail(e_, #call);             \
    } while (0)

hm_status dev_alloc(hm_matrix h, void **p, size_t bytes);

// kernels launchers (k_solve.cu)
void launch_permute_in(const void *b, int64_t ldb, void *xt, int64_t pN, const int32_t *pperm,
                       int nrhs, bool fp64, cudaStream_t s);
void launch_permute_out(const void *xt, int64_t pN, void *x, int64_t ldx, const int32_t *pperm,
                        int nrhs, bool fp64, cudaStream_t s);
void launch_zero(void *p, size_t bytes, cudaStream_t s);
// z (+)= M_level x  for one item list; z must be pre-zeroed by the caller
// rb: -1 = default choice by nrhs, 0 = one right-hand side at a time for every block,
// 8 / 16 / 32 = shared-memory multi-RHS kernel with that chunk for the blocks it takes.
// Returns the number of kernels it enqueued.
int launch_apply_items(hm_matrix h, const LevelList &L, const void *x, void *z, int nrhs, bool fp64,
                        cudaStream_t s, int rb = -1);
// FP64-class (Dot2) products of every block of a level into its partial slots (no atomics)
// warps of the FP32 product kernel's persistent grid (k_product.cu) and of the
// FP64-class residual kernel's (k_residual.cu)
int64_t product_warps(hm_matrix h);
int64_t residual_warps(hm_matrix h);
// the residual products' block bounds of items[0 .. n) (k_residual.cu)
void launch_item_bounds(const Item *items, int64_t n, const float2 *pool, float4 *bnd, cudaStream_t s);
int launch_apply_items_partials(hm_matrix h, const LevelList &L, const float2 *x, dot2::cdf *part, int64_t pstride,
                                int nrhs, cudaStream_t s, int rb = -1);   // returns the kernels enqueued
// per leaf: acc = D x + sum of the leaf's partial slots of levels 1..m (double-float, fixed order);
// out = b - acc (+ norms) when b is given, else out = acc (rounded to complex64)
void launch_gather_acc64(hm_matrix h, const float2 *x, int m, const dot2::cdf *part, int64_t pstride,
                         const float2 *b, float2 *out, double *norms, int nrhs, cudaStream_t s);
void launch_apply_self_f32(hm_matrix h, const float2 *x, float2 *acc, int nrhs, cudaStream_t s);
// per leaf: out = (y ? y - Dinv zin : Dinv zin); if zero_in, zin is cleared afterwards
// the last series step out = y - D^{-1} z (z cleared) and the end of the solve (v = base + out
// or out, finiteness into the status word, x = P^T v) in one pass per leaf (complex64; k_solve.cu)
void launch_leaf_finish(hm_matrix h, const float2 *y, float2 *z, float2 *out, const float2 *base, float2 *x,
                        int64_t ldx, int nrhs, cudaStream_t s);
// bt = P b and y = D^{-1} bt in one pass per leaf (complex64; k_solve.cu)
void launch_permute_leaf(hm_matrix h, const float2 *b, int64_t ldb, float2 *bt, float2 *y, int nrhs, cudaStream_t s);
// the residual gather (out = b - acc, norms) and y = D^{-1} out in one pass per leaf (k_residual.cu)
void launch_gather_leaf_update(hm_matrix h, const float2 *x, int m, const dot2::cdf *part, int64_t pstride,
                               const float2 *b, float2 *out, double *norms, float2 *y, int nrhs, cudaStream_t s);
void launch_leaf_update(hm_matrix h, const void *y, void *zin, void *out, int nrhs, bool zero_in, bool fp64,
                        cudaStream_t s);
// out = y - w
void launch_sub(const void *y, const void *w, void *out, int64_t n, bool fp64, cudaStream_t s);
void launch_add_inplace(void *x, const void *dx, int64_t n, bool fp64, cudaStream_t s);
void launch_check_finite(const void *x, int64_t n, bool fp64, int *status, cudaStream_t s);
// complex64: v = xt (+ dx if given), non-finite -> HM_ERR_DIVERGED, x[r * ldx + pperm[p]] = v
void launch_finish(const float2 *xt, const float2 *dx, int64_t pN, float2 *x, int64_t ldx, const int32_t *pperm,
                   int nrhs, int *status, cudaStream_t s);
void launch_convert_f64_to_f32(const double2 *a, float2 *b, int64_t n, cudaStream_t s);
void launch_convert_f32_to_f64(const float2 *a, double2 *b, int64_t n, cudaStream_t s);

// factorisation (k_factor.cu)
int factor_max_leaf();
hm_status launch_factor(hm_matrix h, cudaStream_t s);

// unknown count of a mesh (RWG edges or SWG faces) with the checks of hm_build (k_build.cu)
hm_status count_unknowns(const hm_mesh *mesh, int64_t *n);

// plane-wave right-hand sides (k_build.cu)
void launch_rhs_plane_wave(hm_matrix h, const double *d_k, const double *d_p, int nrhs, float2 *b, int64_t ldb,
                           cudaStream_t s);

// GPU build from a mesh (k_build.cu dispatches; the SWG volume build is in k_build_swg.cu)
hm_status build_from_mesh(const hm_mesh *mesh, const hm_build_opts *opts, cudaStream_t s, hm_matrix *out);
hm_status build_from_tets(const hm_mesh *mesh, const hm_build_opts *opts, cudaStream_t s, hm_matrix *out);
// SWG faces of a tetrahedral mesh (sorted vertex triples; T+ = lower tetrahedron,
// T- = -1 on the boundary); HM_ERR_ARG for a face of more than two tetrahedra
hm_status swg_faces(int64_t nv, int64_t nt, const int32_t *tet, std::vector<int32_t> &fv, std::vector<int32_t> &ftet,
                    std::vector<int32_t> &ffree);

// shared construction helpers (hm_api.cu)
hm_status finalize_layout(hm_matrix h, cudaStream_t s);
// assigns the partial slots (Item::pad) and uploads the per-leaf slot lists;
// call after every level list is complete and before the items are uploaded
hm_status prepare_partials(hm_matrix h, cudaStream_t s);
// uploads every level's item list and its multi-RHS split (small / big)
hm_status upload_item_lists(hm_matrix h, cudaStream_t s);
// multi-right-hand-side product of the small items of a level (k_mrhs.cu):
// z (+)= M_level x for right-hand sides [0, nrhs), blocks read once per chunk of rb
void launch_apply_items_mrhs(hm_matrix h, const LevelList &L, const float2 *x, float2 *z, int nrhs, int rb,
                             cudaStream_t s);
// the same for an explicit list of small items (k_mrhs.cu)
void launch_apply_list_mrhs(hm_matrix h, const LevelList &L, const Item *items, int64_t n_items, const float2 *x,
                            float2 *z, int nrhs, int rb, cudaStream_t s);
// owner-computes FP64-class products of a level's small items into own ([RHS][pN]) and the gather
// out = b - (D x + sum of the m levels' owner sums) (k_resid_own.cu)
void launch_resid_own(hm_matrix h, const LevelList &L, const float2 *x, double2 *own, int nrhs, cudaStream_t s);
// the owner-computes products' common-grid bounds of prods[0 .. n) (k_resid_own.cu)
void launch_prod_bounds(const TcProd *prods, int64_t n, const float2 *pool, float2 *out, cudaStream_t s);
void launch_gather_own(hm_matrix h, const float2 *x, int m, const double2 *own, int64_t lstride, const float2 *b,
                       float2 *out, double *norms, int nrhs, cudaStream_t s);
// level-operator norm estimate (k_norm.cu): start vector (zero pads), |v|^2 into one device double
// (cleared first), dst = op(src) / sqrt(*nrm2) with op = conjugation or identity
void launch_seed_vector(float2 *v, const int32_t *pperm, int64_t pN, uint32_t seed, cudaStream_t s);
void launch_norm2(const float2 *v, int64_t n, double *out, cudaStream_t s);
void launch_conj_scale(const float2 *src, float2 *dst, int64_t n, const double *nrm2, bool conj, cudaStream_t s);
// one-launch solve (k_persist.cu): whether the operator's leaves fit it, and one
// cooperative launch running the phases (device array) with grid barriers between them;
// units = the widest phase's work units (caps the grid)
bool persist_supported(hm_matrix h);
void persist_ctx(hm_matrix h, PersistCtx *c);
// the recorded phase list of a one-launch solve of b -> x (device pointers, ld = N), made on
// first use (which may grow the handle's workspace and launches nothing) (hm_api.cu)
hm_status persist_phases(hm_matrix h, const void *b, void *x, int nrhs, const hm_solve_opts *o,
                         const Phase **phases, int *n_phases);
// the request loop: grid size (cooperative, all CTAs resident) and one launch
int serve_loop_grid(int num_sms);
hm_status launch_serve_loop(LoopEntry *ring, int ring_size, LoopCtl *ctl, LoopDev *dv, unsigned *bar, int *loop_status,
                            int grid, uint32_t idle_polls, cudaStream_t s);
hm_status launch_persist(hm_matrix h, const Phase *d_phases, int n_phases, int units, cudaStream_t s);
// bytes of the split-x workspace of the tensor-core product for n_xch chunks and nrhs (k_mrhs_tc.cu)
size_t tc_xplane_bytes(int64_t n_xch, int nrhs);
// bytes of its stage-1 workspace for n_tchunk T chunks and nrhs (k_mrhs_tc.cu)
size_t tc_t_bytes(int64_t n_tchunk, int nrhs);
// tensor-core products of a level's small items for all right-hand sides (k_mrhs_tc.cu);
// z accumulates (vector atomics); needs the split-x and stage-1 workspaces for nrhs
int launch_apply_tc(hm_matrix h, const LevelList &L, const float2 *x, float2 *z, int nrhs, cudaStream_t s);
// the FP64-class partial-slot products of the small items for many right-hand sides (k_mrhs.cu)
void launch_apply_items_partials_mrhs(hm_matrix h, const LevelList &L, const float2 *x, dot2::cdf *part,
                                      int64_t pstride, int nrhs, cudaStream_t s, int rb = -1);

} // namespace hm
