/*
 * hmps.h — C ABI of the GB300 (sm_103a) multi-level power-series solver for
 * surface EFIE H-Matrices (arxiv 2307.03968, "Multi-Level Power Series
 * Solution for Large Surface and Volume Electric Field Integral Equation").
 *
 * Problem (paper §II eq. 5, §III eq. 6): Z x = b with Z = Z_N + Z_F, the
 * Galerkin RWG discretisation of the S-EFIE (eq. 3) of a closed PEC surface,
 * Z_N dense near-field leaf blocks and Z_F low-rank far-field blocks U V
 * grouped by tree level (eq. 8).  The solve (§IV eqs. 12-22) applies the leaf
 * self-block inverses D^{-1} and a fixed number K of power-series terms of
 * the H-Matrix product, level by level from the leaf level.
 *
 * Conventions used by every call
 *  - Unknowns are RWG functions numbered in the ORIGINAL order: interior edges
 *    of the triangle mesh sorted by (smaller vertex id, larger vertex id); T+ is
 *    the triangle with the lower index.  The tree permutation is internal.
 *  - Vectors are column-major N x nrhs arrays of interleaved complex numbers:
 *    complex64 (float re, float im) unless a call says otherwise; leading
 *    dimension ld >= N counted in complex elements.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Device work is
 *    stream ordered; calls return after enqueueing unless they say they
 *    synchronise.
 *  - Ownership: an hm_matrix owns all device memory of one operator and its
 *    workspaces; caller buffers are never retained after a call returns.
 *  - Errors: every call returns an hm_status.  Argument and state errors are
 *    detected on the host and returned before any work is enqueued.  Errors
 *    found on the device (singular leaf block, non-finite values, wait
 *    time-outs) are recorded in the handle's device status word and returned
 *    by hm_sync_status() (which synchronises the stream) and by the next call
 *    that synchronises.  hm_last_error() gives a message for the last failing
 *    call of the calling thread.
 *  - One handle must not be used concurrently from several host threads.
 */
#ifndef HMPS_H
#define HMPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hm_matrix_s *hm_matrix;

typedef enum {
    HM_OK = 0,
    HM_ERR_ARG = 1,       /* invalid argument (null pointer, size, option) */
    HM_ERR_OOM = 2,       /* device or pinned host allocation failed */
    HM_ERR_CUDA = 3,      /* a CUDA runtime call failed */
    HM_ERR_STATE = 4,     /* call out of order (e.g. solve before hm_factor_leaf) */
    HM_ERR_SINGULAR = 5,  /* a leaf self block has a zero pivot (hm_factor_leaf) */
    HM_ERR_DIVERGED = 6,  /* non-finite values in a solve result */
    HM_ERR_TIMEOUT = 7    /* a bounded device wait gave up */
} hm_status;

/* ---------------------------------------------------------------- build --- */

/* Basis and integral equation of a mesh (paper §II). */
typedef enum {
    HM_RWG = 0,   /* closed PEC surface, triangles, RWG basis, S-EFIE (eq. 3) */
    HM_SWG = 1    /* inhomogeneous dielectric volume, tetrahedra, SWG basis, V-EFIE (eq. 4) */
} hm_basis;

/*
 * Mesh of the scatterer, in metres.
 *   HM_RWG: cells are triangles (3 vertex ids each, counter-clockwise seen from
 *           outside); one unknown per edge shared by exactly two triangles,
 *           ordered by (lower vertex id, higher vertex id).
 *   HM_SWG: cells are tetrahedra (4 vertex ids each, either orientation) with a
 *           real relative permittivity eps_r > 0 per tetrahedron; one unknown
 *           per face (interior and boundary), ordered by the ascending vertex
 *           triple.  The unknowns x give the electric flux density
 *           D = eps0 sum_n x_n f_n, and the equation is tested with
 *           kappa f_m, kappa = 1 - 1/eps_r, so that the matrix is complex
 *           symmetric (the half storage of §III).
 * All pointers are host memory, read during the call only.
 */
typedef struct {
    int basis;              /* hm_basis */
    int64_t n_vert;
    const double *xyz;      /* 3*n_vert */
    int64_t n_cell;
    const int32_t *cells;   /* 3*n_cell (HM_RWG) or 4*n_cell (HM_SWG) vertex ids */
    const double *eps_r;    /* HM_SWG: n_cell relative permittivities; HM_RWG: ignored (NULL) */
    double wavelength;      /* free-space wavelength; k = 2 pi / wavelength, eta = 376.73 ohm */
} hm_mesh;

/* Tree, admissibility (eq. 7) and compression (§III) options. */
typedef struct {
    int leaf_size;     /* split clusters until every leaf holds <= leaf_size unknowns;
                          1..1536 (HM_ERR_ARG otherwise) */
    int arity;         /* 2 = binary tree (the paper's runs), 4, or 8 = octree */
    double adm;        /* c in dist(t,s) >= c * min(diam t, diam s); the paper's
                          eta = 1 is c = 1, the 2-diameter rule is c = 2 */
    double aca_tol;    /* relative Frobenius tolerance of ACA and of re-compression */
    int levels;        /* far-field levels to compute: 1 = leaf level only (the
                          paper's runs skip the coarser levels), -1 = all */
    int keep_fp64;     /* also keep a complex128 copy of every block (for the
                          plain FP64 solve path) */
} hm_build_opts;

/*
 * Build the H-Matrix of `mesh` on the GPU: RWG or SWG basis, cluster tree,
 * eq. 7 partition, near-field fill and ACA + re-compression of the far blocks,
 * all on the device (§III).  Synchronises `stream` before returning.
 * HM_ERR_ARG for an empty or malformed mesh (vertex id out of range, a
 * degenerate cell, eps_r missing or not > 0 for HM_SWG, a face shared by more
 * than two tetrahedra).
 */
hm_status hm_build(const hm_mesh *mesh, const hm_build_opts *opts, void *stream, hm_matrix *out);

/*
 * Import an H-Matrix given as explicit blocks (complex128, host memory), e.g.
 * one assembled by another program, so that solves of the same operator can be
 * compared.  Layout (all host pointers, read during the call only):
 *   perm[N]                    tree position p -> original unknown perm[p]
 *   leaf_off[n_leaves+1]       leaf i covers tree positions [leaf_off[i], leaf_off[i+1])
 *   self[]                     leaf self blocks D_i, row-major n_i x n_i, concatenated
 *   near: n_near pairs         rows [near_row0[b], +near_m[b]), cols [near_col0[b], +near_n[b]),
 *                              values near_vals (row-major m x n, concatenated);
 *                              the row block must lie before the column block (half storage:
 *                              the mirrored block is the transpose)
 *   far:  n_far blocks         level far_level[b] (1 = leaf level, counted upward), rows/cols as
 *                              for near, rank far_rank[b]; far_u = U (m x k, row-major),
 *                              far_v = V (k x n, row-major), concatenated; block ~ U V
 * Blocks of any level are accepted; hm_build_opts is not used.
 */
typedef struct {
    int64_t n;
    const int64_t *perm;
    int64_t n_leaves;
    const int64_t *leaf_off;
    const double *self;             /* complex128 interleaved */
    int64_t n_near;
    const int64_t *near_row0, *near_col0;
    const int32_t *near_m, *near_n;
    const double *near_vals;        /* complex128 interleaved */
    int64_t n_far;
    const int32_t *far_level;
    const int64_t *far_row0, *far_col0;
    const int32_t *far_m, *far_n, *far_rank;
    const double *far_u, *far_v;    /* complex128 interleaved */
    int keep_fp64;
} hm_blocks;

hm_status hm_build_from_blocks(const hm_blocks *blocks, void *stream, hm_matrix *out);

/* --------------------------------------------------------------- factor --- */

/*
 * Factor the leaf self blocks (paper eq. 12, [Z~_N]^{-1}): FP64 Gauss-Jordan
 * with partial pivoting on the device; the explicit inverse is kept in
 * complex64 (and complex128 with keep_fp64).  Leaves of up to 112 unknowns are
 * inverted in shared memory, one block per CTA.  Larger leaves (up to 1536)
 * are copied into a device workspace of 16 n^2 bytes per leaf, allocated here
 * and freed before return (HM_ERR_OOM if it cannot be had), and eliminated one
 * pivot step at a time across all of them.  Then estimates the level
 * operators' norms and spectral radii as hm_estimate_norms does, with
 * HM_NORM_ITERS_DEFAULT steps.  Synchronises; returns HM_ERR_SINGULAR if a
 * pivot is exactly zero, HM_ERR_ARG for a leaf above 1536.
 */
hm_status hm_factor_leaf(hm_matrix h, void *stream);

#define HM_NORM_ITERS_DEFAULT 32

/*
 * Convergence of the series (paper §IV, eqs. 20-22: the power series of
 * (I + U)^{-1}; §V sets its operating bound as a norm of the level operator
 * below 0.1).  For every level l with blocks, U_l = D^{-1} M_l (l = 1: the
 * non-self near blocks and the leaf-level far blocks; l > 1: the far blocks
 * l - 1 levels above the leaves).  Two power iterations of n_iter steps each,
 * on the device with the solve's own product and leaf-inverse kernels
 * (complex64 vectors, FP64 norms), from fixed start vectors:
 *   norm_est[l-1]  |U_l v| for the unit iterate v of (U_l^H U_l)^k v0: a lower
 *                  bound of ||U_l||_2 that rises toward it as n_iter grows
 *                  (U^H is applied through the complex symmetry of M and D);
 *   rho_est[l-1]   the geometric-mean growth |U_l v| of the iterates of U_l over
 *                  the second half of the steps: an estimate of the spectral
 *                  radius of U_l, which decides whether the series converges
 *                  (it converges for rho < 1, the K-term result is computed and
 *                  returned either way).
 * The results go to hm_info (norm_est, rho_est, norm_iters) and to every
 * hm_solve_info.  Costs 3 n_iter products of each level.  Synchronises.
 * HM_ERR_STATE before hm_factor_leaf, HM_ERR_ARG for n_iter outside [2, 4096].
 */
hm_status hm_estimate_norms(hm_matrix h, int n_iter, void *stream);

/* ---------------------------------------------------------------- solve --- */

typedef struct {
    int n_terms;   /* K: power-series terms (applications of the level operator),
                      the paper's "two fixed iterations" is 2 */
    int n_levels;  /* m: 1 = leaf level only (the paper's runs), -1 = all levels */
    int nested;    /* 1 = literal nested form of eq. 19 (each level's operator is
                      preconditioned by the full lower-level series),
                      0 = flat form S_K(D^{-1}(A_m - D)) D^{-1} (identical for m = 1) */
    int refine;    /* 1 = one refinement step: r = b - A_m x with FP64 accumulation,
                      x += (same series)(r) */
    int fp64;      /* 1 = plain FP64 path: b, x are complex128 and the operator's
                      complex128 copy is used (needs keep_fp64) */
    int graph;     /* 1 = capture the whole solve (every kernel of every term and
                      level) into a CUDA graph on first use and replay it on later
                      calls with the same pointers, sizes and options; 0 = launch
                      kernels one by one.  Ignored while hm_profile is enabled or
                      when info is requested. */
    int persistent; /* 1 = run the whole solve (every term, level, the residual and
                      the refinement) as ONE cooperative kernel whose CTAs walk the
                      solve's steps with a grid-wide barrier between consecutive
                      steps (bounded waits: HM_ERR_TIMEOUT through the status word);
                      the block products run one right-hand side at a time.  The
                      step list is recorded on first use per pointers, sizes and
                      options.  Complex64 only, leaves of at most 128 padded
                      unknowns; otherwise the solve runs as separate kernels.
                      Combines with graph (the launch is then graph-replayed). */
} hm_solve_opts;

typedef struct {
    double rel_residual;     /* |b - A_m x| / |b| (max over columns), FP64; only if refine */
    int levels_used;         /* m after clamping to the levels present */
    int64_t bytes_streamed;  /* algorithmic operator + vector bytes of this solve */
    int64_t kernel_launches; /* kernels enqueued by this call */
    double norm_est[16];     /* levels 1..levels_used: the handle's estimate of ||D^{-1} M_l||_2
                                (hm_estimate_norms), index l - 1; 0 beyond */
    double rho_est[16];      /* the same levels: estimated spectral radius of D^{-1} M_l */
    int convergent;          /* 1: every rho_est of the levels used is below 1 (the series
                                converges as K grows); 0: some level's is not, so the K-term
                                result departs from A_m^{-1} b as K grows; -1: not estimated */
} hm_solve_info;

/*
 * x = power-series solution of A_m x = b (paper eq. 19 with the fixed-term
 * series of §IV).  b, x: DEVICE pointers, nrhs columns.  b is not modified;
 * b and x must not overlap.  `info` may be NULL; when given, the call
 * synchronises and fills it.
 */
hm_status hm_powerseries_solve(hm_matrix h, const void *b, int64_t ldb, void *x, int64_t ldx,
                               int nrhs, const hm_solve_opts *opts, void *stream, hm_solve_info *info);

/*
 * Same as hm_powerseries_solve with HOST buffers b and x (any host memory):
 * copies b to the device, solves, copies x back, and synchronises before
 * returning.  A buffer that is page-locked (cudaMallocHost / cudaHostRegister)
 * and has leading dimension N is copied directly; any other goes through the
 * handle's page-locked staging buffer (allocated on first use, kept).
 */
hm_status hm_powerseries_solve_host(hm_matrix h, const void *b, int64_t ldb, void *x, int64_t ldx,
                                    int nrhs, const hm_solve_opts *opts, void *stream);

/*
 * y = A_m x (the H-Matrix product of §IV, "the solution process only depends
 * on the matrix-vector product"), x, y DEVICE complex64, original order.
 * n_levels as in hm_solve_opts.  fp64_accumulate = 1 accumulates in FP64.
 */
hm_status hm_apply(hm_matrix h, const void *x, int64_t ldx, void *y, int64_t ldy, int nrhs,
                   int n_levels, int fp64_accumulate, void *stream);

/*
 * r = b - A_m x, the residual of the refinement step, accumulated to FP64-class
 * accuracy without FP64 arithmetic in the block products: complex64 blocks and
 * vectors; inside each block the products are summed in short error-free runs
 * (each exact product rounded onto a power-of-two grid bounded by the run's
 * own terms, ExtractScalar of Rump, Ogita & Oishi 2008 through the FMA, with
 * the remainders below the grid summed apart) folded into double-float sums.
 * A block sum errs by at most 2^-39 of sum |a b| (typically 2^-45..2^-47).
 * Sums across blocks and b - A x are formed in FP64, in a fixed order (no
 * atomics on the sums).  b, x, r: DEVICE complex64,
 * original order; r must not overlap b or x.  norms: NULL, or HOST array of
 * 2*nrhs doubles receiving |r_j|^2 and |b_j|^2 (the call then synchronises).
 * Needs hm_factor_leaf (it prepares the complex64 copy of D).
 */
hm_status hm_residual(hm_matrix h, const void *b, int64_t ldb, const void *x, int64_t ldx, void *r, int64_t ldr,
                      int nrhs, int n_levels, double *norms, void *stream);

/*
 * hm_residual_noalloc: the same residual as hm_residual (same arguments, same
 * result), for callers that must not allocate device memory after start-up.
 * One example is a serving process whose memory is reserved up front by a
 * framework's caching allocator, where a late cudaMalloc may fail or stall the
 * device mid-request.  Real-time loops are another.  hm_residual may grow the
 * handle's workspace; this call never allocates (no cudaMalloc, cudaFree or
 * allocating library routine).  It keeps all temporary data in one fixed
 * 32 MiB array in device memory that every GPU loading the library holds until
 * the process exits.  Calls whose operator and nrhs need more than that
 * (3 complex64 vectors of padded length x nrhs, 2 doubles per right-hand side,
 * and the FP64 partial slots of one right-hand side) return HM_ERR_ARG before
 * any device work.
 * The first call on each device does a one-off set-up: it looks up the array's
 * device address.  Under CUDA's lazy module loading (the default) that lookup
 * loads the part of the library's device code that holds the array, which
 * commits the 32 MiB, and the call's first kernel launches may load the device
 * code of the residual kernels if no residual or refined solve has run yet.
 * That set-up can allocate device memory, so make the first call at start-up:
 * before a caching allocator reserves the device's memory, and before any
 * stream capture.  Later calls allocate nothing.  The looked-up address is
 * cached per device for the life of the process; after a cudaDeviceReset in
 * the calling process it is stale, so do not call this entry point after one.
 * All calls share the one array and it keeps the previous call's contents:
 * calls that may overlap on the GPU (other streams, other threads, other
 * handles) race and must be serialised by the caller.  The paper has no
 * counterpart; this is an interface of this library.
 */
hm_status hm_residual_noalloc(hm_matrix h, const void *b, int64_t ldb, const void *x, int64_t ldx, void *r,
                              int64_t ldr, int nrhs, int n_levels, double *norms, void *stream);

/* ------------------------------------------------------------ excitation --- */

/*
 * Right-hand sides of eq. 5 for incident plane waves (paper §II, eq. 5: the
 * excitation b is the tested incident plane wave), unit amplitude: for HM_RWG
 *   b_m = Int f_m . p_hat exp(-jk k_hat . r) dS     (7-point triangle rule),
 * for HM_SWG
 *   b_m = Int kappa f_m . p_hat exp(-jk k_hat . r) dV (4-point tetrahedron rule),
 * the same rules as the fill.  khat, phat:
 * HOST arrays of 3*nrhs doubles (unit propagation direction, unit polarisation).
 * b: DEVICE complex64, column-major N x nrhs in the original order, leading
 * dimension ldb.  Only for operators made by hm_build (the mesh is kept).
 */
hm_status hm_rhs_plane_wave(hm_matrix h, const double *khat, const double *phat, int nrhs, void *b, int64_t ldb,
                            void *stream);

/* ------------------------------------------------------------- profiling --- */

/*
 * Opt-in timing of the block-product kernel (the near/far-field H-Matrix product
 * of every series term): while enabled, every launch of that kernel made by
 * hm_powerseries_solve is bracketed by CUDA events recorded on the launching
 * stream.  enable = 1 starts a new measurement (counters reset), 0 stops.
 */
hm_status hm_profile(hm_matrix h, int enable);

/*
 * Synchronises the recorded events and returns the summed kernel time (ms), the
 * number of timed launches, and the algorithmic bytes those launches had to move
 * (complex64 block elements at their unpadded sizes, plus one read of x and one
 * write of z per right-hand side).
 */
hm_status hm_profile_read(hm_matrix h, double *product_ms, int64_t *launches, int64_t *bytes);

/* --------------------------------------------------------------- serving --- */

/*
 * Continuous-batching solve server.  Operators are registered as meshes (with
 * build and solve options) and built on the GPU on first use.  Requests carry
 * nrhs right-hand sides in host memory and are queued per operator.  A
 * scheduler thread merges the queued requests of one operator, in arrival
 * order, into one multi-RHS solve of at most max_batch_rhs columns.  It runs
 * batches of different operators concurrently on n_slots CUDA streams (their
 * kernels overlap on the device).  Before building an operator it evicts idle
 * least-recently-used operators until the resident device bytes fit
 * hbm_budget_bytes (a target: an operator larger than the budget is still
 * admitted when nothing else is resident).  Requests that arrive while
 * others run join the next batch of their operator.  Complex64 only.
 * The server owns its operators; all calls are thread safe.
 */
typedef struct hm_server_s *hm_server;
typedef struct {
    int64_t batches, solved_rhs, builds, evictions, resident_bytes, peak_resident_bytes;
    int64_t loop_launches;   /* device-loop mode: launches of the request loop kernel */
    int64_t loop_stops;      /* device-loop mode: stops for host-side GPU work (builds, allocation) */
} hm_server_info;

hm_status hm_server_create(int n_slots, int64_t hbm_budget_bytes, int max_batch_rhs, hm_server *out);

/*
 * The same server with device_loop = 1: a device-resident request loop.  One
 * cooperative kernel stays on the GPU and serves the batches from a ring in
 * mapped pinned host memory, with no kernel launch per batch: the scheduler
 * thread copies a batch's right-hand sides to its slot's device buffer, writes
 * the ring entry (the batch's one-launch solve, recorded for every right-hand-side
 * count rounded up to a multiple of 4 when the operator is built, the slot's
 * buffers and the operator's context) and marks it ready; the kernel runs it
 * between grid barriers and marks it done; the scheduler copies the solutions
 * out.  Batches run one after another on the whole GPU (n_slots batches can be
 * queued in the ring).  Builds (with their recordings), evictions and slot
 * buffer growth stop the loop (a stop entry after everything queued) and run on
 * the host side; an idle loop leaves by itself after about a second and is
 * launched again by the next batch.  Every
 * wait of the kernel is bounded; a wait that gives up fails the batch it was
 * serving with HM_ERR_TIMEOUT.  The solve options of every operator must fit the
 * one-launch solve (complex64, leaves of at most 128 padded unknowns; HM_ERR_ARG
 * for the batch otherwise).  device_loop = 0 is hm_server_create.
 */
hm_status hm_server_create_ex(int n_slots, int64_t hbm_budget_bytes, int max_batch_rhs, int device_loop,
                              hm_server *out);
/* Registers a mesh (either basis); *n_unknowns receives its unknown count N (the length of every
 * right-hand side of this operator). */
hm_status hm_server_add_mesh(hm_server s, const hm_mesh *mesh, const hm_build_opts *bo, const hm_solve_opts *so,
                             int *op_id, int64_t *n_unknowns);
/* Queues nrhs right-hand sides b (host, complex64, N x nrhs column-major, copied
 * during the call); n must equal the operator's N.  HM_ERR_OOM, before anything is
 * queued, when the request alone needs more device memory than the HBM budget (at
 * least 8 N (2 + 4 (m + 1) + 8) bytes per right-hand side for its buffers and the
 * solve's work vectors, m = the operator's solve levels, 1 if all); other requests
 * are not affected. */
hm_status hm_server_submit(hm_server s, int op_id, const void *b, int64_t n, int nrhs, int64_t *req_id);
/* Blocks until the request is solved (at most 600 s), copies its solution to x
 * (host, N x nrhs) and gives the submit-to-completion latency in ms. */
hm_status hm_server_wait(hm_server s, int64_t req_id, void *x, double *latency_ms);
hm_status hm_server_get_info(hm_server s, hm_server_info *info);
void hm_server_destroy(hm_server s);

/* ---------------------------------------------------------- inspection --- */

typedef struct {
    int64_t n;               /* unknowns */
    int64_t n_leaves;
    int depth;               /* tree depth L (root = 0) */
    int n_levels;            /* far-field levels present (1 = leaf level only) */
    int64_t n_near;          /* stored (half) near blocks */
    int64_t n_far[16];       /* stored far blocks per level (index 0 = level 1) */
    int64_t near_elems;      /* complex elements of the near blocks */
    int64_t far_elems[16];   /* complex elements k (m + n) per level */
    int64_t self_elems;      /* sum n_i^2 */
    int max_rank;
    int factored;
    int has_fp64;
    int64_t device_bytes;    /* device memory held by the handle */
    double norm_est[16];     /* per level (index l - 1): estimate of ||D^{-1} M_l||_2 (hm_estimate_norms) */
    double rho_est[16];      /* per level: estimated spectral radius of D^{-1} M_l */
    int norm_iters;          /* steps of the last estimate, 0 if none was made */
} hm_info;

hm_status hm_get_info(hm_matrix h, hm_info *info);

/*
 * Kernel choice of the built-in autotuner for `nrhs` right-hand sides (no
 * counterpart in the paper: it concerns how this GPU implementation batches the
 * block products of eqs. 6 and 8).  Right-hand-side counts share a choice per
 * bucket (the next power of two >= nrhs, at least 4).  The first complex64
 * solve, product or residual in a bucket on an operator times the candidate
 * kernels on that operator at the bucket's size (with CUDA events on the
 * caller's stream, which it synchronises once) and keeps the fastest: for the product and for the
 * FP64-class residual products, 0 = one right-hand side at a time, 8 / 16 / 32 =
 * blocks staged once in shared memory per chunk of that many right-hand sides,
 * 1016 (product only, timed from 32 right-hand sides on) = the blocks of at most
 * 64 x 64 (rank <= 32) on the tensor cores in tiles of 128 right-hand sides;
 * 1017 (residual only, where every level of the call holds only such blocks) =
 * owner-computes FP64-class products, one CTA per output cluster and group of 16
 * right-hand sides, no partial slots.  res_ms of the owner kernel covers all
 * nrhs right-hand sides at once, of the others one chunk of at most 16.
 * prod_ms / res_ms: the measured time of one leaf-level launch of the choice.
 * Any output pointer may be NULL.  HM_ERR_STATE if no call with that nrhs has
 * been made yet (or nrhs < 4, which needs no choice).
 */
hm_status hm_get_tuning(hm_matrix h, int nrhs, int *prod_rb, int *res_rb, double *prod_ms, double *res_ms);

/*
 * Pin the kernel choice for the bucket of `nrhs` right-hand sides instead of
 * letting the autotuner time it (e.g. for reproducible benchmarks or to test a
 * kernel): prod_rb 0 (one right-hand side at a time), 8 / 16 / 32 (shared-memory
 * SIMT chunks) or 1016 (tensor-core products of the blocks of at most 64 x 64 and
 * rank <= 32, dense and low-rank, tiles of 128 right-hand sides, tcgen05 3xTF32;
 * the first call that runs it allocates its stage-1 workspace: the low-rank
 * intermediates, 8 KB per 8 rank rows of every low-rank block side and per tile,
 * counted in hm_info.device_bytes);
 * res_rb 0, 8, 16 or 1017 (owner-computes; calls whose levels hold larger blocks
 * fall back to the partial-slot kernel of one right-hand side at a time).  Drops captured solve graphs.  HM_ERR_ARG for nrhs < 4 or
 * another value.
 */
hm_status hm_set_tuning(hm_matrix h, int nrhs, int prod_rb, int res_rb);

/*
 * Bound of the device waits of this library's kernels (no counterpart in the
 * paper).  Two kernels wait on other parts of the GPU:
 *  - the tensor-core product (hm_set_tuning choice 1016): its roles (copies,
 *    operand conversion, MMA issue) hand shared-memory slots to one another
 *    through mbarriers.  On a time-out every role of the CTA leaves, the
 *    copies and MMAs already in flight are waited for at the full bound, and
 *    the tensor memory is freed;
 *  - the one-launch solve (hm_solve_opts.persistent): its CTAs meet at a
 *    grid-wide barrier between steps.  A CTA that gives up leaves the kernel,
 *    so every other CTA gives up at its next barrier.
 * Each wait polls at most `polls` times (default 2^24, a few seconds), then the
 * kernel records HM_ERR_TIMEOUT in the device status word (returned by
 * hm_sync_status and by the next synchronising call); the result is then
 * incomplete.  polls < 0 restores the default; 0 makes every such wait give up
 * at once (to exercise the error path).  Drops captured solve graphs.
 * HM_ERR_ARG above 2^32 - 1.
 */
hm_status hm_set_wait_limit(hm_matrix h, int64_t polls);

/* Tree permutation (tree position -> original unknown), host int64[n]. */
hm_status hm_get_perm(hm_matrix h, int64_t *perm);

/* Leaf offsets, host int64[n_leaves + 1]. */
hm_status hm_get_leaves(hm_matrix h, int64_t *leaf_off);

/*
 * Block list of level `level` (1 = leaf level; level 1 lists the near blocks
 * first, rank 0), host arrays of length count (query count with NULL arrays):
 * row0, col0 (tree positions), m, n, rank.
 */
hm_status hm_get_blocks(hm_matrix h, int level, int64_t *count, int64_t *row0, int64_t *col0,
                        int32_t *m, int32_t *n, int32_t *rank);

/*
 * Copy one stored block to host complex128 memory: dense blocks as row-major
 * m x n into `a` (b unused); low-rank blocks as U (m x k row-major) into `a`
 * and V (k x n row-major) into `b`.  index as in hm_get_blocks.
 */
hm_status hm_get_block(hm_matrix h, int level, int64_t index, double *a, double *b);

/* Device status word: synchronises `stream`, returns and clears the first
 * device-side error recorded since the last call. */
hm_status hm_sync_status(hm_matrix h, void *stream);

int64_t hm_size(hm_matrix h);
void hm_destroy(hm_matrix h);
const char *hm_last_error(void);
const char *hm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* HMPS_H */
