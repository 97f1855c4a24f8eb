// Tensor-core block products for many right-hand sides (arxiv 2307.03968 eq. 6
// and §III: the near blocks and the low-rank far blocks U(V x) of one level,
// half stored, each block used for both mirrored products):
//     Z_I += B X_J,   Z_J += B^T X_I
// on the 5th-generation tensor cores (tcgen05.mma kind::tf32, accumulators in
// tensor memory).
//
// Orientation.  The right-hand sides are the M dimension: a tile of 128 of them
// gives the 128 rows of the accumulator (tensor-memory lane r = right-hand side
// r of the tile).
//
// Complex arithmetic.  With X = Xr + i Xi (tile rows x input) and B = Br + i Bi
// (output x input), the accumulator [Re Z | Im Z] (128 x 2*m8) is
//     Xr [Br ; Bi]^T + Xi [-Bi ; Br]^T
// where [Br ; Bi] stacks the planes along N.  The B operand of a K step holds the
// three planes -Bi, Br, Bi one after another, so both products are windows of
// the same shared-memory rows (start at -Bi or at Br, N = 2*m8).
//
// Two launches per product.
//  - k_tc_stage1: stage 1 of every low-rank directed product (B = Y W, rank k;
//    W = V and Y = U forward, W = U^T and Y = V^T mirrored), T = X W^T, batched over
//    the products that share an input cluster: their W rows are stacked along N
//    (roundup8(k) rows each, at most 64 in all), so one K chunk of split x feeds
//    MMAs of N up to 128 instead of one product's 2*roundup8(k).  Each batch's
//    accumulator (two alternate in tensor memory) is stored in HBM as T chunks of 8
//    rank rows: for the 128 RHS of the tile, a plane of Re T and a plane of Im T in
//    the layout of an A operand plane (poff).
//  - k_apply_tc: per output cluster, work units of its dense products and second
//    stages Z += T Y^T.  A second stage's A operand is a T chunk copied in raw and
//    split by the converters in place: thread r reads row r's 16 values and writes
//    the four split planes at row r's own positions, so no thread reads what another
//    writes.  One CTA keeps the sum for (cluster, RHS tile) in tensor memory while it
//    streams the unit, and adds it into z once.
//
// Precision (3xTF32): every FP32 operand a is split as a = hi + lo, hi = a
// rounded to TF32 (|a - hi| <= 2^-11 |a|), lo = a - hi rounded to TF32 too; each
// K step accumulates hi*hi + hi*lo + lo*hi in FP32 (the dropped lo*lo and the
// rounding of lo are <= 2^-22 |a b| each).  T is held in FP32 between the stages,
// as it was when it stayed in tensor memory.  The larger error is the tensor core's
// FP32 accumulation, which loses a little on every MMA added into a large running
// sum: measured against the oracle, the product erred 7.4e-6 (relative, 60-unknown
// leaves) when a work unit summed 256 K chunks in tensor memory, and a refined
// solve 1.2e-4, above the 1e-4 bar; with units of at most 64 chunks
// (TC_UNIT_CHUNKS: each unit's sum is drained into z in FP32) the product errs
// 1.9e-6, and the 181-RHS sweep of the 30,720-unknown sphere stays within 2.3e-5 of
// the oracle (16-chunk units: 5.4e-7 and 7e-6, at 31 % more time per launch); in two
// launches, whose units gather about five times as many low-rank products (only their
// second-stage chunks count), the sweep stays within 2.9e-5.
// Adding the lo*lo products changed neither (same errors to four digits).
//
// Pipeline (both kernels; warp-specialised, mbarrier hand-offs, no CTA-wide barrier
// per chunk).  K goes in chunks of 8 (one MMA K step) through a ring of shared-memory
// slots.  Before the launches, x is split once into hi/lo planes per (input-cluster
// K chunk, RHS tile), already in the operand layout (k_split_x).  Warp 0 (producer)
// copies a chunk's A planes (split x, or a raw T chunk) with one cp.async.bulk and
// the raw complex64 rows of the block or factor with cp.async.  Warps 1-4
// (converters) split the block rows into the B planes (and a raw T chunk into the A
// planes), and store finished accumulators (into z, or as T chunks).  Warp 5 issues
// the six MMAs of a chunk and commits them to the slot's "empty" mbarrier.  Two CTAs
// share an SM.  Every pipeline wait is bounded by a number of polls given at launch
// (hm_set_wait_limit; default 2^24): on timeout the kernel records HM_ERR_TIMEOUT in
// the status word and all roles leave their loops.  Before the CTA ends, the
// producer waits for its bulk copies in flight and the MMA issuer for its MMAs in
// flight, both at the full bound (2^24 polls) whatever the pipeline limit, and only
// then is the tensor memory freed.
#include "k_common.cuh"

namespace hm {
namespace {

using namespace kc;
constexpr int NWARP = 6;                         // 0 producer, 1-4 converters (tensor-memory lanes 32(w%4)..), 5 MMA
constexpr int TT = NWARP * 32;
constexpr int NCV = 128;                         // converter threads
constexpr int NCW = NCV / 32;                    // converter warps: the arrivals on ready and acc_empty
constexpr int TM = 128;                          // MMA M: right-hand sides per tile
constexpr int KCH = 8;                           // K per chunk (complex unknowns; one MMA K step)
constexpr int NSLOT = 3;
constexpr int A_PLANE = TM * KCH * 4;            // bytes of one A plane (Xr/Xi x hi/lo): 4 KB
constexpr int A_BYTES = 4 * A_PLANE;             // 16 KB, one bulk copy
constexpr int B_ROWS = 3 * 64;                   // -Bi, Br, Bi rows of one B plane (<= 64 rows each)
constexpr int B_PLANE = B_ROWS * KCH * 4;        // bytes of one B plane (hi or lo): 6 KB
constexpr int B_RAW = 64 * KCH * 8;              // raw complex64 block / factor rows: 4 KB
constexpr int SLOT = A_BYTES + 2 * B_PLANE + B_RAW;   // 32 KB
constexpr int OFF_B = A_BYTES, OFF_RAW = A_BYTES + 2 * B_PLANE;
constexpr int SMEM = NSLOT * SLOT;
constexpr uint32_t TMEM_COLS = 128;              // k_apply_tc: the output accumulator (N = 2*m8 <= 128)
constexpr uint32_t S1_TMEM_COLS = 256;           // k_tc_stage1: two alternate accumulators at columns 0 and 128
constexpr int S1_ROWS = 64;                      // stacked W rows of a stage-1 batch, at most
constexpr int T_PLANE = TM * KCH;                // floats of one plane (Re or Im) of a T chunk
constexpr uint32_t GROUP_BYTES = 2 * 128;        // one 8-row group: two K-adjacent core matrices
constexpr uint32_t WAIT_LIMIT = 1u << 24;
static_assert(TC_MAX_DIM <= 64 && TC_MAX_RANK <= 32, "operand planes and tensor-memory columns");
static_assert(2 * T_PLANE == TC_T_CHUNK && 2 * T_PLANE * 4 <= A_BYTES, "a raw T chunk fits the A planes it becomes");
static_assert(3 * S1_ROWS <= B_ROWS && S1_ROWS <= 64, "stacked rows fit the B planes and the raw rows");

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void split_tf32(float a, float &hi, float &lo)
{
    uint32_t h, l;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(a));
    hi = __uint_as_float(h);
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(__fsub_rn(a, hi)));
    lo = __uint_as_float(l);
}

// shared-memory matrix descriptor, K-major, no swizzle: core matrices of 8 rows x
// 16 bytes, K-adjacent cores 128 B apart, 8-row groups GROUP_BYTES apart
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr)
{
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)(128u >> 4) << 16;
    d |= (uint64_t)((GROUP_BYTES >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// float offset of (row, K index k < 8) in a plane
__device__ __forceinline__ int poff(int row, int k) { return (((row >> 3) * 2 + (k >> 2)) << 5) + ((row & 7) << 2) + (k & 3); }

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity)
{
    uint32_t done;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
    return done != 0;
}

// bounded wait on an mbarrier phase of the pipeline (at most `limit` polls, 0 = give up
// at once); gives up early once another role aborted
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, volatile int *abort, uint32_t limit)
{
    for (uint32_t it = 0; it < limit; ++it) {
        if (mbar_try(mbar, parity)) return true;
        if (*abort) return false;
    }
    *abort = 1;
    return false;
}

// converter warp: the bounded wait taken by the whole warp, so that its lanes leave
// together (they go on to warp-collective steps: tcgen05.ld, one arrival per warp)
__device__ __forceinline__ bool warp_wait(uint32_t mbar, uint32_t parity, volatile int *abort, uint32_t limit)
{
    const bool ok = mbar_wait(mbar, parity, abort, limit);
    return __all_sync(0xffffffffu, ok);
}
__device__ __forceinline__ bool warp_aborted(volatile int *abort) { return __any_sync(0xffffffffu, *abort != 0); }

// wait for asynchronous work this thread issued (bulk copies, MMAs) before the CTA
// frees what that work writes: the full bound, not cut short by an abort
__device__ __forceinline__ void mbar_drain(uint32_t mbar, uint32_t parity, volatile int *abort)
{
    for (uint32_t it = 0; it < WAIT_LIMIT; ++it)
        if (mbar_try(mbar, parity)) return;
    *abort = 1;
}

__device__ __forceinline__ void arrive(uint32_t mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}
// converter warp: one arrival for the warp once every lane is past its writes (each lane
// has fenced its own shared-memory writes to the async proxy, or its tensor-memory loads,
// before the warp synchronises; the arrival releases them all)
__device__ __forceinline__ void warp_arrive(uint32_t mbar, int lane)
{
    __syncwarp();
    if (lane == 0) arrive(mbar);
}
__device__ __forceinline__ void commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tld8(uint32_t taddr, float (&v)[8])
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 16-byte copy (bytes < 16: zero-filled) with an L2 eviction policy
__device__ __forceinline__ void cp16(uint32_t dst, const void *src, int bytes, uint64_t pol)
{
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2, %3;" ::"r"(dst), "l"(src), "r"(bytes),
                 "l"(pol) : "memory");
}
__device__ __forceinline__ int clamp16(int bytes) { return bytes < 0 ? 0 : bytes > 16 ? 16 : bytes; }

// the A planes of tile row r from 8 complex values: Xr hi, Xr lo, Xi hi, Xi lo
// (4 planes of A_PLANE bytes, plane-major; the same layout in shared and global memory)
__device__ __forceinline__ void put_a_row(float4 *p, int r, const float (&re)[8], const float (&im)[8])
{
    constexpr int PF4 = A_PLANE / 16;            // float4 per plane
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        float rh[4], rl[4], ih[4], il[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            split_tf32(re[4 * c + j], rh[j], rl[j]);
            split_tf32(im[4 * c + j], ih[j], il[j]);
        }
        const int o = poff(r, 4 * c) >> 2;
        p[o] = make_float4(rh[0], rh[1], rh[2], rh[3]);
        p[PF4 + o] = make_float4(rl[0], rl[1], rl[2], rl[3]);
        p[2 * PF4 + o] = make_float4(ih[0], ih[1], ih[2], ih[3]);
        p[3 * PF4 + o] = make_float4(il[0], il[1], il[2], il[3]);
    }
}

// split x once per launch: chunk g of the input clusters (unknowns off .. off+valid-1)
// for RHS tile t (rows r0 .. r0+127) -> xpl[(t * n_xch + g)], A_BYTES each
__global__ void __launch_bounds__(TM)
k_split_x(const XChunk *__restrict__ xch, int64_t n_xch, const float2 *__restrict__ x, int64_t ldx, int nrhs,
          float *__restrict__ xpl)
{
    const int64_t g = blockIdx.x;
    const int t = blockIdx.y, r = threadIdx.x, r0 = t * TM;
    const XChunk ch = xch[g];
    float re[8], im[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) { re[j] = 0.f; im[j] = 0.f; }
    if (r0 + r < nrhs) {
        const float2 *src = x + (int64_t)(r0 + r) * ldx + ch.off;
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (j < ch.len) { const float2 v = __ldg(src + j); re[j] = v.x; im[j] = v.y; }
    }
    put_a_row(reinterpret_cast<float4 *>(xpl + ((int64_t)t * n_xch + g) * (A_BYTES / 4)), r, re, im);
}

// Raw B layouts (16-byte pieces, swizzled so that the conversion reads are free of
// bank conflicts):
//   natural: row rho, complex q .. q+1 (piece q/2) at  rho*64 + ((q/2) ^ ((rho>>1)&3))*16
//   transposed: K row k, rows row .. row+1 (piece row/2) at  k*512 + ((row/2) ^ k)*16
__device__ __forceinline__ int swz_n(int r, int pc) { return r * 64 + ((pc ^ ((r >> 1) & 3)) << 4); }
__device__ __forceinline__ int swz_t(int k, int pc) { return k * 512 + ((pc ^ k) << 4); }

// producer lane: raw B rows, natural orientation: element (row, q) = src[row * ld + q]
// for row < rows_valid, q = k0 + j < klen (else zero); rows < R8
__device__ __forceinline__ void fetch_b_nat(uint32_t raw, int lane, const float2 *__restrict__ src, int ld, int R8,
                                            int rows_valid, int k0, int klen, uint64_t pol)
{
    for (int id = lane; id < 4 * R8; id += 32) {
        const int row = id >> 2, pc = id & 3;
        const int q = k0 + 2 * pc;
        const int bytes = row < rows_valid ? clamp16((klen - q) * 8) : 0;
        cp16(raw + swz_n(row, pc), bytes > 0 ? (const void *)(src + (int64_t)row * ld + q) : (const void *)src, bytes,
             pol);
    }
}

// producer lane: raw B rows, transposed orientation: element (row, q) = src[q * ld + row]
// for row < rows_valid, q = k0 + k < klen (else zero); rows < R8
__device__ __forceinline__ void fetch_b_tr(uint32_t raw, int lane, const float2 *__restrict__ src, int ld, int R8,
                                           int rows_valid, int k0, int klen, uint64_t pol)
{
    const int k = lane & 7;
    const bool kv = k0 + k < klen;
    const float2 *p = src + (int64_t)(k0 + k) * ld;
    for (int pc = lane >> 3; 2 * pc < R8; pc += 4) {
        const int row = 2 * pc;
        const int bytes = kv ? clamp16((rows_valid - row) * 8) : 0;
        cp16(raw + swz_t(k, pc), bytes > 0 ? (const void *)(p + row) : (const void *)src, bytes, pol);
    }
}

// producer lane: the stacked W rows of a stage-1 batch, natural orientation: element
// (row, q) = pool[rs + q] for q = k0 + j < klen, with rs the row's W offset (-1: a zero
// row).  The lane's rows are (lane >> 2) + 8 i (offsets in rs[i]), its 16-byte piece
// lane & 3: the same pieces fetch_b_nat gives it.
__device__ __forceinline__ void fetch_b_rows(uint32_t raw, int lane, const float2 *__restrict__ pool,
                                             const int64_t (&rs)[8], int R8, int k0, int klen, uint64_t pol)
{
    const int pc = lane & 3, q = k0 + 2 * pc;
    const int bytes_k = clamp16((klen - q) * 8);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int row = (lane >> 2) + 8 * i;
        if (row >= R8) break;
        const int bytes = rs[i] >= 0 ? bytes_k : 0;
        cp16(raw + swz_n(row, pc), bytes > 0 ? (const void *)(pool + rs[i] + q) : (const void *)pool, bytes, pol);
    }
}

// converter thread r (0..127): the A planes of row r from a raw T chunk in the same
// slot (Re T in plane 0, Im T in plane 1, both at the positions poff(r, k)).  Row r's
// 16 values are read before any is written, and put_a_row writes only row r's
// positions, so the split runs in place without a barrier between threads.
__device__ __forceinline__ void conv_a_raw(float *slot, int r)
{
    const float4 *p = reinterpret_cast<const float4 *>(slot);
    const int o0 = poff(r, 0) >> 2, o1 = poff(r, 4) >> 2;
    const float4 a = p[o0], b = p[o1], c = p[T_PLANE / 4 + o0], d = p[T_PLANE / 4 + o1];
    const float re[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    const float im[8] = {c.x, c.y, c.z, c.w, d.x, d.y, d.z, d.w};
    put_a_row(reinterpret_cast<float4 *>(slot), r, re, im);
}

// converter thread t (0..127): B planes from a raw natural chunk (rows < R8): row t/2,
// K indices 4*(t&1) .. +3
__device__ __forceinline__ void conv_b_nat(float *bhi, float *blo, const unsigned char *raw, int R8, int t);

// the B planes of 4 K-consecutive elements of one row (K indices 4*half .. 4*half+3)
__device__ __forceinline__ void put_b4(float *bhi, float *blo, int row, int R8, int half, const float (&v)[8])
{
    float nh[4], nl[4], rh[4], rl[4], ih[4], il[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        split_tf32(v[2 * j], rh[j], rl[j]);
        split_tf32(v[2 * j + 1], ih[j], il[j]);
        nh[j] = -ih[j]; nl[j] = -il[j];
    }
    float4 *H = reinterpret_cast<float4 *>(bhi), *L = reinterpret_cast<float4 *>(blo);
    int o = poff(row, 4 * half) >> 2;
    H[o] = make_float4(nh[0], nh[1], nh[2], nh[3]); L[o] = make_float4(nl[0], nl[1], nl[2], nl[3]);
    o = poff(R8 + row, 4 * half) >> 2;
    H[o] = make_float4(rh[0], rh[1], rh[2], rh[3]); L[o] = make_float4(rl[0], rl[1], rl[2], rl[3]);
    o = poff(2 * R8 + row, 4 * half) >> 2;
    H[o] = make_float4(ih[0], ih[1], ih[2], ih[3]); L[o] = make_float4(il[0], il[1], il[2], il[3]);
}

// converter thread t (0..127): B planes from a raw transposed chunk (rows < R8): row t/2,
// K indices 4*(t&1) .. +3, one 8-byte element from each of four K rows
__device__ __forceinline__ void conv_b_tr(float *bhi, float *blo, const unsigned char *raw, int R8, int t)
{
    const int row = t >> 1, half = t & 1;
    if (row >= R8) return;
    float v[8];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int k = 4 * half + j;
        const float2 e = *reinterpret_cast<const float2 *>(raw + swz_t(k, row >> 1) + ((row & 1) << 3));
        v[2 * j] = e.x;
        v[2 * j + 1] = e.y;
    }
    put_b4(bhi, blo, row, R8, half, v);
}

__device__ __forceinline__ void conv_b_nat(float *bhi, float *blo, const unsigned char *raw, int R8, int t)
{
    const int row = t >> 1, half = t & 1;
    if (row >= R8) return;
    const float4 a = *reinterpret_cast<const float4 *>(raw + swz_n(row, 2 * half));
    const float4 b = *reinterpret_cast<const float4 *>(raw + swz_n(row, 2 * half + 1));
    const float v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    put_b4(bhi, blo, row, R8, half, v);
}

// the six MMAs of one chunk into the accumulator at tensor-memory address acc:
// acc (+)= Xr [Br;Bi]^T + Xi [-Bi;Br]^T in 3xTF32 (N = 2 R8)
__device__ __forceinline__ void issue_chunk(uint32_t slot, uint32_t acc, int R8, bool accumulate)
{
    const uint32_t N = 2u * (uint32_t)R8;
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((N >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
    const uint32_t a0 = slot, b0 = slot + OFF_B;
    const uint32_t pos = (uint32_t)(R8 >> 3) * GROUP_BYTES;      // the [Br;Bi] window
    const uint64_t xr_h = smem_desc(a0), xr_l = smem_desc(a0 + A_PLANE);
    const uint64_t xi_h = smem_desc(a0 + 2 * A_PLANE), xi_l = smem_desc(a0 + 3 * A_PLANE);
    const uint64_t bp_h = smem_desc(b0 + pos), bp_l = smem_desc(b0 + B_PLANE + pos);
    const uint64_t bn_h = smem_desc(b0), bn_l = smem_desc(b0 + B_PLANE);
    const uint32_t first = accumulate ? 1u : 0u;
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc), "l"(xr_h), "l"(bp_h),
                 "r"(idesc), "r"(first));
    asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;\n" ::"r"(acc), "l"(xr_h), "l"(bp_l), "r"(idesc));
    asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;\n" ::"r"(acc), "l"(xr_l), "l"(bp_h), "r"(idesc));
    asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;\n" ::"r"(acc), "l"(xi_h), "l"(bn_h), "r"(idesc));
    asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;\n" ::"r"(acc), "l"(xi_h), "l"(bn_l), "r"(idesc));
    asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;\n" ::"r"(acc), "l"(xi_l), "l"(bn_h), "r"(idesc));
}

// converter: add the output accumulator rows of lane quadrant quad (tile rows < nr,
// outputs < mlen) into z
__device__ __forceinline__ void drain(uint32_t tmem, int quad, int lane, int m8, int mlen, float2 *__restrict__ z,
                                      int64_t ldz, int r0, int nr, int out0)
{
    const int r = 32 * quad + lane;
    const uint32_t lane_base = (uint32_t)(32 * quad) << 16;
    float2 *zr = z + (int64_t)(r0 + r) * ldz + out0;
    for (int i0 = 0; i0 < m8; i0 += 8) {
        float re[8], im[8];
        tld8(tmem + lane_base + (uint32_t)i0, re);
        tld8(tmem + lane_base + (uint32_t)(m8 + i0), im);
        tld_wait();
        if (r < nr) {
#pragma unroll
            for (int j = 0; j < 8; j += 2) {
                const int i = i0 + j;
                if (i + 1 < mlen) red2(zr + i, make_float2(re[j], im[j]), make_float2(re[j + 1], im[j + 1]));
                else if (i < mlen) red1(zr + i, make_float2(re[j], im[j]));
            }
        }
    }
}

// converter: store a stage-1 accumulator (tensor-memory column acc, rows of lane
// quadrant quad, R8 stacked rows) as T chunks: group g of 8 rows -> chunk tch[g] of the
// tile's T (tbase), Re and Im planes at row r's positions poff(r, k)
__device__ __forceinline__ void store_t(uint32_t tmem, uint32_t acc, int quad, int lane, int R8,
                                        const int32_t (&tch)[S1_ROWS / 8], float *__restrict__ tbase)
{
    const int r = 32 * quad + lane;
    const uint32_t lane_base = (uint32_t)(32 * quad) << 16;
    const int o0 = poff(r, 0) >> 2, o1 = poff(r, 4) >> 2;
#pragma unroll
    for (int g = 0; g < S1_ROWS / 8; ++g) {
        if (8 * g >= R8) break;
        float re[8], im[8];
        tld8(tmem + lane_base + acc + (uint32_t)(8 * g), re);
        tld8(tmem + lane_base + acc + (uint32_t)(R8 + 8 * g), im);
        const int64_t chunk = tch[g];
        tld_wait();
        // streaming stores (evict first): T passes through L2 once, the split x stays
        float4 *d = reinterpret_cast<float4 *>(tbase + chunk * TC_T_CHUNK);
        __stcs(d + o0, make_float4(re[0], re[1], re[2], re[3]));
        __stcs(d + o1, make_float4(re[4], re[5], re[6], re[7]));
        __stcs(d + T_PLANE / 4 + o0, make_float4(im[0], im[1], im[2], im[3]));
        __stcs(d + T_PLANE / 4 + o1, make_float4(im[4], im[5], im[6], im[7]));
    }
}

// the mbarriers and tensor-memory allocation of a CTA of either kernel
__device__ __forceinline__ void init_pipeline(uint64_t *full, uint64_t *ready, uint64_t *empty, uint64_t *acc_full,
                                              uint64_t *acc_empty, int n_acc, uint64_t *fin, volatile int *abort_flag)
{
    for (int s = 0; s < NSLOT; ++s) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&full[s])), "r"(33));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&ready[s])), "r"(NCW));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&empty[s])));
    }
    for (int b = 0; b < n_acc; ++b) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&acc_full[b])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&acc_empty[b])), "r"(NCW));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(fin)));
    asm volatile("fence.mbarrier_init.release.cluster;");
    *abort_flag = 0;
}

// producer lane 0: one bulk copy of `bytes` into the slot, completing on full
__device__ __forceinline__ void bulk_in(uint32_t slot, const float *src, uint32_t bytes, uint64_t *full, uint64_t pol)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(full)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
                 " [%0], [%1], %2, [%3], %4;"
                 ::"r"(slot), "l"(src), "r"(bytes), "r"(su32(full)), "l"(pol) : "memory");
}

// producer, after its loop: its cp.async copies, and the slot fills still in flight,
// land before the CTA may end (their full phases complete on the copies alone)
__device__ __forceinline__ void producer_drain(uint64_t *full, uint32_t n, int lane, volatile int *abort_flag)
{
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (lane == 0)
        for (uint32_t f = n > (uint32_t)NSLOT ? n - NSLOT : 0; f < n; ++f)
            mbar_drain(su32(&full[f % NSLOT]), (f / NSLOT) & 1, abort_flag);
    __syncwarp();
}

// ---- k_tc_stage1: T = X W^T for batches of stacked W rows --------------------------

// Position in a CTA's chunk sequence: batch-tile u (taken in turn with stride
// gridDim.x, tile-major), chunk c of nch; the next batch's record is loaded when a
// batch begins.  Every role walks the same sequence.
struct S1Pos {
    int64_t u;
    int c, nch, tile;
    bool valid, has_next;
    TcBatch B, Bn;
};

struct S1Seq {
    const TcBatch *batches;
    int n_batches;
    int64_t total;
    __device__ void enter(S1Pos &q) const
    {
        q.tile = (int)(q.u / n_batches);
        q.c = 0;
        q.nch = (q.B.klen + KCH - 1) / KCH;
        const int64_t un = q.u + gridDim.x;
        q.has_next = un < total;
        if (q.has_next) q.Bn = batches[un % n_batches];
    }
    __device__ void first(S1Pos &q) const
    {
        q.valid = q.u < total;
        if (!q.valid) return;
        q.B = batches[q.u % n_batches];
        enter(q);
    }
    __device__ void next(S1Pos &q) const
    {
        if (++q.c < q.nch) return;
        q.u += gridDim.x;
        q.valid = q.has_next;
        if (!q.valid) return;
        q.B = q.Bn;
        enter(q);
    }
};

// producer lane: the W offsets of its stacked rows (lane >> 2) + 8 i of batch B
__device__ __forceinline__ void load_rows(int64_t (&rs)[8], const int64_t *__restrict__ rows, const TcBatch &B, int lane)
{
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int row = (lane >> 2) + 8 * i;
        rs[i] = row < B.nrows ? rows[B.row0 + row] : -1;
    }
}

__global__ void __launch_bounds__(TT, 2)
k_tc_stage1(const TcBatch *__restrict__ batches, int n_batches, const int64_t *__restrict__ rows,
            const int32_t *__restrict__ tchunks, int64_t n_xch, const float *__restrict__ xpl,
            const float2 *__restrict__ pool, float *__restrict__ tct, int64_t n_tchunk, int n_tiles, int *status,
            uint32_t wait_limit)
{
    extern __shared__ __align__(1024) unsigned char smraw[];
    __shared__ __align__(8) uint64_t full[NSLOT], ready[NSLOT], empty[NSLOT];
    __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2], fin;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    if (tid == 0) init_pipeline(full, ready, empty, acc_full, acc_empty, 2, &fin, &abort_flag);
    if (w == NWARP - 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                     "n"(S1_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t sm0 = su32(smraw);
    const S1Seq seq{batches, n_batches, (int64_t)n_batches * n_tiles};
    S1Pos q;
    q.u = blockIdx.x;
    seq.first(q);
    uint32_t n = 0;

    if (w == 0) {
        // ---- producer: split x (one bulk copy) and the stacked W rows into slot n % NSLOT
        uint64_t keep, stream;
        asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(keep));
        asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(stream));
        // the row offsets of the current batch (rs) and, loaded while its first chunk goes
        // out, of the next one (rsn)
        int64_t rs[8], rsn[8];
        if (q.valid) load_rows(rsn, rows, q.B, lane);
        while (q.valid && !abort_flag) {
            const int s = (int)(n % NSLOT);
            if (n >= NSLOT && !mbar_wait(su32(&empty[s]), ((n / NSLOT) + 1) & 1, &abort_flag, wait_limit)) break;
            if (q.c == 0) {
#pragma unroll
                for (int i = 0; i < 8; ++i) rs[i] = rsn[i];
            }
            const uint32_t slot = sm0 + (uint32_t)(s * SLOT);
            if (lane == 0)
                bulk_in(slot, xpl + ((int64_t)q.tile * n_xch + q.B.xg0 + q.c) * (A_BYTES / 4), A_BYTES, &full[s], keep);
            fetch_b_rows(slot + OFF_RAW, lane, pool, rs, q.B.nrows, q.c * KCH, q.B.klen, stream);
            asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(su32(&full[s])) : "memory");
            if (q.c == 0 && q.has_next) load_rows(rsn, rows, q.Bn, lane);
            ++n;
            seq.next(q);
        }
        producer_drain(full, n, lane, &abort_flag);
    } else if (w <= 4) {
        // ---- converters: B planes, then each finished batch's T chunks
        const int t = tid - 32, quad = w & 3;
        uint32_t nb = 0;
        int32_t tch[S1_ROWS / 8];   // the batch's T chunks, loaded at its first chunk, stored at its last
        while (q.valid && !warp_aborted(&abort_flag)) {
            const int s = (int)(n % NSLOT);
            if (q.c == 0) {
#pragma unroll
                for (int g = 0; g < S1_ROWS / 8; ++g) tch[g] = 8 * g < q.B.nrows ? tchunks[q.B.row0 / 8 + g] : 0;
            }
            if (!warp_wait(su32(&full[s]), (n / NSLOT) & 1, &abort_flag, wait_limit)) break;
            float *bh = reinterpret_cast<float *>(smraw + s * SLOT + OFF_B), *bl = bh + B_PLANE / 4;
            conv_b_nat(bh, bl, smraw + s * SLOT + OFF_RAW, q.B.nrows, t);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            warp_arrive(su32(&ready[s]), lane);
            if (q.c == q.nch - 1) {
                const int b = (int)(nb & 1);
                if (!warp_wait(su32(&acc_full[b]), (nb >> 1) & 1, &abort_flag, wait_limit)) break;
                fence_after();
                store_t(tmem, (uint32_t)(128 * b), quad, lane, q.B.nrows, tch, tct + (int64_t)q.tile * n_tchunk * TC_T_CHUNK);
                fence_before();
                warp_arrive(su32(&acc_empty[b]), lane);
                ++nb;
            }
            ++n;
            seq.next(q);
        }
    } else if (lane == 0) {
        // ---- MMA issuer: batch j into accumulator j % 2, once its previous contents are stored
        uint32_t nb = 0;
        while (q.valid && !abort_flag) {
            const int s = (int)(n % NSLOT);
            const int b = (int)(nb & 1);
            if (q.c == 0 && nb >= 2 && !mbar_wait(su32(&acc_empty[b]), ((nb >> 1) - 1) & 1, &abort_flag, wait_limit))
                break;
            if (!mbar_wait(su32(&ready[s]), (n / NSLOT) & 1, &abort_flag, wait_limit)) break;
            fence_after();
            issue_chunk(sm0 + (uint32_t)(s * SLOT), tmem + (uint32_t)(128 * b), q.B.nrows, q.c > 0);
            commit(su32(&empty[s]));
            if (q.c == q.nch - 1) {
                commit(su32(&acc_full[b]));
                ++nb;
            }
            ++n;
            seq.next(q);
        }
        commit(su32(&fin));                         // every MMA issued, then a bounded wait before freeing
        mbar_drain(su32(&fin), 0, &abort_flag);
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (abort_flag && status && tid == 0) atomicCAS(status, 0, (int)HM_ERR_TIMEOUT);
    if (w == NWARP - 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(S1_TMEM_COLS));
}

// ---- k_apply_tc: dense products and second stages, by output cluster ---------------

// Position in a CTA's chunk sequence: unit-tile u (units taken in turn with stride
// gridDim.x, tile-major so that one RHS tile's split x stays in L2), operation p of
// the unit, chunk c of nch.  The next unit's record is loaded when a unit begins, the
// next operation's (of this unit or the next) when an operation begins.  Every role
// walks the same sequence.
struct Pos {
    int64_t u;
    int p, c, nch;
    int tile, r0, nr, m8;
    bool valid, has_next;
    TcUnit U, Un;
    TcOp P, Pn;
    __device__ bool last_of_unit() const { return c == nch - 1 && p == U.p1 - 1; }
};

struct Seq {
    const TcUnit *units;
    const TcOp *ops;
    int n_units, nrhs;
    int64_t total;
    __device__ void start(Pos &q) const
    {
        if (q.p + 1 < q.U.p1) q.Pn = ops[q.p + 1];
        else if (q.has_next) q.Pn = ops[q.Un.p0];
        q.c = 0;
        q.nch = (q.P.klen + KCH - 1) / KCH;
    }
    __device__ void enter(Pos &q) const
    {
        q.tile = (int)(q.u / n_units);
        q.r0 = q.tile * TM;
        q.nr = min(TM, nrhs - q.r0);
        q.m8 = (q.U.mlen + 7) & ~7;
        q.p = q.U.p0;
        const int64_t un = q.u + gridDim.x;
        q.has_next = un < total;
        if (q.has_next) q.Un = units[un % n_units];
    }
    __device__ void first(Pos &q) const
    {
        q.valid = q.u < total;
        if (!q.valid) return;
        q.U = units[q.u % n_units];
        enter(q);
        q.P = ops[q.p];
        start(q);
    }
    __device__ void next(Pos &q) const
    {
        if (++q.c < q.nch) return;
        if (++q.p < q.U.p1) {
            q.P = q.Pn;
            start(q);
            return;
        }
        q.u += gridDim.x;
        q.valid = q.has_next;
        if (!q.valid) return;
        q.U = q.Un;
        enter(q);
        q.P = q.Pn;
        start(q);
    }
};

__global__ void __launch_bounds__(TT, 2)
k_apply_tc(const TcUnit *__restrict__ units, int n_units, const TcOp *__restrict__ ops, int64_t n_xch,
           const float *__restrict__ xpl, const float *__restrict__ tct, int64_t n_tchunk,
           const float2 *__restrict__ pool, float2 *__restrict__ z, int64_t ldz, int nrhs, int *status,
           uint32_t wait_limit)
{
    extern __shared__ __align__(1024) unsigned char smraw[];
    __shared__ __align__(8) uint64_t full[NSLOT], ready[NSLOT], empty[NSLOT];
    __shared__ __align__(8) uint64_t acc_full, acc_empty, fin;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    if (tid == 0) init_pipeline(full, ready, empty, &acc_full, &acc_empty, 1, &fin, &abort_flag);
    if (w == NWARP - 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                     "n"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t sm0 = su32(smraw);
    const Seq seq{units, ops, n_units, nrhs, (int64_t)n_units * ((nrhs + TM - 1) / TM)};
    Pos q;
    q.u = blockIdx.x;
    seq.first(q);
    uint32_t n = 0;

    if (w == 0) {
        // ---- producer: the A planes (split x, or a raw T chunk; one bulk copy) and the raw
        // B rows into slot n % NSLOT; the split x is kept in L2 (evict last), T and the
        // block stream are not (evict first)
        uint64_t keep, stream;
        asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(keep));
        asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(stream));
        while (q.valid && !abort_flag) {
            const int s = (int)(n % NSLOT);
            if (n >= NSLOT && !mbar_wait(su32(&empty[s]), ((n / NSLOT) + 1) & 1, &abort_flag, wait_limit)) break;
            const uint32_t slot = sm0 + (uint32_t)(s * SLOT);
            const int k0 = q.c * KCH;
            if (lane == 0) {
                if (q.P.kind == 2)
                    bulk_in(slot, tct + ((int64_t)q.tile * n_tchunk + q.P.t0 + q.c) * TC_T_CHUNK, TC_T_CHUNK * 4,
                            &full[s], stream);
                else
                    bulk_in(slot, xpl + ((int64_t)q.tile * n_xch + q.P.xg0 + q.c) * (A_BYTES / 4), A_BYTES, &full[s],
                            keep);
            }
            const uint32_t raw = slot + OFF_RAW;
            if (q.P.kind == 0) fetch_b_nat(raw, lane, pool + q.P.src, q.P.ld, q.m8, q.P.olen, k0, q.P.klen, stream);
            else fetch_b_tr(raw, lane, pool + q.P.src, q.P.ld, q.m8, q.P.olen, k0, q.P.klen, stream);
            asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(su32(&full[s])) : "memory");
            ++n;
            seq.next(q);
        }
        producer_drain(full, n, lane, &abort_flag);
    } else if (w <= 4) {
        // ---- converters: B planes (and A planes from a raw T chunk), accumulators into z
        const int t = tid - 32, quad = w & 3;
        uint32_t n_u = 0;
        while (q.valid && !warp_aborted(&abort_flag)) {
            const int s = (int)(n % NSLOT);
            if (!warp_wait(su32(&full[s]), (n / NSLOT) & 1, &abort_flag, wait_limit)) break;
            float *slot = reinterpret_cast<float *>(smraw + s * SLOT);
            const unsigned char *raw = smraw + s * SLOT + OFF_RAW;
            float *bh = reinterpret_cast<float *>(smraw + s * SLOT + OFF_B), *bl = bh + B_PLANE / 4;
            if (q.P.kind == 2) conv_a_raw(slot, t);
            if (q.P.kind == 0) conv_b_nat(bh, bl, raw, q.m8, t);
            else conv_b_tr(bh, bl, raw, q.m8, t);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            warp_arrive(su32(&ready[s]), lane);
            if (q.last_of_unit()) {
                if (!warp_wait(su32(&acc_full), n_u & 1, &abort_flag, wait_limit)) break;
                fence_after();
                drain(tmem, quad, lane, q.m8, q.U.mlen, z, ldz, q.r0, q.nr, q.U.out0);
                fence_before();
                warp_arrive(su32(&acc_empty), lane);
                ++n_u;
            }
            ++n;
            seq.next(q);
        }
    } else if (lane == 0) {
        // ---- MMA issuer
        uint32_t n_u = 0;
        bool started = false;
        while (q.valid && !abort_flag) {
            const int s = (int)(n % NSLOT);
            if (!started && n_u > 0 && !mbar_wait(su32(&acc_empty), (n_u - 1) & 1, &abort_flag, wait_limit)) break;
            if (!mbar_wait(su32(&ready[s]), (n / NSLOT) & 1, &abort_flag, wait_limit)) break;
            fence_after();
            issue_chunk(sm0 + (uint32_t)(s * SLOT), tmem, q.m8, started);
            commit(su32(&empty[s]));
            started = true;
            if (q.last_of_unit()) {
                commit(su32(&acc_full));
                ++n_u;
                started = false;
            }
            ++n;
            seq.next(q);
        }
        commit(su32(&fin));                         // every MMA issued, then a bounded wait before freeing
        mbar_drain(su32(&fin), 0, &abort_flag);
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (abort_flag && status && tid == 0) atomicCAS(status, 0, (int)HM_ERR_TIMEOUT);
    if (w == NWARP - 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(TMEM_COLS));
}

// records a status code in the device status word (first error wins)
__global__ void k_set_status(int *status, int code)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) atomicCAS(status, 0, code);
}

} // namespace

size_t tc_xplane_bytes(int64_t n_xch, int nrhs) { return (size_t)A_BYTES * (size_t)n_xch * (size_t)((nrhs + TM - 1) / TM); }

size_t tc_t_bytes(int64_t n_tchunk, int nrhs)
{
    return sizeof(float) * (size_t)TC_T_CHUNK * (size_t)n_tchunk * (size_t)((nrhs + TM - 1) / TM);
}

// tensor-core products of the level's small items (dense and low-rank) for all
// right-hand sides, in tiles of 128: split x, stage 1 of the low-rank products, then
// the dense products and second stages
int launch_apply_tc(hm_matrix h, const LevelList &L, const float2 *x, float2 *z, int nrhs, cudaStream_t s)
{
    if (L.n_tcu == 0 || nrhs <= 0) return 0;
    const bool have_x = h->ws.d_xpl && h->ws.xpl_bytes >= tc_xplane_bytes(L.n_xch, nrhs);
    const bool have_t = L.n_tcb == 0 || (h->ws.d_tct && h->ws.tct_bytes >= tc_t_bytes(L.n_tchunk, nrhs));
    if (!have_x || !have_t) {
        // not reached through the API (the workspaces are sized before every product); the call
        // reports HM_ERR_STATE through the status word instead of returning an incomplete product
        fail(HM_ERR_STATE, "tensor-core product without its split-x or stage-1 workspace");
        k_set_status<<<1, 32, 0, s>>>(h->d_status, (int)HM_ERR_STATE);
        return 1;
    }
    static bool attr = false;
    if (!attr) {   // two CTAs of ~98 KB per SM need the largest shared-memory carveout
        for (const void *k : {(const void *)k_apply_tc, (const void *)k_tc_stage1}) {
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
            cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
        }
        attr = true;
    }
    const int n_tiles = (nrhs + TM - 1) / TM;
    const uint32_t limit = h->tc_wait_limit < 0 ? WAIT_LIMIT : (uint32_t)h->tc_wait_limit;
    k_split_x<<<dim3((unsigned)L.n_xch, (unsigned)n_tiles), TM, 0, s>>>(L.d_xch, L.n_xch, x, h->pN, nrhs, h->ws.d_xpl);
    // two CTAs per SM in both launches: shared memory 2 x ~98 KB of 228 KB, tensor memory
    // 2 x 256 (stage 1) or 2 x 128 columns of 512; the persistent loops are correct for any grid
    const int64_t per_sm = 2 * (int64_t)(h->num_sms > 0 ? h->num_sms : 1);
    if (L.n_tcb > 0) {
        const int64_t g1 = std::min<int64_t>(per_sm, L.n_tcb * (int64_t)n_tiles);
        k_tc_stage1<<<(unsigned)g1, TT, SMEM, s>>>(L.d_tcb, (int)L.n_tcb, L.d_tcr, L.d_tcc, L.n_xch, h->ws.d_xpl,
                                                 h->d_pool32, h->ws.d_tct, L.n_tchunk, n_tiles, h->d_status, limit);
    }
    const int64_t g = std::min<int64_t>(per_sm, L.n_tcu * (int64_t)n_tiles);
    k_apply_tc<<<(unsigned)g, TT, SMEM, s>>>(L.d_tcu, (int)L.n_tcu, L.d_tco, L.n_xch, h->ws.d_xpl, h->ws.d_tct,
                                           L.n_tchunk, h->d_pool32, z, h->pN, nrhs, h->d_status, limit);
    return L.n_tcb > 0 ? 3 : 2;
}

} // namespace hm
