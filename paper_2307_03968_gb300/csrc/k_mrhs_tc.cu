// Tensor-core block product for many right-hand sides (arxiv 2307.03968 eq. 6,
// the dense near blocks, with the half storage of §III):
//     Z_I += B X_J,   Z_J += B^T X_I        (B complex m x n, m, n <= 64)
// for a chunk of RB right-hand sides, on the 5th-generation tensor cores
// (tcgen05.mma kind::tf32, accumulators in tensor memory).
//
// Complex products as real GEMMs.  With B = Br + i Bi and X = Xr + i Xi, the
// direct product is D = A B' with
//     A  (64 x 2n8):   [Br | Bi]                       (rows i, K index = plane, j)
//     B' (2n8 x 2RB):  column 2q   = [ Xr[:,q] ; -Xi[:,q] ]
//                      column 2q+1 = [ Xi[:,q] ;  Xr[:,q] ]
// so that D[i][2q] = Re Z_I[i][q] and D[i][2q+1] = Im Z_I[i][q] (n8 = n rounded up
// to 8, zero padded).  The mirror product uses the transposed planes [Br^T | Bi^T]
// and the panel of X_I.  Both operands are in shared memory in the K-major
// layout without swizzle: 8-row x 16-byte core matrices, K-adjacent cores 128 B
// apart (leading byte offset), 8-row groups KCmax * 128 B apart (stride offset).
//
// Precision (3xTF32): every FP32 operand a is split as a = hi + lo, hi = a rounded
// to TF32 (10 mantissa bits), lo = a - hi (exact); each K step accumulates
// hi*hi + hi*lo + lo*hi in FP32 in tensor memory, which keeps the product within
// a few FP32 ulps (the dropped lo*lo term and the TF32 rounding of lo are ~2^-22).
//
// One CTA of 128 threads per block, persistent; thread 0 issues the MMAs, whose
// completion arrives on an mbarrier; the accumulator (M = 64) sits in tensor-memory
// lanes 32w .. 32w+15 of warp w, rows 16w .. 16w+15.  Every wait is bounded: on
// timeout the kernel records HM_ERR_TIMEOUT in the status word, frees its tensor
// memory and returns.
#include "k_common.cuh"

namespace hm {
namespace {

using namespace kc;
constexpr int TT = 128;                  // threads per CTA
constexpr int TM = 64;                   // MMA M (rows of A)
constexpr uint32_t WAIT_LIMIT = 1u << 24;

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void split_tf32(float a, float &hi, float &lo)
{
    uint32_t h;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(a));
    hi = __uint_as_float(h);
    lo = __fsub_rn(a, hi);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t sbo)
{
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)(128u >> 4) << 16;              // leading byte offset: K-adjacent core matrices
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;    // stride byte offset: 8-row groups
    d |= (uint64_t)1 << 46;                        // descriptor version (tcgen05)
    return d;                                      // no swizzle, base offset 0
}

// float offset of element (row r, K index k) in a K-major operand with kc K-cores per row
__device__ __forceinline__ int koff(int r, int k, int kc)
{
    return (((r >> 3) * kc + (k >> 2)) << 5) + ((r & 7) << 2) + (k & 3);
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity)
{
    for (uint32_t it = 0; it < WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

// RHS operand B' for a panel of `len` unknowns at `base` (K = 2*len8): rows nn = 2q + s
template <int RB>
__device__ __forceinline__ void stage_rhs(const float2 *__restrict__ x, int64_t ldx, int base, int len, int len8,
                                          int nr, float *Bhi, float *Blo, int kc)
{
    constexpr int NR = 2 * RB;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int rr = lane >> 2, kk = lane & 3;
    const int kcores = (2 * len8) >> 2;
    const int units = (NR >> 3) * kcores;
    for (int u = w; u < units; u += TT / 32) {
        const int gn = u / kcores, c = u - gn * kcores;
        const int nn = 8 * gn + rr, k = 4 * c + kk;
        const int q = nn >> 1, s = nn & 1;
        const int half = k >= len8, j = k - half * len8;
        float v = 0.f;
        if (q < nr && j < len) {
            const float2 xv = x[(int64_t)q * ldx + base + j];
            v = half == 0 ? (s == 0 ? xv.x : xv.y) : (s == 0 ? -xv.y : xv.x);
        }
        float h, l;
        split_tf32(v, h, l);
        const int o = ((gn * kc + c) << 5) + lane;   // == koff(nn, k, kc)
        Bhi[o] = h;
        Blo[o] = l;
    }
}

// issue the 3xTF32 MMAs of one product (K = 2*len8) into tensor-memory columns at tmem
template <int RB>
__device__ __forceinline__ void issue_mma(uint32_t tmem, uint32_t aHi, uint32_t aLo, uint32_t bHi, uint32_t bLo,
                                          int len8, uint32_t sbo_a, uint32_t sbo_b, uint32_t mbar)
{
    constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)((2 * RB) >> 3) << 17) |
                               ((uint32_t)(TM >> 4) << 24);
    const int steps = (2 * len8) >> 3;
    for (int st = 0; st < steps; ++st) {
        const uint32_t ko = (uint32_t)st * 256u;     // two K-cores of 128 B per K step of 8
        const uint64_t ah = smem_desc(aHi + ko, sbo_a), al = smem_desc(aLo + ko, sbo_a);
        const uint64_t bh = smem_desc(bHi + ko, sbo_b), bl = smem_desc(bLo + ko, sbo_b);
        const uint32_t acc0 = st > 0 ? 1u : 0u;
        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                     "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem), "l"(ah), "l"(bh),
                     "r"(IDESC), "r"(acc0));
        asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;\n" ::"r"(tmem), "l"(ah), "l"(bl),
                     "r"(IDESC));
        asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;\n" ::"r"(tmem), "l"(al), "l"(bh),
                     "r"(IDESC));
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

// add the accumulator (rows < rows_valid) into z: row r, right-hand side q at z[q*ldz + base + r]
template <int RB>
__device__ __forceinline__ void drain(uint32_t taddr, int rows_valid, float2 *z, int64_t ldz, int base, int nr)
{
    static_assert(RB == 16, "one 32-column load per warp");
    uint32_t v[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                   "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                   "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                   "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int row = 16 * w + lane;
    if (lane < 16 && row < rows_valid) {
#pragma unroll
        for (int q = 0; q < RB; ++q)
            if (q < nr) red1(z + (int64_t)q * ldz + base + row, make_float2(__uint_as_float(v[2 * q]),
                                                                              __uint_as_float(v[2 * q + 1])));
    }
}

template <int RB>
__global__ void __launch_bounds__(TT)
k_apply_mrhs_tc(const Item *__restrict__ items, int64_t n_items, const float2 *__restrict__ pool,
                const float2 *__restrict__ x, int64_t ldx, float2 *__restrict__ z, int64_t ldz, int nr, int kcmax,
                int *status)
{
    constexpr int NR = 2 * RB;
    constexpr int MAXU = (TM / 8) * (TM / 4) / (TT / 32);   // block units per warp (8 x 4 elements each)
    extern __shared__ __align__(1024) float smtc[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int kd = 4 * kcmax;                                // K floats per operand row
    float *Ahi = smtc, *Alo = Ahi + TM * kd, *Bhi = Alo + TM * kd, *Blo = Bhi + NR * kd;
    const uint32_t sbo_a = (uint32_t)kcmax * 128u, sbo_b = sbo_a;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (int i = tid; i < (2 * TM + 2 * NR) * kd; i += TT) smtc[i] = 0.f;   // pads stay finite
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (w == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                     "n"(2 * NR));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    const uint32_t mb = su32(&mbar);
    const uint32_t aHi = su32(Ahi), aLo = su32(Alo), bHi = su32(Bhi), bLo = su32(Blo);
    const int rr = lane >> 2, kk = lane & 3;
    uint32_t phase = 0;
    bool ok = true;
    for (int64_t b = blockIdx.x; b < n_items && ok; b += gridDim.x) {
        const Item it = items[b];
        const int m = it.m, n = it.n, m8 = (m + 7) & ~7, n8 = (n + 7) & ~7;
        const int ld = (int)even(n);
        const float2 *B = pool + it.off;
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();                                     // previous item: tensor memory read, shared free
        asm volatile("tcgen05.fence::after_thread_sync;");
        // ---- block -> registers and the direct operand [Br | Bi]
        const int gm = m8 >> 3, cn = n8 >> 2, units = gm * cn;
        float2 hold[MAXU];
#pragma unroll
        for (int t = 0; t < MAXU; ++t) {
            const int u = w + t * (TT / 32);
            hold[t] = make_float2(0.f, 0.f);
            if (u < units) {
                const int g = u / cn, c = u - g * cn;
                const int i = 8 * g + rr, j = 4 * c + kk;
                if (i < m && j < n) hold[t] = __ldcs(B + (int64_t)i * ld + j);
                float h, l;
                split_tf32(hold[t].x, h, l);
                int o = ((g * kcmax + c) << 5) + lane;        // (row i, K index j)
                Ahi[o] = h; Alo[o] = l;
                split_tf32(hold[t].y, h, l);
                o = ((g * kcmax + c + (n8 >> 2)) << 5) + lane; // (row i, K index n8 + j)
                Ahi[o] = h; Alo[o] = l;
            }
        }
        stage_rhs<RB>(x, ldx, it.col0, n, n8, nr, Bhi, Blo, kcmax);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0) issue_mma<RB>(tmem, aHi, aLo, bHi, bLo, n8, sbo_a, sbo_b, mb);
        if (!__syncthreads_and(mbar_wait(mb, phase))) { ok = false; break; }   // uniform decision
        phase ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;");
        drain<RB>(tmem + ((uint32_t)(32 * w) << 16), m, z, ldz, it.row0, nr);
        // ---- the mirror operand [Br^T | Bi^T] from the held block, and the panel of X_I
        const int kcm = m8 >> 2;
#pragma unroll
        for (int t = 0; t < MAXU; ++t) {
            const int u = w + t * (TT / 32);
            if (u < units) {
                const int g = u / cn, c = u - g * cn;
                const int i = 8 * g + rr, j = 4 * c + kk;
                float h, l;
                split_tf32(hold[t].x, h, l);
                int o = koff(j, i, kcmax);                    // (row j, K index i)
                Ahi[o] = h; Alo[o] = l;
                split_tf32(hold[t].y, h, l);
                o = koff(j, i + 4 * kcm, kcmax);              // (row j, K index m8 + i)
                Ahi[o] = h; Alo[o] = l;
            }
        }
        stage_rhs<RB>(x, ldx, it.row0, m, m8, nr, Bhi, Blo, kcmax);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0) issue_mma<RB>(tmem + NR, aHi, aLo, bHi, bLo, m8, sbo_a, sbo_b, mb);
        if (!__syncthreads_and(mbar_wait(mb, phase))) { ok = false; break; }
        phase ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;");
        drain<RB>(tmem + ((uint32_t)(32 * w) << 16) + NR, n, z, ldz, it.col0, nr);
    }
    if (!ok && status) atomicCAS(status, 0, (int)HM_ERR_TIMEOUT);
    if (!ok) {   // an MMA may still be in flight: wait (bounded) for it before freeing tensor memory
        mbar_wait(mb, phase);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(2 * NR));
}

} // namespace

// dense items with m, n <= 64: tensor-core products, RHS in chunks of 16
void launch_apply_dense_tc(hm_matrix h, const Item *items, int64_t n_items, int dim, const float2 *x, float2 *z,
                           int nrhs, cudaStream_t s)
{
    constexpr int RB = 16;
    if (n_items == 0 || nrhs <= 0) return;
    const int kcmax = 2 * ((dim + 7) & ~7) / 4;          // K-cores per operand row: 2 * round8(dim) floats
    const size_t sm = sizeof(float) * (size_t)(2 * TM + 4 * RB) * (size_t)(4 * kcmax);
    static size_t attr = 0;
    if (sm > attr) {
        cudaFuncSetAttribute(k_apply_mrhs_tc<RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        attr = sm;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_apply_mrhs_tc<RB>, TT, sm) != cudaSuccess) {
        cudaGetLastError();
        per_sm = (int)((227u << 10) / (sm + (2u << 10)));  // shared memory bound, with the static part
    }
    if (per_sm < 1) per_sm = 1;
    if (per_sm > 4) per_sm = 4;                           // tensor memory: 4 x 64 columns of 512
    int64_t g = (int64_t)per_sm * (h->num_sms > 0 ? h->num_sms : 1);
    if (g > n_items) g = n_items;
    for (int r0 = 0; r0 < nrhs; r0 += RB) {
        const int nr = nrhs - r0 < RB ? nrhs - r0 : RB;
        k_apply_mrhs_tc<RB><<<(unsigned)g, TT, sm, s>>>(items, n_items, h->d_pool32, x + (int64_t)r0 * h->pN, h->pN,
                                                        z + (int64_t)r0 * h->pN, h->pN, nr, kcmax, h->d_status);
    }
}

} // namespace hm
