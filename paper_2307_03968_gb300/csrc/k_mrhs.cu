// Block product z += M x for many right-hand sides (arxiv 2307.03968 eqs. 6
// and 8 with the half storage of §III), reading every stored block once per
// chunk of RB right-hand sides instead of once per right-hand side:
//     dense  B (I,J):  Z_I += B X_J,            Z_J += B^T X_I
//     low rank U V:    Z_I += U (V X_J),        Z_J += V^T (U^T X_I)
// with X_I, X_J the row / column cluster panels of the RB right-hand sides.
//
// One CTA of 128 threads per block, persistent over the item list.  The block
// (or both low-rank panels) and the two RHS panels are copied to shared memory
// with cp.async; each small product is then a SIMT GEMM.  In the FP32 product a
// thread owns 4 rows x RB/4 right-hand sides of the output (the two mirrored
// products run side by side on the two halves of the CTA), so every
// shared-memory load of the block feeds RB/4 complex FMAs; in the FP64-class
// residual (compensated Dot2 sums, double-float partial slots) it owns 2 rows x RB/4.
// Block rows have an odd stride (complex elements) so that the rows a warp
// touches fall in distinct banks, and the shared buffers are sized for the
// largest block and rank of the level, so that several CTAs per SM overlap one
// block's copy with another's arithmetic.
// Results go to z with vector atomics, as in the single-RHS kernel.  Blocks
// larger than MRHS_MAX_DIM or of rank above MRHS_MAX_RANK stay on the
// single-RHS kernel.
#include "k_common.cuh"
#include "k_dot2.cuh"

namespace hm {
namespace {

using namespace kc;
constexpr int MT = 128;   // threads per CTA

struct Geom {             // shared-memory geometry of one launch (complex-element units)
    int sld;              // block row stride: dim + 1 (odd)
    int xld;              // RHS panel row stride: RB + 1 (odd)
    int kmax;             // rows reserved for U^T (V follows)
    int srows;            // rows of the block area
    int dim;              // rows of each RHS panel
};

__device__ __forceinline__ void cma(float2 &acc, float2 a, float2 b)   // acc += a b
{
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}

__device__ __forceinline__ void cp_async8(float2 *dst, const float2 *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Wider tiles for the FP32 product: 64 threads per product (tid in [0, 64)), each
// owning 4 rows (or columns) x RB/4 right-hand sides.  Operands are addressed as
// 32-bit offsets into the kernel's shared array (so that every access is a
// shared-space load with an immediate offset), and the RHS panels have an even
// row stride so that a thread's right-hand sides load as 128-bit pairs.
extern __shared__ __align__(16) float2 smf2[];

template <int RB>
__device__ __forceinline__ void ld_x(int xi, float2 (&xv)[RB / 4])
{
#pragma unroll
    for (int q = 0; q < RB / 4; q += 2) {
        const float4 v = *reinterpret_cast<const float4 *>(&smf2[xi + q]);
        xv[q] = make_float2(v.x, v.y);
        xv[q + 1] = make_float2(v.z, v.w);
    }
}

// Y[r][q] (yo >= 0: shared offset of Y, row stride xld) or z (yo < 0) = sum_c S[r][c] X[c][q], rows r < R
template <int RB>
__device__ __forceinline__ void mm4_rows(int tid, int so, int sld, int R, int C, int xo, int xld, int yo, float2 *z,
                                         int64_t ldz, int base, int nr)
{
    constexpr int TQ = RB / 4;
    const int q0 = (tid & 3) * TQ, r = 4 * (tid >> 2);
    if (r >= R) return;
    float2 a[4][TQ];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < TQ; ++q) a[i][q] = make_float2(0.f, 0.f);
    int si[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) si[i] = so + (r + i < R ? r + i : R - 1) * sld;
    int xi = xo + q0;
#pragma unroll 2
    for (int c = 0; c < C; ++c, xi += xld) {
        float2 xv[TQ];
        ld_x<RB>(xi, xv);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 b = smf2[si[i] + c];
#pragma unroll
            for (int q = 0; q < TQ; ++q) cma(a[i][q], b, xv[q]);
        }
    }
    if (yo < 0) {
#pragma unroll
        for (int q = 0; q < TQ; ++q) {
            if (q0 + q >= nr) break;
            float2 *zz = z + (int64_t)(q0 + q) * ldz + base + r;
#pragma unroll
            for (int i = 0; i < 4; i += 2) {
                if (r + i + 1 < R) red2(zz + i, a[i][q], a[i + 1][q]);
                else if (r + i < R) red1(zz + i, a[i][q]);
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (r + i < R)
#pragma unroll
                for (int q = 0; q < TQ; ++q) smf2[yo + (r + i) * xld + q0 + q] = a[i][q];
    }
}

// z[q*ldz + base + c] += sum_r S[r][c] X[r][q], columns c < C, rows r < R
template <int RB>
__device__ __forceinline__ void mm4_cols(int tid, int so, int sld, int R, int C, int xo, int xld, float2 *z,
                                         int64_t ldz, int base, int nr)
{
    constexpr int TQ = RB / 4;
    const int q0 = (tid & 3) * TQ, c = 4 * (tid >> 2);
    if (c >= C) return;
    float2 a[4][TQ];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < TQ; ++q) a[i][q] = make_float2(0.f, 0.f);
    int cc[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) cc[i] = so + (c + i < C ? c + i : C - 1);
    int xi = xo + q0, srow = 0;
#pragma unroll 2
    for (int r = 0; r < R; ++r, xi += xld, srow += sld) {
        float2 xv[TQ];
        ld_x<RB>(xi, xv);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 b = smf2[cc[i] + srow];
#pragma unroll
            for (int q = 0; q < TQ; ++q) cma(a[i][q], b, xv[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < TQ; ++q) {
        if (q0 + q >= nr) break;
        float2 *zz = z + (int64_t)(q0 + q) * ldz + base + c;
#pragma unroll
        for (int i = 0; i < 4; i += 2) {
            if (c + i + 1 < C) red2(zz + i, a[i][q], a[i + 1][q]);
            else if (c + i < C) red1(zz + i, a[i][q]);
        }
    }
}

// rows x cols complex matrix (row stride ld in global memory) -> S (row stride sld);
// warp w copies rows w, w+4, ..., lanes the columns
__device__ __forceinline__ void stage(const float2 *__restrict__ g, int rows, int cols, int ld, float2 *S, int sld)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int r = w; r < rows; r += MT / 32)
        for (int c = lane; c < cols; c += 32) cp_async8(S + r * sld + c, g + (int64_t)r * ld + c);
}

// RHS panel X[i][q] = x[q * ldx + base + i] for i < len, q < RB (zero for q >= nr)
template <int RB>
__device__ __forceinline__ void stage_x(const float2 *__restrict__ x, int64_t ldx, int base, int len, int nr,
                                        float2 *X, int xld)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int q = w; q < RB; q += MT / 32)
        for (int i = lane; i < len; i += 32) {
            if (q < nr) cp_async8(X + i * xld + q, x + (int64_t)q * ldx + base + i);
            else X[i * xld + q] = make_float2(0.f, 0.f);
        }
}

template <int RB>
__global__ void __launch_bounds__(MT)
k_apply_mrhs(const Item *__restrict__ items, int64_t n_items, const float2 *__restrict__ pool,
             const float2 *__restrict__ x, int64_t ldx, float2 *__restrict__ z, int64_t ldz, int nr, Geom gm)
{
    // shared offsets (complex elements): the block, or U^T then V; the RHS panels; V X_J and U^T X_I
    const int oS = 0, oSV = gm.kmax * gm.sld, oXI = gm.srows * gm.sld, oXJ = oXI + gm.dim * gm.xld;
    const int oT = oXJ + gm.dim * gm.xld, oTP = oT + gm.kmax * gm.xld;
    const int tid = threadIdx.x & 63;
    const bool lo = threadIdx.x < 64;
    for (int64_t b = blockIdx.x; b < n_items; b += gridDim.x) {
        const Item it = items[b];
        __syncthreads();                              // the previous item is done with shared memory
        stage_x<RB>(x, ldx, it.row0, it.m, nr, smf2 + oXI, gm.xld);
        stage_x<RB>(x, ldx, it.col0, it.n, nr, smf2 + oXJ, gm.xld);
        if (it.k == 0) {
            stage(pool + it.off, it.m, it.n, (int)even(it.n), smf2 + oS, gm.sld);
            cp_async_wait_all();
            __syncthreads();
            // the two mirrored products run side by side on the two halves of the CTA
            if (lo) mm4_rows<RB>(tid, oS, gm.sld, it.m, it.n, oXJ, gm.xld, -1, z, ldz, it.row0, nr);   // Z_I += B X_J
            else mm4_cols<RB>(tid, oS, gm.sld, it.m, it.n, oXI, gm.xld, z, ldz, it.col0, nr);         // Z_J += B^T X_I
        } else {
            const float2 *UT = pool + it.off;
            const float2 *V = UT + (int64_t)it.k * it.m;
            stage(UT, it.k, it.m, it.m, smf2 + oS, gm.sld);
            stage(V, it.k, it.n, it.n, smf2 + oSV, gm.sld);
            cp_async_wait_all();
            __syncthreads();
            if (lo) mm4_rows<RB>(tid, oSV, gm.sld, it.k, it.n, oXJ, gm.xld, oT, nullptr, 0, 0, nr);    // T  = V X_J
            else mm4_rows<RB>(tid, oS, gm.sld, it.k, it.m, oXI, gm.xld, oTP, nullptr, 0, 0, nr);      // T' = U^T X_I
            __syncthreads();
            if (lo) mm4_cols<RB>(tid, oS, gm.sld, it.k, it.m, oT, gm.xld, z, ldz, it.row0, nr);        // Z_I += U T
            else mm4_cols<RB>(tid, oSV, gm.sld, it.k, it.n, oTP, gm.xld, z, ldz, it.col0, nr);        // Z_J += V^T T'
        }
    }
}

// ------------------------------------------------------------------------------
// FP64-class residual products for many right-hand sides: the same staging, the
// products accumulated in short error-free chains of four terms (biased
// accumulator, k_dot2.cuh) folded into double-float sums, each block's results
// stored in its double-float partial slots (row side: even(m) slots from it.pad, column
// side: even(n) slots after them; no atomics, so the per-leaf FP64 gather that
// follows stays deterministic).  Right-hand side q of the chunk writes
// part[q * pstride + slot].

// slots[q*pstride + r] = sum_c S[r][c] X[c][q] for r < Rs (rows R .. Rs-1 are zero).
// Y given (double-float staging, row stride xld) instead of slots: store there.
template <int RB>
__device__ __forceinline__ void mm_rows_c(const float2 *S, int sld, int R, int Rs, int C, const float2 *X, int xld,
                                          dot2::cdf *Y, dot2::cdf *slots, int64_t pstride, int nr)
{
    using namespace dot2;
    constexpr int TC = RB / 4;
    const int t = threadIdx.x, q0 = (t & 3) * TC;
    const int r = 2 * (t >> 2);
    if (r >= Rs) return;
    cdf a0[TC], a1[TC];
#pragma unroll
    for (int q = 0; q < TC; ++q) { a0[q] = cdf_zero(); a1[q] = cdf_zero(); }
    if (r < R) {
        const float2 *s0 = S + r * sld, *s1 = s0 + sld;
        for (int c0 = 0; c0 < C; c0 += 4) {
            // row r + 1 may be past R (its sums are then discarded), columns past C are zero
            float2 b0[4], b1[4], xv[4][TC];
            float sa0 = 0.f, sa1 = 0.f, mq[TC];
#pragma unroll
            for (int q = 0; q < TC; ++q) mq[q] = 0.f;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool ok = c0 + u < C;
                b0[u] = ok ? s0[c0 + u] : make_float2(0.f, 0.f);
                b1[u] = ok ? s1[c0 + u] : make_float2(0.f, 0.f);
                sa0 = __fadd_rn(sa0, l1(b0[u]));
                sa1 = __fadd_rn(sa1, l1(b1[u]));
#pragma unroll
                for (int q = 0; q < TC; ++q) {
                    xv[u][q] = ok ? X[(c0 + u) * xld + q0 + q] : make_float2(0.f, 0.f);
                    mq[q] = fmaxf(mq[q], linf(xv[u][q]));
                }
            }
#pragma unroll
            for (int q = 0; q < TC; ++q) {
                const float g0 = chain_sigma(sa0, mq[q]), g1 = chain_sigma(sa1, mq[q]);
                cxacc k0, k1;
                cxfirst(k0, g0, b0[0], xv[0][q]);
                cxfirst(k1, g1, b1[0], xv[0][q]);
#pragma unroll
                for (int u = 1; u < 4; ++u) {
                    cxstep(k0, b0[u], xv[u][q]);
                    cxstep(k1, b1[u], xv[u][q]);
                }
                a0[q] = cdf_add(a0[q], cxclose(k0, g0));
                a1[q] = cdf_add(a1[q], cxclose(k1, g1));
            }
        }
    }
    const bool two = r + 1 < R;   // else row r+1 (if < Rs) is a zero pad slot
#pragma unroll
    for (int q = 0; q < TC; ++q) {
        if (Y) {
            Y[r * xld + q0 + q] = a0[q];
            if (r + 1 < Rs) Y[(r + 1) * xld + q0 + q] = two ? a1[q] : cdf_zero();
        } else {
            if (q0 + q >= nr) break;
            dot2::cdf *o = slots + (int64_t)(q0 + q) * pstride + r;
            o[0] = a0[q];
            if (r + 1 < Rs) o[1] = two ? a1[q] : cdf_zero();
        }
    }
}

// slots[q*pstride + c] = sum_r S[r][c] X[r][q] for c < Cs (columns C .. Cs-1 zero);
// X in FP32 (XF) or double-float (XD).
template <int RB>
__device__ __forceinline__ void mm_cols_c(const float2 *S, int sld, int R, int C, int Cs, const float2 *XF,
                                          const dot2::cdf *XD, int xld, dot2::cdf *slots, int64_t pstride, int nr)
{
    using namespace dot2;
    constexpr int TC = RB / 4;
    const int t = threadIdx.x, q0 = (t & 3) * TC;
    const int c = 2 * (t >> 2);
    if (c >= Cs) return;
    cdf a0[TC], a1[TC];
#pragma unroll
    for (int q = 0; q < TC; ++q) { a0[q] = cdf_zero(); a1[q] = cdf_zero(); }
    if (c < C) {
        const float2 *sc = S + c;
        for (int r0 = 0; r0 < R; r0 += 4) {
            // column c + 1 may be past C (its sums are then discarded), rows past R are zero
            float2 b0[4], b1[4];
            float sa0 = 0.f, sa1 = 0.f, mq[TC];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool ok = r0 + u < R;
                b0[u] = ok ? sc[(r0 + u) * sld] : make_float2(0.f, 0.f);
                b1[u] = ok ? sc[(r0 + u) * sld + 1] : make_float2(0.f, 0.f);
                sa0 = __fadd_rn(sa0, l1(b0[u]));
                sa1 = __fadd_rn(sa1, l1(b1[u]));
            }
#pragma unroll
            for (int q = 0; q < TC; ++q) mq[q] = 0.f;
            if (XD) {
                // the chain bound uses the leading parts; the trailing parts go to the remainders
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (r0 + u < R)
#pragma unroll
                        for (int q = 0; q < TC; ++q) {
                            const cdf v = XD[(r0 + u) * xld + q0 + q];
                            mq[q] = fmaxf(mq[q], fmaxf(fabsf(v.re.hi), fabsf(v.im.hi)));
                        }
#pragma unroll
                for (int q = 0; q < TC; ++q) {
                    const float g0 = chain_sigma(sa0, mq[q]), g1 = chain_sigma(sa1, mq[q]);
                    cxacc k0, k1;
                    const cdf v0 = XD[r0 * xld + q0 + q];
                    cxfirst_df(k0, g0, b0[0], v0);
                    cxfirst_df(k1, g1, b1[0], v0);
#pragma unroll
                    for (int u = 1; u < 4; ++u) {
                        const cdf v = r0 + u < R ? XD[(r0 + u) * xld + q0 + q] : cdf_zero();
                        cxstep_df(k0, b0[u], v);
                        cxstep_df(k1, b1[u], v);
                    }
                    a0[q] = cdf_add(a0[q], cxclose(k0, g0));
                    a1[q] = cdf_add(a1[q], cxclose(k1, g1));
                }
            } else {
                float2 xv[4][TC];
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int q = 0; q < TC; ++q) {
                        xv[u][q] = r0 + u < R ? XF[(r0 + u) * xld + q0 + q] : make_float2(0.f, 0.f);
                        mq[q] = fmaxf(mq[q], linf(xv[u][q]));
                    }
#pragma unroll
                for (int q = 0; q < TC; ++q) {
                    const float g0 = chain_sigma(sa0, mq[q]), g1 = chain_sigma(sa1, mq[q]);
                    cxacc k0, k1;
                    cxfirst(k0, g0, b0[0], xv[0][q]);
                    cxfirst(k1, g1, b1[0], xv[0][q]);
#pragma unroll
                    for (int u = 1; u < 4; ++u) {
                        cxstep(k0, b0[u], xv[u][q]);
                        cxstep(k1, b1[u], xv[u][q]);
                    }
                    a0[q] = cdf_add(a0[q], cxclose(k0, g0));
                    a1[q] = cdf_add(a1[q], cxclose(k1, g1));
                }
            }
        }
    }
    const bool two = c + 1 < C;
#pragma unroll
    for (int q = 0; q < TC; ++q) {
        if (q0 + q >= nr) break;
        dot2::cdf *o = slots + (int64_t)(q0 + q) * pstride + c;
        o[0] = a0[q];
        if (c + 1 < Cs) o[1] = two ? a1[q] : cdf_zero();
    }
}

template <int RB>
__global__ void __launch_bounds__(MT)
k_residual_mrhs(const Item *__restrict__ items, int64_t n_items, const float2 *__restrict__ pool,
                const float2 *__restrict__ x, int64_t ldx, dot2::cdf *__restrict__ part, int64_t pstride, int nr,
                Geom gm)
{
    using dot2::cdf;
    float2 *S = smf2;
    float2 *SV = S + gm.kmax * gm.sld;
    float2 *XI = S + gm.srows * gm.sld;
    float2 *XJ = XI + gm.dim * gm.xld;
    cdf *T = reinterpret_cast<cdf *>(XJ + gm.dim * gm.xld);    // kmax x xld (double-float)
    cdf *TP = T + gm.kmax * gm.xld;
    for (int64_t b = blockIdx.x; b < n_items; b += gridDim.x) {
        const Item it = items[b];
        __syncthreads();
        stage_x<RB>(x, ldx, it.row0, it.m, nr, XI, gm.xld);
        stage_x<RB>(x, ldx, it.col0, it.n, nr, XJ, gm.xld);
        dot2::cdf *rows = part + it.pad;
        if (it.k == 0) {
            const int em = (int)even(it.m), en = (int)even(it.n);
            stage(pool + it.off, it.m, it.n, en, S, gm.sld);
            cp_async_wait_all();
            __syncthreads();
            mm_rows_c<RB>(S, gm.sld, it.m, em, it.n, XJ, gm.xld, nullptr, rows, pstride, nr);          // B x_J
            mm_cols_c<RB>(S, gm.sld, it.m, it.n, en, XI, nullptr, gm.xld, rows + em, pstride, nr);    // B^T x_I
        } else {
            const float2 *UT = pool + it.off;
            const float2 *V = UT + (int64_t)it.k * it.m;
            stage(UT, it.k, it.m, it.m, S, gm.sld);
            stage(V, it.k, it.n, it.n, SV, gm.sld);
            cp_async_wait_all();
            __syncthreads();
            mm_rows_c<RB>(SV, gm.sld, it.k, it.k, it.n, XJ, gm.xld, T, nullptr, 0, nr);               // T  = V x_J
            mm_rows_c<RB>(S, gm.sld, it.k, it.k, it.m, XI, gm.xld, TP, nullptr, 0, nr);               // T' = U^T x_I
            __syncthreads();
            mm_cols_c<RB>(S, gm.sld, it.k, it.m, it.m, nullptr, T, gm.xld, rows, pstride, nr);        // U T
            mm_cols_c<RB>(SV, gm.sld, it.k, it.n, it.n, nullptr, TP, gm.xld, rows + it.m, pstride, nr); // V^T T'
        }
    }
}

Geom level_geom(const LevelList &L, int xld, size_t t_elem, size_t &bytes)
{
    Geom gm;
    gm.dim = L.small_dim;                              // even, <= MRHS_MAX_DIM
    gm.sld = gm.dim + 1;
    gm.xld = xld;
    gm.kmax = L.small_rank;
    gm.srows = std::max(gm.dim, 2 * gm.kmax) + 1;     // one spare row: a thread's second row may be read past the end
    if ((gm.srows * gm.sld) & 1) ++gm.srows;           // keep the RHS panels that follow 16-byte aligned
    bytes = sizeof(float2) * ((size_t)gm.srows * gm.sld + 2 * (size_t)gm.dim * gm.xld) +
            t_elem * 2 * (size_t)std::max(gm.kmax, 1) * gm.xld;
    return gm;
}

template <int RB>
void launch_resid_rb(hm_matrix h, const LevelList &L, const float2 *x, dot2::cdf *part, int64_t pstride, int nrhs,
                     cudaStream_t s)
{
    size_t sm = 0;
    const Geom gm = level_geom(L, RB + 1, sizeof(dot2::cdf), sm);
    static size_t attr = 0;
    if (sm > attr) {
        cudaFuncSetAttribute(k_residual_mrhs<RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        cudaFuncSetAttribute(k_residual_mrhs<RB>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);   // several CTAs per SM
        attr = sm;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_residual_mrhs<RB>, MT, sm);
    if (per_sm < 1) per_sm = 1;
    int64_t g = (int64_t)per_sm * (h->num_sms > 0 ? h->num_sms : 1);
    if (g > L.n_small) g = L.n_small;
    for (int r0 = 0; r0 < nrhs; r0 += RB) {
        const int nr = nrhs - r0 < RB ? nrhs - r0 : RB;
        k_residual_mrhs<RB><<<(unsigned)g, MT, sm, s>>>(L.d_small, L.n_small, h->d_pool32, x + (int64_t)r0 * h->pN,
                                                        h->pN, part + (int64_t)r0 * pstride, pstride, nr, gm);
    }
}

template <int RB>
void launch_rb(hm_matrix h, const LevelList &L, const Item *items, int64_t n_items, const float2 *x, float2 *z,
               int nrhs, cudaStream_t s)
{
    size_t sm = 0;
    const Geom gm = level_geom(L, RB + 2, sizeof(float2), sm);   // even panel stride: 16-byte aligned rows
    static size_t attr = 0;                                      // largest dynamic size enabled so far
    if (sm > attr) {
        cudaFuncSetAttribute(k_apply_mrhs<RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        cudaFuncSetAttribute(k_apply_mrhs<RB>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);   // several CTAs per SM
        attr = sm;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_apply_mrhs<RB>, MT, sm);
    if (per_sm < 1) per_sm = 1;
    int64_t g = (int64_t)per_sm * (h->num_sms > 0 ? h->num_sms : 1);
    if (g > n_items) g = n_items;
    for (int r0 = 0; r0 < nrhs; r0 += RB) {
        const int nr = nrhs - r0 < RB ? nrhs - r0 : RB;
        k_apply_mrhs<RB><<<(unsigned)g, MT, sm, s>>>(items, n_items, h->d_pool32, x + (int64_t)r0 * h->pN,
                                                     h->pN, z + (int64_t)r0 * h->pN, h->pN, nr, gm);
    }
}

} // namespace

void launch_apply_items_mrhs(hm_matrix h, const LevelList &L, const float2 *x, float2 *z, int nrhs, int rb,
                             cudaStream_t s)
{
    launch_apply_list_mrhs(h, L, L.d_small, L.n_small, x, z, nrhs, rb, s);
}

void launch_apply_list_mrhs(hm_matrix h, const LevelList &L, const Item *items, int64_t n_items, const float2 *x,
                            float2 *z, int nrhs, int rb, cudaStream_t s)
{
    if (n_items == 0 || nrhs <= 0) return;
    if (rb <= 8) launch_rb<8>(h, L, items, n_items, x, z, nrhs, s);
    else if (rb <= 16) launch_rb<16>(h, L, items, n_items, x, z, nrhs, s);
    else launch_rb<32>(h, L, items, n_items, x, z, nrhs, s);
}

} // namespace hm

namespace hm {

void launch_apply_items_partials_mrhs(hm_matrix h, const LevelList &L, const float2 *x, dot2::cdf *part,
                                      int64_t pstride, int nrhs, cudaStream_t s, int rb)
{
    if (L.n_small == 0 || nrhs <= 0) return;
    if (rb < 0) rb = nrhs <= 8 ? 8 : 16;
    if (rb <= 8) launch_resid_rb<8>(h, L, x, part, pstride, nrhs, s);
    else launch_resid_rb<16>(h, L, x, part, pstride, nrhs, s);
}

} // namespace hm
