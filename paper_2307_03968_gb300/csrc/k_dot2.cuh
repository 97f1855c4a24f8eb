// Error-free FP32 arithmetic for the FP64-class residual products
// (shared by the single- and multi-right-hand-side residual kernels).
#pragma once

#include "k_common.cuh"

namespace hm {
namespace dot2 {

using kc::FULL;

// ---------------------------------------------------------------------------
// FP64-class products for the refinement residual (complex64 data).
//
// GB300 runs FP64 at a small fraction of its FP32 rate, so a full-operator pass
// in FP64 arithmetic costs many times its HBM time.  The residual products
// therefore use error-free transformations in FP32 (Ogita, Rump & Oishi,
// "Accurate sum and dot product", SIAM J. Sci. Comput. 2005, algorithm Dot2):
// every product a*b is split exactly into p + e with e = fma(a, b, -p), and
// every sum is compensated (Knuth's TwoSum), so the sums are as accurate as if
// computed in twice the working precision.  Dot2 serves the leaf gathers
// (D x) and the low-rank blocks larger than 64 x 64; the block products of
// the residual kernels use the cheaper biased chains further down, folded into
// double-float sums (df_add).  df, cdf: hm_internal.h

// The error-free transformations below must not be contracted into FMAs or
// reassociated, so every operation is an explicitly rounded intrinsic.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// acc += a * b  (Dot2 step): p + ep == a * b exactly
__device__ __forceinline__ void dot2(df &acc, float a, float b)
{
    const float p = __fmul_rn(a, b);
    const float ep = __fmaf_rn(a, b, -p);
    float s, q;
    two_sum(acc.hi, p, s, q);
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(q, ep));
}
// acc += a * b for complex a (FP32) and b (FP32)
__device__ __forceinline__ void cdot2(cdf &acc, float2 a, float2 b)
{
    dot2(acc.re, a.x, b.x);
    dot2(acc.re, -a.y, b.y);
    dot2(acc.im, a.x, b.y);
    dot2(acc.im, a.y, b.x);
}
// acc += a * (bh + bl) for complex a and a double-float complex b
__device__ __forceinline__ void cdot2_df(cdf &acc, float2 a, const cdf &b)
{
    cdot2(acc, a, make_float2(b.re.hi, b.im.hi));
    acc.re.lo += a.x * b.re.lo - a.y * b.im.lo;
    acc.im.lo += a.x * b.im.lo + a.y * b.re.lo;
}
// a + b for double-float numbers: the leading parts summed exactly (TwoSum), the
// error and trailing parts added into the trailing part.  The result is not
// renormalised: its trailing part stays within a few ulps of the leading one over
// the short sums it is used in (lane reductions), and hi + lo converts to FP64
// exactly as it stands.
__device__ __forceinline__ df df_add(df a, df b)
{
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    return {s, __fadd_rn(e, __fadd_rn(a.lo, b.lo))};
}
__device__ __forceinline__ cdf cdf_add(const cdf &a, const cdf &b) { return {df_add(a.re, b.re), df_add(a.im, b.im)}; }

// ---------------------------------------------------------------------------
// Short error-free chains with a biased accumulator (four operations per real
// product against ten for Dot2).
//
// For a short sum s = sum_k a_k b_k with sum_k |a_k b_k| < sigma / 2, sigma a
// power of two, the accumulator tau starts at sigma and stays within
// [1/2, 3/2] sigma, where every float is a multiple of 2^-24 sigma.  Each step
//   tau' = fma(a, b, tau)     the exact product rounded once onto tau's grid,
//   q    = tau' - tau         exact (a multiple of 2^-24 sigma, |q| <= sigma / 2),
//   r   += fma(a, b, -q)      the product's remainder below the grid,
// leaves s = (tau - sigma) + r with tau - sigma exact; only r, whose terms are
// at most ulp(sigma) ~ 2^-23 sigma, is rounded.  The grid extraction is the
// ExtractScalar step of Rump, Ogita & Oishi ("Accurate floating-point
// summation part I: faithful rounding", SIAM J. Sci. Comput. 31(1), 2008),
// applied here to each exact product through the FMA.  sigma comes from a
// bound of the chain's own terms (sum of |a|_1 times max |b|_inf), so the
// grid follows the data.  Each remainder is rounded once, on a grid of about
// 2^-23 sigma with sigma 5-15 times the terms' size: over chains of 4-8 real
// terms the error is typically 1.5-6 units of 2^-48 of sum |a_k b_k| and stays
// within 2^-39, against a few units for Dot2 (an exact model of both is in the
// tests).  That is 10^4 times and more below FP32 summation, and below the
// complex64 rounding of the residual these sums feed.
struct xacc { float tau, r; };
struct cxacc { xacc re, im; };

// the least power of two >= v for finite v >= 0 (0 for 0, 2^-126 for subnormals)
__device__ __forceinline__ float pow2_ceil(float v)
{
    return __uint_as_float((__float_as_uint(v) + 0x007FFFFFu) & 0xFF800000u);
}
__device__ __forceinline__ float l1(float2 a) { return __fadd_rn(fabsf(a.x), fabsf(a.y)); }
__device__ __forceinline__ float linf(float2 a) { return fmaxf(fabsf(a.x), fabsf(a.y)); }
// sigma for a chain of complex products a_k b_k with sum_k |a_k|_1 = sa and
// max_k |b_k|_inf = mb (each real part and each imaginary part sums at most
// sa * mb): twice the bound, raised by 2^-17 against the rounding of sa, of the
// two products and of the grid parts q, so that tau never drops below sigma / 2
constexpr float CHAIN_MARGIN = 2.0f + 0x1p-16f;
__device__ __forceinline__ float chain_sigma(float sa, float mb) { return pow2_ceil(CHAIN_MARGIN * sa * mb); }

__device__ __forceinline__ void xfirst(xacc &c, float sigma, float a, float b)
{
    c.tau = __fmaf_rn(a, b, sigma);
    c.r = __fmaf_rn(a, b, -__fsub_rn(c.tau, sigma));
}
__device__ __forceinline__ void xstep(xacc &c, float a, float b)
{
    const float t2 = __fmaf_rn(a, b, c.tau);
    c.r = __fadd_rn(c.r, __fmaf_rn(a, b, -__fsub_rn(t2, c.tau)));
    c.tau = t2;
}
// c = a * b (the chain's first complex term)
__device__ __forceinline__ void cxfirst(cxacc &c, float sigma, float2 a, float2 b)
{
    xfirst(c.re, sigma, a.x, b.x);
    xstep(c.re, -a.y, b.y);
    xfirst(c.im, sigma, a.x, b.y);
    xstep(c.im, a.y, b.x);
}
// c += a * b
__device__ __forceinline__ void cxstep(cxacc &c, float2 a, float2 b)
{
    xstep(c.re, a.x, b.x);
    xstep(c.re, -a.y, b.y);
    xstep(c.im, a.x, b.y);
    xstep(c.im, a.y, b.x);
}
// c += a * (b.hi + b.lo) for a double-float b: the leading part through the
// chain (its bound uses |b.hi|), the trailing part (2^-24 of it) into r
__device__ __forceinline__ void cx_lo(cxacc &c, float2 a, const cdf &b)
{
    c.re.r = __fmaf_rn(a.x, b.re.lo, c.re.r);
    c.re.r = __fmaf_rn(-a.y, b.im.lo, c.re.r);
    c.im.r = __fmaf_rn(a.x, b.im.lo, c.im.r);
    c.im.r = __fmaf_rn(a.y, b.re.lo, c.im.r);
}
__device__ __forceinline__ void cxfirst_df(cxacc &c, float sigma, float2 a, const cdf &b)
{
    cxfirst(c, sigma, a, make_float2(b.re.hi, b.im.hi));
    cx_lo(c, a, b);
}
__device__ __forceinline__ void cxstep_df(cxacc &c, float2 a, const cdf &b)
{
    cxstep(c, a, make_float2(b.re.hi, b.im.hi));
    cx_lo(c, a, b);
}
// the chain's sum as a double-float: the exact grid part and the remainder
__device__ __forceinline__ cdf cxclose(const cxacc &c, float sigma)
{
    return {{__fsub_rn(c.re.tau, sigma), c.re.r}, {__fsub_rn(c.im.tau, sigma), c.im.r}};
}
// ---------------------------------------------------------------------------
// Chains on a common grid.  When every chain that feeds one output sum takes the
// same sigma, and sigma bounds the whole output sum (all its terms, whichever
// lane or chain holds them), the chains' grid parts tau - sigma are multiples of
// 2^-24 sigma and so is every partial sum of them, of magnitude at most sigma / 2:
// the grid parts of the lanes then add EXACTLY in plain FP32, and only the
// remainders r are rounded.  sigma comes from a bound of the block (its largest
// row or column 1-norm, precomputed per block in FP64 and rounded up) times the
// largest input component.  A chain of L real steps drifts from the exact grid
// sum by at most L 2^-24 sigma, so the margin 2 + 2^-10 keeps tau within
// [1/2, 3/2] sigma for output sums of up to 2^12 real steps per part (2,048
// complex products).  The error of a sum is then a few units of 2^-48 sigma per
// chain step, sigma being at most 4.01 times the bound of the sum.
constexpr float GRID_MARGIN = 2.0f + 0x1p-10f;
__device__ __forceinline__ float grid_sigma(float bound, float mb) { return pow2_ceil(GRID_MARGIN * bound * mb); }
__device__ __forceinline__ void cx_start(cxacc &c, float sigma) { c = {{sigma, 0.f}, {sigma, 0.f}}; }
// one step of a transposing warp reduction: of the pair (v[j], v[j + H]) this lane
// keeps the upper one when its lane bit `mask` is set, and adds the partner lane's
// copy of it; after the steps for masks M, M/2, ..., 1 over V values, each lane
// holds V / (2M) sums over the 2M lanes, the value index bits above taken from the
// lane bits (exact for the grid parts of a common grid)
template <int H>
__device__ __forceinline__ void xreduce_step(float *v, int lane, int mask)
{
    const bool up = (lane & mask) != 0;
#pragma unroll
    for (int j = 0; j < H; ++j) {
        const float send = up ? v[j] : v[j + H];
        const float keep = up ? v[j + H] : v[j];
        v[j] = __fadd_rn(keep, __shfl_xor_sync(FULL, send, mask));
    }
}
__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) v = fmaxf(v, __shfl_xor_sync(FULL, v, s));
    return v;
}

// 1-norm bounds of a row-major rows x cols array (row stride ld): the largest row
// sum and the largest column sum of |re| + |im|, in FP64 (warp-wide results)
__device__ __forceinline__ void l1_bounds(const float2 *__restrict__ A, int rows, int cols, int ld, double &rmax,
                                          double &cmax, int lane)
{
    rmax = 0.0;
    for (int i = 0; i < rows; ++i) {
        double v = 0.0;
        for (int j = lane; j < cols; j += 32) {
            const float2 a = A[(int64_t)i * ld + j];
            v += (double)fabsf(a.x) + (double)fabsf(a.y);
        }
        for (int s = 16; s >= 1; s >>= 1) v += __shfl_xor_sync(FULL, v, s);
        rmax = fmax(rmax, v);
    }
    cmax = 0.0;
    for (int j = lane; j < cols; j += 32) {
        double v = 0.0;
        for (int i = 0; i < rows; ++i) {
            const float2 a = A[(int64_t)i * ld + j];
            v += (double)fabsf(a.x) + (double)fabsf(a.y);
        }
        cmax = fmax(cmax, v);
    }
    for (int s = 16; s >= 1; s >>= 1) cmax = fmax(cmax, __shfl_xor_sync(FULL, cmax, s));
}

__device__ __forceinline__ cdf cdf_zero() { return {{0.f, 0.f}, {0.f, 0.f}}; }
__device__ __forceinline__ cdf shfl_xor(const cdf &v, int s)
{
    return {{__shfl_xor_sync(FULL, v.re.hi, s), __shfl_xor_sync(FULL, v.re.lo, s)},
            {__shfl_xor_sync(FULL, v.im.hi, s), __shfl_xor_sync(FULL, v.im.lo, s)}};
}
__device__ __forceinline__ cdf shfl_idx(const cdf &v, int l)
{
    return {{__shfl_sync(FULL, v.re.hi, l), __shfl_sync(FULL, v.re.lo, l)},
            {__shfl_sync(FULL, v.im.hi, l), __shfl_sync(FULL, v.im.lo, l)}};
}
__device__ __forceinline__ double2 to_d2(const cdf &v)
{
    return make_double2((double)v.re.hi + (double)v.re.lo, (double)v.im.hi + (double)v.im.lo);
}
// lane l ends with the sum over all lanes of v[l & (S-1)] in v[0] (S = 8 or 4)
template <int S>
__device__ __forceinline__ void reduce_cdf(cdf (&v)[S], int lane)
{
#pragma unroll
    for (int s = S / 2; s >= 1; s >>= 1) {
        const bool up = (lane & s) != 0;
#pragma unroll
        for (int j = 0; j < s; ++j) {
            const cdf send = up ? v[j] : v[j + s];
            const cdf keep = up ? v[j + s] : v[j];
            v[j] = cdf_add(keep, shfl_xor(send, s));
        }
    }
#pragma unroll
    for (int s = S; s < 32; s <<= 1) v[0] = cdf_add(v[0], shfl_xor(v[0], s));
}

} // namespace dot2
} // namespace hm
