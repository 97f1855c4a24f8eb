// Basis-independent parts of the GPU H-Matrix construction (arxiv 2307.03968
// §III, eqs. 6-7), shared by the surface (RWG) and volume (SWG) builds.
//
//   k_fill       near-field blocks (complex64) and leaf self blocks
//                (complex128, upper half filled and mirrored) from the basis
//                geometry's entry function;
//   k_aca        partially pivoted adaptive cross approximation of every far
//                block, one CTA per block (§III, refs. [22,23]);
//   k_recompress re-compression of each ACA pair (ref. [24]): QR of both
//                factors by twice-iterated Gram-Schmidt, SVD of the small core
//                by one-sided Jacobi rotations, truncation at the tolerance;
//   k_pack_far   copy of the compressed factors into the padded pool;
//   host         cluster tree, eq. 7 block partition and the packed layout.
//
// A basis geometry G is a struct of device pointers with a member `perm`
// (tree position -> original unknown) and a device member template
//   template <class R> CX<R> entry(int m, int n) const
// returning the Galerkin matrix entry Z[m][n] of original unknowns m, n.
#pragma once

#include "hm_internal.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <numeric>

namespace hm {
namespace {

constexpr int ACA_THREADS = 128;
constexpr int ACA_KCAP = 48;
constexpr int RC_THREADS = 256;

template <class R> struct CX { R re, im; };

__device__ __forceinline__ float sqrtR(float v) { return sqrtf(v); }
__device__ __forceinline__ double sqrtR(double v) { return sqrt(v); }
__device__ __forceinline__ float logR(float v) { return logf(v); }
__device__ __forceinline__ double logR(double v) { return log(v); }
__device__ __forceinline__ float atanR(float v) { return atanf(v); }
__device__ __forceinline__ double atanR(double v) { return atan(v); }
__device__ __forceinline__ void sincosR(float v, float *s, float *c) { sincosf(v, s, c); }
__device__ __forceinline__ void sincosR(double v, double *s, double *c) { sincos(v, s, c); }
__device__ __forceinline__ float sinR(float v) { return sinf(v); }
__device__ __forceinline__ double sinR(double v) { return sin(v); }
__device__ __forceinline__ float absR(float v) { return fabsf(v); }
__device__ __forceinline__ double absR(double v) { return fabs(v); }

// ---------------------------------------------------------------- fill ----------
struct FillJob {
    int64_t out;     // element offset (pool for near, self64 for self)
    int64_t first;   // first flat entry index of this job
    int32_t r0, c0;  // tree positions of the row / column leaf starts
    int32_t m, n;    // true sizes
    int32_t ld;      // output row stride (near) ; unused for self
    int32_t self;    // 1 = self block (complex128, upper half + mirror)
};

// One thread per entry.  SELF = false: complex64 near blocks (row-major, row
// stride ld); SELF = true: complex128 leaf self blocks, the upper triangle
// (i <= j) enumerated row by row and mirrored.  Separate instantiations keep
// the FP32 near fill free of the FP64 path's registers.
template <class G, bool SELF>
__global__ void k_fill(G g, const FillJob *__restrict__ jobs, int njobs, int64_t total, float2 *pool,
                       double2 *self64)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = njobs - 1;
        while (lo < hi) {   // last job with first <= t
            const int mid = (lo + hi + 1) >> 1;
            if (jobs[mid].first <= t) lo = mid; else hi = mid - 1;
        }
        const FillJob J = jobs[lo];
        const int64_t e = t - J.first;
        if (SELF) {
            int i = 0;
            int64_t rem = e;
            while (rem >= J.n - i) { rem -= J.n - i; ++i; }
            const int j = i + (int)rem;
            const CX<double> v = g.template entry<double>(g.perm[J.r0 + i], g.perm[J.c0 + j]);
            self64[J.out + (int64_t)i * J.n + j] = make_double2(v.re, v.im);
            if (i != j) self64[J.out + (int64_t)j * J.n + i] = make_double2(v.re, v.im);
        } else {
            const int i = (int)(e / J.n), j = (int)(e - (int64_t)i * J.n);
            const CX<float> v = g.template entry<float>(g.perm[J.r0 + i], g.perm[J.c0 + j]);
            pool[J.out + (int64_t)i * J.ld + j] = make_float2(v.re, v.im);
        }
    }
}

// ---------------------------------------------------------------- ACA -----------
struct AcaJob {
    int64_t off;     // scratch offset: U^T (kmax x m) then V (kmax x n)
    int32_t r0, c0;  // tree positions
    int32_t m, n, kmax, pad;
};

__device__ __forceinline__ float cabs2(float2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ float2 cmulf(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ float2 cconjmul(float2 a, float2 b)   // conj(a) * b
{
    return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

// block-wide argmax of v (ties: lowest index); returns (value, index) to all threads
__device__ void block_argmax(float v, int idx, float *sv, int *si, float &ov, int &oi)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int s = 16; s >= 1; s >>= 1) {
        const float v2 = __shfl_xor_sync(0xffffffffu, v, s);
        const int i2 = __shfl_xor_sync(0xffffffffu, idx, s);
        if (v2 > v || (v2 == v && i2 < idx)) { v = v2; idx = i2; }
    }
    __syncthreads();
    if (lane == 0) { sv[w] = v; si[w] = idx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        float bv = sv[0];
        int bi = si[0];
        for (int q = 1; q < nw; ++q)
            if (sv[q] > bv || (sv[q] == bv && si[q] < bi)) { bv = sv[q]; bi = si[q]; }
        sv[0] = bv; si[0] = bi;
    }
    __syncthreads();
    ov = sv[0];
    oi = si[0];
}

// block-wide sum of a complex value (double accumulation across the block)
__device__ double2 block_sum(double2 v, double2 *sbuf)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int s = 16; s >= 1; s >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, s);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, s);
    }
    __syncthreads();
    if (lane == 0) sbuf[w] = v;
    __syncthreads();
    double2 r = make_double2(0, 0);
    for (int q = 0; q < nw; ++q) { r.x += sbuf[q].x; r.y += sbuf[q].y; }
    __syncthreads();
    return r;
}

// Partially pivoted ACA: Z[rows, cols] ~ sum_l u_l v_l^T with u_l stored as the
// row l of U^T (length m) and v_l as row l of V (length n).
template <class G>
__global__ void __launch_bounds__(ACA_THREADS)
k_aca(G g, const AcaJob *__restrict__ jobs, float2 *scratch, int32_t *ranks, float tol)
{
    const AcaJob J = jobs[blockIdx.x];
    float2 *UT = scratch + J.off;
    float2 *V = UT + (int64_t)J.kmax * J.m;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *used = smem_raw;           // [m]
    __shared__ float sv[32];
    __shared__ int si[32];
    __shared__ double2 sb[32];
    for (int i = threadIdx.x; i < J.m; i += blockDim.x) used[i] = 0;
    __syncthreads();
    int k = 0, istar = 0;
    double s2 = 0.0;
    int guard = 0;
    while (k < J.kmax && guard < J.m + J.kmax) {
        ++guard;
        float2 *v = V + (int64_t)k * J.n;
        float2 *u = UT + (int64_t)k * J.m;
        // residual row istar
        float best = -1.f;
        int bj = 0;
        for (int j = threadIdx.x; j < J.n; j += blockDim.x) {
            const CX<float> z = g.template entry<float>(g.perm[J.r0 + istar], g.perm[J.c0 + j]);
            float2 r = make_float2(z.re, z.im);
            for (int l = 0; l < k; ++l) {
                const float2 p = cmulf(UT[(int64_t)l * J.m + istar], V[(int64_t)l * J.n + j]);
                r.x -= p.x;
                r.y -= p.y;
            }
            v[j] = r;
            const float a = cabs2(r);
            if (a > best) { best = a; bj = j; }
        }
        __syncthreads();
        if (threadIdx.x == 0) used[istar] = 1;
        float pv;
        int jstar;
        block_argmax(best, bj, sv, si, pv, jstar);
        if (!(pv > 0.f)) {
            int next = -1;
            for (int i = 0; i < J.m; ++i)
                if (!used[i]) { next = i; break; }
            if (next < 0) break;
            istar = next;
            __syncthreads();
            continue;
        }
        const float2 piv = v[jstar];
        __syncthreads();
        const float pn = cabs2(piv);
        const float2 ipiv = make_float2(piv.x / pn, -piv.y / pn);
        for (int j = threadIdx.x; j < J.n; j += blockDim.x) v[j] = cmulf(v[j], ipiv);
        // residual column jstar
        for (int i = threadIdx.x; i < J.m; i += blockDim.x) {
            const CX<float> z = g.template entry<float>(g.perm[J.r0 + i], g.perm[J.c0 + jstar]);
            float2 c = make_float2(z.re, z.im);
            for (int l = 0; l < k; ++l) {
                const float2 p = cmulf(V[(int64_t)l * J.n + jstar], UT[(int64_t)l * J.m + i]);
                c.x -= p.x;
                c.y -= p.y;
            }
            u[i] = c;
        }
        __syncthreads();
        // norms and the cross terms of |S_k|_F^2
        double2 a = make_double2(0, 0);
        for (int i = threadIdx.x; i < J.m; i += blockDim.x) a.x += cabs2(u[i]);
        for (int j = threadIdx.x; j < J.n; j += blockDim.x) a.y += cabs2(v[j]);
        const double2 nuv = block_sum(a, sb);
        double cross = 0.0;
        for (int l = 0; l < k; ++l) {
            double2 pu = make_double2(0, 0), pv2 = make_double2(0, 0);
            for (int i = threadIdx.x; i < J.m; i += blockDim.x) {
                const float2 t = cconjmul(UT[(int64_t)l * J.m + i], u[i]);
                pu.x += t.x; pu.y += t.y;
            }
            const double2 su = block_sum(pu, sb);
            for (int j = threadIdx.x; j < J.n; j += blockDim.x) {
                const float2 t = cconjmul(V[(int64_t)l * J.n + j], v[j]);
                pv2.x += t.x; pv2.y += t.y;
            }
            const double2 svv = block_sum(pv2, sb);
            cross += su.x * svv.x - su.y * svv.y;   // Re(su * svv)
        }
        s2 += 2.0 * cross + nuv.x * nuv.y;
        ++k;
        if (sqrt(nuv.x * nuv.y) <= (double)tol * sqrt(fmax(s2, 0.0))) break;
        // next pivot row: largest |u_i| over unused rows
        float bu = -1.f;
        int bi = -1;
        for (int i = threadIdx.x; i < J.m; i += blockDim.x)
            if (!used[i]) {
                const float a2 = cabs2(u[i]);
                if (a2 > bu) { bu = a2; bi = i; }
            }
        float ov;
        int oi;
        block_argmax(bu, bi < 0 ? 0x7fffffff : bi, sv, si, ov, oi);
        if (ov < 0.f) break;
        istar = oi;
        __syncthreads();
    }
    if (threadIdx.x == 0) ranks[blockIdx.x] = k;
}

// ------------------------------------------------------------ re-compression ----
// One CTA per block.  Orthonormalise the rows of U^T (k x m) and of V (k x n) in
// place by Gram-Schmidt applied twice (R factors in shared memory, FP64), form
// the core C = R_U R_V^T, orthogonalise its columns by one-sided Jacobi
// rotations (C W = [sigma_i w_i]), keep the smallest rank r whose discarded
// singular values have Frobenius norm <= tol * total, and overwrite the rows:
//   U'^T[l] = sum_t (C W)[t][p_l] q_t      V'[l] = sum_t conj(W[t][p_l]) q'_t
// (p = singular values sorted descending), so that U'^T^T V' = Q_U C Q_V^T.
__device__ void gram_schmidt_rows(float2 *Q, int k, int len, double2 *Rm /* k x k, Rm[t*k + l] */,
                                  double2 *coef, double2 *sb)
{
    for (int l = 0; l < k; ++l)
        for (int t = threadIdx.x; t < k; t += blockDim.x) Rm[t * k + l] = make_double2(0, 0);
    __syncthreads();
    for (int l = 0; l < k; ++l) {
        float2 *ql = Q + (int64_t)l * len;
        for (int pass = 0; pass < 2; ++pass) {
            for (int t = 0; t < l; ++t) {
                const float2 *qt = Q + (int64_t)t * len;
                double2 a = make_double2(0, 0);
                for (int i = threadIdx.x; i < len; i += blockDim.x) {
                    const float2 c = cconjmul(qt[i], ql[i]);
                    a.x += c.x; a.y += c.y;
                }
                const double2 s = block_sum(a, sb);
                if (threadIdx.x == 0) {
                    coef[t] = s;
                    Rm[t * k + l].x += s.x;
                    Rm[t * k + l].y += s.y;
                }
            }
            __syncthreads();
            for (int i = threadIdx.x; i < len; i += blockDim.x) {
                float2 v = ql[i];
                for (int t = 0; t < l; ++t) {
                    const float2 q = Q[(int64_t)t * len + i];
                    const float cr = (float)coef[t].x, ci = (float)coef[t].y;
                    v.x -= cr * q.x - ci * q.y;
                    v.y -= cr * q.y + ci * q.x;
                }
                ql[i] = v;
            }
            __syncthreads();
        }
        double2 a = make_double2(0, 0);
        for (int i = threadIdx.x; i < len; i += blockDim.x) a.x += cabs2(ql[i]);
        const double nrm = sqrt(block_sum(a, sb).x);
        if (threadIdx.x == 0) Rm[l * k + l] = make_double2(nrm, 0.0);
        const float inv = nrm > 0.0 ? (float)(1.0 / nrm) : 0.f;
        for (int i = threadIdx.x; i < len; i += blockDim.x) {
            ql[i].x *= inv;
            ql[i].y *= inv;
        }
        __syncthreads();
    }
}

__device__ __forceinline__ double2 zmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 zcmul(double2 a, double2 b) { return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }  // conj(a) b

__global__ void __launch_bounds__(RC_THREADS)
k_recompress(const AcaJob *__restrict__ jobs, float2 *scratch, int32_t *ranks, float tol)
{
    const AcaJob J = jobs[blockIdx.x];
    const int k = ranks[blockIdx.x];
    if (k <= 1) return;
    float2 *UT = scratch + J.off;
    float2 *V = UT + (int64_t)J.kmax * J.m;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2 *Ru = reinterpret_cast<double2 *>(smem_raw);   // k x k
    double2 *Rv = Ru + k * k;                              // k x k
    double2 *C = Rv + k * k;                               // k x k, column-major C[col*k + row]
    double2 *W = C + k * k;                                // k x k, column-major
    double2 *coef = W + k * k;                             // k
    double *sig = reinterpret_cast<double *>(coef + k);    // k
    int *order = reinterpret_cast<int *>(sig + k);         // k
    __shared__ double2 sb[32];
    __shared__ int s_r;
    __shared__ int s_rot;
    gram_schmidt_rows(UT, k, J.m, Ru, coef, sb);
    gram_schmidt_rows(V, k, J.n, Rv, coef, sb);
    // C = Ru Rv^T (both upper triangular, Rm[t*k + l] = R[t][l])
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
        const int row = e % k, col = e / k;
        double2 s = make_double2(0, 0);
        for (int t = 0; t < k; ++t) {
            const double2 p = zmul(Ru[row * k + t], Rv[col * k + t]);
            s.x += p.x; s.y += p.y;
        }
        C[col * k + row] = s;
        W[col * k + row] = make_double2(row == col ? 1.0 : 0.0, 0.0);
    }
    __syncthreads();
    // one-sided Jacobi on the columns of C (cyclic sweeps over pairs p < q);
    // warp 0 forms the 2x2 Gram entries, the whole CTA applies the rotation
    for (int sweep = 0; sweep < 20; ++sweep) {
        if (threadIdx.x == 0) s_rot = 0;
        __syncthreads();
        for (int p = 0; p < k - 1; ++p)
            for (int q = p + 1; q < k; ++q) {
                if (threadIdx.x < 32) {
                    double al = 0, be = 0, gr = 0, gi = 0;
                    for (int t = threadIdx.x; t < k; t += 32) {
                        const double2 cp = C[p * k + t], cq = C[q * k + t];
                        al += cp.x * cp.x + cp.y * cp.y;
                        be += cq.x * cq.x + cq.y * cq.y;
                        gr += cp.x * cq.x + cp.y * cq.y;
                        gi += cp.x * cq.y - cp.y * cq.x;
                    }
                    for (int o = 16; o >= 1; o >>= 1) {
                        al += __shfl_xor_sync(0xffffffffu, al, o);
                        be += __shfl_xor_sync(0xffffffffu, be, o);
                        gr += __shfl_xor_sync(0xffffffffu, gr, o);
                        gi += __shfl_xor_sync(0xffffffffu, gi, o);
                    }
                    if (threadIdx.x == 0) {
                        const double gabs = sqrt(gr * gr + gi * gi);
                        double c = 1.0, sr = 0.0, si = 0.0;
                        if (gabs > 1e-12 * sqrt(al * be) && gabs > 0.0) {
                            const double zeta = (be - al) / (2.0 * gabs);
                            const double tt = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                            c = 1.0 / sqrt(1.0 + tt * tt);
                            const double sv_ = c * tt;
                            sr = sv_ * gr / gabs;   // s = |s| gamma / |gamma|
                            si = sv_ * gi / gabs;
                            s_rot = 1;
                        }
                        coef[0] = make_double2(c, 0.0);
                        coef[1] = make_double2(sr, si);
                    }
                }
                __syncthreads();
                const double c = coef[0].x;
                const double2 sv2 = coef[1];
                if (c != 1.0)
                    for (int t = threadIdx.x; t < 2 * k; t += blockDim.x) {
                        double2 *M = t < k ? C : W;
                        const int r = t < k ? t : t - k;
                        const double2 a = M[p * k + r], b = M[q * k + r];
                        // [a b] <- [a b] [[c, s], [-conj(s), c]]
                        const double2 csb = zcmul(sv2, b);   // conj(s) b
                        const double2 sa = zmul(sv2, a);
                        M[p * k + r] = make_double2(c * a.x - csb.x, c * a.y - csb.y);
                        M[q * k + r] = make_double2(sa.x + c * b.x, sa.y + c * b.y);
                    }
                __syncthreads();
            }
        if (!s_rot) break;
        __syncthreads();
    }
    // singular values and truncation
    for (int l = threadIdx.x; l < k; l += blockDim.x) {
        double a = 0;
        for (int t = 0; t < k; ++t) a += C[l * k + t].x * C[l * k + t].x + C[l * k + t].y * C[l * k + t].y;
        sig[l] = sqrt(a);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int l = 0; l < k; ++l) order[l] = l;
        for (int a = 1; a < k; ++a) {   // insertion sort, descending
            const int key = order[a];
            int b = a - 1;
            while (b >= 0 && sig[order[b]] < sig[key]) { order[b + 1] = order[b]; --b; }
            order[b + 1] = key;
        }
        double total = 0;
        for (int l = 0; l < k; ++l) total += sig[l] * sig[l];
        double tail = total;
        int r = k;
        for (int l = 0; l < k; ++l) {   // tail = sum of sig[order[l..]]^2
            if (l >= 1 && sqrt(fmax(tail, 0.0)) <= tol * sqrt(total)) { r = l; break; }
            tail -= sig[order[l]] * sig[order[l]];
        }
        if (r < 1) r = 1;
        s_r = r;
    }
    __syncthreads();
    const int r = s_r;
    // rows of U'^T and V' : each thread owns one position and transforms its k-vector
    for (int side = 0; side < 2; ++side) {
        float2 *Q = side == 0 ? UT : V;
        const int len = side == 0 ? J.m : J.n;
        for (int i = threadIdx.x; i < len; i += blockDim.x) {
            float2 qv[ACA_KCAP];
            for (int t = 0; t < k; ++t) qv[t] = Q[(int64_t)t * len + i];
            for (int l = 0; l < r; ++l) {
                const int pl = order[l];
                double2 s = make_double2(0, 0);
                for (int t = 0; t < k; ++t) {
                    const double2 q = make_double2(qv[t].x, qv[t].y);
                    const double2 m = side == 0 ? C[pl * k + t] : make_double2(W[pl * k + t].x, -W[pl * k + t].y);
                    const double2 p = zmul(m, q);
                    s.x += p.x; s.y += p.y;
                }
                Q[(int64_t)l * len + i] = make_float2((float)s.x, (float)s.y);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) ranks[blockIdx.x] = r;
}

// copy rank-r factors from the ACA scratch into the padded pool
struct PackJob {
    int64_t src;     // scratch offset (U^T kmax x m, V kmax x n)
    int64_t dst;     // pool offset (U^T r x pm, V r x pn)
    int32_t r0, c0;  // tree positions (true)
    int32_t pr0, pc0;// padded positions
    int32_t m, n, pm, pn, kmax, r;
};

__global__ void k_pack_far(const PackJob *__restrict__ jobs, const float2 *__restrict__ scratch,
                           const int32_t *__restrict__ ptree, float2 *pool)
{
    const PackJob J = jobs[blockIdx.x];
    const int64_t nu = (int64_t)J.r * J.pm, nv = (int64_t)J.r * J.pn;
    for (int64_t e = threadIdx.x; e < nu + nv; e += blockDim.x) {
        float2 v = make_float2(0.f, 0.f);
        if (e < nu) {
            const int l = (int)(e / J.pm), pi = (int)(e - (int64_t)l * J.pm);
            const int tp = ptree[J.pr0 + pi];
            if (tp >= 0) v = scratch[J.src + (int64_t)l * J.m + (tp - J.r0)];
        } else {
            const int64_t e2 = e - nu;
            const int l = (int)(e2 / J.pn), pj = (int)(e2 - (int64_t)l * J.pn);
            const int tp = ptree[J.pc0 + pj];
            if (tp >= 0) v = scratch[J.src + (int64_t)J.kmax * J.m + (int64_t)l * J.n + (tp - J.c0)];
        }
        pool[J.dst + e] = v;
    }
}

// ------------------------------------------------------------ host side ---------
struct HostTree {
    std::vector<std::vector<std::pair<int64_t, int64_t>>> levels;   // (offset, size) per depth
    std::vector<std::vector<std::vector<int>>> children;           // per depth
    std::vector<std::vector<std::array<double, 6>>> box;           // lo[3], hi[3]
    std::vector<int64_t> perm;
    int depth = 0;
};


// bisect idx along the longest axis of the bounding box of its centres; ties in
// the axis go to the lower axis; sort key (coordinate, original index); cut at n/2
void bisect(const std::vector<int64_t> &idx, const std::vector<double> &cen, std::vector<int64_t> &a,
            std::vector<int64_t> &b)
{
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t v : idx)
        for (int d = 0; d < 3; ++d) {
            lo[d] = std::min(lo[d], cen[3 * v + d]);
            hi[d] = std::max(hi[d], cen[3 * v + d]);
        }
    int axis = 0;
    double best = hi[0] - lo[0];
    for (int d = 1; d < 3; ++d)
        if (hi[d] - lo[d] > best) { best = hi[d] - lo[d]; axis = d; }
    std::vector<int64_t> s = idx;
    std::sort(s.begin(), s.end(), [&](int64_t x, int64_t y) {
        const double cx = cen[3 * x + axis], cy = cen[3 * y + axis];
        return cx < cy || (cx == cy && x < y);
    });
    const size_t h = s.size() / 2;
    a.assign(s.begin(), s.begin() + h);
    b.assign(s.begin() + h, s.end());
}

hm_status build_tree(const std::vector<double> &cen, const std::vector<double> &blo, const std::vector<double> &bhi,
                     int64_t N, int leaf_size, int arity, HostTree &T)
{
    const int splits = arity == 2 ? 1 : arity == 4 ? 2 : 3;
    std::vector<std::vector<int64_t>> clusters(1);
    clusters[0].resize(N);
    std::iota(clusters[0].begin(), clusters[0].end(), 0);
    std::vector<std::vector<std::vector<int64_t>>> lv{clusters};
    while (true) {
        size_t mx = 0;
        for (auto &c : clusters) mx = std::max(mx, c.size());
        if ((int64_t)mx <= leaf_size) break;
        std::vector<std::vector<int64_t>> nxt;
        std::vector<std::vector<int>> ch;
        for (auto &c : clusters) {
            std::vector<std::vector<int64_t>> parts{c};
            for (int s = 0; s < splits; ++s) {
                std::vector<std::vector<int64_t>> np;
                for (auto &p : parts) {
                    std::vector<int64_t> a, b;
                    bisect(p, cen, a, b);
                    np.push_back(std::move(a));
                    np.push_back(std::move(b));
                }
                parts.swap(np);
            }
            std::vector<int> kids;
            for (auto &p : parts) {
                if (p.empty()) return fail(HM_ERR_ARG, "leaf_size too small for this arity: a cluster would be empty");
                kids.push_back((int)nxt.size());
                nxt.push_back(std::move(p));
            }
            ch.push_back(kids);
        }
        T.children.push_back(ch);
        clusters.swap(nxt);
        lv.push_back(clusters);
    }
    T.depth = (int)lv.size() - 1;
    T.perm.clear();
    for (auto &c : clusters) T.perm.insert(T.perm.end(), c.begin(), c.end());
    std::vector<int64_t> pos(N);
    for (int64_t p = 0; p < N; ++p) pos[T.perm[p]] = p;
    for (auto &cl : lv) {
        std::vector<std::pair<int64_t, int64_t>> L;
        std::vector<std::array<double, 6>> B;
        for (auto &c : cl) {
            int64_t mn = N;
            std::array<double, 6> bx{INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
            for (int64_t v : c) {
                mn = std::min(mn, pos[v]);
                for (int d = 0; d < 3; ++d) {
                    bx[d] = std::min(bx[d], blo[3 * v + d]);
                    bx[3 + d] = std::max(bx[3 + d], bhi[3 * v + d]);
                }
            }
            L.push_back({mn, (int64_t)c.size()});
            B.push_back(bx);
        }
        T.levels.push_back(L);
        T.box.push_back(B);
    }
    return HM_OK;
}

bool admissible(const HostTree &T, int d, int t, int s, double c)
{
    const auto &a = T.box[d][t], &b = T.box[d][s];
    double g2 = 0, da = 0, db = 0;
    for (int x = 0; x < 3; ++x) {
        const double gap = std::max(0.0, std::max(b[x] - a[3 + x], a[x] - b[3 + x]));
        g2 = g2 + gap * gap;
        const double ea = a[3 + x] - a[x], eb = b[3 + x] - b[x];
        da = da + ea * ea;
        db = db + eb * eb;
    }
    const double dist = std::sqrt(g2);
    return dist > 0.0 && dist >= c * std::min(std::sqrt(da), std::sqrt(db));
}

void partition(const HostTree &T, double c, int d, int t, int s, std::vector<std::pair<int, int>> &near,
               std::map<int, std::vector<std::pair<int, int>>> &far)
{
    if (t != s && admissible(T, d, t, s, c)) {
        far[d].push_back({t, s});
        return;
    }
    if (d == T.depth) {
        if (t != s) near.push_back({t, s});
        return;
    }
    for (int ct : T.children[d][t])
        for (int cs : T.children[d][s]) {
            if (t == s && ct > cs) continue;
            partition(T, c, d + 1, ct, cs, near, far);
        }
}

template <class T> hm_status up(hm_matrix h, T **dst, const std::vector<T> &src, cudaStream_t s)
{
    hm_status st = dev_alloc(h, (void **)dst, std::max<size_t>(1, src.size()) * sizeof(T));
    if (st != HM_OK) return st;
    if (!src.empty()) HM_CUDA(cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return HM_OK;
}

struct TmpBuffers {
    std::vector<void *> ptrs;
    ~TmpBuffers() { for (void *p : ptrs) cudaFree(p); }
    template <class T> hm_status up(T **dst, const std::vector<T> &src, cudaStream_t s)
    {
        void *p = nullptr;
        const size_t bytes = std::max<size_t>(1, src.size()) * sizeof(T);
        HM_CUDA(cudaMalloc(&p, bytes));
        ptrs.push_back(p);
        *dst = (T *)p;
        if (!src.empty()) HM_CUDA(cudaMemcpyAsync(p, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s));
        return HM_OK;
    }
    hm_status alloc(void **dst, size_t bytes)
    {
        HM_CUDA(cudaMalloc(dst, std::max<size_t>(bytes, 16)));
        ptrs.push_back(*dst);
        return HM_OK;
    }
};

// Host description of the unknowns of one basis: the point each unknown is
// sorted by in the tree and its support box, plus what the operator keeps for
// plane-wave excitation (b_m = sum over the two sides of ucoef * sum_q w_q
// (r_q - v) . p exp(-jk k . r_q) over the side's cell).
struct BasisData {
    int64_t N = 0;
    std::vector<double> cen, blo, bhi;   // N x 3 each
    int nq = 0;                          // quadrature points per cell
    std::vector<double> qw;              // nq weights (sum 1)
    std::vector<double> qpd;             // n_cell x nq x 3 points
    std::vector<double> vtx;             // n_vert x 3
    std::vector<int32_t> ucell, ufree;   // N x 2: cell and free vertex of each side (-1: no side)
    std::vector<double> ucoef;           // N x 2
};

// Tree, partition, packed layout, far-field ACA + re-compression and near fill
// for the basis geometry g (all device pointers set except g.perm).
template <class G>
hm_status assemble(BasisData &B, G g, const hm_build_opts *o, TmpBuffers &tmp, cudaStream_t s, hm_matrix *out)
{
    const int64_t N = B.N;
    HostTree T;
    hm_status st = build_tree(B.cen, B.blo, B.bhi, N, o->leaf_size, o->arity, T);
    if (st != HM_OK) return st;
    std::vector<std::pair<int, int>> near;
    std::map<int, std::vector<std::pair<int, int>>> farp;
    partition(T, o->adm, 0, 0, 0, near, farp);

    hm_matrix h = new hm_matrix_s();
    struct Guard { hm_matrix h; bool keep = false; ~Guard() { if (!keep && h) hm_destroy(h); } } guard{h};
    h->N = N;
    h->perm = T.perm;
    h->n_leaves = (int64_t)T.levels[T.depth].size();
    h->leaf_off.resize(h->n_leaves + 1);
    for (int64_t i = 0; i < h->n_leaves; ++i) h->leaf_off[i] = T.levels[T.depth][i].first;
    h->leaf_off[h->n_leaves] = N;
    h->has_fp64 = o->keep_fp64 != 0;
    if ((st = finalize_layout(h, s)) != HM_OK) return st;
    h->depth = T.depth;

    std::vector<int32_t> perm32(T.perm.begin(), T.perm.end());
    int32_t *d_perm = nullptr;
    if ((st = tmp.up(&d_perm, perm32, s)) != HM_OK) return st;
    g.perm = d_perm;

    // ---- far blocks: ACA + re-compression into scratch
    const int max_level_keep = o->levels < 0 ? 1 << 20 : o->levels;
    struct FarRec { int level; int64_t r0, m, c0, n; };
    std::vector<FarRec> fars;
    for (auto &kv : farp) {
        const int lev = T.depth - kv.first + 1;
        if (lev > max_level_keep) continue;
        for (auto &pr : kv.second) {
            const auto &a = T.levels[kv.first][pr.first], &b = T.levels[kv.first][pr.second];
            fars.push_back({lev, a.first, a.second, b.first, b.second});
        }
    }
    std::vector<AcaJob> aj(fars.size());
    int64_t scr = 0;
    for (size_t b = 0; b < fars.size(); ++b) {
        const int kmax = (int)std::min<int64_t>(ACA_KCAP, std::min(fars[b].m, fars[b].n));
        aj[b] = {scr, (int32_t)fars[b].r0, (int32_t)fars[b].c0, (int32_t)fars[b].m, (int32_t)fars[b].n, kmax, 0};
        scr += (int64_t)kmax * (fars[b].m + fars[b].n);
    }
    float2 *d_scr = nullptr;
    int32_t *d_ranks = nullptr;
    AcaJob *d_aj = nullptr;
    std::vector<int32_t> ranks(fars.size(), 0);
    if (!fars.empty()) {
        if ((st = tmp.alloc((void **)&d_scr, sizeof(float2) * scr)) != HM_OK) return st;
        if ((st = tmp.alloc((void **)&d_ranks, sizeof(int32_t) * fars.size())) != HM_OK) return st;
        if ((st = tmp.up(&d_aj, aj, s)) != HM_OK) return st;
        int64_t maxm = 0;
        for (auto &j : aj) maxm = std::max<int64_t>(maxm, j.m);
        k_aca<G><<<(unsigned)fars.size(), ACA_THREADS, maxm, s>>>(g, d_aj, d_scr, d_ranks, (float)o->aca_tol);
        HM_CUDA(cudaGetLastError());
        HM_CUDA(cudaMemcpyAsync(ranks.data(), d_ranks, sizeof(int32_t) * fars.size(), cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaStreamSynchronize(s));
        // re-compression, launched per rank bucket so that shared memory fits the bucket
        const int bounds[] = {8, 16, 32, ACA_KCAP};
        int lo = 1;
        for (int bk : bounds) {
            std::vector<AcaJob> jb;
            std::vector<int32_t> rb;
            std::vector<size_t> where;
            for (size_t b = 0; b < fars.size(); ++b)
                if (ranks[b] > lo && ranks[b] <= bk) { jb.push_back(aj[b]); rb.push_back(ranks[b]); where.push_back(b); }
            lo = bk;
            if (jb.empty()) continue;
            AcaJob *d_jb = nullptr;
            int32_t *d_rb = nullptr;
            if ((st = tmp.up(&d_jb, jb, s)) != HM_OK) return st;
            if ((st = tmp.up(&d_rb, rb, s)) != HM_OK) return st;
            const size_t rsm = 4 * (size_t)bk * bk * sizeof(double2) + bk * (sizeof(double2) + sizeof(double) + sizeof(int)) + 64;
            HM_CUDA(cudaFuncSetAttribute(k_recompress, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm));
            k_recompress<<<(unsigned)jb.size(), RC_THREADS, rsm, s>>>(d_jb, d_scr, d_rb, (float)o->aca_tol);
            HM_CUDA(cudaGetLastError());
            HM_CUDA(cudaMemcpyAsync(rb.data(), d_rb, sizeof(int32_t) * rb.size(), cudaMemcpyDeviceToHost, s));
            HM_CUDA(cudaStreamSynchronize(s));
            for (size_t q = 0; q < where.size(); ++q) ranks[where[q]] = rb[q];
        }
    }

    // ---- pool layout: near blocks (level 1) then far blocks, by level
    std::map<int64_t, int64_t> leaf_start, leaf_end;
    for (int64_t i = 0; i < h->n_leaves; ++i) {
        leaf_start[h->leaf_off[i]] = i;
        leaf_end[h->leaf_off[i + 1]] = i;
    }
    auto padded = [&](int64_t r0, int64_t m, int64_t &pr0, int64_t &pm) {
        const int64_t a = leaf_start.at(r0), b = leaf_end.at(r0 + m);
        pr0 = h->pleaf_off[a];
        pm = h->pleaf_off[b + 1] - pr0;
    };
    int64_t pool = 0;
    std::vector<FillJob> fj, fs;   // near jobs, self jobs
    int64_t flat = 0, flat_self = 0;
    for (auto &pr : near) {
        const auto &a = T.levels[T.depth][pr.first], &b = T.levels[T.depth][pr.second];
        Item it{};
        int64_t pr0, pm, pc0, pn;
        padded(a.first, a.second, pr0, pm);
        padded(b.first, b.second, pc0, pn);
        it.off = pool; it.row0 = (int32_t)pr0; it.col0 = (int32_t)pc0;
        it.m = (int32_t)a.second; it.n = (int32_t)b.second; it.k = 0;
        fj.push_back({it.off, flat, (int32_t)a.first, (int32_t)b.first, it.m, it.n, (int32_t)even(it.n), 0});
        flat += (int64_t)it.m * it.n;
        pool += item_elems(it);
        LevelList &L = h->levels[1];
        L.items.push_back(it); L.true_m.push_back(it.m); L.true_n.push_back(it.n);
        L.elems += item_elems(it); L.n_dense++;
        L.alg_elems += (int64_t)it.m * it.n;
    }
    std::vector<PackJob> pj;
    int max_level = 1, max_rank = 0;
    for (size_t b = 0; b < fars.size(); ++b) {
        const FarRec &f = fars[b];
        Item it{};
        int64_t pr0, pm, pc0, pn;
        padded(f.r0, f.m, pr0, pm);
        padded(f.c0, f.n, pc0, pn);
        it.off = pool; it.row0 = (int32_t)pr0; it.col0 = (int32_t)pc0;
        it.m = (int32_t)pm; it.n = (int32_t)pn; it.k = ranks[b];
        if (it.k < 1) continue;   // an exactly zero block
        pj.push_back({aj[b].off, it.off, (int32_t)f.r0, (int32_t)f.c0, (int32_t)pr0, (int32_t)pc0, (int32_t)f.m,
                      (int32_t)f.n, (int32_t)pm, (int32_t)pn, aj[b].kmax, it.k});
        pool += item_elems(it);
        LevelList &L = h->levels[f.level];
        L.items.push_back(it); L.true_m.push_back((int32_t)f.m); L.true_n.push_back((int32_t)f.n);
        L.elems += item_elems(it); L.n_lowrank++;
        L.alg_elems += (int64_t)it.k * (f.m + f.n);
        max_level = std::max(max_level, f.level);
        max_rank = std::max(max_rank, it.k);
    }
    // self blocks (complex128, upper half + mirror)
    for (int64_t i = 0; i < h->n_leaves; ++i) {
        const int64_t n = h->leaf_off[i + 1] - h->leaf_off[i];
        fs.push_back({h->self_off[i], flat_self, (int32_t)h->leaf_off[i], (int32_t)h->leaf_off[i], (int32_t)n,
                      (int32_t)n, 0, 1});
        flat_self += n * (n + 1) / 2;
    }
    h->pool_elems = pool;
    h->n_levels = max_level;
    h->max_rank = max_rank;
    if ((st = dev_alloc(h, (void **)&h->d_pool32, sizeof(float2) * std::max<int64_t>(pool, 1))) != HM_OK) return st;
    HM_CUDA(cudaMemsetAsync(h->d_pool32, 0, sizeof(float2) * std::max<int64_t>(pool, 1), s));
    if ((st = dev_alloc(h, (void **)&h->d_self64, sizeof(double2) * h->self_elems)) != HM_OK) return st;
    FillJob *d_fj = nullptr, *d_fs = nullptr;
    if ((st = tmp.up(&d_fj, fj, s)) != HM_OK) return st;
    if ((st = tmp.up(&d_fs, fs, s)) != HM_OK) return st;
    if (flat > 0) {
        const int grid = (int)std::min<int64_t>((flat + 255) / 256, 152 * 64);
        k_fill<G, false><<<grid, 256, 0, s>>>(g, d_fj, (int)fj.size(), flat, h->d_pool32, h->d_self64);
        HM_CUDA(cudaGetLastError());
    }
    if (flat_self > 0) {
        const int grid = (int)std::min<int64_t>((flat_self + 255) / 256, 152 * 64);
        k_fill<G, true><<<grid, 256, 0, s>>>(g, d_fs, (int)fs.size(), flat_self, h->d_pool32, h->d_self64);
        HM_CUDA(cudaGetLastError());
    }
    if (!pj.empty()) {
        std::vector<int32_t> ptree(h->pN, -1);
        for (int64_t i = 0; i < h->n_leaves; ++i)
            for (int64_t p = h->leaf_off[i]; p < h->leaf_off[i + 1]; ++p)
                ptree[h->pleaf_off[i] + (p - h->leaf_off[i])] = (int32_t)p;
        int32_t *d_ptree = nullptr;
        PackJob *d_pj = nullptr;
        if ((st = tmp.up(&d_ptree, ptree, s)) != HM_OK) return st;
        if ((st = tmp.up(&d_pj, pj, s)) != HM_OK) return st;
        k_pack_far<<<(unsigned)pj.size(), 256, 0, s>>>(d_pj, d_scr, d_ptree, h->d_pool32);
        HM_CUDA(cudaGetLastError());
    }
    if (h->has_fp64) {   // complex128 copy of the same (complex64-filled) blocks for the FP64 path
        if ((st = dev_alloc(h, (void **)&h->d_pool64, sizeof(double2) * std::max<int64_t>(pool, 1))) != HM_OK)
            return st;
        launch_convert_f32_to_f64(h->d_pool32, h->d_pool64, std::max<int64_t>(pool, 1), s);
    }
    if ((st = prepare_partials(h, s)) != HM_OK) return st;
    if ((st = upload_item_lists(h, s)) != HM_OK) return st;
    // geometry kept for the plane-wave excitation
    if ((st = up(h, &h->d_qpd, B.qpd, s)) != HM_OK || (st = up(h, &h->d_vtx, B.vtx, s)) != HM_OK ||
        (st = up(h, &h->d_ucell, B.ucell, s)) != HM_OK || (st = up(h, &h->d_ufree, B.ufree, s)) != HM_OK ||
        (st = up(h, &h->d_ucoef, B.ucoef, s)) != HM_OK || (st = up(h, &h->d_rhs_w, B.qw, s)) != HM_OK)
        return st;
    h->rhs_nq = B.nq;
    h->has_mesh = true;
    h->wavenumber = g.k;
    HM_CUDA(cudaStreamSynchronize(s));
    guard.keep = true;
    *out = h;
    return HM_OK;
}

} // namespace
} // namespace hm
