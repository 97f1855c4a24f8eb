// FP64-class residual products for many right-hand sides, owner-computes form
// (the refinement residual r = b - A_m x of the solve; the block products are
// eq. 6 and eq. 8 of arxiv 2307.03968 with the half storage of §III).
//
// A work unit is one output cluster O of a level and one group of RG right-hand
// sides (16, or 8 for calls with few right-hand sides, so that there are enough
// units to balance).  The CTA walks every directed product into O (the stored
// blocks with O as row cluster, and mirrored, those with O as column cluster;
// dense or low-rank), in a fixed order, and keeps the sums in registers as
// double-float complex numbers.  Each directed product is summed, per output row
// and right-hand side, as one error-free chain on a common grid (k_dot2.cuh: every
// product rounded exactly onto a power-of-two grid whose sigma comes from the
// product's precomputed bound, k_prod_bounds, and the input's largest component;
// the remainders summed apart), folded once into the double-float sum with a
// compensated addition.  Thread t of the RT-thread CTA (RT = 128 or 256) owns
// output row t % 64 and the right-hand sides QN (t / 64) .. + QN - 1 of the group,
// QN = RG / (RT / 64).  The unit's sums are stored once, in FP64, into the level's
// [RHS][pN] array: no partial slots, no atomics, and the result is independent of
// scheduling.  k_gather_own then forms b - (D x + sum over levels) in FP64.
//
// Shared-memory staging keeps every compute read consecutive along the output
// row: a dense block is stored K-major (element (K index j, output i) at
// j * 65 + i), whichever orientation the product reads it in; a low-rank
// block's input-side factor W is stored K-major over its rank rows and its
// output-side factor Y rank-major.
#include "k_dot2.cuh"

#include <algorithm>

namespace hm {
namespace {

using namespace kc;
using namespace dot2;
constexpr int RGMAX = 16;        // right-hand sides per unit (at most)
constexpr int BS = 65;           // float2 stride of a staged K row of a block (odd: conflict-free staging)
constexpr int WS = 33;           // float2 stride of a staged K row of W (rank <= 32)
constexpr int XS = 18;           // float2 stride of a staged K row of x (16 RHS, 16-byte aligned rows)
constexpr int SM_B = 64 * WS + 32 * BS;   // float2: W (64 x WS) then Y (32 x BS), or a dense block (64 x BS)
constexpr int SM_X = 64 * XS;
constexpr int SM_T = 32 * RGMAX; // cdf: T = W x (rank x RG RHS)
static_assert(64 * BS <= SM_B, "a dense block fits the block area");

struct alignas(16) Smem {
    float2 b[SM_B];
    float2 x[SM_X];
    cdf t[SM_T];
    float mx[2 * RGMAX];         // max |x|_inf over K indices 32h..32h+31 (h = 0, 1), per right-hand side
};

// stage x of the input cluster: xs[j * XS + q] = x[(r0 + q) * ldx + in0 + j] for j < klen, q < nr,
// 0 for the rest of j < roundup4(klen); mx[2 q + h] = max over j = 32h..32h+31 of |x|_inf.
// Every thread runs the same number of iterations (RG * 64 is a multiple of RT), and a warp
// covers 32 consecutive j of one q.
template <int RG, int RT>
__device__ __forceinline__ void stage_x(float2 *xs, float *mx, const float2 *__restrict__ x, int64_t ldx, int r0,
                                        int nr, int in0, int klen)
{
    static_assert((RG * 64) % RT == 0, "uniform staging loop");
    const int k4 = (klen + 3) & ~3;
    for (int e = threadIdx.x; e < RG * 64; e += RT) {
        const int q = e >> 6, j = e & 63;
        const float2 v = (j < klen && q < nr) ? x[(int64_t)(r0 + q) * ldx + in0 + j] : make_float2(0.f, 0.f);
        if (j < k4) xs[j * XS + q] = v;
        const float m = warp_max(linf(v));
        if ((j & 31) == 0) mx[2 * q + (j >> 5)] = m;
    }
}
// the largest |x|_inf of right-hand side q over the staged input
__device__ __forceinline__ float x_max(const float *mx, int q) { return fmaxf(mx[2 * q], mx[2 * q + 1]); }

template <int RG, int RT>
__global__ void __launch_bounds__(RT, 4)
k_resid_own(const TcUnit *__restrict__ units, int n_units, const TcProd *__restrict__ prods,
            const float2 *__restrict__ pbnd, const float2 *__restrict__ pool, const float2 *__restrict__ x,
            int64_t ldx, int nrhs, double2 *__restrict__ own, int64_t ldo)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    Smem &S = *reinterpret_cast<Smem *>(smraw);
    constexpr int QN = RG / (RT / 64);   // right-hand sides per thread
    const int tid = threadIdx.x, i = tid & 63, hh = tid >> 6;
    const int n_groups = (nrhs + RG - 1) / RG;
    const int64_t total = (int64_t)n_units * n_groups;
    // cluster-major: the RHS groups of one output cluster are consecutive units, so they
    // run on neighbouring CTAs at the same time and read the cluster's blocks from DRAM
    // once between them (the later reads hit L2)
    for (int64_t u = blockIdx.x; u < total; u += gridDim.x) {
        const TcUnit U = units[u / n_groups];
        const int r0 = (int)(u % n_groups) * RG, nr = min(RG, nrhs - r0);
        cdf acc[QN];
#pragma unroll
        for (int q = 0; q < QN; ++q) acc[q] = cdf_zero();
        for (int p = U.p0; p < U.p1; ++p) {
            const TcProd P = prods[p];
            __syncthreads();                                  // the previous product's reads are done
            stage_x<RG, RT>(S.x, S.mx, x, ldx, r0, nr, P.in0, P.klen);
            if (P.rank == 0) {
                // block elements (output i < olen, K j < klen) into b[j * BS + i]
                const float2 *B = pool + P.b_off;
                const int rows = P.trans ? P.klen : P.olen;
                for (int e = tid; e < rows * 64; e += RT) {
                    const int a = e >> 6, c = e & 63;         // source row a, column c (coalesced along c)
                    if (P.trans) {                            // element (i = c, j = a) = B[a][c]
                        if (a < P.klen && c < P.olen) S.b[a * BS + c] = B[(int64_t)a * P.b_ld + c];
                    } else {                                  // element (i = a, j = c) = B[a][c]
                        if (a < P.olen && c < P.klen) S.b[c * BS + a] = B[(int64_t)a * P.b_ld + c];
                    }
                }
                __syncthreads();
                if (i < P.olen) {
                    // one chain per right-hand side over all K indices, on the grid of the
                    // product's largest output-row 1-norm times the input's largest component
                    const float bo = pbnd[p].x;
                    float sg[QN];
                    cxacc c[QN];
#pragma unroll
                    for (int q = 0; q < QN; ++q) {
                        sg[q] = grid_sigma(bo, x_max(S.mx, QN * hh + q));
                        cx_start(c[q], sg[q]);
                    }
#pragma unroll 4
                    for (int j = 0; j < P.klen; ++j) {
                        const float2 bv = S.b[j * BS + i];
                        const float4 *xv = reinterpret_cast<const float4 *>(S.x + j * XS + QN * hh);
#pragma unroll
                        for (int q = 0; q < QN / 2; ++q) {
                            const float4 v = xv[q];
                            cxstep(c[2 * q], bv, make_float2(v.x, v.y));
                            cxstep(c[2 * q + 1], bv, make_float2(v.z, v.w));
                        }
                    }
#pragma unroll
                    for (int q = 0; q < QN; ++q) acc[q] = cdf_add(acc[q], cxclose(c[q], sg[q]));
                }
            } else {
                // W (rank rows l, K j) into b[j * WS + l]; Y (element (i, l) = Y[l][i]) into y[l * BS + i]
                float2 *Wsm = S.b, *Ysm = S.b + 64 * WS;
                const float2 *W = pool + P.b_off, *Y = pool + P.y_off;
                for (int e = tid; e < P.rank * 64; e += RT) {
                    const int l = e >> 6, c = e & 63;
                    if (c < P.klen) Wsm[c * WS + l] = W[(int64_t)l * P.b_ld + c];
                    if (c < P.olen) Ysm[l * BS + c] = Y[(int64_t)l * P.y_ld + c];
                }
                __syncthreads();
                // stage 1: T[l][q] = sum_j W[l][j] x[j][q]; a round covers 128 / (4 RG) rank rows;
                // thread (row l0 + tid / (4 RG), q = (tid / 4) % RG, K slice ks = tid % 4: j = ks,
                // ks + 4, ...); the four slices' chains share the grid of W's largest rank-row
                // 1-norm times x's largest component, so their grid parts add exactly across lanes
                const float2 bb = pbnd[p];
                {
                    constexpr int NS = 2;                          // K slices per rank row and RHS
                    constexpr int LR = RT / (NS * RG);             // rank rows per round
                    const int ks = tid % NS, q = (tid / NS) % RG, lr = tid / (NS * RG);
                    const float s1 = grid_sigma(bb.x, x_max(S.mx, q));
                    for (int l0 = 0; l0 < P.rank; l0 += LR) {
                        const int l = l0 + lr;
                        cxacc c;
                        cx_start(c, s1);
                        if (l < P.rank)
                            for (int j = ks; j < P.klen; j += NS) cxstep(c, Wsm[j * WS + l], S.x[j * XS + q]);
                        float v[4] = {__fsub_rn(c.re.tau, s1), c.re.r, __fsub_rn(c.im.tau, s1), c.im.r};
#pragma unroll
                        for (int sh = 1; sh < NS; sh <<= 1)
#pragma unroll
                            for (int e = 0; e < 4; ++e) v[e] = __fadd_rn(v[e], __shfl_xor_sync(FULL, v[e], sh));
                        if (ks == 0 && l < P.rank) S.t[l * RG + q] = {{v[0], v[1]}, {v[2], v[3]}};
                    }
                }
                __syncthreads();
                // stage 2: out[i][q] += sum_l Y[i][l] T[l][q], one chain per right-hand side over
                // all rank rows: the leading part of T[l][q] is a grid sum, at most half of
                // stage 1's sigma, which bounds the inputs with Y's largest output-row 1-norm
                if (i < P.olen) {
                    float sg[QN];
                    cxacc c[QN];
#pragma unroll
                    for (int q = 0; q < QN; ++q) {
                        sg[q] = grid_sigma(bb.y, 0.5f * grid_sigma(bb.x, x_max(S.mx, QN * hh + q)));
                        cx_start(c[q], sg[q]);
                    }
                    for (int l = 0; l < P.rank; ++l) {
                        const float2 yv = Ysm[l * BS + i];
#pragma unroll
                        for (int q = 0; q < QN; ++q) cxstep_df(c[q], yv, S.t[l * RG + QN * hh + q]);
                    }
#pragma unroll
                    for (int q = 0; q < QN; ++q) acc[q] = cdf_add(acc[q], cxclose(c[q], sg[q]));
                }
            }
        }
        if (i < U.mlen) {
#pragma unroll
            for (int q = 0; q < QN; ++q) {
                const int r = QN * hh + q;
                if (r < nr) own[(int64_t)(r0 + r) * ldo + U.out0 + i] = to_d2(acc[q]);
            }
        }
    }
}

// Per leaf (blockIdx.x) and right-hand side (blockIdx.y): acc = D_I x_I (Dot2) +
// the owner sums of levels 1..m at the leaf's rows (FP64), in a fixed order.  If b
// is given, out = b - acc (FP64, rounded to complex64) and |r|^2, |b|^2 go to
// norms; else out = acc (complex64).  x of the leaf is staged in dynamic shared
// memory (np entries).
__global__ void __launch_bounds__(64)
k_gather_own(const int32_t *__restrict__ pleaf_off, const int64_t *__restrict__ dinv_off,
             const float2 *__restrict__ self32, const float2 *__restrict__ x, int64_t ld, int m,
             const double2 *__restrict__ own, int64_t lstride, const float2 *__restrict__ b, float2 *__restrict__ out,
             double *norms)
{
    extern __shared__ __align__(16) unsigned char gsm[];
    float2 *xs = reinterpret_cast<float2 *>(gsm);
    const int leaf = blockIdx.x, r = blockIdx.y, tid = threadIdx.x, lane = tid & 31;
    const int o = pleaf_off[leaf], np = pleaf_off[leaf + 1] - o;
    double rr = 0.0, bb = 0.0;
    for (int j = tid; j < np; j += 64) xs[j] = x[r * ld + o + j];
    __syncthreads();
    const float2 *Sd = self32 + dinv_off[leaf];                 // column-major np x np
    for (int i = tid; i < np; i += 64) {
        const int64_t g = r * ld + o + i;
        cdf dx = cdf_zero();
        for (int j = 0; j < np; ++j) cdot2(dx, Sd[(int64_t)j * np + i], xs[j]);
        double2 acc = to_d2(dx);
        for (int lev = 0; lev < m; ++lev) acc = cadd(acc, own[lev * lstride + g]);
        if (b) {
            const double2 bv = conv<double2>(b[g]);
            const double2 rv = csub(bv, acc);
            out[g] = make_float2((float)rv.x, (float)rv.y);
            rr += rv.x * rv.x + rv.y * rv.y;
            bb += bv.x * bv.x + bv.y * bv.y;
        } else {
            out[g] = make_float2((float)acc.x, (float)acc.y);
        }
    }
    if (norms) {
        for (int s = 16; s >= 1; s >>= 1) {
            rr += __shfl_xor_sync(FULL, rr, s);
            bb += __shfl_xor_sync(FULL, bb, s);
        }
        if (lane == 0) {
            atomicAdd(&norms[2 * r], rr);
            atomicAdd(&norms[2 * r + 1], bb);
        }
    }
}

// Per directed product, the bounds its common grids take (k_resid_own): x = the
// largest 1-norm of an output row of the oriented block (dense) or of a rank row of
// the input-side factor W (low-rank, stage 1); y = the largest 1-norm, over the rank
// rows, of an output row of Y (low-rank, stage 2).  FP64 sums rounded up; one warp
// per product.
__global__ void __launch_bounds__(256)
k_prod_bounds(const TcProd *__restrict__ prods, int64_t n, const float2 *__restrict__ pool, float2 *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < n; t += nw) {
        const TcProd P = prods[t];
        double a = 0.0, b = 0.0, c = 0.0, d = 0.0;
        if (P.rank == 0) {
            if (P.trans) l1_bounds(pool + P.b_off, P.klen, P.olen, P.b_ld, c, a, lane);   // output i = column i
            else l1_bounds(pool + P.b_off, P.olen, P.klen, P.b_ld, a, c, lane);
        } else {
            l1_bounds(pool + P.b_off, P.rank, P.klen, P.b_ld, a, c, lane);
            l1_bounds(pool + P.y_off, P.rank, P.olen, P.y_ld, d, b, lane);
        }
        if (lane == 0) out[t] = make_float2(__double2float_ru(a), __double2float_ru(b));
    }
}

} // namespace

void launch_prod_bounds(const TcProd *prods, int64_t n, const float2 *pool, float2 *out, cudaStream_t s)
{
    if (n <= 0) return;
    const int g = (int)std::min<int64_t>((n + 7) / 8, 152 * 16);
    k_prod_bounds<<<g, 256, 0, s>>>(prods, n, pool, out);
}

// owner-computes FP64-class products of a level's small items: own[r * pN + i] = (M_level x_r)_i
// for the level's output rows (a level whose items are all small; the rest of own is untouched)
void launch_resid_own(hm_matrix h, const LevelList &L, const float2 *x, double2 *own, int nrhs, cudaStream_t s)
{
    if (L.n_rcu == 0 || nrhs <= 0) return;
    constexpr int SMEM = (int)sizeof(Smem);
    static bool attr = false;
    if (!attr) {
        for (const void *f : {(const void *)k_resid_own<8, 128>, (const void *)k_resid_own<16, 128>,
                              (const void *)k_resid_own<8, 256>, (const void *)k_resid_own<16, 256>}) {
            cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
            cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
        }
        attr = true;
    }
    // groups of 8 right-hand sides up to 32 of them, so that small calls still have enough units.
    // four CTAs of ~50 KB per SM: of 256 threads (4 RHS per thread, 64 registers) up to 128 RHS,
    // of 128 threads (8 RHS per thread) above: measured on the 30,720-unknown sphere, 0.499 /
    // 0.365 ms per RHS at 16 / 64 RHS against 0.587 / 0.406 for 128 threads, and 0.382 against
    // 0.386 for 256 threads at 181
    const int rg = nrhs <= 32 ? 8 : 16;
    const bool wide = nrhs <= 128;
    const int64_t units = L.n_rcu * (int64_t)((nrhs + rg - 1) / rg);
    int64_t g = 4 * (int64_t)(h->num_sms > 0 ? h->num_sms : 1);
    if (g > units) g = units;
    auto go = [&](auto kern, int rt) {
        kern<<<(unsigned)g, rt, SMEM, s>>>(L.d_rcu, (int)L.n_rcu, L.d_rcp, L.d_rcb, h->d_pool32, x, h->pN, nrhs, own,
                                           h->pN);
    };
    if (rg == 8) wide ? go(k_resid_own<8, 256>, 256) : go(k_resid_own<8, 128>, 128);
    else wide ? go(k_resid_own<16, 256>, 256) : go(k_resid_own<16, 128>, 128);
}

void launch_gather_own(hm_matrix h, const float2 *x, int m, const double2 *own, int64_t lstride, const float2 *b,
                       float2 *out, double *norms, int nrhs, cudaStream_t s)
{
    dim3 grid((unsigned)h->n_leaves, (unsigned)nrhs);
    int64_t maxnp = 0;
    for (int64_t i = 0; i < h->n_leaves; ++i) maxnp = std::max<int64_t>(maxnp, h->pleaf_off[i + 1] - h->pleaf_off[i]);
    k_gather_own<<<grid, 64, sizeof(float2) * (size_t)std::max<int64_t>(maxnp, 1), s>>>(
        h->d_pleaf_off, h->d_dinv_off, h->d_self32, x, h->pN, m, own, lstride, b, out, norms);
}

} // namespace hm
