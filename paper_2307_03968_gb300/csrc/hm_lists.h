// Work lists of the block products: the host logic that orders the stored blocks
// for the kernels (plain C++, no CUDA types, so that the CPU tests compile it with
// the host compiler; hm_internal.h includes it).
//  - Item: one stored block, the work item of the product and residual kernels.
//  - TcProd / TcUnit: the directed products of the small blocks (each block gives two,
//    eq. 6 and eq. 8 with the half storage of §III of arxiv 2307.03968), grouped by
//    output cluster.
//  - TcOp / TcBatch / XChunk: the tensor-core product's two launches (k_mrhs_tc.cu).
#pragma once

#include <algorithm>
#include <climits>
#include <cstdint>
#include <map>
#include <utility>
#include <vector>

#ifdef __CUDACC__
#define HM_HD __host__ __device__
#else
#define HM_HD
#endif

namespace hm {

constexpr int MRHS_MAX_DIM = 64;    // largest block side of the multi-RHS product kernel
constexpr int MRHS_MAX_RANK = 32;   // largest rank of a low-rank block it takes
constexpr int TC_MAX_DIM = MRHS_MAX_DIM;    // the tensor-core product takes the same small items
constexpr int TC_MAX_RANK = MRHS_MAX_RANK;
constexpr int TC_UNIT_CHUNKS = 64;  // K chunks (of 8) a tensor-core work unit sums in tensor memory

// One stored block = one work item of the product kernels (32 bytes).
struct Item {
    int64_t off;    // complex-element offset into the pool
    int32_t row0;   // padded-tree offset of the row cluster
    int32_t col0;   // padded-tree offset of the column cluster
    int32_t m, n;   // padded cluster lengths (dense: m = true rows, n = true cols)
    int32_t k;      // rank; 0 = dense block
    int32_t pad;    // offset of the block's partial slots (row side, then column side)
};
static_assert(sizeof(Item) == 32, "Item layout");

// One directed product of a small stored block into an output cluster (the
// owner-computes residual, k_resid_own.cu): Z_out += B X_in with B the block (dense,
// read row-major or transposed) or, for a low-rank block, Y (W X_in) with the
// input-side factor W read row-major (rank rows) and the output-side factor Y
// read transposed.
struct TcProd {
    int64_t b_off;   // complex offset of the block (dense) or of W (low-rank)
    int64_t y_off;   // complex offset of Y (low-rank)
    int32_t in0;     // padded-tree offset of the input cluster
    int32_t klen;    // input length (K of the dense product and of stage 1)
    int32_t rank;    // 0 = dense
    int32_t b_ld;    // row stride of the block / of W
    int32_t y_ld;    // row stride of Y as stored (rank rows)
    int32_t trans;   // dense: 1 = element (out i, in j) is block[j][i] (the mirror product)
    int32_t olen;    // output length of this product
    int32_t xg0;     // first K chunk of the input cluster in the level's split-x chunk list
};
static_assert(sizeof(TcProd) == 48, "TcProd layout");
// a work unit: products [p0, p1) into the output cluster at out0 (mlen = largest olen)
struct TcUnit { int32_t out0, mlen, p0, p1; };

// The tensor-core product (k_mrhs_tc.cu) in two launches.  The first runs stage 1 of
// every low-rank directed product, T = W X_in, batched over the products that share
// an input cluster (their W rows stacked along N); it stores T in chunks of 8 rank
// rows (TC_T_CHUNK floats per chunk and RHS tile).  The second runs, per output
// cluster, the dense products and the second stages Y T, which read T back.
constexpr int TC_T_CHUNK = 2 * 128 * 8;   // floats of one T chunk: Re and Im planes of 128 RHS x 8 rank rows
// one operation of the second launch
struct TcOp {
    int64_t src;     // complex offset of the dense block, or of Y (low-rank second stage)
    int64_t t0;      // low-rank: first T chunk of the product (per RHS tile)
    int32_t kind;    // 0 dense (element (out i, in j) = block[i][j]), 1 dense mirror (= block[j][i]), 2 Y T
    int32_t klen;    // K length: the input length (dense) or the rank
    int32_t ld;      // row stride of the block or of Y as stored (rank rows)
    int32_t olen;    // output length
    int32_t xg0;     // dense: first split-x chunk of the input cluster
    int32_t pad;
};
static_assert(sizeof(TcOp) == 40, "TcOp layout");
// a batch of the first launch: stacked rows [row0, row0 + nrows) (nrows a multiple of
// 8, at most 64) of the row table, all over one input cluster (split-x chunks from xg0,
// K length klen); each row's W offset (-1: a zero row) is in the row table, each group
// of 8 rows' T chunk in the chunk table (index row / 8)
struct TcBatch { int32_t xg0, klen, row0, nrows; };
// a K chunk of an input cluster for the split x: padded-tree offset and valid length (<= 8)
struct XChunk { int32_t off, len; };

HM_HD inline int64_t even(int64_t v) { return (v + 1) & ~int64_t(1); }

HM_HD inline int64_t item_elems(const Item &it)
{
    if (it.k == 0) return int64_t(it.m) * even(it.n);
    return int64_t(it.k) * (even(it.m) + even(it.n));
}

// The directed products of the small items: every item gives two (into its row
// cluster and, mirrored, into its column cluster), grouped by output cluster.
inline std::map<int32_t, std::vector<TcProd>> directed_products(const std::vector<Item> &small)
{
    std::map<int32_t, std::vector<TcProd>> by_out;
    auto add = [&](int32_t out0, const TcProd &p) {
        if (p.klen > 0 && p.olen > 0) by_out[out0].push_back(p);
    };
    for (const Item &it : small) {
        if (it.k == 0) {
            const int32_t ld = (int32_t)even(it.n);
            add(it.row0, TcProd{it.off, 0, it.col0, it.n, 0, ld, 0, 0, it.m, 0});
            add(it.col0, TcProd{it.off, 0, it.row0, it.m, 0, ld, 0, 1, it.n, 0});
        } else {
            const int32_t lm = (int32_t)even(it.m), ln = (int32_t)even(it.n);
            const int64_t uoff = it.off, voff = it.off + (int64_t)it.k * lm;
            add(it.row0, TcProd{voff, uoff, it.col0, it.n, it.k, ln, lm, 0, it.m, 0});   // U (V x_J)
            add(it.col0, TcProd{uoff, voff, it.row0, it.m, it.k, lm, ln, 0, it.n, 0});   // V^T (U^T x_I)
        }
    }
    return by_out;
}

// The owner-computes residual's list: one unit per output cluster (every output row
// summed by one CTA in a fixed order), largest first.
inline void build_owner_lists(const std::map<int32_t, std::vector<TcProd>> &by_out, std::vector<TcUnit> &runits,
                              std::vector<TcProd> &rprods)
{
    auto cost = [](const TcProd &p) {
        return (int64_t)((p.klen + 7) / 8) + (p.rank > 0 ? (int64_t)((p.rank + 7) / 8) : 0);
    };
    struct R { TcUnit u; int64_t c; const std::vector<TcProd> *p; };
    std::vector<R> rs;
    for (auto &kv : by_out) {
        R r{TcUnit{kv.first, 0, 0, 0}, 0, &kv.second};
        for (const TcProd &p : kv.second) { r.u.mlen = std::max(r.u.mlen, p.olen); r.c += cost(p); }
        rs.push_back(r);
    }
    std::stable_sort(rs.begin(), rs.end(), [](const R &a, const R &b) { return a.c > b.c; });
    runits.clear();
    rprods.clear();
    for (R &r : rs) {
        r.u.p0 = (int32_t)rprods.size();
        rprods.insert(rprods.end(), r.p->begin(), r.p->end());
        r.u.p1 = (int32_t)rprods.size();
        runits.push_back(r.u);
    }
}

// The tensor-core product's lists (k_mrhs_tc.cu), two launches.
//  - Stage 1 of every low-rank directed product, T = W X_in (W = V forward, U^T mirrored),
//    is batched over the products that share an input cluster: each product takes
//    roundup8(rank) stacked rows (rows past its rank are zero) and as many T chunks, and a
//    batch stacks up to 64 rows, so one K chunk of split x feeds MMAs of N up to 128.
//  - The second launch takes, per output cluster, the dense products and the second
//    stages Y T (Y = U forward, V^T mirrored; T read back by chunk), cut into units of at
//    most TC_UNIT_CHUNKS K chunks (units of one cluster add into z with atomics) and sorted
//    by cost, largest first, so that the persistent CTAs taking units in turn stay balanced.
// Returns false when a list would break an index bound the kernels rely on.
struct TcLists {
    std::vector<TcUnit> units;
    std::vector<TcOp> ops;
    std::vector<XChunk> xch;
    std::vector<TcBatch> batches;
    std::vector<int64_t> rows;
    std::vector<int32_t> tchunks;
    int64_t n_tchunk = 0;
};
inline bool build_tc_lists(const std::map<int32_t, std::vector<TcProd>> &by_out, TcLists &T)
{
    // K chunks of the input clusters (each cluster's longest input length)
    std::map<int32_t, int32_t> in_len;
    for (auto &kv : by_out)
        for (const TcProd &p : kv.second) in_len[p.in0] = std::max(in_len[p.in0], p.klen);
    std::map<int32_t, int32_t> in_g0;
    T.xch.clear();
    for (auto &kv : in_len) {
        in_g0[kv.first] = (int32_t)T.xch.size();
        for (int32_t c = 0; c < kv.second; c += 8) T.xch.push_back(XChunk{kv.first + c, std::min(8, kv.second - c)});
    }
    // stage-1 jobs by (input cluster, K length), each with its first T chunk
    struct Job { int64_t w_off; int32_t w_ld, rank; int64_t t0; };
    std::map<std::pair<int32_t, int32_t>, std::vector<Job>> by_in;
    T.n_tchunk = 0;
    // second-launch operations per output cluster
    auto chunks = [](int32_t klen) { return (int64_t)((klen + 7) / 8); };
    const int64_t cap = TC_UNIT_CHUNKS;
    struct U { TcUnit u; int64_t c; std::vector<TcOp> p; };
    std::vector<U> us;
    for (auto &kv : by_out) {
        int32_t mlen = 0;
        for (const TcProd &p : kv.second) mlen = std::max(mlen, p.olen);
        U cur{TcUnit{kv.first, mlen, 0, 0}, 0, {}};
        for (const TcProd &p : kv.second) {
            TcOp op{};
            op.olen = p.olen;
            if (p.rank == 0) {
                op.src = p.b_off;
                op.kind = p.trans ? 1 : 0;
                op.klen = p.klen;
                op.ld = p.b_ld;
                op.xg0 = in_g0[p.in0];
            } else {
                op.src = p.y_off;
                op.t0 = T.n_tchunk;
                op.kind = 2;
                op.klen = p.rank;
                op.ld = p.y_ld;
                by_in[{p.in0, p.klen}].push_back(Job{p.b_off, p.b_ld, p.rank, T.n_tchunk});
                T.n_tchunk += chunks(p.rank);
            }
            // Units of at most TC_UNIT_CHUNKS K chunks: the tensor cores' FP32 accumulator loses
            // a little on every MMA it adds into a large running sum (measured: the product's
            // error grows in proportion to the chunks summed in tensor memory, 7.4e-6 relative
            // at 256 chunks, 1.9e-6 at 64, 5.4e-7 at 16 on 60-unknown leaves), so a unit's sum
            // leaves tensor memory (added into z in FP32) every TC_UNIT_CHUNKS chunks.
            if (cur.c > 0 && cur.c + chunks(op.klen) > cap) {
                us.push_back(cur);
                cur.c = 0;
                cur.p.clear();
            }
            cur.p.push_back(op);
            cur.c += chunks(op.klen);
        }
        if (!cur.p.empty()) us.push_back(cur);
    }
    std::stable_sort(us.begin(), us.end(), [](const U &a, const U &b) { return a.c > b.c; });
    T.units.clear();
    T.ops.clear();
    for (U &x : us) {
        x.u.p0 = (int32_t)T.ops.size();
        T.ops.insert(T.ops.end(), x.p.begin(), x.p.end());
        x.u.p1 = (int32_t)T.ops.size();
        T.units.push_back(x.u);
    }
    // stage-1 batches of at most 64 stacked rows
    T.batches.clear();
    T.rows.clear();
    T.tchunks.clear();
    for (auto &kv : by_in) {
        const int32_t xg0 = in_g0[kv.first.first], klen = kv.first.second;
        TcBatch b{xg0, klen, (int32_t)T.rows.size(), 0};
        for (const Job &j : kv.second) {
            const int32_t k8 = (j.rank + 7) & ~7;
            if (b.nrows + k8 > 64) {
                T.batches.push_back(b);
                b = TcBatch{xg0, klen, (int32_t)T.rows.size(), 0};
            }
            for (int32_t l = 0; l < k8; ++l) T.rows.push_back(l < j.rank ? j.w_off + (int64_t)l * j.w_ld : -1);
            for (int32_t g = 0; g < k8 / 8; ++g) T.tchunks.push_back((int32_t)(j.t0 + g));
            b.nrows += k8;
        }
        if (b.nrows > 0) T.batches.push_back(b);
    }
    // the bounds the kernels index by
    if (T.n_tchunk > INT32_MAX || (int64_t)T.rows.size() > INT32_MAX || T.ops.size() > (size_t)INT32_MAX) return false;
    if ((int64_t)T.tchunks.size() * 8 != (int64_t)T.rows.size()) return false;
    for (const TcBatch &b : T.batches)
        if (b.nrows <= 0 || b.nrows > 64 || (b.nrows & 7) || b.row0 < 0 || (b.row0 & 7) ||
            b.row0 + (int64_t)b.nrows > (int64_t)T.rows.size() ||
            b.xg0 + chunks(b.klen) > (int64_t)T.xch.size())
            return false;
    for (int32_t t : T.tchunks)
        if (t < 0 || t >= T.n_tchunk) return false;
    for (const TcOp &o : T.ops) {
        if (o.olen <= 0 || o.olen > TC_MAX_DIM || o.klen <= 0) return false;
        if (o.kind == 2 ? (o.klen > TC_MAX_RANK || o.t0 + chunks(o.klen) > T.n_tchunk)
                        : (o.klen > TC_MAX_DIM || o.xg0 + chunks(o.klen) > (int64_t)T.xch.size()))
            return false;
    }
    for (const TcUnit &u : T.units)
        if (u.mlen > TC_MAX_DIM || u.p0 < 0 || u.p1 <= u.p0 || u.p1 > (int32_t)T.ops.size()) return false;
    return true;
}

// items reordered for a persistent kernel whose nw warps take items t, t + nw, ...:
// sorted by cost, largest first, and every odd round of nw reversed (a snake), so that
// the warps' sums match.  Cost of the product: stored bytes plus a fixed 2 KB for the
// per-block latencies; of the FP64-class residual (instruction-bound): about 39 lane
// instructions per stored element of a dense block, 52 of a low-rank one, plus 3,000.
inline int64_t product_cost(const Item &it) { return item_elems(it) * 8 + 2048; }
inline int64_t residual_cost(const Item &it) { return item_elems(it) * (it.k == 0 ? 39 : 52) + 3000; }
template <class Cost>
inline std::vector<Item> balanced_order(const std::vector<Item> &in, int64_t nw, Cost cost)
{
    std::vector<Item> v = in;
    std::stable_sort(v.begin(), v.end(), [&](const Item &a, const Item &b) { return cost(a) > cost(b); });
    const int64_t n = (int64_t)v.size();
    nw = std::min<int64_t>(std::max<int64_t>(nw, 1), std::max<int64_t>(n, 1));
    std::vector<Item> out(v.size());
    for (int64_t t = 0; t < n; ++t) {
        const int64_t q = t / nw, p = t % nw, rem = std::min<int64_t>(nw, n - q * nw);
        out[t] = v[q * nw + ((q & 1) ? rem - 1 - p : p)];
    }
    return out;
}

} // namespace hm
