// Host-side check of the block products' work lists (csrc/hm_lists.h): builds the
// directed products, the owner-computes residual's units and the tensor-core
// product's two-launch lists for a random set of small blocks, and checks every
// property the kernels rely on; also the snake order the persistent product and
// residual kernels take their blocks in (each block once, warp sums within the
// largest cost of one another).  Prints "ok ..." and exits 0, or prints the first
// violation and exits 1.
//
// usage: tc_lists_check <seed> <mode>
//   mode 0: random cluster lengths 1..64, dense and low-rank blocks, ranks 1..32
//   mode 1: every rank 32 (batches of two products of 32 rows)
//   mode 2: every rank 1 (batches of eight products of one row and seven zero rows)
//   mode 3: no blocks at all
//   mode 4: one dense block on the diagonal cluster pair (both directed products into one cluster)
//   mode 5: mode 0 with two entries of the chunk table swapped after the build (must FAIL)
//   mode 6: mode 0 with one batch moved by a group of 8 rows after the build (must FAIL)
//   mode 7: mode 0 with the blocks handed out in build order, unsorted (must FAIL the
//           balance check)
#include "hm_lists.h"

#include <cstdio>
#include <cstdlib>
#include <random>
#include <set>
#include <tuple>

using namespace hm;

static int fail(const char *what)
{
    std::printf("FAIL %s\n", what);
    return 1;
}

int main(int argc, char **argv)
{
    if (argc < 3) return fail("usage");
    const int seed = std::atoi(argv[1]), mode = std::atoi(argv[2]);
    std::mt19937 rng(seed);
    auto uni = [&](int lo, int hi) { return std::uniform_int_distribution<int>(lo, hi)(rng); };

    // clusters at padded offsets 64 apart, lengths 1..64; blocks on random cluster pairs
    const int ncl = 48;
    std::vector<int> len(ncl), off(ncl);
    for (int i = 0; i < ncl; ++i) {
        len[i] = uni(1, 64);
        off[i] = 64 * i;
    }
    std::vector<Item> items;
    int64_t pool = 0;
    auto add = [&](int i, int j, int k) {
        Item it{pool, off[i], off[j], len[i], len[j], k, 0};
        pool += item_elems(it) + (item_elems(it) & 1);
        items.push_back(it);
    };
    if (mode == 4) {
        add(3, 3, 0);
    } else if (mode != 3) {
        for (int i = 0; i < ncl; ++i)
            for (int j = i; j < ncl; ++j) {
                if (uni(0, 2) != 0) continue;
                const int k = mode == 1 ? 32 : mode == 2 ? 1 : (uni(0, 1) ? uni(1, 32) : 0);   // modes 0, 5-7
                add(i, j, k);
            }
    }

    const auto by_out = directed_products(items);
    std::vector<TcUnit> runits;
    std::vector<TcProd> rprods;
    build_owner_lists(by_out, runits, rprods);
    TcLists T;
    if (!build_tc_lists(by_out, T)) return fail("builder rejected its own lists");
    if (mode == 5 && T.tchunks.size() >= 2) std::swap(T.tchunks[0], T.tchunks[1]);
    if (mode == 6 && T.batches.size() >= 2) T.batches[1].row0 += 8;

    // directed products: two per block, into its row and its column cluster
    size_t nprod = 0;
    for (auto &kv : by_out) nprod += kv.second.size();
    if (nprod != 2 * items.size()) return fail("two directed products per block");

    // owner lists: every directed product once, units by output cluster, largest first
    if (rprods.size() != nprod || runits.size() != by_out.size()) return fail("owner list sizes");
    int64_t last_cost = INT64_MAX;
    for (const TcUnit &u : runits) {
        const auto &want = by_out.at(u.out0);
        if (u.p1 - u.p0 != (int32_t)want.size()) return fail("owner unit size");
        int64_t c = 0;
        int32_t mlen = 0;
        for (int32_t p = u.p0; p < u.p1; ++p) {
            const TcProd &P = rprods[p];
            c += (P.klen + 7) / 8 + (P.rank > 0 ? (P.rank + 7) / 8 : 0);
            mlen = std::max(mlen, P.olen);
        }
        if (c > last_cost) return fail("owner units not largest first");
        if (mlen != u.mlen) return fail("owner unit mlen");
        last_cost = c;
    }

    // split-x chunks: each input cluster's chunks cover its longest input in steps of 8
    std::map<int32_t, int32_t> in_len;
    for (auto &kv : by_out)
        for (const TcProd &p : kv.second) in_len[p.in0] = std::max(in_len[p.in0], p.klen);
    {
        size_t g = 0;
        for (auto &kv : in_len)
            for (int32_t c = 0; c < kv.second; c += 8, ++g) {
                if (g >= T.xch.size()) return fail("split-x chunk count");
                if (T.xch[g].off != kv.first + c || T.xch[g].len != std::min(8, kv.second - c))
                    return fail("split-x chunk");
            }
        if (g != T.xch.size()) return fail("split-x chunk count");
    }

    // batches: whole 8-row groups, at most 64 rows, every T chunk exactly once
    std::vector<std::pair<int, int>> chunk_at(T.n_tchunk, {-1, -1});   // T chunk -> (first row, batch)
    for (size_t b = 0; b < T.batches.size(); ++b) {
        const TcBatch &B = T.batches[b];
        if (B.nrows <= 0 || B.nrows > 64 || (B.nrows & 7) || (B.row0 & 7)) return fail("batch shape");
        if (B.xg0 < 0 || B.xg0 + (B.klen + 7) / 8 > (int64_t)T.xch.size()) return fail("batch split-x range");
        for (int g = 0; g < B.nrows / 8; ++g) {
            const int32_t t = T.tchunks[B.row0 / 8 + g];
            if (t < 0 || t >= T.n_tchunk) return fail("T chunk out of range");
            if (chunk_at[t].first >= 0) return fail("T chunk written twice");
            chunk_at[t] = {B.row0 + 8 * g, (int)b};
        }
    }
    for (auto &c : chunk_at)
        if (c.first < 0) return fail("T chunk never written");
    if ((int64_t)T.tchunks.size() * 8 != (int64_t)T.rows.size()) return fail("chunk table size");

    // second-launch operations: exactly the directed products, each in a unit of its output cluster
    using Key = std::tuple<int64_t, int32_t, int32_t, int32_t, int32_t>;   // src, kind, klen, ld, olen
    std::map<int32_t, std::multiset<Key>> want_ops;
    std::map<int64_t, TcProd> lowrank_by_y;
    for (auto &kv : by_out)
        for (const TcProd &p : kv.second) {
            if (p.rank == 0) {
                want_ops[kv.first].insert(Key{p.b_off, p.trans ? 1 : 0, p.klen, p.b_ld, p.olen});
            } else {
                want_ops[kv.first].insert(Key{p.y_off, 2, p.rank, p.y_ld, p.olen});
                if (lowrank_by_y.count(p.y_off)) return fail("two low-rank products with one Y");
                lowrank_by_y[p.y_off] = p;
            }
        }
    std::map<int32_t, std::multiset<Key>> got_ops;
    std::vector<int> seen(T.ops.size(), 0);
    for (const TcUnit &u : T.units) {
        if (u.p0 < 0 || u.p1 <= u.p0 || u.p1 > (int32_t)T.ops.size()) return fail("unit range");
        int64_t c = 0;
        for (int32_t p = u.p0; p < u.p1; ++p) {
            const TcOp &o = T.ops[p];
            ++seen[p];
            c += (o.klen + 7) / 8;
            if (o.olen > u.mlen) return fail("operation longer than its unit");
            got_ops[u.out0].insert(Key{o.src, o.kind, o.klen, o.ld, o.olen});
            if (o.kind == 2) {
                // its T chunks hold its W rows in order, zero rows past the rank, in batches
                // over its own input cluster and length
                const TcProd &P = lowrank_by_y.at(o.src);
                for (int l = 0; l < ((P.rank + 7) & ~7); ++l) {
                    const auto at = chunk_at[o.t0 + l / 8];
                    const int64_t row = T.rows[at.first + l % 8];
                    const int64_t want = l < P.rank ? P.b_off + (int64_t)l * P.b_ld : -1;
                    if (row != want) return fail("stacked row");
                    const TcBatch &B = T.batches[at.second];
                    if (B.klen != P.klen || T.xch[B.xg0].off != P.in0) return fail("batch input cluster");
                }
            } else if (o.xg0 < 0 || o.xg0 + (o.klen + 7) / 8 > (int64_t)T.xch.size()) {
                return fail("dense operation's split-x range");
            }
        }
        if (c > TC_UNIT_CHUNKS && u.p1 - u.p0 > 1) return fail("unit over the chunk cap");
    }
    for (int v : seen)
        if (v != 1) return fail("operation not in exactly one unit");
    if (got_ops != want_ops) return fail("operations differ from the directed products");
    // dense operations read the split x of their own input cluster
    for (auto &kv : by_out)
        for (const TcProd &p : kv.second)
            if (p.rank == 0) {
                bool found = false;
                for (const TcOp &o : T.ops)
                    if (o.kind != 2 && o.src == p.b_off && o.kind == (p.trans ? 1 : 0))
                        found = found || T.xch[o.xg0].off == p.in0;
                if (!found) return fail("dense operation's split x");
            }

    // snake order for nw round-robin warps: a permutation of the blocks, and no two warps'
    // cost sums more than the largest cost apart
    for (int pass = 0; pass < 2; ++pass)
        for (int64_t nw : {1, 7, 64, 1000}) {
            auto cost = [&](const Item &it) { return pass == 0 ? product_cost(it) : residual_cost(it); };
            std::vector<Item> ord = balanced_order(items, nw, cost);
            if (mode == 7) ord = items;
            if (ord.size() != items.size()) return fail("snake order size");
            std::multiset<int64_t> a, b;
            for (const Item &it : items) a.insert(it.off);
            for (const Item &it : ord) b.insert(it.off);
            if (a != b) return fail("snake order is not a permutation");
            const int64_t w = std::min<int64_t>(nw, std::max<int64_t>((int64_t)ord.size(), 1));
            std::vector<int64_t> sum(w, 0);
            int64_t cmax = 0;
            for (size_t t = 0; t < ord.size(); ++t) {
                sum[t % w] += cost(ord[t]);
                cmax = std::max(cmax, cost(ord[t]));
            }
            if (!ord.empty() && *std::max_element(sum.begin(), sum.end()) - *std::min_element(sum.begin(), sum.end()) > cmax)
                return fail("snake order unbalanced");
        }

    std::printf("ok blocks=%zu ops=%zu units=%zu batches=%zu rows=%zu tchunks=%lld\n", items.size(), T.ops.size(),
                T.units.size(), T.batches.size(), T.rows.size(), (long long)T.n_tchunk);
    return 0;
}
