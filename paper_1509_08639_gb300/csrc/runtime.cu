// runtime.cu -- host side of the miner: the C ABI of include/mine.h.
//
// Contexts own a stream, a growable scratch arena for the synchronous batch
// calls, two sets of buffers (and a copy stream each way) for host-buffer
// batch calls in flight, and a serving engine: a host thread that forms
// batches from submitted article pairs (continuous batching), admits them
// against a fixed device-memory pool (the budget), runs up to max_inflight
// batches at once on their own streams, and hands results to mine_poll.
#include "internal.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

using namespace mine;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

#define CK(call)                                                                       \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return fail(MINE_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

int ceil_log2_host(int64_t x)
{
    return x <= 1 ? 0 : 64 - __builtin_clzll((unsigned long long)(x - 1));
}

int64_t align_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// ------------------------------------------------------------------ buffers

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
    ~DevBuf()
    {
        if (p) cudaFree(p);
    }
};

int ensure_dev(DevBuf &b, size_t bytes)
{
    if (bytes <= b.cap && b.p) return 0;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
    const size_t nb = std::max<size_t>(bytes + bytes / 4, 1 << 16);
    CK(cudaMalloc(&b.p, nb));
    b.cap = nb;
    return 0;
}

struct HostBuf {
    void *p = nullptr;
    size_t cap = 0;
    ~HostBuf()
    {
        if (p) cudaFreeHost(p);
    }
};

int ensure_host(HostBuf &b, size_t bytes)
{
    if (bytes <= b.cap && b.p) return 0;
    if (b.p) cudaFreeHost(b.p);
    b.p = nullptr;
    b.cap = 0;
    const size_t nb = std::max<size_t>(bytes + bytes / 4, 1 << 16);
    CK(cudaMallocHost(&b.p, nb));
    b.cap = nb;
    return 0;
}

// ------------------------------------------------------------------ plan

using Setting = std::pair<int32_t, int32_t>;   // (gap, threshold)

struct Plan {
    int32_t P = 0;
    std::vector<PairPlan> pairs;
    std::vector<PairBases> pbases;  // per pair: where its alignment buffers start
    std::vector<ScoreItem> pitems;  // 32-row items of the preparation kernel
    std::vector<ScoreItem> sitems;  // 64-row items of the score kernel
    std::vector<int32_t> dorder;    // pairs by sentence count, longest first; wide targets first
    int32_t n_dwide = 0;            // pairs of more than kWideArticleSent target sentences
    std::vector<NwItem> nitems;
    std::vector<TileItem> tiles;    // of the tiled alignments (the last n_tiled items)
    int32_t n_tiled = 0;
    int64_t tb_words = 0;
    std::vector<int32_t> set_gap, set_thr, gap_val;
    std::vector<int32_t> set_perm, gap_sfirst;   // each list's settings by gap; where each gap's start
    int64_t m_elems = 0, code_words = 0, match_words = 0, sel_cap = 0;
    int32_t R = 0;
    int32_t n_grp[kNwGroups] = {0, 0, 0, 0};   // alignments by pipelines of 8, 4, 2, 1 warps (from 0, in order)
    int64_t n_sent = 0, n_tok = 0;

    // empty again, keeping the vectors' storage (a plan reused call after
    // call allocates nothing once it has grown)
    void reset()
    {
        P = 0;
        pairs.clear();
        pbases.clear();
        pitems.clear();
        sitems.clear();
        dorder.clear();
        n_dwide = 0;
        nitems.clear();
        tiles.clear();
        n_tiled = 0;
        tb_words = 0;
        set_gap.clear();
        set_perm.clear();
        gap_sfirst.clear();
        set_thr.clear();
        gap_val.clear();
        m_elems = code_words = match_words = sel_cap = 0;
        R = 0;
        for (int k = 0; k < kNwGroups; ++k) n_grp[k] = 0;
        n_sent = n_tok = 0;
    }
};

// A pair's settings list, checked once for every pair that has the same
// list: each setting's gap as an index into the list's distinct gaps (in
// order of first appearance) and the largest |gap|; where the list sits in
// the plan (every pair with the same list shares it).
struct SettingsSeen {
    const Setting *last = nullptr;   // the array the list was last read from
    std::vector<Setting> list;
    std::vector<int32_t> local, thr, gaps;
    int64_t max_g = 0;
    int32_t gap0 = 0, slist0 = 0;
    bool valid = false;
};

// Validate a pair's settings and add them to the plan: the list's distinct
// gaps (their indices start at gap0) and its settings, each as (its gap's
// index among them, θ), from slist0.  `seen` keeps the last list checked: a
// pair with the same list only has its size bound checked and shares the
// list's place in the plan.
int add_settings(Plan &pl, SettingsSeen &seen, const Setting *set, int n, int32_t S, int32_t T,
                 int64_t max_abs_s, bool mined, int32_t &gap0, int32_t &ngap, int32_t &slist0)
{
    if (n < 1 || n > 256) return fail(MINE_EINVAL, "settings count must be in [1, 256]");
    // (the same array as the pair before: the same list, not compared again)
    if (!seen.valid || (int)seen.list.size() != n ||
        (set != seen.last && !std::equal(set, set + n, seen.list.begin()))) {
        seen.valid = false;
        seen.list.assign(set, set + n);
        seen.local.resize(n);
        seen.thr.resize(n);
        seen.gaps.clear();
        seen.max_g = 0;
        for (int k = 0; k < n; ++k) {
            const int32_t g = set[k].first, th = set[k].second;
            if (g > 0) return fail(MINE_EINVAL, "gap must be <= 0");
            if (mined && (th < 0 || th > 65536))
                return fail(MINE_EINVAL, "threshold must be in [0, 65536]");
            const auto it = std::find(seen.gaps.begin(), seen.gaps.end(), g);
            seen.local[k] = (int32_t)(it - seen.gaps.begin());
            seen.thr[k] = th;
            if (it == seen.gaps.end()) seen.gaps.push_back(g);
            seen.max_g = std::max(seen.max_g, -(int64_t)g);
        }
        seen.gap0 = (int32_t)pl.gap_val.size();
        pl.gap_val.insert(pl.gap_val.end(), seen.gaps.begin(), seen.gaps.end());
        seen.slist0 = (int32_t)pl.set_gap.size();
        pl.set_gap.insert(pl.set_gap.end(), seen.local.begin(), seen.local.end());
        pl.set_thr.insert(pl.set_thr.end(), seen.thr.begin(), seen.thr.end());
        // the settings by gap (a counting sort, stable), and where each gap's start
        const int ng = (int)seen.gaps.size();
        std::vector<int32_t> start(ng + 1, 0);
        for (int k = 0; k < n; ++k) ++start[seen.local[k] + 1];
        for (int g = 0; g < ng; ++g) start[g + 1] += start[g];
        pl.gap_sfirst.insert(pl.gap_sfirst.end(), start.begin(), start.begin() + ng);
        const size_t at = pl.set_perm.size();
        pl.set_perm.resize(at + n);
        for (int k = 0; k < n; ++k) pl.set_perm[at + start[seen.local[k]]++] = k;
        seen.valid = true;
    }
    seen.last = set;
    // the bound grows with |gap|: the largest decides for every setting
    const int64_t bound = (int64_t)(S + T) * seen.max_g + (int64_t)std::min(S, T) * max_abs_s;
    if (bound >= (int64_t(1) << 31))
        return fail(MINE_EOVERFLOW, "(S+T)*|gap| + min(S,T)*max|s| reaches 2^31");
    gap0 = seen.gap0;
    slist0 = seen.slist0;
    ngap = (int32_t)seen.gaps.size();
    return 0;
}

// settings_of(p) -> (pointer, count) of pair p's settings (arrays that stay
// unchanged during the call: pairs given the same array share one list);
// swap: every pair's two articles exchange roles (the target article is the
// source)
template <class F>
int build_plan(Plan &pl, int32_t P, const int32_t *doc_off, int64_t n_sent, F settings_of,
               int64_t max_abs_s, bool mined, const int8_t *align_tab = nullptr, bool swap = false)
{
    pl.reset();
    pl.P = P;
    pl.n_sent = n_sent;
    if (P < 0) return fail(MINE_EINVAL, "negative pair count");
    if (doc_off[0] != 0) return fail(MINE_EINVAL, "doc_off[0] must be 0");
    for (int64_t d = 0; d < 2 * (int64_t)P; ++d) {
        const int64_t n = (int64_t)doc_off[d + 1] - doc_off[d];
        if (n < 0 || n > MINE_MAX_SENTENCES)
            return fail(MINE_EINVAL, "article sentence count out of range at document " + std::to_string(d));
    }
    if ((int64_t)doc_off[2 * (int64_t)P] != n_sent)
        return fail(MINE_EINVAL, "doc_off[2P] must equal n_sent");
    pl.pairs.resize(P);
    pl.pbases.assign(P, PairBases{0, 0, 0});
    SettingsSeen seen;
    std::vector<int> bucketS(P), bucketC(P), bucketD(P);
    std::vector<int8_t> kind(P);
    int64_t n_pitems = 0, n_sitems = 0;
    for (int32_t p = 0; p < P; ++p) {
        PairPlan &pp = pl.pairs[p];
        pp.s0 = doc_off[2 * p];
        pp.S = doc_off[2 * p + 1] - pp.s0;
        pp.t0 = doc_off[2 * p + 1];
        pp.T = doc_off[2 * p + 2] - pp.t0;
        if (swap) {   // mining in the other direction: the target article is the source
            std::swap(pp.s0, pp.t0);
            std::swap(pp.S, pp.T);
        }
        const Setting *set;
        int n;
        settings_of(p, set, n);
        pp.set0 = pl.R;
        pp.nset = n;
        int rc = add_settings(pl, seen, set, n, pp.S, pp.T, max_abs_s, mined, pp.gap0, pp.ngap, pp.slist0);
        if (rc) return rc;
        pl.R += n;
        pp.m_off = pl.m_elems;
        pl.m_elems += (int64_t)((pp.S + kTile - 1) / kTile) * ((pp.T + kTile - 1) / kTile) * kTileElems;
        pp.sel_base = pl.sel_cap;
        pl.sel_cap += (int64_t)n * std::min(pp.S, pp.T);
        bucketS[p] = ceil_log2_host((int64_t)pp.T + 1);
        bucketC[p] = ceil_log2_host((int64_t)pp.S * pp.T + 1);
        bucketD[p] = ceil_log2_host((int64_t)pp.S + pp.T + 1);
        kind[p] = (int8_t)align_kind(align_tab, pp.S, pp.T);
        n_pitems += (pp.S + 31) / 32;
        n_sitems += (int64_t)((pp.S + 63) / 64) * ((std::max(pp.T, 1) + kScoreColChunk - 1) / kScoreColChunk);
    }
    pl.pitems.reserve(n_pitems);
    pl.sitems.reserve(n_sitems);
    // longest-first orders (counting sort on the bit length of the work)
    auto order_by = [&](const std::vector<int> &key) {
        std::vector<int> cnt(66, 0), ord(P);
        for (int p = 0; p < P; ++p) cnt[65 - key[p]]++;
        for (int k = 1; k < 66; ++k) cnt[k] += cnt[k - 1];
        for (int p = P - 1; p >= 0; --p) ord[--cnt[65 - key[p]]] = p;
        return ord;
    };
    pl.dorder = order_by(bucketD);
    // the pairs of the wide-article preparation first, each part longest first
    pl.n_dwide = (int32_t)(std::stable_partition(pl.dorder.begin(), pl.dorder.end(),
                                                 [&](int p) { return pl.pairs[p].T > kWideArticleSent; }) -
                           pl.dorder.begin());
    for (int p : order_by(bucketS)) {
        const PairPlan &pp = pl.pairs[p];
        for (int r0 = 0; r0 < pp.S; r0 += 32) pl.pitems.push_back(ScoreItem{p, r0, 0, 0});
        for (int r0 = 0; r0 < pp.S; r0 += 64)
            for (int c0 = 0; c0 < std::max(pp.T, 1); c0 += kScoreColChunk)
                pl.sitems.push_back(ScoreItem{p, r0, c0, std::min(pp.T, c0 + kScoreColChunk)});
    }
    // alignments: pipelines of 8, 4 and 2 warps, then one warp each, each
    // longest first, then the tiled ones
    const std::vector<int> ord = order_by(bucketC);
    const int kind_of_pass[kNwGroups + 1] = {AF_WARP8, AF_WARP4, AF_WARP2, AF_WARP1, AF_TILED};
    std::vector<TileItem> tl;
    std::vector<int32_t> tdiag;
    int64_t n_items = 0;
    for (int p = 0; p < P; ++p) n_items += pl.pairs[p].ngap;
    pl.nitems.reserve(n_items);
    for (int pass = 0; pass < kNwGroups + 1; ++pass) {
        for (int p : ord) {
            const PairPlan &pp = pl.pairs[p];
            if (kind[p] != kind_of_pass[pass]) continue;
            // the pair's gaps one after another in each buffer
            PairBases &pb = pl.pbases[p];
            const int64_t CW = (pp.T + 15) >> 4;
            pb.codes = pl.code_words;
            pl.code_words += pp.ngap * (int64_t)pp.S * CW;
            pb.matches = pl.match_words;
            pl.match_words += pp.ngap * (int64_t)std::min(pp.S, pp.T);
            pb.tb = 0;
            if (pass == kNwGroups) {
                pb.tb = pl.tb_words;
                pl.tb_words += pp.ngap * tb_words_of(pp.S, pp.T);
            }
            for (int g = 0; g < pp.ngap; ++g) {
                if (pass == kNwGroups) {
                    const int64_t NR = tile_rows_of(pp.S), NC = tile_cols_of(pp.T);
                    for (int R = 0; R < NR; ++R)
                        for (int C = 0; C < NC; ++C) {
                            tl.push_back(TileItem{(int32_t)pl.nitems.size(), (int16_t)R, (int16_t)C});
                            tdiag.push_back(R + C);
                        }
                }
                pl.nitems.push_back(NwItem{p, pp.gap0 + g});
            }
        }
        if (pass < kNwGroups) {
            int32_t before = 0;
            for (int k = 0; k < pass; ++k) before += pl.n_grp[k];
            pl.n_grp[pass] = (int32_t)pl.nitems.size() - before;
        }
        if (pass == kNwGroups - 1) pl.n_tiled = -(int32_t)pl.nitems.size();
    }
    pl.n_tiled += (int32_t)pl.nitems.size();
    // tiles in order of their anti-diagonal: a tile's predecessors come first
    std::vector<int32_t> idx(tl.size());
    for (size_t k = 0; k < idx.size(); ++k) idx[k] = (int32_t)k;
    std::stable_sort(idx.begin(), idx.end(), [&](int32_t x, int32_t y) { return tdiag[x] < tdiag[y]; });
    pl.tiles.resize(tl.size());
    for (size_t k = 0; k < idx.size(); ++k) pl.tiles[k] = tl[idx[k]];
    return 0;
}

// Byte layout of one batch's device region.
struct Layout {
    int64_t plan = 0, plan_bytes = 0;
    int64_t sent_off = 0, tokens = 0;           // only when the inputs are copied in
    int64_t elems = 0, sinfo = 0, order = 0, tdoc = 0, pdoc = 0, witems = 0, xwl = 0, kitems = 0;
    int64_t M = 0, Mrow = 0, codes = 0, matches = 0, hfin = 0;
    int64_t counters = 0, nw = 0, nsel = 0, sel = 0;
    int64_t total = 0;
    // offsets inside the plan blob
    int64_t o_pairs = 0, o_pbases = 0, o_sitems = 0, o_nitems = 0, o_setgap = 0, o_setthr = 0, o_gapval = 0;
    int64_t o_setperm = 0, o_gapsfirst = 0;
    int64_t o_dorder = 0, o_pitems = 0, o_tiles = 0, tbnd = 0;
};

Layout make_layout(const Plan &pl, int32_t kmax, bool copy_inputs, bool own_sel, bool scoring)
{
    Layout L;
    int64_t o = 0;
    auto take = [&](int64_t bytes) {
        const int64_t at = o;
        o = align_up(o + std::max<int64_t>(bytes, 0), 256);
        return at;
    };
    int64_t q = 0;
    auto sub = [&](int64_t bytes) {
        const int64_t at = q;
        q = align_up(q + bytes, 16);
        return at;
    };
    L.o_pairs = sub(sizeof(PairPlan) * pl.pairs.size());
    L.o_pbases = sub(sizeof(PairBases) * pl.pbases.size());
    L.o_sitems = sub(sizeof(ScoreItem) * pl.sitems.size());
    L.o_nitems = sub(sizeof(NwItem) * pl.nitems.size());
    L.o_setgap = sub(4 * pl.set_gap.size());
    L.o_setthr = sub(4 * pl.set_thr.size());
    L.o_gapval = sub(4 * pl.gap_val.size());
    L.o_setperm = sub(4 * pl.set_perm.size());
    L.o_gapsfirst = sub(4 * pl.gap_sfirst.size());
    L.o_dorder = sub(4 * pl.dorder.size());
    L.o_pitems = sub(sizeof(ScoreItem) * pl.pitems.size());
    L.o_tiles = sub(sizeof(TileItem) * pl.tiles.size());
    L.plan_bytes = q;
    L.plan = take(q);
    if (copy_inputs) {
        L.sent_off = take(4 * (pl.n_sent + 1));
        L.tokens = take(4 * pl.n_tok + 16);
    }
    if (scoring) {
        L.elems = take(4 * (pl.n_tok * kmax + 3 * pl.n_sent + 16));
        L.sinfo = take(16 * pl.n_sent);
        L.order = take(4 * pl.n_sent + 16);
        L.tdoc = take(2 * pl.n_tok + 64);   // bulk copies round up past the end
        L.pdoc = take(4 * (int64_t)pl.P + 16);
        L.witems = take(sizeof(ScoreItem) * (pl.sitems.size() + 1));
        L.xwl = take(4 * (int64_t)pl.P + 16);
        L.kitems = take(sizeof(ScoreItem) * (pl.pitems.size() + 1));
    } else {
        // a caller-supplied row-major matrix is copied here, then tiled
        int64_t rows = 0;
        for (const PairPlan &pp : pl.pairs) rows += (int64_t)pp.S * pp.T;
        L.Mrow = take(4 * rows + 16);
    }
    L.M = take(4 * pl.m_elems + 16);
    L.codes = take(4 * pl.code_words + 16);
    L.matches = take(4 * pl.match_words + 16);
    L.hfin = take(4 * (int64_t)pl.nitems.size() + 16);
    L.tbnd = take(4 * pl.tb_words + 16);
    L.counters = take(4 * kCounters);
    L.nw = take(4 * (int64_t)pl.R);
    L.nsel = take(4 * (int64_t)pl.R);
    if (own_sel) L.sel = take(12 * pl.sel_cap + 16);
    L.total = o;
    return L;
}

void pack_plan(const Plan &pl, const Layout &L, char *dst)
{
    std::memcpy(dst + L.o_pairs, pl.pairs.data(), sizeof(PairPlan) * pl.pairs.size());
    std::memcpy(dst + L.o_pbases, pl.pbases.data(), sizeof(PairBases) * pl.pbases.size());
    std::memcpy(dst + L.o_sitems, pl.sitems.data(), sizeof(ScoreItem) * pl.sitems.size());
    std::memcpy(dst + L.o_nitems, pl.nitems.data(), sizeof(NwItem) * pl.nitems.size());
    std::memcpy(dst + L.o_setgap, pl.set_gap.data(), 4 * pl.set_gap.size());
    std::memcpy(dst + L.o_setthr, pl.set_thr.data(), 4 * pl.set_thr.size());
    std::memcpy(dst + L.o_gapval, pl.gap_val.data(), 4 * pl.gap_val.size());
    std::memcpy(dst + L.o_setperm, pl.set_perm.data(), 4 * pl.set_perm.size());
    std::memcpy(dst + L.o_gapsfirst, pl.gap_sfirst.data(), 4 * pl.gap_sfirst.size());
    std::memcpy(dst + L.o_dorder, pl.dorder.data(), 4 * pl.dorder.size());
    std::memcpy(dst + L.o_pitems, pl.pitems.data(), sizeof(ScoreItem) * pl.pitems.size());
    std::memcpy(dst + L.o_tiles, pl.tiles.data(), sizeof(TileItem) * pl.tiles.size());
}

BatchDev make_batchdev(const Plan &pl, const Layout &L, char *base, const int32_t *sent_off,
                       const int32_t *tokens, int32_t *sel, const uint64_t *recip, void *gscratch)
{
    BatchDev b{};
    b.recip = recip;
    b.recip31 = recip ? reinterpret_cast<const uint32_t *>(recip + kMaxSentTokens + 1) : nullptr;
    b.gscratch = static_cast<int2 *>(gscratch);
    char *plan = base + L.plan;
    b.sent_off = sent_off;
    b.tokens = tokens;
    b.n_tok = pl.n_tok;
    b.n_pairs = pl.P;
    b.n_dwide = pl.n_dwide;
    b.pairs = reinterpret_cast<const PairPlan *>(plan + L.o_pairs);
    b.pbases = reinterpret_cast<const PairBases *>(plan + L.o_pbases);
    b.prep_items = reinterpret_cast<const ScoreItem *>(plan + L.o_pitems);
    b.n_prep_items = (int32_t)pl.pitems.size();
    b.score_items = reinterpret_cast<const ScoreItem *>(plan + L.o_sitems);
    b.n_score_items = (int32_t)pl.sitems.size();
    b.nw_items = reinterpret_cast<const NwItem *>(plan + L.o_nitems);
    b.n_nw_items = (int32_t)pl.nitems.size();
    for (int k = 0; k < kNwGroups; ++k) b.n_nw_grp[k] = pl.n_grp[k];
    b.n_nw_tiled = pl.n_tiled;
    b.tiles = reinterpret_cast<const TileItem *>(plan + L.o_tiles);
    b.n_tiles = (int32_t)pl.tiles.size();
    b.tbnd = reinterpret_cast<int32_t *>(base + L.tbnd);
    b.n_tbnd = pl.tb_words;
    b.set_gap = reinterpret_cast<const int32_t *>(plan + L.o_setgap);
    b.set_thr = reinterpret_cast<const int32_t *>(plan + L.o_setthr);
    b.gap_val = reinterpret_cast<const int32_t *>(plan + L.o_gapval);
    b.set_perm = reinterpret_cast<const int32_t *>(plan + L.o_setperm);
    b.gap_sfirst = reinterpret_cast<const int32_t *>(plan + L.o_gapsfirst);
    b.elems = reinterpret_cast<uint32_t *>(base + L.elems);
    b.sinfo = reinterpret_cast<int4 *>(base + L.sinfo);
    b.row_order = reinterpret_cast<int32_t *>(base + L.order);
    b.tdoc = reinterpret_cast<uint16_t *>(base + L.tdoc);
    b.pdoc = reinterpret_cast<int32_t *>(base + L.pdoc);
    b.wide_items = reinterpret_cast<ScoreItem *>(base + L.witems);
    b.xw_list = reinterpret_cast<int32_t *>(base + L.xwl);
    b.keyed_items = reinterpret_cast<ScoreItem *>(base + L.kitems);
    b.dorder = reinterpret_cast<const int32_t *>(plan + L.o_dorder);
    b.M = reinterpret_cast<int32_t *>(base + L.M);
    b.codes = reinterpret_cast<uint32_t *>(base + L.codes);
    b.matches = reinterpret_cast<uint32_t *>(base + L.matches);
    b.hfin = reinterpret_cast<int32_t *>(base + L.hfin);
    b.counters = reinterpret_cast<int32_t *>(base + L.counters);
    b.err = b.counters + 8;
    b.nw_score = reinterpret_cast<int32_t *>(base + L.nw);
    b.n_sel = reinterpret_cast<int32_t *>(base + L.nsel);
    b.sel = sel ? sel : reinterpret_cast<int32_t *>(base + L.sel);
    return b;
}

const char *device_err_text(int32_t e)
{
    switch (e) {
    case ERR_DUP_KEY: return "duplicate dictionary key";
    case ERR_BAD_OFFSETS: return "malformed sentence offsets (sent_off must start at 0, not decrease, end at n_tok, and give <= 1024 tokens per sentence)";
    case ERR_BAD_TOKEN: return "token id outside [0, 2^30)";
    case ERR_TIMEOUT: return "a bounded device wait ran out";
    default: return "device error";
    }
}

// The ABI code of a device error word: MINE_ETIMEDOUT for a bounded wait that
// ran out, MINE_EINVAL for malformed inputs found on the device.
int device_fail(int32_t e)
{
    return fail(e == ERR_TIMEOUT ? MINE_ETIMEDOUT : MINE_EINVAL, device_err_text(e));
}

// ------------------------------------------------------------------ pool

// First-fit allocator over one device region: the serving budget.
struct Pool {
    char *base = nullptr;
    int64_t size = 0;
    std::map<int64_t, int64_t> free_;   // offset -> bytes
    int64_t used = 0;

    int64_t alloc(int64_t bytes)
    {
        bytes = align_up(bytes, 256);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const int64_t off = it->first, rest = it->second - bytes;
                free_.erase(it);
                if (rest > 0) free_[off + bytes] = rest;
                used += bytes;
                return off;
            }
        }
        return -1;
    }
    void release(int64_t off, int64_t bytes)
    {
        bytes = align_up(bytes, 256);
        used -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

}  // namespace

void mine::set_last_error(const char *msg) { g_err = msg ? msg : ""; }

// ------------------------------------------------------------------ objects

struct mine_dict {
    DevDict d{};
    void *slots_mem = nullptr;
    void *trans_mem = nullptr;
    std::atomic<int64_t> inflight{0};
    uint64_t serial = 0;               // unique per context, for cached graphs
};

namespace {

struct Request {
    uint64_t ticket = 0;
    std::vector<int32_t> src_off, src_tok, tgt_off, tgt_tok;
    const mine_dict *dict = nullptr;
    std::vector<Setting> settings;
    int64_t footprint = 0;
    std::chrono::steady_clock::time_point t_submit;
};

// A second stream beside a launch stream: the wide-article launches of a
// batch run on it next to the others (fork and join by events), so that their
// few long pairs do not hold up the rest of the GPU.
struct Fork {
    cudaStream_t st = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};

int fork_create(Fork &f)
{
    if (cudaStreamCreateWithFlags(&f.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&f.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&f.join, cudaEventDisableTiming) != cudaSuccess)
        return fail(MINE_ECUDA, "stream or event creation failed");
    return 0;
}

void fork_destroy(Fork &f)
{
    if (f.st) cudaStreamDestroy(f.st);
    if (f.fork) cudaEventDestroy(f.fork);
    if (f.join) cudaEventDestroy(f.join);
    f = Fork{};
}

struct Slot {
    cudaStream_t st = nullptr;
    Fork fork;                         // beside st
    cudaEvent_t ev = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;   // timed: before the first copy, after the last
    bool busy = false;
    std::vector<Request> reqs;
    int64_t pool_off = -1, pool_bytes = 0;
    HostBuf pin_in, pin_out;
    Plan plan;
    Layout lay;
    int64_t out_nw = 0, out_nsel = 0, out_sel = 0, out_err = 0;
    void *gscratch = nullptr;          // score-kernel tables for long sentences
};

// Result bookkeeping of one enqueued host-buffer batch call.
struct HostCallOut {
    int64_t R = 0;                     // result rows (pairs x settings)
    int32_t *h_err = nullptr;          // pinned copy of the device error word
    int64_t h2d = 0, d2h = 0;          // bytes copied each way
    const int32_t *d_sel = nullptr;    // packed triples left on the device (copied by the caller)
};

// One host-buffer batch call in flight (mine_run_batch_async): its own
// input buffer, scratch, staging and long-sentence tables, so that its
// input copies can run while the kernels of the call before it run.
struct AsyncCall {
    bool busy = false, waiting = false;
    uint64_t ticket = 0;
    DevBuf inbuf, arena;
    HostBuf pin;
    Plan plan;                         // reused call after call (its storage stays)
    void *gscratch = nullptr;
    cudaEvent_t in_ready = nullptr;    // inputs and plan on the device (input stream)
    cudaEvent_t packed = nullptr;      // results packed (context stream)
    cudaEvent_t done = nullptr;        // last result copy (output stream)
    const mine_dict *dict = nullptr;
    const int64_t *sel_off = nullptr;
    const mine_pair *sel = nullptr;
    int64_t sel_cap = 0;
    HostCallOut out;
};

}  // namespace

struct mine_ctx {
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    Fork fork;                         // beside stream
    std::mutex api_mu;                 // synchronous calls
    DevBuf arena;                      // scratch of the synchronous calls
    DevBuf inbuf;                      // inputs of the host-buffer batch call
    HostBuf pin;                       // staging of the synchronous calls
    Plan plan;                         // of the synchronous host-buffer batch call
    std::atomic<int64_t> launches{0};
    // test fault injection (mine_test_inject): the checked CUDA call of a
    // host-buffer batch call at which a failure is faked, counting down
    std::atomic<int32_t> inject_cuda_at{0};
    // host-buffer batch calls still to run with withheld pipeline rows and
    // short device waits (mine_test_inject, MINE_INJECT_WITHHOLD_ROWS)
    std::atomic<int32_t> inject_withhold{0};
    std::atomic<int64_t> h2d_bytes{0}, d2h_bytes{0};   // host-buffer batch calls
    // per-kernel timing (CUDA events on the launching stream)
    std::mutex prof_mu;
    bool prof_on = false;
    struct Mark { int kid; cudaEvent_t a, b; };
    std::vector<Mark> prof_pending;
    std::vector<cudaEvent_t> prof_free;
    double prof_ms[KID_COUNT] = {0};
    int64_t prof_n[KID_COUNT] = {0};
    int64_t err_off = -1;              // offset of the last device batch's error word
    uint64_t arena_gen = 0;            // bumped whenever a call rewrites arena / pin
    int8_t align_tab[kAlignBins];      // alignment strategy per size bin (-1: built-in rule)
    uint64_t dict_serial = 0;
    // The last device-buffer batch as a CUDA graph (plan upload + kernels);
    // replayed when the next call repeats it byte for byte.
    struct Graph {
        cudaGraphExec_t exec = nullptr;
        uint64_t dict_serial = 0, gen = 0;
        int32_t P = 0;
        int64_t n_sent = 0, n_tok = 0, sel_cap = 0, err_off = -1;
        std::vector<int32_t> doc_off, gaps, thr;
        const void *sent_off = nullptr, *tokens = nullptr, *nw = nullptr, *ns = nullptr, *sel = nullptr;
        cudaStream_t stream = nullptr;
        int launches = 0;
    } graph;

    // serving
    mine_config cfg{};
    Pool pool;
    void *pool_mem = nullptr;
    uint64_t *recip = nullptr;         // device table of ceil(2^48 / m), m <= kMaxSentTokens
    void *gscratch = nullptr;          // score-kernel tables for long sentences (synchronous calls)
    size_t gscratch_bytes = 0;
    std::vector<std::unique_ptr<Slot>> slots;
    std::mutex q_mu;
    std::condition_variable q_cv;      // pending work / stop
    std::condition_variable r_cv;      // results ready
    std::deque<Request> pending;
    std::deque<mine_result> ready;
    int64_t in_flight_reqs = 0;        // submitted, not yet turned into results
    bool stop = false;
    uint64_t next_ticket = 1;
    std::thread worker;
    std::vector<mine_dict *> dicts;
    // device time span of every served batch (ms after `origin`), for the
    // overlap statistic of mine_serving_stats (guarded by q_mu)
    cudaEvent_t origin = nullptr;
    std::vector<std::pair<float, float>> spans;
    int64_t n_batches = 0;

    // host-buffer batch calls in flight (mine_run_batch_async)
    cudaStream_t cstream = nullptr;    // their input copies
    cudaStream_t ostream = nullptr;    // their result copies
    AsyncCall acall[MINE_ASYNC_DEPTH];
    uint64_t next_async = 1;
};

namespace {

int set_device(mine_ctx *ctx)
{
    CK(cudaSetDevice(ctx->device));
    return 0;
}

// True for the checked CUDA call at which mine_test_inject asked for a
// failure (the call is then not made).
bool inject_cuda_error(mine_ctx *ctx)
{
    if (ctx->inject_cuda_at.load(std::memory_order_relaxed) <= 0) return false;
    return ctx->inject_cuda_at.fetch_sub(1) == 1;
}

cudaEvent_t prof_event(mine_ctx *ctx)
{
    if (!ctx->prof_free.empty()) {
        cudaEvent_t e = ctx->prof_free.back();
        ctx->prof_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Launch one kernel through `fn`, bracketed by events when profiling is on.
template <class F>
int timed_launch(mine_ctx *ctx, int kid, cudaStream_t st, F fn)
{
    std::unique_lock<std::mutex> lk(ctx->prof_mu, std::defer_lock);
    bool on = false;
    {
        std::lock_guard<std::mutex> g(ctx->prof_mu);
        on = ctx->prof_on;
    }
    if (!on) return fn();
    cudaEvent_t a, b;
    {
        std::lock_guard<std::mutex> g(ctx->prof_mu);
        a = prof_event(ctx);
        b = prof_event(ctx);
    }
    cudaEventRecord(a, st);
    const int n = fn();
    cudaEventRecord(b, st);
    std::lock_guard<std::mutex> g(ctx->prof_mu);
    if (n > 0) {
        ctx->prof_pending.push_back({kid, a, b});
    } else {
        ctx->prof_free.push_back(a);
        ctx->prof_free.push_back(b);
    }
    return n;
}

// Enqueue the kernels of one batch whose plan is already on the device.
// With a fork stream, the wide-article preparation and score launches run on
// it beside the small-article ones (launched first: their long pairs start
// early and finish while the others run); each pair of launches is joined
// before the next step.
int enqueue_kernels(mine_ctx *ctx, const BatchDev &b, const mine_dict *dict, int64_t n_sent,
                    int64_t n_tok, bool scoring, cudaStream_t st, bool aligning = true,
                    const Fork *fk = nullptr)
{
    int n = 0;
    CK(cudaMemsetAsync(b.counters, 0, 4 * kCounters, st));
    if (scoring) {
        n += timed_launch(ctx, KID_VALIDATE, st, [&] { return launch_validate(b.sent_off, n_sent, n_tok, b.err, st); });
        BatchDev bd = b;
        bd.kmax = dict->d.kmax;
        // (with per-kernel events every launch runs alone: its time is its own)
        bool prof = false;
        {
            std::lock_guard<std::mutex> g(ctx->prof_mu);
            prof = ctx->prof_on;
        }
        const bool par = fk && fk->st && !prof;
        const cudaStream_t sw = par ? fk->st : st;
        if (par) {
            CK(cudaEventRecord(fk->fork, st));
            CK(cudaStreamWaitEvent(sw, fk->fork, 0));
        }
        n += timed_launch(ctx, KID_DOC_WIDE, sw, [&] { return launch_pairprep_wide(bd, dict->d, ctx->num_sms, sw); });
        n += timed_launch(ctx, KID_DOC, st, [&] { return launch_pairprep(bd, dict->d, ctx->num_sms, st); });
        if (par) {
            CK(cudaEventRecord(fk->join, sw));
            CK(cudaStreamWaitEvent(st, fk->join, 0));
        }
        n += timed_launch(ctx, KID_DOC_XWIDE, st, [&] { return launch_pairprep_xwide(bd, dict->d, ctx->num_sms, st); });
        n += timed_launch(ctx, KID_PREP, st, [&] { return launch_prep(bd, dict->d, ctx->num_sms, st); });
        n += timed_launch(ctx, KID_ORDER, st, [&] { return launch_order(bd, ctx->num_sms, st); });
        if (par) {
            CK(cudaEventRecord(fk->fork, st));
            CK(cudaStreamWaitEvent(sw, fk->fork, 0));
        }
        n += timed_launch(ctx, KID_SCORE_WIDE, sw, [&] { return launch_score_wide(bd, ctx->num_sms, sw); });
        n += timed_launch(ctx, KID_SCORE, st, [&] { return launch_score(bd, ctx->num_sms, st); });
        n += timed_launch(ctx, KID_SCORE_XWIDE, st, [&] { return launch_score_xwide(bd, ctx->num_sms, st); });
        if (par) {
            CK(cudaEventRecord(fk->join, sw));
            CK(cudaStreamWaitEvent(st, fk->join, 0));
        }
    }
    if (aligning) {
        if (b.n_tiles > 0) CK(cudaMemsetAsync(b.tbnd, 0, 4 * b.n_tbnd, st));
        n += timed_launch(ctx, KID_ALIGN, st, [&] { return launch_align(b, ctx->num_sms, st); });
        n += timed_launch(ctx, KID_ALIGN_TILED, st, [&] { return launch_align_tiled(b, ctx->num_sms, st); });
        n += timed_launch(ctx, KID_TRACE, st, [&] { return launch_trace(b, ctx->num_sms, st); });
    }
    CK(cudaGetLastError());
    ctx->launches += n;
    return 0;
}

int64_t request_footprint(const Plan &pl, int32_t kmax)
{
    return make_layout(pl, kmax, true, true, true).total;
}

}  // namespace

static void serving_loop(mine_ctx *ctx);

// ====================================================================== ABI

extern "C" {

const char *mine_last_error(void) { return g_err.c_str(); }

int64_t mine_launch_count(mine_ctx *ctx) { return ctx ? ctx->launches.load() : 0; }

namespace {

// Device time (ms, mean of three launches after a warm-up) of the alignment
// kernel over P random side x side matrices, every pair aligned in form
// `form` (AF_*).
int time_align(mine_ctx *ctx, int bin, int side, int32_t P, int form, cudaEvent_t e0, cudaEvent_t e1,
               float &ms)
{
    std::vector<int32_t> doc(2 * (size_t)P + 1);
    for (size_t k = 0; k < doc.size(); ++k) doc[k] = (int32_t)k * side;
    int8_t tab[kAlignBins];
    std::fill(tab, tab + kAlignBins, (int8_t)-1);
    tab[bin] = (int8_t)form;
    const Setting set(-65536, 0);
    Plan pl;
    int rc = build_plan(pl, P, doc.data(), (int64_t)doc.back(),
                        [&](int32_t, const Setting *&s, int &cnt) { s = &set; cnt = 1; }, 65536, false, tab);
    if (rc) return rc;
    const Layout L = make_layout(pl, 1, false, true, false);
    if ((rc = ensure_dev(ctx->arena, L.total))) return rc;
    if ((rc = ensure_host(ctx->pin, L.plan_bytes + 64))) return rc;
    cudaStream_t st = ctx->stream;
    CK(cudaStreamSynchronize(st));
    char *hp = static_cast<char *>(ctx->pin.p);
    pack_plan(pl, L, hp);
    char *base = static_cast<char *>(ctx->arena.p);
    CK(cudaMemcpyAsync(base + L.plan, hp, L.plan_bytes, cudaMemcpyHostToDevice, st));
    BatchDev b = make_batchdev(pl, L, base, nullptr, nullptr, nullptr, ctx->recip, ctx->gscratch);
    launch_fill_scores(b.M, pl.m_elems, 0x5EEDu + (uint32_t)bin, st);
    for (int rep = 0; rep < 4; ++rep) {
        CK(cudaMemsetAsync(b.counters, 0, 4 * kCounters, st));
        if (rep == 1) CK(cudaEventRecord(e0, st));
        ctx->launches += launch_align(b, ctx->num_sms, st);
        ctx->launches += launch_trace(b, ctx->num_sms, st);   // part of each form's cost
    }
    CK(cudaEventRecord(e1, st));
    CK(cudaEventSynchronize(e1));
    CK(cudaGetLastError());
    int32_t derr = 0;
    CK(cudaMemcpy(&derr, b.err, 4, cudaMemcpyDeviceToHost));
    if (derr) return fail(MINE_ETIMEDOUT, "a bounded device wait ran out while tuning");
    CK(cudaEventElapsedTime(&ms, e0, e1));
    ms /= 3.0f;
    return 0;
}

}  // namespace

int mine_autotune(mine_ctx *ctx)
{
    if (!ctx) return fail(MINE_EINVAL, "null context");
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    int rc = set_device(ctx);
    if (rc) return rc;
    ++ctx->arena_gen;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(MINE_ECUDA, "cudaEventCreate failed");
    }
    int8_t tab[kAlignBins];
    std::copy(ctx->align_tab, ctx->align_tab + kAlignBins, tab);
    for (int bin = 6; bin <= 17 && rc == 0; ++bin) {
        // square pairs whose cell count falls in the bin: 2^(bin-1) < side^2 + 1 <= 2^bin
        int side = 1;
        while ((int64_t)(side + 1) * (side + 1) + 1 <= (int64_t(1) << bin)) ++side;
        const int64_t cells = (int64_t)side * side;
        const int32_t P = (int32_t)std::min<int64_t>(8192, std::max<int64_t>(64, (int64_t(1) << 23) / cells));
        // pipelines of 1, 2, 4 and 8 warps (as far as the side allows)
        const int forms[4] = {AF_WARP1, AF_WARP2, AF_WARP4, AF_WARP8};
        float tbest = 0.f;
        int fbest = -1;
        for (int fi = 0; fi < 4 && rc == 0; ++fi) {
            int8_t one[kAlignBins];
            std::fill(one, one + kAlignBins, (int8_t)-1);
            one[bin] = (int8_t)forms[fi];
            if (align_kind(one, side, side) != forms[fi]) continue;
            float t = 0.f;
            rc = time_align(ctx, bin, side, P, forms[fi], e0, e1, t);
            if (rc == 0 && (fbest < 0 || t < tbest)) {
                tbest = t;
                fbest = forms[fi];
            }
        }
        if (rc == 0 && fbest >= 0) tab[bin] = (int8_t)fbest;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    std::copy(tab, tab + kAlignBins, ctx->align_tab);
    return MINE_OK;
}

static int check_batch(const mine_batch *b);
static int check_settings(const mine_settings *s);

int mine_autotune_batch(mine_ctx *ctx, const mine_dict *dict, const mine_batch *batch,
                        const mine_settings *settings)
{
    if (!ctx || !dict) return fail(MINE_EINVAL, "null context or dictionary");
    int rc = check_batch(batch);
    if (rc) return rc;
    if (settings && (rc = check_settings(settings))) return rc;
    const int32_t P = batch->n_pairs;
    if (P == 0) return MINE_OK;
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    if ((rc = set_device(ctx))) return rc;
    ++ctx->arena_gen;
    // the settings the batch will be mined with: their distinct gaps are
    // the alignments each pair gets
    std::vector<Setting> set;
    if (settings) {
        for (int k = 0; k < settings->n; ++k) set.push_back(Setting(settings->gaps[k], settings->thresholds[k]));
    } else {
        set.push_back(Setting(-65536, 32768));
    }
    const int nset = (int)set.size();
    auto plan_with = [&](Plan &pl, const int8_t *tab) {
        int r = build_plan(pl, P, batch->doc_off, batch->n_sent,
                           [&](int32_t, const Setting *&s, int &cnt) { s = set.data(); cnt = nset; }, 65536,
                           true, tab);
        pl.n_tok = batch->n_tok;
        return r;
    };
    int8_t tab[kAlignBins];
    std::copy(ctx->align_tab, ctx->align_tab + kAlignBins, tab);
    Plan pl;
    if ((rc = plan_with(pl, tab))) return rc;
    // the scratch layout of the plan with every pair that can be tiled tiled:
    // the largest tile area and tile list of all the plans tried below
    int8_t all_tiles[kAlignBins];
    std::fill(all_tiles, all_tiles + kAlignBins, (int8_t)2);
    Plan pmax;
    if ((rc = plan_with(pmax, all_tiles))) return rc;
    const Layout L = make_layout(pmax, dict->d.kmax, true, true, true);
    if ((rc = ensure_dev(ctx->arena, L.total))) return rc;
    if ((rc = ensure_host(ctx->pin, L.plan_bytes + 64))) return rc;
    char *hp = static_cast<char *>(ctx->pin.p);
    char *base = static_cast<char *>(ctx->arena.p);
    cudaStream_t st = ctx->stream;
    pack_plan(pl, L, hp);
    int32_t *d_sent = reinterpret_cast<int32_t *>(base + L.sent_off);
    int32_t *d_tok = reinterpret_cast<int32_t *>(base + L.tokens);
    CK(cudaMemcpyAsync(base + L.plan, hp, L.plan_bytes, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_sent, batch->sent_off, 4 * (batch->n_sent + 1), cudaMemcpyHostToDevice, st));
    if (batch->n_tok > 0)
        CK(cudaMemcpyAsync(d_tok, batch->tokens, 4 * batch->n_tok, cudaMemcpyHostToDevice, st));
    // the batch's score matrices, once
    BatchDev b = make_batchdev(pl, L, base, d_sent, d_tok, nullptr, ctx->recip, ctx->gscratch);
    if ((rc = enqueue_kernels(ctx, b, dict, batch->n_sent, batch->n_tok, true, st, false, &ctx->fork))) return rc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(MINE_ECUDA, "cudaEventCreate failed");
    }
    // device time of the batch's alignment under a strategy table (the plan's
    // alignment items change with it; score matrices and their layout do not)
    auto time_with = [&](const int8_t *t, float &ms) -> int {
        Plan q;
        int r = plan_with(q, t);
        if (r) return r;
        CK(cudaStreamSynchronize(st));
        pack_plan(q, L, hp);
        CK(cudaMemcpyAsync(base + L.plan, hp, L.plan_bytes, cudaMemcpyHostToDevice, st));
        BatchDev bq = make_batchdev(q, L, base, d_sent, d_tok, nullptr, ctx->recip, ctx->gscratch);
        for (int rep = 0; rep < 5; ++rep) {   // one untimed, four timed
            // queue heads (the error word at index 8 is kept)
            CK(cudaMemsetAsync(bq.counters, 0, 4 * 8, st));
            CK(cudaMemsetAsync(bq.counters + 16, 0, 4 * (kCounters - 16), st));
            if (bq.n_tiles > 0) CK(cudaMemsetAsync(bq.tbnd, 0, 4 * bq.n_tbnd, st));
            if (rep == 1) CK(cudaEventRecord(e0, st));
            ctx->launches += launch_align(bq, ctx->num_sms, st);
            ctx->launches += launch_align_tiled(bq, ctx->num_sms, st);
            ctx->launches += launch_trace(bq, ctx->num_sms, st);   // one-warp forms trace inside k_align
        }
        CK(cudaEventRecord(e1, st));
        CK(cudaEventSynchronize(e1));
        CK(cudaGetLastError());
        int32_t derr = 0;
        CK(cudaMemcpy(&derr, bq.err, 4, cudaMemcpyDeviceToHost));
        if (derr) return device_fail(derr);
        CK(cudaEventElapsedTime(&ms, e0, e1));
        ms /= 4.0f;
        return 0;
    };
    // the forms open to some pair of each bin present in the batch.  A whole
    // CTA pipelines its warps over 32-row stripes: for a pair of one stripe
    // seven of its eight warps would idle, so that form is tried only for
    // bins holding a pair of more rows.
    // the forms open to some pair of each bin present in the batch (a form
    // a pair cannot take is narrowed for it, so trying it would repeat
    // another form's timing)
    bool present[kAlignBins] = {};
    bool can[kAlignBins][AF_FORMS] = {};
    for (const PairPlan &pp : pl.pairs) {
        const int64_t c = (int64_t)pp.S * pp.T;
        int bin = 0;
        while (bin < 63 && (int64_t(1) << bin) < c + 1) ++bin;
        if (bin >= kAlignBins) continue;
        present[bin] = true;
        for (int f = 0; f < AF_FORMS; ++f) {
            int8_t one[kAlignBins];
            std::fill(one, one + kAlignBins, (int8_t)-1);
            one[bin] = (int8_t)f;
            if (align_kind(one, pp.S, pp.T) == f) can[bin][f] = true;
        }
    }
    float best = 0.f;
    rc = time_with(tab, best);
    const int order[AF_FORMS] = {AF_WARP1, AF_WARP2, AF_WARP4, AF_WARP8, AF_TILED};
    for (int bin = 0; bin < kAlignBins && rc == 0; ++bin) {
        if (!present[bin]) continue;
        // the entry the bin has now (-1: the built-in rule), then each form
        int keep = tab[bin];
        for (int fi = 0; fi < AF_FORMS && rc == 0; ++fi) {
            const int f = order[fi];
            if (f == tab[bin] || !can[bin][f]) continue;
            int8_t trial[kAlignBins];
            std::copy(tab, tab + kAlignBins, trial);
            trial[bin] = (int8_t)f;
            float t = 0.f;
            if ((rc = time_with(trial, t))) break;
            if (t < 0.97f * best) {
                best = t;
                keep = f;
            }
        }
        tab[bin] = (int8_t)keep;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    std::copy(tab, tab + kAlignBins, ctx->align_tab);
    return MINE_OK;
}

}  // extern "C"

namespace {

// The strategy table as a small JSON document,
//   {"format": "mine-align-strategy", "bins": [t0, t1, ..., t39]},
// entries -1 .. AF_FORMS - 1 as in mine_align_strategy.
std::string strategy_json(const int8_t *tab)
{
    std::string s = "{\"format\": \"mine-align-strategy\", \"bins\": [";
    for (int b = 0; b < kAlignBins; ++b) {
        if (b) s += ", ";
        s += std::to_string((int)tab[b]);
    }
    s += "]}\n";
    return s;
}

// Parse a document of that form (any white space between its tokens) into
// tab; false, with tab unchanged, for anything else.
bool strategy_parse(const std::string &t, int8_t *tab)
{
    size_t i = 0;
    auto ws = [&] {
        while (i < t.size() && (t[i] == ' ' || t[i] == '\t' || t[i] == '\n' || t[i] == '\r')) ++i;
    };
    auto lit = [&](const char *x) {
        ws();
        const size_t n = std::strlen(x);
        if (t.compare(i, n, x) != 0) return false;
        i += n;
        return true;
    };
    int8_t v[kAlignBins];
    if (!lit("{") || !lit("\"format\"") || !lit(":") || !lit("\"mine-align-strategy\"") || !lit(",") ||
        !lit("\"bins\"") || !lit(":") || !lit("["))
        return false;
    for (int n = 0;; ++n) {
        ws();
        const bool neg = i < t.size() && t[i] == '-';
        if (neg) ++i;
        int x = 0, digits = 0;
        while (i < t.size() && t[i] >= '0' && t[i] <= '9' && digits < 3) x = 10 * x + (t[i++] - '0'), ++digits;
        if (digits == 0 || n >= kAlignBins) return false;
        x = neg ? -x : x;
        if (x < -1 || x >= AF_FORMS) return false;
        v[n] = (int8_t)x;
        if (lit(",")) continue;
        if (!lit("]") || n + 1 != kAlignBins) return false;
        break;
    }
    if (!lit("}")) return false;
    ws();
    if (i != t.size()) return false;
    std::copy(v, v + kAlignBins, tab);
    return true;
}

}  // namespace

extern "C" {

int mine_align_strategy_save(mine_ctx *ctx, const char *path)
{
    if (!ctx || !path) return fail(MINE_EINVAL, "null context or path");
    int8_t tab[kAlignBins];
    {
        std::lock_guard<std::mutex> lk(ctx->api_mu);
        std::copy(ctx->align_tab, ctx->align_tab + kAlignBins, tab);
    }
    const std::string s = strategy_json(tab);
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(MINE_EINVAL, std::string("cannot open ") + path);
    const size_t w = std::fwrite(s.data(), 1, s.size(), f);
    if (std::fclose(f) != 0 || w != s.size()) return fail(MINE_EINVAL, std::string("cannot write ") + path);
    return MINE_OK;
}

int mine_align_strategy_load(mine_ctx *ctx, const char *path)
{
    if (!ctx || !path) return fail(MINE_EINVAL, "null context or path");
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(MINE_EINVAL, std::string("cannot open ") + path);
    std::string t;
    char buf[4096];
    size_t r;
    while ((r = std::fread(buf, 1, sizeof buf, f)) > 0 && t.size() < (1u << 16)) t.append(buf, r);
    std::fclose(f);
    int8_t tab[kAlignBins];
    if (!strategy_parse(t, tab)) return fail(MINE_EINVAL, std::string("not a strategy table: ") + path);
    return mine_align_strategy(ctx, tab, kAlignBins, 0);
}

int mine_align_strategy(mine_ctx *ctx, int8_t *tab, int32_t n, int32_t get)
{
    if (!ctx || !tab || n < 0 || n > kAlignBins) return fail(MINE_EINVAL, "bad argument");
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    if (get) {
        std::copy(ctx->align_tab, ctx->align_tab + n, tab);
    } else {
        for (int k = 0; k < n; ++k)
            if (tab[k] < -1 || tab[k] >= AF_FORMS) return fail(MINE_EINVAL, "strategy entries are -1 .. 4");
        std::copy(tab, tab + n, ctx->align_tab);
        ++ctx->arena_gen;   // cached graphs hold plans of the old table
    }
    return MINE_OK;
}

int mine_open(const mine_config *cfg, mine_ctx **out)
{
    if (!out) return fail(MINE_EINVAL, "out is NULL");
    *out = nullptr;
    std::unique_ptr<mine_ctx> ctx(new mine_ctx());
    std::fill(ctx->align_tab, ctx->align_tab + kAlignBins, (int8_t)-1);
    mine_config c{};
    if (cfg) c = *cfg;
    else c.device = -1;
    if (c.device_budget_bytes <= 0) c.device_budget_bytes = int64_t(8) << 30;
    if (c.max_inflight <= 0) c.max_inflight = 3;
    if (c.max_batch_pairs <= 0) c.max_batch_pairs = 4096;
    if (c.batch_window_us <= 0) c.batch_window_us = 200;
    ctx->cfg = c;
    if (c.device < 0) {
        CK(cudaGetDevice(&ctx->device));
    } else {
        ctx->device = c.device;
    }
    CK(cudaSetDevice(ctx->device));
    CK(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device));
    CK(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
    if (int frc = fork_create(ctx->fork)) return frc;
    CK(cudaMalloc(&ctx->pool_mem, (size_t)c.device_budget_bytes));
    {
        // exact fixed-point reciprocals: floor(x * 65536 / m) == (x * K[m]) >> 32
        // for 0 <= x <= m <= kMaxSentTokens (error of K below 1/m)
        // and the 32-bit form floor(x * 65536 / m) == umulhi(x << 17, R[m]),
        // R[m] = ceil(2^31 / m), for m <= kRecip31Max (after K in the same block)
        std::vector<uint64_t> K(kMaxSentTokens + 1, 0);
        for (int m = 1; m <= kMaxSentTokens; ++m) K[m] = ((uint64_t(1) << 48) + m - 1) / m;
        std::vector<uint32_t> R(kMaxSentTokens + 1, 0);
        for (int m = 1; m <= kMaxSentTokens; ++m) R[m] = (uint32_t)(((uint64_t(1) << 31) + m - 1) / m);
        CK(cudaMalloc(&ctx->recip, sizeof(uint64_t) * K.size() + sizeof(uint32_t) * R.size()));
        CK(cudaMemcpy(ctx->recip, K.data(), sizeof(uint64_t) * K.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(ctx->recip + K.size(), R.data(), sizeof(uint32_t) * R.size(), cudaMemcpyHostToDevice));
    }
    ctx->pool.base = static_cast<char *>(ctx->pool_mem);
    ctx->pool.size = c.device_budget_bytes;
    ctx->pool.free_[0] = c.device_budget_bytes;
    // one set of per-warp long-sentence tables per batch that can run at once
    ctx->gscratch_bytes = (size_t)ctx->num_sms * kGScratchWarpsPerSm * kScoreScratchPerWarp;
    CK(cudaMalloc(&ctx->gscratch, ctx->gscratch_bytes));
    CK(cudaEventCreate(&ctx->origin));
    CK(cudaEventRecord(ctx->origin, ctx->stream));
    for (int k = 0; k < c.max_inflight; ++k) {
        std::unique_ptr<Slot> s(new Slot());
        CK(cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking));
        if (int frc = fork_create(s->fork)) return frc;
        CK(cudaEventCreateWithFlags(&s->ev, cudaEventDisableTiming));
        CK(cudaEventCreate(&s->t0));
        CK(cudaEventCreate(&s->t1));
        CK(cudaMalloc(&s->gscratch, ctx->gscratch_bytes));
        ctx->slots.push_back(std::move(s));
    }
    mine_ctx *raw = ctx.release();
    raw->worker = std::thread(serving_loop, raw);
    *out = raw;
    return MINE_OK;
}

int mine_close(mine_ctx *ctx)
{
    if (!ctx) return MINE_OK;
    {
        std::lock_guard<std::mutex> lk(ctx->q_mu);
        ctx->stop = true;
    }
    ctx->q_cv.notify_all();
    if (ctx->worker.joinable()) ctx->worker.join();
    cudaSetDevice(ctx->device);
    // host-buffer batch calls still in flight: wait for them (the caller
    // keeps their arrays until this returns)
    for (AsyncCall &a : ctx->acall) {
        if (a.busy) {
            cudaEventSynchronize(a.done);
            const_cast<mine_dict *>(a.dict)->inflight--;
            a.busy = false;
        }
        if (a.in_ready) cudaEventDestroy(a.in_ready);
        if (a.packed) cudaEventDestroy(a.packed);
        if (a.done) cudaEventDestroy(a.done);
        if (a.gscratch) cudaFree(a.gscratch);
    }
    if (ctx->cstream) cudaStreamDestroy(ctx->cstream);
    if (ctx->ostream) cudaStreamDestroy(ctx->ostream);
    for (mine_result &r : ctx->ready) std::free(r.pairs);
    ctx->ready.clear();
    for (mine_dict *d : ctx->dicts) {
        cudaFree(d->slots_mem);
        cudaFree(d->trans_mem);
        delete d;
    }
    for (auto &s : ctx->slots) {
        cudaStreamDestroy(s->st);
        fork_destroy(s->fork);
        cudaEventDestroy(s->ev);
        if (s->t0) cudaEventDestroy(s->t0);
        if (s->t1) cudaEventDestroy(s->t1);
        cudaFree(s->gscratch);
    }
    if (ctx->origin) cudaEventDestroy(ctx->origin);
    cudaFree(ctx->gscratch);
    if (ctx->graph.exec) cudaGraphExecDestroy(ctx->graph.exec);
    ctx->slots.clear();
    for (auto &m : ctx->prof_pending) {
        cudaEventDestroy(m.a);
        cudaEventDestroy(m.b);
    }
    for (cudaEvent_t e : ctx->prof_free) cudaEventDestroy(e);
    cudaFree(ctx->pool_mem);
    cudaFree(ctx->recip);
    cudaStreamDestroy(ctx->stream);
    fork_destroy(ctx->fork);
    delete ctx;
    return MINE_OK;
}

int mine_dict_create(mine_ctx *ctx, const int32_t *keys, const int32_t *trans_off,
                     const int32_t *trans, int32_t n_keys, mine_dict **out)
{
    if (!ctx || !out || n_keys < 0 || (n_keys > 0 && (!keys || !trans_off)))
        return fail(MINE_EINVAL, "null argument or negative key count");
    *out = nullptr;
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    int rc = set_device(ctx);
    if (rc) return rc;
    if (n_keys > 0 && trans_off[0] != 0) return fail(MINE_EINVAL, "trans_off[0] must be 0");
    int kmax = 1;
    for (int32_t k = 0; k < n_keys; ++k) {
        if (keys[k] < 0 || keys[k] > MINE_MAX_TOKEN_ID) return fail(MINE_EINVAL, "key outside [0, 2^30)");
        const int32_t c = trans_off[k + 1] - trans_off[k];
        if (c < 0 || c > MINE_MAX_TRANS) return fail(MINE_EINVAL, "translation count outside [0, 32]");
        kmax = std::max(kmax, (int)c);
    }
    const int64_t n_trans = n_keys > 0 ? trans_off[n_keys] : 0;
    if (n_trans >= (int64_t(1) << 26)) return fail(MINE_EINVAL, "more than 2^26 translations");
    if (n_trans > 0 && !trans) return fail(MINE_EINVAL, "trans is NULL");
    for (int64_t k = 0; k < n_trans; ++k)
        if (trans[k] < 0 || trans[k] > MINE_MAX_TOKEN_ID) return fail(MINE_EINVAL, "translation outside [0, 2^30)");
    std::unique_ptr<mine_dict> d(new mine_dict());
    d->serial = ++ctx->dict_serial;
    // buckets of 8 slots, at most a quarter full on average
    d->d.log2 = std::max(4, ceil_log2_host(4 * (int64_t)n_keys));
    d->d.kmax = kmax;
    d->d.n_trans = n_trans;
    const size_t slots_bytes = sizeof(int2) << d->d.log2;
    // inline table: two entries per 64-byte bucket, at most half of them used
    d->d.inl_log2 = std::max(4, ceil_log2_host((int64_t)n_keys));
    const size_t inl_bytes = (size_t)64 << d->d.inl_log2;
    CK(cudaMalloc(&d->slots_mem, slots_bytes + inl_bytes));
    CK(cudaMalloc(&d->trans_mem, 4 * (size_t)std::max<int64_t>(n_trans, 1)));
    d->d.slots = static_cast<int2 *>(d->slots_mem);
    d->d.inl = reinterpret_cast<int4 *>(static_cast<char *>(d->slots_mem) + slots_bytes);
    d->d.trans = static_cast<int32_t *>(d->trans_mem);
    cudaStream_t st = ctx->stream;
    CK(cudaMemsetAsync(d->slots_mem, 0xff, slots_bytes + inl_bytes, st));
    if (n_trans > 0) CK(cudaMemcpyAsync(d->trans_mem, trans, 4 * n_trans, cudaMemcpyHostToDevice, st));
    if (n_keys > 0) {
        void *tmp = nullptr;
        const size_t kb = 4 * (size_t)n_keys, ob = 4 * ((size_t)n_keys + 1);
        CK(cudaMalloc(&tmp, kb + ob + 16));
        int32_t *dk = static_cast<int32_t *>(tmp);
        int32_t *doff = dk + n_keys;
        int32_t *derr = doff + n_keys + 1;
        CK(cudaMemcpyAsync(dk, keys, kb, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(doff, trans_off, ob, cudaMemcpyHostToDevice, st));
        CK(cudaMemsetAsync(derr, 0, 4, st));
        ctx->launches += timed_launch(ctx, KID_DICT, st, [&] { return launch_dict_build(dk, doff, n_keys, d->d, derr, st); });
        int32_t herr = 0;
        CK(cudaMemcpyAsync(&herr, derr, 4, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        cudaFree(tmp);
        if (herr) {
            cudaFree(d->slots_mem);
            cudaFree(d->trans_mem);
            return device_fail(herr);
        }
    }
    CK(cudaStreamSynchronize(st));
    mine_dict *raw = d.release();
    {
        std::lock_guard<std::mutex> q(ctx->q_mu);
        ctx->dicts.push_back(raw);
    }
    *out = raw;
    return MINE_OK;
}

int mine_dict_destroy(mine_ctx *ctx, mine_dict *dict)
{
    if (!ctx || !dict) return fail(MINE_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    std::lock_guard<std::mutex> q(ctx->q_mu);
    if (dict->inflight.load() > 0) return fail(MINE_EBUSY, "dictionary used by requests in flight");
    auto it = std::find(ctx->dicts.begin(), ctx->dicts.end(), dict);
    if (it == ctx->dicts.end()) return fail(MINE_EINVAL, "unknown dictionary");
    ctx->dicts.erase(it);
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    cudaFree(dict->slots_mem);
    cudaFree(dict->trans_mem);
    delete dict;
    return MINE_OK;
}

int64_t mine_batch_capacity(const int32_t *doc_off, int32_t n_pairs, int32_t n_settings)
{
    if (!doc_off || n_pairs < 0 || n_settings < 0) return 0;
    int64_t cap = 0;
    for (int32_t p = 0; p < n_pairs; ++p) {
        const int64_t S = doc_off[2 * p + 1] - doc_off[2 * p];
        const int64_t T = doc_off[2 * p + 2] - doc_off[2 * p + 1];
        cap += (int64_t)n_settings * std::max<int64_t>(0, std::min(S, T));
    }
    return cap;
}

static int check_settings(const mine_settings *s)
{
    if (!s || s->n < 1 || s->n > 256 || !s->gaps || !s->thresholds)
        return fail(MINE_EINVAL, "settings must hold 1..256 (gap, threshold) pairs");
    return 0;
}

static int check_batch(const mine_batch *b)
{
    if (!b || b->n_pairs < 0 || !b->doc_off || b->n_sent < 0 || b->n_tok < 0 ||
        (b->n_sent > 0 && !b->sent_off) || (b->n_tok > 0 && !b->tokens))
        return fail(MINE_EINVAL, "malformed batch");
    if (b->n_tok >= (int64_t(1) << 31) || b->n_sent >= (int64_t(1) << 31))
        return fail(MINE_EINVAL, "batch larger than 2^31 tokens or sentences");
    return 0;
}

// Buffers and streams of one host-buffer batch call.
struct HostCallRes {
    DevBuf *inbuf, *arena;
    HostBuf *pin;
    Plan *plan;
    void *gscratch;
    cudaStream_t st;         // kernels
    cudaStream_t cst;        // input and plan copies (st itself for a synchronous call)
    cudaEvent_t in_ready;    // recorded on cst after them when cst != st
    cudaStream_t ost;        // result copies (st itself for a synchronous call)
    cudaEvent_t packed;      // recorded on st after the packing when ost != st
    bool exact_sel = false;  // leave the triples on the device: the caller copies exactly their total
};

// Enqueue one host-buffer batch call of P > 0 pairs: the inputs go first,
// into their own buffer (their copy overlaps the planning), then the plan;
// the kernels and the packing of the selections follow on res.st, the copies
// of every result into the caller's arrays on res.ost.  Nothing waits for the device
// unless a step fails: then both streams are synchronised, so the caller may
// free its inputs on return.
static int enqueue_host_batch(mine_ctx *ctx, const mine_dict *dict, const mine_batch *batch,
                              const mine_settings *settings, mine_q16 *nw_score, int32_t *n_sel,
                              int64_t *sel_off, mine_pair *sel, int64_t sel_cap,
                              const HostCallRes &res, HostCallOut &out)
{
    const int32_t P = batch->n_pairs;
    const int n = settings->n;
    const cudaStream_t st = res.st, cst = res.cst;
    int rc = 0;
    const int64_t in_tok_at = align_up(4 * (batch->n_sent + 1), 256);
    if ((rc = ensure_dev(*res.inbuf, in_tok_at + 4 * batch->n_tok + 16))) return rc;
    int32_t *d_sent = static_cast<int32_t *>(res.inbuf->p);
    int32_t *d_tok = reinterpret_cast<int32_t *>(static_cast<char *>(res.inbuf->p) + in_tok_at);
    // from the first copy on, every failure waits for the copies and kernels
    // already enqueued on the call's streams before it returns: the caller may
    // free or reuse its arrays as soon as the call has returned
    auto bail = [&](int code) {
        cudaStreamSynchronize(cst);
        if (st != cst) cudaStreamSynchronize(st);
        if (res.ost != st) cudaStreamSynchronize(res.ost);
        return code;
    };
#define CKB(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = inject_cuda_error(ctx) ? cudaErrorInvalidValue : (call);                  \
        if (e_ != cudaSuccess)                                                                     \
            return bail(fail(MINE_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)));     \
    } while (0)
    CKB(cudaMemcpyAsync(d_sent, batch->sent_off, 4 * (batch->n_sent + 1), cudaMemcpyHostToDevice, cst));
    if (batch->n_tok > 0)
        CKB(cudaMemcpyAsync(d_tok, batch->tokens, 4 * batch->n_tok, cudaMemcpyHostToDevice, cst));
    std::vector<Setting> set(n);
    for (int k = 0; k < n; ++k) set[k] = Setting(settings->gaps[k], settings->thresholds[k]);
    Plan &pl = *res.plan;
    rc = build_plan(pl, P, batch->doc_off, batch->n_sent,
                    [&](int32_t, const Setting *&s, int &cnt) { s = set.data(); cnt = n; }, 65536, true,
                    ctx->align_tab);
    if (rc) return bail(rc);
    pl.n_tok = batch->n_tok;
    const int32_t R = pl.R;
    Layout L = make_layout(pl, dict->d.kmax, false, true, true);
    // packed outputs: offsets, triples, block sums
    const int64_t o_off = align_up(L.total, 256);
    const int64_t o_pk = o_off + align_up(8 * ((int64_t)R + 1), 256);
    const int64_t o_bs = o_pk + align_up(12 * pl.sel_cap + 16, 256);
    const int64_t total = o_bs + 4 * ((int64_t)R / 1024 + 1) + 16;
    const int64_t err_at = align_up(L.plan_bytes, 64);   // the error word after the plan
    if ((rc = ensure_dev(*res.arena, total))) return bail(rc);
    if ((rc = ensure_host(*res.pin, err_at + 64))) return bail(rc);
    char *hp = static_cast<char *>(res.pin->p);
    pack_plan(pl, L, hp);
    int32_t *h_err = reinterpret_cast<int32_t *>(hp + err_at);
    *h_err = 0;
    char *base = static_cast<char *>(res.arena->p);
    CKB(cudaMemcpyAsync(base + L.plan, hp, L.plan_bytes, cudaMemcpyHostToDevice, cst));
    if (cst != st) {
        CKB(cudaEventRecord(res.in_ready, cst));
        CKB(cudaStreamWaitEvent(st, res.in_ready, 0));
    }
    BatchDev b = make_batchdev(pl, L, base, d_sent, d_tok, nullptr, ctx->recip, res.gscratch);
    if (ctx->inject_withhold.load() > 0 && ctx->inject_withhold.fetch_sub(1) > 0) {
        b.test_withhold = 1;
        b.wait_spins = kTestWaitSpins;
    }
    if ((rc = enqueue_kernels(ctx, b, dict, batch->n_sent, batch->n_tok, true, st, true, &ctx->fork)))
        return bail(rc);
    int64_t *d_off = reinterpret_cast<int64_t *>(base + o_off);
    int32_t *d_pk = reinterpret_cast<int32_t *>(base + o_pk);
    int32_t *d_bs = reinterpret_cast<int32_t *>(base + o_bs);
    ctx->launches += timed_launch(ctx, KID_PACK, st, [&] { return launch_pack(b, n, R, d_bs, d_off, d_pk, st); });
    CKB(cudaGetLastError());
    // results straight into the caller's arrays
    const cudaStream_t ost = res.ost;
    if (ost != st) {
        CKB(cudaEventRecord(res.packed, st));
        CKB(cudaStreamWaitEvent(ost, res.packed, 0));
    }
    const int64_t cp = std::min(sel_cap, pl.sel_cap);
    CKB(cudaMemcpyAsync(nw_score, b.nw_score, 4 * (size_t)R, cudaMemcpyDeviceToHost, ost));
    CKB(cudaMemcpyAsync(n_sel, b.n_sel, 4 * (size_t)R, cudaMemcpyDeviceToHost, ost));
    CKB(cudaMemcpyAsync(sel_off, d_off, 8 * ((size_t)R + 1), cudaMemcpyDeviceToHost, ost));
    if (cp > 0 && sel && !res.exact_sel)
        CKB(cudaMemcpyAsync(sel, d_pk, 12 * (size_t)cp, cudaMemcpyDeviceToHost, ost));
    CKB(cudaMemcpyAsync(h_err, b.err, 4, cudaMemcpyDeviceToHost, ost));
    out.R = R;
    out.h_err = h_err;
    out.d_sel = res.exact_sel ? d_pk : nullptr;
    out.h2d = L.plan_bytes + 4 * (batch->n_sent + 1) + 4 * batch->n_tok;
    out.d2h = 8 * (int64_t)R + 8 * ((int64_t)R + 1) + 4 + (sel && !res.exact_sel ? 12 * cp : 0);
#undef CKB
    return MINE_OK;
}

// Status of a completed host-buffer batch call.
static int finish_host_batch(const HostCallOut &o, const int64_t *sel_off, const mine_pair *sel,
                             int64_t sel_cap)
{
    if (!o.h_err) return MINE_OK;   // no pairs
    if (*o.h_err) return device_fail(*o.h_err);
    const int64_t tot = sel_off[o.R];
    if (tot > sel_cap || (tot > 0 && !sel)) return fail(MINE_EINVAL, "sel_cap too small");
    return MINE_OK;
}

int mine_run_batch(mine_ctx *ctx, const mine_dict *dict, const mine_batch *batch,
                   const mine_settings *settings, mine_q16 *nw_score, int32_t *n_sel,
                   int64_t *sel_off, mine_pair *sel, int64_t sel_cap)
{
    if (!ctx || !dict) return fail(MINE_EINVAL, "null context or dictionary");
    int rc = check_batch(batch);
    if (rc) return rc;
    if ((rc = check_settings(settings))) return rc;
    const int32_t P = batch->n_pairs;
    if (P > 0 && (!nw_score || !n_sel || !sel_off)) return fail(MINE_EINVAL, "null output");
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    if ((rc = set_device(ctx))) return rc;
    ++ctx->arena_gen;
    sel_off[0] = 0;
    if (P == 0) return MINE_OK;
    // synchronous: once the offsets are back, copy exactly the selected
    // triples (a sweep's capacity, settings x min(S,T) per pair, is mostly
    // unused)
    HostCallRes res{&ctx->inbuf, &ctx->arena, &ctx->pin, &ctx->plan, ctx->gscratch, ctx->stream,
                    ctx->stream, nullptr, ctx->stream, nullptr};
    res.exact_sel = true;
    HostCallOut o;
    if ((rc = enqueue_host_batch(ctx, dict, batch, settings, nw_score, n_sel, sel_off, sel, sel_cap, res, o)))
        return rc;
    CK(cudaStreamSynchronize(ctx->stream));
    if ((rc = finish_host_batch(o, sel_off, sel, sel_cap))) return rc;
    const int64_t tot = sel_off[o.R];
    if (tot > 0) {
        const cudaError_t e = inject_cuda_error(ctx)
                                  ? cudaErrorInvalidValue
                                  : cudaMemcpy(sel, o.d_sel, 12 * (size_t)tot, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return fail(MINE_ECUDA, std::string("selected pairs copy: ") + cudaGetErrorString(e));
    }
    ctx->h2d_bytes += o.h2d;
    ctx->d2h_bytes += o.d2h + 12 * tot;
    return MINE_OK;
}

int mine_run_batch_async(mine_ctx *ctx, const mine_dict *dict, const mine_batch *batch,
                         const mine_settings *settings, mine_q16 *nw_score, int32_t *n_sel,
                         int64_t *sel_off, mine_pair *sel, int64_t sel_cap, uint64_t *ticket)
{
    if (!ctx || !dict || !ticket) return fail(MINE_EINVAL, "null context, dictionary or ticket");
    *ticket = 0;
    int rc = check_batch(batch);
    if (rc) return rc;
    if ((rc = check_settings(settings))) return rc;
    const int32_t P = batch->n_pairs;
    if (P > 0 && (!nw_score || !n_sel || !sel_off)) return fail(MINE_EINVAL, "null output");
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    if ((rc = set_device(ctx))) return rc;
    AsyncCall *c = nullptr;
    for (AsyncCall &a : ctx->acall)
        if (!a.busy) {
            c = &a;
            break;
        }
    if (!c) return fail(MINE_EAGAIN, "MINE_ASYNC_DEPTH batch calls in flight: wait for one first");
    if (!ctx->cstream) CK(cudaStreamCreateWithFlags(&ctx->cstream, cudaStreamNonBlocking));
    if (!ctx->ostream) CK(cudaStreamCreateWithFlags(&ctx->ostream, cudaStreamNonBlocking));
    if (!c->in_ready) CK(cudaEventCreateWithFlags(&c->in_ready, cudaEventDisableTiming));
    if (!c->packed) CK(cudaEventCreateWithFlags(&c->packed, cudaEventDisableTiming));
    if (!c->done) CK(cudaEventCreateWithFlags(&c->done, cudaEventDisableTiming));
    if (!c->gscratch) CK(cudaMalloc(&c->gscratch, ctx->gscratch_bytes));
    sel_off[0] = 0;
    c->out = HostCallOut{};
    if (P > 0) {
        const HostCallRes res{&c->inbuf, &c->arena, &c->pin, &c->plan, c->gscratch, ctx->stream,
                              ctx->cstream, c->in_ready, ctx->ostream, c->packed};
        if ((rc = enqueue_host_batch(ctx, dict, batch, settings, nw_score, n_sel, sel_off, sel, sel_cap,
                                     res, c->out)))
            return rc;
        ctx->h2d_bytes += c->out.h2d;
        ctx->d2h_bytes += c->out.d2h;
    }
    // P == 0: nothing was enqueued; the event still orders the wait after
    // earlier work of the context
    const cudaError_t er = cudaEventRecord(c->done, P > 0 ? ctx->ostream : ctx->stream);
    if (er != cudaSuccess) {   // nothing to wait on: finish the enqueued work here
        cudaStreamSynchronize(ctx->cstream);
        cudaStreamSynchronize(ctx->stream);
        cudaStreamSynchronize(ctx->ostream);
        return fail(MINE_ECUDA, std::string("cudaEventRecord: ") + cudaGetErrorString(er));
    }
    c->busy = true;
    c->waiting = false;
    c->ticket = ctx->next_async++;
    c->dict = dict;
    const_cast<mine_dict *>(dict)->inflight++;
    c->sel_off = sel_off;
    c->sel = sel;
    c->sel_cap = sel_cap;
    *ticket = c->ticket;
    return MINE_OK;
}

int mine_batch_wait(mine_ctx *ctx, uint64_t ticket)
{
    if (!ctx) return fail(MINE_EINVAL, "null context");
    AsyncCall *c = nullptr;
    {
        std::lock_guard<std::mutex> lk(ctx->api_mu);
        for (AsyncCall &a : ctx->acall)
            if (a.busy && !a.waiting && a.ticket == ticket) {
                c = &a;
                break;
            }
        if (!c) return fail(MINE_EINVAL, "no batch call in flight with this ticket");
        c->waiting = true;   // the slot stays taken while this thread waits without the lock
    }
    const cudaError_t e = cudaEventSynchronize(c->done);
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    const int rc = e == cudaSuccess ? finish_host_batch(c->out, c->sel_off, c->sel, c->sel_cap)
                                    : fail(MINE_ECUDA, std::string("cudaEventSynchronize: ") +
                                                           cudaGetErrorString(e));
    const_cast<mine_dict *>(c->dict)->inflight--;
    c->busy = c->waiting = false;
    return rc;
}

// The score matrices of a host batch, row-major pair after pair, as Q16
// integers (f32 = 0) or single-precision floats (f32 = 1); out holds 4-byte
// cells.
static int score_matrices(mine_ctx *ctx, const mine_dict *dict, const mine_batch *batch, void *out,
                          int64_t out_len, int f32)
{
    if (!ctx || !dict) return fail(MINE_EINVAL, "null context or dictionary");
    int rc = check_batch(batch);
    if (rc) return rc;
    const int32_t P = batch->n_pairs;
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    if ((rc = set_device(ctx))) return rc;
    ++ctx->arena_gen;
    const Setting set(-65536, 0);
    Plan pl;
    rc = build_plan(pl, P, batch->doc_off, batch->n_sent,
                    [&](int32_t, const Setting *&s, int &cnt) { s = &set; cnt = 1; }, 65536, true,
                    ctx->align_tab);
    if (rc) return rc;
    pl.n_tok = batch->n_tok;
    int64_t cells = 0;
    for (const PairPlan &pp : pl.pairs) cells += (int64_t)pp.S * pp.T;
    if (out_len < cells || (cells > 0 && !out)) return fail(MINE_EINVAL, "out shorter than the sum of S*T");
    if (P == 0 || cells == 0) return MINE_OK;
    const Layout L = make_layout(pl, dict->d.kmax, true, true, true);
    if ((rc = ensure_dev(ctx->arena, L.total))) return rc;
    const int64_t m_bytes = 4 * pl.m_elems;
    if ((rc = ensure_host(ctx->pin, align_up(L.plan_bytes, 64) + m_bytes + 64))) return rc;
    char *hp = static_cast<char *>(ctx->pin.p);
    pack_plan(pl, L, hp);
    char *base = static_cast<char *>(ctx->arena.p);
    cudaStream_t st = ctx->stream;
    int32_t *d_sent = reinterpret_cast<int32_t *>(base + L.sent_off);
    int32_t *d_tok = reinterpret_cast<int32_t *>(base + L.tokens);
    CK(cudaMemcpyAsync(base + L.plan, hp, L.plan_bytes, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_sent, batch->sent_off, 4 * (batch->n_sent + 1), cudaMemcpyHostToDevice, st));
    if (batch->n_tok > 0)
        CK(cudaMemcpyAsync(d_tok, batch->tokens, 4 * batch->n_tok, cudaMemcpyHostToDevice, st));
    BatchDev b = make_batchdev(pl, L, base, d_sent, d_tok, nullptr, ctx->recip, ctx->gscratch);
    b.f32 = f32;
    if ((rc = enqueue_kernels(ctx, b, dict, batch->n_sent, batch->n_tok, true, st, false, &ctx->fork))) return rc;
    int32_t *h_err = reinterpret_cast<int32_t *>(hp + align_up(L.plan_bytes, 64));
    const int32_t *h_m = h_err + 16;
    CK(cudaMemcpyAsync(h_err, b.err, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(const_cast<int32_t *>(h_m), b.M, m_bytes, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (*h_err) return device_fail(*h_err);
    // tiles -> row-major, pair after pair (4-byte cells copied as they are)
    int32_t *o32 = static_cast<int32_t *>(out);
    int64_t o = 0;
    for (const PairPlan &pp : pl.pairs) {
        const int TT = (pp.T + kTile - 1) / kTile;
        for (int i = 0; i < pp.S; ++i)
            for (int j = 0; j < pp.T; ++j) o32[o++] = h_m[m_cell(pp.m_off, TT, i, j)];
    }
    return MINE_OK;
}

int mine_score_f32(mine_ctx *ctx, const mine_dict *dict, const mine_batch *batch, float *out,
                   int64_t out_len)
{
    return score_matrices(ctx, dict, batch, out, out_len, 1);
}

int mine_score_q16(mine_ctx *ctx, const mine_dict *dict, const mine_batch *batch, mine_q16 *out,
                   int64_t out_len)
{
    return score_matrices(ctx, dict, batch, out, out_len, 0);
}

int mine_test_inject(mine_ctx *ctx, int32_t kind, int32_t count)
{
    if (!ctx || count < 0) return fail(MINE_EINVAL, "null context or negative count");
    if (kind == MINE_INJECT_CUDA_CALL) {
        ctx->inject_cuda_at.store(count);
    } else if (kind == MINE_INJECT_WITHHOLD_ROWS) {
        ctx->inject_withhold.store(count);
    } else {
        return fail(MINE_EINVAL, "unknown injection kind");
    }
    return MINE_OK;
}

int mine_run_batch_bidi(mine_ctx *ctx, const mine_dict *fwd, const mine_dict *bwd,
                        const mine_batch *batch, const mine_settings *settings, mine_q16 *nw_fwd,
                        mine_q16 *nw_bwd, int32_t *n_sel, int64_t *sel_off, mine_pair *sel,
                        int64_t sel_cap)
{
    if (!ctx || !fwd || !bwd) return fail(MINE_EINVAL, "null context or dictionary");
    int rc = check_batch(batch);
    if (rc) return rc;
    if ((rc = check_settings(settings))) return rc;
    const int32_t P = batch->n_pairs;
    const int n = settings->n;
    if (P > 0 && (!nw_fwd || !nw_bwd || !n_sel || !sel_off)) return fail(MINE_EINVAL, "null output");
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    if ((rc = set_device(ctx))) return rc;
    ++ctx->arena_gen;
    std::vector<Setting> set(n);
    for (int k = 0; k < n; ++k) set[k] = Setting(settings->gaps[k], settings->thresholds[k]);
    auto all = [&](int32_t, const Setting *&s, int &cnt) { s = set.data(); cnt = n; };
    Plan pf, pb;
    if ((rc = build_plan(pf, P, batch->doc_off, batch->n_sent, all, 65536, true, ctx->align_tab))) return rc;
    if ((rc = build_plan(pb, P, batch->doc_off, batch->n_sent, all, 65536, true, ctx->align_tab, true)))
        return rc;
    pf.n_tok = pb.n_tok = batch->n_tok;
    sel_off[0] = 0;
    if (P == 0) return MINE_OK;
    // one arena: the forward batch (with the inputs), the backward batch
    // (reading the same inputs), then the union and its counts
    const Layout Lf = make_layout(pf, fwd->d.kmax, true, true, true);
    const Layout Lb = make_layout(pb, bwd->d.kmax, false, true, true);
    const int64_t ob = align_up(Lf.total, 256);
    const int64_t ou = ob + align_up(Lb.total, 256);
    const int64_t on = ou + align_up(12 * 2 * pf.sel_cap + 16, 256);
    if ((rc = ensure_dev(ctx->arena, on + 4 * (int64_t)pf.R + 16))) return rc;
    const int64_t pb_at = align_up(Lf.plan_bytes, 64);
    const int64_t ho_at = pb_at + align_up(Lb.plan_bytes, 64);
    const int64_t out_bytes = 12 * (int64_t)pf.R + 16 + 24 * pf.sel_cap + 64;
    if ((rc = ensure_host(ctx->pin, ho_at + out_bytes))) return rc;
    char *hp = static_cast<char *>(ctx->pin.p);
    pack_plan(pf, Lf, hp);
    pack_plan(pb, Lb, hp + pb_at);
    char *base = static_cast<char *>(ctx->arena.p);
    cudaStream_t st = ctx->stream;
    int32_t *d_sent = reinterpret_cast<int32_t *>(base + Lf.sent_off);
    int32_t *d_tok = reinterpret_cast<int32_t *>(base + Lf.tokens);
    CK(cudaMemcpyAsync(base + Lf.plan, hp, Lf.plan_bytes, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(base + ob + Lb.plan, hp + pb_at, Lb.plan_bytes, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_sent, batch->sent_off, 4 * (batch->n_sent + 1), cudaMemcpyHostToDevice, st));
    if (batch->n_tok > 0)
        CK(cudaMemcpyAsync(d_tok, batch->tokens, 4 * batch->n_tok, cudaMemcpyHostToDevice, st));
    BatchDev bf = make_batchdev(pf, Lf, base, d_sent, d_tok, nullptr, ctx->recip, ctx->gscratch);
    BatchDev bb = make_batchdev(pb, Lb, base + ob, d_sent, d_tok, nullptr, ctx->recip, ctx->gscratch);
    if ((rc = enqueue_kernels(ctx, bf, fwd, batch->n_sent, batch->n_tok, true, st, true, &ctx->fork))) return rc;
    if ((rc = enqueue_kernels(ctx, bb, bwd, batch->n_sent, batch->n_tok, true, st, true, &ctx->fork))) return rc;
    UnionDev u;
    u.fwd = bf.pairs;
    u.bwd = bb.pairs;
    u.n_pairs = P;
    u.nset = n;
    u.sel_f = bf.sel;
    u.sel_b = bb.sel;
    u.nsel_f = bf.n_sel;
    u.nsel_b = bb.n_sel;
    u.out = reinterpret_cast<int32_t *>(base + ou);
    u.n_out = reinterpret_cast<int32_t *>(base + on);
    u.err_f = bf.err;
    u.err_b = bb.err;
    ctx->launches += timed_launch(ctx, KID_UNION, st, [&] { return launch_union(u, ctx->num_sms, st); });
    CK(cudaGetLastError());
    char *ho = hp + ho_at;
    int32_t *h_nwf = reinterpret_cast<int32_t *>(ho);
    int32_t *h_nwb = h_nwf + pf.R;
    int32_t *h_ns = h_nwb + pf.R;
    int32_t *h_err = h_ns + pf.R;
    int32_t *h_sel = h_err + 4;
    CK(cudaMemcpyAsync(h_nwf, bf.nw_score, 4 * pf.R, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(h_nwb, bb.nw_score, 4 * pf.R, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(h_ns, u.n_out, 4 * pf.R, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(h_err, bf.err, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(h_err + 1, bb.err, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(h_sel, u.out, 24 * pf.sel_cap, cudaMemcpyDeviceToHost, st));
    ctx->h2d_bytes += Lf.plan_bytes + Lb.plan_bytes + 4 * (batch->n_sent + 1) + 4 * batch->n_tok;
    ctx->d2h_bytes += 12 * (int64_t)pf.R + 8 + 24 * pf.sel_cap;
    CK(cudaStreamSynchronize(st));
    if (h_err[0]) return device_fail(h_err[0]);
    if (h_err[1]) return device_fail(h_err[1]);
    int64_t tot = 0;
    for (int32_t r = 0; r < pf.R; ++r) tot += h_ns[r];
    if (tot > sel_cap || (tot > 0 && !sel)) return fail(MINE_EINVAL, "sel_cap too small");
    int64_t o = 0;
    for (int32_t p = 0; p < P; ++p) {
        const PairPlan &pp = pf.pairs[p];
        const int64_t cap = std::min(pp.S, pp.T);
        for (int k = 0; k < n; ++k) {
            const int64_t r = (int64_t)p * n + k;
            nw_fwd[r] = h_nwf[r];
            nw_bwd[r] = h_nwb[r];
            n_sel[r] = h_ns[r];
            sel_off[r] = o;
            std::memcpy(sel + o, h_sel + 3 * 2 * (pp.sel_base + k * cap), 12 * (size_t)h_ns[r]);
            o += h_ns[r];
        }
    }
    sel_off[(int64_t)P * n] = o;
    return MINE_OK;
}

int mine_tune_f1(mine_ctx *ctx, const mine_dict *dict, const mine_batch *batch,
                 const mine_settings *settings, const int32_t *truth, int64_t *tp,
                 int64_t *n_selected, int64_t *n_truth, int32_t *best)
{
    if (!ctx || !dict) return fail(MINE_EINVAL, "null context or dictionary");
    int rc = check_batch(batch);
    if (rc) return rc;
    if ((rc = check_settings(settings))) return rc;
    const int32_t P = batch->n_pairs;
    const int n = settings->n;
    if (!tp || !n_selected || !n_truth || !best || (batch->n_sent > 0 && !truth))
        return fail(MINE_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    if ((rc = set_device(ctx))) return rc;
    ++ctx->arena_gen;
    std::vector<Setting> set(n);
    for (int k = 0; k < n; ++k) set[k] = Setting(settings->gaps[k], settings->thresholds[k]);
    Plan pl;
    rc = build_plan(pl, P, batch->doc_off, batch->n_sent,
                    [&](int32_t, const Setting *&s, int &cnt) { s = set.data(); cnt = n; }, 65536, true,
                    ctx->align_tab);
    if (rc) return rc;
    pl.n_tok = batch->n_tok;
    // a known pair names a target sentence of its own pair (or -1)
    for (const PairPlan &pp : pl.pairs)
        for (int32_t i = 0; i < pp.S; ++i) {
            const int32_t v = truth[pp.s0 + i];
            if (v < -1 || v >= pp.T) return fail(MINE_EINVAL, "truth entry outside [-1, T) of its pair");
        }
    for (int k = 0; k < n; ++k) tp[k] = n_selected[k] = 0;
    *n_truth = 0;
    *best = 0;
    if (P == 0) return MINE_OK;
    const Layout L = make_layout(pl, dict->d.kmax, true, true, true);
    const int64_t o_truth = align_up(L.total, 256);
    const int64_t o_acc = o_truth + align_up(4 * batch->n_sent + 16, 256);
    const int64_t acc_bytes = 8 * (2 * (int64_t)n + 1) + 16;
    if ((rc = ensure_dev(ctx->arena, o_acc + acc_bytes))) return rc;
    const int64_t ho_at = align_up(L.plan_bytes, 64);
    if ((rc = ensure_host(ctx->pin, ho_at + acc_bytes + 64))) return rc;
    char *hp = static_cast<char *>(ctx->pin.p);
    pack_plan(pl, L, hp);
    char *base = static_cast<char *>(ctx->arena.p);
    cudaStream_t st = ctx->stream;
    int32_t *d_sent = reinterpret_cast<int32_t *>(base + L.sent_off);
    int32_t *d_tok = reinterpret_cast<int32_t *>(base + L.tokens);
    int32_t *d_truth = reinterpret_cast<int32_t *>(base + o_truth);
    unsigned long long *d_acc = reinterpret_cast<unsigned long long *>(base + o_acc);
    CK(cudaMemcpyAsync(base + L.plan, hp, L.plan_bytes, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_sent, batch->sent_off, 4 * (batch->n_sent + 1), cudaMemcpyHostToDevice, st));
    if (batch->n_tok > 0)
        CK(cudaMemcpyAsync(d_tok, batch->tokens, 4 * batch->n_tok, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_truth, truth, 4 * batch->n_sent, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(d_acc, 0, acc_bytes, st));
    BatchDev b = make_batchdev(pl, L, base, d_sent, d_tok, nullptr, ctx->recip, ctx->gscratch);
    if ((rc = enqueue_kernels(ctx, b, dict, batch->n_sent, batch->n_tok, true, st, true, &ctx->fork))) return rc;
    F1Dev f;
    f.pairs = b.pairs;
    f.n_pairs = P;
    f.nset = n;
    f.sel = b.sel;
    f.n_sel = b.n_sel;
    f.truth = d_truth;
    f.acc = d_acc;
    f.best = reinterpret_cast<int32_t *>(d_acc + 2 * n + 1);
    f.err = b.err;
    ctx->launches += timed_launch(ctx, KID_F1, st, [&] { return launch_f1(f, ctx->num_sms, st); });
    CK(cudaGetLastError());
    unsigned long long *h_acc = reinterpret_cast<unsigned long long *>(hp + ho_at);
    int32_t *h_err = reinterpret_cast<int32_t *>(h_acc + 2 * n + 2);
    CK(cudaMemcpyAsync(h_acc, d_acc, 8 * (2 * (int64_t)n + 2), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(h_err, b.err, 4, cudaMemcpyDeviceToHost, st));
    ctx->h2d_bytes += L.plan_bytes + 4 * (batch->n_sent + 1) + 4 * batch->n_tok + 4 * batch->n_sent;
    ctx->d2h_bytes += 8 * (2 * (int64_t)n + 2) + 4;
    CK(cudaStreamSynchronize(st));
    if (*h_err) return device_fail(*h_err);
    for (int k = 0; k < n; ++k) {
        tp[k] = (int64_t)h_acc[k];
        n_selected[k] = (int64_t)h_acc[n + k];
    }
    *n_truth = (int64_t)h_acc[2 * n];
    *best = *reinterpret_cast<const int32_t *>(h_acc + 2 * n + 1);
    return MINE_OK;
}

int mine_best_match(mine_ctx *ctx, const mine_dict *dict, const mine_batch *batch, mine_q16 threshold,
                    int32_t *n_sel, int32_t *repeated, int64_t *sel_off, mine_pair *sel, int64_t sel_cap)
{
    if (!ctx || !dict) return fail(MINE_EINVAL, "null context or dictionary");
    int rc = check_batch(batch);
    if (rc) return rc;
    const int32_t P = batch->n_pairs;
    if (P > 0 && (!n_sel || !repeated || !sel_off)) return fail(MINE_EINVAL, "null output");
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    if ((rc = set_device(ctx))) return rc;
    ++ctx->arena_gen;
    const Setting set(-65536, threshold);   // validates the threshold; no alignment runs
    Plan pl;
    rc = build_plan(pl, P, batch->doc_off, batch->n_sent,
                    [&](int32_t, const Setting *&s, int &cnt) { s = &set; cnt = 1; }, 65536, true,
                    ctx->align_tab);
    if (rc) return rc;
    pl.n_tok = batch->n_tok;
    if (sel_off) sel_off[0] = 0;
    if (P == 0) return MINE_OK;
    const Layout L = make_layout(pl, dict->d.kmax, true, false, true);
    const int64_t ns = batch->n_sent;
    const int64_t words = ns / 32 + 1;
    const int64_t o_best = align_up(L.total, 256);
    const int64_t o_out = o_best + align_up(8 * ns + 16, 256);
    const int64_t o_cnt = o_out + align_up(12 * ns + 16, 256);
    const int64_t o_bits = o_cnt + align_up(8 * (int64_t)P + 16, 256);
    if ((rc = ensure_dev(ctx->arena, o_bits + 8 * words + 16))) return rc;
    const int64_t ho = align_up(L.plan_bytes, 64);
    if ((rc = ensure_host(ctx->pin, ho + 8 * (int64_t)P + 12 * ns + 64))) return rc;
    char *hp = static_cast<char *>(ctx->pin.p);
    pack_plan(pl, L, hp);
    char *base = static_cast<char *>(ctx->arena.p);
    cudaStream_t st = ctx->stream;
    int32_t *d_sent = reinterpret_cast<int32_t *>(base + L.sent_off);
    int32_t *d_tok = reinterpret_cast<int32_t *>(base + L.tokens);
    CK(cudaMemcpyAsync(base + L.plan, hp, L.plan_bytes, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_sent, batch->sent_off, 4 * (batch->n_sent + 1), cudaMemcpyHostToDevice, st));
    if (batch->n_tok > 0)
        CK(cudaMemcpyAsync(d_tok, batch->tokens, 4 * batch->n_tok, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(base + o_bits, 0, 8 * words, st));
    BatchDev b = make_batchdev(pl, L, base, d_sent, d_tok, nullptr, ctx->recip, ctx->gscratch);
    if ((rc = enqueue_kernels(ctx, b, dict, batch->n_sent, batch->n_tok, true, st, false, &ctx->fork))) return rc;
    BestDev d;
    d.pairs = b.pairs;
    d.n_pairs = P;
    d.items = b.prep_items;
    d.n_items = b.n_prep_items;
    d.M = b.M;
    d.thr = threshold;
    d.best = reinterpret_cast<int2 *>(base + o_best);
    d.out = reinterpret_cast<int32_t *>(base + o_out);
    d.n_sel = reinterpret_cast<int32_t *>(base + o_cnt);
    d.rep = d.n_sel + P;
    d.seen1 = reinterpret_cast<uint32_t *>(base + o_bits);
    d.seen2 = d.seen1 + words;
    d.err = b.err;
    ctx->launches += timed_launch(ctx, KID_BEST, st, [&] { return launch_best(d, ctx->num_sms, st); });
    CK(cudaGetLastError());
    int32_t *h_cnt = reinterpret_cast<int32_t *>(hp + ho);
    int32_t *h_out = h_cnt + 2 * P;
    int32_t h_err = 0;
    CK(cudaMemcpyAsync(h_cnt, d.n_sel, 8 * (size_t)P, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(h_out, d.out, 12 * (size_t)ns, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&h_err, b.err, 4, cudaMemcpyDeviceToHost, st));
    ctx->h2d_bytes += L.plan_bytes + 4 * (batch->n_sent + 1) + 4 * batch->n_tok;
    ctx->d2h_bytes += 8 * (int64_t)P + 12 * ns + 4;
    CK(cudaStreamSynchronize(st));
    if (h_err) return device_fail(h_err);
    int64_t tot = 0;
    for (int32_t p = 0; p < P; ++p) tot += h_cnt[p];
    if (tot > sel_cap || (tot > 0 && !sel)) return fail(MINE_EINVAL, "sel_cap too small");
    int64_t o = 0;
    for (int32_t p = 0; p < P; ++p) {
        n_sel[p] = h_cnt[p];
        repeated[p] = h_cnt[P + p];
        sel_off[p] = o;
        std::memcpy(sel + o, h_out + 3 * (int64_t)pl.pairs[p].s0, 12 * (size_t)h_cnt[p]);
        o += h_cnt[p];
    }
    sel_off[P] = o;
    return MINE_OK;
}

int mine_run_batch_device(mine_ctx *ctx, const mine_dict *dict, const mine_batch *batch,
                          const int32_t *doc_off_host, const mine_settings *settings,
                          mine_q16 *nw_score, int32_t *n_sel, mine_pair *sel, int64_t sel_cap,
                          void *stream)
{
    if (!ctx || !dict || !doc_off_host || !batch) return fail(MINE_EINVAL, "null argument");
    mine_batch bh = *batch;          // only the host copy of doc_off is read
    bh.doc_off = doc_off_host;
    int rc = check_batch(&bh);
    if (rc) return rc;
    if ((rc = check_settings(settings))) return rc;
    const int32_t P = batch->n_pairs;
    const int n = settings->n;
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    if ((rc = set_device(ctx))) return rc;
    cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : ctx->stream;
    mine_ctx::Graph &G = ctx->graph;
    // the same batch, settings, buffers and stream as the captured call, and
    // nothing rewrote the scratch since: replay (every kernel runs again)
    if (!ctx->prof_on && G.exec && G.gen == ctx->arena_gen && G.dict_serial == dict->serial &&
        G.P == P && G.n_sent == batch->n_sent && G.n_tok == batch->n_tok && G.sel_cap == sel_cap &&
        G.sent_off == batch->sent_off && G.tokens == batch->tokens && G.nw == nw_score &&
        G.ns == n_sel && G.sel == sel && G.stream == st && (int)G.gaps.size() == n &&
        std::equal(G.gaps.begin(), G.gaps.end(), settings->gaps) &&
        std::equal(G.thr.begin(), G.thr.end(), settings->thresholds) &&
        std::equal(G.doc_off.begin(), G.doc_off.end(), doc_off_host)) {
        CK(cudaGraphLaunch(G.exec, st));
        ctx->launches += G.launches;
        ctx->err_off = G.err_off;
        return MINE_OK;
    }
    ++ctx->arena_gen;
    std::vector<Setting> set(n);
    for (int k = 0; k < n; ++k) set[k] = Setting(settings->gaps[k], settings->thresholds[k]);
    Plan pl;
    rc = build_plan(pl, P, doc_off_host, batch->n_sent,
                    [&](int32_t, const Setting *&s, int &cnt) { s = set.data(); cnt = n; }, 65536, true,
                    ctx->align_tab);
    if (rc) return rc;
    pl.n_tok = batch->n_tok;
    if (P == 0) return MINE_OK;
    if (sel_cap < pl.sel_cap || !sel || !nw_score || !n_sel)
        return fail(MINE_EINVAL, "sel_cap below mine_batch_capacity() or null output");
    const Layout L = make_layout(pl, dict->d.kmax, false, false, true);
    if ((rc = ensure_dev(ctx->arena, L.total))) return rc;
    if ((rc = ensure_host(ctx->pin, L.plan_bytes + 64))) return rc;
    // the staging buffer may still feed the previous call's copy
    CK(cudaStreamSynchronize(st));
    char *hp = static_cast<char *>(ctx->pin.p);
    pack_plan(pl, L, hp);
    char *base = static_cast<char *>(ctx->arena.p);
    BatchDev b = make_batchdev(pl, L, base, batch->sent_off, batch->tokens,
                               reinterpret_cast<int32_t *>(sel), ctx->recip, ctx->gscratch);
    b.nw_score = nw_score;
    b.n_sel = n_sel;
    ctx->err_off = L.counters + 4 * 8;
    if (ctx->prof_on) {   // per-kernel events: plain launches
        CK(cudaMemcpyAsync(base + L.plan, hp, L.plan_bytes, cudaMemcpyHostToDevice, st));
        return enqueue_kernels(ctx, b, dict, batch->n_sent, batch->n_tok, true, st, true, &ctx->fork);
    }
    // capture the plan upload and the kernels as one graph, then launch it
    if (G.exec) {
        cudaGraphExecDestroy(G.exec);
        G.exec = nullptr;
    }
    const int64_t before = ctx->launches.load();
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
    cudaError_t ce = cudaMemcpyAsync(base + L.plan, hp, L.plan_bytes, cudaMemcpyHostToDevice, st);
    rc = ce == cudaSuccess ? enqueue_kernels(ctx, b, dict, batch->n_sent, batch->n_tok, true, st, true, &ctx->fork)
                           : fail(MINE_ECUDA, cudaGetErrorString(ce));
    cudaGraph_t graph = nullptr;
    ce = cudaStreamEndCapture(st, &graph);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (ce != cudaSuccess) return fail(MINE_ECUDA, cudaGetErrorString(ce));
    cudaGraphExec_t exec = nullptr;
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return fail(MINE_ECUDA, cudaGetErrorString(ce));
    CK(cudaGraphLaunch(exec, st));
    G.exec = exec;
    G.gen = ctx->arena_gen;
    G.dict_serial = dict->serial;
    G.P = P;
    G.n_sent = batch->n_sent;
    G.n_tok = batch->n_tok;
    G.sel_cap = sel_cap;
    G.sent_off = batch->sent_off;
    G.tokens = batch->tokens;
    G.nw = nw_score;
    G.ns = n_sel;
    G.sel = sel;
    G.stream = st;
    G.gaps.assign(settings->gaps, settings->gaps + n);
    G.thr.assign(settings->thresholds, settings->thresholds + n);
    G.doc_off.assign(doc_off_host, doc_off_host + 2 * (int64_t)P + 1);
    G.launches = (int)(ctx->launches.load() - before);
    G.err_off = ctx->err_off;
    return MINE_OK;
}

int mine_align_matrix(mine_ctx *ctx, const mine_q16 *M, int32_t S, int32_t T, mine_q16 gap,
                      mine_q16 threshold, mine_pair *out, int32_t *n_out, mine_q16 *nw_score)
{
    if (!ctx || !n_out || !nw_score || S < 0 || T < 0 || S > MINE_MAX_SENTENCES ||
        T > MINE_MAX_SENTENCES || (S > 0 && T > 0 && !M))
        return fail(MINE_EINVAL, "bad argument");
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    int rc = set_device(ctx);
    if (rc) return rc;
    ++ctx->arena_gen;
    int64_t maxabs = 0;
    for (int64_t k = 0; k < (int64_t)S * T; ++k)
        maxabs = std::max<int64_t>(maxabs, M[k] < 0 ? -(int64_t)M[k] : (int64_t)M[k]);
    const int32_t doc_off[3] = {0, S, S + T};
    const Setting set(gap, threshold);
    Plan pl;
    rc = build_plan(pl, 1, doc_off, (int64_t)S + T,
                    [&](int32_t, const Setting *&s, int &cnt) { s = &set; cnt = 1; }, maxabs, false,
                    ctx->align_tab);
    if (rc) return rc;
    if (std::min(S, T) > 0 && !out) return fail(MINE_EINVAL, "out is NULL");
    const Layout L = make_layout(pl, 1, false, true, false);
    if ((rc = ensure_dev(ctx->arena, L.total))) return rc;
    const int64_t out_bytes = 8 + 12 * pl.sel_cap + 64;
    if ((rc = ensure_host(ctx->pin, L.plan_bytes + out_bytes))) return rc;
    char *hp = static_cast<char *>(ctx->pin.p);
    pack_plan(pl, L, hp);
    char *base = static_cast<char *>(ctx->arena.p);
    cudaStream_t st = ctx->stream;
    CK(cudaMemcpyAsync(base + L.plan, hp, L.plan_bytes, cudaMemcpyHostToDevice, st));
    BatchDev b = make_batchdev(pl, L, base, nullptr, nullptr, nullptr, ctx->recip, ctx->gscratch);
    if (S > 0 && T > 0) {
        int32_t *mrow = reinterpret_cast<int32_t *>(base + L.Mrow);
        CK(cudaMemcpyAsync(mrow, M, 4 * (size_t)S * T, cudaMemcpyHostToDevice, st));
        ctx->launches += timed_launch(ctx, KID_TILE, st, [&] { return launch_tile(mrow, S, T, b.M, st); });
    }
    if ((rc = enqueue_kernels(ctx, b, nullptr, 0, 0, false, st))) return rc;
    char *ho = hp + align_up(L.plan_bytes, 64);
    int32_t *h = reinterpret_cast<int32_t *>(ho);
    CK(cudaMemcpyAsync(h, b.nw_score, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(h + 1, b.n_sel, 4, cudaMemcpyDeviceToHost, st));
    if (pl.sel_cap > 0)
        CK(cudaMemcpyAsync(h + 2, b.sel, 12 * pl.sel_cap, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *nw_score = h[0];
    *n_out = h[1];
    if (h[1] > 0) std::memcpy(out, h + 2, 12 * (size_t)h[1]);
    return MINE_OK;
}

int mine_check(mine_ctx *ctx)
{
    if (!ctx) return fail(MINE_EINVAL, "null context");
    std::lock_guard<std::mutex> lk(ctx->api_mu);
    int rc = set_device(ctx);
    if (rc) return rc;
    CK(cudaDeviceSynchronize());
    if (ctx->err_off >= 0 && ctx->arena.p) {
        int32_t e = 0;
        CK(cudaMemcpy(&e, static_cast<char *>(ctx->arena.p) + ctx->err_off, 4, cudaMemcpyDeviceToHost));
        if (e) return device_fail(e);
    }
    return MINE_OK;
}

int mine_io_bytes(mine_ctx *ctx, int64_t *h2d, int64_t *d2h)
{
    if (!ctx || !h2d || !d2h) return fail(MINE_EINVAL, "null argument");
    *h2d = ctx->h2d_bytes.load();
    *d2h = ctx->d2h_bytes.load();
    return MINE_OK;
}

int mine_profile(mine_ctx *ctx, int32_t enable)
{
    if (!ctx) return fail(MINE_EINVAL, "null context");
    std::lock_guard<std::mutex> g(ctx->prof_mu);
    ctx->prof_on = enable != 0;
    return MINE_OK;
}

int mine_profile_read(mine_ctx *ctx, double *ms, int64_t *launches, int32_t n)
{
    if (!ctx || n < 0 || (n > 0 && (!ms || !launches))) return fail(MINE_EINVAL, "bad argument");
    std::vector<mine_ctx::Mark> marks;
    {
        std::lock_guard<std::mutex> g(ctx->prof_mu);
        marks.swap(ctx->prof_pending);
    }
    cudaSetDevice(ctx->device);
    for (auto &m : marks) {
        CK(cudaEventSynchronize(m.b));
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, m.a, m.b));
        std::lock_guard<std::mutex> g(ctx->prof_mu);
        ctx->prof_ms[m.kid] += t;
        ctx->prof_n[m.kid] += 1;
        ctx->prof_free.push_back(m.a);
        ctx->prof_free.push_back(m.b);
    }
    std::lock_guard<std::mutex> g(ctx->prof_mu);
    for (int k = 0; k < n && k < KID_COUNT; ++k) {
        ms[k] = ctx->prof_ms[k];
        launches[k] = ctx->prof_n[k];
    }
    for (int k = 0; k < KID_COUNT; ++k) {
        ctx->prof_ms[k] = 0;
        ctx->prof_n[k] = 0;
    }
    return KID_COUNT;
}

const char *mine_kernel_name(int32_t id)
{
    static const char *names[KID_COUNT] = {"k_dict_build", "k_validate", "k_prep", "k_score",
                                           "k_align", "k_tile", "k_trace", "k_order",
                                           "k_pairprep", "k_score_wide", "k_align_tiled",
                                           "k_union", "k_f1", "k_pairprep_wide", "k_pack", "k_best",
                                           "k_pairprep_xwide", "k_score_xwide"};
    return (id >= 0 && id < KID_COUNT) ? names[id] : "";
}

// ------------------------------------------------------------------ serving

static int copy_doc(const mine_doc *d, std::vector<int32_t> &off, std::vector<int32_t> &tok)
{
    if (!d || d->n_sent < 0 || d->n_sent > MINE_MAX_SENTENCES || (d->n_sent > 0 && !d->sent_off))
        return fail(MINE_EINVAL, "malformed document");
    if (d->n_sent == 0) {
        off.assign(1, 0);
        tok.clear();
        return 0;
    }
    if (d->sent_off[0] != 0) return fail(MINE_EINVAL, "sent_off[0] must be 0");
    for (int32_t k = 0; k < d->n_sent; ++k) {
        const int64_t L = (int64_t)d->sent_off[k + 1] - d->sent_off[k];
        if (L < 0 || L > MINE_MAX_SENT_TOKENS) return fail(MINE_EINVAL, "sentence length outside [0, 1024]");
    }
    const int64_t nt = d->sent_off[d->n_sent];
    if (nt > 0 && !d->tokens) return fail(MINE_EINVAL, "tokens is NULL");
    for (int64_t k = 0; k < nt; ++k)
        if (d->tokens[k] < 0 || d->tokens[k] > MINE_MAX_TOKEN_ID) return fail(MINE_EINVAL, "token outside [0, 2^30)");
    off.assign(d->sent_off, d->sent_off + d->n_sent + 1);
    tok.assign(d->tokens, d->tokens + nt);
    return 0;
}

int mine_submit_sweep(mine_ctx *ctx, const mine_doc *src, const mine_doc *tgt,
                      const mine_dict *dict, int32_t n, const mine_q16 *gaps,
                      const mine_q16 *thresholds, uint64_t *ticket)
{
    if (!ctx || !dict || !ticket || n < 1 || n > 256 || !gaps || !thresholds)
        return fail(MINE_EINVAL, "bad argument");
    Request rq;
    int rc = copy_doc(src, rq.src_off, rq.src_tok);
    if (rc) return rc;
    if ((rc = copy_doc(tgt, rq.tgt_off, rq.tgt_tok))) return rc;
    rq.dict = dict;
    rq.settings.resize(n);
    for (int k = 0; k < n; ++k) rq.settings[k] = Setting(gaps[k], thresholds[k]);
    // footprint of the request alone (also validates gap/threshold/overflow)
    const int32_t S = (int32_t)rq.src_off.size() - 1, T = (int32_t)rq.tgt_off.size() - 1;
    const int32_t doc_off[3] = {0, S, S + T};
    Plan pl;
    rc = build_plan(pl, 1, doc_off, (int64_t)S + T,
                    [&](int32_t, const Setting *&s, int &cnt) { s = rq.settings.data(); cnt = n; },
                    65536, true);
    if (rc) return rc;
    pl.n_tok = (int64_t)rq.src_tok.size() + (int64_t)rq.tgt_tok.size();
    rq.footprint = request_footprint(pl, dict->d.kmax);
    if (rq.footprint > ctx->pool.size) return fail(MINE_ENOMEM, "request alone exceeds the device budget");
    rq.t_submit = std::chrono::steady_clock::now();
    {
        std::lock_guard<std::mutex> lk(ctx->q_mu);
        if (ctx->stop) return fail(MINE_EINVAL, "context is closing");
        rq.ticket = ctx->next_ticket++;
        *ticket = rq.ticket;
        const_cast<mine_dict *>(dict)->inflight++;
        ctx->in_flight_reqs++;
        ctx->pending.push_back(std::move(rq));
    }
    ctx->q_cv.notify_all();
    return MINE_OK;
}

int mine_submit(mine_ctx *ctx, const mine_doc *src, const mine_doc *tgt, const mine_dict *dict,
                mine_q16 gap, mine_q16 threshold, uint64_t *ticket)
{
    return mine_submit_sweep(ctx, src, tgt, dict, 1, &gap, &threshold, ticket);
}

int mine_poll(mine_ctx *ctx, mine_result *out, int32_t max_out, int32_t timeout_us)
{
    if (!ctx || (max_out > 0 && !out) || max_out < 0) return fail(MINE_EINVAL, "bad argument");
    std::unique_lock<std::mutex> lk(ctx->q_mu);
    auto have = [&] { return !ctx->ready.empty() || (timeout_us < 0 && ctx->in_flight_reqs == 0); };
    if (timeout_us > 0) {
        ctx->r_cv.wait_for(lk, std::chrono::microseconds(timeout_us), have);
    } else if (timeout_us < 0) {
        ctx->r_cv.wait(lk, have);
    }
    int got = 0;
    while (got < max_out && !ctx->ready.empty()) {
        out[got++] = ctx->ready.front();
        ctx->ready.pop_front();
    }
    return got;
}

int mine_serving_stats(mine_ctx *ctx, int64_t *batches, int32_t *max_overlap)
{
    if (!ctx) return fail(MINE_EINVAL, "null context");
    std::vector<std::pair<float, int>> ev;
    int64_t nb = 0;
    {
        std::lock_guard<std::mutex> lk(ctx->q_mu);
        nb = ctx->n_batches;
        ev.reserve(2 * ctx->spans.size());
        for (const auto &sp : ctx->spans) {
            ev.emplace_back(sp.first, +1);
            ev.emplace_back(sp.second, -1);
        }
    }
    // sweep over the span ends in time order (an end before a start at the
    // same instant: touching spans do not overlap)
    std::sort(ev.begin(), ev.end());
    int cur = 0, best = 0;
    for (const auto &e : ev) {
        cur += e.second;
        best = std::max(best, cur);
    }
    if (batches) *batches = nb;
    if (max_overlap) *max_overlap = best;
    return MINE_OK;
}

void mine_result_free(mine_ctx *, mine_result *result)
{
    if (!result) return;
    std::free(result->pairs);
    result->pairs = nullptr;
    result->n_pairs = 0;
}

}  // extern "C"

// The serving engine.  Batches are formed from the front of the pending
// queue (same dictionary, at most max_batch_pairs, total footprint that fits
// the free part of the budget pool), launched on a free slot's stream, and
// harvested when their event completes.  While batches run, new arrivals
// wait at most batch_window_us before they form the next batch, which runs
// concurrently on another slot.
namespace {

constexpr size_t kMaxSpans = 1 << 16;   // served batches whose device span is kept

void finish_slot(mine_ctx *ctx, Slot &s)
{
    const char *ho = static_cast<const char *>(s.pin_out.p);
    const int32_t *h_nw = reinterpret_cast<const int32_t *>(ho + s.out_nw);
    const int32_t *h_ns = reinterpret_cast<const int32_t *>(ho + s.out_nsel);
    const int32_t *h_sel = reinterpret_cast<const int32_t *>(ho + s.out_sel);
    const int32_t dev_err = *reinterpret_cast<const int32_t *>(ho + s.out_err);
    const cudaError_t ce = cudaEventQuery(s.ev);
    const auto now = std::chrono::steady_clock::now();
    std::vector<mine_result> res;
    for (size_t p = 0; p < s.reqs.size(); ++p) {
        const Request &rq = s.reqs[p];
        const PairPlan &pp = s.plan.pairs[p];
        const int64_t cap = std::min(pp.S, pp.T);
        for (int k = 0; k < pp.nset; ++k) {
            mine_result r{};
            r.ticket = rq.ticket;
            r.setting = k;
            r.latency_ns = std::chrono::duration_cast<std::chrono::nanoseconds>(now - rq.t_submit).count();
            if (ce != cudaSuccess) {
                r.status = MINE_ECUDA;
            } else if (dev_err) {
                r.status = dev_err == ERR_TIMEOUT ? MINE_ETIMEDOUT : MINE_EINVAL;
            } else {
                const int64_t row = pp.set0 + k;
                r.nw_score = h_nw[row];
                r.n_pairs = h_ns[row];
                if (r.n_pairs > 0) {
                    r.pairs = static_cast<mine_pair *>(std::malloc(sizeof(mine_pair) * r.n_pairs));
                    std::memcpy(r.pairs, h_sel + 3 * (pp.sel_base + k * cap), 12 * (size_t)r.n_pairs);
                }
            }
            res.push_back(r);
        }
    }
    float a = 0.f, z = 0.f;
    const bool timed = ce == cudaSuccess && cudaEventElapsedTime(&a, ctx->origin, s.t0) == cudaSuccess &&
                       cudaEventElapsedTime(&z, ctx->origin, s.t1) == cudaSuccess;
    {
        std::lock_guard<std::mutex> lk(ctx->q_mu);
        ctx->n_batches++;
        if (timed) {
            if (ctx->spans.size() >= kMaxSpans) ctx->spans.erase(ctx->spans.begin(), ctx->spans.begin() + kMaxSpans / 2);
            ctx->spans.emplace_back(a, z);
        }
        for (auto &r : res) ctx->ready.push_back(r);
        for (auto &rq : s.reqs) {
            const_cast<mine_dict *>(rq.dict)->inflight--;
            ctx->in_flight_reqs--;
        }
        ctx->pool.release(s.pool_off, s.pool_bytes);
    }
    s.reqs.clear();
    s.busy = false;
    ctx->r_cv.notify_all();
}

// Pack requests into one batch and launch it on slot s.  Returns 0 or an error.
int launch_slot(mine_ctx *ctx, Slot &s)
{
    const int P = (int)s.reqs.size();
    std::vector<int32_t> doc_off(2 * P + 1, 0);
    int64_t n_sent = 0, n_tok = 0;
    for (int p = 0; p < P; ++p) {
        const Request &rq = s.reqs[p];
        doc_off[2 * p + 1] = doc_off[2 * p] + (int32_t)rq.src_off.size() - 1;
        doc_off[2 * p + 2] = doc_off[2 * p + 1] + (int32_t)rq.tgt_off.size() - 1;
        n_tok += (int64_t)rq.src_tok.size() + (int64_t)rq.tgt_tok.size();
    }
    n_sent = doc_off[2 * P];
    const mine_dict *dict = s.reqs[0].dict;
    int rc = build_plan(s.plan, P, doc_off.data(), n_sent,
                        [&](int32_t p, const Setting *&set, int &cnt) {
                            set = s.reqs[p].settings.data();
                            cnt = (int)s.reqs[p].settings.size();
                        },
                        65536, true, ctx->align_tab);
    if (rc) return rc;
    s.plan.n_tok = n_tok;
    s.lay = make_layout(s.plan, dict->d.kmax, true, true, true);
    const Layout &L = s.lay;
    if (L.total > s.pool_bytes) return fail(MINE_ENOMEM, "batch layout exceeds its budget region");
    // host staging: plan | sent_off | tokens ; outputs: nw | nsel | err | sel
    const int64_t in_bytes = align_up(L.plan_bytes, 64) + 4 * (n_sent + 1) + 4 * n_tok + 64;
    if ((rc = ensure_host(s.pin_in, in_bytes))) return rc;
    s.out_nw = 0;
    s.out_nsel = align_up(4 * (int64_t)s.plan.R, 16);
    s.out_err = s.out_nsel + align_up(4 * (int64_t)s.plan.R, 16);
    s.out_sel = s.out_err + 16;
    if ((rc = ensure_host(s.pin_out, s.out_sel + 12 * s.plan.sel_cap + 16))) return rc;
    char *hi = static_cast<char *>(s.pin_in.p);
    pack_plan(s.plan, L, hi);
    int32_t *h_sent = reinterpret_cast<int32_t *>(hi + align_up(L.plan_bytes, 64));
    int32_t *h_tok = h_sent + n_sent + 1;
    int64_t so = 0, to = 0;
    h_sent[0] = 0;
    for (int p = 0; p < P; ++p) {
        const Request &rq = s.reqs[p];
        for (int side = 0; side < 2; ++side) {
            const std::vector<int32_t> &off = side ? rq.tgt_off : rq.src_off;
            const std::vector<int32_t> &tk = side ? rq.tgt_tok : rq.src_tok;
            const int32_t base = (int32_t)to;
            for (size_t k = 1; k < off.size(); ++k) h_sent[++so] = base + off[k];
            std::memcpy(h_tok + to, tk.data(), 4 * tk.size());
            to += (int64_t)tk.size();
        }
    }
    char *base = ctx->pool.base + s.pool_off;
    int32_t *d_sent = reinterpret_cast<int32_t *>(base + L.sent_off);
    int32_t *d_tok = reinterpret_cast<int32_t *>(base + L.tokens);
    CK(cudaEventRecord(s.t0, s.st));
    CK(cudaMemcpyAsync(base + L.plan, hi, L.plan_bytes, cudaMemcpyHostToDevice, s.st));
    CK(cudaMemcpyAsync(d_sent, h_sent, 4 * (n_sent + 1), cudaMemcpyHostToDevice, s.st));
    if (n_tok > 0) CK(cudaMemcpyAsync(d_tok, h_tok, 4 * n_tok, cudaMemcpyHostToDevice, s.st));
    BatchDev b = make_batchdev(s.plan, L, base, d_sent, d_tok, nullptr, ctx->recip, s.gscratch);
    if ((rc = enqueue_kernels(ctx, b, dict, n_sent, n_tok, true, s.st, true, &s.fork))) return rc;
    char *ho = static_cast<char *>(s.pin_out.p);
    CK(cudaMemcpyAsync(ho + s.out_nw, b.nw_score, 4 * s.plan.R, cudaMemcpyDeviceToHost, s.st));
    CK(cudaMemcpyAsync(ho + s.out_nsel, b.n_sel, 4 * s.plan.R, cudaMemcpyDeviceToHost, s.st));
    CK(cudaMemcpyAsync(ho + s.out_err, b.err, 4, cudaMemcpyDeviceToHost, s.st));
    if (s.plan.sel_cap > 0)
        CK(cudaMemcpyAsync(ho + s.out_sel, b.sel, 12 * s.plan.sel_cap, cudaMemcpyDeviceToHost, s.st));
    CK(cudaEventRecord(s.t1, s.st));
    CK(cudaEventRecord(s.ev, s.st));
    s.busy = true;
    return 0;
}

}  // namespace

static void serving_loop(mine_ctx *ctx)
{
    cudaSetDevice(ctx->device);
    const auto window = std::chrono::microseconds(ctx->cfg.batch_window_us);
    for (;;) {
        // harvest finished batches
        int nbusy = 0;
        Slot *oldest = nullptr;
        for (auto &sp : ctx->slots) {
            Slot &s = *sp;
            if (s.busy && cudaEventQuery(s.ev) != cudaErrorNotReady) finish_slot(ctx, s);
            if (s.busy) {
                ++nbusy;
                if (!oldest) oldest = &s;
            }
        }
        Slot *free_slot = nullptr;
        for (auto &sp : ctx->slots)
            if (!sp->busy) {
                free_slot = sp.get();
                break;
            }
        std::unique_lock<std::mutex> lk(ctx->q_mu);
        if (ctx->pending.empty()) {
            if (ctx->stop && nbusy == 0) return;
            if (nbusy > 0) {   // poll the running batches, wake early on new work
                ctx->q_cv.wait_for(lk, std::chrono::microseconds(20),
                                   [&] { return ctx->stop || !ctx->pending.empty(); });
                continue;
            }
            ctx->q_cv.wait(lk, [&] { return ctx->stop || !ctx->pending.empty(); });
            continue;
        }
        if (!free_slot) {
            lk.unlock();
            cudaEventSynchronize(oldest->ev);
            continue;
        }
        // let a small batch grow while the device is busy
        if (nbusy > 0 && (int)ctx->pending.size() < ctx->cfg.max_batch_pairs && !ctx->stop) {
            const auto age = std::chrono::steady_clock::now() - ctx->pending.front().t_submit;
            if (age < window) {
                ctx->q_cv.wait_for(lk, window - age, [&] {
                    return ctx->stop || (int)ctx->pending.size() >= ctx->cfg.max_batch_pairs;
                });
                continue;
            }
        }
        // form the batch: same dictionary, fits the free budget
        Slot &s = *free_slot;
        int64_t bytes = 0;
        const mine_dict *dict = ctx->pending.front().dict;
        std::vector<Request> take;
        while (!ctx->pending.empty() && (int)take.size() < ctx->cfg.max_batch_pairs &&
               ctx->pending.front().dict == dict) {
            const int64_t f = ctx->pending.front().footprint;
            if (bytes + f > ctx->pool.size - ctx->pool.used) break;
            bytes += f;
            take.push_back(std::move(ctx->pending.front()));
            ctx->pending.pop_front();
        }
        if (take.empty()) {   // budget held by running batches
            lk.unlock();
            if (oldest) cudaEventSynchronize(oldest->ev);
            continue;
        }
        // the exact layout of the merged batch is a little smaller than the sum
        const int64_t off = ctx->pool.alloc(bytes + (int64_t)take.size() * 4096);
        if (off < 0) {
            for (auto it = take.rbegin(); it != take.rend(); ++it) ctx->pending.push_front(std::move(*it));
            lk.unlock();
            if (oldest) cudaEventSynchronize(oldest->ev);
            else std::this_thread::sleep_for(std::chrono::microseconds(50));
            continue;
        }
        lk.unlock();
        s.reqs = std::move(take);
        s.pool_off = off;
        s.pool_bytes = bytes + (int64_t)s.reqs.size() * 4096;
        int rc = launch_slot(ctx, s);
        if (rc) {
            // report the failure on every request of the batch
            std::lock_guard<std::mutex> q(ctx->q_mu);
            for (auto &rq : s.reqs) {
                for (size_t k = 0; k < rq.settings.size(); ++k) {
                    mine_result r{};
                    r.ticket = rq.ticket;
                    r.setting = (int32_t)k;
                    r.status = rc;
                    ctx->ready.push_back(r);
                }
                const_cast<mine_dict *>(rq.dict)->inflight--;
                ctx->in_flight_reqs--;
            }
            ctx->pool.release(s.pool_off, s.pool_bytes);
            s.reqs.clear();
            s.busy = false;
            ctx->r_cv.notify_all();
        }
    }
}
