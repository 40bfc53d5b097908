// Host-only checks of the runtime's host logic (no GPU needed): the runtime
// translation unit is compiled into this program.
//  - The batch plan: plans for seeded synthetic batches, and their invariants
//    -- every buffer region of every pair and alignment in place and
//    disjoint, every (pair, gap) aligned once, the settings lists and their
//    by-gap index, the tiles of the tiled alignments, the preparation order
//    and the byte layout of the device region.
//  - The alignment forms: every pair shape under every strategy-table entry
//    gets a form the kernels can run.
//  - The plan's input checks: malformed batches and settings refused with
//    their ABI codes, the int32 overflow bound exactly at its edge.
//  - The strategy table's file: save / load round trips through a context
//    built on the host, and malformed documents refused.
//  - The serving budget's first-fit pool: seeded alloc / release sequences
//    against a plain model of the region (256-byte units), checking each
//    offset (the first fit), the used count and that free blocks are merged.
// Exit status 0 and "ok" when every check holds; otherwise the first failed
// check is printed and the status is 1.
#include "runtime.cu"

#include <cstdio>
#include <set>
#include <tuple>

namespace {

int g_fail = 0;

#define EXPECT(cond, ...)                                                                     \
    do {                                                                                      \
        if (!(cond)) {                                                                        \
            if (!g_fail) {                                                                    \
                std::printf("check failed (%s:%d): %s: ", __FILE__, __LINE__, #cond);        \
                std::printf(__VA_ARGS__);                                                     \
                std::printf("\n");                                                            \
            }                                                                                 \
            g_fail = 1;                                                                       \
            return;                                                                           \
        }                                                                                     \
    } while (0)

uint64_t g_lcg = 0x9E3779B97F4A7C15ull;
int rnd(int n)   // in [0, n)
{
    g_lcg = g_lcg * 6364136223846793005ull + 1442695040888963407ull;
    return (int)((g_lcg >> 33) % (uint64_t)n);
}

// [start, start + len) intervals: disjoint, and together exactly [0, total)
void check_tiling(std::vector<std::pair<int64_t, int64_t>> iv, int64_t total, const char *what)
{
    std::sort(iv.begin(), iv.end());
    int64_t at = 0;
    for (const auto &x : iv) {
        if (x.second == 0) continue;
        EXPECT(x.first == at, "%s: region at %lld, expected %lld", what, (long long)x.first, (long long)at);
        at += x.second;
    }
    EXPECT(at == total, "%s: regions end at %lld, total %lld", what, (long long)at, (long long)total);
}

// A batch: pair sizes (S, T) and each pair's settings array; optionally the
// two articles' roles exchanged (the other mining direction) and a
// strategy table of alignment forms per size bin.
struct Case {
    const char *name;
    std::vector<std::pair<int, int>> st;
    std::vector<std::vector<Setting>> lists;   // distinct arrays
    std::vector<int> list_of;                  // per pair: index into lists
    bool swap = false;
    std::vector<int8_t> tab;                   // empty: the built-in rule
};

void check_case(const Case &cs)
{
    const int32_t P = (int32_t)cs.st.size();
    std::vector<int32_t> doc(2 * (size_t)P + 1, 0);
    for (int p = 0; p < P; ++p) {   // (with swap, the target article comes first in doc)
        doc[2 * p + 1] = doc[2 * p] + (cs.swap ? cs.st[p].second : cs.st[p].first);
        doc[2 * p + 2] = doc[2 * p + 1] + (cs.swap ? cs.st[p].first : cs.st[p].second);
    }
    Plan pl;
    const int rc = build_plan(pl, P, doc.data(), (int64_t)doc.back(),
                              [&](int32_t p, const Setting *&s, int &n) {
                                  const auto &l = cs.lists[cs.list_of[p]];
                                  s = l.data();
                                  n = (int)l.size();
                              },
                              65536, true, cs.tab.empty() ? nullptr : cs.tab.data(), cs.swap);
    EXPECT(rc == 0, "%s: build_plan returned %d (%s)", cs.name, rc, g_err.c_str());
    EXPECT((int32_t)pl.pairs.size() == P && (int32_t)pl.pbases.size() == P, "%s: pair tables", cs.name);

    // pairs: sentence ranges, settings rows, score tiles, selection blocks
    std::vector<std::pair<int64_t, int64_t>> m_iv, sel_iv, code_iv, match_iv, tb_iv;
    int32_t rows = 0;
    int64_t n_items_want = 0;
    for (int p = 0; p < P; ++p) {
        const PairPlan &pp = pl.pairs[p];
        const int S = cs.st[p].first, T = cs.st[p].second;
        const int32_t s0 = cs.swap ? doc[2 * p + 1] : doc[2 * p], t0 = cs.swap ? doc[2 * p] : doc[2 * p + 1];
        EXPECT(pp.s0 == s0 && pp.S == S && pp.t0 == t0 && pp.T == T, "%s: pair %d", cs.name, p);
        const auto &l = cs.lists[cs.list_of[p]];
        EXPECT(pp.set0 == rows && pp.nset == (int)l.size(), "%s: settings rows of pair %d", cs.name, p);
        rows += pp.nset;
        // each setting: its gap among the list's distinct gaps, its threshold
        std::vector<int32_t> gaps;
        for (const Setting &s : l)
            if (std::find(gaps.begin(), gaps.end(), s.first) == gaps.end()) gaps.push_back(s.first);
        EXPECT(pp.ngap == (int)gaps.size(), "%s: distinct gaps of pair %d", cs.name, p);
        for (int k = 0; k < pp.nset; ++k) {
            const int lg = pl.set_gap[pp.slist0 + k];
            EXPECT(lg >= 0 && lg < pp.ngap && pl.gap_val[pp.gap0 + lg] == l[k].first &&
                       pl.set_thr[pp.slist0 + k] == l[k].second,
                   "%s: setting %d of pair %d", cs.name, k, p);
        }
        // by gap: set_perm lists the settings grouped by gap, gap_sfirst where each gap starts
        std::vector<int> seen(pp.nset, 0);
        for (int f = 0; f < pp.nset; ++f) {
            const int k = pl.set_perm[pp.slist0 + f];
            EXPECT(k >= 0 && k < pp.nset && !seen[k], "%s: set_perm of pair %d", cs.name, p);
            seen[k] = 1;
            const int g = pl.set_gap[pp.slist0 + k];
            const int first = pl.gap_sfirst[pp.gap0 + g];
            const int last = g + 1 < pp.ngap ? pl.gap_sfirst[pp.gap0 + g + 1] : pp.nset;
            EXPECT(f >= first && f < last, "%s: gap_sfirst of pair %d", cs.name, p);
            if (f > 0) {
                const int k0 = pl.set_perm[pp.slist0 + f - 1];
                EXPECT(pl.set_gap[pp.slist0 + k0] < g || (pl.set_gap[pp.slist0 + k0] == g && k0 < k),
                       "%s: set_perm order of pair %d", cs.name, p);
            }
        }
        n_items_want += pp.ngap;
        const int64_t tiles = (int64_t)((S + 31) / 32) * ((T + 31) / 32) * kTileElems;
        m_iv.push_back({pp.m_off, tiles});
        sel_iv.push_back({pp.sel_base, (int64_t)pp.nset * std::min(S, T)});
        const PairBases &pb = pl.pbases[p];
        code_iv.push_back({pb.codes, (int64_t)pp.ngap * S * ((T + 15) / 16)});
        match_iv.push_back({pb.matches, (int64_t)pp.ngap * std::min(S, T)});
    }
    EXPECT(pl.R == rows, "%s: R", cs.name);
    // pairs given the same array share one settings list
    for (int p = 1; p < P; ++p)
        if (cs.list_of[p] == cs.list_of[p - 1])
            EXPECT(pl.pairs[p].slist0 == pl.pairs[p - 1].slist0 && pl.pairs[p].gap0 == pl.pairs[p - 1].gap0,
                   "%s: pairs %d and %d do not share their list", cs.name, p - 1, p);
    check_tiling(m_iv, pl.m_elems, "score tiles");
    if (g_fail) return;
    check_tiling(sel_iv, pl.sel_cap, "selection blocks");
    if (g_fail) return;
    check_tiling(code_iv, pl.code_words, "direction codes");
    if (g_fail) return;
    check_tiling(match_iv, pl.match_words, "match lists");
    if (g_fail) return;

    // alignments: every (pair, gap) once, runs in order, the tiled ones last
    EXPECT((int64_t)pl.nitems.size() == n_items_want, "%s: %zu items, want %lld", cs.name, pl.nitems.size(),
           (long long)n_items_want);
    int32_t in_runs = 0;
    for (int k = 0; k < kNwGroups; ++k) in_runs += pl.n_grp[k];
    EXPECT(in_runs + pl.n_tiled == (int32_t)pl.nitems.size(), "%s: runs", cs.name);
    std::set<std::pair<int, int>> items;
    std::set<int> tiled_pairs;
    for (size_t x = 0; x < pl.nitems.size(); ++x) {
        const NwItem &it = pl.nitems[x];
        EXPECT(it.pair >= 0 && it.pair < P, "%s: item %zu", cs.name, x);
        const PairPlan &pp = pl.pairs[it.pair];
        EXPECT(it.gap >= pp.gap0 && it.gap < pp.gap0 + pp.ngap, "%s: gap of item %zu", cs.name, x);
        EXPECT(items.insert({it.pair, it.gap}).second, "%s: item %zu repeats", cs.name, x);
        const PairBases &pb = pl.pbases[it.pair];
        const int64_t c = item_codes(pb.codes, pp, it.gap), m = item_matches(pb.matches, pp, it.gap);
        EXPECT(c >= pb.codes && c + (int64_t)pp.S * ((pp.T + 15) / 16) <= pb.codes + (int64_t)pp.ngap * pp.S * ((pp.T + 15) / 16),
               "%s: codes of item %zu", cs.name, x);
        EXPECT(m >= pb.matches && m + std::min(pp.S, pp.T) <= pb.matches + (int64_t)pp.ngap * std::min(pp.S, pp.T),
               "%s: matches of item %zu", cs.name, x);
        if ((int32_t)x >= in_runs && tiled_pairs.insert(it.pair).second)
            tb_iv.push_back({pb.tb, (int64_t)pp.ngap * tb_words_of(pp.S, pp.T)});
    }
    check_tiling(tb_iv, pl.tb_words, "tile boundaries");
    if (g_fail) return;
    // tiles: every tile of every tiled alignment once, in order of R + C
    std::set<std::tuple<int, int, int>> tl;
    for (size_t k = 0; k < pl.tiles.size(); ++k) {
        const TileItem &t = pl.tiles[k];
        EXPECT(t.nw >= in_runs && t.nw < (int32_t)pl.nitems.size(), "%s: tile %zu", cs.name, k);
        const PairPlan &pp = pl.pairs[pl.nitems[t.nw].pair];
        EXPECT(t.R >= 0 && t.R < tile_rows_of(pp.S) && t.C >= 0 && t.C < tile_cols_of(pp.T), "%s: tile %zu", cs.name, k);
        EXPECT(tl.insert({t.nw, t.R, t.C}).second, "%s: tile %zu repeats", cs.name, k);
        if (k > 0) EXPECT(pl.tiles[k - 1].R + pl.tiles[k - 1].C <= t.R + t.C, "%s: tile order", cs.name);
    }
    int64_t tiles_want = 0;
    for (int32_t x = in_runs; x < (int32_t)pl.nitems.size(); ++x) {
        const PairPlan &pp = pl.pairs[pl.nitems[x].pair];
        tiles_want += tile_rows_of(pp.S) * tile_cols_of(pp.T);
    }
    EXPECT((int64_t)tl.size() == tiles_want, "%s: %zu tiles, want %lld", cs.name, tl.size(), (long long)tiles_want);

    // the preparation order: every pair once, the wide targets first
    std::vector<int> once(P, 0);
    for (int k = 0; k < P; ++k) {
        const int p = pl.dorder[k];
        EXPECT(p >= 0 && p < P && !once[p], "%s: dorder", cs.name);
        once[p] = 1;
        EXPECT((k < pl.n_dwide) == (pl.pairs[p].T > kWideArticleSent), "%s: dorder wide part", cs.name);
    }
    // preparation items (32 rows) and score items (64 rows, at most kScoreColChunk columns)
    int64_t prow = 0, scells = 0, cells = 0;
    for (const ScoreItem &it : pl.pitems) prow += std::min(32, pl.pairs[it.pair].S - it.row0);
    for (const ScoreItem &it : pl.sitems) {
        const PairPlan &pp = pl.pairs[it.pair];
        EXPECT(it.c0 < std::max(pp.T, 1) && it.c1 - it.c0 <= kScoreColChunk && it.c1 <= pp.T, "%s: score item", cs.name);
        scells += (int64_t)std::min(64, pp.S - it.row0) * (it.c1 - it.c0);
    }
    int64_t src_rows = 0;
    for (int p = 0; p < P; ++p) {
        cells += (int64_t)cs.st[p].first * cs.st[p].second;
        src_rows += cs.st[p].first;
    }
    EXPECT(prow == src_rows, "%s: preparation items cover %lld source rows of %lld", cs.name, (long long)prow,
           (long long)src_rows);
    EXPECT(scells == cells, "%s: score items cover %lld cells of %lld", cs.name, (long long)scells, (long long)cells);

    // the device region: aligned, disjoint, in the order laid out
    pl.n_sent = doc.back();
    pl.n_tok = 5 * pl.n_sent;
    const Layout L = make_layout(pl, 4, true, true, true);
    const int64_t reg[] = {L.plan, L.sent_off, L.tokens, L.elems, L.sinfo, L.order, L.tdoc, L.pdoc, L.witems,
                           L.xwl, L.kitems, L.M, L.codes, L.matches, L.hfin, L.tbnd, L.counters, L.nw, L.nsel,
                           L.sel, L.total};
    for (size_t k = 0; k + 1 < sizeof(reg) / sizeof(reg[0]); ++k)
        EXPECT(reg[k] % 256 == 0 && reg[k] < reg[k + 1], "%s: device region %zu", cs.name, k);
    EXPECT(L.codes + 4 * pl.code_words <= L.matches && L.matches + 4 * pl.match_words <= L.hfin &&
               L.M + 4 * pl.m_elems <= L.codes && L.tbnd + 4 * pl.tb_words <= L.counters,
           "%s: region sizes", cs.name);
    const int64_t sub[] = {L.o_pairs, L.o_pbases, L.o_sitems, L.o_nitems, L.o_setgap, L.o_setthr, L.o_gapval,
                           L.o_setperm, L.o_gapsfirst, L.o_dorder, L.o_pitems, L.o_tiles, L.plan_bytes};
    for (size_t k = 0; k + 1 < sizeof(sub) / sizeof(sub[0]); ++k)
        EXPECT(sub[k] % 16 == 0 && sub[k] <= sub[k + 1], "%s: plan blob part %zu", cs.name, k);
    EXPECT(L.o_pbases - L.o_pairs >= (int64_t)(sizeof(PairPlan) * P) &&
               L.o_nitems - L.o_sitems >= (int64_t)(sizeof(ScoreItem) * pl.sitems.size()) &&
               L.plan_bytes - L.o_tiles >= (int64_t)(sizeof(TileItem) * pl.tiles.size()),
           "%s: plan blob sizes", cs.name);
}

// The plan's input checks: each malformed batch or settings list is refused
// with its ABI code, and the overflow bound (S+T)|g| + min(S,T) max|s| < 2^31
// holds exactly at its edge.
int plan_rc(std::vector<int32_t> doc, int64_t n_sent, std::vector<Setting> set, bool mined = true)
{
    Plan pl;
    const int32_t P = doc.size() > 1 ? (int32_t)(doc.size() - 1) / 2 : 0;
    return build_plan(pl, P, doc.data(), n_sent,
                      [&](int32_t, const Setting *&s, int &n) {
                          s = set.data();
                          n = (int)set.size();
                      },
                      65536, mined, nullptr);
}

void check_errors()
{
    const std::vector<Setting> one{Setting(-65536, 32768)};
    EXPECT(plan_rc({0, 3, 7}, 7, one) == MINE_OK, "a valid batch");
    EXPECT(plan_rc({0}, 0, one) == MINE_OK, "no pairs");
    EXPECT(plan_rc({1, 3, 7}, 7, one) == MINE_EINVAL, "doc_off[0] != 0");
    EXPECT(plan_rc({0, 3, 2}, 2, one) == MINE_EINVAL, "decreasing doc_off");
    EXPECT(plan_rc({0, 3, 7}, 8, one) == MINE_EINVAL, "doc_off[2P] != n_sent");
    // (a gap of -1/65536: the overflow bound allows these sizes)
    const std::vector<Setting> tiny{Setting(-1, 32768)};
    EXPECT(plan_rc({0, MINE_MAX_SENTENCES, MINE_MAX_SENTENCES + 1}, MINE_MAX_SENTENCES + 1, tiny) == MINE_OK,
           "the largest article");
    EXPECT(plan_rc({0, MINE_MAX_SENTENCES + 1, MINE_MAX_SENTENCES + 2}, MINE_MAX_SENTENCES + 2, tiny) ==
               MINE_EINVAL,
           "an article above the largest");
    EXPECT(plan_rc({0, MINE_MAX_SENTENCES, MINE_MAX_SENTENCES + 1}, MINE_MAX_SENTENCES + 1, one) == MINE_EOVERFLOW,
           "the largest article at gap -1: (S+T)|g| reaches 2^32");
    EXPECT(plan_rc({0, 3, 7}, 7, {}) == MINE_EINVAL, "no settings");
    EXPECT(plan_rc({0, 3, 7}, 7, std::vector<Setting>(256, Setting(-1, 0))) == MINE_OK, "256 settings");
    EXPECT(plan_rc({0, 3, 7}, 7, std::vector<Setting>(257, Setting(-1, 0))) == MINE_EINVAL, "257 settings");
    EXPECT(plan_rc({0, 3, 7}, 7, {Setting(1, 0)}) == MINE_EINVAL, "a positive gap");
    EXPECT(plan_rc({0, 3, 7}, 7, {Setting(0, 0), Setting(0, 65536)}) == MINE_OK, "gap 0, thresholds 0 and 1");
    EXPECT(plan_rc({0, 3, 7}, 7, {Setting(-1, -1)}) == MINE_EINVAL, "a negative threshold");
    EXPECT(plan_rc({0, 3, 7}, 7, {Setting(-1, 65537)}) == MINE_EINVAL, "a threshold above 1");
    EXPECT(plan_rc({0, 3, 7}, 7, {Setting(-1, 65537)}, false) == MINE_OK, "thresholds unused: not checked");
    // S = 1, T = 2: the bound is 3 |g| + 65536
    EXPECT(plan_rc({0, 1, 3}, 3, {Setting(-715806037, 0)}) == MINE_OK, "bound 2^31 - 1");
    EXPECT(plan_rc({0, 1, 3}, 3, {Setting(-715806038, 0)}) == MINE_EOVERFLOW, "bound 2^31 + 2");
    // the largest |gap| decides for every setting of the list
    EXPECT(plan_rc({0, 1, 3}, 3, {Setting(-1, 0), Setting(-715806038, 0)}) == MINE_EOVERFLOW, "a list's largest gap");
}

// The alignment form of every pair shape under every table entry is one the
// kernels can run: tiles only where there are several tile rows and columns;
// one warp only where its own ring holds a row (T < kRing, or one stripe);
// a pipeline only where its first warp can get a whole row ahead of its last
// (every warp one stripe at most, or the row within the rings of the links:
// about 12 tiles of 32 columns per link).
void check_forms()
{
    std::vector<int> sides;
    for (int v : {0, 1, 2, 31, 32, 33, 63, 64, 65, 95, 96, 97, 128, 200, 255, 256, 257, 300, 384, 511, 512, 513,
                  600, 800, 1000, 1023, 1024, 1025, 2000, 2048, 4000, 8192})
        sides.push_back(v);
    std::vector<int8_t> tab(kAlignBins, (int8_t)-1);
    for (int entry = -1; entry < AF_FORMS; ++entry) {
        for (int b = 0; b < kAlignBins; ++b) tab[b] = (int8_t)entry;
        for (int S : sides)
            for (int T : sides) {
                const int f = align_kind(entry < 0 ? nullptr : tab.data(), S, T);
                EXPECT(f == AF_WARP1 || f == AF_WARP2 || f == AF_WARP4 || f == AF_WARP8 || f == AF_TILED,
                       "form %d for %d x %d", f, S, T);
                if (f == AF_TILED) {
                    EXPECT(S > kAlignTileRows && T > kAlignTileCols, "tiles for %d x %d", S, T);
                    continue;
                }
                const int g = form_warps(f), ns = (S + 31) / 32, tt = (T + 31) / 32;
                const int ge = std::max(1, std::min(std::min(g, ns), std::max(1, tt - 1)));
                if (ge == 1)
                    EXPECT(ns <= 1 || T < kRing, "one warp for %d x %d (table entry %d)", S, T, entry);
                else
                    EXPECT(ns <= ge || tt <= 12 * (ge - 1), "%d warps for %d x %d (table entry %d)", ge, S, T, entry);
            }
    }
}

// The strategy table's file: written and read back through a context (one
// built on the host: no device is touched), every table a round trip; the
// documents of any other form refused with the table unchanged.
void check_strategy_file(const char *dir)
{
    const std::string path = std::string(dir) + "/strategy.json";
    mine_ctx ctx;
    for (int rep = 0; rep < 50; ++rep) {
        int8_t tab[kAlignBins], back[kAlignBins];
        for (int b = 0; b < kAlignBins; ++b) tab[b] = (int8_t)(rnd(AF_FORMS + 1) - 1);
        EXPECT(mine_align_strategy(&ctx, tab, kAlignBins, 0) == MINE_OK, "set");
        EXPECT(mine_align_strategy_save(&ctx, path.c_str()) == MINE_OK, "save: %s", mine_last_error());
        int8_t other[kAlignBins];
        std::fill(other, other + kAlignBins, (int8_t)-1);
        EXPECT(mine_align_strategy(&ctx, other, kAlignBins, 0) == MINE_OK, "reset");
        EXPECT(mine_align_strategy_load(&ctx, path.c_str()) == MINE_OK, "load: %s", mine_last_error());
        EXPECT(mine_align_strategy(&ctx, back, kAlignBins, 1) == MINE_OK, "get");
        EXPECT(std::equal(tab, tab + kAlignBins, back), "round trip %d", rep);
    }
    int8_t before[kAlignBins], after[kAlignBins];
    EXPECT(mine_align_strategy(&ctx, before, kAlignBins, 1) == MINE_OK, "get");
    std::string good = strategy_json(before);
    std::string spaced = good;   // white space anywhere between tokens
    for (size_t k = 0; k < spaced.size(); ++k)
        if (spaced[k] == ',' || spaced[k] == ':' || spaced[k] == '[') spaced.insert(++k, "\n\t ");
    std::string list = "";
    for (int b = 0; b < kAlignBins; ++b) list += (b ? ", " : "") + std::to_string((int)before[b]);
    const std::string head = "{\"format\": \"mine-align-strategy\", \"bins\": [";
    const char *bad[] = {"", "{}", "not json", "{\"format\": \"other\", \"bins\": []}"};
    std::vector<std::string> docs(bad, bad + 4);
    docs.push_back(head + list + ", 0]}");                          // 41 entries
    docs.push_back(head + list.substr(0, list.rfind(',')) + "]}");  // 39 entries
    docs.push_back(head + "5" + list.substr(list.find(',')) + "]}");   // a value above the forms
    docs.push_back(head + "-2" + list.substr(list.find(',')) + "]}");  // below -1
    docs.push_back(head + list + ",]}");                            // a trailing comma
    docs.push_back(head + list + "]} x");                           // text after the document
    docs.push_back(good.substr(0, good.size() / 2));                // cut short
    for (size_t k = 0; k <= docs.size(); ++k) {
        const std::string &d = k < docs.size() ? docs[k] : spaced;
        FILE *f = std::fopen(path.c_str(), "wb");
        EXPECT(f && std::fwrite(d.data(), 1, d.size(), f) == d.size() && std::fclose(f) == 0, "write");
        const int rc = mine_align_strategy_load(&ctx, path.c_str());
        EXPECT(rc == (k < docs.size() ? MINE_EINVAL : MINE_OK), "document %zu: rc %d", k, rc);
        EXPECT(mine_align_strategy(&ctx, after, kAlignBins, 1) == MINE_OK, "get");
        EXPECT(std::equal(before, before + kAlignBins, after), "document %zu changed the table", k);
    }
    EXPECT(mine_align_strategy_load(&ctx, (path + ".missing").c_str()) == MINE_EINVAL, "a missing file");
    EXPECT(mine_align_strategy_save(&ctx, (std::string(dir) + "/no/such/dir/s.json").c_str()) == MINE_EINVAL,
           "an unwritable path");
    std::remove(path.c_str());
}

// The first-fit pool against a model: a byte per 256-byte unit (1 = taken).
void check_pool(int64_t units, int steps)
{
    Pool pool;
    pool.size = units * 256;
    pool.free_[0] = pool.size;
    std::vector<char> model(units, 0);
    std::vector<std::pair<int64_t, int64_t>> live;   // (offset, bytes asked)
    int64_t used = 0;
    for (int it = 0; it < steps; ++it) {
        if (live.empty() || rnd(3) != 0) {
            // ask for 1 .. units/4 units' worth, not always a multiple of 256
            const int64_t bytes = 1 + rnd((int)(units * 64));
            const int64_t need = (bytes + 255) / 256;
            int64_t want = -1;   // the model's first fit
            for (int64_t u = 0, run = 0; u < units; ++u) {
                run = model[u] ? 0 : run + 1;
                if (run == need) {
                    want = (u + 1 - need) * 256;
                    break;
                }
            }
            const int64_t off = pool.alloc(bytes);
            EXPECT(off == want, "pool step %d: %lld bytes at %lld, the first fit is %lld", it, (long long)bytes,
                   (long long)off, (long long)want);
            if (off >= 0) {
                for (int64_t u = off / 256; u < off / 256 + need; ++u) model[u] = 1;
                live.push_back({off, bytes});
                used += need * 256;
            }
        } else {
            const int k = rnd((int)live.size());
            const auto x = live[k];
            live.erase(live.begin() + k);
            pool.release(x.first, x.second);
            for (int64_t u = x.first / 256; u < x.first / 256 + (x.second + 255) / 256; ++u) model[u] = 0;
            used -= (x.second + 255) / 256 * 256;
        }
        EXPECT(pool.used == used, "pool step %d: used %lld, want %lld", it, (long long)pool.used, (long long)used);
        // the free list is the model's free runs, each merged with its neighbours
        int64_t at = -1;
        for (const auto &f : pool.free_) {
            EXPECT(f.first > at && f.second > 0 && f.first + f.second <= pool.size, "pool step %d: free block", it);
            EXPECT(f.first == 0 || model[f.first / 256 - 1], "pool step %d: free block at %lld not merged", it,
                   (long long)f.first);
            for (int64_t u = f.first / 256; u < (f.first + f.second) / 256; ++u)
                EXPECT(!model[u], "pool step %d: free block over a taken unit", it);
            EXPECT(f.first + f.second == pool.size || model[(f.first + f.second) / 256], "pool step %d: free run cut",
                   it);
            at = f.first + f.second;
        }
        int64_t free_units = 0;
        for (char m : model) free_units += !m;
        int64_t listed = 0;
        for (const auto &f : pool.free_) listed += f.second / 256;
        EXPECT(listed == free_units, "pool step %d: %lld free units listed, %lld free", it, (long long)listed,
               (long long)free_units);
    }
    for (const auto &x : live) pool.release(x.first, x.second);
    EXPECT(pool.used == 0 && pool.free_.size() == 1 && pool.free_.begin()->first == 0 &&
               pool.free_.begin()->second == pool.size,
           "pool: not one free block after every release");
}

}  // namespace

int main(int argc, char **argv)
{
    check_strategy_file(argc > 1 ? argv[1] : ".");
    if (g_fail) return 1;
    check_errors();
    if (g_fail) return 1;
    check_forms();
    if (g_fail) return 1;
    check_pool(64, 4000);
    check_pool(1000, 4000);
    if (g_fail) return 1;
    std::vector<Case> cases;
    // edge sizes, one shared list of one setting
    {
        Case c{"edges", {}, {{Setting(-65536, 32768)}}, {}};
        const int sz[] = {0, 1, 2, 31, 32, 33, 63, 64, 65, 127, 128, 161, 255, 300};
        for (int s : sz)
            for (int t : sz) c.st.push_back({s, t});
        c.list_of.assign(c.st.size(), 0);
        cases.push_back(c);
    }
    // lognormal-like sizes with a few long and tiled pairs, a 64-setting sweep list
    {
        Case c{"sweep", {}, {{}}, {}};
        for (int g = 1; g <= 8; ++g)
            for (int t = 0; t < 8; ++t) c.lists[0].push_back(Setting(-16384 * g, 19661 + 4681 * t));
        for (int p = 0; p < 600; ++p) {
            const int s = 1 + rnd(rnd(4) == 0 ? 800 : 90), t = 1 + rnd(rnd(4) == 0 ? 800 : 90);
            c.st.push_back({s, t});
        }
        c.st.push_back({1500, 1500});
        c.st.push_back({300, 8000});
        c.st.push_back({2100, 600});
        c.list_of.assign(c.st.size(), 0);
        cases.push_back(c);
    }
    // per-pair lists: runs sharing an array, equal contents in another array,
    // repeated gaps out of order
    {
        Case c{"lists", {}, {}, {}};
        c.lists.push_back({Setting(-65536, 32768)});
        c.lists.push_back({Setting(-65536, 32768)});
        c.lists.push_back({Setting(-32768, 10000), Setting(-65536, 20000), Setting(-32768, 30000),
                           Setting(-131072, 0), Setting(-65536, 65536)});
        c.lists.push_back({Setting(0, 5), Setting(0, 6)});
        for (int p = 0; p < 200; ++p) {
            c.st.push_back({rnd(200), rnd(200)});
            c.list_of.push_back(p < 40 ? 0 : p < 80 ? 1 : (p / 7) % 4);
        }
        cases.push_back(c);
    }
    // the other direction (each pair's articles exchanged), and a strategy
    // table that sends some size bins to other forms
    {
        Case c = cases[1];
        c.name = "sweep-swapped";
        c.swap = true;
        cases.push_back(c);
        Case d = cases[1];
        d.name = "sweep-table";
        d.tab.assign(kAlignBins, (int8_t)-1);
        d.tab[7] = AF_WARP1;
        d.tab[12] = AF_WARP2;
        d.tab[16] = AF_WARP8;
        d.tab[18] = AF_WARP4;
        d.tab[20] = AF_TILED;
        cases.push_back(d);
    }
    for (const Case &c : cases) {
        check_case(c);
        if (g_fail) return 1;
    }
    std::printf("ok\n");
    return 0;
}
