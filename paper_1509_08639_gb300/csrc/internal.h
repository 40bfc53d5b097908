// internal.h -- device data layout shared by the kernels and the host runtime
// of the miner (not part of the public ABI; see include/mine.h).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "mine.h"

namespace mine {

// Direction codes of the alignment (2 bits per cell, 16 cells per uint32;
// code 2 is unused).
enum : uint32_t { DIR_DIAG = 0, DIR_UP = 1, DIR_LEFT = 3 };

// Source-element flag bits (token IDs are < 2^30, so the two top bits are free).
constexpr uint32_t ELEM_FIRST = 1u << 31;   // first occurrence of this translation in U_i
constexpr uint32_t ELEM_END = 1u << 30;     // last translation of one source token
constexpr uint32_t ELEM_TOKEN = (1u << 30) - 1;

// device error word values (0 = fine)
constexpr int32_t ERR_DUP_KEY = 1;
constexpr int32_t ERR_BAD_OFFSETS = 2;
constexpr int32_t ERR_BAD_TOKEN = 3;
constexpr int32_t ERR_TIMEOUT = 4;          // a bounded device wait ran out

constexpr int kWarp = 32;
constexpr int kNwGroups = 4;                // alignment pipelines of 8, 4, 2 and 1 warps
constexpr int kTile = 32;                   // score matrices are stored as 32 x 32 tiles
constexpr int kTileElems = kTile * kTile;
constexpr int kColHashSlots = 1024;         // per-warp target-token table of a column block
constexpr int kColTokCap = kColHashSlots / 2;   // tokens per column block at most
constexpr int kMaxSentTokens = MINE_MAX_SENT_TOKENS;
constexpr uint32_t kWaitLimit = 1u << 22;   // bounded spins on shared-memory flags
constexpr uint32_t kWaitHintNs = 100000;     // mbarrier try_wait suspend-time hint (100 us)
constexpr uint32_t kMbarTries = 20000;       // try_wait attempts before giving up (<= ~2 s)
constexpr uint32_t kTestWaitSpins = 20000;   // flag-wait tries of a test with withheld rows (a few ms)
constexpr int kScoreWarps = 4;              // warps per CTA of the score kernel
constexpr int kScoreCtasPerSm = 4;          // CTAs per SM of the preparation kernel (grid = SMs x this)
constexpr int kScoreWarpsScore = 2;         // warps per CTA of the score kernel (64 rows per item)
constexpr int kScoreCtasPerSmScore = 6;     // its resident CTAs per SM
constexpr int kBlkTokCap = 1024;            // tokens of one staged 32-column block at most
constexpr int kPairPrepCtasPerSm = 2;       // CTAs (16 warps each) per SM of the pair preparation
// per-warp global tables: enough for the largest grid of the three kernels using them
constexpr int kGScratchWarpsPerSm = 72;
// Target articles of more than this many sentences are prepared by the
// wide-article launch (bigger tables, fewer CTAs per SM)
constexpr int kWideArticleSent = 160;
// floor(x * 65536 / m) == umulhi(x << 17, ceil(2^31 / m)) for 0 <= x <= m <= this
constexpr int kRecip31Max = 181;
static_assert(kScoreWarpsScore * kScoreCtasPerSmScore <= kGScratchWarpsPerSm &&
                  kScoreWarps * kScoreCtasPerSm <= kGScratchWarpsPerSm &&
                  16 * kPairPrepCtasPerSm <= kGScratchWarpsPerSm,
              "per-warp global tables");
// Target articles with at most kDirect distinct tokens are scored through
// dense document ids (a direct-indexed column mask per id); entry kZeroEnt of
// that mask array is never set.
constexpr int kDirect = 8192;
constexpr uint32_t kZeroEnt = kDirect;
// Articles with more distinct tokens, up to kDirectX, are prepared again by a
// third launch with a larger table and scored through a larger mask array.
constexpr int kDirectX = 16384;
// per-warp global table of the score kernel: 2 * kMaxSentTokens (key, mask) entries
constexpr int64_t kScoreScratchPerWarp = 2 * (int64_t)kMaxSentTokens * 8;

// Resident dictionary: table of (key, off << 6 | cnt) slots in buckets of 8,
// bucket = key * 0x9E3779B1 >> (35 - log2), overflow into the next bucket.
// Empty key = -1.
struct DevDict {
    int2 *slots;        // [1 << log2]
    int32_t *trans;     // translations
    int32_t log2;
    int32_t kmax;       // largest translation count of any key
    int64_t n_trans;
    // The same keys with their first kInlineTrans translations inline:
    // 64-byte buckets of two 32-byte entries (key, off << 6 | cnt, t0..t5),
    // bucket = key * 0x9E3779B1 >> (32 - inl_log2), overflow into the next
    // bucket; empty key = -1.  One bucket read gives a key's translations.
    int4 *inl;          // [4 << inl_log2]
    int32_t inl_log2;
};
constexpr int kInlineTrans = 6;

struct PairPlan {       // 56 bytes
    int32_t s0, S;      // source sentences [s0, s0+S) (global sentence index)
    int32_t t0, T;      // target sentences [t0, t0+T)
    int32_t set0, nset; // settings rows [set0, set0+nset) (the outputs)
    int32_t gap0, ngap; // distinct gaps [gap0, gap0+ngap) of this pair (shared by the pairs
                        // with the same settings list)
    int32_t slist0;     // its settings: set_gap / set_thr [slist0, slist0+nset) (shared too)
    int32_t pad_;
    int64_t m_off;      // int32 offset of M: ceil(S/32) x ceil(T/32) tiles of 32 x 32
    int64_t sel_base;   // mine_pair offset of the selection block (nset * min(S,T))
};

// Where a pair's alignment buffers start (read by the alignment kernels only)
struct PairBases {
    int64_t codes;      // uint32 offset of the direction codes of its first gap (then one
                        // block of S rows x ceil(T/16) words per gap, in gap order)
    int64_t matches;    // uint32 offset of its match lists (min(S,T) entries per gap)
    int64_t tb;         // tiled alignments: int32 offset of the tile boundaries and flags
                        // of its first gap (tb_words_of(S, T) per gap)
};

// Offset of cell (r, c) (0-based) of a tiled score matrix with TT column tiles.
__host__ __device__ __forceinline__ int64_t m_cell(int64_t m_off, int TT, int r, int c)
{
    return m_off + ((int64_t)(r >> 5) * TT + (c >> 5)) * kTileElems + (r & 31) * kTile + (c & 31);
}

struct NwItem {         // one alignment: (pair, gap); its buffers follow from the pair's PairBases
    int32_t pair;
    int32_t gap;        // global gap index
};

// A tiled alignment is cut into tiles of kAlignTileRows x kAlignTileCols
// cells computed by different CTAs: tile (R, C) starts once (R-1, C) and
// (R, C-1) are done.  Between tiles: the last row of every tile row, the
// last column of every tile column (global memory), a done flag per tile.
constexpr int kAlignTileRows = 256;        // 8 stripes of 32 rows: one CTA of 8 warps
constexpr int kAlignTileCols = 512;        // = the shared ring of one stripe
constexpr int64_t kTiledCells = int64_t(1) << 21;
struct TileItem {
    int32_t nw;         // alignment item
    int16_t R, C;       // tile row and column
};
// boundary area of an S x T tiled alignment: rows (NR-1) x (T+1), columns
// (NC-1) x (S+1), flags NR x NC (int32 each)
__host__ __device__ inline int64_t tile_rows_of(int32_t S) { return (S + kAlignTileRows - 1) / kAlignTileRows; }
__host__ __device__ inline int64_t tile_cols_of(int32_t T) { return (T + kAlignTileCols - 1) / kAlignTileCols; }
// int32 words of one tiled alignment's boundaries and flags: the last row of
// every tile row but the last ((NR-1) x (T+1)), the last column of every tile
// column but the last ((NC-1) x (S+1)), a done flag per tile; a multiple of 4
__host__ __device__ inline int64_t tb_words_of(int32_t S, int32_t T)
{
    const int64_t NR = tile_rows_of(S), NC = tile_cols_of(T);
    return ((NR - 1) * (T + 1) + (NC - 1) * (S + 1) + NR * NC + 3) & ~int64_t(3);
}
// Offsets of the buffers of alignment (pair pp, global gap index gap), from
// the pair's base of that buffer
__host__ __device__ inline int64_t item_codes(int64_t base, const PairPlan &pp, int32_t gap)
{
    return base + (int64_t)(gap - pp.gap0) * pp.S * ((pp.T + 15) >> 4);
}
__host__ __device__ inline int64_t item_matches(int64_t base, const PairPlan &pp, int32_t gap)
{
    return base + (int64_t)(gap - pp.gap0) * (pp.S < pp.T ? pp.S : pp.T);
}
__host__ __device__ inline int64_t item_tb(int64_t base, const PairPlan &pp, int32_t gap)
{
    return base + (int64_t)(gap - pp.gap0) * tb_words_of(pp.S, pp.T);
}

struct ScoreItem {      // 32 (preparation) or 64 (scoring) source rows of one pair
    int32_t pair;
    int32_t row0;
    int32_t c0, c1;     // scoring: target columns [c0, c1)
};

// A score item covers at most this many target columns (long articles are cut
// so that no item is much longer than the others).
constexpr int kScoreColChunk = 256;

struct BatchDev {
    // inputs
    const int32_t *sent_off;     // [n_sent+1]
    const int32_t *tokens;       // [n_tok]
    int64_t n_tok;
    int32_t n_pairs;
    // plan
    const PairPlan *pairs;
    const PairBases *pbases;         // [n_pairs] where each pair's alignment buffers start
    const ScoreItem *prep_items;     // 32 rows each
    int32_t n_prep_items;
    const ScoreItem *score_items;    // 64 rows each
    int32_t n_score_items;
    ScoreItem *wide_items;           // the items of the score launches for larger articles
                                     // (built on the device; their count in counters[18])
    const NwItem *nw_items;
    int32_t n_nw_items;
    int32_t n_nw_grp[kNwGroups]; // items aligned by pipelines of 8, 4, 2 warps and by one warp, in that order from 0
    int32_t n_nw_tiled;          // the last n_nw_tiled items are aligned tile by tile
    const TileItem *tiles;       // tiles of the tiled items, in order of R + C
    int32_t n_tiles;
    int32_t *tbnd;               // tile boundaries and flags (zeroed per batch)
    int64_t n_tbnd;              // their int32 count
    const int32_t *set_gap;      // settings lists (PairPlan::slist0): each setting's gap as an
    const int32_t *set_thr;      // index among its pair's distinct gaps, and its threshold
    const int32_t *gap_val;      // [G]
    const int32_t *set_perm;     // per settings list, its settings ordered by gap (stable)
    const int32_t *gap_sfirst;   // [G] where a gap's settings start in set_perm (list-relative)
    // scratch
    uint32_t *elems;             // source elements (see elem_base)
    int4 *sinfo;                 // [n_sent] (n_i, #elements, |U_i|, 0) of source sentences
    int32_t *row_order;          // [n_sent] per pair, source rows by element count (longest first)
    uint16_t *tdoc;              // [n_tok + 32] document id of each target token
    int32_t *pdoc;               // [n_pairs] distinct target tokens D, or -1 (token-keyed path)
    int32_t *xw_list;            // [n_pairs] pairs left to the extra-wide preparation (counters[21])
    ScoreItem *keyed_items;      // [n_prep_items] 32-row groups left to k_prep (counters[22])
    const int32_t *dorder;       // [n_pairs] pairs by article size, longest first: the n_dwide
                                 // pairs of more than kWideArticleSent target sentences, then the rest
    int32_t n_dwide;
    int32_t kmax;                // largest translation count of the dictionary
    int32_t *M;                  // tiled scores
    uint32_t *codes;             // directions
    uint32_t *matches;           // traceback matches (i << 16 | j), decreasing i
    int32_t *hfin;               // [n_nw_items] H[S][T] of a tiled alignment (unused by the others)
    const uint64_t *recip;       // [kMaxSentTokens + 1]: ceil(2^48 / m), 0 for m = 0
    const uint32_t *recip31;     // [kMaxSentTokens + 1]: ceil(2^31 / m), 0 for m = 0 (after recip)
    int2 *gscratch;              // per-warp tables for sentences longer than the shared ones
    int32_t f32;                 // score kernel writes single-precision scores (float bits) into M
    int32_t *counters;           // [8] work-queue heads
    int32_t *err;                // error word (0 = fine)
    uint32_t wait_spins;         // tries of a bounded flag wait (0: kWaitLimit)
    int32_t test_withhold;       // testing only: warp 0 of every warp pipeline publishes no rows
    // outputs
    int32_t *nw_score;           // [R]
    int32_t *n_sel;              // [R]
    int32_t *sel;                // mine_pair triples
};

// Alignment forms (the values of the strategy table, mine_align_strategy):
// a pipeline of 1, 2, 4 or 8 warps (warp w of a pipeline of G takes stripes
// w, w + G, ... of 32 rows), or tiles over many CTAs.  A one-warp alignment
// keeps the previous stripe's last row in a ring of kRing entries, so a pair
// with more than 32 source sentences and T >= kRing target sentences needs a
// pipeline of two or more warps; a pipeline of G warps needs G stripes and
// more than G tiles of 32 columns per row.
enum : int { AF_WARP1 = 0, AF_WARP8 = 1, AF_TILED = 2, AF_WARP2 = 3, AF_WARP4 = 4, AF_FORMS = 5 };
constexpr int kRing = 512;
constexpr int kNwPipe = 8;                  // warps of the widest pipeline (a CTA)
__host__ __device__ inline int form_warps(int f)
{
    return f == AF_WARP8 ? 8 : f == AF_WARP4 ? 4 : f == AF_WARP2 ? 2 : f == AF_WARP1 ? 1 : 0;
}
// queue heads of the alignment groups (pipelines of 8, 4, 2, 1 warps) in the
// batch's counters
__host__ __device__ constexpr int ctr_nw(int gi) { return gi == 0 ? 2 : gi == 1 ? 16 : gi == 2 ? 17 : 3; }
constexpr int kCounters = 32;               // queue heads and flags of a batch (index 8: error word)
constexpr int kAlignBins = MINE_ALIGN_BINS;

// Alignment form of an S x T pair: the tuned choice of its size bin (tab
// may be null; -1 keeps the built-in rule: tiles from kTiledCells, else
// about 2^14 cells or more per warp of a pipeline), made feasible: tiles
// need more than one tile row and column; a pipeline is narrowed (by powers
// of two) to at most the stripes and the column tiles - 1 of the pair, and
// widened to two warps where one warp cannot hold the ring.
inline int align_kind(const int8_t *tab, int32_t S, int32_t T)
{
    const int64_t c = (int64_t)S * T;
    const bool can_tile = S > kAlignTileRows && T > kAlignTileCols;
    const int bin = c > 0 ? 64 - __builtin_clzll((unsigned long long)c) : 0;   // 2^bin > c
    int v = (tab && bin < kAlignBins) ? tab[bin] : -1;
    if (v < 0)
        v = (can_tile && c >= kTiledCells) ? AF_TILED
            : c >= (int64_t(1) << 17) ? AF_WARP8 : c >= (int64_t(1) << 16) ? AF_WARP4
            : c >= (int64_t(1) << 15) ? AF_WARP2 : AF_WARP1;
    if (v == AF_TILED && !can_tile) v = AF_WARP8;
    if (v == AF_TILED) return v;
    const int ns = (S + 31) >> 5, tt = (T + 31) >> 5;
    // a pipeline whose warps take several stripes each hands the rows of its
    // last warp to its first one through rings of kRing entries: the first
    // warp must get a whole row (tt tiles) ahead of the last one, which the
    // ring space between the G - 1 links allows up to about 12 (G - 1) tiles.
    // The kernel runs min(g, ns, tt - 1) warps of a pipeline of g.
    auto feasible = [&](int g) {
        const int ge = g < ns ? (g < tt - 1 ? g : tt - 1) : (ns < tt - 1 ? ns : tt - 1);
        if (ge <= 1) return !(S > kTile && T >= kRing);
        return ns <= ge || tt <= 12 * (ge - 1);
    };
    int g = form_warps(v);
    while (g > 1 && (g > ns || g > tt - 1)) g >>= 1;   // no idle warps where a narrower one does
    if (!feasible(g)) {
        if (feasible(8)) g = 8;
        else if (can_tile) return AF_TILED;
        else g = 1;   // (a pair that reaches here has T <= 64)
    }
    return g == 8 ? AF_WARP8 : g == 4 ? AF_WARP4 : g == 2 ? AF_WARP2 : AF_WARP1;
}

// Union of the selections of a batch mined in both directions (the second
// plan has every pair's articles exchanged; same pairs, same settings).
struct UnionDev {
    const PairPlan *fwd, *bwd;
    int32_t n_pairs, nset;
    const int32_t *sel_f, *sel_b;    // selected triples of each direction
    const int32_t *nsel_f, *nsel_b;  // their counts, row set0 + k of each plan
    int32_t *out;                    // row (p, k) at 2 (sel_base + k min(S,T)) triples
    int32_t *n_out;                  // [rows of the forward plan]
    const int32_t *err_f, *err_b;    // error words of the two batches (nothing is done if set)
};

// Tuning objective: true positives and sizes of the selections per setting.
struct F1Dev {
    const PairPlan *pairs;
    int32_t n_pairs, nset;
    const int32_t *sel, *n_sel;
    const int32_t *truth;            // [n_sent] known target sentence of a source sentence, or -1
    unsigned long long *acc;         // [2 nset + 1]: tp per setting, selected per setting, known
    int32_t *best;                   // [1]
    const int32_t *err;              // error word of the batch (nothing is done if set)
};

// Contrast without the path constraint: each source sentence's best target.
struct BestDev {
    const PairPlan *pairs;
    int32_t n_pairs;
    const ScoreItem *items;          // 32-row groups of source sentences (the preparation items)
    int32_t n_items;
    const int32_t *M;                // tiled scores
    int32_t thr;
    int2 *best;                      // [n_sent] (target, score) of a source sentence, or (-1, 0)
    int32_t *out;                    // [3 n_sent] selected (i, j, s) of pair p from 3 s0 on
    int32_t *n_sel, *rep;            // [n_pairs] selected pairs, target sentences taken twice or more
    uint32_t *seen1, *seen2;         // [n_sent / 32 + 1] each, zeroed: targets taken once, twice
    const int32_t *err;              // error word of the scoring (nothing is done if set)
};

// launchers (kernels.cu, bidi_tune.cu, best_match.cu); each returns the number of kernels launched
int launch_dict_build(const int32_t *keys, const int32_t *trans_off, int32_t n_keys, DevDict d,
                      int32_t *err, cudaStream_t st);
int launch_validate(const int32_t *sent_off, int64_t n_sent, int64_t n_tok, int32_t *err,
                    cudaStream_t st);
int launch_prep(const BatchDev &b, const DevDict &d, int num_sms, cudaStream_t st);
int launch_pairprep_wide(const BatchDev &b, const DevDict &d, int num_sms, cudaStream_t st);
int launch_pairprep(const BatchDev &b, const DevDict &d, int num_sms, cudaStream_t st);
int launch_pairprep_xwide(const BatchDev &b, const DevDict &d, int num_sms, cudaStream_t st);
int launch_order(const BatchDev &b, int num_sms, cudaStream_t st);
int launch_score(const BatchDev &b, int num_sms, cudaStream_t st);        // small articles
int launch_score_wide(const BatchDev &b, int num_sms, cudaStream_t st);   // all other items
int launch_score_xwide(const BatchDev &b, int num_sms, cudaStream_t st);  // kDirect < ids <= kDirectX
int launch_align(const BatchDev &b, int num_sms, cudaStream_t st);
int launch_align_tiled(const BatchDev &b, int num_sms, cudaStream_t st);
int launch_trace(const BatchDev &b, int num_sms, cudaStream_t st);
int launch_tile(const int32_t *src, int32_t S, int32_t T, int32_t *dst, cudaStream_t st);
int launch_fill_scores(int32_t *M, int64_t n, uint32_t seed, cudaStream_t st);
int launch_union(const UnionDev &u, int num_sms, cudaStream_t st);
// packed outputs of the host call: rows r = p n + k, offsets off[0..R], triples in out
int launch_pack(const BatchDev &b, int32_t n, int32_t R, int32_t *bsum, int64_t *off, int32_t *out,
                cudaStream_t st);
int launch_f1(const F1Dev &f, int num_sms, cudaStream_t st);
int launch_best(const BestDev &d, int num_sms, cudaStream_t st);

// Record the text returned by mine_last_error() for this thread (runtime.cu).
void set_last_error(const char *msg);

// kernel identities for per-kernel timing
enum KernelId { KID_DICT = 0, KID_VALIDATE = 1, KID_PREP = 2, KID_SCORE = 3, KID_ALIGN = 4,
                KID_TILE = 5, KID_TRACE = 6, KID_ORDER = 7, KID_DOC = 8,
                KID_SCORE_WIDE = 9, KID_ALIGN_TILED = 10, KID_UNION = 11, KID_F1 = 12,
                KID_DOC_WIDE = 13, KID_PACK = 14, KID_BEST = 15, KID_DOC_XWIDE = 16,
                KID_SCORE_XWIDE = 17, KID_COUNT = 18 };

}  // namespace mine
