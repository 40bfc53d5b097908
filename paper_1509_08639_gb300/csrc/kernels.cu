// kernels.cu -- the miner's hot path on sm_103a.
//
// Per article pair (Section 4 of Wolk & Marasek): the sentence-pair score
// matrix M (token overlap through the bilingual dictionary + length, fixed
// point), then a Needleman-Wunsch global alignment over M with gap penalty g
// (monotone paths: "cannot go upward or leftward"), the traceback, and the
// selection of aligned pairs whose score passes the threshold.
//
// Kernels, in launch order (the wide-article preparation and score launches
// run on a second stream beside the small-article ones):
//   k_dict_build  once per dictionary: bucketed table (8 slots per 64-byte
//                 bucket) of key -> (offset, count) of its translations, and
//                 the inline table (two keys with their first translations)
//   k_validate    sentence offsets are sane (later kernels trust them)
//   k_pairprep    one CTA per pair, largest first, three launches (target
//                 articles of at most / more than 160 sentences, then the
//                 ones with too many distinct tokens for those): the target
//                 article's distinct tokens get dense ids (ranks of occupied
//                 slots of a shared table); every target token's id; one warp
//                 per source row: distinct tokens, dictionary lookups, and
//                 the translations the target article holds written as (id |
//                 FIRST | END) -- the only ones that can overlap
//   k_prep        the same for articles with more than 16384 distinct target
//                 tokens, keeping every translation (token-keyed path)
//   k_order       per pair, source rows by list length; the score items of
//                 the larger articles, listed for their launches
//   k_score       three launches (articles with at most 4096 distinct target
//                 tokens, from the plan's items; more, from k_order's list;
//                 8193-16384, by CTAs of 8 warps): per item of 64 (256)
//                 source rows and one range of target columns, block by block
//                 of 32 target sentences, a column mask per id
//                 (direct-indexed shared array, block ids TMA-staged), every
//                 lane adds the masks of its row's kept ids into bit-sliced
//                 carry-save counters, 8 x 8 bit transposes give the counts,
//                 exact reciprocal multiplies the ratios; 32 x 32 tiles of M.
//                 Articles beyond 16384 ids use a per-block hashed token ->
//                 column mask table instead.
//   k_nw          (align.cu) persistent wavefront fill: a pair by one warp or
//                 by a pipeline of 2, 4 or 8 warps over its 32-row stripes
//   k_align_tiled very large pairs: 256 x 512-cell tiles over many CTAs, in
//                 anti-diagonal order with bounded flag waits on the tiles
//                 above and on the left
//   k_trace       one warp per alignment: traceback over the packed codes and
//                 the threshold selection of every setting that shares the gap
#include "internal.h"
#include "async_copy.cuh"

#include <algorithm>
#include <cstdint>

namespace mine {

namespace {

constexpr uint32_t kFull = 0xffffffffu;

__device__ __forceinline__ uint32_t hmul(int32_t key) { return (uint32_t)key * 0x9E3779B1u; }

__device__ __forceinline__ int ceil_log2(int x)
{
    int l = 0;
    while ((1 << l) < x) ++l;
    return l;
}

// floor(x * 65536 / m) for 0 <= x <= m <= 1024, given K = ceil(2^48 / m)
// (the host-built reciprocal table; K = 0 for m = 0): the scaled reciprocal
// errs by less than x / 2^32 <= 1/m, which cannot carry the quotient past an
// integer.
__device__ __forceinline__ uint32_t mul_q16(uint32_t x, uint64_t K)
{
    return (uint32_t)(((uint64_t)x * K) >> 32);
}

// ---------------------------------------------------------------- dictionary

// The dictionary table is made of buckets of 8 (key, off << 6 | cnt) slots
// (64 bytes, read at once); a key lives in its hash bucket or, when that is
// full, in the next ones.  Slots of a bucket fill in order, so a bucket with
// an empty last slot ends every search.
constexpr int kDictBucket = 8;

__device__ __forceinline__ uint32_t dict_bucket(const DevDict &d, int32_t key)
{
    return hmul(key) >> (32 - (d.log2 - 3));
}

__device__ __forceinline__ void dict_load(const DevDict &d, uint32_t bk, int4 (&q)[4])
{
    const int4 *p = reinterpret_cast<const int4 *>(d.slots + (size_t)kDictBucket * bk);
#pragma unroll
    for (int i = 0; i < 4; ++i) q[i] = __ldg(p + i);
}

// (off, cnt) of `key` from its loaded bucket; `more` when the bucket is full
// without it (the search goes on in the next bucket).
__device__ __forceinline__ int2 dict_match(const int4 (&q)[4], int32_t key, bool &more)
{
    int32_t v = -1;
    bool hit = false;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (q[i].x == key) { v = q[i].y; hit = true; }
        if (q[i].z == key) { v = q[i].w; hit = true; }
    }
    more = !hit && q[3].z != -1;
    return hit ? make_int2((int32_t)((uint32_t)v >> 6), v & 63) : make_int2(0, 0);
}

__device__ __forceinline__ int2 dict_find(const DevDict &d, int32_t key)
{
    const uint32_t nbm = (1u << (d.log2 - 3)) - 1u;
    uint32_t bk = dict_bucket(d, key);
    for (;;) {   // ends: the table is at most half full
        int4 q[4];
        dict_load(d, bk, q);
        bool more;
        const int2 oc = dict_match(q, key, more);
        if (!more) return oc;
        bk = (bk + 1) & nbm;
    }
}

// Inline table: the bucket of `key` and, from its 64 loaded bytes, the
// entry holding it (0 or 1), -1 when the key is absent, or -2 when the bucket
// is full without it (the search goes on in the next bucket).
__device__ __forceinline__ uint32_t inl_bucket(const DevDict &d, int32_t key)
{
    return hmul(key) >> (32 - d.inl_log2);
}

__device__ __forceinline__ void inl_load(const DevDict &d, uint32_t bk, int4 (&q)[4])
{
    const int4 *p = d.inl + 4 * (size_t)bk;
#pragma unroll
    for (int i = 0; i < 4; ++i) q[i] = __ldg(p + i);
}

__device__ __forceinline__ int inl_match(const int4 (&q)[4], int32_t key)
{
    if (q[0].x == key) return 0;
    if (q[2].x == key) return 1;
    return q[2].x == -1 ? -1 : -2;
}

// (off, cnt) and the first four translations of `key` (0 past cnt) from its
// bucket chain in the inline table; cnt = 0 when the key is absent.
__device__ __forceinline__ int2 inl_find(const DevDict &d, int32_t key, int32_t (&u)[4])
{
    const uint32_t nbm = (1u << d.inl_log2) - 1u;
    uint32_t bk = inl_bucket(d, key);
    for (;;) {   // ends: the table is at most half full
        int4 q[4];
        inl_load(d, bk, q);
        const int e = inl_match(q, key);
        if (e != -2) {
            if (e < 0) {
                u[0] = u[1] = u[2] = u[3] = 0;
                return make_int2(0, 0);
            }
            const int4 h = q[2 * e], t = q[2 * e + 1];
            u[0] = h.z;
            u[1] = h.w;
            u[2] = t.x;
            u[3] = t.y;
            return make_int2((int32_t)((uint32_t)h.y >> 6), h.y & 63);
        }
        bk = (bk + 1) & nbm;
    }
}

__global__ void k_dict_build(const int32_t *__restrict__ keys, const int32_t *__restrict__ trans_off,
                             int32_t n_keys, DevDict d, int32_t *err)
{
    const uint32_t nbm = (1u << (d.log2 - 3)) - 1u;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_keys;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t key = keys[k];
        const int32_t off = trans_off[k];
        const int32_t cnt = trans_off[k + 1] - off;
        uint32_t bk = dict_bucket(d, key);
        bool done = false;
        for (uint32_t probe = 0; probe <= nbm && !done; ++probe) {
            for (int sl = 0; sl < kDictBucket; ++sl) {
                int2 *slot = d.slots + (size_t)kDictBucket * bk + sl;
                const int32_t old = atomicCAS(&slot->x, -1, key);
                if (old == -1) {
                    slot->y = (int32_t)(((uint32_t)off << 6) | (uint32_t)cnt);
                    done = true;
                    break;
                }
                if (old == key) {
                    atomicCAS(err, 0, ERR_DUP_KEY);
                    done = true;
                    break;
                }
            }
            bk = (bk + 1) & nbm;
        }
        // the inline table (a repeated key was reported above)
        const uint32_t ibm = (1u << d.inl_log2) - 1u;
        uint32_t ib = inl_bucket(d, key);
        done = false;
        for (uint32_t probe = 0; probe <= ibm && !done; ++probe) {
            for (int e = 0; e < 2 && !done; ++e) {
                int32_t *ent = reinterpret_cast<int32_t *>(d.inl + 4 * (size_t)ib + 2 * e);
                const int32_t old = atomicCAS(ent, -1, key);
                if (old == -1) {
                    ent[1] = (int32_t)(((uint32_t)off << 6) | (uint32_t)cnt);
                    for (int t = 0; t < kInlineTrans; ++t) ent[2 + t] = t < cnt ? d.trans[off + t] : 0;
                    done = true;
                } else if (old == key) {
                    done = true;
                }
            }
            ib = (ib + 1) & ibm;
        }
    }
}

// ---------------------------------------------------------------- shared hashes
// Open addressing, linear probing; callers keep the load factor <= 1/2, so
// every probe sequence meets an empty slot.

// Table entries are (key, 32-bit mask) pairs, so one 64-bit shared load
// answers a probe.  Keys are written once (CAS from -1) and never change.
__device__ __forceinline__ int tab_slot(int2 *tab, int log2, int32_t key)
{
    const uint32_t mask = (1u << log2) - 1u;
    uint32_t h = hmul(key) >> (32 - log2);
    for (;;) {
        int32_t k = tab[h].x;
        if (k == -1) {
            k = atomicCAS(&tab[h].x, -1, key);
            if (k == -1) return (int)h;
        }
        if (k == key) return (int)h;
        h = (h + 1) & mask;
    }
}

__device__ __forceinline__ void tab_clear(int2 *tab, int n, int lane)
{
    int4 *t4 = reinterpret_cast<int4 *>(tab);
    for (int q = lane; q < n / 2; q += 32) t4[q] = make_int4(-1, 0, -1, 0);
}

// Element list of source sentence `sent` (first token at tok_off): 16-byte
// aligned with room for L * kmax elements before the next sentence's list
// (the buffer holds n_tok * kmax + 3 * n_sent + 16 words).
__device__ __forceinline__ int64_t elem_base(int64_t tok_off, int64_t sent, int32_t kmax)
{
    return (tok_off * kmax + 3 * sent + 3) & ~(int64_t)3;
}

// ---------------------------------------------------------------- validation

__global__ void k_validate(const int32_t *__restrict__ sent_off, int64_t n_sent, int64_t n_tok,
                           int32_t *err)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_sent;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = sent_off[k], b = sent_off[k + 1];
        const bool bad = (k == 0 && a != 0) || (b < a) || (b - a > kMaxSentTokens) ||
                         (k == n_sent - 1 && (int64_t)b != n_tok);
        if (bad) atomicCAS(err, 0, ERR_BAD_OFFSETS);
    }
}

// ---------------------------------------------------------------- row preparation

constexpr int kSW = kScoreWarps;
constexpr int kSWS = kScoreWarpsScore;
constexpr int kPrepTok = 256;                    // tokens per preparation round
constexpr int kPrepElem = kColHashSlots / 2;     // translations per dedupe round
constexpr int kGTabSlots = 2 * kMaxSentTokens;   // per-warp global table for long sentences

// Per-warp shared memory of k_prep.  The table maps a source token to the
// mask of rows holding it, then a translation to the mask of rows whose U_i
// holds it.  grp lists the distinct (row, token) pairs of a round, then
// their dictionary entries (off << 6 | cnt, row | pos << 5).
struct alignas(16) PrepWarpSmem {
    int2 tab[kColHashSlots];
    int32_t tok[kPrepTok + 8];                   // TMA staging of a round's tokens
    int2 grp[kPrepTok];
    uint8_t rowmap[kPrepTok];                    // row of each staged token
    unsigned long long bar;
    int32_t rtok[33];
    int32_t rcnt[32], recnt[32], rU[32];
    int32_t ngrp;
};

// Set `bit` in the mask of `key`; true when it was not set before.
__device__ __forceinline__ bool tab_set(int2 *tab, int lg, int32_t key, uint32_t bit)
{
    const int slot = tab_slot(tab, lg, key);
    return !(atomicOr((uint32_t *)&tab[slot].y, bit) & bit);
}

// Stage tokens [tok0, tok0 + ntok) into dst with a TMA bulk copy (the bulk
// part is 16-byte aligned; the few tokens past the last 16-byte boundary of
// the token array are copied by lanes, which sets `generic`).  A buffer that
// generic stores wrote before gets a proxy fence first.  Returns the offset
// of tok0 in dst.
__device__ __forceinline__ int stage_tokens(const BatchDev &b, int32_t *dst,
                                            unsigned long long *bar, int64_t tok0, int ntok,
                                            int lane, bool &generic)
{
    const int64_t a0 = tok0 & ~(int64_t)3;
    const int64_t end = tok0 + ntok;
    const int64_t a1 = min((end + 3) & ~(int64_t)3, b.n_tok & ~(int64_t)3);
    const uint32_t bytes = a1 > a0 ? (uint32_t)(4 * (a1 - a0)) : 0u;
    if (generic) fence_proxy_async();
    generic = max(a1, a0) < end;
    __syncwarp();
    if (lane == 0) {
        mbar_expect_tx(bar, bytes);
        if (bytes) bulk_g2s(dst, b.tokens + a0, bytes, bar);
    }
    for (int64_t p = max(a1, a0) + lane; p < end; p += 32) dst[p - a0] = b.tokens[p];
    return (int)(tok0 - a0);
}

// Mark the first copy of every translation in out[0..nel) (one row) with
// ELEM_FIRST, using the per-warp global table, or a scan when even that is
// too small.  Returns the number of first copies (|U_i|).
__device__ int mark_first_copies(uint32_t *out, int nel, int2 *gtab, int lane)
{
    int firsts = 0;
    if (nel <= kGTabSlots / 2) {
        const int lgE = max(6, ceil_log2(2 * max(nel, 1)));
        tab_clear(gtab, 1 << lgE, lane);
        __syncwarp();
        for (int e = lane; e < nel; e += 32) {
            const int slot = tab_slot(gtab, lgE, (int32_t)(out[e] & ELEM_TOKEN));
            if (!(atomicOr((uint32_t *)&gtab[slot].y, 1u) & 1u)) {
                ++firsts;
                atomicOr(&out[e], ELEM_FIRST);
            }
        }
    } else {
        for (int e = lane; e < nel; e += 32) {
            const uint32_t u = out[e] & ELEM_TOKEN;
            bool first = true;
            for (int q = 0; q < e && first; ++q) first = (out[q] & ELEM_TOKEN) != u;
            firsts += first;
            if (first) atomicOr(&out[e], ELEM_FIRST);
        }
    }
    const int f = __reduce_add_sync(kFull, firsts);
    __syncwarp();
    return f;
}

// One warp per 32 source rows of a pair: distinct tokens X_i (n_i), their
// translations grouped per token with FIRST / END flags (U_i), written to the
// row's element list, and (n_i, #elements, |U_i|) to sinfo.
__global__ void __launch_bounds__(kSW * 32)
k_prep(BatchDev b, DevDict d)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    PrepWarpSmem &sm = reinterpret_cast<PrepWarpSmem *>(smem_raw)[wib];
    int2 *gtab = b.gscratch + (int64_t)(blockIdx.x * kSW + wib) * kGTabSlots;
    const int kmax = d.kmax;
    if (lane == 0) {
        mbar_init(&sm.bar, 1);
        fence_barrier_init();
    }
    __syncwarp();
    uint32_t parity = 0u;
    bool generic = false;
    // nothing to do unless k_pairprep left an article with too many distinct tokens
    if (*(volatile int32_t *)b.err || *(volatile int32_t *)&b.counters[14] == 0) return;

    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(&b.counters[0], 1);
        item = __shfl_sync(kFull, item, 0);
        // the 32-row groups of the pairs the extra-wide preparation listed
        if (item >= b.counters[22]) break;
        const ScoreItem si = b.keyed_items[item];
        if (b.pdoc[si.pair] >= 0) continue;   // prepared by k_pairprep
        const PairPlan pp = b.pairs[si.pair];
        const int nrows = min(32, pp.S - si.row0);
        const int64_t s_first = (int64_t)pp.s0 + si.row0;
        int32_t a_tok = 0, e_tok = 0;
        if (lane < nrows) {
            a_tok = b.sent_off[s_first + lane];
            e_tok = b.sent_off[s_first + lane + 1];
        }
        const int32_t tA = __shfl_sync(kFull, a_tok, 0);
        if (lane < nrows) sm.rtok[lane] = a_tok - tA;
        if (lane == nrows - 1) sm.rtok[nrows] = e_tok - tA;
        sm.rcnt[lane] = 0;
        sm.recnt[lane] = 0;
        sm.rU[lane] = 0;
        __syncwarp();
        for (int rA = 0; rA < nrows;) {
            // rows [rA, rB) with at most kPrepTok tokens, or one longer row alone
            const int cand = rA + 1 + lane;
            const bool okr = cand <= nrows && sm.rtok[cand] - sm.rtok[rA] <= kPrepTok;
            const int rB = rA + max(1, __popc(__ballot_sync(kFull, okr)));
            const int tbase = sm.rtok[rA];
            const int ntok = sm.rtok[rB] - tbase;
            if (ntok > kPrepTok) {
                // one long row, read from global memory, deduplicated in the
                // per-warp global table; translations written as found
                const int32_t *gtk = b.tokens + tA + tbase;
                uint32_t *out = b.elems + elem_base(tA + tbase, s_first + rA, kmax);
                const int lgT = max(6, ceil_log2(2 * ntok));
                tab_clear(gtab, 1 << lgT, lane);
                __syncwarp();
                int newc = 0;
                for (int k = lane; k < ntok; k += 32) {
                    const int32_t tok = gtk[k];
                    if ((uint32_t)tok > ELEM_TOKEN) atomicCAS(b.err, 0, ERR_BAD_TOKEN);
                    if (tab_set(gtab, lgT, tok & (int32_t)ELEM_TOKEN, 1u)) {
                        ++newc;
                        const int2 oc = dict_find(d, tok & (int32_t)ELEM_TOKEN);
                        const int pos = atomicAdd(&sm.recnt[rA], oc.y);
                        for (int q = 0; q < oc.y; ++q)
                            out[pos + q] = (uint32_t)__ldg(&d.trans[oc.x + q]) |
                                           (q == oc.y - 1 ? ELEM_END : 0u);
                    }
                }
                const int nd = __reduce_add_sync(kFull, newc);
                if (lane == 0) sm.rcnt[rA] = nd;
                __syncwarp();
                const int f = mark_first_copies(out, sm.recnt[rA], gtab, lane);
                if (lane == 0) sm.rU[rA] = f;
                __syncwarp();
                rA = rB;
                continue;
            }
            const int lead = stage_tokens(b, sm.tok, &sm.bar, (int64_t)tA + tbase, ntok, lane, generic);
            const int lg = max(6, ceil_log2(2 * max(ntok, 1)));
            tab_clear(sm.tab, 1 << lg, lane);
            if (lane == 0) sm.ngrp = 0;
            if (!mbar_wait(&sm.bar, parity, b.err)) return;
            parity ^= 1u;
            __syncwarp();
            // row of every staged token (each lane marks its row's range)
            if (lane >= rA && lane < rB) {
                const int k1 = sm.rtok[lane + 1] - tbase;
                for (int k = sm.rtok[lane] - tbase; k < k1; ++k) sm.rowmap[k] = (uint8_t)lane;
            }
            __syncwarp();
            // distinct (row, token), all lanes over the tokens: the table maps a
            // token to the mask of rows holding it
            {
                const int32_t *stk = sm.tok + lead;
                for (int k = lane; k < ntok; k += 32) {
                    const int32_t tok = stk[k];
                    if ((uint32_t)tok > ELEM_TOKEN) atomicCAS(b.err, 0, ERR_BAD_TOKEN);
                    const int r = sm.rowmap[k];
                    if (tab_set(sm.tab, lg, tok & (int32_t)ELEM_TOKEN, 1u << r)) {
                        atomicAdd(&sm.rcnt[r], 1);
                        sm.grp[atomicAdd(&sm.ngrp, 1)] = make_int2(tok & (int32_t)ELEM_TOKEN, r);
                    }
                }
            }
            __syncwarp();
            const int ng = sm.ngrp;
            // dictionary lookups
            for (int g0 = 0; g0 < ng; g0 += 64) {
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int g = g0 + q * 32 + lane;
                    if (g < ng) {
                        const int2 oc = dict_find(d, sm.grp[g].x);
                        const int r = sm.grp[g].y;
                        const int pos = atomicAdd(&sm.recnt[r], oc.y);
                        sm.grp[g] = make_int2((int32_t)(((uint32_t)oc.x << 6) | (uint32_t)oc.y),
                                              r | (pos << 5));
                    }
                }
            }
            __syncwarp();
            // translations of rows [eA, eB), at most kPrepElem of them per round;
            // one row with more goes alone (global table or scan)
            for (int eA = rA; eA < rB;) {
                const int v = (eA + lane < rB) ? sm.recnt[eA + lane] : 0;
                int incl = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(kFull, incl, o);
                    if (lane >= o) incl += y;
                }
                const bool fits = (eA + lane < rB) && incl <= kPrepElem;
                const int eB = eA + max(1, __popc(__ballot_sync(kFull, fits)));
                const int nel = __shfl_sync(kFull, incl, eB - eA - 1);
                const bool alone = nel > kPrepElem;
                const int lgE = max(6, ceil_log2(2 * max(nel, 1)));
                if (!alone) {
                    tab_clear(sm.tab, 1 << lgE, lane);
                    __syncwarp();
                }
                for (int g = lane; g < ng; g += 32) {
                    const int2 gr = sm.grp[g];
                    const int r = gr.y & 31;
                    if (r < eA || r >= eB) continue;
                    const uint32_t pk = (uint32_t)gr.x;
                    const int off = (int)(pk >> 6), cnt = (int)(pk & 63u);
                    uint32_t *out = b.elems + elem_base(tA + sm.rtok[r], s_first + r, kmax) + (gr.y >> 5);
                    const uint32_t bit = 1u << r;
                    int firsts = 0;
                    for (int k = 0; k < cnt; ++k) {
                        const int32_t u = __ldg(&d.trans[off + k]);
                        const bool first = !alone && tab_set(sm.tab, lgE, u, bit);
                        firsts += first;
                        out[k] = (uint32_t)u | (first ? ELEM_FIRST : 0u) | (k == cnt - 1 ? ELEM_END : 0u);
                    }
                    if (firsts) atomicAdd(&sm.rU[r], firsts);
                }
                __syncwarp();
                if (alone) {
                    uint32_t *out = b.elems + elem_base(tA + sm.rtok[eA], s_first + eA, kmax);
                    const int f = mark_first_copies(out, nel, gtab, lane);
                    if (lane == 0) sm.rU[eA] = f;
                    __syncwarp();
                }
                eA = eB;
            }
            rA = rB;
        }
        __syncwarp();
        if (lane < nrows) b.sinfo[s_first + lane] = make_int4(sm.rcnt[lane], sm.recnt[lane], sm.rU[lane], 0);
        __syncwarp();
    }
}

// ---------------------------------------------------------------- k_pairprep

// Two launches: target articles of at most kWideArticleSent sentences by
// CTAs of 8 warps with a table of kSmallSlots slots (five CTAs per SM, the
// most their shared memory allows, with registers capped to fit: more pairs
// in flight and fewer warps waiting at a pair's barriers), the others by
// CTAs of 16 warps with a table of 2 kDirect slots.  A small article stops
// once it has more than kSmallIds distinct tokens (before its table fills)
// and goes to the extra-wide launch.
constexpr int kSmallSlots = 8192;
constexpr int kSmallIds = 6144;
constexpr int kRowSetBig = 2 * kMaxSentTokens;     // rows of > 64 tokens: per-warp table in global memory
static_assert(kRowSetBig * 8 <= kScoreScratchPerWarp, "per-warp global table too small");

template <int WARPS, int SLOTS, int IDS>
struct alignas(16) PairPrepSmem {
    static constexpr int kIds = IDS;           // document ids below this
    int32_t key[SLOTS];                        // target tokens of the article
    uint32_t occ[SLOTS / 32];                  // occupied slots
    uint16_t rank[SLOTS / 32];                 // occupied slots before each word
    uint32_t seen[WARPS][IDS / 32];            // ids already kept in the warp's current row
    int32_t cbuf[WARPS][64];                   // distinct tokens of the row, compacted
    int32_t nd;
    int32_t item;
};

// Document id of target token `tok` (the rank of its slot among the
// occupied ones), or -1 when the article lacks it.
template <class SM>
__device__ __forceinline__ int doc_id(const SM &sm, int lg, int32_t tok)
{
    const uint32_t mask = (1u << lg) - 1u;
    uint32_t h = hmul(tok) >> (32 - lg);
    for (;;) {   // ends: the table always has empty slots
        const int32_t k = sm.key[h];
        if (k == tok) {
            const uint32_t w = h >> 5;
            return (int)sm.rank[w] + __popc(sm.occ[w] & ((1u << (h & 31)) - 1u));
        }
        if (k == -1) return -1;
        h = (h + 1) & mask;
    }
}

// Insert target token `tok`; returns its slot, and `added` is set when this
// call added it (the caller counts the additions, one atomic per warp).
template <class SM>
__device__ __forceinline__ uint32_t doc_insert(SM &sm, int lg, int32_t tok, bool &added)
{
    const uint32_t mask = (1u << lg) - 1u;
    uint32_t h = hmul(tok) >> (32 - lg);
    volatile int32_t *key = sm.key;
    added = false;
    for (;;) {
        const int32_t k = key[h];
        if (k == tok) return h;
        if (k == -1) {
            const int32_t old = atomicCAS(&sm.key[h], -1, tok);
            if (old == -1) {
                added = true;
                return h;
            }
            if (old == tok) return h;
        }
        h = (h + 1) & mask;
    }
}

// Insert `tok` into a row set whose live entries carry `stamp`; true when
// the token is new in this row.  Entries of earlier rows count as empty.
__device__ __forceinline__ bool rset_insert(int2 *set, int lg, int32_t tok, int32_t stamp)
{
    const uint32_t mask = (1u << lg) - 1u;
    uint32_t h = hmul(tok) >> (32 - lg);
    unsigned long long *s64 = reinterpret_cast<unsigned long long *>(set);
    const unsigned long long mine = ((unsigned long long)(uint32_t)stamp << 32) | (uint32_t)tok;
    unsigned long long cur = *reinterpret_cast<volatile unsigned long long *>(&s64[h]);
    for (;;) {
        if ((int32_t)(cur >> 32) != stamp) {
            const unsigned long long old = atomicCAS(&s64[h], cur, mine);
            if (old == cur) return true;
            cur = old;   // taken meanwhile: look at it again
            continue;
        }
        if ((uint32_t)cur == (uint32_t)tok) return false;
        h = (h + 1) & mask;
        cur = *reinterpret_cast<volatile unsigned long long *>(&s64[h]);
    }
}

// Distinct tokens of a row of L <= 64 tokens (t0: tokens 0..31, t1: 32..63,
// one per lane), compacted into cb[0..n); returns n.  ht: 256 zero words of
// shared memory (zero again on return), a small table for rows of more than
// 32 tokens.
__device__ __forceinline__ int distinct64(int32_t t0, int32_t t1, int L, int lane, int32_t *cb,
                                          uint32_t *ht)
{
    const bool v0 = lane < L, v1 = 32 + lane < L;
    const int32_t k0 = v0 ? t0 : -1 - lane;   // tokens are >= 0: sentinels never match one
    // every lane takes part in the match (no short-circuit around it)
    const uint32_t m0 = __match_any_sync(kFull, k0);
    const bool lead0 = v0 && (__ffs(m0) - 1 == lane);
    bool lead1 = false;
    if (L > 32) {
        const int32_t k1 = v1 ? t1 : -1 - lane;
        const uint32_t m1 = __match_any_sync(kFull, k1);
        lead1 = v1 && (__ffs(m1) - 1 == lane);
        // a second-half token already in the first half: the first half's
        // distinct tokens (keys token + 1) go into the table, the second
        // half's look them up, and the table is cleared again
        int slot0 = -1;
        if (lead0) {
            uint32_t h = hmul(t0) >> 24;
            while (atomicCAS(&ht[h], 0u, (uint32_t)t0 + 1u) != 0u) h = (h + 1) & 255u;   // keys differ
            slot0 = (int)h;
        }
        __syncwarp();
        bool dup = false;
        if (lead1) {
            uint32_t h = hmul(t1) >> 24;
            for (;;) {   // ends: at most 32 of the 256 slots are used
                const uint32_t v = ht[h];
                if (v == (uint32_t)t1 + 1u) {
                    dup = true;
                    break;
                }
                if (v == 0u) break;
                h = (h + 1) & 255u;
            }
        }
        lead1 = lead1 && !dup;
        __syncwarp();
        if (slot0 >= 0) ht[slot0] = 0u;
        __syncwarp();
    }
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t b0 = __ballot_sync(kFull, lead0), b1 = __ballot_sync(kFull, lead1);
    const int n0 = __popc(b0);
    if (lead0) cb[__popc(b0 & lt)] = t0;
    if (lead1) cb[n0 + __popc(b1 & lt)] = t1;
    __syncwarp();
    return n0 + __popc(b1);
}

// Kept translations of one distinct source token per lane (first four given
// in u, the rest read again): write them from position out + (earlier lanes'
// kept count) as (id | FIRST | END); advances out by the warp's total.
template <class SM>
__device__ __forceinline__ void emit_kept(const BatchDev &b, const DevDict &d, const SM &sm,
                                          int lg, const int32_t (&u)[4], int2 oc, uint32_t *seen,
                                          uint32_t *el, int &out, int &nf, int lane)
{
    int id[4];
    int kc = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        id[q] = q < oc.y ? doc_id(sm, lg, u[q]) : -1;
        kc += id[q] >= 0 ? 1 : 0;
    }
    for (int q = 4; q < oc.y; ++q) kc += doc_id(sm, lg, __ldg(&d.trans[oc.x + q])) >= 0 ? 1 : 0;
    int incl = kc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    int pos = out + incl - kc;
    out += __shfl_sync(kFull, incl, 31);
    int left = kc;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (id[q] >= 0) {
            const uint32_t bit = 1u << (id[q] & 31);
            const bool first = !(atomicOr(&seen[id[q] >> 5], bit) & bit);
            nf += first ? 1 : 0;
            --left;
            el[pos++] = (uint32_t)id[q] | (first ? ELEM_FIRST : 0u) | (left == 0 ? ELEM_END : 0u);
        }
    }
    for (int q = 4; q < oc.y; ++q) {
        const int idv = doc_id(sm, lg, __ldg(&d.trans[oc.x + q]));
        if (idv >= 0) {
            const uint32_t bit = 1u << (idv & 31);
            const bool first = !(atomicOr(&seen[idv >> 5], bit) & bit);
            nf += first ? 1 : 0;
            --left;
            el[pos++] = (uint32_t)idv | (first ? ELEM_FIRST : 0u) | (left == 0 ? ELEM_END : 0u);
        }
    }
}

// One source row of <= 64 tokens: tokens, distinct tokens (warp match, no
// table), dictionary buckets, translations, then the kept translations.
template <class SM>
__device__ void prep_row_short(const BatchDev &b, const DevDict &d, const SM &sm, int lg,
                               int64_t s, int32_t a, int32_t L, int32_t t0, int32_t t1, int lane,
                               uint32_t *seen, int32_t *cb, int kmax)
{
    // t0, t1: tokens a+lane and a+32+lane of the row (0 past its end)
    if (((uint32_t)t0 | (uint32_t)t1) > ELEM_TOKEN) {
        atomicCAS(b.err, 0, ERR_BAD_TOKEN);
        t0 &= (int32_t)ELEM_TOKEN;
        t1 &= (int32_t)ELEM_TOKEN;
    }
    const int n = distinct64(t0, t1, L, lane, cb, seen);   // (the row's id bitmap is zero here)
    uint32_t *el = b.elems + elem_base(a, s, kmax);
    int out = 0, nf = 0;
    for (int g = 0; 32 * g < n; ++g) {
        const int k = 32 * g + lane;
        const bool v = k < n;
        const int32_t key = v ? cb[k] : 0;
        int2 oc = make_int2(0, 0);
        int32_t u[4] = {0, 0, 0, 0};
        if (v) oc = inl_find(d, key, u);
        emit_kept(b, d, sm, lg, u, oc, seen, el, out, nf, lane);
    }
    nf = (int)__reduce_add_sync(kFull, (unsigned)nf);
    if (lane == 0) b.sinfo[s] = make_int4(n, out, nf, 0);
    __syncwarp();
    uint4 *sz = reinterpret_cast<uint4 *>(seen);
    for (int q = lane; q < SM::kIds / 128; q += 32) sz[q] = make_uint4(0u, 0u, 0u, 0u);
    __syncwarp();
}

// One source row of any length (distinct tokens through a per-warp table in
// global memory whose live entries carry the row's stamp).
template <class SM>
__device__ void prep_row_long(const BatchDev &b, const DevDict &d, const SM &sm, int lg,
                              int64_t s, int32_t a, int32_t L, int lane, int2 *gset,
                              bool &gset_clean, int32_t stamp, uint32_t *seen)
{
    if (!gset_clean) {
        int4 *gz = reinterpret_cast<int4 *>(gset);
        for (int k = lane; k < kRowSetBig / 2; k += 32) gz[k] = make_int4(-1, 0, -1, 0);
        __syncwarp();
        gset_clean = true;
    }
    uint32_t *el = b.elems + elem_base(a, s, b.kmax);
    int n_i = 0, out = 0, nf = 0;
    for (int c = 0; c < L; c += 32) {
        const bool valid = c + lane < L;
        int32_t tok = valid ? b.tokens[a + c + lane] : 0;
        if ((uint32_t)tok > ELEM_TOKEN) {
            atomicCAS(b.err, 0, ERR_BAD_TOKEN);
            tok &= (int32_t)ELEM_TOKEN;
        }
        const bool isnew = valid && rset_insert(gset, 11, tok, stamp);
        n_i += __popc(__ballot_sync(kFull, isnew));
        int2 oc = make_int2(0, 0);
        int32_t u[4] = {0, 0, 0, 0};
        if (isnew) oc = inl_find(d, tok, u);
        emit_kept(b, d, sm, lg, u, oc, seen, el, out, nf, lane);
    }
    nf = (int)__reduce_add_sync(kFull, (unsigned)nf);
    if (lane == 0) b.sinfo[s] = make_int4(n_i, out, nf, 0);
    __syncwarp();
    uint4 *sz = reinterpret_cast<uint4 *>(seen);
    for (int q = lane; q < SM::kIds / 128; q += 32) sz[q] = make_uint4(0u, 0u, 0u, 0u);
    __syncwarp();
}

// Modes of the preparation launches: target articles of more than
// kWideArticleSent sentences (wide), the others (small), and the articles
// those found to hold too many distinct tokens (extra wide: up to kDirectX
// ids, a table of 2 kDirectX slots, one CTA per SM).
constexpr int kModeWide = 0, kModeSmall = 1, kModeXWide = 2;

// One CTA per pair (largest first), for every pair whose target article has
// at most kDirect (kDirectX in the extra-wide mode) distinct tokens:
//  1. the article's distinct tokens go into a shared table; their dense ids
//     are the ranks of the occupied slots (pdoc[p] = D, the count);
//  2. every target token's id goes to tdoc;
//  3. one warp per source row: distinct tokens (n_i), their dictionary
//     translations, of which only those the target article holds are kept,
//     written as (id | FIRST | END) -- FIRST on the first copy of an id in the
//     row, END on the last kept translation of each source token -- with
//     (n_i, #kept, #kept FIRST) in sinfo.
// A larger article gets pdoc[p] = -1 and is left to the extra-wide launch,
// then to k_prep and the token-keyed score path.
template <int WARPS, int SLOTS, int CTAS, int MODE>
__global__ void __launch_bounds__(WARPS * 32, CTAS)
k_pairprep(BatchDev b, DevDict d)
{
    constexpr bool SMALL = MODE == kModeSmall, XW = MODE == kModeXWide;
    constexpr int IDS = XW ? kDirectX : kDirect;
    constexpr int kPPWarps = WARPS, kPPThreads = WARPS * 32;
    // the most distinct target tokens an article of this launch may have
    constexpr int kCap = SMALL ? kSmallIds : IDS;
    static_assert(kCap <= IDS && kCap + 4 * kPPThreads < SLOTS, "the target table never fills");
    // nothing to do unless another launch left an article with too many ids
    // (their pairs listed in xw_list, counters[21] of them)
    if (XW && *(volatile int32_t *)&b.counters[9] == 0) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PairPrepSmem<WARPS, SLOTS, IDS> &sm = *reinterpret_cast<PairPrepSmem<WARPS, SLOTS, IDS> *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    int2 *gset = b.gscratch + (int64_t)(blockIdx.x * kPPWarps + wib) * kGTabSlots;
    bool gset_clean = false;
    int32_t stamp = 0;
    for (int k = tid; k < kPPWarps * (IDS / 32); k += kPPThreads) (&sm.seen[0][0])[k] = 0u;
    const int kmax = b.kmax;
    for (;;) {
        if (__syncthreads_or(*(volatile int32_t *)b.err != 0)) break;
        // items: the wide launch takes dorder[0, n_dwide), the small one the
        // rest, the extra-wide one every pair the others left
        if (tid == 0) {
            sm.item = atomicAdd(&b.counters[SMALL ? 5 : (XW ? 11 : 10)], 1) + (SMALL ? b.n_dwide : 0);
            sm.nd = 0;
        }
        __syncthreads();
        const int item = sm.item;
        if (item >= (MODE == kModeWide ? b.n_dwide : (XW ? b.counters[21] : b.n_pairs))) break;
        const int p = XW ? b.xw_list[item] : b.dorder[item];
        if (XW && b.pdoc[p] != -1) continue;    // prepared by one of the other launches
        const PairPlan pp = b.pairs[p];
        const int32_t ta = b.sent_off[pp.t0], tb = b.sent_off[pp.t0 + pp.T];
        // at most a quarter of the slots used where the table allows (the
        // probes of absent translations, the common case, end sooner)
        const int lg = min(max(ceil_log2(4 * max(tb - ta, 1)), 10), SMALL ? 13 : (XW ? 15 : 14));
        const int NS = 1 << lg;
        int4 *kz = reinterpret_cast<int4 *>(sm.key);
        for (int k = tid; k < NS / 4; k += kPPThreads) kz[k] = make_int4(-1, -1, -1, -1);
        __syncthreads();
        // 1. distinct target tokens; four loads in flight per thread; the
        //    warp adds its new tokens to the count at once; an article stops
        //    once its tokens cannot all get ids (before its table fills: at
        //    most 4 kPPThreads more insertions than kCap)
        for (int32_t kw = ta + (tid & ~31); kw < tb; kw += 4 * kPPThreads) {   // warp-uniform
            if (__shfl_sync(kFull, *(volatile int32_t *)&sm.nd, 0) > kCap) break;
            const int32_t k = kw + lane;
            int32_t tk[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int32_t kk = k + q * kPPThreads;
                tk[q] = kk < tb ? b.tokens[kk] : -1;
            }
            unsigned added = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int32_t kk = k + q * kPPThreads;
                if (kk < tb) {
                    uint32_t h = 0;
                    if ((uint32_t)tk[q] > ELEM_TOKEN) {
                        atomicCAS(b.err, 0, ERR_BAD_TOKEN);
                    } else {
                        bool a;
                        h = doc_insert(sm, lg, tk[q], a);
                        added += a ? 1u : 0u;
                    }
                    b.tdoc[kk] = (uint16_t)h;   // the slot; its rank replaces it below
                }
            }
            added = __reduce_add_sync(kFull, added);
            if (lane == 0 && added) atomicAdd(&sm.nd, (int)added);
        }
        __syncthreads();
        const int D = sm.nd;
        if (tid == 0) {
            if (!XW) {
                b.pdoc[p] = D <= kCap ? D : -1;
                if (D > kCap) {   // the extra-wide launch has work: this pair
                    b.xw_list[atomicAdd(&b.counters[21], 1)] = p;
                    atomicExch(&b.counters[9], 1);
                }
            } else if (D <= kCap) {
                b.pdoc[p] = D;
                // so has the extra-wide score launch, unless another one takes it
                if (D > kDirect) atomicExch(&b.counters[13], 1);
            } else {
                // k_prep has work (pdoc stays -1): this pair's 32-row groups
                const int n = (pp.S + 31) >> 5;
                const int at = atomicAdd(&b.counters[22], n);
                for (int k = 0; k < n; ++k) b.keyed_items[at + k] = ScoreItem{p, 32 * k, 0, 0};
                atomicExch(&b.counters[14], 1);
            }
        }
        if (D > kCap) continue;
        const int NW = NS >> 5;
        for (int w = wib; w < NW; w += kPPWarps)
            sm.occ[w] = __ballot_sync(kFull, sm.key[32 * w + lane] != -1);
        __syncthreads();
        if (wib == 0) {
            const int per = NW >> 5;   // NW >= 32
            int run = 0;
            for (int q = 0; q < per; ++q) run += __popc(sm.occ[lane * per + q]);
            int incl = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += y;
            }
            int base = incl - run;
            for (int q = 0; q < per; ++q) {
                sm.rank[lane * per + q] = (uint16_t)base;
                base += __popc(sm.occ[lane * per + q]);
            }
        }
        __syncthreads();
        // 2. id of every target token: the rank of the slot phase 1 found for
        //    it (each thread rewrites the entries it wrote there)
        for (int32_t k = ta + tid; k < tb; k += 4 * kPPThreads) {
            uint32_t hs[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int32_t kk = k + q * kPPThreads;
                hs[q] = kk < tb ? b.tdoc[kk] : 0u;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int32_t kk = k + q * kPPThreads;
                const uint32_t h = hs[q] & ((1u << lg) - 1u);
                const uint32_t w = h >> 5;
                if (kk < tb) b.tdoc[kk] = (uint16_t)((int)sm.rank[w] + __popc(sm.occ[w] & ((1u << (h & 31)) - 1u)));
            }
        }
        // 3. source rows, one warp each (rows wib, wib + kPPWarps, ...).  The
        //    loads of the next row's tokens and of the offsets of the row after
        //    it are in flight while a row is prepared.
        auto offsets = [&](int j) {   // lanes 0, 1: start and end of row j
            int32_t v = 0;
            if (j < pp.S && lane < 2) v = b.sent_off[(int64_t)pp.s0 + j + lane];
            return v;
        };
        auto tokens_of = [&](int32_t a, int32_t L, int32_t &t0, int32_t &t1) {
            t0 = (L <= 64 && lane < L) ? b.tokens[a + lane] : 0;
            t1 = (L <= 64 && 32 + lane < L) ? b.tokens[a + 32 + lane] : 0;
        };
        int32_t v = offsets(wib);
        int32_t a = __shfl_sync(kFull, v, 0), L = __shfl_sync(kFull, v, 1) - a;
        int32_t t0, t1;
        tokens_of(a, L, t0, t1);
        v = offsets(wib + kPPWarps);
        for (int j = wib; j < pp.S; j += kPPWarps) {
            const int32_t an = __shfl_sync(kFull, v, 0), Ln = __shfl_sync(kFull, v, 1) - an;
            int32_t n0, n1;
            tokens_of(an, Ln, n0, n1);               // row j + kPPWarps
            v = offsets(j + 2 * kPPWarps);          // row j + 2 kPPWarps
            const int64_t sj = (int64_t)pp.s0 + j;
            if (L > 64)
                prep_row_long(b, d, sm, lg, sj, a, L, lane, gset, gset_clean, ++stamp, sm.seen[wib]);
            else
                prep_row_short(b, d, sm, lg, sj, a, L, t0, t1, lane, sm.seen[wib], sm.cbuf[wib], kmax);
            a = an;
            L = Ln;
            t0 = n0;
            t1 = n1;
        }
    }
}

// ---------------------------------------------------------------- k_order

// Score launches: articles of at most kDirectSmall distinct target tokens
// (from the plan's item list), and the others (from a list k_order builds).
constexpr int kDirectSmall = 4096;
constexpr int kScoreWarpsX = 8;   // warps per CTA of the extra-wide score launch

// Per pair, the source rows sorted by element count, longest first (counting
// sort on min(count, 1023); ties in any order), written to row_order[s0 ..
// s0+S); and the score items of the pairs with more than kDirectSmall
// distinct target tokens (or the token-keyed path) appended to wide_items.
// One warp per pair.
__global__ void __launch_bounds__(256)
k_order(BatchDev b)
{
    __shared__ int32_t hist_all[8][1024];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    int32_t *hist = hist_all[wib];
    if (*(volatile int32_t *)b.err) return;
    for (int p = (blockIdx.x * 8 + wib); p < b.n_pairs; p += gridDim.x * 8) {
        const PairPlan pp = b.pairs[p];
        const int S = pp.S;
        const int D = b.pdoc[p];
        if (D < 0 || D > kDirectSmall) {
            // the pair's score items, for the launches of larger articles:
            // 32 rows per warp of the launch that takes them (64, or 32
            // kScoreWarpsX for the extra-wide ones) by kScoreColChunk columns
            const int rows = D > kDirect ? 32 * kScoreWarpsX : 64;
            const int nc = (max(pp.T, 1) + kScoreColChunk - 1) / kScoreColChunk, n = ((S + rows - 1) / rows) * nc;
            int base = 0;
            if (lane == 0 && n > 0) base = atomicAdd(&b.counters[18], n);
            base = __shfl_sync(kFull, base, 0);
            for (int k = lane; k < n; k += 32) {
                const int c0 = kScoreColChunk * (k % nc);
                b.wide_items[base + k] = ScoreItem{p, rows * (k / nc), c0, min(pp.T, c0 + kScoreColChunk)};
            }
        }
        int32_t *ord = b.row_order + pp.s0;
        if (S <= 32) {
            if (lane < S) ord[lane] = lane;
            continue;
        }
        for (int k = lane; k < 1024; k += 32) hist[k] = 0;
        __syncwarp();
        for (int r = lane; r < S; r += 32) {
            const int key = 1023 - min(b.sinfo[(int64_t)pp.s0 + r].y, 1023);
            atomicAdd(&hist[key], 1);
        }
        __syncwarp();
        // exclusive scan of 1024 buckets: 32 per lane, then across lanes
        int run = 0;
        for (int k = 0; k < 32; ++k) {
            const int v = hist[lane * 32 + k];
            hist[lane * 32 + k] = run;
            run += v;
        }
        int incl = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        const int base = incl - run;
        for (int k = 0; k < 32; ++k) hist[lane * 32 + k] += base;
        __syncwarp();
        for (int r = lane; r < S; r += 32) {
            const int key = 1023 - min(b.sinfo[(int64_t)pp.s0 + r].y, 1023);
            ord[atomicAdd(&hist[key], 1)] = r;
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------- k_score

// Per-warp buffers of the token-keyed path: the column-block table (target
// token -> mask of the block's columns holding it), two TMA staging buffers,
// the column of each staged token and the block's column data.
struct alignas(16) KeyedWarp {
    int2 tab[kColHashSlots];
    int32_t tok[2][kColTokCap + 8];
    uint8_t colmap[kColTokCap];
    int32_t soff[2][33];
    uint64_t Km[32];        // reciprocal of m_j
    uint64_t KL[32];        // reciprocal of L'_j
    int32_t Lt[32];
    int32_t mcnt[32];       // m_j of the block being built
};

// CTA buffers of the document-id path: a column mask per document id below
// DIRECT (entry DIRECT stays zero), the TMA-staged ids of one block's tokens
// and the block's column data.
template <int DIRECT>
struct alignas(16) DirectCta {
    uint32_t mask[DIRECT + 16];
    uint16_t ids[kBlkTokCap + 32];
    uint64_t Km[32];
    uint64_t KL[32];
    int32_t Lt[32];
    int32_t Mj[32];          // m_j (single-precision scores)
    uint32_t Rm[32];         // the 32-bit reciprocals of m_j and L'_j (kRecip31Max at most)
    uint32_t RL[32];
};

// Shared memory of one k_score CTA (W warps).  The mbarriers stay outside
// the union: both paths write it with generic stores.  Without the
// token-keyed path (KEYED false) the per-warp buffers are not needed.
template <int DIRECT, bool KEYED, int W>
struct alignas(16) ScoreSmem {
    union {
        KeyedWarp kw[KEYED ? W : 1];
        DirectCta<DIRECT> d;
    };
    unsigned long long bar[W][2];      // token-keyed path, per warp
    unsigned long long dbar;           // document-id path
    int32_t item;
};

// The two score launches: articles with at most kDirectSmall distinct target
// tokens (small mask array, more CTAs per SM), and all others.

__device__ __forceinline__ void csa(uint32_t &carry, uint32_t &sum, uint32_t a, uint32_t b,
                                    uint32_t c)
{
    const uint32_t u = a ^ b;
    carry = (a & b) | (u & c);
    sum = u ^ c;
}

// Counts of columns 8m .. 8m+7 from eight bit planes: gather byte m of every
// plane into a 64-bit 8 x 8 bit matrix (row k = plane k) and transpose it;
// byte c of (lo, hi) is then the count of column 8m + c.
__device__ __forceinline__ void planes_to_bytes(const uint32_t (&P)[8], int m, uint32_t &lo,
                                                uint32_t &hi)
{
    const uint32_t sel = (uint32_t)m | ((uint32_t)(m + 4) << 4);
    const uint32_t t01 = __byte_perm(P[0], P[1], sel), t23 = __byte_perm(P[2], P[3], sel);
    const uint32_t t45 = __byte_perm(P[4], P[5], sel), t67 = __byte_perm(P[6], P[7], sel);
    lo = __byte_perm(t01, t23, 0x5410);
    hi = __byte_perm(t45, t67, 0x5410);
    uint32_t t;
    t = (lo ^ (lo >> 7)) & 0x00AA00AAu;  lo ^= t ^ (t << 7);
    t = (hi ^ (hi >> 7)) & 0x00AA00AAu;  hi ^= t ^ (t << 7);
    t = (lo ^ (lo >> 14)) & 0x0000CCCCu; lo ^= t ^ (t << 14);
    t = (hi ^ (hi >> 14)) & 0x0000CCCCu; hi ^= t ^ (t << 14);
    t = (lo ^ (hi << 4)) & 0xF0F0F0F0u;
    lo ^= t;
    hi ^= t >> 4;
}

template <int NPL>
__device__ __forceinline__ uint32_t plane_value(const uint32_t (&P)[NPL], int col)
{
    uint32_t v = 0;
#pragma unroll
    for (int k = 0; k < NPL; ++k) v |= ((P[k] >> col) & 1u) << k;
    return v;
}

__device__ __forceinline__ int32_t cell_score(uint32_t a, uint32_t bb, uint64_t Km, uint64_t Ks,
                                              int Ls, int Lt, uint64_t KLs, uint64_t KLt)
{
    const uint32_t q_t = mul_q16(a, Km);
    const uint32_t q_s = mul_q16(bb, Ks);
    uint32_t q_l;
    if (Ls == 0 && Lt == 0) {
        q_l = 65536u;
    } else {
        const uint32_t lmin = (uint32_t)min(Ls, Lt);
        q_l = mul_q16(lmin, Ls >= Lt ? KLs : KLt);
    }
    const uint32_t h = (q_t + q_s) >> 1;
    // (49152 * h + 16384 * q_l) >> 16 == (3h + q_l) >> 2
    return (int32_t)((3u * h + q_l) >> 2);
}

// The same score with 32-bit reciprocals, for counts and lengths of at most
// kRecip31Max: R = ceil(2^31 / m) = 2^31 / m + e (0 <= e < 1), so
// (x 2^17) R / 2^32 = x 2^16 / m + x e / 2^15, and x e / 2^15 < m / 2^15 < 1 / m
// when m^2 < 2^15 (m <= 181): below the distance from x 2^16 / m to the next
// integer, so the high word is the floor (m = 0: R = 0 and x = 0).
__device__ __forceinline__ int32_t cell_score32(uint32_t a, uint32_t bb, uint32_t Rm, uint32_t Rs, int Ls,
                                                int Lt, uint32_t RLs, uint32_t RLt)
{
    const uint32_t q_t = __umulhi(a << 17, Rm);
    const uint32_t q_s = __umulhi(bb << 17, Rs);
    const uint32_t q_l = (Ls == 0 && Lt == 0) ? 65536u
                                              : __umulhi((uint32_t)min(Ls, Lt) << 17, Ls >= Lt ? RLs : RLt);
    const uint32_t h = (q_t + q_s) >> 1;
    return (int32_t)((3u * h + q_l) >> 2);
}

// Single-precision score of one cell from the same counts: the coverage and
// length ratios by correctly rounded division, then 0.375 (q_t + q_s) +
// 0.25 q_l (the fixed-point weights 49152/2 and 16384 over 65536).
__device__ __forceinline__ float cell_score_f32(uint32_t a, uint32_t bb, int m, int n, int Ls, int Lt)
{
    const float rt = m > 0 ? __fdiv_rn((float)a, (float)m) : 0.f;
    const float rs = n > 0 ? __fdiv_rn((float)bb, (float)n) : 0.f;
    const int lmax = max(Ls, Lt);
    const float rl = lmax > 0 ? __fdiv_rn((float)min(Ls, Lt), (float)lmax) : 1.f;
    return 0.375f * (rt + rs) + 0.25f * rl;
}

// Column mask of `key` in the block table (valid lanes only).  The first
// slot settles almost every probe without a branch; lanes whose key sits
// further along continue in a loop that the warp enters only when needed.
__device__ __forceinline__ uint32_t probe2(const int2 *tab, uint32_t mask, int lg, int32_t key,
                                           bool valid)
{
    uint32_t h = hmul(key) >> (32 - lg);
    const int2 e0 = valid ? tab[h] : make_int2(key, 0);
    uint32_t o = e0.x == key ? (uint32_t)e0.y : 0u;
    bool more = e0.x != key && e0.x != -1;
    if (__any_sync(kFull, more)) {
        while (more) {
            h = (h + 1) & mask;
            const int2 e = tab[h];
            o = e.x == key ? (uint32_t)e.y : 0u;
            more = e.x != key && e.x != -1;
        }
    }
    return o;
}

// Add two 32-lane bit vectors to the bit-sliced counter P: a carry-save
// adder for plane 0, then a ripple.
template <int NPL>
__device__ __forceinline__ void add2(uint32_t (&P)[NPL], uint32_t x, uint32_t y)
{
    uint32_t c;
    csa(c, P[0], P[0], x, y);
#pragma unroll
    for (int k = 1; k < NPL; ++k) {
        const uint32_t n = P[k] & c;
        P[k] ^= c;
        c = n;
    }
}

template <int NPL, bool F32>
__device__ __forceinline__ void emit_row(const uint32_t (&A)[NPL], const uint32_t (&B)[NPL],
                                         const uint64_t *Km, const uint64_t *KL, const int32_t *Lt,
                                         uint64_t Ks, uint64_t KLs, int Ls, int ncols,
                                         int32_t *mrow, int c0, const int32_t *Mj, int n_i);

// emit_row with the single-precision form chosen at run time (uniform per launch)
template <int NPL>
__device__ __forceinline__ void emit_row_any(const uint32_t (&A)[NPL], const uint32_t (&B)[NPL],
                                             const uint64_t *Km, const uint64_t *KL, const int32_t *Lt,
                                             uint64_t Ks, uint64_t KLs, int Ls, int ncols, int32_t *mrow,
                                             int c0, bool f32, const int32_t *Mj, int n_i)
{
    if (f32) emit_row<NPL, true>(A, B, Km, KL, Lt, Ks, KLs, Ls, ncols, mrow, c0, Mj, n_i);
    else emit_row<NPL, false>(A, B, Km, KL, Lt, Ks, KLs, Ls, ncols, mrow, c0, Mj, n_i);
}

// Accumulate the overlap counts of one column block and score its cells
// into row `lane` of the score tiles (mrow points at column tile 0).
// NPL <= 8: bit planes are turned into byte counts by 8 x 8 transposes.
template <int NPL>
__device__ __forceinline__ void score_block(const KeyedWarp &sm, const int2 *tab, int lg,
                                         const uint32_t *el, int n_elem, int nE2, int ncols,
                                         bool row_ok, uint64_t Ks, uint64_t KLs, int Ls,
                                         int32_t *mrow, int c0, bool f32, int n_i)
{
    uint32_t A[NPL], B[NPL];
#pragma unroll
    for (int k = 0; k < NPL; ++k) A[k] = B[k] = 0u;
    const uint32_t mask = (1u << lg) - 1u;
    uint32_t hit = 0;
    uint2 nx = make_uint2(0, 0);
    if (0 < n_elem) nx = *reinterpret_cast<const uint2 *>(el);
    for (int e0 = 0; e0 < nE2; e0 += 2) {
        const uint2 v = nx;
        if (e0 + 2 < n_elem) nx = *reinterpret_cast<const uint2 *>(el + e0 + 2);   // prefetch
        // validity comes from the index: token 0 without flags is a real element
        const bool va = e0 < n_elem, vb = e0 + 1 < n_elem;
        const uint32_t ea = va ? v.x : 0u;
        const uint32_t eb = vb ? v.y : 0u;
        const uint32_t oa = probe2(tab, mask, lg, (int32_t)(ea & ELEM_TOKEN), va);
        const uint32_t ob = probe2(tab, mask, lg, (int32_t)(eb & ELEM_TOKEN), vb);
        const uint32_t xa0 = (ea & ELEM_FIRST) ? oa : 0u;
        hit |= oa;
        const uint32_t xb0 = (ea & ELEM_END) ? hit : 0u;
        hit = (ea & ELEM_END) ? 0u : hit;
        const uint32_t xa1 = (eb & ELEM_FIRST) ? ob : 0u;
        hit |= ob;
        const uint32_t xb1 = (eb & ELEM_END) ? hit : 0u;
        hit = (eb & ELEM_END) ? 0u : hit;
        add2<NPL>(A, xa0, xa1);
        add2<NPL>(B, xb0, xb1);
    }
    if (!row_ok) return;
    emit_row_any<NPL>(A, B, sm.Km, sm.KL, sm.Lt, Ks, KLs, Ls, ncols, mrow, c0, f32, sm.mcnt, n_i);
}

// Score the cells of one row and one column block from its bit-sliced counts
// A (|U_i and X_j|) and B (source tokens with a translation in X_j) into the
// row's score tiles (mrow points at column tile 0).  NPL <= 8: bit planes are
// turned into byte counts by 8 x 8 transposes.
template <int NPL, bool F32>
__device__ __forceinline__ void emit_row(const uint32_t (&A)[NPL], const uint32_t (&B)[NPL],
                                         const uint64_t *Km, const uint64_t *KL, const int32_t *Lt,
                                         uint64_t Ks, uint64_t KLs, int Ls, int ncols,
                                         int32_t *mrow, int c0, const int32_t *Mj, int n_i)
{
    const bool whole = ncols == 32 && (c0 & 31) == 0;   // one whole row of one tile
    if constexpr (NPL <= 8) {
        uint32_t A8[8], B8[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            A8[k] = k < NPL ? A[k] : 0u;
            B8[k] = k < NPL ? B[k] : 0u;
        }
#pragma unroll 1
        for (int m = 0; m < 4 && 8 * m < ncols; ++m) {
            uint32_t alo, ahi, blo, bhi;
            planes_to_bytes(A8, m, alo, ahi);
            planes_to_bytes(B8, m, blo, bhi);
            int32_t v[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int jj = 8 * m + c;
                const uint32_t a = ((c < 4 ? alo : ahi) >> (8 * (c & 3))) & 0xffu;
                const uint32_t bb = ((c < 4 ? blo : bhi) >> (8 * (c & 3))) & 0xffu;
                if constexpr (F32) v[c] = __float_as_int(cell_score_f32(a, bb, Mj[jj], n_i, Ls, Lt[jj]));
                else v[c] = cell_score(a, bb, Km[jj], Ks, Ls, Lt[jj], KLs, KL[jj]);
            }
            if (whole) {
                int4 *dst = reinterpret_cast<int4 *>(mrow + (int64_t)(c0 >> 5) * kTileElems + 8 * m);
                dst[0] = make_int4(v[0], v[1], v[2], v[3]);
                dst[1] = make_int4(v[4], v[5], v[6], v[7]);
            } else {
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int jj = 8 * m + c;
                    if (jj < ncols) {
                        const int col = c0 + jj;
                        mrow[(int64_t)(col >> 5) * kTileElems + (col & 31)] = v[c];
                    }
                }
            }
        }
    } else {
        for (int jj = 0; jj < ncols; ++jj) {
            const uint32_t a = plane_value<NPL>(A, jj), bb = plane_value<NPL>(B, jj);
            int32_t v;
            if constexpr (F32) v = __float_as_int(cell_score_f32(a, bb, Mj[jj], n_i, Ls, Lt[jj]));
            else v = cell_score(a, bb, Km[jj], Ks, Ls, Lt[jj], KLs, KL[jj]);
            const int col = c0 + jj;
            mrow[(int64_t)(col >> 5) * kTileElems + (col & 31)] = v;
        }
    }
}

// emit_row (NPL = 8, fixed point) with the 32-bit reciprocals of cell_score32
__device__ __forceinline__ void emit_row32(const uint32_t (&A)[8], const uint32_t (&B)[8], const uint32_t *Rm,
                                           const uint32_t *RL, const int32_t *Lt, uint32_t Rs, uint32_t RLs,
                                           int Ls, int ncols, int32_t *mrow, int c0)
{
    const bool whole = ncols == 32 && (c0 & 31) == 0;   // one whole row of one tile
#pragma unroll 1
    for (int m = 0; m < 4 && 8 * m < ncols; ++m) {
        uint32_t alo, ahi, blo, bhi;
        planes_to_bytes(A, m, alo, ahi);
        planes_to_bytes(B, m, blo, bhi);
        int32_t v[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int jj = 8 * m + c;
            const uint32_t a = ((c < 4 ? alo : ahi) >> (8 * (c & 3))) & 0xffu;
            const uint32_t bb = ((c < 4 ? blo : bhi) >> (8 * (c & 3))) & 0xffu;
            v[c] = cell_score32(a, bb, Rm[jj], Rs, Ls, Lt[jj], RLs, RL[jj]);
        }
        if (whole) {
            int4 *dst = reinterpret_cast<int4 *>(mrow + (int64_t)(c0 >> 5) * kTileElems + 8 * m);
            dst[0] = make_int4(v[0], v[1], v[2], v[3]);
            dst[1] = make_int4(v[4], v[5], v[6], v[7]);
        } else {
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int jj = 8 * m + c;
                if (jj < ncols) {
                    const int col = c0 + jj;
                    mrow[(int64_t)(col >> 5) * kTileElems + (col & 31)] = v[c];
                }
            }
        }
    }
}

// Add eight 32-lane bit vectors to the bit-sliced counter P (planes 0..2 are
// the ones / twos / fours of a carry-save tree; the weight-8 carry ripples
// into the planes above).
template <int NPL>
__device__ __forceinline__ void add8(uint32_t (&P)[NPL], const uint32_t (&x)[8])
{
    uint32_t t1, t2, f1, f2, e;
    csa(t1, P[0], P[0], x[0], x[1]);
    csa(t2, P[0], P[0], x[2], x[3]);
    csa(f1, P[1], P[1], t1, t2);
    csa(t1, P[0], P[0], x[4], x[5]);
    csa(t2, P[0], P[0], x[6], x[7]);
    csa(f2, P[1], P[1], t1, t2);
    csa(e, P[2], P[2], f1, f2);
#pragma unroll
    for (int k = 3; k < NPL; ++k) {
        const uint32_t n = P[k] & e;
        P[k] ^= e;
        e = n;
    }
}

// Overlap counts of one row and one 32-column block on the document-id path:
// the row's hit list (document id | FIRST | END of its token group) is read
// eight entries at a time; each id's column mask comes from the block's mask
// array.  A counts FIRST entries, B counts token groups with any hit.
template <int NPL, int ZERO>
__device__ __forceinline__ void direct_counts(const uint32_t *mask, const uint32_t *hl, int n_h,
                                              int nIt, uint4 f0, uint4 f1, uint32_t (&A)[NPL],
                                              uint32_t (&B)[NPL])
{
#pragma unroll
    for (int k = 0; k < NPL; ++k) A[k] = B[k] = 0u;
    uint32_t hit = 0;
    // entries 0..7 stay in registers for the whole item; later ones are read
    // one step ahead
    uint4 n0 = make_uint4(0u, 0u, 0u, 0u), n1 = n0;
    if (8 < n_h) {
        n0 = *reinterpret_cast<const uint4 *>(hl + 8);
        n1 = *reinterpret_cast<const uint4 *>(hl + 12);
    }
#pragma unroll 1
    for (int it = 0; it < nIt; ++it) {
        const int k0 = it * 8;
        uint4 v0 = f0, v1 = f1;
        if (it > 0) {
            v0 = n0;
            v1 = n1;
            if (k0 + 8 < n_h) {
                n0 = *reinterpret_cast<const uint4 *>(hl + k0 + 8);
                n1 = *reinterpret_cast<const uint4 *>(hl + k0 + 12);
            }
        }
        const uint32_t ev[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
        uint32_t xa[8], xb[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const bool ok = k0 + q < n_h;
            const uint32_t en = ok ? ev[q] : 0u;
            const uint32_t m = mask[ok ? min(en & ELEM_TOKEN, (uint32_t)ZERO) : (uint32_t)ZERO];
            xa[q] = (en & ELEM_FIRST) ? m : 0u;
            hit |= m;
            xb[q] = (en & ELEM_END) ? hit : 0u;
            hit = (en & ELEM_END) ? 0u : hit;
        }
        add8<NPL>(A, xa);
        add8<NPL>(B, xb);
    }
}

// Stage the document ids of tokens [k0, k1) into ids[] (one bulk copy of the
// 16-byte aligned range around them); returns the offset of k0 in ids[].
__device__ __forceinline__ int stage_ids(const BatchDev &b, uint16_t *ids, unsigned long long *bar,
                                         int32_t k0, int32_t k1, bool issue)
{
    const int32_t a0 = k0 & ~7, a1 = (k1 + 7) & ~7;   // the id array is padded past n_tok
    if (issue) {
        const uint32_t bytes = (uint32_t)(2 * (a1 - a0));
        mbar_expect_tx(bar, bytes);
        if (bytes) bulk_g2s(ids, b.tdoc + a0, bytes, bar);
    }
    return k0 - a0;
}

// One score item (up to 32 W source rows) on the document-id path, block by
// block (32 columns), by the whole CTA: the block's ids are staged by TMA
// (one block ahead); threads W j .. W j + W - 1 set bit j in the mask of
// every id of target sentence j and count m_j on the way; every warp counts the hits of
// its 32 rows and scores their cells; the masks of ids [0, D) are cleared
// again.  A block with more than kBlkTokCap tokens reads its ids from global
// memory.  Returns false (on every thread) when a bounded wait ran out.
template <int DIRECT, int W>
__device__ bool score_item_direct(const BatchDev &b, DirectCta<DIRECT> &sd, unsigned long long *dbar,
                                  uint32_t &dparity, const PairPlan &pp, int D, int tid, int nrows,
                                  bool row_ok, const uint32_t *hl, int n_h, int n_i, uint64_t Ks,
                                  uint64_t KLs, int Ls, int32_t *mrow, int cbeg, int cend)
{
    const int maxH = (int)__reduce_max_sync(kFull, (unsigned)n_h);   // this warp's rows
    // this warp's rows short enough for the 32-bit reciprocals (n_i <= Ls)
    const bool rows32 = __all_sync(kFull, !row_ok || Ls <= kRecip31Max);
    const uint32_t Rs = b.recip31[min(n_i, kRecip31Max)], RLs = b.recip31[min(Ls, kRecip31Max)];
    const int nIt = (maxH + 7) >> 3;
    uint4 f0 = make_uint4(0u, 0u, 0u, 0u), f1 = f0;
    if (0 < n_h) {
        f0 = *reinterpret_cast<const uint4 *>(hl);
        f1 = *reinterpret_cast<const uint4 *>(hl + 4);
    }
    // W threads per target column of the block (tid = W col + part)
    const int col = tid / W, part = tid % W;
    const int64_t t0 = pp.t0;
    int32_t k0 = b.sent_off[t0 + cbeg], k1 = b.sent_off[t0 + cbeg + max(0, min(32, cend - cbeg))];
    // a copy is issued only for a block the loop below consumes (and waits for)
    bool staged = cbeg < cend && k1 - k0 <= kBlkTokCap;
    int lead = staged ? stage_ids(b, sd.ids, dbar, k0, k1, tid == 0) : 0;
    for (int c0 = cbeg; c0 < cend; c0 += 32) {
        const int ncols = min(32, cend - c0);
        const int64_t j0 = t0 + c0;
        int32_t a = 0, e = 0;
        if (col < ncols) {
            a = b.sent_off[j0 + col];
            e = b.sent_off[j0 + col + 1];
        }
        // next block's token range, read while this one is in flight
        const bool more = c0 + 32 < cend;
        int32_t nk1 = 0;
        if (more) nk1 = b.sent_off[j0 + 32 + min(32, cend - c0 - 32)];
        bool ok = true;
        if (staged) {
            ok = mbar_wait(dbar, dparity, b.err);
            dparity ^= 1u;
        }
        if (!__syncthreads_and(ok)) return false;
        const uint32_t bit = 1u << col;
        int m = 0;
        if (staged) {
            const uint16_t *ids = sd.ids + lead - k0;
            for (int32_t k = a + part; k < e; k += W)
                m += (atomicOr(&sd.mask[min((uint32_t)ids[k], (uint32_t)DIRECT - 1)], bit) & bit) ? 0 : 1;
        } else {
            for (int32_t k = a + part; k < e; k += W)
                m += (atomicOr(&sd.mask[min((uint32_t)b.tdoc[k], (uint32_t)DIRECT - 1)], bit) & bit) ? 0 : 1;
        }
#pragma unroll
        for (int o = 1; o < W; o <<= 1) m += __shfl_xor_sync(kFull, m, o);
        if (part == 0 && col < ncols) {
            sd.Km[col] = __ldg(&b.recip[m]);
            sd.KL[col] = __ldg(&b.recip[e - a]);
            sd.Lt[col] = e - a;
            sd.Mj[col] = m;
            sd.Rm[col] = __ldg(&b.recip31[min(m, kRecip31Max)]);
            sd.RL[col] = __ldg(&b.recip31[min(e - a, kRecip31Max)]);
        }
        // every column of the block short enough for the 32-bit reciprocals (m_j <= L'_j)
        const bool cols32 = __syncthreads_and(part != 0 || col >= ncols || e - a <= kRecip31Max);
        // the ids are in the masks now: stage the next block's
        if (more) {
            k0 = k1;
            k1 = nk1;
            staged = k1 - k0 <= kBlkTokCap;
            if (staged) lead = stage_ids(b, sd.ids, dbar, k0, k1, tid == 0);
        }
        if (nrows > 0) {
            if (maxH < 256) {
                uint32_t A[8], B[8];
                direct_counts<8, DIRECT>(sd.mask, hl, n_h, nIt, f0, f1, A, B);
                if (rows32 && cols32 && !b.f32) {
                    if (row_ok) emit_row32(A, B, sd.Rm, sd.RL, sd.Lt, Rs, RLs, Ls, ncols, mrow, c0);
                } else if (row_ok) {
                    emit_row_any<8>(A, B, sd.Km, sd.KL, sd.Lt, Ks, KLs, Ls, ncols, mrow, c0, b.f32 != 0,
                                    sd.Mj, n_i);
                }
            } else {
                uint32_t A[11], B[11];
                direct_counts<11, DIRECT>(sd.mask, hl, n_h, nIt, f0, f1, A, B);
                if (row_ok)
                    emit_row_any<11>(A, B, sd.Km, sd.KL, sd.Lt, Ks, KLs, Ls, ncols, mrow, c0, b.f32 != 0,
                                     sd.Mj, n_i);
            }
        }
        __syncthreads();
        uint4 *mz = reinterpret_cast<uint4 *>(sd.mask);
        for (int k = tid; k < (D + 3) >> 2; k += W * 32) mz[k] = make_uint4(0u, 0u, 0u, 0u);
        __syncthreads();
    }
    return true;
}

__device__ __forceinline__ int plan_block(const BatchDev &b, KeyedWarp &sm, unsigned long long *bar,
                                          int buf, int64_t tcol0, int c0, int T, int lane, int &ntok,
                                          int &lead, bool &generic, bool &staged, int64_t &tok0);

// One score item on the token-keyed path, one warp for its 32 rows.
// Returns false when a bounded wait ran out.
__device__ bool score_item_keyed(const BatchDev &b, KeyedWarp &sm, unsigned long long *bar,
                                 uint32_t (&parity)[2], bool (&generic)[2], int2 *gtab,
                                 const PairPlan &pp, int lane, bool row_ok, const uint32_t *el,
                                 int n_elem, int nU, int n_i, uint64_t Ks, uint64_t KLs, int Ls,
                                 int32_t *mrow, int cbeg, int cend)
{
    const int T = cend;   // blocks end at the item's last column
    const int64_t tcol0 = pp.t0;
    const uint64_t *recip = b.recip;
    const int nE2 = (int)((__reduce_max_sync(kFull, (unsigned)n_elem) + 1) & ~1u);
    const int maxU = (int)__reduce_max_sync(kFull, (unsigned)nU);
    const int maxN = (int)__reduce_max_sync(kFull, (unsigned)n_i);
    int cur = 0;
    int c0 = cbeg, ntok = 0, lead = 0, ncols = 0;
    bool staged = false;
    int64_t tok0 = 0;
    if (c0 < T)
        ncols = plan_block(b, sm, bar, 0, tcol0, c0, T, lane, ntok, lead, generic[0], staged, tok0);
    bool pending = ncols > 0 && staged;   // a copy in flight into buffer `cur`
    while (c0 < T) {
        if (ncols == 0) {
            if (lane == 0) atomicCAS(b.err, 0, ERR_BAD_OFFSETS);
            break;
        }
        int2 *tab = staged ? sm.tab : gtab;
        const int lg = max(6, ceil_log2(2 * max(ntok, 1)));
        tab_clear(tab, 1 << lg, lane);
        // prefetch the next block into the other buffer while this one is built and scored
        const int nc0 = c0 + ncols;
        int n_ncols = 0, n_ntok = 0, n_lead = 0;
        bool n_staged = false;
        int64_t n_tok0 = 0;
        if (nc0 < T)
            n_ncols = plan_block(b, sm, bar, cur ^ 1, tcol0, nc0, T, lane, n_ntok, n_lead,
                                 generic[cur ^ 1], n_staged, n_tok0);
        if (staged) {
            if (!mbar_wait(&bar[cur], parity[cur], b.err)) return false;
            parity[cur] ^= 1u;
        }
        pending = n_ncols > 0 && n_staged;
        __syncwarp();
        // column of every staged token, then all lanes insert the block's
        // tokens (token -> column mask) and count each column's distinct ones
        const int32_t *tks = staged ? sm.tok[cur] + lead : b.tokens + tok0;
        sm.mcnt[lane] = 0;
        if (staged && lane < ncols) {
            const int k1 = sm.soff[cur][lane + 1];
            for (int k = sm.soff[cur][lane]; k < k1; ++k) sm.colmap[k] = (uint8_t)lane;
        }
        __syncwarp();
        for (int k = lane; k < ntok; k += 32) {
            const int32_t tok = tks[k];
            if ((uint32_t)tok > ELEM_TOKEN) atomicCAS(b.err, 0, ERR_BAD_TOKEN);
            const int col = staged ? sm.colmap[k] : 0;
            if (tab_set(tab, lg, tok & (int32_t)ELEM_TOKEN, 1u << col)) atomicAdd(&sm.mcnt[col], 1);
        }
        __syncwarp();
        int m = 0;
        if (lane < ncols) {
            m = sm.mcnt[lane];
            const int Lt = sm.soff[cur][lane + 1] - sm.soff[cur][lane];
            sm.Km[lane] = __ldg(&recip[m]);
            sm.KL[lane] = __ldg(&recip[Lt]);
            sm.Lt[lane] = Lt;
        }
        const int maxM = (int)__reduce_max_sync(kFull, (unsigned)m);
        __syncwarp();
        const int bound = max(min(maxU, maxM), maxN);
        if (bound < 256) {
            score_block<8>(sm, tab, lg, el, n_elem, nE2, ncols, row_ok, Ks, KLs, Ls, mrow, c0,
                           b.f32 != 0, n_i);
        } else {
            score_block<11>(sm, tab, lg, el, n_elem, nE2, ncols, row_ok, Ks, KLs, Ls, mrow, c0,
                            b.f32 != 0, n_i);
        }
        __syncwarp();
        c0 = nc0;
        ncols = n_ncols;
        ntok = n_ntok;
        lead = n_lead;
        staged = n_staged;
        tok0 = n_tok0;
        cur ^= 1;
    }
    if (pending) {   // a block was staged but not used (bad offsets): let it land
        const bool ok = mbar_wait(&bar[cur], parity[cur], b.err);
        parity[cur] ^= 1u;
        if (!ok) return false;
    }
    __syncwarp();
    return true;
}

// Plan the column block starting at c0: widest run of <= 32 target sentences
// whose tokens fit the table; stage its tokens into buffer `buf`.  A single
// column longer than kColTokCap becomes an unstaged block (staged = false)
// read from global memory into the per-warp global table.  Returns ncols
// (>= 1, or 0 on bad offsets); tok0 receives the block's first token index.
__device__ __forceinline__ int plan_block(const BatchDev &b, KeyedWarp &sm, unsigned long long *bar,
                                          int buf, int64_t tcol0, int c0, int T, int lane, int &ntok,
                                          int &lead, bool &generic, bool &staged, int64_t &tok0)
{
    tok0 = b.sent_off[tcol0 + c0];
    int cum = 0x7fffffff;
    if (c0 + lane < T) cum = b.sent_off[tcol0 + c0 + lane + 1] - (int32_t)tok0;
    int ncols = __popc(__ballot_sync(kFull, cum <= kColTokCap));
    staged = ncols > 0;
    if (!staged) {
        const int first = __shfl_sync(kFull, cum, 0);
        if (c0 >= T || first < 0 || first > kMaxSentTokens) return 0;
        ncols = 1;
    }
    ntok = __shfl_sync(kFull, cum, ncols - 1);
    if (lane < ncols) sm.soff[buf][lane + 1] = cum;
    if (lane == 0) sm.soff[buf][0] = 0;
    lead = 0;
    if (staged) lead = stage_tokens(b, sm.tok[buf], &bar[buf], tok0, ntok, lane, generic);
    return ncols;
}

// DIRECT = kDirectSmall: items of articles with at most that many distinct
// target tokens (queue counters[1]); DIRECT = kDirectX: articles with more
// than kDirect and at most kDirectX (queue counters[12]); DIRECT = kDirect
// with KEYED: all other items, document-id or token-keyed (queue counters[6]).
// W warps per CTA, 32 rows each: 2 (items of 64 rows), or kScoreWarpsX for
// the extra-wide articles, whose 64 KB mask array leaves room for 3 CTAs per
// SM (items of 32 kScoreWarpsX rows, from k_order's list).
template <int DIRECT, bool KEYED, int W>
__global__ void __launch_bounds__(W * 32, KEYED ? 1 : (W == 2 ? 11 : 3))   // 11 small-launch CTAs per SM fit
k_score(BatchDev b)
{
    constexpr bool XW = !KEYED && DIRECT == kDirectX;
    if (XW && *(volatile int32_t *)&b.counters[13] == 0) return;   // no such article
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ScoreSmem<DIRECT, KEYED, W> &S = *reinterpret_cast<ScoreSmem<DIRECT, KEYED, W> *>(smem_raw);
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int wib = tid >> 5;
    KeyedWarp &kw = S.kw[wib];
    unsigned long long *kbar = S.bar[wib];
    int2 *gtab = b.gscratch + (int64_t)(blockIdx.x * W + wib) * kGTabSlots;
    const uint64_t *recip = b.recip;
    const int kmax = b.kmax;
    if (lane == 0) {
        mbar_init(&kbar[0], 1);
        mbar_init(&kbar[1], 1);
        if (wib == 0) mbar_init(&S.dbar, 1);
        fence_barrier_init();
    }
    uint32_t parity[2] = {0u, 0u}, dparity = 0u;
    bool generic[2] = {false, false};   // generic stores wrote into kw.tok[buf] since its last copy
    bool mask_clean = false;            // S.d.mask is all zero
    bool ok = true;

    for (;;) {
        // every thread leaves together: on an error (here or in another CTA)
        // or when the queue is empty
        if (__syncthreads_or(!ok || *(volatile int32_t *)b.err != 0)) break;
        if (tid == 0) S.item = atomicAdd(&b.counters[KEYED ? 6 : (XW ? 12 : 1)], 1);
        __syncthreads();
        const int item = S.item;
        // the larger articles' launches take the list k_order built
        constexpr bool kWideList = KEYED || XW;
        if (item >= (kWideList ? b.counters[18] : b.n_score_items)) break;
        const ScoreItem si = kWideList ? b.wide_items[item] : b.score_items[item];
        const int D = b.pdoc[si.pair];
        if (KEYED ? (D >= 0 && (D <= kDirectSmall || D > kDirect))
                  : (XW ? (D <= kDirect || D > kDirectX) : (D < 0 || D > kDirectSmall)))
            continue;   // another launch's item
        const PairPlan pp = b.pairs[si.pair];
        const int TT = (pp.T + 31) >> 5;
        // this warp's 32 rows, in the pair's order of element counts (the
        // rows of one warp have lists of similar length)
        const int row0 = si.row0 + 32 * wib;
        const int nrows = max(0, min(32, pp.S - row0));
        const bool row_ok = lane < nrows;
        const int r = row_ok ? b.row_order[(int64_t)pp.s0 + row0 + lane] : 0;
        const int64_t s_row = (int64_t)pp.s0 + r;
        int4 inf = make_int4(0, 0, 0, 0);
        int32_t a_tok = 0, e_tok = 0;
        if (row_ok) {
            inf = b.sinfo[s_row];
            a_tok = b.sent_off[s_row];
            e_tok = b.sent_off[s_row + 1];
        }
        const int n_i = inf.x, n_elem = inf.y, nU = inf.z;
        const int Ls = e_tok - a_tok;
        const uint32_t *el = row_ok ? b.elems + elem_base(a_tok, s_row, kmax) : b.elems;
        const uint64_t Ks = __ldg(&recip[n_i]);
        const uint64_t KLs = __ldg(&recip[Ls]);
        int32_t *mrow = b.M + pp.m_off + (int64_t)(r >> 5) * TT * kTileElems + (r & 31) * kTile;

        if (D >= 0) {
            // document-id path (the element list holds the row's hits)
            if (!mask_clean) {
                // the token-keyed path wrote these bytes with generic stores
                uint4 *mz = reinterpret_cast<uint4 *>(S.d.mask);
                for (int k = tid; k < (DIRECT + 16) / 4; k += W * 32) mz[k] = make_uint4(0u, 0u, 0u, 0u);
                fence_proxy_async();
                __syncthreads();
                mask_clean = true;
            }
            // generic stores now cover the keyed staging buffers: fence before their next copy
            generic[0] = generic[1] = true;
            ok = score_item_direct<DIRECT, W>(b, S.d, &S.dbar, dparity, pp, D, tid, nrows, row_ok, el,
                                           n_elem, n_i, Ks, KLs, Ls, mrow, si.c0, si.c1);
            continue;
        }
        if constexpr (KEYED) {
            mask_clean = false;
            if (nrows > 0)
                ok = score_item_keyed(b, kw, kbar, parity, generic, gtab, pp, lane, row_ok, el, n_elem,
                                      nU, n_i, Ks, KLs, Ls, mrow, si.c0, si.c1);
        }
    }
}

// ---------------------------------------------------------------- k_tile

__global__ void k_tile(const int32_t *__restrict__ src, int32_t S, int32_t T, int32_t *__restrict__ dst)
{
    const int TT = (T + 31) >> 5;
    const int64_t n = (int64_t)S * T;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(k / T), c = (int)(k % T);
        dst[m_cell(0, TT, r, c)] = src[k];
    }
}

// ---------------------------------------------------------------- k_align

constexpr int kAW = 8;      // warps per CTA (pipeline depth of a large alignment)
constexpr int kMBuf = 3;    // score tiles in flight per warp

struct AlignSmem {
    int32_t tile[kAW][kMBuf][kTileElems];
    int32_t ring[kAW][kRing];
    unsigned long long bar[kAW][kMBuf];
    int32_t prod[kAW];      // stream values published by warp w (its last rows)
    int32_t cons[kAW];      // stream values warp w consumed from its predecessor
    int32_t item;
};


// One chunk of 32 wavefront steps of a stripe.  At step u lane L is at
// column cidx = 32c + u - L; its score comes from tile c-1 (u < L) or tile c
// (base_prev / base_cur already point at column u = 0 of the lane's row).
// Direction codes are shifted into `word` (two bits per cell, the oldest in
// the low bits; a zero for a step outside the matrix), so after steps 15 and
// 31 every lane holds 16 codes starting at its own column offset; joined with
// the previous 16 (`prev`) by a funnel shift of 2 (L & 15) they give the
// aligned 16-column word 2c - 1 - L/16 (step 15) or 2c - L/16 (step 31) of
// the lane's row, stored when it lies in [mlo, mhi).  Columns [clo, chi)
// are filled.  GUARD = false for chunks in which every lane is inside them
// and every word stored lies in [mlo, mhi).  TILE: the cell values of the
// bottom row go to gbot (lane 31 of a tile's last stripe; null otherwise)
// and those of column chi-1 to *gright (null when no tile follows on the
// right).
template <bool GUARD, bool TILE = false>
__device__ __forceinline__ void stripe_chunk(int c, int lane, int clo, int chi, bool row_ok, int32_t g,
                                             int32_t up_val, const int32_t *base_prev,
                                             const int32_t *base_cur, uint32_t *cr, int mlo, int mhi,
                                             int32_t *ring, int32_t qm, bool publish, int32_t &h_left,
                                             int32_t &up_prev, int32_t &h_out, uint32_t &word,
                                             uint32_t &prev, int32_t *gbot = nullptr,
                                             int32_t *gright = nullptr)
{
    const uint32_t sh = 2u * (uint32_t)(lane & 15);
    const int mb = 2 * c - (lane >> 4);
    // step u is inside [clo, chi) when u + voff, taken unsigned, is below vspan
    const int voff = 32 * c - lane - clo;
    const uint32_t vspan = (row_ok && chi > clo) ? (uint32_t)(chi - clo) : 0u;
#pragma unroll 8
    for (int u = 0; u < 32; ++u) {
        int32_t up_in = __shfl_up_sync(kFull, h_out, 1);
        const int32_t from_above = __shfl_sync(kFull, up_val, u);
        up_in = (lane == 0) ? from_above : up_in;
        const int cidx = 32 * c + u - lane;
        const bool valid = !GUARD || (uint32_t)(u + voff) < vspan;
        uint32_t code = 0u;
        if (valid) {
            const int32_t sv = (u < lane ? base_prev : base_cur)[u];
            const int32_t cd = up_prev + sv;
            const int32_t cu = up_in + g;
            const int32_t cl = h_left + g;
            const int32_t cg = max(cu, cl);
            const int32_t best = max(cd, cg);
            code = cd >= cg ? DIR_DIAG : (cu >= cl ? DIR_UP : DIR_LEFT);
            if (publish) ring[(qm + cidx) & (kRing - 1)] = best;
            if constexpr (TILE) {
                if (gbot) gbot[cidx + 1] = best;
                if (gright && cidx == chi - 1) *gright = best;
            }
            h_left = best;
            h_out = best;
            up_prev = up_in;
        }
        word = __funnelshift_r(word, code, 2);
        if ((u & 15) == 15) {   // the same step for every lane
            const int m = mb - (u == 15 ? 1 : 0);
            if (!GUARD || (row_ok && m >= mlo && m < mhi)) cr[m] = __funnelshift_r(prev, word, sh);
            prev = word;
        }
    }
}

// The last aligned word of a lane's row after its final chunk c (the 16
// codes of `prev` shifted down, zeros above).
__device__ __forceinline__ void stripe_flush(int c, int lane, bool row_ok, uint32_t *cr, int mlo, int mhi,
                                             uint32_t prev)
{
    const int m = 2 * c + 1 - (lane >> 4);
    if (row_ok && m >= mlo && m < mhi) cr[m] = __funnelshift_r(prev, 0u, 2u * (uint32_t)(lane & 15));
}

// H[S][T] of the alignment is the score of its optimal path: the scores of
// the path's diagonal steps (the matches) plus g for each of its
// S + T - 2 nm gap steps.  The selection keeps, per setting sharing the gap,
// the matches whose score passes the threshold.
__device__ __forceinline__ void select_and_emit(const BatchDev &b, const PairPlan &pp,
                                                int gap_idx, const uint32_t *matches,
                                                int nm, int lane)
{
    const int cap = min(pp.S, pp.T);
    const int TT = (pp.T + 31) >> 5;
    // the first 64 matches in increasing-i order (lane and lane + 32), kept
    // in registers for every setting of the gap
    int i0 = 0, j0 = 0, i1 = 0, j1 = 0;
    int32_t s0 = 0, s1 = 0;
    if (lane < nm) {
        const uint32_t ij = matches[nm - 1 - lane];
        i0 = (int)(ij >> 16);
        j0 = (int)(ij & 0xffffu);
        s0 = b.M[m_cell(pp.m_off, TT, i0 - 1, j0 - 1)];
    }
    if (32 + lane < nm) {
        const uint32_t ij = matches[nm - 33 - lane];
        i1 = (int)(ij >> 16);
        j1 = (int)(ij & 0xffffu);
        s1 = b.M[m_cell(pp.m_off, TT, i1 - 1, j1 - 1)];
    }
    int32_t sum = s0 + s1;
    for (int q = 64 + lane; q < nm; q += 32) {
        const uint32_t ij = matches[nm - 1 - q];
        sum += b.M[m_cell(pp.m_off, TT, (int)(ij >> 16) - 1, (int)(ij & 0xffffu) - 1)];
    }
    sum = (int32_t)__reduce_add_sync(kFull, (uint32_t)sum);
    const int32_t H = sum + b.gap_val[gap_idx] * (pp.S + pp.T - 2 * nm);
    // the settings of this gap: set_perm[slist0 + first .. slist0 + last)
    const int lg = gap_idx - pp.gap0;
    const int first = b.gap_sfirst[gap_idx];
    const int last = lg + 1 < pp.ngap ? b.gap_sfirst[gap_idx + 1] : pp.nset;
    for (int f = first; f < last; ++f) {
        const int k = b.set_perm[pp.slist0 + f];
        const int row = pp.set0 + k;
        const int32_t thr = b.set_thr[pp.slist0 + k];
        int32_t *out = b.sel + 3 * (pp.sel_base + (int64_t)k * cap);
        int cnt = 0;
        for (int c = 0; c < nm; c += 32) {
            const int q = c + lane;   // position in increasing-i order
            bool take = false;
            int i = 0, j = 0;
            int32_t sc = 0;
            if (c < 64) {   // (c warp-uniform)
                i = c == 0 ? i0 : i1;
                j = c == 0 ? j0 : j1;
                sc = c == 0 ? s0 : s1;
                take = q < nm && sc > thr;
            } else if (q < nm) {
                const uint32_t ij = matches[nm - 1 - q];
                i = (int)(ij >> 16);
                j = (int)(ij & 0xffffu);
                sc = b.M[m_cell(pp.m_off, TT, i - 1, j - 1)];
                take = sc > thr;
            }
            const uint32_t bal = __ballot_sync(kFull, take);
            if (take) {
                const int pos = cnt + __popc(bal & ((1u << lane) - 1u));
                out[3 * pos + 0] = i - 1;
                out[3 * pos + 1] = j - 1;
                out[3 * pos + 2] = sc;
            }
            cnt += __popc(bal);
        }
        if (lane == 0) {
            b.nw_score[row] = H;
            b.n_sel[row] = cnt;
        }
    }
}

// Traceback from (S,T): blocks of 32 rows x 16 columns of codes held in
// registers, one lane per row; then the selection.
__device__ void trace_and_select(const BatchDev &b, const NwItem &it, const PairPlan &pp, int lane)
{
    const int S = pp.S, T = pp.T;
    const PairBases pb = b.pbases[it.pair];
    uint32_t *matches = b.matches + item_matches(pb.matches, pp, it.gap);
    const uint32_t *codes = b.codes + item_codes(pb.codes, pp, it.gap);
    const int CW = (T + 15) >> 4;
    int i = S, j = T, nm = 0;
    while (i > 0 && j > 0) {
        const int rb = max(1, i - 31);
        const int w = (j - 1) >> 4;
        uint32_t wd = 0;
        if (rb + lane <= i) wd = codes[(int64_t)(rb + lane - 1) * CW + w];
        do {
            const uint32_t word = __shfl_sync(kFull, wd, i - rb);
            const uint32_t dir = (word >> (2 * ((j - 1) & 15))) & 3u;
            if (dir == DIR_DIAG) {
                if (lane == 0) matches[nm] = ((uint32_t)i << 16) | (uint32_t)j;
                ++nm;
                --i;
                --j;
            } else if (dir == DIR_UP) {
                --i;
            } else {
                --j;
            }
        } while (i >= rb && i > 0 && j > 0 && ((j - 1) >> 4) == w);
    }
    __syncwarp();
    select_and_emit(b, pp, it.gap, matches, nm, lane);
}

// Bounded wait until *flag != 0 (a flag another CTA sets); false when the
// wait ran out (error word set).
__device__ __forceinline__ bool flag_wait_set(const int32_t *flag, int32_t *err)
{
    for (uint32_t it = 0; it < kWaitLimit; ++it) {
        if (*(volatile const int32_t *)flag != 0) return true;
        __nanosleep(64);
    }
    atomicCAS(err, 0, ERR_TIMEOUT);
    return false;
}

// One tile (R, C) of a tiled alignment by the whole CTA: warp w fills stripe
// 8R + w over the columns [512C, min(512C + 512, T)), the first stripe takes
// its row above from the tile row above (global), every stripe its column
// on the left from the tile on the left (global) and the stripes pass rows
// to each other through the shared rings as in a whole-CTA alignment.  The
// tile's last row and column go to global memory for the tiles below and to
// the right.  Returns false (on every thread) when a bounded wait ran out.
__device__ bool align_tile(const BatchDev &b, AlignSmem &sm, int wib, int lane, const TileItem &ti,
                           uint32_t (&uses)[kMBuf])
{
    const uint64_t pol = l2_evict_first();   // score tiles are read once
    const NwItem it = b.nw_items[ti.nw];
    const PairPlan pp = b.pairs[it.pair];
    const int S = pp.S, T = pp.T;
    const int R = ti.R, C = ti.C;
    const int NR = (int)tile_rows_of(S), NC = (int)tile_cols_of(T);
    int32_t *hb = b.tbnd + item_tb(b.pbases[it.pair].tb, pp, it.gap);   // rows: (NR-1) x (T+1)
    int32_t *vb = hb + (int64_t)(NR - 1) * (T + 1);                 // columns: (NC-1) x (S+1)
    int32_t *fl = vb + (int64_t)(NC - 1) * (S + 1);                 // flags: NR x NC
    // wait for the tiles above and on the left
    bool ok = true;
    if (threadIdx.x == 0) {
        if (R > 0) ok = flag_wait_set(&fl[(R - 1) * NC + C], b.err);
        if (ok && C > 0) ok = flag_wait_set(&fl[R * NC + C - 1], b.err);
        __threadfence();
    }
    if (threadIdx.x < kAW) {
        sm.prod[threadIdx.x] = 0;
        sm.cons[threadIdx.x] = 0;
    }
    if (!__syncthreads_and(ok)) return false;

    const int32_t g = b.gap_val[it.gap];
    const int TT = (T + 31) >> 5;
    const int TS = (S + 31) >> 5;
    const int CW = (T + 15) >> 4;
    const int clo = kAlignTileCols * C, chi = min(T, clo + kAlignTileCols);
    const int cb = clo >> 5, ce = (chi + 31) >> 5;           // score tiles of the columns
    const int s = (kAlignTileRows / 32) * R + wib;            // this warp's stripe
    if (s < TS) {
        uint32_t *codes = b.codes + item_codes(b.pbases[it.pair].codes, pp, it.gap);
        const int32_t *Mp = b.M + pp.m_off;
        const int mlo = clo >> 4, mhi = (chi + 15) >> 4;   // code words of the tile's columns
        const int i0 = 32 * s;
        const int row = i0 + lane + 1;
        const bool row_ok = row <= S;
        const bool full_stripe = i0 + 32 <= S;
        const bool has_above = wib > 0;                        // in this CTA
        const bool has_below = wib + 1 < kAW && s + 1 < TS;    // in this CTA
        const int32_t qbase = -clo;                            // ring positions relative to clo
        const int pred = wib - 1, succ = wib + 1;
        uint32_t *cr = codes + (int64_t)(row - 1) * CW;
        int32_t *gbot = (wib + 1 == kAW && s + 1 < TS && lane == 31) ? hb + (int64_t)R * (T + 1) : nullptr;
        int32_t *gright = (C + 1 < NC && row_ok) ? vb + (int64_t)C * (S + 1) + row : nullptr;
        __syncwarp();
        if (lane == 0) {
            for (int k = 0; k < kMBuf && cb + k < ce; ++k) {
                mbar_expect_tx(&sm.bar[wib][k], kTileElems * 4);
                bulk_g2s_once(sm.tile[wib][k], Mp + ((int64_t)s * TT + cb + k) * kTileElems, kTileElems * 4,
                         &sm.bar[wib][k], pol);
            }
        }
        for (int k = 0; k < kMBuf && cb + k < ce; ++k) uses[k]++;
        // the column on the left: H[row][clo] and H[row-1][clo]
        const int32_t *vl = C > 0 ? vb + (int64_t)(C - 1) * (S + 1) : nullptr;
        int32_t h_left = vl ? (row_ok ? vl[row] : 0) : row * g;
        int32_t up_prev = vl ? (row - 1 == 0 ? clo * g : (row_ok ? vl[row - 1] : 0)) : (row - 1) * g;
        int32_t h_out = 0;
        uint32_t word = 0, prev = 0;
        const int nchunks = ((chi + 31 + 31) >> 5) - cb;
        const int32_t *hrow = (R > 0 && wib == 0) ? hb + (int64_t)(R - 1) * (T + 1) : nullptr;
        int b_cur = 0;
        for (int cc = 0; cc < nchunks; ++cc) {
            const int c = cb + cc;
            if (c < ce) {
                if (!mbar_wait(&sm.bar[wib][b_cur], (uses[b_cur] - 1) & 1u, b.err)) { ok = false; break; }
            }
            const int b_prev = b_cur == 0 ? kMBuf - 1 : b_cur - 1;
            if (cc >= 2 && c + 1 < ce) {
                const int bb = b_cur == kMBuf - 1 ? 0 : b_cur + 1;
                __syncwarp();
                if (lane == 0) {
                    mbar_expect_tx(&sm.bar[wib][bb], kTileElems * 4);
                    bulk_g2s_once(sm.tile[wib][bb], Mp + ((int64_t)s * TT + c + 1) * kTileElems, kTileElems * 4,
                             &sm.bar[wib][bb], pol);
                }
                uses[bb]++;
            }
            // the row above for columns 32c+1 .. 32c+32 (lane k holds column 32c+1+k)
            const int jcol = 32 * c + 1 + lane;
            int32_t up_val;
            if (has_above) {
                const int32_t need = qbase + min(32 * c + 32, chi);
                if (!flag_wait_ge(&sm.prod[pred], need, b.err)) { ok = false; break; }
                up_val = (jcol > clo && jcol <= chi) ? sm.ring[pred][(qbase + jcol - 1) & (kRing - 1)] : 0;
                __syncwarp();
                if (lane == 0) *(volatile int32_t *)&sm.cons[wib] = need;
            } else if (hrow) {
                up_val = (jcol > clo && jcol <= chi) ? hrow[jcol] : 0;
            } else {
                up_val = jcol * g;
            }
            if (has_below) {
                const int jmax = min(32 * c + 1, chi);
                if (jmax > clo && !flag_wait_ge(&sm.cons[succ], qbase + jmax - kRing, b.err)) { ok = false; break; }
            }
            const int32_t *base_prev = sm.tile[wib][b_prev] + lane * kTile + 32 - lane;
            const int32_t *base_cur = sm.tile[wib][b_cur] + lane * kTile - lane;
            const bool publish = has_below && lane == 31;
            if (full_stripe && cc >= 1 && 32 * (c + 1) <= chi)
                stripe_chunk<false, true>(c, lane, clo, chi, row_ok, g, up_val, base_prev, base_cur, cr, mlo,
                                          mhi, sm.ring[wib], qbase, publish, h_left, up_prev, h_out, word,
                                          prev, gbot, gright);
            else
                stripe_chunk<true, true>(c, lane, clo, chi, row_ok, g, up_val, base_prev, base_cur, cr, mlo,
                                         mhi, sm.ring[wib], qbase, publish, h_left, up_prev, h_out, word,
                                         prev, gbot, gright);
            __syncwarp();
            if (publish) {
                const int jdone = min(32 * c + 1, chi);
                if (jdone > clo) {
                    __threadfence_block();
                    *(volatile int32_t *)&sm.prod[wib] = qbase + jdone;
                }
            }
            b_cur = b_cur == kMBuf - 1 ? 0 : b_cur + 1;
        }
        if (ok) {
            stripe_flush(cb + nchunks - 1, lane, row_ok, cr, mlo, mhi, prev);
            if (s == TS - 1 && row == S && chi == T) b.hfin[ti.nw] = h_left;
        }
        __syncwarp();
    }
    // publish: rows and columns written above, then the flag
    if (!__syncthreads_and(ok)) return false;
    if (threadIdx.x == 0) {
        __threadfence();
        *(volatile int32_t *)&fl[R * NC + C] = 1;
    }
    return true;
}

// Tiled alignments: persistent CTAs take tiles in order of their
// anti-diagonal (a tile's predecessors were taken by running CTAs before it).
__global__ void __launch_bounds__(kAW * 32)
k_align_tiled(BatchDev b)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AlignSmem &sm = *reinterpret_cast<AlignSmem *>(smem_raw);
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    if (lane == 0) {
        for (int k = 0; k < kMBuf; ++k) mbar_init(&sm.bar[wib][k], 1);
        fence_barrier_init();
    }
    uint32_t uses[kMBuf] = {0u, 0u, 0u};
    for (;;) {
        if (__syncthreads_or(*(volatile int32_t *)b.err != 0)) break;
        if (threadIdx.x == 0) sm.item = atomicAdd(&b.counters[7], 1);
        __syncthreads();
        const int t = sm.item;
        if (t >= b.n_tiles) break;
        if (!align_tile(b, sm, wib, lane, b.tiles[t], uses)) break;
    }
}

// Traceback and selection of every alignment, one warp each.
__global__ void __launch_bounds__(128)
k_trace(BatchDev b)
{
    const int lane = threadIdx.x & 31;
    if (*(volatile int32_t *)b.err) return;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(&b.counters[4], 1);
        item = __shfl_sync(kFull, item, 0);
        if (item >= b.n_nw_items) break;
        const NwItem it = b.nw_items[item];
        const PairPlan pp = b.pairs[it.pair];
        if (pp.S == 0 || pp.T == 0) {
            select_and_emit(b, pp, it.gap, nullptr, 0, lane);
            continue;
        }
        trace_and_select(b, it, pp, lane);
    }
}

}  // namespace

// ---------------------------------------------------------------- launchers

int launch_dict_build(const int32_t *keys, const int32_t *trans_off, int32_t n_keys, DevDict d,
                      int32_t *err, cudaStream_t st)
{
    if (n_keys <= 0) return 0;
    const int threads = 256;
    const int blocks = (int)((n_keys + threads - 1) / threads);
    k_dict_build<<<blocks, threads, 0, st>>>(keys, trans_off, n_keys, d, err);
    return 1;
}

int launch_validate(const int32_t *sent_off, int64_t n_sent, int64_t n_tok, int32_t *err,
                    cudaStream_t st)
{
    if (n_sent <= 0) return 0;
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>(4096, (n_sent + threads - 1) / threads);
    k_validate<<<blocks, threads, 0, st>>>(sent_off, n_sent, n_tok, err);
    return 1;
}

int launch_prep(const BatchDev &b, const DevDict &d, int num_sms, cudaStream_t st)
{
    if (b.n_prep_items <= 0) return 0;
    const size_t smem = sizeof(PrepWarpSmem) * kSW;
    cudaFuncSetAttribute(k_prep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int need = (b.n_prep_items + kSW - 1) / kSW;
    const int grid = std::max(1, std::min(num_sms * kScoreCtasPerSm, need));
    k_prep<<<grid, kSW * 32, smem, st>>>(b, d);
    return 1;
}

template <int WARPS, int SLOTS, int CTAS, int MODE>
int launch_pairprep_one(const BatchDev &b, const DevDict &d, int num_sms, cudaStream_t st)
{
    const size_t smem = sizeof(PairPrepSmem<WARPS, SLOTS, MODE == kModeXWide ? kDirectX : kDirect>);
    cudaFuncSetAttribute(k_pairprep<WARPS, SLOTS, CTAS, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    const int grid = std::max(1, std::min(num_sms * CTAS, b.n_pairs));
    k_pairprep<WARPS, SLOTS, CTAS, MODE><<<grid, WARPS * 32, smem, st>>>(b, d);
    return 1;
}

// per-warp global tables (rows of more than 64 tokens): the small-article
// launch takes the first 40 per SM, the wide-article launch, which may run
// beside it, the next 32; the extra-wide launch runs after both
constexpr int kSmallPrepScratchWarps = 8 * 5;
static_assert(kSmallPrepScratchWarps + 16 * 2 <= kGScratchWarpsPerSm, "per-warp global tables");

int launch_pairprep_wide(const BatchDev &b, const DevDict &d, int num_sms, cudaStream_t st)
{
    if (b.n_pairs <= 0) return 0;
    BatchDev bw = b;
    bw.gscratch += (int64_t)num_sms * kSmallPrepScratchWarps * kGTabSlots;
    return launch_pairprep_one<16, 2 * kDirect, 2, kModeWide>(bw, d, num_sms, st);
}

int launch_pairprep(const BatchDev &b, const DevDict &d, int num_sms, cudaStream_t st)
{
    if (b.n_pairs <= 0) return 0;
    return launch_pairprep_one<8, kSmallSlots, 5, kModeSmall>(b, d, num_sms, st);
}

int launch_pairprep_xwide(const BatchDev &b, const DevDict &d, int num_sms, cudaStream_t st)
{
    if (b.n_pairs <= 0) return 0;
    return launch_pairprep_one<16, 2 * kDirectX, 1, kModeXWide>(b, d, num_sms, st);
}

int launch_order(const BatchDev &b, int num_sms, cudaStream_t st)
{
    if (b.n_pairs <= 0) return 0;
    const int grid = std::max(1, std::min(num_sms * 4, (b.n_pairs + 7) / 8));
    k_order<<<grid, 256, 0, st>>>(b);
    return 1;
}

template <int DIRECT, bool KEYED, int W>
int launch_score_one(const BatchDev &b, int num_sms, cudaStream_t st)
{
    const size_t smem = sizeof(ScoreSmem<DIRECT, KEYED, W>);
    static int per_sm = 0;   // resident CTAs per SM of this variant (queried once)
    if (per_sm == 0) {
        cudaFuncSetAttribute(k_score<DIRECT, KEYED, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_score<DIRECT, KEYED, W>, W * 32, smem) !=
                cudaSuccess || n < 1)
            n = 1;
        per_sm = std::min(n, kGScratchWarpsPerSm / W);
    }
    const int grid = std::max(1, std::min(num_sms * per_sm, b.n_score_items));
    k_score<DIRECT, KEYED, W><<<grid, W * 32, smem, st>>>(b);
    return 1;
}

int launch_score(const BatchDev &b, int num_sms, cudaStream_t st)
{
    if (b.n_score_items <= 0) return 0;
    return launch_score_one<kDirectSmall, false, kSWS>(b, num_sms, st);
}

int launch_score_wide(const BatchDev &b, int num_sms, cudaStream_t st)
{
    if (b.n_score_items <= 0) return 0;
    return launch_score_one<kDirect, true, kSWS>(b, num_sms, st);
}

int launch_score_xwide(const BatchDev &b, int num_sms, cudaStream_t st)
{
    if (b.n_score_items <= 0) return 0;
    return launch_score_one<kDirectX, false, kScoreWarpsX>(b, num_sms, st);
}

int launch_align_tiled(const BatchDev &b, int num_sms, cudaStream_t st)
{
    if (b.n_tiles <= 0) return 0;
    const size_t smem = sizeof(AlignSmem);
    cudaFuncSetAttribute(k_align_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int grid = std::max(1, std::min(num_sms * 2, b.n_tiles));
    k_align_tiled<<<grid, kAW * 32, smem, st>>>(b);
    return 1;
}

int launch_trace(const BatchDev &b, int num_sms, cudaStream_t st)
{
    const int n = b.n_nw_items;
    if (n <= 0) return 0;
    const int need = (n + 3) / 4;
    const int grid = std::max(1, std::min(num_sms * 8, need));
    k_trace<<<grid, 128, 0, st>>>(b);
    return 1;
}

// Outputs of a batch in the host call's packed form: row r = p n + k (n
// settings per pair) has its n_sel[r] selected triples at off[r] of `out`,
// off[R] = their total.  Two passes over blocks of 1024 rows: the sums per
// block, then each block's offsets (after the blocks before it) and the copy
// of its rows' triples, one warp per row.  Nothing is done after a device
// error: the counts of a batch whose alignment stopped are not written.
constexpr int kPackBlock = 1024;

__global__ void __launch_bounds__(kPackBlock) k_pack_sums(const int32_t *__restrict__ n_sel, int32_t R,
                                                          int32_t *__restrict__ bsum, const int32_t *err)
{
    __shared__ int part[kPackBlock / 32];
    if (*(volatile const int32_t *)err) return;
    const int r = blockIdx.x * kPackBlock + threadIdx.x;
    const int v = r < R ? n_sel[r] : 0;
    const int w = (int)__reduce_add_sync(kFull, (unsigned)v);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = w;
    __syncthreads();
    if (threadIdx.x < 32) {
        const int t = (int)__reduce_add_sync(kFull, (unsigned)part[threadIdx.x]);
        if (threadIdx.x == 0) bsum[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(kPackBlock) k_pack_place(BatchDev b, int32_t n, int32_t R,
                                                           const int32_t *__restrict__ bsum,
                                                           int64_t *__restrict__ off, int32_t *__restrict__ out)
{
    __shared__ int wsum[32];
    __shared__ int64_t base;
    __shared__ int64_t roff[kPackBlock];
    if (*(volatile const int32_t *)b.err) return;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (w == 0) {
        int64_t before = 0, all = 0;
        const int nblk = (R + kPackBlock - 1) / kPackBlock;
        for (int c = lane; c < nblk; c += 32) {
            const int64_t v = bsum[c];
            all += v;
            if (c < (int)blockIdx.x) before += v;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            before += __shfl_xor_sync(kFull, before, o);
            all += __shfl_xor_sync(kFull, all, o);
        }
        if (lane == 0) {
            base = before;
            if (blockIdx.x == gridDim.x - 1) off[R] = all;
        }
    }
    const int r = blockIdx.x * kPackBlock + tid;
    const int v = r < R ? b.n_sel[r] : 0;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        const int x = wsum[lane];
        int xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, xi, o);
            if (lane >= o) xi += y;
        }
        wsum[lane] = xi - x;
    }
    __syncthreads();
    const int64_t o = base + wsum[w] + incl - v;
    roff[tid] = o;
    if (r < R) off[r] = o;
    __syncthreads();
    // copy the triples of the block's rows, one warp per row
    const int rows = min(kPackBlock, R - (int)blockIdx.x * kPackBlock);
    for (int q = w; q < rows; q += kPackBlock / 32) {
        const int rr = blockIdx.x * kPackBlock + q;
        const int p = rr / n, k = rr - p * n;
        const PairPlan pp = b.pairs[p];
        const int64_t cap = min(pp.S, pp.T);
        const int cnt = b.n_sel[rr];
        const int32_t *src = b.sel + 3 * (pp.sel_base + k * cap);
        int32_t *dst = out + 3 * roff[q];
        for (int e = lane; e < 3 * cnt; e += 32) dst[e] = src[e];
    }
}

int launch_pack(const BatchDev &b, int32_t n, int32_t R, int32_t *bsum, int64_t *off, int32_t *out,
                cudaStream_t st)
{
    if (R <= 0) return 0;
    const int nblk = (R + kPackBlock - 1) / kPackBlock;
    k_pack_sums<<<nblk, kPackBlock, 0, st>>>(b.n_sel, R, bsum, b.err);
    k_pack_place<<<nblk, kPackBlock, 0, st>>>(b, n, R, bsum, off, out);
    return 2;
}

// Random scores in [0, 65536) for timing (a multiplicative hash of the index).
__global__ void k_fill_scores(int32_t *__restrict__ M, int64_t n, uint32_t seed)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        uint32_t x = (uint32_t)k * 0x9E3779B1u ^ seed;
        x ^= x >> 15;
        x *= 0x2C1B3C6Du;
        x ^= x >> 12;
        M[k] = (int32_t)(x & 0xFFFFu);
    }
}

int launch_fill_scores(int32_t *M, int64_t n, uint32_t seed, cudaStream_t st)
{
    if (n <= 0) return 0;
    const int blocks = (int)std::min<int64_t>(4096, (n + 255) / 256);
    k_fill_scores<<<blocks, 256, 0, st>>>(M, n, seed);
    return 1;
}

int launch_tile(const int32_t *src, int32_t S, int32_t T, int32_t *dst, cudaStream_t st)
{
    const int64_t n = (int64_t)S * T;
    if (n <= 0) return 0;
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>(4096, (n + threads - 1) / threads);
    k_tile<<<blocks, threads, 0, st>>>(src, S, T, dst);
    return 1;
}

}  // namespace mine
