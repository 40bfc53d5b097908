// kernels.cu -- the miner's hot path on sm_103a.
//
// Per article pair (Section 4 of Wolk & Marasek): the sentence-pair score
// matrix M (token overlap through the bilingual dictionary + length, fixed
// point), then a Needleman-Wunsch global alignment over M with gap penalty g
// (monotone paths: "cannot go upward or leftward"), the traceback, and the
// selection of aligned pairs whose score passes the threshold.
//
// Kernels:
//   k_dict_build  one thread per dictionary key -> open-addressed HBM table
//   k_prep        one warp per source sentence: distinct tokens X_i and their
//                 translations grouped per token, flagged FIRST (first copy of
//                 a translation in U_i) and END (last translation of a token)
//   k_score       one warp per 32 source rows of a pair; for each block of up
//                 to 32 target sentences a per-warp shared-memory hash of the
//                 block's target tokens maps token -> 32-bit column mask; each
//                 lane (one source row) probes its elements and accumulates the
//                 overlap counts of all 32 columns at once in bit-sliced
//                 carry-save counters, then scores and stores its 32 cells
//   k_align       one warp per (pair, gap): anti-diagonal wavefront over
//                 stripes of 32 rows (lane = row, the cell above passed by
//                 __shfl_up_sync, the row kept in registers), 2-bit direction
//                 codes packed 16 per word, a warp-cooperative traceback and
//                 the threshold selection of every setting sharing the gap
#include "internal.h"

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

// ceil(2^48 / m) for 1 <= m < 2^16, 0 for m == 0.  For every 0 <= x <= m,
// floor(x * 65536 / m) == (x * K) >> 32: the scaled reciprocal errs by less
// than x / 2^32 <= 1/m, which cannot carry the quotient past an integer.
__device__ __forceinline__ uint64_t recip48(uint32_t m)
{
    return m ? ((1ull << 48) + m - 1) / m : 0ull;
}

__device__ __forceinline__ uint32_t mul_q16(uint32_t x, uint64_t K)
{
    return (uint32_t)(((uint64_t)x * K) >> 32);
}

// ---------------------------------------------------------------- dictionary

__device__ __forceinline__ int2 dict_find(const DevDict &d, int32_t key)
{
    const uint32_t mask = (1u << d.log2) - 1u;
    uint32_t h = hmul(key) >> (32 - d.log2);
    for (;;) {
        int2 e = __ldg(&d.slots[h]);
        if (e.x == key) return make_int2((int32_t)((uint32_t)e.y >> 6), e.y & 63);
        if (e.x == -1) return make_int2(0, 0);
        h = (h + 1) & mask;
    }
}

__global__ void k_dict_build(const int32_t *__restrict__ keys, const int32_t *__restrict__ trans_off,
                             int32_t n_keys, DevDict d, int32_t *err)
{
    const uint32_t mask = (1u << d.log2) - 1u;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_keys;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t key = keys[k];
        const int32_t off = trans_off[k];
        const int32_t cnt = trans_off[k + 1] - off;
        uint32_t h = hmul(key) >> (32 - d.log2);
        for (uint32_t probe = 0; probe <= mask; ++probe) {
            int32_t old = atomicCAS(&d.slots[h].x, -1, key);
            if (old == -1) {
                d.slots[h].y = (int32_t)(((uint32_t)off << 6) | (uint32_t)cnt);
                break;
            }
            if (old == key) {  // duplicate key
                atomicCAS(err, 0, ERR_DUP_KEY);
                break;
            }
            h = (h + 1) & mask;
        }
    }
}

// ---------------------------------------------------------------- shared hash

// Insert key into an open-addressed shared-memory set; true if it was new.
// The caller keeps the load factor <= 1/2, so an empty slot always exists.
__device__ __forceinline__ bool set_insert(int32_t *tab, int log2, int32_t key)
{
    const uint32_t mask = (1u << log2) - 1u;
    uint32_t h = hmul(key) >> (32 - log2);
    for (;;) {
        int32_t old = atomicCAS(&tab[h], -1, key);
        if (old == -1) return true;
        if (old == key) return false;
        h = (h + 1) & mask;
    }
}

__device__ __forceinline__ int slot_of(int32_t *keys, int log2, int32_t key)
{
    const uint32_t mask = (1u << log2) - 1u;
    uint32_t h = hmul(key) >> (32 - log2);
    for (;;) {
        int32_t old = atomicCAS(&keys[h], -1, key);
        if (old == -1 || old == key) return (int)h;
        h = (h + 1) & mask;
    }
}

__device__ __forceinline__ uint32_t probe_occ(const int32_t *keys, const uint32_t *occ, int log2,
                                              int32_t key)
{
    const uint32_t mask = (1u << log2) - 1u;
    uint32_t h = hmul(key) >> (32 - log2);
    for (;;) {
        const int32_t k = keys[h];
        if (k == key) return occ[h];
        if (k == -1) return 0u;
        h = (h + 1) & mask;
    }
}

__device__ __forceinline__ int64_t elem_base(int64_t tok_off, int64_t sent, int32_t kmax)
{
    // 16-byte aligned start with room for L * kmax elements before the next
    // sentence's start (the buffer holds n_tok * kmax + 3 * n_sent + 16 words)
    return (tok_off * kmax + 3 * sent + 3) & ~(int64_t)3;
}

__device__ __forceinline__ int warp_excl_scan(int v, int lane, int *total)
{
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    *total = __shfl_sync(kFull, x, 31);
    return x - v;
}

// ---------------------------------------------------------------- k_prep

struct PrepSmem {
    int32_t tab[kPrepHashSlots];
    int32_t xs[kMaxSentTokens];      // distinct tokens, then packed (off << 6 | cnt)
    int32_t goff[kMaxSentTokens];    // element offset of each token's group
};

constexpr int kPrepWarps = 4;

__global__ void __launch_bounds__(kPrepWarps * 32)
k_prep(BatchDev b, DevDict d)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    PrepSmem &sm = reinterpret_cast<PrepSmem *>(smem_raw)[wib];
    const int kmax = d.kmax;
    if (*(volatile int32_t *)b.err) return;

    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(&b.counters[0], 1);
        item = __shfl_sync(kFull, item, 0);
        if (item >= b.n_score_items) break;
        const ScoreItem si = b.score_items[item];
        const PairPlan pp = b.pairs[si.pair];
        const int rows = min(32, pp.S - si.row0);
        for (int r = 0; r < rows; ++r) {
            const int64_t s = (int64_t)pp.s0 + si.row0 + r;
            const int32_t t_beg = b.sent_off[s];
            const int L = b.sent_off[s + 1] - t_beg;
            // 1. distinct tokens X_i
            const int lg_a = max(6, ceil_log2(2 * L));
            for (int k = lane; k < (1 << lg_a); k += 32) sm.tab[k] = -1;
            __syncwarp();
            int n_i = 0;
            for (int k0 = 0; k0 < L; k0 += 32) {
                const int k = k0 + lane;
                bool is_new = false;
                int32_t tok = 0;
                if (k < L) {
                    tok = b.tokens[t_beg + k];
                    if ((uint32_t)tok > (uint32_t)ELEM_TOKEN) atomicCAS(b.err, 0, ERR_BAD_TOKEN);
                    is_new = set_insert(sm.tab, lg_a, tok);
                }
                const uint32_t bal = __ballot_sync(kFull, is_new);
                if (is_new) sm.xs[n_i + __popc(bal & ((1u << lane) - 1u))] = tok;
                n_i += __popc(bal);
            }
            __syncwarp();
            // 2. dictionary lookups, group offsets
            int n_elem = 0;
            for (int p0 = 0; p0 < n_i; p0 += 32) {
                const int p = p0 + lane;
                int cnt = 0;
                int32_t packed = 0;
                if (p < n_i) {
                    const int2 oc = dict_find(d, sm.xs[p]);
                    cnt = oc.y;
                    packed = (int32_t)(((uint32_t)oc.x << 6) | (uint32_t)oc.y);
                }
                int tot;
                const int off = warp_excl_scan(cnt, lane, &tot);
                if (p < n_i) {
                    sm.xs[p] = packed;
                    sm.goff[p] = n_elem + off;
                }
                n_elem += tot;
            }
            __syncwarp();
            // 3. elements with FIRST / END flags
            uint32_t *out = b.elems + elem_base(t_beg, s, kmax);
            int nU = 0;
            if (n_elem <= kPrepElemCap) {
                const int lg_b = max(6, ceil_log2(2 * n_elem));
                for (int k = lane; k < (1 << lg_b); k += 32) sm.tab[k] = -1;
                __syncwarp();
                int firsts = 0;
                for (int p = lane; p < n_i; p += 32) {
                    const uint32_t pk = (uint32_t)sm.xs[p];
                    const int off = (int)(pk >> 6), cnt = (int)(pk & 63u);
                    const int go = sm.goff[p];
                    for (int k = 0; k < cnt; ++k) {
                        const int32_t u = __ldg(&d.trans[off + k]);
                        const bool first = set_insert(sm.tab, lg_b, u);
                        firsts += first;
                        out[go + k] = (uint32_t)u | (first ? ELEM_FIRST : 0u) |
                                      (k == cnt - 1 ? ELEM_END : 0u);
                    }
                }
                nU = __reduce_add_sync(kFull, firsts);
            } else {
                // rare long element lists: write, then mark first copies by scanning
                for (int p = lane; p < n_i; p += 32) {
                    const uint32_t pk = (uint32_t)sm.xs[p];
                    const int off = (int)(pk >> 6), cnt = (int)(pk & 63u);
                    const int go = sm.goff[p];
                    for (int k = 0; k < cnt; ++k)
                        out[go + k] = (uint32_t)__ldg(&d.trans[off + k]) |
                                      (k == cnt - 1 ? ELEM_END : 0u);
                }
                __syncwarp();
                int firsts = 0;
                for (int e = lane; e < n_elem; e += 32) {
                    const uint32_t u = out[e] & ELEM_TOKEN;
                    bool first = true;
                    for (int q = 0; q < e && first; ++q) first = (out[q] & ELEM_TOKEN) != u;
                    firsts += first;
                    if (first) atomicOr(&out[e], ELEM_FIRST);
                }
                nU = __reduce_add_sync(kFull, firsts);
            }
            if (lane == 0) b.sinfo[s] = make_int4(n_i, n_elem, nU, 0);
            __syncwarp();
        }
    }
}

// ---------------------------------------------------------------- k_score

struct ScoreSmem {
    int32_t keys[kColHashSlots];
    uint32_t occ[kColHashSlots];
    uint64_t Km[32];        // reciprocal of m_j
    uint64_t KL[32];        // reciprocal of L'_j
    int32_t Lt[32];
    int32_t mcnt[32];
    int32_t soff[33];
};

constexpr int kScoreWarps = 4;

__device__ __forceinline__ void csa(uint32_t &carry, uint32_t &sum, uint32_t a, uint32_t b,
                                    uint32_t c)
{
    const uint32_t u = a ^ b;
    carry = (a & b) | (u & c);
    sum = u ^ c;
}

// Add eight 32-lane bit vectors x[0..7] to the bit-sliced counter P (plane k
// holds bit k of 32 counts): carry-save adders for the three low planes, a
// ripple for the rest (Harley-Seal).
template <int NPL>
__device__ __forceinline__ void add8(uint32_t (&P)[NPL], const uint32_t (&x)[8])
{
    uint32_t t1a, t1b, t2a, t2b, t4;
    csa(t1a, P[0], P[0], x[0], x[1]);
    csa(t1b, P[0], P[0], x[2], x[3]);
    csa(t2a, P[1], P[1], t1a, t1b);
    csa(t1a, P[0], P[0], x[4], x[5]);
    csa(t1b, P[0], P[0], x[6], x[7]);
    csa(t2b, P[1], P[1], t1a, t1b);
    csa(t4, P[2], P[2], t2a, t2b);
    uint32_t c = t4;
#pragma unroll
    for (int k = 3; k < NPL; ++k) {
        const uint32_t n = P[k] & c;
        P[k] ^= c;
        c = n;
    }
}

template <int NPL>
__device__ __forceinline__ uint32_t plane_value(const uint32_t (&P)[NPL], int col)
{
    uint32_t v = 0;
#pragma unroll
    for (int k = 0; k < NPL; ++k) v |= ((P[k] >> col) & 1u) << k;
    return v;
}

// One column block: accumulate, score, store.
template <int NPL>
__device__ __forceinline__ void score_block(const ScoreSmem &sm, int lg, const uint32_t *el,
                                            int n_elem, int nE8, int ncols, bool row_ok,
                                            uint64_t Ks, uint64_t KLs, int Ls, int32_t *mrow)
{
    uint32_t A[NPL], B[NPL];
#pragma unroll
    for (int k = 0; k < NPL; ++k) A[k] = B[k] = 0u;
    uint32_t hit = 0;
    for (int e0 = 0; e0 < nE8; e0 += 8) {
        uint32_t xa[8], xb[8];
        uint4 v0 = make_uint4(0, 0, 0, 0), v1 = make_uint4(0, 0, 0, 0);
        if (e0 < n_elem) {
            v0 = *reinterpret_cast<const uint4 *>(el + e0);
            v1 = *reinterpret_cast<const uint4 *>(el + e0 + 4);
        }
        const uint32_t ev[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const bool ok = (e0 + q) < n_elem;
            const uint32_t e = ok ? ev[q] : 0u;
            const uint32_t o = ok ? probe_occ(sm.keys, sm.occ, lg, (int32_t)(e & ELEM_TOKEN)) : 0u;
            xa[q] = (e & ELEM_FIRST) ? o : 0u;
            hit |= o;
            xb[q] = (e & ELEM_END) ? hit : 0u;
            hit = (e & ELEM_END) ? 0u : hit;
        }
        add8<NPL>(A, xa);
        add8<NPL>(B, xb);
    }
    if (!row_ok) return;
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) {
        if (jj < ncols) {
            const uint32_t a = plane_value<NPL>(A, jj);
            const uint32_t bb = plane_value<NPL>(B, jj);
            const uint32_t q_t = mul_q16(a, sm.Km[jj]);
            const uint32_t q_s = mul_q16(bb, Ks);
            const int Lt = sm.Lt[jj];
            uint32_t q_l;
            if (Ls == 0 && Lt == 0) {
                q_l = 65536u;
            } else {
                const uint32_t lmin = (uint32_t)min(Ls, Lt);
                q_l = mul_q16(lmin, Ls >= Lt ? KLs : sm.KL[jj]);
            }
            const uint32_t h = (q_t + q_s) >> 1;
            mrow[jj] = (int32_t)((3u * h + q_l) >> 2);
        }
    }
}

__global__ void __launch_bounds__(kScoreWarps * 32)
k_score(BatchDev b, DevDict d)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    ScoreSmem &sm = reinterpret_cast<ScoreSmem *>(smem_raw)[wib];
    const int kmax = d.kmax;
    if (*(volatile int32_t *)b.err) return;

    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(&b.counters[1], 1);
        item = __shfl_sync(kFull, item, 0);
        if (item >= b.n_score_items) break;
        const ScoreItem si = b.score_items[item];
        const PairPlan pp = b.pairs[si.pair];
        const int S = pp.S, T = pp.T;
        const int Tp = (T + 3) & ~3;
        const int r = si.row0 + lane;
        const bool row_ok = r < S;
        // this lane's source row
        int n_i = 0, n_elem = 0, nU = 0, Ls = 0;
        const uint32_t *el = b.elems;
        if (row_ok) {
            const int64_t s = (int64_t)pp.s0 + r;
            const int4 inf = b.sinfo[s];
            n_i = inf.x;
            n_elem = inf.y;
            nU = inf.z;
            const int32_t tb = b.sent_off[s];
            Ls = b.sent_off[s + 1] - tb;
            el = b.elems + elem_base(tb, s, kmax);
        }
        const uint64_t Ks = recip48((uint32_t)n_i);
        const uint64_t KLs = recip48((uint32_t)Ls);
        const int nE8 = (__reduce_max_sync(kFull, (unsigned)n_elem) + 7) & ~7;
        const int maxU = (int)__reduce_max_sync(kFull, (unsigned)nU);
        const int maxN = (int)__reduce_max_sync(kFull, (unsigned)n_i);
        int32_t *mrow = b.M + pp.m_off + (int64_t)r * Tp;

        for (int c0 = 0; c0 < T; ) {
            // widest block of <= 32 columns whose tokens fit the table
            const int64_t tcol = (int64_t)pp.t0 + c0;
            const int32_t tok0 = b.sent_off[tcol];
            int cum = 0x7fffffff;
            if (c0 + lane < T) cum = b.sent_off[tcol + lane + 1] - tok0;
            const int ncols = __popc(__ballot_sync(kFull, cum <= kColTokCap));
            if (ncols == 0) {  // cannot happen for validated offsets
                if (lane == 0) atomicCAS(b.err, 0, ERR_BAD_OFFSETS);
                break;
            }
            const int ntok = __shfl_sync(kFull, cum, ncols - 1);
            // column offsets (relative to tok0) for the token -> column search
            if (lane < ncols) sm.soff[lane + 1] = cum;
            if (lane == 0) sm.soff[0] = 0;
            const int lg = max(6, ceil_log2(2 * max(ntok, 1)));
            for (int k = lane; k < (1 << lg); k += 32) {
                sm.keys[k] = -1;
                sm.occ[k] = 0u;
            }
            if (lane < 32) sm.mcnt[lane] = 0;
            __syncwarp();
            // build: token -> slot, set the column bit, count distinct per column
            for (int k = lane; k < ntok; k += 32) {
                const int32_t tok = b.tokens[tok0 + k];
                if ((uint32_t)tok > (uint32_t)ELEM_TOKEN) atomicCAS(b.err, 0, ERR_BAD_TOKEN);
                int lo = 0, hi = ncols - 1;   // column: last c with soff[c] <= k
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (sm.soff[mid] <= k) lo = mid; else hi = mid - 1;
                }
                const int slot = slot_of(sm.keys, lg, tok);
                const uint32_t bit = 1u << lo;
                const uint32_t old = atomicOr(&sm.occ[slot], bit);
                if (!(old & bit)) atomicAdd(&sm.mcnt[lo], 1);
            }
            __syncwarp();
            int maxM = 0;
            if (lane < ncols) {
                const int m = sm.mcnt[lane];
                const int Lt = sm.soff[lane + 1] - sm.soff[lane];
                sm.Km[lane] = recip48((uint32_t)m);
                sm.KL[lane] = recip48((uint32_t)Lt);
                sm.Lt[lane] = Lt;
                maxM = m;
            }
            maxM = (int)__reduce_max_sync(kFull, (unsigned)maxM);
            __syncwarp();
            const int bound = max(min(maxU, maxM), maxN);
            int32_t *dst = mrow + c0;
            if (bound < 64) {
                score_block<6>(sm, lg, el, n_elem, nE8, ncols, row_ok, Ks, KLs, Ls, dst);
            } else if (bound < 256) {
                score_block<8>(sm, lg, el, n_elem, nE8, ncols, row_ok, Ks, KLs, Ls, dst);
            } else {
                score_block<11>(sm, lg, el, n_elem, nE8, ncols, row_ok, Ks, KLs, Ls, dst);
            }
            __syncwarp();
            c0 += ncols;
        }
    }
}

// ---------------------------------------------------------------- k_align

constexpr int kAlignWarps = 4;

__device__ __forceinline__ void select_and_emit(const BatchDev &b, const PairPlan &pp,
                                                int gap_idx, int32_t H, const uint32_t *matches,
                                                int nm, int lane)
{
    const int cap = min(pp.S, pp.T);
    const int Tp = (pp.T + 3) & ~3;
    const int32_t *Mp = b.M + pp.m_off;
    for (int k = 0; k < pp.nset; ++k) {
        const int row = pp.set0 + k;
        if (b.set_gap[row] != gap_idx) continue;
        const int32_t thr = b.set_thr[row];
        int32_t *out = b.sel + 3 * (pp.sel_base + (int64_t)k * cap);
        int cnt = 0;
        for (int c = 0; c < nm; c += 32) {
            const int q = c + lane;                   // position in increasing-i order
            bool take = false;
            int i = 0, j = 0;
            int32_t sc = 0;
            if (q < nm) {
                const uint32_t ij = matches[nm - 1 - q];
                i = (int)(ij >> 16);
                j = (int)(ij & 0xffffu);
                sc = Mp[(int64_t)(i - 1) * Tp + (j - 1)];
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

__global__ void __launch_bounds__(kAlignWarps * 32)
k_align(BatchDev b)
{
    const int lane = threadIdx.x & 31;
    if (*(volatile int32_t *)b.err) return;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(&b.counters[2], 1);
        item = __shfl_sync(kFull, item, 0);
        if (item >= b.n_nw_items) break;
        const NwItem it = b.nw_items[item];
        const PairPlan pp = b.pairs[it.pair];
        const int S = pp.S, T = pp.T;
        const int32_t g = b.gap_val[it.gap];
        uint32_t *matches = b.matches + it.match_off;
        if (S == 0 || T == 0) {
            select_and_emit(b, pp, it.gap, (S + T) * g, matches, 0, lane);
            continue;
        }
        const int Tp = (T + 3) & ~3;
        const int CW = (T + 15) >> 4;
        const int32_t *Mp = b.M + pp.m_off;
        uint32_t *codes = b.codes + it.code_off;
        int32_t *hrow = b.hrow + it.hrow_off;
        for (int j = lane; j <= T; j += 32) hrow[j] = j * g;
        __syncwarp();
        int32_t Hfinal = 0;
        for (int i0 = 0; i0 < S; i0 += 32) {
            const int row = i0 + lane + 1;          // 1-based
            const bool row_ok = row <= S;
            const int32_t *mr = Mp + (int64_t)(row - 1) * Tp;
            uint32_t *cr = codes + (int64_t)(row - 1) * CW;
            int32_t h_left = row * g;               // H[row][j-1]
            int32_t up_prev = (row - 1) * g;        // H[row-1][j-1]
            int32_t h_out = 0;                      // value handed to the next lane
            uint32_t word = 0;
            const int nsteps = T + 31;
            int32_t cur_s[8], cur_u[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int j = u - lane + 1;
                const bool ok = row_ok && j >= 1 && j <= T;
                cur_s[u] = ok ? __ldg(mr + j - 1) : 0;
                cur_u[u] = (lane == 0 && j >= 1 && j <= T) ? hrow[j] : 0;
            }
            for (int t0 = 0; t0 < nsteps; t0 += 8) {
                int32_t nxt_s[8], nxt_u[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int j = t0 + 8 + u - lane + 1;
                    const bool ok = row_ok && j >= 1 && j <= T;
                    nxt_s[u] = ok ? __ldg(mr + j - 1) : 0;
                    nxt_u[u] = (lane == 0 && j >= 1 && j <= T) ? hrow[j] : 0;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int t = t0 + u;
                    const int j = t - lane + 1;
                    int32_t up_in = __shfl_up_sync(kFull, h_out, 1);
                    if (lane == 0) up_in = cur_u[u];
                    if (t < nsteps && row_ok && j >= 1 && j <= T) {
                        const int32_t cd = up_prev + cur_s[u];
                        const int32_t cu = up_in + g;
                        const int32_t cl = h_left + g;
                        const bool upw = cu >= cl;
                        const int32_t cg = upw ? cu : cl;
                        const bool dg = cd >= cg;
                        const int32_t best = dg ? cd : cg;
                        const uint32_t dir = dg ? DIR_DIAG : (upw ? DIR_UP : DIR_LEFT);
                        word |= dir << (2 * ((j - 1) & 15));
                        if (((j - 1) & 15) == 15 || j == T) {
                            cr[(j - 1) >> 4] = word;
                            word = 0;
                        }
                        if (lane == 31) hrow[j] = best;
                        h_left = best;
                        h_out = best;
                        up_prev = up_in;
                    }
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    cur_s[u] = nxt_s[u];
                    cur_u[u] = nxt_u[u];
                }
            }
            const int last_lane = (S - 1 - i0) < 32 ? (S - 1 - i0) : 31;
            Hfinal = __shfl_sync(kFull, h_left, last_lane);
            __syncwarp();
        }
        // traceback: walk blocks of 32 rows x 16 columns of codes held in registers
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
        select_and_emit(b, pp, it.gap, Hfinal, matches, nm, lane);
    }
}

// ---------------------------------------------------------------- validation

// Sentence offsets must start at 0, never decrease, end at n_tok and give at
// most MINE_MAX_SENT_TOKENS tokens per sentence; later kernels trust them.
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

// ---------------------------------------------------------------- compaction

__global__ void k_compact(const int32_t *__restrict__ src, const int64_t *__restrict__ src_off,
                          const int64_t *__restrict__ dst_off, const int32_t *__restrict__ counts,
                          int32_t n_rows, int32_t *__restrict__ dst)
{
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int r = warp; r < n_rows; r += nwarps) {
        const int64_t n = 3 * (int64_t)counts[r];
        const int32_t *s = src + 3 * src_off[r];
        int32_t *d = dst + 3 * dst_off[r];
        for (int64_t k = lane; k < n; k += 32) d[k] = s[k];
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

static int grid_for(int num_sms, int per_sm, int items, int warps_per_cta)
{
    const int need = (items + warps_per_cta - 1) / warps_per_cta;
    return max(1, min(num_sms * per_sm, need));
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
    if (b.n_score_items <= 0) return 0;
    const size_t smem = sizeof(PrepSmem) * kPrepWarps;
    cudaFuncSetAttribute(k_prep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_prep<<<grid_for(num_sms, 2, b.n_score_items, kPrepWarps), kPrepWarps * 32, smem, st>>>(b, d);
    return 1;
}

int launch_score(const BatchDev &b, const DevDict &d, int num_sms, cudaStream_t st)
{
    if (b.n_score_items <= 0) return 0;
    const size_t smem = sizeof(ScoreSmem) * kScoreWarps;
    cudaFuncSetAttribute(k_score, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_score<<<grid_for(num_sms, 3, b.n_score_items, kScoreWarps), kScoreWarps * 32, smem, st>>>(b, d);
    return 1;
}

int launch_align(const BatchDev &b, int num_sms, cudaStream_t st)
{
    if (b.n_nw_items <= 0) return 0;
    k_align<<<grid_for(num_sms, 8, b.n_nw_items, kAlignWarps), kAlignWarps * 32, 0, st>>>(b);
    return 1;
}

int launch_compact(const int32_t *src, const int64_t *src_off, const int64_t *dst_off,
                   const int32_t *counts, int32_t n_rows, int32_t *dst, cudaStream_t st)
{
    if (n_rows <= 0) return 0;
    const int threads = 256;
    const int blocks = min(4096, (n_rows * 32 + threads - 1) / threads);
    k_compact<<<blocks, threads, 0, st>>>(src, src_off, dst_off, counts, n_rows, dst);
    return 1;
}

}  // namespace mine
