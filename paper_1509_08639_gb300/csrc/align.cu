// align.cu -- the Needleman-Wunsch fill of the miner (Section 4 of Wolk &
// Marasek: global alignment of the sentence-pair score matrix M with the
// Penalty as gap cost; a path never moves upward or leftward).
//
//   H[0][0] = 0, H[i][0] = i g, H[0][j] = j g,
//   H[i][j] = max(H[i-1][j-1] + s(i,j), H[i-1][j] + g, H[i][j-1] + g),
//   direction DIAG if the diagonal attains the maximum, else UP if the cell
//   above does, else LEFT; 2-bit codes, 16 per word, row-major per alignment.
//
// Wavefront.  One lane per row, 32 rows (a stripe) per warp; lane L is L
// steps behind lane 0, so at every step each lane holds the cell above its
// next one in lane L-1 (one shuffle).  A warp runs on from one of its stripes
// into the next without draining: lane L's virtual column v = t - L walks
// stripe after stripe (each T' = T rounded up to 32 columns wide), and lane 0
// takes the row above a stripe from lane 31 of the stripe before it through
// a ring in shared memory that lane 31 both writes (its own row) and reads
// (the value lane 0 needs at the next step), handing it over in the same
// rotation shuffle: the lane-0 boundary costs one store, one load and one
// select per step, and no warp-level synchronisation (one thread owns the
// ring).  A pipeline of G warps shares a pair: warp w takes stripes w, w+G,
// ... and reads the ring of warp w-1 (bounded flag waits once per 32 steps).
//
// Scores.  The 32 x 32 tiles of M come in by one 4 KB bulk copy each, one
// tile ahead, three slots per warp; in a chunk of 32 steps lane L reads the
// tile before for its first L steps and the current one after (the skew puts
// the 32 lanes' reads in distinct banks).
//
// Per step a lane issues the shuffle, the score load, three integer
// operations for the cell (add; max of up and left with the up-wins flag;
// fused add-then-max), the code select and shift, and the lane-31 ring
// store, load and select.
#include "async_copy.cuh"
#include "internal.h"

#include <algorithm>
#include <climits>

namespace mine {
namespace {

constexpr uint32_t kFullMaskA = 0xffffffffu;
constexpr int kNwWarps = kNwPipe;    // warps per CTA (two CTAs per SM)
constexpr int kNwSlots = 3;          // score tiles resident per warp (two read, one in flight)
constexpr int kNwRing = 512;         // boundary ring entries per warp

template <int K>
struct NwSmem {
    int32_t tile[K][kNwSlots][kTileElems];   // 32 x 32 score tiles, row-major
    int32_t ring[K][kNwRing];
    unsigned long long bar[K][kNwSlots];
    int32_t prod[K];                 // keys published by warp w's lane 31 (INT_MAX: done)
    int32_t cons[K];                 // keys warp w has read from its predecessor (INT_MAX: done)
    int32_t gitem[kNwGroups][K];     // the item a group (at its first warp) took, per run
};

// Where lane 0's up value comes from in a chunk of 32 steps: the ring (the
// chunk's 32 values read at its start, one per lane, and shuffled to lane 0
// step by step), H[0][j] of the pair's first stripe, or -- stripes one tile
// wide -- lane 31's value of the step before, which is exactly the row above.
enum XSrc { X_RING = 0, X_ARITH = 1, X_ROT = 2 };

// 32 wavefront steps.  Lane L's score at step u is bp[u] (u < L: the tile
// before, at column 32 - L + u of its row) or bc[u] (u >= L: column u - L of
// the current tile); the skew keeps the 32 lanes' reads in distinct banks.  rw:
// lane 31 writes its value of step u to rw[u] (the ring read by the next
// stripe's lane 0).  rv: lane k holds lane 0's up value of step k (X_RING).
// xa: H[0][j] of lane 0's cell at u = 0 (X_ARITH; + u g at step u).  RESET:
// lanes start a stripe at step u = lane (h = row g, the diagonal (row - 1) g).
// a1 / a2: where the aligned code words completed at steps 15 and 31 go
// (null: not stored).
template <bool RESET, int XS>
__device__ __forceinline__ void nw_chunk(const int32_t *__restrict__ bp, const int32_t *__restrict__ bc,
                                         int32_t *__restrict__ rw, int32_t rv,
                                         int lane, int src, int32_t g, int32_t rh, int32_t xa,
                                         uint32_t sh, uint32_t *__restrict__ a1, uint32_t *__restrict__ a2, int32_t &h,
                                         int32_t &up_prev, uint32_t &word, uint32_t &prev)
{
#pragma unroll
    for (int u = 0; u < 32; ++u) {
        const int32_t rot = __shfl_sync(kFullMaskA, h, src);   // the cell above, from lane - 1
        int32_t up_in;
        if (XS == X_ROT) {
            up_in = rot;
        } else {
            const int32_t l0 = XS == X_ARITH ? xa + u * g : __shfl_sync(kFullMaskA, rv, u);
            up_in = lane == 0 ? l0 : rot;
        }
        if (RESET && u == lane) {
            h = rh;
            up_prev = rh - g;
        }
        const int32_t sv = (u < lane ? bp : bc)[u];
        const int32_t cd = up_prev + sv;
        // the diagonal and the left cell do not wait for the shuffle: one
        // fused add-then-max after it
        const int32_t dl = __viaddmax_s32(h, g, cd);          // max(left + g, diag + s)
        const int32_t best = __viaddmax_s32(up_in, g, dl);    // max(up + g, that)
        const uint32_t code = best == cd ? DIR_DIAG : (up_in >= h ? DIR_UP : DIR_LEFT);
        word = __funnelshift_r(word, code, 2);
        h = best;
        up_prev = up_in;
        if (XS != X_ROT && lane == 31) rw[u] = best;
        if (u == 15) {
            if (a1) *a1 = __funnelshift_r(prev, word, sh);
            prev = word;
        } else if (u == 31) {
            if (a2) *a2 = __funnelshift_r(prev, word, sh);
            prev = word;
        }
    }
}

// Wait (bounded) until every tile copy this warp has in flight has landed,
// so that the CTA may end after an error.
// tiles: the number of tiles this warp has issued so far; the j-th tile it
// issued went into slot j % 3 and completes that slot's phase j / 3.
template <int K>
__device__ void nw_drain(NwSmem<K> &sm, int w, uint32_t tiles, int32_t *err)
{
    for (uint32_t j = tiles > kNwSlots ? tiles - kNwSlots : 0; j < tiles; ++j)
        mbar_wait(&sm.bar[w][j % kNwSlots], (j / kNwSlots) & 1u, err);
}

// Fill H for one alignment by warp wg of a pipeline of G warps (w = its
// warp in the CTA; the pipeline is warps w - wg .. w - wg + G - 1).  Returns
// false when a bounded wait ran out (error word set).
template <int K>
__device__ bool nw_run(const BatchDev &b, NwSmem<K> &sm, int w, int wg, int G, int lane, const NwItem &it,
                       const PairPlan &pp, uint32_t &tiles, uint64_t pol)
{
    const int S = pp.S, T = pp.T;
    const int TT = (T + 31) >> 5;           // column tiles; stripes are Tp = 32 TT wide
    const int Tp = TT << 5;
    const int NS = (S + 31) >> 5;           // stripes of the pair
    const bool self = G == 1;
    int32_t *prod_mine = &sm.prod[w];
    int32_t *cons_mine = &sm.cons[w];
    if (wg >= NS) {   // nothing for this warp: its partners must not wait on it
        if (lane == 0) {
            *(volatile int32_t *)prod_mine = INT_MAX;
            *(volatile int32_t *)cons_mine = INT_MAX;
        }
        __syncwarp();
        return true;
    }
    const int nq = (NS - wg + G - 1) / G;   // stripes of this warp: wg, wg + G, ...
    const int32_t g = b.gap_val[it.gap];
    const int CW = (T + 15) >> 4;
    uint32_t *codes = b.codes + item_codes(b.pbases[it.pair].codes, pp, it.gap);
    const int32_t *Mp = b.M + pp.m_off;
    const int base_w = w - wg;
    const int pw = self ? w : base_w + (wg == 0 ? G - 1 : wg - 1);
    const int sw = self ? w : base_w + (wg == G - 1 ? 0 : wg + 1);
    int32_t *ring_out = sm.ring[w];
    const int32_t *ring_in = sm.ring[pw];
    const int32_t *prod_pred = &sm.prod[pw];
    const int32_t *cons_succ = &sm.cons[sw];
    // the consumer's key of a value lane 31 writes at virtual column v is
    // v + off_out (the next stripe of the same warp, or warp 0's next one)
    const int32_t off_out = (self || wg == G - 1) ? Tp : 0;
    // keys the successor reads from this warp's ring: all of its stripes'
    // keys, except that warp 0 takes its first stripe's from row 0
    const int nq_succ = wg == G - 1 ? (NS + G - 1) / G : (NS - wg - 1 + G - 1) / G;
    const int32_t succ_first = wg == G - 1 ? Tp : 0;
    const int32_t succ_last = nq_succ * Tp - 1;
    const int src = (lane + 31) & 31;
    // testing the bounded waits: the first warp of a pipeline keeps its rows
    // to itself, so the next warp's wait runs out
    const bool publish = !(b.test_withhold && !self && wg == 0);
    const uint32_t sh = 2u * (uint32_t)(lane & 15);
    const int ntile = nq * TT;              // virtual tiles of this warp
    const int nchunks = ntile + 1;

    // virtual tile k of this warp (the warp's tile t0 + k) into slot
    // (t0 + k) % 3: one bulk copy of the tile's rows inside the pair (4 KB
    // but in the last stripe; the lanes past the last row read stale rows,
    // and rows never feed the rows above them)
    const uint32_t t0 = tiles;
    auto issue = [&](int k) {
        const int q = k / TT;
        const int C = k - q * TT;
        const int s = wg + q * G;
        const int slot = (int)((t0 + k) % kNwSlots);
        const uint32_t bytes = (uint32_t)min(kTile, pp.S - kTile * s) * (kTile * 4);
        __syncwarp();
        if (lane == 0) {
            mbar_expect_tx(&sm.bar[w][slot], bytes);
            bulk_g2s_once(sm.tile[w][slot], Mp + ((int64_t)s * TT + C) * kTileElems, bytes, &sm.bar[w][slot],
                          pol);
        }
        tiles = t0 + k + 1;
    };

    int32_t h = 0, up_prev = 0;
    uint32_t word = 0, prev = 0;
    issue(0);
    for (int c = 0; c < nchunks; ++c) {
        if (c + 1 < ntile) issue(c + 1);
        const uint32_t tc = t0 + c;                   // the warp's tile of this chunk
        if (c < ntile && !mbar_wait(&sm.bar[w][tc % kNwSlots], (tc / kNwSlots) & 1u, b.err)) return false;
        const int q = c / TT;                      // stripe (of this warp) lane 0 is in
        const int r = c - q * TT;
        const bool reset = r == 0 && q < nq;
        // lane 0's up values of this chunk: keys 32c .. 32c + 31
        int xs = X_RING;
        if (wg == 0 && c < TT) xs = X_ARITH;       // the pair's first stripe: H[0][j]
        else if (Tp == 32) xs = X_ROT;            // (one warp) lane 31's previous value
        if (c == ntile) xs = X_ARITH;              // lane 0 is past its last stripe
        if (!self) {
            if (xs == X_RING && !flag_wait_ge(prod_pred, 32 * c + 31, b.err, b.wait_spins)) return false;
            // lane 31 overwrites keys need - 31 .. need in this chunk: wait
            // until the successor has read those of them it reads at all
            const int32_t need = 32 * c + off_out - kNwRing;
            if (succ_first <= succ_last && need >= succ_first && need - 31 <= succ_last &&
                !flag_wait_ge(cons_succ, min(need, succ_last), b.err, b.wait_spins))
                return false;
            __threadfence_block();
        } else {
            __syncwarp();   // lane 31's ring stores of earlier chunks, read by every lane below
        }
        // lane k: key 32c + k, stored at slot key - 1
        const int32_t rv = xs == X_RING ? ring_in[(32 * c + lane - 1) & (kNwRing - 1)] : 0;
        const int32_t *bp = sm.tile[w][(tc + kNwSlots - 1) % kNwSlots] + lane * kTile + 32 - lane;
        const int32_t *bc = sm.tile[w][tc % kNwSlots] + lane * kTile - lane;
        int32_t *rw = ring_out + ((32 * c - 32 + off_out) & (kNwRing - 1));
        const int32_t xa = (32 * c + 1) * g;
        // the new stripe of a reset chunk, for the row of each lane
        const int32_t rh = (int32_t)(32 * (wg + q * G) + lane + 1) * g;
        // aligned code words completed at steps 15 and 31
        uint32_t *a1 = nullptr, *a2 = nullptr;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int m = 2 * c - 1 + e - (lane >> 4);
            uint32_t *ad = nullptr;
            const int qm = m < 2 * TT * q ? q - 1 : q;
            const int wi = m - 2 * TT * qm;
            const int row = 32 * (wg + qm * G) + lane + 1;
            if (m >= 0 && qm < nq && wi < CW && row <= S) ad = codes + (int64_t)(row - 1) * CW + wi;
            if (e == 0) a1 = ad;
            else a2 = ad;
        }
        if (reset) {
            if (xs == X_RING)
                nw_chunk<true, X_RING>(bp, bc, rw, rv, lane, src, g, rh, xa, sh, a1, a2, h, up_prev, word, prev);
            else if (xs == X_ARITH)
                nw_chunk<true, X_ARITH>(bp, bc, rw, rv, lane, src, g, rh, xa, sh, a1, a2, h, up_prev, word, prev);
            else
                nw_chunk<true, X_ROT>(bp, bc, rw, rv, lane, src, g, rh, xa, sh, a1, a2, h, up_prev, word, prev);
        } else {
            if (xs == X_RING)
                nw_chunk<false, X_RING>(bp, bc, rw, rv, lane, src, g, rh, xa, sh, a1, a2, h, up_prev, word, prev);
            else if (xs == X_ARITH)
                nw_chunk<false, X_ARITH>(bp, bc, rw, rv, lane, src, g, rh, xa, sh, a1, a2, h, up_prev, word, prev);
            else
                nw_chunk<false, X_ROT>(bp, bc, rw, rv, lane, src, g, rh, xa, sh, a1, a2, h, up_prev, word, prev);
        }
        if (!self) {
            __syncwarp();
            if (lane == 31) {
                __threadfence_block();
                if (publish) *(volatile int32_t *)prod_mine = 32 * c + off_out;
                *(volatile int32_t *)cons_mine = 32 * c + 31;
            }
        }
    }
    if (!self) {
        __syncwarp();
        if (lane == 31) {
            __threadfence_block();
            if (publish) *(volatile int32_t *)prod_mine = INT_MAX;
            *(volatile int32_t *)cons_mine = INT_MAX;
        }
    }
    __syncwarp();
    return true;
}

// Named barrier of a pipeline group: id 1 for the whole CTA (8 warps), 2-3
// for groups of 4, 4-7 for groups of 2.
__device__ __forceinline__ void group_sync(int G, int base_w)
{
    if (G == 1) {
        __syncwarp();
    } else {
        const int id = (kNwPipe / G) + base_w / G;
        asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(G * 32) : "memory");
    }
}

// Persistent alignment kernel.  The items come in four runs: pairs aligned
// by pipelines of 8, 4 and 2 warps, then one warp per pair.  The CTA first
// works as one group of 8 warps on the first run; a group whose run is empty
// splits in two and each half takes the next run, without waiting for the
// other groups.  Tracebacks follow in k_trace.
template <int K>
__global__ void __launch_bounds__(K * 32, 2) k_nw(BatchDev b)
{
    static_assert(K == kNwPipe, "groups of 8, 4, 2, 1 warps");
    extern __shared__ __align__(128) unsigned char nw_smem_raw[];
    NwSmem<K> &sm = *reinterpret_cast<NwSmem<K> *>(nw_smem_raw);
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    if (lane == 0) {
        for (int k = 0; k < kNwSlots; ++k) mbar_init(&sm.bar[w][k], 1);
        fence_barrier_init();
    }
    uint32_t tiles = 0;                       // tiles this warp has issued
    const uint64_t pol = l2_evict_first();   // score tiles are read once per gap
    __syncthreads();
    if (*(volatile int32_t *)b.err) return;

    int beg = 0;
    for (int gi = 0; gi < kNwGroups; ++gi) {
        const int G = K >> gi;
        const int end = beg + b.n_nw_grp[gi];
        const int base_w = w - w % G, wg = w - base_w;
        while (beg < end) {
            // the group's first warp takes the next item of the run
            if (wg == 0 && lane == 0) sm.gitem[gi][base_w] = atomicAdd(&b.counters[ctr_nw(gi)], 1);
            if (lane == 0) {
                sm.prod[w] = -1;   // keys <= -1 published / consumed: none
                sm.cons[w] = -1;
            }
            group_sync(G, base_w);
            const int item = beg + *(volatile int32_t *)&sm.gitem[gi][base_w];
            if (item >= end) break;
            const NwItem it = b.nw_items[item];
            const PairPlan pp = b.pairs[it.pair];
            // warp 0 of a pipeline of Ge warps needs the row above its second
            // stripe from warp Ge - 1 before it has filled Ge of its own
            // chunks: Ge < T'/32 keeps that dependency acyclic
            const int Ge = min(min(G, (pp.S + 31) >> 5), max(1, ((pp.T + 31) >> 5) - 1));
            bool ok = true;
            if (pp.S > 0 && pp.T > 0 && wg < Ge) ok = nw_run<K>(b, sm, w, wg, Ge, lane, it, pp, tiles, pol);
            if (!ok) atomicCAS(b.err, 0, ERR_TIMEOUT);
            group_sync(G, base_w);
            if (*(volatile int32_t *)b.err) {
                nw_drain<K>(sm, w, tiles, b.err);
                return;
            }
        }
        beg = end;
    }
}

}  // namespace

int launch_align(const BatchDev &b, int num_sms, cudaStream_t st)
{
    const int items = b.n_nw_items - b.n_nw_tiled;
    if (items <= 0) return 0;
    const size_t smem = sizeof(NwSmem<kNwWarps>);
    cudaFuncSetAttribute(k_nw<kNwWarps>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    // CTAs that have work in the first run they can take part in
    int need = 0;
    for (int gi = 0; gi < kNwGroups; ++gi) {
        const int per_cta = 1 << gi;   // groups of 8 >> gi warps per CTA
        need = std::max(need, (b.n_nw_grp[gi] + per_cta - 1) / per_cta);
    }
    const int grid = std::max(1, std::min(2 * num_sms, need));
    k_nw<kNwWarps><<<grid, kNwWarps * 32, smem, st>>>(b);
    return 1;
}

}  // namespace mine
