// best_match.cu -- the contrast to the monotone alignment that the paper
// draws in Section 4: Yalign's A* search does not keep its path from going
// upward or leftward in the score matrix, so it can come back to sentences
// it has matched already, and the same phrase can be repeated.  Without the
// path constraint, in the limit, every source sentence takes its
// best-scoring target sentence.
//
//   k_best       one warp per 32 source rows of a pair: each lane scans its
//                row of the score tiles for the highest score (the lowest
//                column among equal ones)
//   k_best_pack  one warp per pair: the rows above the threshold, compacted
//                in row order, and the target sentences taken more than once
#include "internal.h"

#include <algorithm>

namespace mine {
namespace {

constexpr unsigned kAll = 0xffffffffu;

__global__ void __launch_bounds__(256) k_best(BestDev d)
{
    const int lane = threadIdx.x & 31;
    if (*(volatile const int32_t *)d.err) return;   // scores not written
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < d.n_items; w += warps) {
        const ScoreItem si = d.items[w];
        const PairPlan pp = d.pairs[si.pair];
        const int TT = (pp.T + kTile - 1) / kTile;
        const int row = si.row0 + lane;
        int32_t best = 0;
        int bj = -1;
        const int32_t *tile_row = d.M + pp.m_off + (int64_t)(si.row0 >> 5) * TT * kTileElems + lane * kTile;
        for (int c = 0; c < TT; ++c) {
            const int ncol = min(kTile, pp.T - c * kTile);
            const int4 *src = reinterpret_cast<const int4 *>(tile_row + (int64_t)c * kTileElems);
            int32_t v[32];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int4 x = src[q];
                v[4 * q] = x.x;
                v[4 * q + 1] = x.y;
                v[4 * q + 2] = x.z;
                v[4 * q + 3] = x.w;
            }
#pragma unroll
            for (int k = 0; k < 32; ++k)
                if (k < ncol && (bj < 0 || v[k] > best)) {
                    best = v[k];
                    bj = c * kTile + k;
                }
        }
        if (row < pp.S)
            d.best[pp.s0 + row] = (bj >= 0 && best > d.thr) ? make_int2(bj, best) : make_int2(-1, 0);
    }
}

__global__ void __launch_bounds__(256) k_best_pack(BestDev d)
{
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    if (*(volatile const int32_t *)d.err) return;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < d.n_pairs; p += warps) {
        const PairPlan pp = d.pairs[p];
        int cnt = 0;
        unsigned rep = 0;
        for (int r0 = 0; r0 < pp.S; r0 += 32) {
            const int row = r0 + lane;
            const int2 e = row < pp.S ? d.best[pp.s0 + row] : make_int2(-1, 0);
            const bool take = e.x >= 0;
            const uint32_t bal = __ballot_sync(kAll, take);
            if (take) {
                const int64_t pos = pp.s0 + cnt + __popc(bal & lt);
                d.out[3 * pos] = row;
                d.out[3 * pos + 1] = e.x;
                d.out[3 * pos + 2] = e.y;
                // target sentences taken twice or more: a second bitmap
                // records the second time
                const int64_t t = (int64_t)pp.t0 + e.x;
                const uint32_t m = 1u << (t & 31);
                if (atomicOr(&d.seen1[t >> 5], m) & m)
                    if (!(atomicOr(&d.seen2[t >> 5], m) & m)) ++rep;
            }
            cnt += __popc(bal);
        }
        rep = __reduce_add_sync(kAll, rep);
        if (lane == 0) {
            d.n_sel[p] = cnt;
            d.rep[p] = (int32_t)rep;
        }
    }
}

int warps_grid(int64_t warps, int num_sms)
{
    const int64_t blocks = (warps * 32 + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)num_sms * 16));
}

}  // namespace

int launch_best(const BestDev &d, int num_sms, cudaStream_t st)
{
    if (d.n_pairs <= 0) return 0;
    int n = 0;
    if (d.n_items > 0) {
        k_best<<<warps_grid(d.n_items, num_sms), 256, 0, st>>>(d);
        ++n;
    }
    k_best_pack<<<warps_grid(d.n_pairs, num_sms), 256, 0, st>>>(d);
    return n + 1;
}

}  // namespace mine
