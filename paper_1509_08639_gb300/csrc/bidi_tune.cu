// bidi_tune.cu -- the two steps that follow the per-setting selections of a
// batch: the union of the selections mined in both directions (Section 6:
// classifiers trained from either language find additional bi-sentences,
// Table 2 "BI"; Section 7), and the objective by which Threshold and Penalty
// are tuned (Section 4; Table 2 "NWT"): per setting, F1 of the selected pairs
// against known translation pairs, and the best setting.
//
//   k_union    one warp per (pair, setting): merge of the two selections
//   k_f1       one warp per (pair, setting): true positives and counts
//   k_f1_best  one warp: the setting of highest F1
#include "internal.h"

#include <algorithm>

namespace mine {
namespace {

constexpr unsigned kFullMask = 0xffffffffu;

// Key of a selected pair in forward coordinates, (source << 16 | target):
// sentence indices are < 2^16.  A forward entry is (i, j, s); a backward
// entry is (j, i, s) (its source is the forward target article).
__device__ __forceinline__ uint32_t key_fwd(const int32_t *t)
{
    return ((uint32_t)t[0] << 16) | (uint32_t)t[1];
}
__device__ __forceinline__ uint32_t key_bwd(const int32_t *t)
{
    return ((uint32_t)t[1] << 16) | (uint32_t)t[0];
}

// Number of the n entries of list L (triples, keys strictly increasing) whose
// key is below x.
template <bool BWD>
__device__ __forceinline__ int keys_below(const int32_t *L, int n, uint32_t x)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const uint32_t k = BWD ? key_bwd(L + 3 * mid) : key_fwd(L + 3 * mid);
        if (k < x)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// Union of two selections of one (pair, setting).  Along a monotone
// alignment both indices increase, so each list is sorted by its key in
// forward coordinates.  Entry a of the forward list lands at a + (backward
// keys below it) - (keys of both lists below it); a backward entry whose key
// the forward list also holds is dropped, and the forward entry takes the
// larger of the two scores.
__global__ void __launch_bounds__(256) k_union(UnionDev u)
{
    // the selections of a batch whose alignment stopped are not written
    if (*(volatile const int32_t *)u.err_f || *(volatile const int32_t *)u.err_b) return;
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    const int64_t rows = (int64_t)u.n_pairs * u.nset;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < rows; w += warps) {
        const int p = (int)(w / u.nset), k = (int)(w % u.nset);
        const PairPlan pf = u.fwd[p], pb = u.bwd[p];
        const int64_t cap = min(pf.S, pf.T);
        const int32_t *F = u.sel_f + 3 * (pf.sel_base + k * cap);
        const int32_t *B = u.sel_b + 3 * (pb.sel_base + k * cap);
        const int nf = u.nsel_f[pf.set0 + k], nb = u.nsel_b[pb.set0 + k];
        int32_t *O = u.out + 3 * (2 * (pf.sel_base + k * cap));
        int dup_f = 0;
        for (int a0 = 0; a0 < nf; a0 += 32) {
            const int a = a0 + lane;
            bool dup = false;
            int32_t i = 0, j = 0, s = 0;
            int pos = 0;
            if (a < nf) {
                i = F[3 * a];
                j = F[3 * a + 1];
                s = F[3 * a + 2];
                const uint32_t key = ((uint32_t)i << 16) | (uint32_t)j;
                const int lb = keys_below<true>(B, nb, key);
                dup = lb < nb && key_bwd(B + 3 * lb) == key;
                if (dup) s = max(s, B[3 * lb + 2]);
                pos = a + lb;
            }
            const uint32_t bal = __ballot_sync(kFullMask, dup);
            if (a < nf) {
                pos -= dup_f + __popc(bal & lt);
                O[3 * pos] = i;
                O[3 * pos + 1] = j;
                O[3 * pos + 2] = s;
            }
            dup_f += __popc(bal);
        }
        int dup_b = 0;
        for (int c0 = 0; c0 < nb; c0 += 32) {
            const int c = c0 + lane;
            bool dup = false;
            int32_t i = 0, j = 0, s = 0;
            int pos = 0;
            if (c < nb) {
                j = B[3 * c];
                i = B[3 * c + 1];
                s = B[3 * c + 2];
                const uint32_t key = ((uint32_t)i << 16) | (uint32_t)j;
                const int lf = keys_below<false>(F, nf, key);
                dup = lf < nf && key_fwd(F + 3 * lf) == key;
                pos = c + lf;
            }
            const uint32_t bal = __ballot_sync(kFullMask, dup);
            if (c < nb && !dup) {
                pos -= dup_b + __popc(bal & lt);
                O[3 * pos] = i;
                O[3 * pos + 1] = j;
                O[3 * pos + 2] = s;
            }
            dup_b += __popc(bal);
        }
        if (lane == 0) u.n_out[pf.set0 + k] = nf + nb - dup_f;
    }
}

// Per (pair, setting): the selected pairs (i, j) with truth[s0 + i] == j, and
// the selection's size, added into the setting's sums; the warp of setting 0
// also counts the pair's known pairs (source sentences with truth >= 0).
// The sums gather in shared memory first (settings <= kMaxSettings), so each
// block adds each of its sums into global memory once.
constexpr int kMaxSettings = 256;

__global__ void __launch_bounds__(256) k_f1(F1Dev f)
{
    __shared__ unsigned long long acc[2 * kMaxSettings + 1];
    if (*(volatile const int32_t *)f.err) return;   // selections not written
    const int lane = threadIdx.x & 31;
    const int nacc = 2 * f.nset + 1;
    for (int q = threadIdx.x; q < nacc; q += blockDim.x) acc[q] = 0ull;
    __syncthreads();
    const int64_t rows = (int64_t)f.n_pairs * f.nset;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < rows; w += warps) {
        const int p = (int)(w / f.nset), k = (int)(w % f.nset);
        const PairPlan pp = f.pairs[p];
        const int64_t cap = min(pp.S, pp.T);
        const int n = f.n_sel[pp.set0 + k];
        const int32_t *L = f.sel + 3 * (pp.sel_base + k * cap);
        unsigned tp = 0;
        for (int a = lane; a < n; a += 32) tp += f.truth[pp.s0 + L[3 * a]] == L[3 * a + 1] ? 1u : 0u;
        tp = __reduce_add_sync(kFullMask, tp);
        if (lane == 0) {
            atomicAdd(&acc[k], (unsigned long long)tp);
            atomicAdd(&acc[f.nset + k], (unsigned long long)n);
        }
        if (k == 0) {
            unsigned known = 0;
            for (int q = lane; q < pp.S; q += 32) known += f.truth[pp.s0 + q] >= 0 ? 1u : 0u;
            known = __reduce_add_sync(kFullMask, known);
            if (lane == 0) atomicAdd(&acc[2 * f.nset], (unsigned long long)known);
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nacc; q += blockDim.x)
        if (acc[q]) atomicAdd(&f.acc[q], acc[q]);
}

// F1_k = 2 tp_k / (selected_k + known) as the exact fraction (num, den);
// 0/1 when both counts are 0.
struct F1Frac {
    unsigned long long num, den;
    int k;
};

__device__ __forceinline__ bool f1_better(const F1Frac &a, const F1Frac &b)
{
    const unsigned __int128 x = (unsigned __int128)a.num * b.den;
    const unsigned __int128 y = (unsigned __int128)b.num * a.den;
    return x > y || (x == y && a.k < b.k);
}

// One warp: the setting of highest F1, the lowest index among equals.
__global__ void __launch_bounds__(32) k_f1_best(F1Dev f)
{
    if (*(volatile const int32_t *)f.err) return;
    const int lane = threadIdx.x;
    const unsigned long long known = f.acc[2 * f.nset];
    F1Frac best{0ull, 1ull, 1 << 30};
    for (int k = lane; k < f.nset; k += 32) {
        F1Frac c{2ull * f.acc[k], f.acc[f.nset + k] + known, k};
        if (c.den == 0) c = F1Frac{0ull, 1ull, k};
        if (f1_better(c, best)) best = c;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        F1Frac c;
        c.num = __shfl_xor_sync(kFullMask, best.num, o);
        c.den = __shfl_xor_sync(kFullMask, best.den, o);
        c.k = __shfl_xor_sync(kFullMask, best.k, o);
        if (f1_better(c, best)) best = c;
    }
    if (lane == 0) f.best[0] = best.k < f.nset ? best.k : 0;
}

int rows_grid(int64_t rows, int num_sms)
{
    const int64_t blocks = (rows * 32 + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)num_sms * 8));
}

}  // namespace

int launch_union(const UnionDev &u, int num_sms, cudaStream_t st)
{
    const int64_t rows = (int64_t)u.n_pairs * u.nset;
    if (rows <= 0) return 0;
    k_union<<<rows_grid(rows, num_sms), 256, 0, st>>>(u);
    return 1;
}

int launch_f1(const F1Dev &f, int num_sms, cudaStream_t st)
{
    const int64_t rows = (int64_t)f.n_pairs * f.nset;
    int n = 0;
    if (rows > 0) {
        k_f1<<<rows_grid(rows, num_sms), 256, 0, st>>>(f);
        ++n;
    }
    k_f1_best<<<1, 32, 0, st>>>(f);
    return n + 1;
}

}  // namespace mine
