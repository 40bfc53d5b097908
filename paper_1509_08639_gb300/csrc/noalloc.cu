// noalloc.cu -- alignment of a caller-supplied score matrix without any
// device allocation.
//
// Some callers cannot allocate device memory at the time they call in: code
// that runs under a memory manager which owns the whole device heap (a
// serving process that reserved its pool up front), code inside a region
// where an allocation would synchronize the device or fail (for example while
// another component holds every byte it may use), or code that must not
// touch the allocator at all for latency reasons.  For them this file keeps
// its scratch in one file-scope static device array, sized for matrices of
// at most kNoAllocMaxDim x kNoAllocMaxDim cells, which every GPU that loads
// the library holds until the process exits.
#include "internal.h"

#include <algorithm>
#include <cstdint>
#include <mutex>

namespace mine {
namespace {

constexpr int kNoAllocMaxDim = 1024;                 // S and T at most
constexpr int64_t kTilesMax = (int64_t)(kNoAllocMaxDim / kTile) * (kNoAllocMaxDim / kTile);

// Scratch layout (int32 words), each region 256-byte aligned.
constexpr int64_t kOffM = 0;                                              // tiled scores
constexpr int64_t kOffMrow = kOffM + kTilesMax * kTileElems;              // row-major copy
constexpr int64_t kOffCodes = kOffMrow + (int64_t)kNoAllocMaxDim * kNoAllocMaxDim;
constexpr int64_t kOffMatch = kOffCodes + (int64_t)kNoAllocMaxDim * (kNoAllocMaxDim / 16);
constexpr int64_t kOffSel = kOffMatch + kNoAllocMaxDim;
constexpr int64_t kOffOut = kOffSel + 3 * kNoAllocMaxDim;                 // nw_score, n_sel, hfin
constexpr int64_t kOffPlan = kOffOut + 64;                                // PairPlan, NwItem, settings, PairBases
constexpr int kPlanBasesAt = 128;                                         // byte offset of PairBases in the plan region
constexpr int64_t kOffCounters = kOffPlan + 64;
constexpr int64_t kScratchWords = kOffCounters + 64;
static_assert(kOffMrow % 64 == 0 && kOffCodes % 64 == 0 && kOffMatch % 64 == 0 &&
                  kOffSel % 64 == 0 && kOffOut % 64 == 0 && kOffPlan % 64 == 0 &&
                  kOffCounters % 64 == 0,
              "scratch regions must stay 256-byte aligned");
static_assert(sizeof(PairPlan) + sizeof(NwItem) + 20 <= kPlanBasesAt && kPlanBasesAt + sizeof(PairBases) <= 64 * 4,
              "plan region too small");

static __device__ __align__(256) int32_t g_noalloc_scratch[kScratchWords];

// The plan of a single pair with a single (gap, threshold) setting, and the
// work-queue counters and error word cleared: the array keeps whatever the
// previous call left there.
__global__ void k_noalloc_setup(int32_t *scratch, int32_t S, int32_t T, int32_t gap, int32_t thr)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    char *plan = reinterpret_cast<char *>(scratch + kOffPlan);
    PairPlan *pp = reinterpret_cast<PairPlan *>(plan);
    NwItem *it = reinterpret_cast<NwItem *>(plan + sizeof(PairPlan));
    int32_t *set = reinterpret_cast<int32_t *>(plan + sizeof(PairPlan) + sizeof(NwItem));
    *reinterpret_cast<PairBases *>(plan + kPlanBasesAt) = PairBases{0, 0, 0};
    pp->s0 = 0;
    pp->S = S;
    pp->t0 = S;
    pp->T = T;
    pp->set0 = 0;
    pp->nset = 1;
    pp->gap0 = 0;
    pp->ngap = 1;
    pp->slist0 = 0;
    pp->pad_ = 0;
    pp->m_off = kOffM;
    pp->sel_base = 0;
    it->pair = 0;
    it->gap = 0;
    set[0] = 0;     // set_gap
    set[1] = thr;   // set_thr
    set[2] = gap;   // gap_val
    set[3] = 0;     // set_perm
    set[4] = 0;     // gap_sfirst
    for (int k = 0; k < 64; ++k) scratch[kOffCounters + k] = 0;
    scratch[kOffOut] = 0;
    scratch[kOffOut + 1] = 0;
    scratch[kOffOut + 2] = 0;
}

struct DeviceScratch {
    int32_t *ptr = nullptr;
    int num_sms = 0;
};

std::mutex g_mu;
DeviceScratch g_dev[64];

int fail_na(int code, const char *msg)
{
    set_last_error(msg);
    return code;
}

// Device address of the static array on the current device (looked up once
// per device: in host code the array's name is only a stand-in).  The
// address is kept for the life of the process, so a device reset
// (cudaDeviceReset) after the first call on that device is not supported.
int scratch_of_current_device(DeviceScratch &out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return fail_na(MINE_ECUDA, "no current CUDA device");
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceScratch &d = g_dev[dev];
    if (!d.ptr) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return fail_na(MINE_ECUDA, cudaGetErrorString(e));
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return fail_na(MINE_ECUDA, cudaGetErrorString(e));
        d.ptr = static_cast<int32_t *>(p);
        d.num_sms = sms;
    }
    out = d;
    return MINE_OK;
}

}  // namespace
}  // namespace mine

using namespace mine;

extern "C" int mine_align_matrix_noalloc(const mine_q16 *M, int32_t S, int32_t T, mine_q16 gap,
                                         mine_q16 threshold, mine_pair *out, int32_t *n_out,
                                         mine_q16 *nw_score, void *stream)
{
    if (!n_out || !nw_score || S < 0 || T < 0 || (S > 0 && T > 0 && !M))
        return fail_na(MINE_EINVAL, "null argument or negative size");
    if (S > kNoAllocMaxDim || T > kNoAllocMaxDim)
        return fail_na(MINE_EINVAL, "S and T must be at most 1024 for the allocation-free alignment");
    if (gap > 0) return fail_na(MINE_EINVAL, "gap must be <= 0");
    if (std::min(S, T) > 0 && !out) return fail_na(MINE_EINVAL, "out is NULL");
    int64_t maxabs = 0;
    for (int64_t k = 0; k < (int64_t)S * T; ++k)
        maxabs = std::max<int64_t>(maxabs, M[k] < 0 ? -(int64_t)M[k] : (int64_t)M[k]);
    if ((int64_t)(S + T) * (-(int64_t)gap) + (int64_t)std::min(S, T) * maxabs >= (int64_t(1) << 31))
        return fail_na(MINE_EOVERFLOW, "(S+T)*|gap| + min(S,T)*max|s| reaches 2^31");
    DeviceScratch ds;
    int rc = scratch_of_current_device(ds);
    if (rc) return rc;
    // a launch error left behind by some earlier, unrelated call must not be
    // taken for one of ours: clear it, then check each launch of this call
    (void)cudaGetLastError();
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int32_t *sc = ds.ptr;
    char *plan = reinterpret_cast<char *>(sc + kOffPlan);
    k_noalloc_setup<<<1, 32, 0, st>>>(sc, S, T, gap, threshold);
    if (cudaGetLastError() != cudaSuccess) return fail_na(MINE_ECUDA, "set-up kernel launch failed");
    if (S > 0 && T > 0) {
        if (cudaMemcpyAsync(sc + kOffMrow, M, 4 * (size_t)S * T, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return fail_na(MINE_ECUDA, "copy of the matrix failed");
        launch_tile(sc + kOffMrow, S, T, sc + kOffM, st);
        if (cudaGetLastError() != cudaSuccess) return fail_na(MINE_ECUDA, "tiling kernel launch failed");
    }
    BatchDev b{};
    b.n_pairs = 1;
    b.pairs = reinterpret_cast<const PairPlan *>(plan);
    b.nw_items = reinterpret_cast<const NwItem *>(plan + sizeof(PairPlan));
    b.pbases = reinterpret_cast<const PairBases *>(plan + kPlanBasesAt);
    b.n_nw_items = 1;
    // the built-in alignment form of the pair (never tiles at these sizes)
    int form = align_kind(nullptr, S, T);
    if (form == AF_TILED) form = AF_WARP8;
    const int g = form_warps(form);
    b.n_nw_grp[g == 8 ? 0 : g == 4 ? 1 : g == 2 ? 2 : 3] = 1;
    const int32_t *set = reinterpret_cast<const int32_t *>(plan + sizeof(PairPlan) + sizeof(NwItem));
    b.set_gap = set;
    b.set_thr = set + 1;
    b.gap_val = set + 2;
    b.set_perm = set + 3;
    b.gap_sfirst = set + 4;
    b.M = sc + kOffM;
    b.codes = reinterpret_cast<uint32_t *>(sc + kOffCodes);
    b.matches = reinterpret_cast<uint32_t *>(sc + kOffMatch);
    b.counters = sc + kOffCounters;
    b.err = b.counters + 8;
    b.nw_score = sc + kOffOut;
    b.n_sel = sc + kOffOut + 1;
    b.sel = sc + kOffSel;
    b.hfin = sc + kOffOut + 2;
    launch_align(b, ds.num_sms, st);
    if (cudaGetLastError() != cudaSuccess) return fail_na(MINE_ECUDA, "alignment kernel launch failed");
    launch_trace(b, ds.num_sms, st);
    if (cudaGetLastError() != cudaSuccess) return fail_na(MINE_ECUDA, "traceback kernel launch failed");
    int32_t head[2] = {0, 0}, derr = 0;
    if (cudaMemcpyAsync(head, sc + kOffOut, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&derr, sc + kOffCounters + 8, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return fail_na(MINE_ECUDA, "alignment failed on the device");
    if (derr) return fail_na(MINE_ETIMEDOUT, "a bounded device wait ran out");
    *nw_score = head[0];
    *n_out = head[1];
    if (head[1] > 0) {
        if (cudaMemcpyAsync(out, sc + kOffSel, 12 * (size_t)head[1], cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return fail_na(MINE_ECUDA, "copy of the selection failed");
    }
    return MINE_OK;
}
