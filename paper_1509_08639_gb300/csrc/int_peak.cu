// int_peak.cu -- on-device measurement of the integer add/max throughput that
// bounds the alignment kernels.
//
// The Needleman-Wunsch fill costs four essential int32 operations per cell
// (the diagonal add, the gap add, two maxima); its roofline is the rate at
// which the SMs can execute such operations.  No vendor figure states that
// rate for this part, so it is measured: every thread of a full grid runs
// many independent chains of the same add/max pattern, timed with CUDA
// events, and the operations written in the source are counted (an add and a
// max count as two, whether the compiler issues them as two instructions or
// as one fused add-then-max).  Three forms are timed and the fastest is the
// peak:
//   0  x = max(x + g, y), y = max(y + g, x)          (plain C; the compiler's choice)
//   1  the same through the add-then-max intrinsic   (__viaddmax_s32)
//   2  x = max(x, y) + g, y = max(y, x) + g          (max first, then add)
#include "internal.h"

#include <algorithm>

namespace mine {
namespace {

constexpr int kChains = 8;          // independent chains per thread
constexpr int kPeakThreads = 256;   // threads per block

template <int FORM>
__global__ void __launch_bounds__(kPeakThreads) k_int_peak(int32_t *out, int iters, int32_t g)
{
    int32_t x[kChains], y[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
        x[k] = (int32_t)(threadIdx.x * 7 + k);
        y[k] = (int32_t)(blockIdx.x * 3 - k);
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) {
                if constexpr (FORM == 0) {
                    x[k] = max(x[k] + g, y[k]);
                    y[k] = max(y[k] + g, x[k]);
                } else if constexpr (FORM == 1) {
                    x[k] = __viaddmax_s32(x[k], g, y[k]);
                    y[k] = __viaddmax_s32(y[k], g, x[k]);
                } else {
                    x[k] = max(x[k], y[k]) + g;
                    y[k] = max(y[k], x[k]) + g;
                }
            }
        }
    }
    int32_t acc = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc ^= x[k] ^ y[k];
    if (acc == 0x7fffffff) out[blockIdx.x * blockDim.x + threadIdx.x] = acc;   // keeps the chains live
}

// int32 operations one launch executes: per thread and iteration,
// 4 unrolled rounds x kChains chains x 2 statements x (1 add + 1 max).
double ops_of(int blocks, int iters)
{
    return (double)blocks * kPeakThreads * iters * 4.0 * kChains * 4.0;
}

}  // namespace
}  // namespace mine

using namespace mine;

extern "C" int mine_int_peak(int32_t device, double *ops_per_s, double *per_form, int32_t n_form)
{
    if (!ops_per_s) {
        set_last_error("ops_per_s is NULL");
        return MINE_EINVAL;
    }
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess) {
        set_last_error("no CUDA device");
        return MINE_ECUDA;
    }
    if (device >= 0 && cudaSetDevice(device) != cudaSuccess) {
        set_last_error("cudaSetDevice failed");
        return MINE_ECUDA;
    }
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device >= 0 ? device : prev);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, device >= 0 ? device : prev);
    const int blocks = std::max(1, sms * std::max(1, per_sm / kPeakThreads));
    const int iters = 128;   // about 0.1-0.3 s per launch
    int32_t *out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = MINE_OK;
    double best = 0.0;
    if (cudaMalloc(&out, sizeof(int32_t) * (size_t)blocks * kPeakThreads) != cudaSuccess ||
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        set_last_error("allocation of the measurement's buffers failed");
        rc = MINE_ECUDA;
    }
    for (int form = 0; form < 3 && rc == MINE_OK; ++form) {
        float ms_best = 1e30f;
        for (int rep = 0; rep < 4 && rc == MINE_OK; ++rep) {   // the first is a warm-up
            cudaEventRecord(e0, st);
            if (form == 0) k_int_peak<0><<<blocks, kPeakThreads, 0, st>>>(out, iters, -3);
            if (form == 1) k_int_peak<1><<<blocks, kPeakThreads, 0, st>>>(out, iters, -3);
            if (form == 2) k_int_peak<2><<<blocks, kPeakThreads, 0, st>>>(out, iters, -3);
            cudaEventRecord(e1, st);
            float ms = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                set_last_error("timing of the measurement kernel failed");
                rc = MINE_ECUDA;
                break;
            }
            if (rep > 0) ms_best = std::min(ms_best, ms);
        }
        if (rc != MINE_OK) break;
        const double r = ops_of(blocks, iters) / (ms_best * 1e-3);
        if (per_form && form < n_form) per_form[form] = r;
        best = std::max(best, r);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (out) cudaFree(out);
    if (device >= 0) cudaSetDevice(prev);
    if (rc == MINE_OK) *ops_per_s = best;
    return rc;
}
