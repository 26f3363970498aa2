// FP32 FMA throughput microbenchmark: the measured denominator of the ALU roofline that the
// eigensolve and the plain FP32 Gram are reported against.  Not part of the method.
//
// Every thread runs kChains independent chains x <- fma(x, a, b) for iters rounds.  The chains
// are independent so that the FMA pipe, not the 4-cycle dependent latency, bounds the rate;
// a = 1 - 2^-20 and b = 2^-20 keep every value near 1 (no denormals, no overflow), and the
// sum of the chains is stored so that no chain can be removed.  The grid is enough resident
// blocks to fill every SM.
#include "common.cuh"
#include "letkf.h"

namespace lk {
namespace {

constexpr int kChains = 16;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) fma_peak_kernel(int iters, float a, float b,
                                                            float *out) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1.0f + (float)(threadIdx.x * kChains + c) * 1e-7f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[(size_t)blockIdx.x * kThreads + threadIdx.x] = s;
}

}  // namespace
}  // namespace lk

extern "C" int letkf_fp32_peak_grid(int32_t *blocks, int32_t *threads) {
    if (!blocks || !threads) return LETKF_EINVAL;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lk::fma_peak_kernel, lk::kThreads,
                                                      0) != cudaSuccess)
        return LETKF_ECUDA;
    *blocks = sms * (per_sm > 0 ? per_sm : 1);
    *threads = lk::kThreads;
    return LETKF_OK;
}

extern "C" int letkf_fp32_peak_run(int32_t iters, float *out, int64_t *flops, void *stream) {
    if (iters < 1 || !out || !flops) return LETKF_EINVAL;
    int32_t blocks = 0, threads = 0;
    const int rc = letkf_fp32_peak_grid(&blocks, &threads);
    if (rc != LETKF_OK) return rc;
    const float a = 1.0f - 1.0f / 1048576.0f, b = 1.0f / 1048576.0f;
    lk::fma_peak_kernel<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(iters, a, b,
                                                                                   out);
    if (cudaGetLastError() != cudaSuccess) return LETKF_ECUDA;
    *flops = (int64_t)blocks * threads * iters * 8 * lk::kChains * 2;
    return LETKF_OK;
}
