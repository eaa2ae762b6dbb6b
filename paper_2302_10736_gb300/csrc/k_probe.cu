// k_probe.cu - measurement kernel: the FP64 fused multiply-add throughput of
// the device, the denominator of the FP64 roofline this library reports (the
// method's kernels are bound by the FP64 pipe, not by HBM, on GB300).
//
// Every thread runs 8 independent chains x = x * m + c (enough to cover the
// pipe's latency) for `iters` rounds of 16 steps; the result is kept alive by
// a store that never happens (the chains cannot reach the compared value).
#include "pf_internal.h"

namespace pf {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8, kProbeUnroll = 16;

__global__ void __launch_bounds__(kProbeThreads) k_fp64_peak(int iters, double *sink)
{
    double x[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
    const double m = 0.9999999, a = 1e-9;
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kProbeUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kProbeChains; ++c) x[c] = fma(x[c], m, a);
        }
    }
    double r = 0.0;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) r += x[c];
    if (r == -1.0) *sink = r;   // every chain stays positive: never taken
}

}  // namespace pf

PF_API pf_status fp64_peak_probe(int32_t ctas, int32_t iters, double *sink, int64_t *dfma_per_launch,
                                 pf_stream stream)
{
    using namespace pf;
    if (ctas <= 0 || iters <= 0 || !sink)
        return set_error(PF_EINVAL, "fp64_peak_probe: ctas = %d, iters = %d, sink %s", ctas, iters,
                         sink ? "set" : "NULL");
    if (dfma_per_launch)
        *dfma_per_launch = (int64_t)ctas * kProbeThreads * iters * kProbeUnroll * kProbeChains;
    k_fp64_peak<<<(unsigned)ctas, kProbeThreads, 0, (cudaStream_t)stream>>>(iters, sink);
    PF_CUDA(cudaGetLastError());
    return PF_OK;
}
