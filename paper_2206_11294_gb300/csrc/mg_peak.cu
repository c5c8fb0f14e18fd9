// mg_fp64_fma_rate: the device's FP64 FMA issue rate, measured.  Most kernels
// of the solver are bound by GB300's FP64 pipe rather than by HBM, so their
// roofline denominator is this rate: a kernel whose threads run independent
// chains of register-resident FMAs (no memory traffic), timed with CUDA events.
#include <string>

#include "coupledmg.h"
#include "mg_host.h"

namespace {

constexpr int kChains = 8;          // independent FMA chains per thread
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 4;

__global__ void __launch_bounds__(kThreads) k_fp64_fma_chains(double *sink, int iters, double a, double c) {
    double v[kChains];
#pragma unroll
    for (int q = 0; q < kChains; q++) v[q] = 1e-3 * (threadIdx.x + q);
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int q = 0; q < kChains; q++) v[q] = fma(v[q], a, c);
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kChains; q++) s += v[q];
    if (s == -1.0) sink[threadIdx.x] = s;   // never true for these inputs; keeps the chains live
}

}  // namespace

extern "C" mg_status mg_fp64_fma_rate(void *stream, int repeats, double *g_fma_per_s) {
    using cmg::set_error;
    if (!g_fma_per_s || repeats < 1 || repeats > 100) return set_error(MG_ERR_INVALID_ARG, "repeats in 1..100, out non-NULL");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return set_error(MG_ERR_CUDA, cudaGetErrorString(e));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int blocks = sms * kBlocksPerSM, iters = 4096;
    const double fmas = (double)blocks * kThreads * kChains * iters;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double best = 0.0;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // one untimed launch, then the fastest of `repeats` timed ones (a burst rate)
    for (int r = -1; r < repeats && e == cudaSuccess; r++) {
        e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) {
            k_fp64_fma_chains<<<blocks, kThreads, 0, s>>>(nullptr, iters, 0.999999, 1e-7);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && r >= 0 && ms > 0.f) best = std::max(best, fmas / (ms * 1e-3) / 1e9);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return set_error(MG_ERR_CUDA, (std::string("FP64 rate kernel: ") + cudaGetErrorString(e)).c_str());
    *g_fma_per_s = best;
    return MG_OK;
}
