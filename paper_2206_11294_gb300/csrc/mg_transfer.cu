// mg_copy_h2d_async: a host-to-device copy done by the SMs, which load from
// page-locked host memory over the CPU-GPU link.  The copy engines serve
// their queue in order, so a copy enqueued behind a large transfer on another
// stream waits for all of it; a kernel on a high-priority stream instead runs
// beside that transfer and shares the link with it.
#include <algorithm>
#include <cstdint>
#include <string>

#include "coupledmg.h"
#include "mg_host.h"

namespace {

constexpr int kThreads = 256;

// dst[i] = src[i] for 16-byte words, grid-stride; the last `tail` (< 16)
// bytes one by one in block 0.
__global__ void __launch_bounds__(kThreads) k_copy_words(uint4 *__restrict__ dst, const uint4 *__restrict__ src,
                                                         size_t words, unsigned char *__restrict__ dtail,
                                                         const unsigned char *__restrict__ stail, int tail) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += stride) dst[i] = src[i];
    if (blockIdx.x == 0 && (int)threadIdx.x < tail) dtail[threadIdx.x] = stail[threadIdx.x];
}

}  // namespace

extern "C" mg_status mg_copy_h2d_async(void *dst, const void *src, size_t bytes, void *stream) {
    using cmg::set_error;
    if (bytes == 0) return MG_OK;
    if (!dst || !src) return set_error(MG_ERR_INVALID_ARG, "NULL pointer");
    if ((reinterpret_cast<uintptr_t>(dst) & 15u) || (reinterpret_cast<uintptr_t>(src) & 15u))
        return set_error(MG_ERR_INVALID_ARG, "source and destination must be 16-byte aligned");
    cudaPointerAttributes as, ad;
    cudaError_t e = cudaPointerGetAttributes(&as, src);
    if (e == cudaSuccess) e = cudaPointerGetAttributes(&ad, dst);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(MG_ERR_INVALID_ARG, (std::string("pointer query: ") + cudaGetErrorString(e)).c_str());
    }
    if (as.type != cudaMemoryTypeHost || !as.devicePointer)
        return set_error(MG_ERR_INVALID_ARG, "the source must be page-locked host memory mapped for the device");
    if (ad.type != cudaMemoryTypeDevice) return set_error(MG_ERR_INVALID_ARG, "the destination must be device memory");
    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return set_error(MG_ERR_CUDA, cudaGetErrorString(e));
    if (ad.device != dev) return set_error(MG_ERR_INVALID_ARG, "the destination is on another device");
    const size_t words = bytes / 16;
    const int tail = (int)(bytes % 16);
    const size_t want = (words + kThreads - 1) / kThreads;
    // up to 4 blocks per SM; a copy of a few KB takes one block
    const unsigned blocks = (unsigned)std::max<size_t>(1, std::min<size_t>(want, (size_t)sms * 4));
    const unsigned char *s8 = static_cast<const unsigned char *>(as.devicePointer);
    unsigned char *d8 = static_cast<unsigned char *>(dst);
    k_copy_words<<<blocks, kThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<uint4 *>(d8), reinterpret_cast<const uint4 *>(s8), words, d8 + 16 * words,
        s8 + 16 * words, tail);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(MG_ERR_CUDA, cudaGetErrorString(e));
    return MG_OK;
}
