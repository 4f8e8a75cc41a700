// cwo_launch.cuh -- once-per-device launch configuration of a kernel: the dynamic shared-memory
// opt-in and the number of CTAs the whole GPU holds at once (for persistent grids), computed on
// the first launch on each device and reused, so that a launch costs no attribute or occupancy
// query on the host.
#pragma once
#include <cuda_runtime.h>

#include <atomic>

namespace cwo {

constexpr int kMaxDevices = 64;

template <auto Kernel>
cudaError_t kernel_setup(size_t smem, int threads, int* resident_ctas) {
    static std::atomic<int> cache[kMaxDevices];   // per device: resident CTAs + 1 (0: not yet)
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int c = (dev >= 0 && dev < kMaxDevices) ? cache[dev].load(std::memory_order_acquire) : 0;
    if (c == 0) {
        if (smem > 48 * 1024 &&
            (e = cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
        int sms = 0, per_sm = 0;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
            (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, Kernel, threads, smem)) != cudaSuccess)
            return e;
        c = sms * per_sm + 1;
        if (dev >= 0 && dev < kMaxDevices) cache[dev].store(c, std::memory_order_release);
    }
    if (resident_ctas) *resident_ctas = c - 1;
    return cudaSuccess;
}

}  // namespace cwo
