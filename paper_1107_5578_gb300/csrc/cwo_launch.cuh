// cwo_launch.cuh -- once-per-device launch configuration of a kernel: the dynamic shared-memory
// opt-in and the number of CTAs the whole GPU holds at once (for persistent grids), computed on
// the first launch on each device and reused, so that a launch costs no attribute or occupancy
// query on the host.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <utility>

namespace cwo {

// Programmatic dependent launch: every hot kernel waits for the grid before it in the stream
// (griddepcontrol.wait, the first thing it does, so that grid's memory is complete and visible),
// and is launched with programmatic stream serialisation, so its launch is processed while the
// previous grid runs.  No kernel triggers its dependents early (griddepcontrol.launch_dependents):
// measured on GB300, every placement of the trigger cost time (up to 2 us per 2048^2 field) or
// gained nothing, while the launch overlap alone takes 512^2 propagations from 22.6 to 15.2 us.
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// grids of more CTAs than this are launched plainly (many waves: nothing to overlap)
constexpr unsigned kPdlMaxCtas = 4096;

template <typename... KArgs, typename... Args>
cudaError_t pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    const bool pdl = (unsigned long long)grid.x * grid.y * grid.z <= kPdlMaxCtas;
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}
#endif

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

// the same for a kernel with compile-time cluster dimensions: the number of its clusters the GPU
// holds at once
template <auto Kernel>
cudaError_t cluster_setup(size_t smem, int threads, int* clusters) {
    static std::atomic<int> cache[kMaxDevices];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int c = (dev >= 0 && dev < kMaxDevices) ? cache[dev].load(std::memory_order_acquire) : 0;
    if (c == 0) {
        if (smem > 48 * 1024 &&
            (e = cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2);
        cfg.blockDim = dim3(threads);
        cfg.dynamicSmemBytes = smem;
        int n = 0;
        if ((e = cudaOccupancyMaxActiveClusters(&n, Kernel, &cfg)) != cudaSuccess) return e;
        c = n + 1;
        if (dev >= 0 && dev < kMaxDevices) cache[dev].store(c, std::memory_order_release);
    }
    *clusters = c - 1;
    return cudaSuccess;
}

}  // namespace cwo
