// cwo_calib.cu -- FP32 issue-rate calibration for the arithmetic roofline of the FFT passes.
// Every thread runs `iters` (a multiple of 8) steps of sixteen independent fused multiply-add
// chains -- enough independent work per warp to keep the FMA pipes busy, with one loop branch per
// 128 FFMAs -- and writes one value so that nothing is removed by the compiler.  The caller times
// the launch; the FP32 instruction count is blocks * 256 * iters * 16.
#include <cuda_runtime.h>

#include "../../include/cwo.h"
#include "../../include/cwo_debug.h"
#include "cwo_internal.h"

namespace cwo {

__global__ void __launch_bounds__(256) k_ffma_rate(float* __restrict__ out, int iters, float b, float c) {
    float a[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k] = threadIdx.x * 1e-3f + k;
#pragma unroll 1
    for (int i = 0; i < iters; i += 8) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int k = 0; k < 16; ++k) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 16; ++k) s += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace cwo

extern "C" cwo_status cwo_debug_ffma_rate(int blocks, int iters, float* out_dev, void* cuda_stream) {
    if (blocks < 1 || blocks > (1 << 20) || iters < 8 || iters > (1 << 24) || iters % 8 || !out_dev) {
        cwo::set_last_error("cwo_debug_ffma_rate: blocks in [1, 2^20], iters a multiple of 8 in [8, 2^24], out_dev required");
        return CWO_ERR_INVALID_ARG;
    }
    const int dev = [] { int d = 0; cudaGetDevice(&d); return d; }();
    const int st = cwo::check_device_buffer(out_dev, (size_t)blocks * 256 * sizeof(float), dev, "out_dev");
    if (st) return (cwo_status)st;
    cwo::k_ffma_rate<<<blocks, 256, 0, (cudaStream_t)cuda_stream>>>(out_dev, iters, 0.999999f, 1e-7f);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        cwo::set_last_error(cudaGetErrorString(e));
        return CWO_ERR_CUDA;
    }
    return CWO_OK;
}
