// cwo_copy.cu -- field gather / scatter for the serving runtime: up to kCopyMaxFields fields of
// `elems` complex64 values copied between arbitrary device addresses, so that the requests of
// one mixed batch reach the slot's contiguous input buffer, and its outputs the callers' buffers,
// in one launch each.  The addresses travel in the kernel parameters (no upload); plain
// coalesced copies with 16-byte accesses where both addresses allow them.
#include <cuda_runtime.h>
#include <stdint.h>

#include "cwo_internal.h"
#include "cwo_launch.cuh"

namespace cwo {

__global__ void __launch_bounds__(256) k_copy_fields(const CopyList list, long long elems) {
    pdl_wait();
    const float2* s = list.src[blockIdx.y];
    float2* d = list.dst[blockIdx.y];
    if (!d || !s) return;                                    // a NULL address skips the item
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (((((uintptr_t)s) | ((uintptr_t)d)) & 15) == 0 && (elems & 1) == 0) {
        const float4* s4 = reinterpret_cast<const float4*>(s);
        float4* d4 = reinterpret_cast<float4*>(d);
        for (long long k = i0; k < elems / 2; k += stride) d4[k] = __ldcs(s4 + k);
    } else {
        for (long long k = i0; k < elems; k += stride) d[k] = __ldcs(s + k);
    }
}

cudaError_t launch_copy_fields(const CopyList& list, int fields, long long elems, cudaStream_t st) {
    if (fields < 1 || fields > kCopyMaxFields || elems < 1) return cudaErrorInvalidValue;
    const long long per_block = 256LL * 8;                   // ~8 float4 per thread
    const unsigned bx = (unsigned)std::min<long long>((elems / 2 + per_block - 1) / per_block, 1024);
    const cudaError_t e = pdl_launch(k_copy_fields, dim3(std::max(bx, 1u), (unsigned)fields), dim3(256), 0, st, list, elems);
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace cwo
