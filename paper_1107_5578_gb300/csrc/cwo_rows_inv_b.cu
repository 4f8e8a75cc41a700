// cwo_rows_inv_b.cu -- the inverse row pass for Px >= 2048 (every output epilogue).
#include "cwo_rows.cuh"

namespace cwo {

cudaError_t launch_row_inv_b(int px, const CUtensorMap* wmap, int item_off, float2* out, long long out_item_stride,
                             int ny, int items, float scale, const float4* tw, int* status, cudaStream_t st,
                             const Epilogue& ep) {
    switch (px) {
#define CASE(P) case P: return row_inv_impl<P>(wmap, item_off, out, out_item_stride, ny, items, scale, tw, status, ep, st);
        CASE(2048) CASE(4096) CASE(8192)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cwo
