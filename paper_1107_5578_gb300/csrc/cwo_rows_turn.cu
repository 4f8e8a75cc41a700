// cwo_rows_turn.cu -- the turn from one propagation to the next of a constrained loop (k_row_turn).
#include "cwo_rows.cuh"

namespace cwo {

// a CTA of at least one whole warp; above Px = 2048 the persistent row passes, which overlap one
// group's memory traffic with another's transforms, are as fast as the turn (GS at 2048^2,
// 40 iterations: 10.72 ms fused, 10.68 ms separate; 512^2: 1.09 against 1.30 ms)
bool row_turn_supported(int px) { return px >= 64 && px <= 2048; }

cudaError_t launch_row_turn(int px, const CUtensorMap* wmap, int ny, int items, long long field_item_stride, float scale,
                            const float4* tw, int* status, const Epilogue& ep, cudaStream_t st) {
    if (ep.mode != EPI_PHASE && ep.mode != EPI_AMPLITUDE) return cudaErrorInvalidValue;
    switch (px) {
#define CASE(P) case P: return ep.mode == EPI_PHASE \
        ? row_turn_impl<P, EPI_PHASE>(wmap, ny, items, field_item_stride, scale, tw, status, ep, st) \
        : row_turn_impl<P, EPI_AMPLITUDE>(wmap, ny, items, field_item_stride, scale, tw, status, ep, st);
        CASE(64) CASE(128) CASE(256) CASE(512) CASE(1024) CASE(2048) CASE(4096)
#undef CASE
        default: return cudaErrorNotSupported;
    }
}

}  // namespace cwo
