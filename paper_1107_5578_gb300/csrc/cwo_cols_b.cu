// cwo_cols_b.cu -- the column-pass kernels of P = 1024 and 2048 (templates in cwo_cols.cuh).
#include "cwo_cols.cuh"

namespace cwo {

cudaError_t launch_col_b(int py, const float2* win, long long win_item_stride, float2* wout, long long wout_item_stride,
                         int px, int items, const float4* tw, const HParams& hp, cudaStream_t st) {
    switch (py) {
#define CASE(P) case P: return col_impl<P>(win, win_item_stride, wout, wout_item_stride, px, items, tw, hp, st);
        CASE(1024) CASE(2048)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_col_stack_b(int py, const float2* win, float2* wout, long long wout_item_stride, int px, int planes,
                               const float4* tw, const HParams& hp, cudaStream_t st) {
    switch (py) {
#define CASE(P) case P: return col_stack_impl<P>(win, wout, wout_item_stride, px, planes, tw, hp, st);
        CASE(1024) CASE(2048)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cwo
