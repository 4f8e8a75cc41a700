// cwo_cols.cu -- entry points of the column pass: the once-calculation of the ASM transfer
// function (k_build_hcache) and the size dispatch to the translation units that instantiate the
// column kernels (cwo_cols_a/b/c.cu; the kernels themselves are in cwo_cols.cuh).
#include "cwo_cols.cuh"

namespace cwo {

__global__ void k_build_hcache(float2* __restrict__ out, int py, const HParams hp, const int* __restrict__ yidx) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (o >= py) return;
    const int i = yidx ? __ldg(yidx + o) : o;
    const int col = __ldg(hp.pairs + j).x;
    float2 h;
    if (hp.mode == HMODE_ASM_POLY) h = asm_h_reduced<true>(__ldg(hp.ax + col), __ldg(hp.ay + i), __ldg(hp.kf));
    else if (hp.mode == HMODE_ASM_EXACT) h = asm_h_reduced<false>(__ldg(hp.ax + col), __ldg(hp.ay + i), __ldg(hp.kf));
    else if (hp.mode == HMODE_ASM_FP32) h = asm_h_fp32(__ldg(hp.kbx + col), __ldg(hp.kby + i), hp);
    else h = asm_h_fp64(__ldg(hp.kbx + col), __ldg(hp.kby + i), hp.K, hp.sx, hp.sy);
    out[(long long)j * py + o] = h;
}

cudaError_t launch_build_hcache(float2* out, int npairs, int py, const HParams& hp, cudaStream_t st, const int* yidx) {
    if (npairs < 1 || py < 1 || hp.mode > HMODE_ASM_FP64) return cudaErrorInvalidValue;
    k_build_hcache<<<dim3((unsigned)((py + 255) / 256), (unsigned)npairs), 256, 0, st>>>(out, py, hp, yidx);
    return cudaGetLastError();
}

cudaError_t launch_col_stack(int py, const float2* win, float2* wout, long long wout_item_stride, int px, int planes,
                             const float4* tw, const HParams& hp, cudaStream_t st) {
    if (py <= 512) return launch_col_stack_a(py, win, wout, wout_item_stride, px, planes, tw, hp, st);
    if (py <= 2048) return launch_col_stack_b(py, win, wout, wout_item_stride, px, planes, tw, hp, st);
    return launch_col_stack_c(py, win, wout, wout_item_stride, px, planes, tw, hp, st);
}

cudaError_t launch_col(int py, const float2* win, long long win_item_stride, float2* wout,
                       long long wout_item_stride, int px, int items, const float4* tw,
                       const HParams& hp, cudaStream_t st) {
    if (py <= 512) return launch_col_a(py, win, win_item_stride, wout, wout_item_stride, px, items, tw, hp, st);
    if (py <= 2048) return launch_col_b(py, win, win_item_stride, wout, wout_item_stride, px, items, tw, hp, st);
    return launch_col_c(py, win, win_item_stride, wout, wout_item_stride, px, items, tw, hp, st);
}

}  // namespace cwo
