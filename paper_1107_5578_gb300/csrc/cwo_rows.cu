// cwo_rows.cu -- the two row passes of a propagation.
//
//   row forward : zero-pad each Nx-sample row to Px = 2 Nx and take its forward FFT
//                 (steps "expand" and the row half of "FFT" of Eqs. ang3 / fre_conv_fft).
//                 Only the Ny source rows exist; padding rows are never read, written or
//                 transformed.  The padding columns are never read either: the first DIF stage
//                 sees its upper 8 inputs as constant zeros.
//   row inverse : inverse FFT of each of the Ny kept rows of the intermediate, keeping the first
//                 Nx outputs ("extract the exact area") and applying the 1/(Px Py) scale.
//
// The intermediate W is [items][Ny][Px] complex64 in "storage order" along x: register e of
// thread t of the last forward stage (DIF position 16 t + e) is stored at column e * T + t, which
// makes every global access of both passes a fully coalesced 256-byte warp transaction.
#include "cwo_fft.cuh"
#include "cwo_internal.h"

namespace cwo {

template <int P> constexpr int rows_per_block() {
    constexpr int T = P / 16;
    constexpr int r = 256 / T;
    return r < 1 ? 1 : (r > 16 ? 16 : r);
}

template <int P, int RPB>
__global__ void __launch_bounds__(RPB * (P / 16))
k_row_fwd(const float2* __restrict__ in, long long in_item_stride, float2* __restrict__ w,
          long long w_item_stride, const float2* __restrict__ tw) {
    constexpr int T = P / 16, N = P / 2;
    extern __shared__ float2 sm[];
    const int t = threadIdx.x % T, r = threadIdx.x / T;
    const long long row = (long long)blockIdx.x * RPB + r;
    const long long item = blockIdx.y;
    const float2* src = in + item * in_item_stride + row * N;
    float2 v[16];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = __ldg(src + t + e * T);   // DIF stage-0 positions t + e P/16
#pragma unroll
    for (int e = 8; e < 16; ++e) v[e] = make_float2(0.f, 0.f);   // zero padding, never loaded
    fwd_from<P, RPB, 0, 8>(v, sm, r, t, tw);
    float2* dst = w + item * w_item_stride + row * P;
#pragma unroll
    for (int e = 0; e < 16; ++e) dst[e * T + t] = v[e];
}

template <int P, int RPB>
__global__ void __launch_bounds__(RPB * (P / 16))
k_row_inv(const float2* __restrict__ w, long long w_item_stride, float2* __restrict__ out,
          long long out_item_stride, float scale, const float2* __restrict__ tw) {
    constexpr int T = P / 16, N = P / 2;
    extern __shared__ float2 sm[];
    const int t = threadIdx.x % T, r = threadIdx.x / T;
    const long long row = (long long)blockIdx.x * RPB + r;
    const long long item = blockIdx.y;
    const float2* src = w + item * w_item_stride + row * P;
    float2 v[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = src[e * T + t];
    inv_from<P, RPB, Geo<P>::NST - 1>(v, sm, r, t, tw);
    float2* dst = out + item * out_item_stride + row * N;
#pragma unroll
    for (int e = 0; e < 8; ++e) dst[t + e * T] = cscale(v[e], scale);   // crop: first Nx outputs
}

template <typename K>
static cudaError_t ensure_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int P>
static cudaError_t row_fwd_impl(const float2* in, long long in_item_stride, float2* w,
                                long long w_item_stride, int ny, int items, const float2* tw,
                                cudaStream_t st) {
    constexpr int RPB = rows_per_block<P>();
    constexpr int T = P / 16;
    const size_t smem = (size_t)RPB * P * sizeof(float2);
    cudaError_t e = ensure_smem(k_row_fwd<P, RPB>, smem);
    if (e != cudaSuccess) return e;
    dim3 grid(ny / RPB, items);
    k_row_fwd<P, RPB><<<grid, RPB * T, smem, st>>>(in, in_item_stride, w, w_item_stride, tw);
    return cudaGetLastError();
}

template <int P>
static cudaError_t row_inv_impl(const float2* w, long long w_item_stride, float2* out,
                                long long out_item_stride, int ny, int items, float scale,
                                const float2* tw, cudaStream_t st) {
    constexpr int RPB = rows_per_block<P>();
    constexpr int T = P / 16;
    const size_t smem = (size_t)RPB * P * sizeof(float2);
    cudaError_t e = ensure_smem(k_row_inv<P, RPB>, smem);
    if (e != cudaSuccess) return e;
    dim3 grid(ny / RPB, items);
    k_row_inv<P, RPB><<<grid, RPB * T, smem, st>>>(w, w_item_stride, out, out_item_stride, scale, tw);
    return cudaGetLastError();
}

#define CWO_P_CASES(X) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096) X(8192)

cudaError_t launch_row_fwd(int px, const float2* in, long long in_item_stride, float2* w,
                           long long w_item_stride, int ny, int items, const float2* tw,
                           cudaStream_t st) {
    switch (px) {
#define CASE(P) case P: return row_fwd_impl<P>(in, in_item_stride, w, w_item_stride, ny, items, tw, st);
        CWO_P_CASES(CASE)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_row_inv(int px, const float2* w, long long w_item_stride, float2* out,
                           long long out_item_stride, int ny, int items, float scale,
                           const float2* tw, cudaStream_t st) {
    switch (px) {
#define CASE(P) case P: return row_inv_impl<P>(w, w_item_stride, out, out_item_stride, ny, items, scale, tw, st);
        CWO_P_CASES(CASE)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cwo
