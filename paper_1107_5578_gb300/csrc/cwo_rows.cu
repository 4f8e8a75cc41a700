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
// The intermediate W is COLUMN-MAJOR, [items][Px][Ny] complex64: storage column st holds the Ny
// values of one frequency kx contiguously, so that the column pass streams whole columns.  Along
// x the storage order is the register order of the last forward stage: register e of thread t
// (DIF position 16 t + e) is storage column e * T + t.  A CTA handles R rows and transposes them
// through a padded shared-memory tile, so that each group of R lanes writes (reads) R
// consecutive values of one storage column: R * 8 contiguous bytes per lane group.
#include "cwo_fft.cuh"
#include "cwo_internal.h"

namespace cwo {

// threads per row-pass CTA (compile-time tuning knob)
#ifndef CWO_ROW_THREADS
#define CWO_ROW_THREADS 1024
#endif
template <int P> constexpr int rows_per_block() {
    constexpr int T = P / 16;
    constexpr int r = CWO_ROW_THREADS / T;
    return r < 1 ? 1 : (r > 8 ? 8 : r);
}

template <int P, int R>
constexpr size_t row_smem_words() {
    return PadLayout<P, R>::WORDS > TileLayout<P, R>::WORDS ? PadLayout<P, R>::WORDS : TileLayout<P, R>::WORDS;
}

template <int P, int R>
__global__ void __launch_bounds__(R * (P / 16))
k_row_fwd(const float2* __restrict__ in, long long in_item_stride, float2* __restrict__ w,
          long long w_item_stride, int ny, const float4* __restrict__ tw) {
    constexpr int T = P / 16, N = P / 2, NT = R * T;
    using Tile = TileLayout<P, R>;
    extern __shared__ float2 sm[];
    const int t = threadIdx.x % T, r = threadIdx.x / T;
    const long long y0 = (long long)blockIdx.x * R;
    const long long item = blockIdx.y;
    const float2* src = in + item * in_item_stride + (y0 + r) * N;
    float2 v[16];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = __ldg(src + t + e * T);   // DIF stage-0 positions t + e P/16
#pragma unroll
    for (int e = 8; e < 16; ++e) v[e] = make_float2(0.f, 0.f);   // zero padding, never loaded
    fwd_from<P, R, PadLayout<P, R>, 0, 8, 0>(v, sm, r, t, TwTable<P>{tw, t});
    // transpose: register e of (r, t) is storage column st = e T + t of row y0 + r
#pragma unroll
    for (int e = 0; e < 16; ++e) sm[Tile::addr(e * T + t, r)] = v[e];
    __syncthreads();
    float2* dst = w + item * w_item_stride + y0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int i = threadIdx.x + k * NT;          // i = st * R + rr
        dst[(long long)(i / R) * ny + (i % R)] = sm[i + (i >> 4)];
    }
}

template <int P, int R>
__global__ void __launch_bounds__(R * (P / 16))
k_row_inv(const float2* __restrict__ w, long long w_item_stride, float2* __restrict__ out,
          long long out_item_stride, int ny, float scale, const float4* __restrict__ tw) {
    constexpr int T = P / 16, N = P / 2, NT = R * T;
    using Tile = TileLayout<P, R>;
    extern __shared__ float2 sm[];
    const int t = threadIdx.x % T, r = threadIdx.x / T;
    const long long y0 = (long long)blockIdx.x * R;
    const long long item = blockIdx.y;
    const float2* src = w + item * w_item_stride + y0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int i = threadIdx.x + k * NT;
        sm[i + (i >> 4)] = src[(long long)(i / R) * ny + (i % R)];
    }
    __syncthreads();
    float2 v[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = sm[Tile::addr(e * T + t, r)];
    __syncthreads();
    inv_from<P, R, PadLayout<P, R>, Geo<P>::NST - 1, 0, 0>(v, sm, r, t, TwTable<P>{tw, t});
    float2* dst = out + item * out_item_stride + (y0 + r) * N;
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
                                long long w_item_stride, int ny, int items, const float4* tw,
                                cudaStream_t st) {
    constexpr int R = rows_per_block<P>();
    constexpr int T = P / 16;
    const size_t smem = row_smem_words<P, R>() * sizeof(float2);
    cudaError_t e = ensure_smem(k_row_fwd<P, R>, smem);
    if (e != cudaSuccess) return e;
    if (ny % R) return cudaErrorInvalidValue;
    dim3 grid(ny / R, items);
    k_row_fwd<P, R><<<grid, R * T, smem, st>>>(in, in_item_stride, w, w_item_stride, ny, tw);
    return cudaGetLastError();
}

template <int P>
static cudaError_t row_inv_impl(const float2* w, long long w_item_stride, float2* out,
                                long long out_item_stride, int ny, int items, float scale,
                                const float4* tw, cudaStream_t st) {
    constexpr int R = rows_per_block<P>();
    constexpr int T = P / 16;
    const size_t smem = row_smem_words<P, R>() * sizeof(float2);
    cudaError_t e = ensure_smem(k_row_inv<P, R>, smem);
    if (e != cudaSuccess) return e;
    if (ny % R) return cudaErrorInvalidValue;
    dim3 grid(ny / R, items);
    k_row_inv<P, R><<<grid, R * T, smem, st>>>(w, w_item_stride, out, out_item_stride, ny, scale, tw);
    return cudaGetLastError();
}

#define CWO_P_CASES(X) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096) X(8192)

cudaError_t launch_row_fwd(int px, const float2* in, long long in_item_stride, float2* w,
                           long long w_item_stride, int ny, int items, const float4* tw,
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
                           const float4* tw, cudaStream_t st) {
    switch (px) {
#define CASE(P) case P: return row_inv_impl<P>(w, w_item_stride, out, out_item_stride, ny, items, scale, tw, st);
        CWO_P_CASES(CASE)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cwo
