// cwo_fourier.cu -- Fresnel diffraction in Fourier form (Section "The Fresnel diffraction
// (Fourier form)", Eqs. fre_fourier2 and fre_fourier3): one unpadded Nx x Ny DFT between two
// chirps, in two passes over an Nx x Ny column-major intermediate.
//
//   rows    : each source row times the source chirp exp(i pi (x1^2 + y1^2) / (lambda z))
//             (per-axis tables), forward DIF FFT of length Nx, transposed through a shared-memory
//             tile and stored with TMA into the intermediate [items][Nx][Ny] (storage column =
//             DIF position of kx, as in the convolution passes).
//   columns : C adjacent OUTPUT columns per CTA (lanes column-fastest): each reads the storage
//             column of its frequency, takes the forward DIF FFT of length Ny, and writes every
//             value to its natural, centred output position (kt + N/2) multiplied by the
//             destination chirp, the coefficient C and the (-1)^kt factors that make the plain
//             DFT a centred one; the C lanes of a row write C * 8 contiguous bytes.
#include "cwo_fft.cuh"
#include "cwo_internal.h"
#include "cwo_launch.cuh"
#include "cwo_tma.cuh"

namespace cwo {

template <int P> constexpr int fourier_rows() { return P >= 256 ? 4 : 8; }
template <int P, int R>
__host__ __device__ constexpr size_t fourier_row_words() {
    return PadLayout<P, R>::WORDS > (size_t)R * P ? PadLayout<P, R>::WORDS : (size_t)R * P;
}
constexpr int kFourierCols = 4;

template <int P, int R>
__global__ void __launch_bounds__(R * (P / 16))
k_fourier_rows(const float2* __restrict__ in, long long in_item_stride, const __grid_constant__ CUtensorMap wmap,
               const float2* __restrict__ pre_x, const float2* __restrict__ pre_y, const float4* __restrict__ tw) {
    pdl_wait();
    constexpr int T = P / 16, NT = R * T;
    constexpr int BOX = P < kTmaBoxCols ? P : kTmaBoxCols;
    extern __shared__ __align__(1024) float2 sm[];
    const int r = threadIdx.x % R, t = threadIdx.x / R;
    const int y0 = blockIdx.x * R;
    const int item = blockIdx.y;
    const float2* src = in + item * in_item_stride + (long long)(y0 + r) * P;
    const float2 cy = __ldg(pre_y + y0 + r);
    float2 v[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = cmul(src[t + e * T], cmul(__ldg(pre_x + t + e * T), cy));
    fwd1_from<P, R, 0, 16>(v, sm, r, t, TwTable<P>{tw, t});
    __syncthreads();   // every exchange read done before the tile (which aliases the region) is written
#pragma unroll
    for (int e = 0; e < 16; ++e) sm[e * NT + threadIdx.x] = v[e];
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll 1
        for (int b = 0; b < P / BOX; ++b) tma_store_3d(&wmap, sm + b * BOX * R, y0, b * BOX, item);
        tma_store_commit_and_drain();
    }
}

template <int P, int C>
__global__ void __launch_bounds__(C * (P / 16))
k_fourier_cols(const float2* __restrict__ win, long long win_item_stride, float2* __restrict__ out,
               long long out_item_stride, int nx, const int* __restrict__ st_of_col, const int* __restrict__ row_of_idx,
               const float2* __restrict__ post_x, const float2* __restrict__ post_y, const float4* __restrict__ tw) {
    pdl_wait();
    constexpr int T = P / 16;
    extern __shared__ float2 smc[];
    const int c = threadIdx.x % C, t = threadIdx.x / C;
    const int col = blockIdx.x * C + c;            // natural, centred output column
    const long long item = blockIdx.y;
    const float2* src = win + item * win_item_stride + (long long)__ldg(st_of_col + col) * P;
    float2 v[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = src[t + e * T];
    fwd1_from<P, C, 0, 16>(v, smc, c, t, TwTable<P>{tw, t});
    const float2 hx = __ldg(post_x + col);
    float2* dst = out + item * out_item_stride + col;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        const int i = e * T + t;                   // axis index of register e
        dst[(long long)__ldg(row_of_idx + i) * nx] = cmul(v[e], cmul(hx, __ldg(post_y + i)));
    }
}


template <int P>
static cudaError_t fourier_rows_impl(const float2* in, long long in_item_stride, const CUtensorMap* wmap, int ny,
                                     int items, const float2* pre_x, const float2* pre_y, const float4* tw,
                                     cudaStream_t st) {
    constexpr int R = fourier_rows<P>();
    if (ny % R || row_block_rows(P, false) != R) return cudaErrorInvalidValue;   // the map's box height
    const size_t smem = fourier_row_words<P, R>() * sizeof(float2);
    cudaError_t e = kernel_setup<k_fourier_rows<P, R>>(smem, R * (P / 16), nullptr);
    if (e != cudaSuccess) return e;
    return pdl_launch(k_fourier_rows<P, R>, dim3(ny / R, items), dim3(R * (P / 16)), smem, st, in, in_item_stride, *wmap,
                      pre_x, pre_y, tw);
}

template <int P>
static cudaError_t fourier_cols_impl(const float2* win, long long win_item_stride, float2* out, long long out_item_stride,
                                     int nx, int items, const int* st_of_col, const int* row_of_idx,
                                     const float2* post_x, const float2* post_y, const float4* tw, cudaStream_t st) {
    constexpr int C = kFourierCols;
    if (nx % C) return cudaErrorInvalidValue;
    const size_t smem = (size_t)PadLayout<P, C>::WORDS * sizeof(float2);
    cudaError_t e = kernel_setup<k_fourier_cols<P, C>>(smem, C * (P / 16), nullptr);
    if (e != cudaSuccess) return e;
    return pdl_launch(k_fourier_cols<P, C>, dim3(nx / C, items), dim3(C * (P / 16)), smem, st, win, win_item_stride, out,
                      out_item_stride, nx, st_of_col, row_of_idx, post_x, post_y, tw);
}

#define CWO_FOURIER_CASES(X) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096)

cudaError_t launch_fourier_rows(int px, const float2* in, long long in_item_stride, const CUtensorMap* wmap, int ny,
                                int items, const float2* pre_x, const float2* pre_y, const float4* tw, cudaStream_t st) {
    switch (px) {
#define CASE(P) case P: return fourier_rows_impl<P>(in, in_item_stride, wmap, ny, items, pre_x, pre_y, tw, st);
        CWO_FOURIER_CASES(CASE)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fourier_cols(int py, const float2* win, long long win_item_stride, float2* out, long long out_item_stride,
                                int nx, int items, const int* st_of_col, const int* row_of_idx, const float2* post_x,
                                const float2* post_y, const float4* tw, cudaStream_t st) {
    switch (py) {
#define CASE(P) case P: return fourier_cols_impl<P>(win, win_item_stride, out, out_item_stride, nx, items, st_of_col, row_of_idx, post_x, post_y, tw, st);
        CWO_FOURIER_CASES(CASE)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cwo
