// cwo_cols.cu -- the column pass: forward FFT down each column, transfer-function multiply,
// inverse FFT, crop to the Ny source rows -- the "FFT", "multiply by H" and "IFFT" steps of
// Eqs. ang3 / fre_conv_fft along y, fused in one kernel.
//
// Each column holds Ny stored rows; rows Ny .. Py-1 are the zero padding, seen as constant
// zeros by the first DIF stage.  The forward transform ends in DIF (digit-reversed) order, the
// transfer function is generated for that order, and the inverse (the exact adjoint of the
// forward stages) starts from it: no reordering and no exchange between the last forward and the
// first inverse stage.  Only the Ny kept rows are written back.
//
// Transfer functions:
//   ASM (Eq. ang2), phase in cycles  psi = K sqrt(1 - s),  K = z / lambda,  s = a_x + a_y,
//   a = lambda^2 f^2.  Split exactly as
//       K sqrt(1-s) = K - [K a_x/2 + K a_x^2/8] - [K a_y/2 + K a_y^2/8] - K a_x a_y / 4 - tail,
//       tail = K s^3 (3 + q) / (8 (1 + q)^3),  q = sqrt(1 - s),
//   the bracketed per-axis terms (up to ~1e4 cycles) and frac(K) are range-reduced in FP64 on
//   the host; the cross term (up to ~12 cycles) is a float-float product of two per-axis values
//   reduced exactly in FP32; the tail is < 1 cycle.  s > 1 (evanescent) gives H = 0.
//   Fresnel (Eq. fre_conv_fft): H = C * Hx[kx] * Hy[ky], the two 1-D DFTs of the sampled
//   impulse response computed in FP64 per plan (h_F is separable).
#include "cwo_fft.cuh"
#include "cwo_internal.h"
#include "cwo_h.cuh"

namespace cwo {

template <int P> constexpr int cols_per_block() {
    constexpr int T = P / 16;
    constexpr int c = 512 / T;
    return c < 1 ? 1 : (c > 32 ? 32 : c);
}

__device__ __forceinline__ float2 asm_h_fp32(int kbx, int kby, const HParams& hp) {
    // Eq. ang2 evaluated literally in single precision (precision-study arm)
    const float fx = (float)kbx * (float)hp.dfx, fy = (float)kby * (float)hp.dfy;
    const float k = (float)hp.k;
    const float fourpi2 = 39.4784176043574344753f;
    const float rad = k * k - fourpi2 * (fx * fx + fy * fy);
    if (rad < 0.0f) return make_float2(0.f, 0.f);
    const float ph = (float)hp.z * sqrtf(rad);
    float sn, cs;
    sincosf(ph, &sn, &cs);
    return make_float2(cs, sn);
}

__device__ __forceinline__ float2 asm_h_fp64(int kbx, int kby, const HParams& hp) {
    // phase K sqrt(1 - s) per element in FP64, reduced to [-1/2, 1/2] cycle (reference arm)
    const double s = hp.sx * (double)kbx * (double)kbx + hp.sy * (double)kby * (double)kby;
    if (s > 1.0) return make_float2(0.f, 0.f);
    double psi = hp.K * sqrt(1.0 - s);
    psi -= rint(psi);
    float sn, cs;
    sincospif(2.0f * (float)psi, &sn, &cs);
    return make_float2(cs, sn);
}

template <int P>
__device__ __forceinline__ void apply_h(float2 (&v)[16], int col, int t, long long item,
                                        const HParams& hp) {
    constexpr int T = P / 16;
    if (hp.mode == HMODE_FRESNEL) {
        const float2 hxc = __ldg(hp.hx + item * hp.x_item_stride + col);
        const float2* hy = hp.hy + item * hp.y_item_stride + t;
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const float2 h = cmul(hxc, __ldg(hy + e * T));
            v[e] = hp.conj ? cmulc(v[e], h) : cmul(v[e], h);
        }
    } else if (hp.mode == HMODE_ASM_REDUCED) {
        const float4 X = __ldg(hp.ax + item * hp.x_item_stride + col);
        const float4* ay = hp.ay + item * hp.y_item_stride + t;
        const float K = __ldg(hp.kf + item * hp.kf_item_stride);
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const float2 h = asm_h_reduced(X, __ldg(ay + e * T), K);
            v[e] = hp.conj ? cmulc(v[e], h) : cmul(v[e], h);
        }
    } else {
        const int kbx = __ldg(hp.kbx + col);
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const int kby = __ldg(hp.kby + e * T + t);
            const float2 h = hp.mode == HMODE_ASM_FP32 ? asm_h_fp32(kbx, kby, hp) : asm_h_fp64(kbx, kby, hp);
            v[e] = hp.conj ? cmulc(v[e], h) : cmul(v[e], h);
        }
    }
}

template <int P, int C>
__global__ void __launch_bounds__(C * (P / 16))
k_col(const float2* __restrict__ win, long long win_item_stride, float2* __restrict__ wout,
      long long wout_item_stride, int px, const float2* __restrict__ tw, const HParams hp) {
    constexpr int T = P / 16;
    extern __shared__ float2 sm[];
    const int c = threadIdx.x % C, t = threadIdx.x / C;
    const int col = blockIdx.x * C + c;
    const long long item = blockIdx.y;
    const float2* src = win + item * win_item_stride + col;
    float2 v[16];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = src[(long long)(t + e * T) * px];   // rows < Ny only
#pragma unroll
    for (int e = 8; e < 16; ++e) v[e] = make_float2(0.f, 0.f);
    fwd_from<P, C, 0, 8>(v, sm, c, t, tw);
    apply_h<P>(v, col, t, item, hp);
    inv_from<P, C, Geo<P>::NST - 1>(v, sm, c, t, tw);
    float2* dst = wout + item * wout_item_stride + col;
#pragma unroll
    for (int e = 0; e < 8; ++e) dst[(long long)(t + e * T) * px] = v[e];   // crop: rows < Ny
}

template <int P>
static cudaError_t col_impl(const float2* win, long long win_item_stride, float2* wout,
                            long long wout_item_stride, int px, int items, const float2* tw,
                            const HParams& hp, cudaStream_t st) {
    constexpr int C = cols_per_block<P>();
    constexpr int T = P / 16;
    const size_t smem = (size_t)C * P * sizeof(float2);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_col<P, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (px % C != 0) return cudaErrorInvalidValue;
    dim3 grid(px / C, items);
    k_col<P, C><<<grid, C * T, smem, st>>>(win, win_item_stride, wout, wout_item_stride, px, tw, hp);
    return cudaGetLastError();
}

cudaError_t launch_col(int py, const float2* win, long long win_item_stride, float2* wout,
                       long long wout_item_stride, int px, int items, const float2* tw,
                       const HParams& hp, cudaStream_t st) {
    switch (py) {
#define CASE(P) case P: return col_impl<P>(win, win_item_stride, wout, wout_item_stride, px, items, tw, hp, st);
        CASE(32) CASE(64) CASE(128) CASE(256) CASE(512) CASE(1024) CASE(2048) CASE(4096) CASE(8192)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cwo
