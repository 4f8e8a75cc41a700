// cwo_cols.cuh -- the column pass: forward FFT down each column, transfer-function multiply,
// inverse FFT, crop to the Ny source rows -- the "FFT", "multiply by H" and "IFFT" steps of
// Eqs. ang3 / fre_conv_fft along y, fused in one kernel.
//
// The intermediate is column-major ([items][Px][Ny]), so each column is Ny contiguous complex64
// values and every global access of this pass is a coalesced 256-byte warp transaction.  Rows
// Ny .. Py-1 are the zero padding, seen as constant zeros by the first DIF stage.  The forward transform ends in DIF (digit-reversed) order, the
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
#pragma once
#include "cwo_fft.cuh"
#include "cwo_internal.h"
#include "cwo_h.cuh"
#include "cwo_launch.cuh"


namespace cwo {

// columns per block (single-column kernel) and mirror pairs per block (paired kernel)
template <int P> constexpr int cols_per_block() {
    constexpr int T = P / 16;
    constexpr int c = 256 / T;
    return c < 1 ? 1 : (c > 16 ? 16 : c);
}
template <int P> constexpr int col_min_blocks() { return (P / 16) * cols_per_block<P>() <= 256 ? 2 : 1; }
// The paired kernel holds 32 values per thread (128 registers): two 256-thread CTAs per SM up to
// P = 4096, one 512-thread CTA at P = 8192 (measured 382 us per 4096^2 field vs 488 for the
// single-column kernel).  Single column per transform: plans whose H is not even in kx.
template <int P, int C, bool MIXED>
__global__ void __launch_bounds__(C * (P / 16), col_min_blocks<P>())
k_col(const float2* __restrict__ win, long long win_item_stride, float2* __restrict__ wout,
      long long wout_item_stride, const float4* __restrict__ tw, const HParams hp) {
    pdl_wait();
    constexpr int T = P / 16, NY = P / 2;
    extern __shared__ float2 sm[];
    const int t = threadIdx.x % T, c = threadIdx.x / T;
    const int col = blockIdx.x * C + c;
    const long long item = blockIdx.y;
    const float2* src = win + item * win_item_stride + (long long)col * NY;
    float2 v[16];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = src[t + e * T];           // rows t + e P/16 < Ny
#pragma unroll
    for (int e = 8; e < 16; ++e) v[e] = make_float2(0.f, 0.f);   // zero padding rows
    const TwTable<P> twt{tw, t};
    fwd1_from<P, C, 0, 8, false>(v, sm, c, t, twt);
    apply_h<P, 1, MIXED>(v, v, col, t, item, hp);
    inv1_from<P, C, Geo<P>::NST - 1, false>(v, sm, c, t, twt);
    float2* dst = wout + item * wout_item_stride + (long long)col * NY;
#pragma unroll
    for (int e = 0; e < 8; ++e) dst[t + e * T] = v[e];           // crop: rows < Ny
}

// Mirror-pair column kernel: a thread transforms the two storage columns of frequencies +kx and
// -kx.  H depends on kx only through kx^2 (both methods), so the transfer function is evaluated
// (or loaded) once for both, and the twiddles of each stage are loaded once for both.  The
// exchanges take one barrier each (warp-wide after the first stage) and move a pair's two values
// at one position with one 128-bit access (P >= 128; at P = 8192 the 128-bit form measured 325
// against 334 us per 4096^2 field for 64-bit accesses, with the transfer function cached).  The
// grid is (items, pair groups), item fastest, so that the CTAs running at one time share few pair
// groups: the transfer-function values of a pair (the
// cached table of a once-calculation plan) are read from HBM once and from L2 by the other items.
// Thread 0 prefetches into L2 the columns of the CTA that will take this CTA's place (`resident`
// CTAs later in launch order), and in the CTA of the first item the cached H rows of its pairs.
// At P = 8192 this kernel serves the per-element transfer functions; a cached one runs the split
// form below.
template <int P, int CP>
constexpr int colp_smem_words() {
    return P >= 128 ? 2 * PairLayout<P, CP>::SLOTS : PadLayout<P, 2 * CP>::WORDS;
}

template <int P, int CP, bool MIXED>
__global__ void __launch_bounds__(CP * (P / 16), CP * (P / 16) >= 512 ? 1 : 2)
k_colp(const float2* __restrict__ win, long long win_item_stride, float2* __restrict__ wout,
       long long wout_item_stride, const float4* __restrict__ tw, const HParams hp, int resident) {
    pdl_wait();
    constexpr int T = P / 16, NY = P / 2;
    extern __shared__ float2 sm[];
    const int t = CP == 1 ? (int)threadIdx.x : (int)threadIdx.x % T;
    const int cp = CP == 1 ? 0 : (int)threadIdx.x / T;
    if (threadIdx.x == 0) {
        if (!MIXED && hp.mode == HMODE_TABLE && blockIdx.x == 0) {
            // the cached H rows of this CTA's pairs, read after the forward transform: requested
            // into L2 by the CTA of the first item, so that none of the items waits for HBM there
            const int j0 = blockIdx.y * CP, nr = min(CP, hp.npairs - j0);
            const float2* hrow = hp.hcache + (long long)j0 * hp.hcache_stride;
            const long long bytes = (long long)nr * hp.hcache_stride * 8;
            if ((((uintptr_t)hrow) & 15) == 0 && bytes % 16 == 0)
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" :: "l"(hrow), "r"((unsigned)bytes) : "memory");
        }
        const long long nb = (long long)blockIdx.y * gridDim.x + blockIdx.x + resident;
        if (nb < (long long)gridDim.x * gridDim.y) {
            const long long itn = nb % gridDim.x;
            const int gn = (int)(nb / gridDim.x);
            for (int c = 0; c < CP; ++c) {
                const int jn = gn * CP + c;
                if (jn >= hp.npairs) break;
                const int2 pn = __ldg(hp.pairs + jn);
                const float2* p0 = win + itn * win_item_stride + (long long)pn.x * NY;
                const float2* p1 = win + itn * win_item_stride + (long long)pn.y * NY;
                if ((((uintptr_t)p0 | (uintptr_t)p1) & 15) == 0) {
                    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" :: "l"(p0), "r"(NY * 8) : "memory");
                    if (pn.y != pn.x)
                        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" :: "l"(p1), "r"(NY * 8) : "memory");
                }
            }
        }
    }
    const int j = blockIdx.y * CP + cp;
    const bool live = j < hp.npairs;
    const int2 pr = __ldg(hp.pairs + (live ? j : 0));
    const long long item = blockIdx.x;
    const float2* sa = win + item * win_item_stride + (long long)pr.x * NY;
    const float2* sb = win + item * win_item_stride + (long long)pr.y * NY;
    float2 a[16], b[16];
#pragma unroll
    for (int e = 0; e < 8; ++e) { a[e] = __ldcg(sa + t + e * T); b[e] = __ldcg(sb + t + e * T); }
#pragma unroll
    for (int e = 8; e < 16; ++e) { a[e] = make_float2(0.f, 0.f); b[e] = make_float2(0.f, 0.f); }
    if constexpr (P >= 128) {
        fwd2v_from<P, CP, 0, 8>(a, b, reinterpret_cast<float4*>(sm), cp, t, tw);
        apply_h<P, 2, MIXED>(a, b, pr.x, t, item, hp);
        inv2v_from<P, CP, Geo<P>::NST - 1>(a, b, reinterpret_cast<float4*>(sm), cp, t, tw);
    } else {
        using Lay = PadLayout<P, 2 * CP>;
        fwd2x_from<P, CP, Lay, 0, 8>(a, b, sm, cp, t, tw);
        apply_h<P, 2, MIXED>(a, b, pr.x, t, item, hp);
        inv2x_from<P, CP, Lay, Geo<P>::NST - 1>(a, b, sm, cp, t, tw);
    }
    if (live) {
        float2* da = wout + item * wout_item_stride + (long long)pr.x * NY;
#pragma unroll
        for (int e = 0; e < 8; ++e) da[t + e * T] = a[e];
        if (pr.y != pr.x) {
            float2* db = wout + item * wout_item_stride + (long long)pr.y * NY;
#pragma unroll
            for (int e = 0; e < 8; ++e) db[t + e * T] = b[e];
        }
    }
}

// Column pass at Py = 8192 with the transfer function cached per plan, in split form.  A column
// holds Ny = 4096 samples zero-padded to 8192, so its DFT is exactly the pair of 4096-point DFTs
// of x_n (the even frequencies) and of x_n W_8192^n (the odd ones), and the cropped inverse is the
// 4096-point inverse of the even half plus W_8192^-n times that of the odd half, for n < 4096.  A
// thread carries both sequences of one column the way the 4096-point kernel carries a mirror pair
// (one twiddle load for both, 128-bit exchanges): two exchanges per direction instead of the
// three of the radix-16,16,16,2 transform, and two 256-thread CTAs per SM.  Grid (items,
// 2 (Px/2 + 1)), item fastest: CTA row c takes side c & 1 of mirror pair c / 2 (the self-paired
// columns kx = 0 and Px/2 once), so that the cached H row of a pair (64 KB, in the split order) is
// read from HBM once and from L2 by the other side and the other items.  The first CTA of a pair
// requests that row into L2 when it starts (without it the CTAs of a pair, which run at the same
// time, all waited for HBM after their forward transforms: 354 against 301 us per 4096^2 field),
// and thread 0 of every CTA prefetches into L2 the column of the CTA that will take its place.  The
// column and the H row are read past L1 (ld.global.cg: each value once), which leaves L1 to the
// twiddle and W_8192^n tables: 300 against 307 us per field.
template <int P>
__global__ void __launch_bounds__(P / 32, 2)
k_col_split(const float2* __restrict__ win, long long win_item_stride, float2* __restrict__ wout,
            long long wout_item_stride, const HParams hp, int resident) {
    pdl_wait();
    constexpr int Q = P / 2, T = Q / 16, NY = P / 2;
    extern __shared__ float2 sm[];
    float4* sx = reinterpret_cast<float4*>(sm);
    const int t = threadIdx.x;
    const int c = blockIdx.y, j = c >> 1;
    const int2 pr = __ldg(hp.pairs + j);
    if ((c & 1) && pr.y == pr.x) return;   // uniform over the CTA, before any barrier
    if (threadIdx.x == 0) {
        // the pair's H row, read after the forward transform: requested into L2 by the first CTA
        // of the pair, so that none of its CTAs waits for HBM there
        const float2* hrow = hp.hcache + (long long)j * hp.hcache_stride;
        if (blockIdx.x == 0 && (c & 1) == 0 && (((uintptr_t)hrow) & 15) == 0)
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" :: "l"(hrow), "r"(P * 8) : "memory");
        const long long nb = (long long)blockIdx.y * gridDim.x + blockIdx.x + resident;
        if (nb < (long long)gridDim.x * gridDim.y) {
            const long long itn = nb % gridDim.x;
            const int cn = (int)(nb / gridDim.x);
            const int2 pn = __ldg(hp.pairs + (cn >> 1));
            const float2* pf = win + itn * win_item_stride + (long long)((cn & 1) ? pn.y : pn.x) * NY;
            if ((((uintptr_t)pf) & 15) == 0)
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" :: "l"(pf), "r"(NY * 8) : "memory");
        }
    }
    const int col = (c & 1) ? pr.y : pr.x;
    const long long item = blockIdx.x;
    const float2* src = win + item * win_item_stride + (long long)col * NY;
    float2 a[16], b[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) a[e] = __ldcg(src + t + e * T);   // n = t + e 256: every sample
#pragma unroll
    for (int e = 0; e < 16; ++e) b[e] = cmul(a[e], __ldg(hp.split_w + t + e * T));
    fwd2v_from<Q, 1, 0, 16>(a, b, sx, 0, t, hp.split_tw);
    const float2* hc = hp.hcache + (long long)j * hp.hcache_stride + t;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        const float2 ha = __ldcg(hc + e * T), hb = __ldcg(hc + Q + e * T);
        a[e] = hp.conj ? cmulc(a[e], ha) : cmul(a[e], ha);
        b[e] = hp.conj ? cmulc(b[e], hb) : cmul(b[e], hb);
    }
    inv2v_from<Q, 1, Geo<Q>::NST - 1>(a, b, sx, 0, t, hp.split_tw);
    float2* dst = wout + item * wout_item_stride + (long long)col * NY;
#pragma unroll
    for (int e = 0; e < 16; ++e) dst[t + e * T] = cadd(a[e], cmulc(b[e], __ldg(hp.split_w + t + e * T)));
}

// Shared-source z-stack: the forward column transform of the source is computed once and kept
// in registers; for each plane the kernel multiplies a copy by that plane's transfer function,
// transforms it back and writes the plane (Section "Three-dimensional diffraction calculations":
// a stack of 2-D diffractions of one source).
template <int P, int C>
__global__ void __launch_bounds__(C * (P / 16), col_min_blocks<P>())
k_col_stack(const float2* __restrict__ win, float2* __restrict__ wout, long long wout_item_stride, int nplanes,
            const float4* __restrict__ tw, const HParams hp) {
    pdl_wait();
    constexpr int T = P / 16, NY = P / 2;
    extern __shared__ float2 sm[];
    const int t = threadIdx.x % T, c = threadIdx.x / T;
    const int col = blockIdx.x * C + c;
    const float2* src = win + (long long)col * NY;
    float2 spec[16];
#pragma unroll
    for (int e = 0; e < 8; ++e) spec[e] = src[t + e * T];
#pragma unroll
    for (int e = 8; e < 16; ++e) spec[e] = make_float2(0.f, 0.f);
    const TwTable<P> twt{tw, t};
    fwd1_from<P, C, 0, 8, false>(spec, sm, c, t, twt);
#pragma unroll 1
    for (int z = 0; z < nplanes; ++z) {
        float2 v[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) v[e] = spec[e];
        apply_h<P, 1>(v, v, col, t, z, hp);
        // the previous plane's last exchange reads are done before this plane's first writes
        if (z > 0) __syncthreads();
        inv1_from<P, C, Geo<P>::NST - 1, false>(v, sm, c, t, twt);
        float2* dst = wout + z * wout_item_stride + (long long)col * NY;
#pragma unroll
        for (int e = 0; e < 8; ++e) dst[t + e * T] = v[e];
    }
}


template <int P, bool MIXED>
static cudaError_t col_impl_t(const float2* win, long long win_item_stride, float2* wout,
                              long long wout_item_stride, int px, int items, const float4* tw,
                              const HParams& hp, cudaStream_t st) {
    constexpr int T = P / 16;
    cudaError_t e;
    if constexpr (P == kSplitColP && !MIXED) {
        if (hp.mode == HMODE_TABLE) {   // the cached H is stored in the split order at this Py
            if (hp.asym || !hp.split_tw || !hp.split_w || !hp.hcache || !hp.pairs || hp.npairs != px / 2 + 1)
                return cudaErrorInvalidValue;
            const size_t smem = (size_t)colp_smem_words<P / 2, 1>() * sizeof(float2);
            int resident = 0;
            if ((e = kernel_setup<k_col_split<P>>(smem, P / 32, &resident))) return e;
            e = pdl_launch(k_col_split<P>, dim3(items, 2 * hp.npairs), dim3(P / 32), smem, st, win, win_item_stride,
                           wout, wout_item_stride, hp, resident);
            if (e != cudaSuccess) return e;
            return cudaGetLastError();
        }
    }
    if (hp.asym) {   // H(kx) != H(-kx): one column per transform
        constexpr int C = cols_per_block<P>();
        if (px % C != 0) return cudaErrorInvalidValue;
        const size_t smem = (size_t)PadLayout<P, C>::WORDS * sizeof(float2);
        if ((e = kernel_setup<k_col<P, C, MIXED>>(smem, C * T, nullptr))) return e;
        e = pdl_launch(k_col<P, C, MIXED>, dim3(px / C, items), dim3(C * T), smem, st, win, win_item_stride, wout,
                       wout_item_stride, tw, hp);
        if (e != cudaSuccess) return e;
    } else {         // H even in kx: mirror pairs
        constexpr int CP = cols_per_block<P>();
        if (hp.npairs != px / 2 + 1 || !hp.pairs) return cudaErrorInvalidValue;
        const size_t smem = (size_t)colp_smem_words<P, CP>() * sizeof(float2);
        int resident = 0;
        if ((e = kernel_setup<k_colp<P, CP, MIXED>>(smem, CP * T, &resident))) return e;
        const unsigned blocks = (unsigned)((hp.npairs + CP - 1) / CP);
        e = pdl_launch(k_colp<P, CP, MIXED>, dim3(items, blocks), dim3(CP * T), smem, st, win, win_item_stride, wout,
                       wout_item_stride, tw, hp, resident);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

template <int P>
static cudaError_t col_impl(const float2* win, long long win_item_stride, float2* wout,
                            long long wout_item_stride, int px, int items, const float4* tw,
                            const HParams& hp, cudaStream_t st) {
    return hp.items ? col_impl_t<P, true>(win, win_item_stride, wout, wout_item_stride, px, items, tw, hp, st)
                    : col_impl_t<P, false>(win, win_item_stride, wout, wout_item_stride, px, items, tw, hp, st);
}

template <int P>
static cudaError_t col_stack_impl(const float2* win, float2* wout, long long wout_item_stride, int px, int planes,
                                  const float4* tw, const HParams& hp, cudaStream_t st) {
    constexpr int C = cols_per_block<P>();
    constexpr int T = P / 16;
    if (px % C != 0) return cudaErrorInvalidValue;
    if (P == kSplitColP && hp.mode == HMODE_TABLE) return cudaErrorInvalidValue;   // cached H in the split order
    const size_t smem = (size_t)PadLayout<P, C>::WORDS * sizeof(float2);
    cudaError_t e;
    if ((e = kernel_setup<k_col_stack<P, C>>(smem, C * T, nullptr))) return e;
    return pdl_launch(k_col_stack<P, C>, dim3(px / C), dim3(C * T), smem, st, win, wout, wout_item_stride, planes, tw, hp);
}

// Launchers of the sizes each translation unit instantiates (cwo_cols_a/b/c.cu: P <= 512,
// P = 1024 and 2048, P = 4096 and 8192), so that the kernels compile in parallel.
cudaError_t launch_col_a(int py, const float2* win, long long win_item_stride, float2* wout, long long wout_item_stride,
                         int px, int items, const float4* tw, const HParams& hp, cudaStream_t st);
cudaError_t launch_col_b(int py, const float2* win, long long win_item_stride, float2* wout, long long wout_item_stride,
                         int px, int items, const float4* tw, const HParams& hp, cudaStream_t st);
cudaError_t launch_col_c(int py, const float2* win, long long win_item_stride, float2* wout, long long wout_item_stride,
                         int px, int items, const float4* tw, const HParams& hp, cudaStream_t st);
cudaError_t launch_col_stack_a(int py, const float2* win, float2* wout, long long wout_item_stride, int px, int planes,
                               const float4* tw, const HParams& hp, cudaStream_t st);
cudaError_t launch_col_stack_b(int py, const float2* win, float2* wout, long long wout_item_stride, int px, int planes,
                               const float4* tw, const HParams& hp, cudaStream_t st);
cudaError_t launch_col_stack_c(int py, const float2* win, float2* wout, long long wout_item_stride, int px, int planes,
                               const float4* tw, const HParams& hp, cudaStream_t st);

}  // namespace cwo
