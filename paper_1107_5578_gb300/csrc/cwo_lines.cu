// cwo_lines.cu -- Fresnel diffraction in the convolution form as two separable line passes.
//
// The sampled Fresnel impulse response of Eq. fre_conv_prop_d is a product of one chirp per axis,
// h_F(x, y) = exp(i pi x^2 / (lambda z)) exp(i pi y^2 / (lambda z)), and the zero-padded FFT method
// of Eq. fre_conv_fft equals the linear convolution of the field with it.  That 2-D convolution
// is exactly a 1-D linear convolution of every row with the x chirp followed by one of every column
// with the y chirp, and each 1-D convolution is again the padded FFT method on a line:
//   expand the line to P = 2N, FFT, multiply by the axis transfer function (the FP64 DFT of the
//   sampled chirp; the x table carries the coefficient C), IFFT, keep the first N samples.
// One kernel does both passes.  Pass 1 takes the Ny rows of the field and stores its results
// transposed into a column-major N x N intermediate; pass 2 takes the Nx contiguous columns of
// that intermediate and stores transposed again, i.e. into the row-major output.  Each pass reads
// and writes 8 N^2 bytes (32 N^2 per propagation against 80 N^2 for the three-pass method with an
// N x 2N intermediate) and transforms half as many lines of length 2N as the column pass.
//
// The shifted Fresnel diffraction (Eqs. shift_fre1 - shift_fre3) is the same convolution between a
// source factor f and a destination factor q, both products of one factor per axis, so each pass
// also multiplies its input samples by f along its axis and its kept outputs by q (FAC).
//
// A CTA holds R lines, loads each thread's 8 nonzero stage-0 samples, runs the forward DIF
// stages, multiplies by the table in DIF order (register e of thread t holds the frequency of axis
// index e T + t), runs the adjoint stages back to natural order, scales, and writes the kept half
// as a dense tile [position][line] that TMA stores as boxes of R lines x min(256, N) positions.
// Three forms: the pair form (512 <= P <= 4096; a thread per pair of lines, loads straight from
// global memory), the persistent form (P = 8192; staged bulk loads, measured 0.36 against 0.42 ms
// per pass of two 4096^2 fields for the pair form there) and the single-line form (P < 512, and
// inputs off a 16-byte boundary at P = 8192).
#include <algorithm>
#include <stdint.h>

#include "cwo_fft.cuh"
#include "cwo_internal.h"
#include "cwo_launch.cuh"
#include "cwo_tma.cuh"

namespace cwo {

// lines per group: 2 from P = 4096 (one pair per thread: two 256-thread CTAs per SM at P = 4096,
// measured 73 against 79 us per 2048^2 field with 4-line groups and their whole-sector column
// pieces), 4 below
template <int P> constexpr int line_rows() { return P >= 4096 ? 2 : (P >= 256 ? 4 : 8); }

template <int P, int R>
__host__ __device__ constexpr size_t line_smem_words() {
    return PadLayout<P, R>::WORDS > (size_t)R * (P / 2) ? PadLayout<P, R>::WORDS : (size_t)R * (P / 2);
}

template <int P, int R, bool FAC>
__global__ void __launch_bounds__(R * (P / 16))
k_line_conv(const float2* __restrict__ in, long long in_item_stride, const __grid_constant__ CUtensorMap omap,
            const float2* __restrict__ h, long long h_item_stride, int conj, float scale,
            const float4* __restrict__ tw, const float2* __restrict__ pre, const float2* __restrict__ post) {
    pdl_wait();
    constexpr int T = P / 16, N = P / 2, NT = R * T;
    constexpr int BOX = N < kTmaBoxCols ? N : kTmaBoxCols;
    extern __shared__ __align__(1024) float2 sm[];
    const int r = threadIdx.x % R, t = threadIdx.x / R;
    const int l0 = blockIdx.x * R;
    const int item = blockIdx.y;
    const float2* src = in + item * in_item_stride + (long long)(l0 + r) * N;
    float2 v[16];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = __ldg(src + t + e * T);   // stage-0 positions t + e P/16 < N
#pragma unroll
    for (int e = 8; e < 16; ++e) v[e] = make_float2(0.f, 0.f);   // the expanded half, never loaded
    if constexpr (FAC) {
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = cmul(v[e], __ldg(pre + t + e * T));
    }
    const TwTable<P> twt{tw, t};
    fwd1_from<P, R, 0, 8>(v, sm, r, t, twt);
    const float2* hh = h + item * h_item_stride + t;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        const float2 w = __ldg(hh + e * T);
        v[e] = conj ? cmulc(v[e], w) : cmul(v[e], w);
    }
    inv1_from<P, R, Geo<P>::NST - 1>(v, sm, r, t, twt);
    // kept positions t + e T (e < 8): tile index (t + e T) R + r = e R T + threadIdx.x; the
    // tile aliases the exchange region, so every exchange read completes first
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const float2 w = cscale(v[e], scale);
        sm[e * NT + threadIdx.x] = FAC ? cmul(w, __ldg(post + t + e * T)) : w;
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll 1
        for (int b = 0; b < N / BOX; ++b) tma_store_3d(&omap, sm + b * BOX * R, l0, b * BOX, item);
        tma_store_commit_and_drain();
    }
}

// Persistent form: each CTA walks groups g = blockIdx.x, + gridDim.x, ... of R lines, each thread
// transforming a pair of lines (c0 = 2 cp and c0 + 1; the pair shares its twiddle and
// transfer-function loads: every line of an item has the same axis table).  The lines of the next
// group are copied into a staging buffer by the bulk-copy engine (one copy per line, completion
// on an mbarrier, bounded wait) while the current group is transformed; the first stage runs in
// registers while the previous group's tile (which aliases the exchange region) drains through
// its TMA stores.  Needs every line on a 16-byte boundary.
template <int P>
__host__ __device__ constexpr int line_stage_stride() { return P / 2 + 4; }

// exchange / tile region of the persistent form: the pair layout of the 128-bit exchanges
// (P >= 128) or the padded layout, and the dense [position][line] tile, which aliases it (the
// larger of the two)
template <int P, int R>
__host__ __device__ constexpr size_t line_p_xwords() {
    return 2 * (size_t)PairLayout<P, (R / 2 > 0 ? R / 2 : 1)>::SLOTS > line_smem_words<P, R>()
               ? 2 * (size_t)PairLayout<P, (R / 2 > 0 ? R / 2 : 1)>::SLOTS
               : line_smem_words<P, R>();
}

template <int P, int R>
__host__ __device__ constexpr size_t line_p_smem_bytes() {
    return (line_p_xwords<P, R>() + (size_t)R * line_stage_stride<P>()) * sizeof(float2) + sizeof(uint64_t);
}

struct LineGroupArgs {
    const float2* in;
    long long in_item_stride;
    const CUtensorMap* omap;
    const float2* h;
    long long h_item_stride;
    const float4* tw;
    const float2* pre;
    const float2* post;
    float2* stage;
    uint64_t* mbar;
    int conj;
    float scale;
    int groups_per_item;
};

// thread 0: the R lines of group g into the staging buffer (completion on the mbarrier)
template <int P, int R>
__device__ __forceinline__ void line_issue(const LineGroupArgs& A, int g) {
    constexpr int N = P / 2, SST = line_stage_stride<P>();
    const int item = g / A.groups_per_item, l0 = (g % A.groups_per_item) * R;
    const float2* src = A.in + item * A.in_item_stride + (long long)l0 * N;
    mbar_arrive_expect_tx(A.mbar, (unsigned)(R * N * sizeof(float2)));
#pragma unroll 1
    for (int rr = 0; rr < R; ++rr) bulk_load(A.stage + rr * SST, src + rr * N, (unsigned)(N * sizeof(float2)), A.mbar);
}

// One group of R lines (P >= 512): read the staged lines, request the next group's, transform,
// multiply by the axis table, transform back, write the kept half into the tile and store it by
// TMA.  Returns false (every thread) when the staged copy did not land.  A separate function
// keeps the loop's state out of the registers the transform needs.
template <int P, int R, bool FAC>
__device__ __noinline__ bool line_group(const LineGroupArgs& A, int g, int gnext, bool ok) {
    constexpr int T = P / 16, N = P / 2, SST = line_stage_stride<P>(), CP = R / 2;
    constexpr int BOX = N < kTmaBoxCols ? N : kTmaBoxCols;
    extern __shared__ __align__(1024) float2 sm[];
    float4* sx = reinterpret_cast<float4*>(sm);
    const int t = threadIdx.x % T, cp = threadIdx.x / T, c0 = 2 * cp;
    float2 a[16], b[16];
#pragma unroll
    for (int e = 0; e < 8; ++e) {   // stage-0 positions t + e P/16 of lines c0 and c0 + 1
        a[e] = A.stage[c0 * SST + t + e * T];
        b[e] = A.stage[(c0 + 1) * SST + t + e * T];
    }
#pragma unroll
    for (int e = 8; e < 16; ++e) { a[e] = make_float2(0.f, 0.f); b[e] = make_float2(0.f, 0.f); }
    if constexpr (FAC) {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const float2 f = __ldg(A.pre + t + e * T);
            a[e] = cmul(a[e], f);
            b[e] = cmul(b[e], f);
        }
    }
    fence_proxy_async_smem();   // these reads of the staging buffer precede the next bulk copy into it
    if (__syncthreads_or(!ok)) return false;                              // a copy did not land
    if (threadIdx.x == 0 && gnext >= 0) line_issue<P, R>(A, gnext);
    stage_butterflies<P, 0, false, 8>(a);
    stage_butterflies<P, 0, false, 8>(b);
    twiddle2<P, 0, false>(a, b, A.tw, t);
    if (threadIdx.x == 0) tma_store_wait_read();                          // previous tile read out
    __syncthreads();
    xch2v<P, CP, 0, 1>(sx, cp, t, a, b);
    fwd2v_from<P, CP, 1, 8>(a, b, sx, cp, t, A.tw);
    {
        const float2* hh = A.h + (g / A.groups_per_item) * A.h_item_stride + t;
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const float2 w = __ldg(hh + e * T);
            a[e] = A.conj ? cmulc(a[e], w) : cmul(a[e], w);
            b[e] = A.conj ? cmulc(b[e], w) : cmul(b[e], w);
        }
    }
    inv2v_from<P, CP, Geo<P>::NST - 1>(a, b, sx, cp, t, A.tw);
    __syncthreads();   // every exchange read done before the tile (which aliases the region) is written
    // kept positions t + e T (e < 8) of lines c0, c0 + 1: tile words (t + e T) R + c0, + 1
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        float2 x = cscale(a[e], A.scale), y = cscale(b[e], A.scale);
        if constexpr (FAC) {
            const float2 q = __ldg(A.post + t + e * T);
            x = cmul(x, q);
            y = cmul(y, q);
        }
        *reinterpret_cast<float4*>(sm + (t + e * T) * R + c0) = make_float4(x.x, x.y, y.x, y.y);
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
        const int item = g / A.groups_per_item, l0 = (g % A.groups_per_item) * R;
#pragma unroll 1
        for (int bx = 0; bx < N / BOX; ++bx) tma_store_3d(A.omap, sm + bx * BOX * R, l0, bx * BOX, item);
        tma_store_commit();
    }
    return true;
}

template <int P, int R, bool FAC>
__global__ void __launch_bounds__((R / 2) * (P / 16), (R / 2) * (P / 16) >= 512 ? 1 : 2)
k_line_conv_p(const float2* __restrict__ in, long long in_item_stride, const __grid_constant__ CUtensorMap omap,
              const float2* __restrict__ h, long long h_item_stride, int conj, float scale,
              const float4* __restrict__ tw, int groups_per_item, int total_groups, int* status,
              const float2* __restrict__ pre, const float2* __restrict__ post) {
    static_assert(P >= 512, "the persistent line pass needs T >= 32");
    pdl_wait();
    constexpr int SST = line_stage_stride<P>();
    extern __shared__ __align__(1024) float2 sm[];
    LineGroupArgs A;
    A.in = in; A.in_item_stride = in_item_stride; A.omap = &omap; A.h = h; A.h_item_stride = h_item_stride;
    A.tw = tw; A.pre = pre; A.post = post; A.conj = conj; A.scale = scale; A.groups_per_item = groups_per_item;
    A.stage = sm + line_p_xwords<P, R>();
    A.mbar = reinterpret_cast<uint64_t*>(A.stage + R * SST);
    if (threadIdx.x == 0) {
        mbar_init(A.mbar, 1);
        if ((int)blockIdx.x < total_groups) line_issue<P, R>(A, blockIdx.x);
    }
    __syncthreads();
    unsigned parity = 0;
#pragma unroll 1
    for (int g = blockIdx.x; g < total_groups; g += gridDim.x, parity ^= 1u) {
        const bool ok = mbar_wait_bounded(A.mbar, parity, status);
        const int gnext = g + (int)gridDim.x < total_groups ? g + (int)gridDim.x : -1;
        if (!line_group<P, R, FAC>(A, g, gnext, ok)) break;
    }
    if (threadIdx.x == 0) tma_store_wait_read();
}

// Pair form, the column pass's scheme applied to lines: each thread transforms a pair of
// neighbouring lines (they share the twiddle and table loads, since every line of an item has the
// same axis table) loaded straight from global memory with coalesced accesses, CP = R / 2 pairs
// per CTA, the grid (items, line groups) with the item fastest.  Thread 0 prefetches into L2 the
// lines of the CTA that will take this CTA's place (`resident` CTAs later in launch order).  The
// kept half goes through the tile (aliasing the exchange region) and one TMA store per box; the
// CTA waits for the tile to be read before it exits.  Measured per pass against the persistent
// form: 2048^2 fields 33.8 against 36.9 us, 1024^2 7.0 against 8.3, 512^2 1.67 against 1.96.
// (Stores of each pair's 16-byte pieces straight from the registers, one scattered sector per
// lane, took 51 us at 2048^2.)
template <int P> constexpr int line_pairs_per_block() { return line_rows<P>() / 2; }
template <int P, int CP>
constexpr int line_pair_smem_words() {
    constexpr int x = 2 * PairLayout<P, CP>::SLOTS;
    constexpr int tile = 2 * CP * (P / 2);
    return x > tile ? x : tile;
}

template <int P, int CP, bool FAC>
__global__ void __launch_bounds__(CP * (P / 16), CP * (P / 16) >= 512 ? 1 : 2)
k_line_pair(const float2* __restrict__ in, long long in_item_stride, const __grid_constant__ CUtensorMap omap,
            const float2* __restrict__ h, long long h_item_stride, int conj, float scale,
            const float4* __restrict__ tw, const float2* __restrict__ pre, const float2* __restrict__ post,
            int resident) {
    static_assert(P >= 512 && P <= 4096, "the pair form serves 512 <= P <= 4096");
    pdl_wait();
    constexpr int T = P / 16, N = P / 2;
    extern __shared__ __align__(1024) float2 sm[];
    const int t = CP == 1 ? (int)threadIdx.x : (int)threadIdx.x % T;
    const int cp = CP == 1 ? 0 : (int)threadIdx.x / T;
    if (threadIdx.x == 0) {
        const long long nb = (long long)blockIdx.y * gridDim.x + blockIdx.x + resident;
        if (nb < (long long)gridDim.x * gridDim.y) {
            const long long itn = nb % gridDim.x;
            const long long ln = (nb / gridDim.x) * (2 * CP);
            const float2* pn = in + itn * in_item_stride + ln * N;
            if (((uintptr_t)pn & 15) == 0)
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" :: "l"(pn), "r"(2 * CP * N * 8) : "memory");
        }
    }
    const int l = 2 * ((int)blockIdx.y * CP + cp);
    const long long item = blockIdx.x;
    const float2* sa = in + item * in_item_stride + (long long)l * N;
    float2 a[16], b[16];
#pragma unroll
    for (int e = 0; e < 8; ++e) { a[e] = sa[t + e * T]; b[e] = sa[N + t + e * T]; }   // positions < N
#pragma unroll
    for (int e = 8; e < 16; ++e) { a[e] = make_float2(0.f, 0.f); b[e] = make_float2(0.f, 0.f); }
    if constexpr (FAC) {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const float2 f = __ldg(pre + t + e * T);
            a[e] = cmul(a[e], f);
            b[e] = cmul(b[e], f);
        }
    }
    auto mul_h = [&]() {
        const float2* hh = h + item * h_item_stride + t;
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const float2 w = __ldg(hh + e * T);
            a[e] = conj ? cmulc(a[e], w) : cmul(a[e], w);
            b[e] = conj ? cmulc(b[e], w) : cmul(b[e], w);
        }
    };
    fwd2v_from<P, CP, 0, 8>(a, b, reinterpret_cast<float4*>(sm), cp, t, tw);
    mul_h();
    inv2v_from<P, CP, Geo<P>::NST - 1>(a, b, reinterpret_cast<float4*>(sm), cp, t, tw);
    constexpr int R = 2 * CP, BOX = N < kTmaBoxCols ? N : kTmaBoxCols;
    __syncthreads();   // every exchange read done before the tile (which aliases the region) is written
#pragma unroll
    for (int e = 0; e < 8; ++e) {   // kept positions t + e T < N: tile words (t + e T) R + 2 cp, + 1
        float2 x = cscale(a[e], scale), y = cscale(b[e], scale);
        if constexpr (FAC) {
            const float2 q = __ldg(post + t + e * T);
            x = cmul(x, q);
            y = cmul(y, q);
        }
        *reinterpret_cast<float4*>(sm + (t + e * T) * R + 2 * cp) = make_float4(x.x, x.y, y.x, y.y);
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll 1
        for (int bx = 0; bx < N / BOX; ++bx) tma_store_3d(&omap, sm + bx * BOX * R, (int)blockIdx.y * R, bx * BOX, (int)item);
        tma_store_commit_and_drain();
    }
}

// Shared-source z-stack, first pass: each source line is transformed once and its spectrum kept in
// registers; for every plane j it is multiplied by that plane's axis table, transformed back and
// stored into plane j's intermediate (item j of omap).  The second pass is the line pass over the
// planes.  One line per thread (spectrum and working copy: 32 values), R lines per group as in
// line_rows (interleaved over the lanes), persistent with staged bulk loads as k_line_conv_p.
// The exchanges take one barrier each (warp-wide where the threads of one block of the earlier
// stage, R lines of them, fit in a warp), and the kept half goes to one of two tiles of its own,
// so that a plane waits only for the TMA store issued two planes before it.  Per plane: the
// exchange into stage 0 (CTA-wide) and the barrier after the tile write, which also separates
// this plane's last exchange reads from the next plane's first exchange writes.
template <int P, int R>
__host__ __device__ constexpr size_t stack_x_words() {
    return ((size_t)PadLayout<P, R>::WORDS + 127) / 128 * 128;
}
template <int P, int R>
__host__ __device__ constexpr size_t stack_smem_bytes() {
    return (stack_x_words<P, R>() + 2 * (size_t)R * (P / 2) + (size_t)R * line_stage_stride<P>()) * sizeof(float2) +
           sizeof(uint64_t);
}

template <int P, int R>
__global__ void __launch_bounds__(R * (P / 16), 1)
k_line_stack_p(const float2* __restrict__ in, const __grid_constant__ CUtensorMap omap, const float2* __restrict__ h,
               long long h_item_stride, int planes, int conj, float scale, const float4* __restrict__ tw,
               int groups, int* status) {
    static_assert(Geo<P>::NST >= 2 && Geo<P>::stride(0) * R > 32, "the exchange into stage 0 is CTA-wide");
    pdl_wait();
    constexpr int T = P / 16, N = P / 2, NT = R * T, SST = line_stage_stride<P>();
    constexpr int BOX = N < kTmaBoxCols ? N : kTmaBoxCols;
    extern __shared__ __align__(1024) float2 sm[];
    float2* tiles = sm + stack_x_words<P, R>();
    float2* stage = tiles + 2 * R * N;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(stage + R * SST);
    const int r = threadIdx.x % R, t = threadIdx.x / R;
    auto issue = [&](int g) {   // thread 0: the R source lines of group g into the staging buffer
        const float2* src = in + (long long)g * R * N;
        mbar_arrive_expect_tx(mbar, (unsigned)(R * N * sizeof(float2)));
#pragma unroll 1
        for (int rr = 0; rr < R; ++rr) bulk_load(stage + rr * SST, src + rr * N, (unsigned)(N * sizeof(float2)), mbar);
    };
    if (threadIdx.x == 0) {
        mbar_init(mbar, 1);
        if ((int)blockIdx.x < groups) issue(blockIdx.x);
    }
    __syncthreads();
    const TwTable<P> twt{tw, t};
    unsigned parity = 0;
    int np = 0;   // planes stored by this CTA so far: plane tiles alternate
#pragma unroll 1
    for (int g = blockIdx.x; g < groups; g += gridDim.x, parity ^= 1u) {
        const bool ok = mbar_wait_bounded(mbar, parity, status);
        float2 spec[16];
#pragma unroll
        for (int e = 0; e < 8; ++e) spec[e] = stage[r * SST + t + e * T];   // stage-0 positions t + e P/16
#pragma unroll
        for (int e = 8; e < 16; ++e) spec[e] = make_float2(0.f, 0.f);
        fence_proxy_async_smem();   // these reads of the staging buffer precede the next bulk copy into it
        if (__syncthreads_or(!ok)) break;                                // a copy did not land
        if (threadIdx.x == 0 && g + (int)gridDim.x < groups) issue(g + gridDim.x);
        fwd1_from<P, R, 0, 8>(spec, sm, r, t, twt);
#pragma unroll 1
        for (int j = 0; j < planes; ++j, ++np) {
            float2* tile = tiles + (np & 1) * R * N;
            // the store of two planes ago read its tile; the CTA-wide exchange below publishes it
            if (threadIdx.x == 0) tma_store_wait_read_1();
            float2 v[16];
            const float2* hh = h + j * h_item_stride + t;
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const float2 w = __ldg(hh + e * T);
                v[e] = conj ? cmulc(spec[e], w) : cmul(spec[e], w);
            }
            inv1_from<P, R, Geo<P>::NST - 1>(v, sm, r, t, twt);
#pragma unroll
            for (int e = 0; e < 8; ++e) tile[e * NT + threadIdx.x] = cscale(v[e], scale);
            fence_proxy_async_smem();
            __syncthreads();
            if (threadIdx.x == 0) {
#pragma unroll 1
                for (int bx = 0; bx < N / BOX; ++bx) tma_store_3d(&omap, tile + bx * BOX * R, g * R, bx * BOX, j);
                tma_store_commit();
            }
        }
    }
    if (threadIdx.x == 0) tma_store_wait_read();
}

template <int P>
static cudaError_t line_stack_impl(const float2* in, const CUtensorMap* omap, int lines, int planes, const float2* h,
                                   long long h_item_stride, int conj, float scale, const float4* tw, int* status,
                                   cudaStream_t st) {
    constexpr int R = line_rows<P>();
    constexpr int T = P / 16;
    if constexpr (P < 512 || P > 4096) {
        return cudaErrorNotSupported;
    } else {
        if (lines % R || planes < 1 || !status || (uintptr_t)in % 16) return cudaErrorInvalidValue;
        const size_t smem = stack_smem_bytes<P, R>();
        int resident = 0;
        cudaError_t e = kernel_setup<k_line_stack_p<P, R>>(smem, R * T, &resident);
        if (e != cudaSuccess) return e;
        const int groups = lines / R;
        const int grid = std::min(groups, resident);
        if (grid < 1) return cudaErrorInvalidConfiguration;
        return pdl_launch(k_line_stack_p<P, R>, dim3(grid), dim3(R * T), smem, st, in, *omap, h, h_item_stride, planes,
                          conj, scale, tw, groups, status);
    }
}

template <int P, bool FAC>
static cudaError_t line_conv_impl(const float2* in, long long in_item_stride, const CUtensorMap* omap, int lines,
                                  int items, const float2* h, long long h_item_stride, int conj, float scale,
                                  const float4* tw, int* status, const float2* pre, const float2* post,
                                  cudaStream_t st) {
    constexpr int R = line_rows<P>();
    constexpr int T = P / 16;
    if (lines % R || items < 1 || items > 65535) return cudaErrorInvalidValue;
    const bool aligned = ((uintptr_t)in % 16 == 0) && (in_item_stride % 2 == 0);
    if constexpr (P >= 512 && P <= 4096) {
    constexpr int CP = line_pairs_per_block<P>();
    static_assert(2 * CP == R, "a CTA's lines are one box of the output map");
    {
        const size_t smem = (size_t)line_pair_smem_words<P, CP>() * sizeof(float2);
        int resident = 0;
        cudaError_t e = kernel_setup<k_line_pair<P, CP, FAC>>(smem, CP * T, &resident);
        if (e != cudaSuccess) return e;
        return pdl_launch(k_line_pair<P, CP, FAC>, dim3(items, lines / R), dim3(CP * T), smem, st, in,
                          in_item_stride, *omap, h, h_item_stride, conj, scale, tw, pre, post, resident);
    }
    }
    if constexpr (P >= 8192) {
    if (aligned && status) {
        const size_t smem = line_p_smem_bytes<P, R>();
        int resident = 0;
        cudaError_t e = kernel_setup<k_line_conv_p<P, R, FAC>>(smem, (R / 2) * T, &resident);
        if (e != cudaSuccess) return e;
        const int groups = (lines / R) * items;
        const int grid = std::min(groups, resident);
        if (grid > 0)
            return pdl_launch(k_line_conv_p<P, R, FAC>, dim3(grid), dim3((R / 2) * T), smem, st, in, in_item_stride,
                              *omap, h, h_item_stride, conj, scale, tw, lines / R, groups, status, pre, post);
    }
    }
    const size_t smem = line_smem_words<P, R>() * sizeof(float2);
    cudaError_t e = kernel_setup<k_line_conv<P, R, FAC>>(smem, R * T, nullptr);
    if (e != cudaSuccess) return e;
    return pdl_launch(k_line_conv<P, R, FAC>, dim3(lines / R, items), dim3(R * T), smem, st, in, in_item_stride,
                      *omap, h, h_item_stride, conj, scale, tw, pre, post);
}

int line_block_rows(int p) {
    switch (p) {
#define CASE(P) case P: return line_rows<P>();
        CASE(32) CASE(64) CASE(128) CASE(256) CASE(512) CASE(1024) CASE(2048) CASE(4096) CASE(8192)
#undef CASE
        default: return 0;
    }
}

bool line_stack_supported(int p) { return p >= 512 && p <= 4096; }

cudaError_t launch_line_stack(int p, const float2* in, const CUtensorMap* omap, int lines, int planes, const float2* h,
                              long long h_item_stride, int conj, float scale, const float4* tw, int* status,
                              cudaStream_t st) {
    switch (p) {
#define CASE(P) case P: return line_stack_impl<P>(in, omap, lines, planes, h, h_item_stride, conj, scale, tw, status, st);
        CASE(32) CASE(64) CASE(128) CASE(256) CASE(512) CASE(1024) CASE(2048) CASE(4096) CASE(8192)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_line_conv(int p, const float2* in, long long in_item_stride, const CUtensorMap* omap, int lines,
                             int items, const float2* h, long long h_item_stride, int conj, float scale,
                             const float4* tw, int* status, const float2* pre, const float2* post, cudaStream_t st) {
    if (!pre != !post) return cudaErrorInvalidValue;
    switch (p) {
#define CASE(P) case P: return pre ? line_conv_impl<P, true>(in, in_item_stride, omap, lines, items, h, h_item_stride, conj, scale, tw, status, pre, post, st) \
                               : line_conv_impl<P, false>(in, in_item_stride, omap, lines, items, h, h_item_stride, conj, scale, tw, status, nullptr, nullptr, st);
        CASE(32) CASE(64) CASE(128) CASE(256) CASE(512) CASE(1024) CASE(2048) CASE(4096) CASE(8192)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cwo
