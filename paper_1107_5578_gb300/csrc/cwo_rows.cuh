// cwo_rows.cuh -- the two row passes of a propagation (kernels and their launch templates; the
// launchers are instantiated by cwo_rows.cu, cwo_rows_inv_a.cu, cwo_rows_inv_b.cu and
// cwo_rows_turn.cu, which compile in parallel).
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
// through a dense shared-memory tile [st][r]; the tile moves to and from the intermediate as TMA
// tensor boxes of R rows x 256 columns (R * 8 contiguous bytes per column), so the transposed
// global side costs the threads no load/store instructions.
#pragma once
#include <algorithm>

#include "cwo.h"
#include "cwo_debug.h"
#include "cwo_fft.cuh"
#include "cwo_internal.h"
#include "cwo_launch.cuh"
#include "cwo_tma.cuh"
#include "cwo_epilogue.cuh"

namespace cwo {

// Rows per CTA of each pass (measured on GB300).  The forward pass stores its tile, and stores of
// less than a 32-byte sector per column are expensive, so it keeps >= 4 rows where a 4-row tile
// fits (P <= 4096); the inverse pass loads, where 2-row tiles (16 bytes per column, the other half
// of each sector served from L2 to the neighbouring CTA) allow more CTAs per SM.  A TMA box must
// span at least 16 contiguous bytes, hence >= 2 rows.
template <int P> constexpr int rows_fwd() { return P >= 256 ? 4 : 8; }
// at P = 8192 a CTA holds 2 rows (a pair per thread, 512 threads, 139 KB of exchange space): a
// cluster of two CTAs forms each 4-row group, so that every stored column piece is a whole
// 32-byte sector
template <int P> constexpr bool rows_fwd_cluster() { return P >= 8192; }
template <int P> constexpr int rows_inv() { return P >= 4096 ? 2 : (P >= 256 ? 4 : 8); }
constexpr bool kRowInvPersistent = true;   // measured: 25.4 -> 23.0 us per 2048^2 field

template <int P, int R>
__host__ __device__ constexpr size_t row_smem_words() {
    return PadLayout<P, R>::WORDS > (size_t)R * P ? PadLayout<P, R>::WORDS : (size_t)R * P;
}

// Lanes are row-fastest (thread = r + R t): the FFT exchanges then see R interleaved transforms,
// for which the padded layout is conflict free, and the dense tile [st][r] used by the transposing
// copies is addressed as e * (R T) + threadIdx.x, i.e. consecutive words across a warp.

template <int P, int R, bool PRE>
__global__ void __launch_bounds__(R * (P / 16))
k_row_fwd(const float2* __restrict__ in, long long in_item_stride, const __grid_constant__ CUtensorMap wmap,
          int item_off, const float4* __restrict__ tw, const Prefactor pre) {
    pdl_wait();
    constexpr int T = P / 16, N = P / 2, NT = R * T;
    constexpr int BOX = P < kTmaBoxCols ? P : kTmaBoxCols;
    extern __shared__ __align__(1024) float2 sm[];
    const int r = threadIdx.x % R, t = threadIdx.x / R;
    const int y0 = blockIdx.x * R;
    const int item = blockIdx.y;
    const float2* src = in + item * in_item_stride + (long long)(y0 + r) * N;
    float2 v[16];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = __ldg(src + t + e * T);   // DIF stage-0 positions t + e P/16
#pragma unroll
    for (int e = 8; e < 16; ++e) v[e] = make_float2(0.f, 0.f);   // zero padding, never loaded
    if constexpr (PRE) {
        const float2 fy = __ldg(pre.fy + y0 + r);
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = cmul(v[e], cmul(__ldg(pre.fx + t + e * T), fy));
    }
    fwd1_from<P, R, 0, 8>(v, sm, r, t, TwTable<P>{tw, t});
    if constexpr (Geo<P>::NST > 1) __syncthreads();   // every exchange read done before the tile is written
    // dense tile [st][r]: register e of (r, t) is storage column st = e T + t of row y0 + r
#pragma unroll
    for (int e = 0; e < 16; ++e) sm[e * NT + threadIdx.x] = v[e];
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {   // R rows x BOX columns per box: R * 8 contiguous bytes per column
#pragma unroll 1
        for (int b = 0; b < P / BOX; ++b) tma_store_3d(&wmap, sm + b * BOX * R, y0, b * BOX, item + item_off);
        tma_store_commit_and_drain();
    }
}

template <int P, int R, int EPI>
__global__ void __launch_bounds__(R * (P / 16))
k_row_inv(const __grid_constant__ CUtensorMap wmap, int item_off, float2* __restrict__ out,
          long long out_item_stride, float scale, const float4* __restrict__ tw, int* status, const Epilogue ep) {
    pdl_wait();
    constexpr int T = P / 16, N = P / 2, NT = R * T;
    constexpr int BOX = P < kTmaBoxCols ? P : kTmaBoxCols;
    extern __shared__ __align__(1024) float2 sm[];
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + row_smem_words<P, R>());   // after the tile
    const int r = threadIdx.x % R, t = threadIdx.x / R;
    const int y0 = blockIdx.x * R;
    const int item = blockIdx.y;
    if (threadIdx.x == 0) mbar_init(mbar, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(mbar, (unsigned)(R * P * sizeof(float2)));
#pragma unroll 1
        for (int b = 0; b < P / BOX; ++b) tma_load_3d(sm + b * BOX * R, &wmap, mbar, y0, b * BOX, item + item_off);
    }
    const bool ok = mbar_wait_bounded(mbar, 0, status);
    float2 v[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = sm[e * NT + threadIdx.x];
    if (__syncthreads_or(!ok)) return;             // a copy did not land: the status word says so
    inv1_from<P, R, Geo<P>::NST - 1>(v, sm, r, t, TwTable<P>{tw, t});
    const long long base = item * out_item_stride + (long long)(y0 + r) * N;
#pragma unroll
    for (int e = 0; e < 8; ++e) epilogue_store<EPI>(out, ep, base + t + e * T, t + e * T, y0 + r, cscale(v[e], scale));   // crop
}

// ------------------------------------------------------------------------------------------
// Persistent row passes: one CTA per SM (or as many as fit) walks groups g = blockIdx.x,
// + gridDim.x, ... of R rows, so that the memory traffic of one group overlaps the FFT of another.
//
// Forward: the R input rows of the NEXT group are copied into a staging buffer by the bulk-copy
// engine (one contiguous copy per row, completion on an mbarrier) while the current group is
// transformed; the transposed tile of a group is written out by TMA stores that drain while the
// next group's input is read from the staging buffer.  Shared memory: exchange region / tile
// (row_smem_words), staging R x (N + 4) (row stride padded so the r-fast reads hit distinct
// banks), one mbarrier.
// ------------------------------------------------------------------------------------------
template <int P, int R>
__host__ __device__ constexpr int stage_stride() { return P / 2 + 4; }

template <int P, int R>
__host__ __device__ constexpr size_t row_fwd_p_smem_bytes() {
    return (row_smem_words<P, R>() + (size_t)R * stage_stride<P, R>()) * sizeof(float2) + sizeof(uint64_t);
}

template <int P, int R, bool PRE>
// two CTAs per SM where a CTA has fewer than 1024 threads (1024^2 fields: 5.8 -> 5.3 us per field)
__global__ void __launch_bounds__(R * (P / 16), R * (P / 16) >= 1024 ? 1 : 2)
k_row_fwd_p(const float2* __restrict__ in, long long in_item_stride, const __grid_constant__ CUtensorMap wmap,
            int item_off, int groups_per_item, int total_groups, const float4* __restrict__ tw, int* status,
            const Prefactor pre) {
    pdl_wait();
    constexpr int T = P / 16, N = P / 2, NT = R * T, SST = stage_stride<P, R>();
    constexpr int BOX = P < kTmaBoxCols ? P : kTmaBoxCols;
    extern __shared__ __align__(1024) float2 sm[];
    float2* stage = sm + row_smem_words<P, R>();
    uint64_t* mbar = reinterpret_cast<uint64_t*>(stage + R * SST);
    const int r = threadIdx.x % R, t = threadIdx.x / R;
    auto issue = [&](int g) {   // thread 0: the R rows of group g into the staging buffer
        const int item = g / groups_per_item, y0 = (g % groups_per_item) * R;
        const float2* src = in + item * in_item_stride + (long long)y0 * N;
        mbar_arrive_expect_tx(mbar, (unsigned)(R * N * sizeof(float2)));
#pragma unroll 1
        for (int rr = 0; rr < R; ++rr) bulk_load(stage + rr * SST, src + rr * N, (unsigned)(N * sizeof(float2)), mbar);
    };
    if (threadIdx.x == 0) {
        mbar_init(mbar, 1);
        if ((int)blockIdx.x < total_groups) issue(blockIdx.x);
    }
    __syncthreads();
    unsigned parity = 0;
#pragma unroll 1
    for (int g = blockIdx.x; g < total_groups; g += gridDim.x, parity ^= 1u) {
        const bool ok = mbar_wait_bounded(mbar, parity, status);
        float2 v[16];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = stage[r * SST + t + e * T];   // DIF stage-0 positions t + e P/16
#pragma unroll
        for (int e = 8; e < 16; ++e) v[e] = make_float2(0.f, 0.f);      // zero padding, never loaded
        if constexpr (PRE) {
            const float2 fy = __ldg(pre.fy + (g % groups_per_item) * R + r);
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = cmul(v[e], cmul(__ldg(pre.fx + t + e * T), fy));
        }
        fence_proxy_async_smem();   // these reads of the staging buffer precede the next bulk copy into it
        if (__syncthreads_or(!ok)) break;                                // a copy did not land
        if (threadIdx.x == 0 && g + (int)gridDim.x < total_groups) issue(g + gridDim.x);
        // first stage in registers while the previous tile's stores drain; the exchange region
        // (which the tile aliases) is rewritten only after the drain
        const TwTable<P> twt{tw, t};
        stage_butterflies<P, 0, false, 8>(v);
        if constexpr (Geo<P>::NST > 1) twt.template apply<0, false>(v);
        if (threadIdx.x == 0) tma_store_wait_read();
        __syncthreads();
        if constexpr (Geo<P>::NST > 1) {
            xch1<P, R, 0, 1>(sm, r, t, v);
            fwd1_from<P, R, 1, 8>(v, sm, r, t, twt);
            __syncthreads();   // every exchange read done before the tile (which aliases the region) is written
        }
#pragma unroll
        for (int e = 0; e < 16; ++e) sm[e * NT + threadIdx.x] = v[e];
        fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            const int item = g / groups_per_item, y0 = (g % groups_per_item) * R;
#pragma unroll 1
            for (int b = 0; b < P / BOX; ++b) tma_store_3d(&wmap, sm + b * BOX * R, y0, b * BOX, item + item_off);
            tma_store_commit();
        }
    }
    if (threadIdx.x == 0) tma_store_wait_read();
}

// Forward, cluster pair (P = 8192): CTA rank q of a two-CTA cluster transforms rows y0 + 2q and
// y0 + 2q + 1 of a 4-row group, one thread per pair of rows (the two rows share every twiddle
// load and move with 128-bit exchanges).  After both CTAs have finished their FFT exchanges
// (cluster barrier), every thread writes both rows' values of each of its storage columns with one
// 16-byte store into the 4-row tile of the CTA that stores that column half -- its own half
// locally, the other half into the partner's shared memory -- and after a second cluster barrier
// each CTA stores its [P/2 columns][4 rows] tile by TMA: 32 contiguous bytes per column.  Both
// CTAs execute the same sequence of cluster barriers on every path (a bounded wait that expires
// leaves the status bit set and the loop running), so neither can wait for a partner that has
// left.  BULK: the rows are staged by bulk copies (16-byte aligned input); otherwise each thread
// loads its own samples.  Measured against one row per thread (1024 threads, 8-byte tile stores):
// 156.5 against 168.3 us per 4096^2 field.
template <int P>
__host__ __device__ constexpr size_t row_fwd_c_xwords() { return 2 * (size_t)PairLayout<P, 1>::SLOTS; }
template <int P>
__host__ __device__ constexpr size_t row_fwd_c_smem_bytes() {
    return (row_fwd_c_xwords<P>() + 2 * (size_t)stage_stride<P, 2>()) * sizeof(float2) + sizeof(uint64_t);
}

template <int P, bool PRE, bool BULK>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(P / 16, 1)
k_row_fwd_c(const float2* __restrict__ in, long long in_item_stride, const __grid_constant__ CUtensorMap wmap,
             int item_off, int groups_per_item, int total_groups, const float4* __restrict__ tw, int* status,
             const Prefactor pre) {
    pdl_wait();
    constexpr int T = P / 16, N = P / 2, SST = stage_stride<P, 2>(), HALF = P / 2;
    constexpr int BOX = kTmaBoxCols;
    constexpr size_t XW = row_fwd_c_xwords<P>();
    static_assert(XW >= (size_t)4 * HALF, "the 4-row half tile fits the exchange region");
    extern __shared__ __align__(1024) float2 sm[];
    float4* sx = reinterpret_cast<float4*>(sm);
    float2* stage = sm + XW;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(stage + 2 * SST);
    const unsigned rank = cluster_ctarank();
    const unsigned tile_remote = cluster_map(smem_u32(sm), rank ^ 1u);
    const int t = threadIdx.x;
    const int cl = blockIdx.x / 2, ncl = gridDim.x / 2;
    auto src_rows = [&](int g) {   // first of this CTA's two rows of group g
        const int item = g / groups_per_item, y0 = (g % groups_per_item) * 4 + 2 * (int)rank;
        return in + item * in_item_stride + (long long)y0 * N;
    };
    auto issue = [&](int g) {
        const float2* src = src_rows(g);
        mbar_arrive_expect_tx(mbar, (unsigned)(2 * N * sizeof(float2)));
        bulk_load(stage, src, (unsigned)(N * sizeof(float2)), mbar);
        bulk_load(stage + SST, src + N, (unsigned)(N * sizeof(float2)), mbar);
    };
    if (threadIdx.x == 0) {
        mbar_init(mbar, 1);
        if (BULK && cl < total_groups) issue(cl);
    }
    __syncthreads();
    unsigned parity = 0;
#pragma unroll 1
    for (int g = cl; g < total_groups; g += ncl, parity ^= 1u) {
        float2 a[16], b[16];
        if constexpr (BULK) {
            mbar_wait_bounded(mbar, parity, status);     // on expiry: status bit set, loop continues
#pragma unroll
            for (int e = 0; e < 8; ++e) { a[e] = stage[t + e * T]; b[e] = stage[SST + t + e * T]; }
            fence_proxy_async_smem();
        } else {
            const float2* src = src_rows(g);
#pragma unroll
            for (int e = 0; e < 8; ++e) { a[e] = __ldg(src + t + e * T); b[e] = __ldg(src + N + t + e * T); }
        }
#pragma unroll
        for (int e = 8; e < 16; ++e) { a[e] = make_float2(0.f, 0.f); b[e] = make_float2(0.f, 0.f); }
        if constexpr (PRE) {
            const int yr = (g % groups_per_item) * 4 + 2 * (int)rank;
            const float2 fy0 = __ldg(pre.fy + yr), fy1 = __ldg(pre.fy + yr + 1);
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const float2 fx = __ldg(pre.fx + t + e * T);
                a[e] = cmul(a[e], cmul(fx, fy0));
                b[e] = cmul(b[e], cmul(fx, fy1));
            }
        }
        __syncthreads();
        if (BULK && threadIdx.x == 0 && g + ncl < total_groups) issue(g + ncl);
        stage_butterflies<P, 0, false, 8>(a);
        stage_butterflies<P, 0, false, 8>(b);
        twiddle2<P, 0, false>(a, b, tw, t);
        if (threadIdx.x == 0) tma_store_wait_read();     // this CTA's previous tile read out
        __syncthreads();
        xch2v<P, 1, 0, 1>(sx, 0, t, a, b);
        fwd2v_from<P, 1, 1, 8>(a, b, sx, 0, t, tw);
        cluster_sync();   // both exchange regions free (every exchange read done); both previous tiles read out
#pragma unroll
        for (int e = 0; e < 16; ++e) {   // storage column e T + t lies in half e / 8; rows 2 rank, + 1
            const int q = ((e & 7) * T + t) * 2 + (int)rank;   // float4 slot of the 4-row tile
            const float4 w = make_float4(a[e].x, a[e].y, b[e].x, b[e].y);
            if ((e >> 3) == (int)rank) sx[q] = w;
            else st_cluster4(tile_remote + (unsigned)(q * sizeof(float4)), w);
        }
        fence_proxy_async_cluster();
        cluster_sync();   // every value of both tiles written
        if (threadIdx.x == 0) {
            const int item = g / groups_per_item, y0 = (g % groups_per_item) * 4;
#pragma unroll 1
            for (int bb = 0; bb < HALF / BOX; ++bb)
                tma_store_3d(&wmap, sm + bb * BOX * 4, y0, (int)rank * HALF + bb * BOX, item + item_off);
            tma_store_commit();
        }
    }
    if (threadIdx.x == 0) tma_store_wait_read();
    cluster_sync();   // no CTA leaves while its partner may still use its shared memory
}

// Inverse, persistent: R rows per group, one tile buffer.  The tile of the NEXT group is
// requested as soon as the last exchange of the current group has been read back, so its load
// overlaps the last stage, the crop and the stores of the current group.
template <int P, int R> constexpr int row_inv_p_min_blocks() { return R * (P / 16) >= 1024 ? 1 : 1024 / (R * (P / 16)); }

template <int P, int R, int EPI>
__global__ void __launch_bounds__(R * (P / 16), row_inv_p_min_blocks<P, R>())
k_row_inv_p(const __grid_constant__ CUtensorMap wmap, int item_off, float2* __restrict__ out,
            long long out_item_stride, int groups_per_item, int total_groups, float scale,
            const float4* __restrict__ tw, int* status, const Epilogue ep) {
    pdl_wait();
    constexpr int T = P / 16, N = P / 2, NT = R * T;
    constexpr int BOX = P < kTmaBoxCols ? P : kTmaBoxCols;
    static_assert(Geo<P>::NST >= 2, "at least two stages");
    extern __shared__ __align__(1024) float2 sm[];
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + row_smem_words<P, R>());   // after the tile
    const int r = threadIdx.x % R, t = threadIdx.x / R;
    auto issue = [&](int g) {   // thread 0: the R-row tile of group g
        const int item = g / groups_per_item, y0 = (g % groups_per_item) * R;
        mbar_arrive_expect_tx(mbar, (unsigned)(R * P * sizeof(float2)));
#pragma unroll 1
        for (int b = 0; b < P / BOX; ++b) tma_load_3d(sm + b * BOX * R, &wmap, mbar, y0, b * BOX, item + item_off);
    };
    if (threadIdx.x == 0) {
        mbar_init(mbar, 1);
        if ((int)blockIdx.x < total_groups) issue(blockIdx.x);
    }
    __syncthreads();
    const TwTable<P> twt{tw, t};
    unsigned parity = 0;
#pragma unroll 1
    for (int g = blockIdx.x; g < total_groups; g += gridDim.x, parity ^= 1u) {
        const bool ok = mbar_wait_bounded(mbar, parity, status);
        float2 v[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) v[e] = sm[e * NT + threadIdx.x];
        if (__syncthreads_or(!ok)) break;          // a copy did not land: the status word says so
        inv1_to_stage0<P, R, Geo<P>::NST - 1>(v, sm, r, t, twt);
        fence_proxy_async_smem();                  // the exchange reads precede the next tile load
        __syncthreads();
        if (threadIdx.x == 0 && g + (int)gridDim.x < total_groups) issue(g + gridDim.x);
        twt.template apply<0, true>(v);
        stage_butterflies<P, 0, true, 16>(v);
        const int item = g / groups_per_item, y0 = (g % groups_per_item) * R;
        const long long base = item * out_item_stride + (long long)(y0 + r) * N;
#pragma unroll
        for (int e = 0; e < 8; ++e) epilogue_store<EPI>(out, ep, base + t + e * T, t + e * T, y0 + r, cscale(v[e], scale));   // crop
    }
}



// Inverse, pair form (P = 8192): each thread transforms two rows of the group (2 cp and 2 cp + 1
// of its CP = R / 2 pairs), which share every twiddle load, and moves both rows' values at one
// position with one 128-bit access -- in the tile read (the tile [st][r] holds the pair at
// st R + 2 cp, + 1) and in the exchanges (PairLayout, one barrier each).  Otherwise as
// k_row_inv_p: one tile buffer aliasing the exchange region, the next group's tile requested after
// the last exchange.  Measured per field against k_row_inv_p: 4096^2 159.6 against 171.5 us; at
// 2048^2 (24.2 against 23.0 us) and 1024^2 (5.85 against 5.70) the half as many warps per SM cost
// more than the shared twiddle loads save.
template <int P, int CP>
__host__ __device__ constexpr size_t row_inv_pp_words() {
    return 2 * (size_t)PairLayout<P, CP>::SLOTS > (size_t)2 * CP * P ? 2 * (size_t)PairLayout<P, CP>::SLOTS
                                                                       : (size_t)2 * CP * P;
}

template <int P, int CP, int EPI>
__global__ void __launch_bounds__(CP * (P / 16), CP * (P / 16) >= 512 ? 1 : 2)
k_row_inv_pp(const __grid_constant__ CUtensorMap wmap, int item_off, float2* __restrict__ out,
             long long out_item_stride, int groups_per_item, int total_groups, float scale,
             const float4* __restrict__ tw, int* status, const Epilogue ep) {
    pdl_wait();
    constexpr int R = 2 * CP, T = P / 16, N = P / 2;
    constexpr int BOX = P < kTmaBoxCols ? P : kTmaBoxCols;
    static_assert(Geo<P>::NST >= 2 && P >= 128, "at least two stages, 128-bit pair exchanges");
    extern __shared__ __align__(1024) float2 sm[];
    float4* sx = reinterpret_cast<float4*>(sm);
    const float4* tile = reinterpret_cast<const float4*>(sm);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + row_inv_pp_words<P, CP>());
    const int t = CP == 1 ? (int)threadIdx.x : (int)threadIdx.x % T;
    const int cp = CP == 1 ? 0 : (int)threadIdx.x / T;
    auto issue = [&](int g) {   // thread 0: the R-row tile of group g
        const int item = g / groups_per_item, y0 = (g % groups_per_item) * R;
        mbar_arrive_expect_tx(mbar, (unsigned)(R * P * sizeof(float2)));
#pragma unroll 1
        for (int b = 0; b < P / BOX; ++b) tma_load_3d(sm + b * BOX * R, &wmap, mbar, y0, b * BOX, item + item_off);
    };
    if (threadIdx.x == 0) {
        mbar_init(mbar, 1);
        if ((int)blockIdx.x < total_groups) issue(blockIdx.x);
    }
    __syncthreads();
    unsigned parity = 0;
#pragma unroll 1
    for (int g = blockIdx.x; g < total_groups; g += gridDim.x, parity ^= 1u) {
        const bool ok = mbar_wait_bounded(mbar, parity, status);
        float2 a[16], b[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const float4 q = tile[(e * T + t) * CP + cp];
            a[e] = make_float2(q.x, q.y);
            b[e] = make_float2(q.z, q.w);
        }
        if (__syncthreads_or(!ok)) break;          // a copy did not land: the status word says so
        inv2v_to_stage0<P, CP, Geo<P>::NST - 1>(a, b, sx, cp, t, tw);
        fence_proxy_async_smem();                  // the exchange reads precede the next tile load
        __syncthreads();
        if (threadIdx.x == 0 && g + (int)gridDim.x < total_groups) issue(g + gridDim.x);
        twiddle2<P, 0, true>(a, b, tw, t);
        stage_butterflies<P, 0, true, 16>(a);
        stage_butterflies<P, 0, true, 16>(b);
        const int item = g / groups_per_item, y0 = (g % groups_per_item) * R + 2 * cp;
        const long long base = item * out_item_stride + (long long)y0 * N;
#pragma unroll
        for (int e = 0; e < 8; ++e) {   // crop: positions t + e T < N of rows y0 and y0 + 1
            epilogue_store<EPI>(out, ep, base + t + e * T, t + e * T, y0, cscale(a[e], scale));
            epilogue_store<EPI>(out, ep, base + N + t + e * T, t + e * T, y0 + 1, cscale(b[e], scale));
        }
    }
}

// Turn (P <= 4096): the inverse row pass of one propagation and the forward row pass of the next
// in one kernel, for loops that constrain the field between propagations (the GS iteration of
// Section "GS algorithm").  A CTA loads its R rows of the intermediate by TMA, takes their
// inverse FFTs, crops to the Nx kept samples, scales, applies the constraint (EPI_PHASE or
// EPI_AMPLITUDE), zero-pads and takes the forward FFTs, and stores the R rows back into the same
// place of the intermediate by TMA (in place: no other CTA touches these rows).  The inverse
// ends with register e of thread t at position t + e T, which is where the forward's first
// stage takes its inputs, so the crop, constraint and padding act on the registers and no
// exchange is added; each row's arithmetic is that of k_row_inv_p followed by k_row_fwd_p, so
// the loop computes bit for bit what the separate passes compute through the stored field.
template <int P, int R, int EPI>
__global__ void __launch_bounds__(R * (P / 16))
k_row_turn(const __grid_constant__ CUtensorMap wmap, int groups_per_item, long long field_item_stride,
           float scale, const float4* __restrict__ tw, int* status, const Epilogue ep) {
    pdl_wait();
    constexpr int T = P / 16, N = P / 2, NT = R * T;
    constexpr int BOX = P < kTmaBoxCols ? P : kTmaBoxCols;
    static_assert(Geo<P>::NST >= 2, "at least two stages");
    extern __shared__ __align__(1024) float2 sm[];
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + row_smem_words<P, R>());   // after the tile
    const int r = threadIdx.x % R, t = threadIdx.x / R;
    const int g = blockIdx.x, item = g / groups_per_item, y0 = (g % groups_per_item) * R;
    if (threadIdx.x == 0) {
        mbar_init(mbar, 1);
        mbar_arrive_expect_tx(mbar, (unsigned)(R * P * sizeof(float2)));
#pragma unroll 1
        for (int b = 0; b < P / BOX; ++b) tma_load_3d(sm + b * BOX * R, &wmap, mbar, y0, b * BOX, item);
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(mbar, 0, status);
    float2 v[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = sm[e * NT + threadIdx.x];
    if (__syncthreads_or(!ok)) return;         // a copy did not land: the status word says so
    const TwTable<P> twt{tw, t};
    inv1_to_stage0<P, R, Geo<P>::NST - 1>(v, sm, r, t, twt);
    twt.template apply<0, true>(v);
    stage_butterflies<P, 0, true, 16>(v);
    const long long base = item * field_item_stride + (long long)(y0 + r) * N;
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = epilogue_value<EPI>(ep, base + t + e * T, cscale(v[e], scale));
#pragma unroll
    for (int e = 8; e < 16; ++e) v[e] = make_float2(0.f, 0.f);   // zero padding of the next transform
    // forward: the first exchange writes the positions this thread read in the last one
    fwd1_from<P, R, 0, 8>(v, sm, r, t, twt);
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

template <int P, int EPI>
static cudaError_t row_turn_impl(const CUtensorMap* wmap, int ny, int items, long long field_item_stride, float scale,
                                 const float4* tw, int* status, const Epilogue& ep, cudaStream_t st) {
    if constexpr (P > 4096 || P < 64) {
        return cudaErrorNotSupported;
    } else {
        constexpr int R = rows_fwd<P>();
        constexpr int T = P / 16;
        if (ny % R || items < 1 || !status) return cudaErrorInvalidValue;
        const size_t smem = row_smem_words<P, R>() * sizeof(float2) + sizeof(uint64_t);
        cudaError_t e = kernel_setup<k_row_turn<P, R, EPI>>(smem, R * T, nullptr);
        if (e != cudaSuccess) return e;
        const int groups = ny / R;
        return pdl_launch(k_row_turn<P, R, EPI>, dim3((unsigned)(groups * items)), dim3(R * T), smem, st, *wmap, groups,
                          field_item_stride, scale, tw, status, ep);
    }
}

template <int P, bool PRE, bool BULK>
static cudaError_t row_fwd_c_launch(const float2* in, long long in_item_stride, const CUtensorMap* wmap, int item_off,
                                    int ny, int items, const float4* tw, int* status, const Prefactor& pre,
                                    cudaStream_t st) {
    constexpr int T = P / 16;
    const int groups = (ny / 4) * items;
    int clusters = 0;
    const size_t smem = row_fwd_c_smem_bytes<P>();
    cudaError_t e = cluster_setup<k_row_fwd_c<P, PRE, BULK>>(smem, T, &clusters);
    if (e != cudaSuccess) return e;
    if (clusters < 1) return cudaErrorInvalidConfiguration;
    const int grid = 2 * std::min(groups, clusters);
    return pdl_launch(k_row_fwd_c<P, PRE, BULK>, dim3(grid), dim3(T), smem, st, in, in_item_stride, *wmap, item_off,
                      ny / 4, groups, tw, status, pre);
}

template <int P, bool PRE>
static cudaError_t row_fwd_impl_t(const float2* in, long long in_item_stride, const CUtensorMap* wmap,
                                  int item_off, int ny, int items, const float4* tw, int* status, const Prefactor& pre,
                                  cudaStream_t st) {
    constexpr int R = rows_fwd<P>();
    constexpr int T = P / 16;
    if (ny % R) return cudaErrorInvalidValue;
    // persistent pipelined kernel where its bulk copies are legal: rows start on 16-byte boundaries
    const bool aligned = ((uintptr_t)in % 16 == 0) && (in_item_stride % 2 == 0);
    if constexpr (rows_fwd_cluster<P>()) {
        return aligned ? row_fwd_c_launch<P, PRE, true>(in, in_item_stride, wmap, item_off, ny, items, tw, status, pre, st)
                       : row_fwd_c_launch<P, PRE, false>(in, in_item_stride, wmap, item_off, ny, items, tw, status, pre, st);
    } else {
    if (P >= 512 && aligned) {
        const size_t smem = row_fwd_p_smem_bytes<P, R>();
        int resident = 0;
        cudaError_t e = kernel_setup<k_row_fwd_p<P, R, PRE>>(smem, R * T, &resident);
        if (e != cudaSuccess) return e;
        const int groups = (ny / R) * items;
        const int grid = std::min(groups, resident);
        if (grid > 0) {
            return pdl_launch(k_row_fwd_p<P, R, PRE>, dim3(grid), dim3(R * T), smem, st, in, in_item_stride, *wmap,
                              item_off, ny / R, groups, tw, status, pre);
        }
    }
    const size_t smem = row_smem_words<P, R>() * sizeof(float2);
    cudaError_t e = kernel_setup<k_row_fwd<P, R, PRE>>(smem, R * T, nullptr);
    if (e != cudaSuccess) return e;
    dim3 grid(ny / R, items);
    return pdl_launch(k_row_fwd<P, R, PRE>, grid, dim3(R * T), smem, st, in, in_item_stride, *wmap, item_off, tw, pre);
    }
}

template <int P>
static cudaError_t row_fwd_impl(const float2* in, long long in_item_stride, const CUtensorMap* wmap,
                                int item_off, int ny, int items, const float4* tw, int* status, const Prefactor& pre,
                                cudaStream_t st) {
    if (pre.fx || pre.fy) {
        if (!pre.fx || !pre.fy) return cudaErrorInvalidValue;
        return row_fwd_impl_t<P, true>(in, in_item_stride, wmap, item_off, ny, items, tw, status, pre, st);
    }
    return row_fwd_impl_t<P, false>(in, in_item_stride, wmap, item_off, ny, items, tw, status, pre, st);
}

template <int P, int EPI>
static cudaError_t row_inv_impl_e(const CUtensorMap* wmap, int item_off, float2* out, long long out_item_stride,
                                  int ny, int items, float scale, const float4* tw, int* status, const Epilogue& ep,
                                  cudaStream_t st) {
    constexpr int R = rows_inv<P>();
    constexpr int T = P / 16;
    const size_t smem = row_smem_words<P, R>() * sizeof(float2) + sizeof(uint64_t);   // tile + mbarrier
    if (ny % R) return cudaErrorInvalidValue;
    if constexpr (P >= 8192 && R % 2 == 0) {
        constexpr int CP = R / 2;
        const size_t psmem = row_inv_pp_words<P, CP>() * sizeof(float2) + sizeof(uint64_t);
        int resident = 0;
        cudaError_t e = kernel_setup<k_row_inv_pp<P, CP, EPI>>(psmem, CP * T, &resident);
        if (e != cudaSuccess) return e;
        const int groups = (ny / R) * items;
        const int grid = std::min(groups, resident);
        if (grid > 0)
            return pdl_launch(k_row_inv_pp<P, CP, EPI>, dim3(grid), dim3(CP * T), psmem, st, *wmap, item_off, out,
                              out_item_stride, ny / R, groups, scale, tw, status, ep);
    }
    if constexpr (kRowInvPersistent && P >= 512) {
        int resident = 0;
        cudaError_t e = kernel_setup<k_row_inv_p<P, R, EPI>>(smem, R * T, &resident);
        if (e != cudaSuccess) return e;
        const int groups = (ny / R) * items;
        const int grid = std::min(groups, resident);
        if (grid > 0) {
            return pdl_launch(k_row_inv_p<P, R, EPI>, dim3(grid), dim3(R * T), smem, st, *wmap, item_off, out,
                              out_item_stride, ny / R, groups, scale, tw, status, ep);
        }
    }
    cudaError_t e = kernel_setup<k_row_inv<P, R, EPI>>(smem, R * T, nullptr);
    if (e != cudaSuccess) return e;
    dim3 grid(ny / R, items);
    return pdl_launch(k_row_inv<P, R, EPI>, grid, dim3(R * T), smem, st, *wmap, item_off, out, out_item_stride, scale, tw,
                      status, ep);
}

template <int P>
static cudaError_t row_inv_impl(const CUtensorMap* wmap, int item_off, float2* out, long long out_item_stride,
                                int ny, int items, float scale, const float4* tw, int* status, const Epilogue& ep,
                                cudaStream_t st) {
    switch (ep.mode) {
        case EPI_NONE: return row_inv_impl_e<P, EPI_NONE>(wmap, item_off, out, out_item_stride, ny, items, scale, tw, status, ep, st);
        case EPI_PHASE: return row_inv_impl_e<P, EPI_PHASE>(wmap, item_off, out, out_item_stride, ny, items, scale, tw, status, ep, st);
        case EPI_AMPLITUDE:
            return row_inv_impl_e<P, EPI_AMPLITUDE>(wmap, item_off, out, out_item_stride, ny, items, scale, tw, status, ep, st);
        case EPI_INTENSITY:
            return row_inv_impl_e<P, EPI_INTENSITY>(wmap, item_off, out, out_item_stride, ny, items, scale, tw, status, ep, st);
        case EPI_SEPARABLE:
            return row_inv_impl_e<P, EPI_SEPARABLE>(wmap, item_off, out, out_item_stride, ny, items, scale, tw, status, ep, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cwo
