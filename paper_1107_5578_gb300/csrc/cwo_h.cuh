// cwo_h.cuh -- per-element angular-spectrum transfer function from the per-axis tables.
//
// H_A = exp(i z sqrt(k^2 - 4 pi^2 (fx^2 + fy^2))) (Eq. ang2) with the phase in cycles written as
// psi = K sqrt(1 - s), K = z / lambda, s = a_x + a_y, a = lambda^2 f^2, and split exactly as
//     K sqrt(1-s) = K - [K a_x/2 + K a_x^2/8] - [K a_y/2 + K a_y^2/8] - K a_x a_y / 4 - tail,
//     tail = K s^3 (3 + q) / (8 (1 + q)^3),  q = sqrt(1 - s).
// Table entry (float4) per axis index: {a, W (- frac K on x), u_hi, u_lo} with
// W = frac(K a/2 + K a^2/8) and u_hi + u_lo = sign * sqrt|K| / 2 * a, all computed in FP64.
// The cross term K a_x a_y / 4 = u_x u_y (up to ~12 cycles) is formed as a float-float product
// whose integer part is removed exactly; the tail is < 1 cycle at every studied size.
#pragma once
#include "cwo_fft.cuh"
#include "cwo_internal.h"
#include <math.h>

namespace cwo {

// Tail term K s^3 (3 + q) / (8 (1 + q)^3), q = sqrt(1 - s).
//   POLY: its Taylor series K (s^3/16 + 5 s^4/128 + 7 s^5/256 + 21 s^6/1024 + 33 s^7/2048)
//         (the coefficients of sqrt(1 - s) = sum_n C(1/2, n) (-s)^n); a plan uses it only where
//         the first omitted term K 429 s^8 / 32768 stays below 1e-8 cycle.
//   exact: the closed form (one square root and one division).
template <bool POLY>
CWO_HD float asm_tail(float s, float K) {
    if constexpr (POLY) {
        const float poly = fmaf(s, fmaf(s, fmaf(s, fmaf(s, 33.0f / 2048.0f, 21.0f / 1024.0f), 7.0f / 256.0f),
                                        5.0f / 128.0f), 1.0f / 16.0f);
        return K * (s * s * s) * poly;
    } else {
        const float q = sqrtf(1.0f - s);
        const float d = 1.0f + q;
        return K * (s * s * s) * (3.0f + q) / (8.0f * d * d * d);
    }
}

template <bool POLY>
CWO_HD float2 asm_h_reduced(float4 X, float4 Y, float K) {
    const float s = X.x + Y.x;
    // cross = (X.z + X.w)(Y.z + Y.w) in float-float, fractional part taken exactly
    const float p = X.z * Y.z;
    const float pe = fmaf(X.z, Y.z, -p);
    const float lo = fmaf(X.z, Y.w, fmaf(X.w, Y.z, pe));
    const float pf = p - rintf(p);
    const float tail = asm_tail<POLY>(s, K);
    float psi = -(X.y + Y.y) - pf - lo - tail;
    psi -= rintf(psi);
    float sn, cs;
#ifdef __CUDA_ARCH__
    __sincosf(6.28318530717958647692f * psi, &sn, &cs);
#else
    sn = sinf(6.28318530717958647692f * psi);
    cs = cosf(6.28318530717958647692f * psi);
#endif
    return s > 1.0f ? make_float2(0.f, 0.f) : make_float2(cs, sn);   // evanescent: H = 0
}

// Literal per-element evaluation of the phase K sqrt(1 - s) in FP64, reduced to [-1/2, 1/2]
// cycle before the sine and cosine (reference arm; automatic where K s^3 is too large for the
// FP32 remainder).  s = sx kbx^2 + sy kby^2 with sx = lambda^2 / (Px dx)^2.
CWO_HD float2 asm_h_fp64(int kbx, int kby, double K, double sx, double sy) {
    const double s = sx * (double)kbx * (double)kbx + sy * (double)kby * (double)kby;
    if (s > 1.0) return make_float2(0.f, 0.f);
    double psi = K * sqrt(1.0 - s);
    psi -= rint(psi);
    float sn, cs;
#ifdef __CUDA_ARCH__
    sincospif(2.0f * (float)psi, &sn, &cs);
#else
    sn = (float)sin(2.0 * 3.14159265358979323846 * psi);
    cs = (float)cos(2.0 * 3.14159265358979323846 * psi);
#endif
    return make_float2(cs, sn);
}

// The same with the shifted ASM's extra phase shx kbx + shy kby cycles (Eq. shift_ang2), in FP64
// before the reduction.
CWO_HD float2 asm_h_fp64_shifted(int kbx, int kby, double K, double sx, double sy, double shx, double shy) {
    const double s = sx * (double)kbx * (double)kbx + sy * (double)kby * (double)kby;
    if (s > 1.0) return make_float2(0.f, 0.f);
    double psi = K * sqrt(1.0 - s) + shx * (double)kbx + shy * (double)kby;
    psi -= rint(psi);
    float sn, cs;
#ifdef __CUDA_ARCH__
    sincospif(2.0f * (float)psi, &sn, &cs);
#else
    sn = (float)sin(2.0 * 3.14159265358979323846 * psi);
    cs = (float)cos(2.0 * 3.14159265358979323846 * psi);
#endif
    return make_float2(cs, sn);
}

#ifdef __CUDACC__
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

// Evaluate the transfer function of storage column `col` at this thread's 16 axis indices
// e * T + t (DIF order) and hand each value to f(e, h).  The mode and tables are the launch's, or
// the item's own in a mixed batch.
template <int P, bool MIXED, class F>
__device__ __forceinline__ void eval_h(int col, int t, long long item, const HParams& hp, F&& f) {
    constexpr int T = P / 16;
    int mode = hp.mode;
    float K = 0.f;
    double Kd = hp.K, sx = hp.sx, sy = hp.sy;
    if (MIXED) {      // mixed batch: this item's own mode and scalars (uniform across the block)
        const ItemParams ip = hp.items[item];
        mode = ip.mode;
        K = ip.kf;
        Kd = ip.K; sx = ip.sx; sy = ip.sy;
    } else if (mode == HMODE_ASM_POLY || mode == HMODE_ASM_EXACT) {
        K = __ldg(hp.kf + item * hp.kf_item_stride);
    }
    if (mode == HMODE_TABLE) {
        const int j = abs(__ldg(hp.kbx + col));
        const float2* hc = hp.hcache + (long long)j * hp.hcache_stride + t;
#pragma unroll
        for (int e = 0; e < 16; ++e) f(e, __ldcg(hc + e * T));
    } else if (mode == HMODE_FRESNEL) {
        if (MIXED) {
            const float4 X = __ldg(hp.ax + item * hp.x_item_stride + col);
            const float2 hxc = make_float2(X.x, X.y);
            const float4* hy = hp.ay + item * hp.y_item_stride + t;
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const float4 Y = __ldg(hy + e * T);
                f(e, cmul(hxc, make_float2(Y.x, Y.y)));
            }
        } else {
            const float2 hxc = __ldg(hp.hx + item * hp.x_item_stride + col);
            const float2* hy = hp.hy + item * hp.y_item_stride + t;
#pragma unroll
            for (int e = 0; e < 16; ++e) f(e, cmul(hxc, __ldg(hy + e * T)));
        }
    } else if (mode == HMODE_ASM_POLY || mode == HMODE_ASM_EXACT) {
        const float4 X = __ldg(hp.ax + item * hp.x_item_stride + col);
        const float4* ay = hp.ay + item * hp.y_item_stride + t;
        if (mode == HMODE_ASM_POLY) {
#pragma unroll
            for (int e = 0; e < 16; ++e) f(e, asm_h_reduced<true>(X, __ldg(ay + e * T), K));
        } else {
#pragma unroll
            for (int e = 0; e < 16; ++e) f(e, asm_h_reduced<false>(X, __ldg(ay + e * T), K));
        }
    } else {
        const int kbx = __ldg(hp.kbx + col);
        if (hp.asym) {   // shifted ASM, per-element FP64: window and shift phase
            const bool inx = kbx >= hp.wxlo && kbx <= hp.wxhi;
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int kby = __ldg(hp.kby + e * T + t);
                const bool in = inx && kby >= hp.wylo && kby <= hp.wyhi;
                f(e, in ? asm_h_fp64_shifted(kbx, kby, Kd, sx, sy, hp.shx, hp.shy) : make_float2(0.f, 0.f));
            }
            return;
        }
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const int kby = __ldg(hp.kby + e * T + t);
            f(e, mode == HMODE_ASM_FP32 ? asm_h_fp32(kbx, kby, hp) : asm_h_fp64(kbx, kby, Kd, sx, sy));
        }
    }
}

// multiply the registers of NV transforms of the same storage column pair (same |kx|) by H
// (by conj(H) for the adjoint)
template <int P, int NV, bool MIXED = false>
__device__ __forceinline__ void apply_h(float2 (&a)[16], float2 (&b)[16], int col, int t, long long item,
                                        const HParams& hp) {
    eval_h<P, MIXED>(col, t, item, hp, [&](int e, float2 h) {
        a[e] = hp.conj ? cmulc(a[e], h) : cmul(a[e], h);
        if (NV == 2) b[e] = hp.conj ? cmulc(b[e], h) : cmul(b[e], h);
    });
}
#endif  // __CUDACC__

}  // namespace cwo
