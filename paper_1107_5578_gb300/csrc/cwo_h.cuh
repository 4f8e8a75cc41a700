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

}  // namespace cwo
