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

CWO_HD float2 asm_h_reduced(float4 X, float4 Y, float K) {
    const float s = X.x + Y.x;
    if (s > 1.0f) return make_float2(0.f, 0.f);          // evanescent
    // cross = (X.z + X.w)(Y.z + Y.w) in float-float, fractional part taken exactly
    const float p = X.z * Y.z;
    const float pe = fmaf(X.z, Y.z, -p);
    const float lo = fmaf(X.z, Y.w, fmaf(X.w, Y.z, pe));
    const float pf = p - rintf(p);
    const float q = sqrtf(1.0f - s);
    const float d = 1.0f + q;
    const float tail = K * (s * s * s) * (3.0f + q) / (8.0f * d * d * d);
    float psi = -(X.y + Y.y) - pf - lo - tail;
    psi -= rintf(psi);
    float sn, cs;
#ifdef __CUDA_ARCH__
    __sincosf(6.28318530717958647692f * psi, &sn, &cs);
#else
    sn = sinf(6.28318530717958647692f * psi);
    cs = cosf(6.28318530717958647692f * psi);
#endif
    return make_float2(cs, sn);
}


}  // namespace cwo
