// cwo_epilogue.cuh -- output epilogues of the inverse row pass (the last step of a propagation).
#pragma once
#include "cwo_fft.cuh"
#include "cwo_internal.h"

namespace cwo {

// Output epilogue of the inverse row pass, applied to the scaled value w of output element idx
// (the GS constraints of Section "GS algorithm" fused into the pass that produces the field):
//   EPI_NONE       out = w
//   EPI_PHASE      out = w / |w|             (phase constraint; |w| = 0 gives 1)
//   EPI_AMPLITUDE  out = amp[idx] w / |w|    (amplitude constraint)
//   EPI_INTENSITY  inten[idx] = |w|^2        (reconstruction; out is not written)
// The constraints round every product on its own (an explicit fused multiply-add for the squared
// magnitude, __fmul_rn, which is never merged into a multiply-add, for the scalings), so that the
// value does not depend on what the kernel does with it next: a fused loop, whose next operation
// is an add of the following transform, computes what the separate passes store.
__device__ __forceinline__ float2 unit_phase(float2 w) {
    const float m2 = fmaf(w.x, w.x, w.y * w.y);
    if (m2 > 0.f) {
        const float r = rsqrtf(m2);
        return make_float2(__fmul_rn(w.x, r), __fmul_rn(w.y, r));
    }
    return make_float2(1.f, 0.f);
}
__device__ __forceinline__ float2 amplitude_phase(float2 w, float a) {
    const float2 u = unit_phase(w);
    return make_float2(__fmul_rn(u.x, a), __fmul_rn(u.y, a));
}

template <int EPI>
__device__ __forceinline__ void epilogue_store(float2* out, const Epilogue& ep, long long idx, int x, int y, float2 w) {
    if constexpr (EPI == EPI_NONE) out[idx] = w;
    else if constexpr (EPI == EPI_SEPARABLE) out[idx] = cmul(w, cmul(__ldg(ep.qx + x), __ldg(ep.qy + y)));
    else if constexpr (EPI == EPI_PHASE) out[idx] = unit_phase(w);
    else if constexpr (EPI == EPI_AMPLITUDE) out[idx] = amplitude_phase(w, __ldg(ep.amp + idx));
    else ep.inten[idx] = w.x * w.x + w.y * w.y;
}

// the constrained value of an epilogue that passes the field on (the same expressions as
// epilogue_store, so that a fused loop computes what the separate passes store)
template <int EPI>
__device__ __forceinline__ float2 epilogue_value(const Epilogue& ep, long long idx, float2 w) {
    if constexpr (EPI == EPI_PHASE) return unit_phase(w);
    else if constexpr (EPI == EPI_AMPLITUDE) return amplitude_phase(w, __ldg(ep.amp + idx));
    else return w;
}

// the same with the mode chosen at run time (a uniform branch)
__device__ __forceinline__ void epilogue_store_rt(int mode, float2* out, const Epilogue& ep, long long idx, int x, int y,
                                                  float2 w) {
    switch (mode) {
        case EPI_PHASE: epilogue_store<EPI_PHASE>(out, ep, idx, x, y, w); break;
        case EPI_AMPLITUDE: epilogue_store<EPI_AMPLITUDE>(out, ep, idx, x, y, w); break;
        case EPI_INTENSITY: epilogue_store<EPI_INTENSITY>(out, ep, idx, x, y, w); break;
        default: epilogue_store<EPI_NONE>(out, ep, idx, x, y, w); break;
    }
}

}  // namespace cwo
