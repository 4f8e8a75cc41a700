// cwo_fft.cuh -- device building blocks of the register/shared-memory FFT used by all passes.
//
// A length-P transform (P = 2^p, 32 <= P <= 8192) is computed by T = P/16 threads that each hold
// 16 complex64 values in registers.  The forward transform is an in-place mixed-radix
// decimation-in-frequency (DIF) FFT: stages 0 .. NST-2 have radix 16, the last stage has radix
// RLAST in {2, 4, 8, 16}.  No digit-reversal pass is made: the forward output stays in DIF
// (digit-reversed) order, the transfer function is applied in that order, and the inverse is the
// exact adjoint of the forward stages (conjugate twiddles, inverse butterflies, stages in reverse),
// which consumes digit-reversed input and returns natural order.  Between stages the values are
// exchanged through shared memory in padded layouts that keep every access bank-conflict free.
//
// Stage s works on sub-transforms of length L_s = P / 16^s with stride S_s = L_s / radix(s).
//   stage s < NST-1 : thread t owns butterfly t: block b = t / S_s, offset j = t % S_s, and its
//                     register e holds position b L_s + j + e S_s; after the radix-16 DFT,
//                     output k' is multiplied by W_{L_s}^{j k'}, W_L = exp(-2 pi i / L).
//   stage NST-1     : thread t owns positions 16 t + e (consecutive butterflies of radix RLAST).
// The DIF position of frequency k = sum_s k_s prod_{i<s} r_i is sum_s k_s P / prod_{i<=s} r_i.
//
// These are the FFT steps of Eqs. ang3 and fre_conv_fft (FFT / IFFT), restated for sm_103a.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define CWO_HD __host__ __device__ __forceinline__

namespace cwo {

__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n / 2); }

template <int P>
struct Geo {
    static constexpr int LOG = ilog2c(P);
    static constexpr int NST = (LOG + 3) / 4;
    static constexpr int RLAST = 1 << (LOG - 4 * (NST - 1));
    static constexpr int T = P / 16;
    static __host__ __device__ constexpr int radix(int s) { return s == NST - 1 ? RLAST : 16; }
    static __host__ __device__ constexpr int len(int s) { return P >> (4 * s); }
    static __host__ __device__ constexpr int stride(int s) { return len(s) / radix(s); }
    // twiddle table: stage s < NST-1 owns 8 * stride(s) float4 starting at tw_off(s)
    static __host__ __device__ constexpr int tw_off(int s) { return s <= 0 ? 0 : tw_off(s - 1) + 8 * stride(s - 1); }
    static constexpr int TW_WORDS = tw_off(NST - 1);
    static_assert(P >= 32 && P <= 8192 && (P & (P - 1)) == 0, "P must be a power of two in [32, 8192]");
};

// ------------------------------------------------------------------------------- complex helpers
CWO_HD float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
CWO_HD float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
CWO_HD float2 cmul(float2 a, float2 w) {
    return make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x));
}
CWO_HD float2 cmulc(float2 a, float2 w) {  // a * conj(w)
    return make_float2(fmaf(a.x, w.x, a.y * w.y), fmaf(a.y, w.x, -a.x * w.y));
}
CWO_HD float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// multiply by W_4 = -i (forward) or +i (inverse)
template <bool INV> CWO_HD float2 mul_w4(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

constexpr float kRsqrt2 = 0.70710678118654752440f;
constexpr float kCos1 = 0.92387953251128675613f;  // cos(pi/8)
constexpr float kSin1 = 0.38268343236508977173f;  // sin(pi/8)

// multiply by W_16^E (E = 0..9), W_16 = exp(-+ 2 pi i / 16) for forward / inverse
template <bool INV, int E> CWO_HD float2 mul_w16(float2 a) {
    constexpr float sg = INV ? 1.0f : -1.0f;
    if constexpr (E == 0) return a;
    else if constexpr (E == 4) return mul_w4<INV>(a);
    else if constexpr (E == 8) return make_float2(-a.x, -a.y);
    else if constexpr (E == 2) {  // (1 -+ i)/sqrt2
        return INV ? make_float2((a.x - a.y) * kRsqrt2, (a.x + a.y) * kRsqrt2)
                   : make_float2((a.x + a.y) * kRsqrt2, (a.y - a.x) * kRsqrt2);
    } else if constexpr (E == 6) {  // (-1 -+ i)/sqrt2
        return INV ? make_float2(-(a.x + a.y) * kRsqrt2, (a.x - a.y) * kRsqrt2)
                   : make_float2((a.y - a.x) * kRsqrt2, -(a.x + a.y) * kRsqrt2);
    } else if constexpr (E == 1) {
        return cmul(a, make_float2(kCos1, sg * kSin1));
    } else if constexpr (E == 3) {
        return cmul(a, make_float2(kSin1, sg * kCos1));
    } else if constexpr (E == 9) {
        return cmul(a, make_float2(-kCos1, -sg * kSin1));
    } else {
        static_assert(E < 0, "unused exponent");
        return a;
    }
}

// ----------------------------------------------------------------------------- small DFTs
// All operate in place on v[B .. B+R) with natural-order input and output.
template <bool INV, int B, int ST = 1>
CWO_HD void dft4(float2 (&v)[16]) {
    float2 a0 = v[B], a1 = v[B + ST], a2 = v[B + 2 * ST], a3 = v[B + 3 * ST];
    float2 t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = mul_w4<INV>(csub(a1, a3));
    v[B] = cadd(t0, t2);
    v[B + ST] = cadd(t1, t3);
    v[B + 2 * ST] = csub(t0, t2);
    v[B + 3 * ST] = csub(t1, t3);
}
// radix-4 whose last two inputs are zero
template <bool INV, int B, int ST = 1>
CWO_HD void dft4_half(float2 (&v)[16]) {
    float2 a0 = v[B], a1 = v[B + ST];
    float2 r = mul_w4<INV>(a1);
    v[B] = cadd(a0, a1);
    v[B + ST] = cadd(a0, r);
    v[B + 2 * ST] = csub(a0, a1);
    v[B + 3 * ST] = csub(a0, r);
}

template <bool INV, int B>
CWO_HD void dft2(float2 (&v)[16]) {
    float2 a = v[B], b = v[B + 1];
    v[B] = cadd(a, b);
    v[B + 1] = csub(a, b);
}

template <bool INV, int B>
CWO_HD void dft8(float2 (&v)[16]) {
    float2 e0 = v[B], e1 = v[B + 2], e2 = v[B + 4], e3 = v[B + 6];
    float2 o0 = v[B + 1], o1 = v[B + 3], o2 = v[B + 5], o3 = v[B + 7];
    {   // even and odd radix-4 DFTs
        float2 t0 = cadd(e0, e2), t1 = csub(e0, e2), t2 = cadd(e1, e3), t3 = mul_w4<INV>(csub(e1, e3));
        e0 = cadd(t0, t2); e1 = cadd(t1, t3); e2 = csub(t0, t2); e3 = csub(t1, t3);
        float2 s0 = cadd(o0, o2), s1 = csub(o0, o2), s2 = cadd(o1, o3), s3 = mul_w4<INV>(csub(o1, o3));
        o0 = cadd(s0, s2); o1 = cadd(s1, s3); o2 = csub(s0, s2); o3 = csub(s1, s3);
    }
    o1 = mul_w16<INV, 2>(o1);
    o2 = mul_w4<INV>(o2);
    o3 = mul_w16<INV, 6>(o3);
    v[B] = cadd(e0, o0); v[B + 4] = csub(e0, o0);
    v[B + 1] = cadd(e1, o1); v[B + 5] = csub(e1, o1);
    v[B + 2] = cadd(e2, o2); v[B + 6] = csub(e2, o2);
    v[B + 3] = cadd(e3, o3); v[B + 7] = csub(e3, o3);
}

// 16-point DFT as 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2.  NZ = 8: inputs 8..15 are zero.
template <bool INV, int NZ>
CWO_HD void dft16(float2 (&v)[16]) {
    if constexpr (NZ == 8) {
        dft4_half<INV, 0, 4>(v); dft4_half<INV, 1, 4>(v); dft4_half<INV, 2, 4>(v); dft4_half<INV, 3, 4>(v);
    } else {
        dft4<INV, 0, 4>(v); dft4<INV, 1, 4>(v); dft4<INV, 2, 4>(v); dft4<INV, 3, 4>(v);
    }
    // v[n2 + 4 k1] *= W16^(n2 k1)
    v[5] = mul_w16<INV, 1>(v[5]);   v[6] = mul_w16<INV, 2>(v[6]);   v[7] = mul_w16<INV, 3>(v[7]);
    v[9] = mul_w16<INV, 2>(v[9]);   v[10] = mul_w16<INV, 4>(v[10]); v[11] = mul_w16<INV, 6>(v[11]);
    v[13] = mul_w16<INV, 3>(v[13]); v[14] = mul_w16<INV, 6>(v[14]); v[15] = mul_w16<INV, 9>(v[15]);
    dft4<INV, 0, 1>(v); dft4<INV, 4, 1>(v); dft4<INV, 8, 1>(v); dft4<INV, 12, 1>(v);
    // X[k1 + 4 k2] sits in v[4 k1 + k2]: transpose the 4 x 4 register block
    float2 w[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) w[i] = v[i];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = w[4 * k1 + k2];
}

// the butterflies of stage S on a thread's 16 registers
template <int P, int S, bool INV, int NZ>
CWO_HD void stage_butterflies(float2 (&v)[16]) {
    constexpr int R = Geo<P>::radix(S);
    if constexpr (R == 16) {
        dft16<INV, NZ>(v);
    } else if constexpr (R == 8) {
        dft8<INV, 0>(v); dft8<INV, 8>(v);
    } else if constexpr (R == 4) {
        dft4<INV, 0>(v); dft4<INV, 4>(v); dft4<INV, 8>(v); dft4<INV, 12>(v);
    } else {
        static_assert(R == 2, "radix");
        dft2<INV, 0>(v); dft2<INV, 2>(v); dft2<INV, 4>(v); dft2<INV, 6>(v);
        dft2<INV, 8>(v); dft2<INV, 10>(v); dft2<INV, 12>(v); dft2<INV, 14>(v);
    }
}

// position held by register e of thread t at stage S
template <int P, int S>
CWO_HD int stage_pos(int t, int e) {
    using G = Geo<P>;
    if constexpr (S == G::NST - 1) {
        return 16 * t + e;
    } else {
        constexpr int L = G::len(S), St = G::stride(S);
        return (t / St) * L + (t % St) + e * St;
    }
}

// Shared-memory layout of C transforms of length P, bank-conflict free at every stage when the C
// transforms are interleaved across a warp's lanes: one pad word per 16 positions plus a
// per-transform shift of 16/C words; the address of register e at any stage is a per-thread base
// plus a compile-time constant, so no per-element address arithmetic is left.
template <int P, int C>
struct PadLayout {
    static constexpr int R = P + P / 16 + (C <= 16 ? 16 / C : 1);
    static constexpr int WORDS = C * R;
    static CWO_HD int addr(int c, int pos) { return c * R + pos + (pos >> 4); }
};

// Tile of R rows x P storage columns used to transpose between the row passes and the
// column-major intermediate: linear index st * R + r plus one pad word per 16, which keeps both
// the per-row access (lanes over st) and the per-column access (lanes over r, then st) free of
// bank conflicts.
template <int P, int R>
struct TileLayout {
    static constexpr int WORDS = P * R + (P * R) / 16;
    static CWO_HD int addr(int st, int r) { const int i = st * R + r; return i + (i >> 4); }
};

#ifdef __CUDACC__
// Inter-stage twiddles W_{L_s}^{(t % S_s) k'}, k' = 1..15, of stage s < NST-1.
// TwTable: per stage a block of 8 S_s float4 laid out [kp][j], kp = 0..7, j = t mod S_s, holding
//          the pair (W^{j (2kp+1)}, W^{j (2kp+2)}): 8 16-byte loads per thread and stage.  Only
//          the S_s distinct j are stored, so the table of P = 4096 is 34 KB, not 64 KB, and
//          stays in L1 next to the transfer-function tables.
template <int P>
struct TwTable {
    const float4* __restrict__ tw;
    int t;
    template <int S, bool INV>
    __device__ __forceinline__ void apply(float2 (&v)[16]) const {
        constexpr int SS = Geo<P>::stride(S);
        const float4* base = tw + Geo<P>::tw_off(S) + (t & (SS - 1));
#pragma unroll
        for (int kp = 0; kp < 8; ++kp) {
            const float4 w = __ldg(base + kp * SS);
            v[2 * kp + 1] = INV ? cmulc(v[2 * kp + 1], make_float2(w.x, w.y)) : cmul(v[2 * kp + 1], make_float2(w.x, w.y));
            if (kp < 7)
                v[2 * kp + 2] = INV ? cmulc(v[2 * kp + 2], make_float2(w.z, w.w)) : cmul(v[2 * kp + 2], make_float2(w.z, w.w));
        }
    }
};

// the same twiddles applied to two transforms held by the same thread (two columns)
template <int P, int S, bool INV>
__device__ __forceinline__ void twiddle2(float2 (&a)[16], float2 (&b)[16], const float4* __restrict__ tw, int t) {
    constexpr int SS = Geo<P>::stride(S);
    const float4* base = tw + Geo<P>::tw_off(S) + (t & (SS - 1));
#pragma unroll
    for (int kp = 0; kp < 8; ++kp) {
        const float4 w = __ldg(base + kp * SS);
        const float2 w0 = make_float2(w.x, w.y), w1 = make_float2(w.z, w.w);
        a[2 * kp + 1] = INV ? cmulc(a[2 * kp + 1], w0) : cmul(a[2 * kp + 1], w0);
        b[2 * kp + 1] = INV ? cmulc(b[2 * kp + 1], w0) : cmul(b[2 * kp + 1], w0);
        if (kp < 7) {
            a[2 * kp + 2] = INV ? cmulc(a[2 * kp + 2], w1) : cmul(a[2 * kp + 2], w1);
            b[2 * kp + 2] = INV ? cmulc(b[2 * kp + 2], w1) : cmul(b[2 * kp + 2], w1);
        }
    }
}

// ---- exchanges with one barrier each
// The positions a thread reads in one exchange (its positions at the stage being entered) are
// exactly the positions it writes in the next exchange (it leaves that stage from the same
// positions), whether the next exchange continues the same transform, turns from the forward to
// the inverse stages, or starts the next transform.  Every position is read by one thread only,
// so no thread can overwrite a value another thread has still to read, and each exchange needs a
// single barrier between its writes and its reads.  The barrier spans only the threads that own
// one block of the earlier stage: Geo<P>::stride(s) threads for stages s and s + 1, which is the
// whole transform (T threads) between stages 0 and 1 and at most one warp between later stages.
// CP transforms pairs of a block use named barriers 1 .. CP when T > 32.
template <int P, int CP, int S>
__device__ __forceinline__ void xsync(int cp) {
    constexpr int G = Geo<P>::stride(S);   // threads sharing one stage-S block
    if constexpr (G <= 32) {
        __syncwarp();
    } else if constexpr (CP == 1) {
        __syncthreads();
    } else {
        static_assert(CP < 16, "named barrier ids");
        asm volatile("bar.sync %0, %1;" :: "r"(1 + cp), "r"(P / 16) : "memory");
    }
}

// The same exchanges for R transforms of one value per thread (PadLayout<P, R>), the CTA's
// R * P/16 threads all in step.  IL: the transforms are interleaved over the lanes (thread =
// r + R t), so a stage-S block is stride(S) threads of each transform, stride(S) * R consecutive
// lanes; otherwise each transform has T consecutive threads (thread = t + T r) and a block is
// stride(S) consecutive lanes.  The barrier is warp-wide where the block fits in a warp of a CTA
// of whole warps, and CTA-wide otherwise.
template <int P, int R, int S, bool IL = true>
__device__ __forceinline__ void xsync_r() {
    constexpr int lanes = IL ? Geo<P>::stride(S) * R : Geo<P>::stride(S);
    if constexpr (lanes <= 32 && R * (P / 16) % 32 == 0) __syncwarp();
    else __syncthreads();
}

template <int P, int R, int SW, int SR, bool IL = true>
__device__ __forceinline__ void xch1(float2* __restrict__ sm, int r, int t, float2 (&v)[16]) {
    using Lay = PadLayout<P, R>;
#pragma unroll
    for (int e = 0; e < 16; ++e) sm[Lay::addr(r, stage_pos<P, SW>(t, e))] = v[e];
    xsync_r<P, R, (SW < SR ? SW : SR), IL>();
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = sm[Lay::addr(r, stage_pos<P, SR>(t, e))];
}

// forward DIF from stage S to the end / adjoint from stage S down to stage 0 (or, for
// inv1_to_stage0, down to and including the exchange into stage 0), with xch1 exchanges
template <int P, int R, int S, int NZ0, bool IL = true, class Tw>
__device__ __forceinline__ void fwd1_from(float2 (&v)[16], float2* __restrict__ sm, int r, int t, const Tw& tw) {
    stage_butterflies<P, S, false, (S == 0 ? NZ0 : 16)>(v);
    if constexpr (S < Geo<P>::NST - 1) {
        tw.template apply<S, false>(v);
        xch1<P, R, S, S + 1, IL>(sm, r, t, v);
        fwd1_from<P, R, S + 1, NZ0, IL>(v, sm, r, t, tw);
    }
}

template <int P, int R, int S, bool IL = true, class Tw>
__device__ __forceinline__ void inv1_from(float2 (&v)[16], float2* __restrict__ sm, int r, int t, const Tw& tw) {
    if constexpr (S < Geo<P>::NST - 1) tw.template apply<S, true>(v);
    stage_butterflies<P, S, true, 16>(v);
    if constexpr (S > 0) {
        xch1<P, R, S, S - 1, IL>(sm, r, t, v);
        inv1_from<P, R, S - 1, IL>(v, sm, r, t, tw);
    }
}

template <int P, int R, int S, class Tw>
__device__ __forceinline__ void inv1_to_stage0(float2 (&v)[16], float2* __restrict__ sm, int r, int t, const Tw& tw) {
    if constexpr (S < Geo<P>::NST - 1) tw.template apply<S, true>(v);
    stage_butterflies<P, S, true, 16>(v);
    xch1<P, R, S, S - 1>(sm, r, t, v);
    if constexpr (S > 1) inv1_to_stage0<P, R, S - 1>(v, sm, r, t, tw);
}

template <int P, int CP, class Lay, int SW, int SR>
__device__ __forceinline__ void xch2(float2* __restrict__ sm, int cp, int t, float2 (&a)[16], float2 (&b)[16]) {
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        sm[Lay::addr(2 * cp, stage_pos<P, SW>(t, e))] = a[e];
        sm[Lay::addr(2 * cp + 1, stage_pos<P, SW>(t, e))] = b[e];
    }
    xsync<P, CP, (SW < SR ? SW : SR)>(cp);
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        a[e] = sm[Lay::addr(2 * cp, stage_pos<P, SR>(t, e))];
        b[e] = sm[Lay::addr(2 * cp + 1, stage_pos<P, SR>(t, e))];
    }
}

// Pair layout for xch2v: the values of both transforms of a pair at one position share one
// 16-byte slot, so an exchange moves them with one 128-bit access each way.  One pad slot per 16
// positions keeps the eight lanes of every quarter-warp on distinct banks at every stage when a
// transform has T >= 8 threads (P >= 128).
template <int P, int CP>
struct PairLayout {
    static constexpr int R = P + P / 16;          // slots per pair
    static constexpr int SLOTS = CP * R;
    static CWO_HD int slot(int cp, int pos) { return cp * R + pos + (pos >> 4); }
};

template <int P, int CP, int SW, int SR>
__device__ __forceinline__ void xch2v(float4* __restrict__ sm, int cp, int t, float2 (&a)[16], float2 (&b)[16]) {
    using L = PairLayout<P, CP>;
#pragma unroll
    for (int e = 0; e < 16; ++e) sm[L::slot(cp, stage_pos<P, SW>(t, e))] = make_float4(a[e].x, a[e].y, b[e].x, b[e].y);
    xsync<P, CP, (SW < SR ? SW : SR)>(cp);
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        const float4 v = sm[L::slot(cp, stage_pos<P, SR>(t, e))];
        a[e] = make_float2(v.x, v.y);
        b[e] = make_float2(v.z, v.w);
    }
}

// forward / inverse stages of a pair with the 128-bit exchange (P >= 128)
template <int P, int CP, int S, int NZ0>
__device__ __forceinline__ void fwd2v_from(float2 (&a)[16], float2 (&b)[16], float4* __restrict__ sm, int cp, int t,
                                           const float4* __restrict__ tw) {
    using G = Geo<P>;
    stage_butterflies<P, S, false, (S == 0 ? NZ0 : 16)>(a);
    stage_butterflies<P, S, false, (S == 0 ? NZ0 : 16)>(b);
    if constexpr (S < G::NST - 1) {
        twiddle2<P, S, false>(a, b, tw, t);
        xch2v<P, CP, S, S + 1>(sm, cp, t, a, b);
        fwd2v_from<P, CP, S + 1, NZ0>(a, b, sm, cp, t, tw);
    }
}

template <int P, int CP, int S>
__device__ __forceinline__ void inv2v_from(float2 (&a)[16], float2 (&b)[16], float4* __restrict__ sm, int cp, int t,
                                           const float4* __restrict__ tw) {
    using G = Geo<P>;
    if constexpr (S < G::NST - 1) twiddle2<P, S, true>(a, b, tw, t);
    stage_butterflies<P, S, true, 16>(a);
    stage_butterflies<P, S, true, 16>(b);
    if constexpr (S > 0) {
        xch2v<P, CP, S, S - 1>(sm, cp, t, a, b);
        inv2v_from<P, CP, S - 1>(a, b, sm, cp, t, tw);
    }
}

// the same down to (and including) the exchange into stage 0; the caller applies the stage-0
// twiddles and butterflies (the inverse row pass requests its next tile before them)
template <int P, int CP, int S>
__device__ __forceinline__ void inv2v_to_stage0(float2 (&a)[16], float2 (&b)[16], float4* __restrict__ sm, int cp,
                                                int t, const float4* __restrict__ tw) {
    if constexpr (S < Geo<P>::NST - 1) twiddle2<P, S, true>(a, b, tw, t);
    stage_butterflies<P, S, true, 16>(a);
    stage_butterflies<P, S, true, 16>(b);
    xch2v<P, CP, S, S - 1>(sm, cp, t, a, b);
    if constexpr (S > 1) inv2v_to_stage0<P, CP, S - 1>(a, b, sm, cp, t, tw);
}

template <int P, int CP, class Lay, int S, int NZ0>
__device__ __forceinline__ void fwd2x_from(float2 (&a)[16], float2 (&b)[16], float2* __restrict__ sm, int cp, int t,
                                           const float4* __restrict__ tw) {
    using G = Geo<P>;
    stage_butterflies<P, S, false, (S == 0 ? NZ0 : 16)>(a);
    stage_butterflies<P, S, false, (S == 0 ? NZ0 : 16)>(b);
    if constexpr (S < G::NST - 1) {
        twiddle2<P, S, false>(a, b, tw, t);
        xch2<P, CP, Lay, S, S + 1>(sm, cp, t, a, b);
        fwd2x_from<P, CP, Lay, S + 1, NZ0>(a, b, sm, cp, t, tw);
    }
}

template <int P, int CP, class Lay, int S>
__device__ __forceinline__ void inv2x_from(float2 (&a)[16], float2 (&b)[16], float2* __restrict__ sm, int cp, int t,
                                           const float4* __restrict__ tw) {
    using G = Geo<P>;
    if constexpr (S < G::NST - 1) twiddle2<P, S, true>(a, b, tw, t);
    stage_butterflies<P, S, true, 16>(a);
    stage_butterflies<P, S, true, 16>(b);
    if constexpr (S > 0) {
        xch2<P, CP, Lay, S, S - 1>(sm, cp, t, a, b);
        inv2x_from<P, CP, Lay, S - 1>(a, b, sm, cp, t, tw);
    }
}

#endif  // __CUDACC__

}  // namespace cwo
