// cwo_emu.cpp -- host emulation of the three CUDA passes (test support).
//
// Runs the same butterflies, stage positions, twiddle tables, transfer-function code and table
// generation as the kernels, one "thread" at a time, with a plain array standing in for shared
// memory.  It lets the host-only test suite check the FFT index logic against the oracle on a
// machine without a GPU.  It is slow and only meant for small fields.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/cwo.h"
#include "../../include/cwo_debug.h"
#include "cwo_fft.cuh"
#include "cwo_h.cuh"
#include "cwo_tables.h"

namespace cwo {
namespace {

struct Regs { float2 v[16]; };

template <int P, int S, bool INV>
void emu_twiddle(std::vector<Regs>& R, const float4* tw) {
    constexpr int T = Geo<P>::T, SS = Geo<P>::stride(S);
    for (int t = 0; t < T; ++t)
        for (int k = 1; k < 16; ++k) {
            const float4 q = tw[Geo<P>::tw_off(S) + ((k - 1) / 2) * SS + (t & (SS - 1))];
            const float2 w = (k & 1) ? make_float2(q.x, q.y) : make_float2(q.z, q.w);
            R[t].v[k] = INV ? cmulc(R[t].v[k], w) : cmul(R[t].v[k], w);
        }
}

template <int P, int SW, int SR>
void emu_exchange(std::vector<Regs>& R) {
    constexpr int T = Geo<P>::T;
    std::vector<float2> sm(PadLayout<P, 1>::WORDS);
    for (int t = 0; t < T; ++t)
        for (int e = 0; e < 16; ++e) sm[PadLayout<P, 1>::addr(0, stage_pos<P, SW>(t, e))] = R[t].v[e];
    for (int t = 0; t < T; ++t)
        for (int e = 0; e < 16; ++e) R[t].v[e] = sm[PadLayout<P, 1>::addr(0, stage_pos<P, SR>(t, e))];
}

template <int P, int S, int NZ0>
void emu_fwd_from(std::vector<Regs>& R, const float4* tw) {
    using G = Geo<P>;
    for (int t = 0; t < G::T; ++t) stage_butterflies<P, S, false, (S == 0 ? NZ0 : 16)>(R[t].v);
    if constexpr (S < G::NST - 1) {
        emu_twiddle<P, S, false>(R, tw);
        emu_exchange<P, S, S + 1>(R);
        emu_fwd_from<P, S + 1, NZ0>(R, tw);
    }
}

template <int P, int S>
void emu_inv_from(std::vector<Regs>& R, const float4* tw) {
    using G = Geo<P>;
    if constexpr (S < G::NST - 1) emu_twiddle<P, S, true>(R, tw);
    for (int t = 0; t < G::T; ++t) stage_butterflies<P, S, true, 16>(R[t].v);
    if constexpr (S > 0) {
        emu_exchange<P, S, S - 1>(R);
        emu_inv_from<P, S - 1>(R, tw);
    }
}

// forward transform of one padded line: in[0..P/2) nonzero; out in axis-index order
template <int P>
void emu_line_fwd(const float2* in, long long in_step, float2* out, long long out_step, const float4* tw) {
    constexpr int T = P / 16;
    std::vector<Regs> R(T);
    for (int t = 0; t < T; ++t)
        for (int e = 0; e < 16; ++e)
            R[t].v[e] = e < 8 ? in[(long long)(t + e * T) * in_step] : make_float2(0.f, 0.f);
    emu_fwd_from<P, 0, 8>(R, tw);
    for (int t = 0; t < T; ++t)
        for (int e = 0; e < 16; ++e) out[(long long)(e * T + t) * out_step] = R[t].v[e];
}

// adjoint transform of one line given in axis-index order; keeps the first P/2 outputs
template <int P>
void emu_line_inv(const float2* in, long long in_step, float2* out, long long out_step, const float4* tw) {
    constexpr int T = P / 16;
    std::vector<Regs> R(T);
    for (int t = 0; t < T; ++t)
        for (int e = 0; e < 16; ++e) R[t].v[e] = in[(long long)(e * T + t) * in_step];
    emu_inv_from<P, Geo<P>::NST - 1>(R, tw);
    for (int t = 0; t < T; ++t)
        for (int e = 0; e < 8; ++e) out[(long long)(t + e * T) * out_step] = R[t].v[e];
}

// the split column pass (k_col_split, P = 2Q): the Q samples x_n of a column (stride `step`) and
// x_n W_P^n take the Q-point forward transforms, are multiplied by H at split index h Q + e T + t
// (hs), take the adjoint stages, and the column becomes the even half plus W_P^-n times the odd half
template <int Q>
void emu_col_split(float2* col, long long step, const float2* w, const float4* twq, const std::vector<float2>& hs,
                   bool adjoint) {
    constexpr int T = Q / 16;
    std::vector<Regs> A(T), B(T);
    for (int t = 0; t < T; ++t)
        for (int e = 0; e < 16; ++e) {
            A[t].v[e] = col[(long long)(t + e * T) * step];
            B[t].v[e] = cmul(A[t].v[e], w[t + e * T]);
        }
    emu_fwd_from<Q, 0, 16>(A, twq);
    emu_fwd_from<Q, 0, 16>(B, twq);
    for (int t = 0; t < T; ++t)
        for (int e = 0; e < 16; ++e) {
            const float2 ha = hs[e * T + t], hb = hs[Q + e * T + t];
            A[t].v[e] = adjoint ? cmulc(A[t].v[e], ha) : cmul(A[t].v[e], ha);
            B[t].v[e] = adjoint ? cmulc(B[t].v[e], hb) : cmul(B[t].v[e], hb);
        }
    emu_inv_from<Q, Geo<Q>::NST - 1>(A, twq);
    emu_inv_from<Q, Geo<Q>::NST - 1>(B, twq);
    for (int t = 0; t < T; ++t)
        for (int e = 0; e < 16; ++e)
            col[(long long)(t + e * T) * step] = cadd(A[t].v[e], cmulc(B[t].v[e], w[t + e * T]));
}

using LineFn = void (*)(const float2*, long long, float2*, long long, const float4*);

LineFn pick_fwd(int p) {
    switch (p) {
        case 32: return emu_line_fwd<32>; case 64: return emu_line_fwd<64>; case 128: return emu_line_fwd<128>;
        case 256: return emu_line_fwd<256>; case 512: return emu_line_fwd<512>; case 1024: return emu_line_fwd<1024>;
        case 2048: return emu_line_fwd<2048>; case 4096: return emu_line_fwd<4096>; case 8192: return emu_line_fwd<8192>;
        default: return nullptr;
    }
}
LineFn pick_inv(int p) {
    switch (p) {
        case 32: return emu_line_inv<32>; case 64: return emu_line_inv<64>; case 128: return emu_line_inv<128>;
        case 256: return emu_line_inv<256>; case 512: return emu_line_inv<512>; case 1024: return emu_line_inv<1024>;
        case 2048: return emu_line_inv<2048>; case 4096: return emu_line_inv<4096>; case 8192: return emu_line_inv<8192>;
        default: return nullptr;
    }
}

}  // namespace
}  // namespace cwo

extern "C" cwo_status cwo_debug_emulate(int nx, int ny, double dx, double dy, double lambda, double z,
                                        int type, unsigned flags, int adjoint, const float* in_ri,
                                        float* out_ri) {
    using namespace cwo;
    using namespace cwo::host;
    if (!in_ri || !out_ri || nx < 16 || ny < 16 || nx > 4096 || ny > 4096 || (nx & (nx - 1)) || (ny & (ny - 1)) ||
        !(dx > 0) || !(dy > 0) || !(lambda > 0) || (type != CWO_ANGULAR && type != CWO_FRESNEL_CONV) ||
        (type == CWO_FRESNEL_CONV && z == 0.0) || (flags & ~(CWO_FLAG_LITERAL_SCALE | CWO_FLAG_CACHE_H)) ||
        ((flags & CWO_FLAG_CACHE_H) && type != CWO_ANGULAR))
        return CWO_ERR_INVALID_ARG;
    const int px = 2 * nx, py = 2 * ny;
    const AxisGeo gx(px), gy(py);
    const std::vector<float4> twx = twiddle_table(gx), twy = twiddle_table(gy);
    std::vector<float4> ax(px), ay(py);
    std::vector<float2> hx(px), hy(py);
    float K = 0.f;
    const bool fresnel = type == CWO_FRESNEL_CONV;
    make_h_tables(px, py, dx, dy, lambda, z, fresnel, (flags & CWO_FLAG_LITERAL_SCALE) != 0,
                  ax.data(), ay.data(), hx.data(), hy.data(), &K);
    const int tmode = asm_tail_mode(px, py, dx, dy, lambda, z);
    const bool poly = tmode == 0;
    const std::vector<int> kbx = bin_table(gx), kby = bin_table(gy);
    const double sx = lambda * lambda / ((double)px * dx * (double)px * dx);
    const double sy = lambda * lambda / ((double)py * dy * (double)py * dy);
    const float2* in = (const float2*)in_ri;
    float2* out = (float2*)out_ri;
    LineFn fx = pick_fwd(px), ix = pick_inv(px), fy = pick_fwd(py), iy = pick_inv(py);
    if (fresnel) {
        // the two separable line passes (cwo_lines.cu): rows with Hx into a column-major Nx x Ny
        // intermediate, then its columns with Hy into the output; each scaled by 1/P of its axis
        std::vector<float2> M((size_t)nx * ny), line((size_t)std::max(px, py)), half((size_t)std::max(nx, ny));
        const float scx = (float)(1.0 / px), scy = (float)(1.0 / py);
        for (int y = 0; y < ny; ++y) {
            fx(in + (size_t)y * nx, 1, line.data(), 1, twx.data());
            for (int i = 0; i < px; ++i) line[i] = adjoint ? cmulc(line[i], hx[i]) : cmul(line[i], hx[i]);
            ix(line.data(), 1, half.data(), 1, twx.data());
            for (int x = 0; x < nx; ++x) M[(size_t)x * ny + y] = cscale(half[x], scx);
        }
        for (int x = 0; x < nx; ++x) {
            fy(M.data() + (size_t)x * ny, 1, line.data(), 1, twy.data());
            for (int i = 0; i < py; ++i) line[i] = adjoint ? cmulc(line[i], hy[i]) : cmul(line[i], hy[i]);
            iy(line.data(), 1, half.data(), 1, twy.data());
            for (int y = 0; y < ny; ++y) out[(size_t)y * nx + x] = cscale(half[y], scy);
        }
        return CWO_OK;
    }
    auto h_at = [&](int c, int i) {   // H of storage column c at y axis index i (the column pass's code)
        if (tmode == 2) return asm_h_fp64(kbx[c], kby[i], z / lambda, sx, sy);
        return poly ? asm_h_reduced<true>(ax[c], ay[i], K) : asm_h_reduced<false>(ax[c], ay[i], K);
    };
    std::vector<float2> W((size_t)ny * px);
    for (int y = 0; y < ny; ++y) fx(in + (size_t)y * nx, 1, W.data() + (size_t)y * px, 1, twx.data());
    if ((flags & CWO_FLAG_CACHE_H) && py == kSplitColP) {
        // the cached transfer function at Py = 8192: the split column pass, its H evaluated as the
        // cache builder does (split index i at the y axis index of its frequency) for the
        // canonical column of the mirror pair
        constexpr int Q = kSplitColP / 2;
        const std::vector<float4> twq = twiddle_table(AxisGeo(Q));
        const std::vector<float2> wn = split_phase(py);
        const std::vector<int> yi = split_axis_index(py);
        const std::vector<int2> prs = mirror_pairs(gx);
        std::vector<float2> hs(py);
        for (const int2& pr : prs) {
            for (int i = 0; i < py; ++i) hs[i] = h_at(pr.x, yi[i]);
            emu_col_split<Q>(W.data() + pr.x, px, wn.data(), twq.data(), hs, adjoint != 0);
            if (pr.y != pr.x) emu_col_split<Q>(W.data() + pr.y, px, wn.data(), twq.data(), hs, adjoint != 0);
        }
    } else {
    std::vector<float2> col(py);
    for (int c = 0; c < px; ++c) {
        fy(W.data() + c, px, col.data(), 1, twy.data());
        for (int i = 0; i < py; ++i) {
            float2 h;
            if (fresnel) h = cmul(hx[c], hy[i]);
            else h = h_at(c, i);
            col[i] = adjoint ? cmulc(col[i], h) : cmul(col[i], h);
        }
        iy(col.data(), 1, W.data() + c, px, twy.data());
    }
    }
    const float scale = (float)(1.0 / ((double)px * (double)py));
    std::vector<float2> line(nx);
    for (int y = 0; y < ny; ++y) {
        ix(W.data() + (size_t)y * px, 1, line.data(), 1, twx.data());
        for (int x = 0; x < nx; ++x) out[(size_t)y * nx + x] = cscale(line[x], scale);
    }
    return CWO_OK;
}

extern "C" cwo_status cwo_debug_emulate_shifted(int nx, int ny, double dx, double dy, double lambda, double z,
                                                const cwo_shift* sh, int adjoint, const float* in_ri, float* out_ri) {
    using namespace cwo;
    using namespace cwo::host;
    if (!sh || !in_ri || !out_ri || nx < 16 || ny < 16 || nx > 4096 || ny > 4096 || (nx & (nx - 1)) ||
        (ny & (ny - 1)) || !(dx > 0) || !(dy > 0) || !(lambda > 0) || !std::isfinite(z))
        return CWO_ERR_INVALID_ARG;
    const int px = 2 * nx, py = 2 * ny;
    const int tmode = asm_tail_mode(px, py, dx, dy, lambda, z);
    if (tmode == 2) return CWO_ERR_UNSUPPORTED;   // the per-element FP64 arm is not emulated here
    const std::vector<float4> twx = twiddle_table(AxisGeo(px)), twy = twiddle_table(AxisGeo(py));
    std::vector<float4> ax(px), ay(py);
    asm_axis_table_shifted(AxisGeo(px), dx, lambda, z, true, sh->ox, sh->cx, sh->wx, ax.data());
    asm_axis_table_shifted(AxisGeo(py), dy, lambda, z, false, sh->oy, sh->cy, sh->wy, ay.data());
    const float K = (float)(z / lambda);
    const float2* in = (const float2*)in_ri;
    float2* out = (float2*)out_ri;
    LineFn fx = pick_fwd(px), ix = pick_inv(px), fy = pick_fwd(py), iy = pick_inv(py);
    // the three passes: rows, columns with H (shift and windows folded into the tables), rows back
    std::vector<float2> W((size_t)ny * px), col(py), line(nx);
    for (int y = 0; y < ny; ++y) fx(in + (size_t)y * nx, 1, W.data() + (size_t)y * px, 1, twx.data());
    for (int c = 0; c < px; ++c) {
        fy(W.data() + c, px, col.data(), 1, twy.data());
        for (int i = 0; i < py; ++i) {
            const float2 h = tmode == 0 ? asm_h_reduced<true>(ax[c], ay[i], K) : asm_h_reduced<false>(ax[c], ay[i], K);
            col[i] = adjoint ? cmulc(col[i], h) : cmul(col[i], h);
        }
        iy(col.data(), 1, W.data() + c, px, twy.data());
    }
    const float scale = (float)(1.0 / ((double)px * (double)py));
    for (int y = 0; y < ny; ++y) {
        ix(W.data() + (size_t)y * px, 1, line.data(), 1, twx.data());
        for (int x = 0; x < nx; ++x) out[(size_t)y * nx + x] = cscale(line[x], scale);
    }
    return CWO_OK;
}

extern "C" cwo_status cwo_debug_emulate_shifted_fresnel(int nx, int ny, double dx0, double dy0, double lambda,
                                                        double z, const cwo_shifted_fresnel* prm, int adjoint,
                                                        const float* in_ri, float* out_ri) {
    using namespace cwo;
    using namespace cwo::host;
    if (!prm || !in_ri || !out_ri || nx < 16 || ny < 16 || nx > 4096 || ny > 4096 || (nx & (nx - 1)) ||
        (ny & (ny - 1)) || !(dx0 > 0) || !(dy0 > 0) || !(prm->dx1 > 0) || !(prm->dy1 > 0) || !(lambda > 0) ||
        !std::isfinite(z) || z == 0.0)
        return CWO_ERR_INVALID_ARG;
    const int px = 2 * nx, py = 2 * ny;
    const std::vector<float4> twx = twiddle_table(AxisGeo(px)), twy = twiddle_table(AxisGeo(py));
    std::vector<float2> fx(nx), fy(ny), qx(nx), qy(ny), hx(px), hy(py);
    const double cph = 6.283185307179586476925286766559 * frac01(z / lambda);
    const cd C = cd(std::cos(cph), std::sin(cph)) / cd(0.0, lambda * z) * (dx0 * dy0);
    shifted_fresnel_axis(nx, dx0, prm->dx1, prm->ox0, prm->ox1, lambda, z, C, fx.data(), qx.data(), hx.data());
    shifted_fresnel_axis(ny, dy0, prm->dy1, prm->oy0, prm->oy1, lambda, z, cd(1.0, 0.0), fy.data(), qy.data(), hy.data());
    auto conj = [](float2 a) { return make_float2(a.x, -a.y); };
    // the two separable line passes of cwo_lines.cu with the factors of their axis:
    // forward pre = f, post = q; adjoint pre = conj(q), post = conj(f), conj(h)
    const float2* in = (const float2*)in_ri;
    float2* out = (float2*)out_ri;
    LineFn fwx = pick_fwd(px), ivx = pick_inv(px), fwy = pick_fwd(py), ivy = pick_inv(py);
    std::vector<float2> M((size_t)nx * ny), src((size_t)std::max(nx, ny)), line((size_t)std::max(px, py)),
        half((size_t)std::max(nx, ny));
    const float scx = (float)(1.0 / px), scy = (float)(1.0 / py);
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) src[x] = cmul(in[(size_t)y * nx + x], adjoint ? conj(qx[x]) : fx[x]);
        fwx(src.data(), 1, line.data(), 1, twx.data());
        for (int i = 0; i < px; ++i) line[i] = adjoint ? cmulc(line[i], hx[i]) : cmul(line[i], hx[i]);
        ivx(line.data(), 1, half.data(), 1, twx.data());
        for (int x = 0; x < nx; ++x) M[(size_t)x * ny + y] = cmul(cscale(half[x], scx), adjoint ? conj(fx[x]) : qx[x]);
    }
    for (int x = 0; x < nx; ++x) {
        for (int y = 0; y < ny; ++y) src[y] = cmul(M[(size_t)x * ny + y], adjoint ? conj(qy[y]) : fy[y]);
        fwy(src.data(), 1, line.data(), 1, twy.data());
        for (int i = 0; i < py; ++i) line[i] = adjoint ? cmulc(line[i], hy[i]) : cmul(line[i], hy[i]);
        ivy(line.data(), 1, half.data(), 1, twy.data());
        for (int y = 0; y < ny; ++y) out[(size_t)y * nx + x] = cmul(cscale(half[y], scy), adjoint ? conj(fy[y]) : qy[y]);
    }
    return CWO_OK;
}

extern "C" cwo_status cwo_debug_asm_h(int px, int py, double dx, double dy, double lambda, double z, int* mode_out,
                                      float* out_ri) {
    using namespace cwo;
    using namespace cwo::host;
    if (!mode_out || !out_ri || px < 32 || py < 32 || px > 8192 || py > 8192 || (px & (px - 1)) ||
        (py & (py - 1)) || !(dx > 0) || !(dy > 0) || !(lambda > 0) || !std::isfinite(z))
        return CWO_ERR_INVALID_ARG;
    std::vector<float4> ax(px), ay(py);
    float K = 0.f;
    make_h_tables(px, py, dx, dy, lambda, z, false, false, ax.data(), ay.data(), nullptr, nullptr, &K);
    const int tmode = asm_tail_mode(px, py, dx, dy, lambda, z);
    const std::vector<int> kbx = bin_table(AxisGeo(px)), kby = bin_table(AxisGeo(py));
    const double sx = lambda * lambda / ((double)px * dx * (double)px * dx);
    const double sy = lambda * lambda / ((double)py * dy * (double)py * dy);
    float2* out = (float2*)out_ri;
    for (int i = 0; i < py; ++i)
        for (int c = 0; c < px; ++c) {
            float2 h;
            if (tmode == 2) h = asm_h_fp64(kbx[c], kby[i], z / lambda, sx, sy);
            else h = tmode == 0 ? asm_h_reduced<true>(ax[c], ay[i], K) : asm_h_reduced<false>(ax[c], ay[i], K);
            out[(size_t)i * px + c] = h;
        }
    *mode_out = tmode;
    return CWO_OK;
}

extern "C" cwo_status cwo_debug_line_fft(int p, int inverse, const float* in_ri, float* out_ri) {
    using namespace cwo;
    using namespace cwo::host;
    if (!in_ri || !out_ri || p < 32 || p > 8192 || (p & (p - 1))) return CWO_ERR_INVALID_ARG;
    const AxisGeo g(p);
    const std::vector<float4> tw = twiddle_table(g);
    if (!inverse) pick_fwd(p)((const float2*)in_ri, 1, (float2*)out_ri, 1, tw.data());
    else pick_inv(p)((const float2*)in_ri, 1, (float2*)out_ri, 1, tw.data());
    return CWO_OK;
}
