// cwo_tables.cpp -- FP64 host computation of the per-plan tables.
//
//  * axis permutation: the forward FFT leaves frequency k at its DIF (digit-reversed) position;
//    the passes store and index it by axis index idx = e*T + t (register e of thread t).
//  * twiddles W_{L_s}^{(t mod S_s) k} of every radix-16 stage, correctly rounded from FP64.
//  * Fresnel (Eq. fre_conv_fft): the separable factors of FFT[h_F] -- 1-D DFTs of
//    h(d) = exp(i pi (d pitch)^2 / (lambda z)) over the padded axis -- and C, with every phase
//    reduced modulo one cycle in FP64.
//  * angular spectrum (Eq. ang2): per-axis parts of the phase K sqrt(1 - s), K = z / lambda,
//    reduced modulo one cycle in FP64 (see cwo_h.cuh for the split).
#include "cwo_tables.h"

#include <algorithm>
#include <cmath>
#include <map>
#include <memory>
#include <mutex>

#include "../../include/cwo.h"

namespace cwo {
namespace host {

namespace {
constexpr double kPi = 3.14159265358979323846264338327950288;
int ilog2i(int n) { int l = 0; while ((1 << l) < n) ++l; return l; }
}  // namespace

double frac01(double x) { return x - std::floor(x); }

AxisGeo::AxisGeo(int p) : P(p), T(p / 16) {
    const int lg = ilog2i(p);
    NST = (lg + 3) / 4;
    RLAST = 1 << (lg - 4 * (NST - 1));
}

// pos = sum_s k_s P / (r_0..r_s)  and  k = sum_s k_s (r_0..r_{s-1})
int AxisGeo::freq_of_pos(int pos) const {
    int k = 0, below = 1, above = P;
    for (int s = 0; s < NST; ++s) {
        const int r = radix(s);
        above /= r;
        const int ks = (pos / above) % r;
        k += ks * below;
        below *= r;
    }
    return k;
}

std::vector<float4> twiddle_table(const AxisGeo& g) {
    // per radix-16 stage s (all but the last): 8 S_s float4 laid out [kp][j], kp = 0..7,
    // j = 0..S_s-1 (= t mod S_s), holding (W_L^{j (2kp+1)}, W_L^{j (2kp+2)}), L = L_s
    std::vector<float4> tw((size_t)g.tw_off(g.NST - 1));
    for (int s = 0; s + 1 < g.NST; ++s) {
        const int L = g.len(s), S = g.stride(s);
        for (int kp = 0; kp < 8; ++kp)
            for (int j = 0; j < S; ++j) {
                double re[2], im[2];
                for (int h = 0; h < 2; ++h) {
                    const long long jk = (long long)j * (2 * kp + 1 + h) % L;
                    const double ang = -2.0 * kPi * (double)jk / (double)L;
                    re[h] = std::cos(ang);
                    im[h] = std::sin(ang);
                }
                tw[(size_t)g.tw_off(s) + (size_t)kp * S + j] =
                    make_float4((float)re[0], (float)im[0], (float)re[1], (float)im[1]);
            }
    }
    return tw;
}

std::vector<int2> mirror_pairs(const AxisGeo& g) {
    std::vector<int> where(g.P);
    for (int i = 0; i < g.P; ++i) where[g.freq_of_idx(i)] = i;
    std::vector<int2> pr;
    pr.reserve(g.P / 2 + 1);
    for (int k = 0; k <= g.P / 2; ++k) pr.push_back(make_int2(where[k], where[(g.P - k) % g.P]));
    return pr;
}

std::vector<int> bin_table(const AxisGeo& g) {
    std::vector<int> b(g.P);
    for (int i = 0; i < g.P; ++i) b[i] = g.signed_bin(g.freq_of_idx(i));
    return b;
}

std::vector<int> split_axis_index(int P) {
    const AxisGeo g(P), gq(P / 2);
    std::vector<int> where(P);
    for (int i = 0; i < P; ++i) where[g.freq_of_idx(i)] = i;
    std::vector<int> out(P);
    for (int i = 0; i < P; ++i) {
        const int h = i / gq.P, idx = i % gq.P;
        out[i] = where[2 * gq.freq_of_idx(idx) + h];
    }
    return out;
}

std::vector<float2> split_phase(int P) {
    std::vector<float2> w(P / 2);
    for (int n = 0; n < P / 2; ++n) {
        const double ang = -2.0 * kPi * (double)n / (double)P;
        w[n] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
    return w;
}

// Per-length caches: twiddles W_P^j (j < P/2) of the FP64 FFT, and the axis-index lists of the
// frequency pairs {+k, -k}.  Built once per length, shared by every thread (read-only after).
namespace {
struct AxisCache {
    std::vector<double> wre, wim;        // W_P^j = exp(-2 pi i j / P), j < P/2
    std::vector<int> kabs;               // |signed bin| of each axis index, 0 .. P/2
    std::vector<int> first, second;      // for |k| = 0 .. P/2: the axis indices of +k and -k
};
std::mutex g_cache_mu;
std::map<int, std::unique_ptr<AxisCache>> g_cache;

const AxisCache& axis_cache(int P) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto& slot = g_cache[P];
    if (!slot) {
        auto c = std::make_unique<AxisCache>();
        c->wre.resize(P / 2);
        c->wim.resize(P / 2);
        for (int j = 0; j < P / 2; ++j) {
            const double ang = -2.0 * kPi * (double)j / (double)P;
            c->wre[j] = std::cos(ang);
            c->wim[j] = std::sin(ang);
        }
        const AxisGeo g(P);
        c->kabs.resize(P);
        c->first.assign(P / 2 + 1, -1);
        c->second.assign(P / 2 + 1, -1);
        for (int i = 0; i < P; ++i) {
            const int k = std::abs(g.signed_bin(g.freq_of_idx(i)));
            c->kabs[i] = k;
            (c->first[k] < 0 ? c->first[k] : c->second[k]) = i;
        }
        slot = std::move(c);
    }
    return *slot;
}
}  // namespace

// Forward DFT in FP64 (self-sorting Stockham form): one radix-2 pass when log2 n is odd, then
// radix-4 passes.  A pass of radix r takes x[j m + k + q l' m] (q < r) to
// y[(r j + q) m + k] = (sum_p x_p W_r^{p q}) W_n^{j q m}, with l' = l / r, for j < l', k < m.
void fft64(std::vector<cd>& xv) {
    const int n = (int)xv.size();
    const AxisCache& c = axis_cache(n);
    std::vector<cd> yv(n);
    double* x = reinterpret_cast<double*>(xv.data());
    double* y = reinterpret_cast<double*>(yv.data());
    auto twid = [&](long long i, double& wr, double& wi) {   // W_n^i, i < n (the table holds i < n/2)
        if (i < n / 2) { wr = c.wre[(size_t)i]; wi = c.wim[(size_t)i]; }
        else { wr = -c.wre[(size_t)(i - n / 2)]; wi = -c.wim[(size_t)(i - n / 2)]; }
    };
    int l = n, m = 1;
    if (ilog2i(n) % 2 == 1) {   // radix 2
        const int lr = l / 2;
        for (int j = 0; j < lr; ++j) {
            double wr, wi;
            twid((long long)j * m, wr, wi);
            const double* a = x + 2 * (size_t)j * m;
            const double* b = x + 2 * ((size_t)j * m + (size_t)lr * m);
            double* o0 = y + 2 * (2 * (size_t)j * m);
            double* o1 = o0 + 2 * (size_t)m;
            for (int k = 0; k < m; ++k) {
                const double ar = a[2 * k], ai = a[2 * k + 1], br = b[2 * k], bi = b[2 * k + 1];
                o0[2 * k] = ar + br;
                o0[2 * k + 1] = ai + bi;
                const double dr = ar - br, di = ai - bi;
                o1[2 * k] = dr * wr - di * wi;
                o1[2 * k + 1] = dr * wi + di * wr;
            }
        }
        std::swap(x, y);
        l = lr;
        m *= 2;
    }
    while (l >= 4) {            // radix 4
        const int lr = l / 4;
        const size_t s = (size_t)lr * m;   // distance between the four inputs
        for (int j = 0; j < lr; ++j) {
            double w1r, w1i, w2r, w2i, w3r, w3i;
            twid((long long)j * m, w1r, w1i);
            twid(2LL * j * m, w2r, w2i);
            twid(3LL * j * m, w3r, w3i);
            const double* a = x + 2 * (size_t)j * m;
            double* o = y + 2 * (4 * (size_t)j * m);
            for (int k = 0; k < m; ++k) {
                const double a0r = a[2 * k], a0i = a[2 * k + 1];
                const double a1r = a[2 * (k + s)], a1i = a[2 * (k + s) + 1];
                const double a2r = a[2 * (k + 2 * s)], a2i = a[2 * (k + 2 * s) + 1];
                const double a3r = a[2 * (k + 3 * s)], a3i = a[2 * (k + 3 * s) + 1];
                const double t0r = a0r + a2r, t0i = a0i + a2i, t1r = a0r - a2r, t1i = a0i - a2i;
                const double t2r = a1r + a3r, t2i = a1i + a3i;
                const double t3r = a1i - a3i, t3i = a3r - a1r;   // -i (a1 - a3)
                o[2 * k] = t0r + t2r;
                o[2 * k + 1] = t0i + t2i;
                const double x1r = t1r + t3r, x1i = t1i + t3i;
                const double x2r = t0r - t2r, x2i = t0i - t2i;
                const double x3r = t1r - t3r, x3i = t1i - t3i;
                o[2 * (k + m)] = x1r * w1r - x1i * w1i;
                o[2 * (k + m) + 1] = x1r * w1i + x1i * w1r;
                o[2 * (k + 2 * m)] = x2r * w2r - x2i * w2i;
                o[2 * (k + 2 * m) + 1] = x2r * w2i + x2i * w2r;
                o[2 * (k + 3 * m)] = x3r * w3r - x3i * w3i;
                o[2 * (k + 3 * m) + 1] = x3r * w3i + x3i * w3r;
            }
        }
        std::swap(x, y);
        l = lr;
        m *= 4;
    }
    if (x != reinterpret_cast<double*>(xv.data())) xv.swap(yv);
}

std::vector<cd> fresnel_axis_dft(int P, double pitch, double lambda, double z) {
    std::vector<cd> h(P);
    const double c = pitch * pitch / (2.0 * lambda * z);   // cycles per d^2
    auto cis = [](double cycles) {
        const double ph = 2.0 * kPi * frac01(cycles);
        return cd(std::cos(ph), std::sin(ph));
    };
    // h(d) = exp(2 pi i c d^2) = h(-d): d = 0 .. P/2, mirrored.  From exact values at every 64th d,
    // h(d + 1) = h(d) s(d) with s(d) = exp(2 pi i c (2d + 1)) and s(d + 1) = s(d) exp(4 pi i c): two
    // complex products per sample instead of a sine and a cosine (relative error below 1e-13)
    const cd r = cis(2.0 * c);
    for (int d0 = 0; d0 <= P / 2; d0 += 64) {
        cd v = cis(c * (double)d0 * (double)d0);
        cd st = cis(c * (2.0 * (double)d0 + 1.0));
        const int d1 = std::min(d0 + 64, P / 2 + 1);
        for (int d = d0; d < d1; ++d) {
            h[d] = v;
            if (d > 0 && d < P / 2) h[P - d] = v;
            v *= st;
            st *= r;
        }
    }
    fft64(h);
    return h;
}

cd fresnel_coeff(double dx, double dy, double lambda, double z, bool literal_scale) {
    const double ph = frac01(z / lambda);
    cd c = cd(std::cos(2.0 * kPi * ph), std::sin(2.0 * kPi * ph)) / cd(0.0, lambda * z);
    if (!literal_scale) c *= dx * dy;
    return c;
}

void asm_axis_table(const AxisGeo& g, double pitch, double lambda, double z, bool is_x, float4* out) {
    const double K = z / lambda;
    const double c0 = is_x ? frac01(K) : 0.0;
    const double sgn = (is_x && K < 0) ? -1.0 : 1.0;
    const double rt = std::sqrt(std::fabs(K)) * 0.5;
    const double Pd = (double)g.P * pitch;
    const double c1 = z * lambda / (2.0 * Pd * Pd);                              // K a / 2   per kt^2
    const double c2 = z * lambda * lambda * lambda / (8.0 * Pd * Pd * Pd * Pd);  // K a^2 / 8 per kt^4
    // every entry depends on kt^2 only: evaluate |kt| = 0 .. P/2 once, store at both indices
    const AxisCache& c = axis_cache(g.P);
    for (int k = 0; k <= g.P / 2; ++k) {
        const double kt = (double)k;
        const double k2 = kt * kt;
        const double a = lambda * lambda * k2 / (Pd * Pd);
        const double W = frac01(frac01(c1 * k2) + frac01(c2 * k2 * k2)) - c0;
        const double u = sgn * rt * a;
        const float uh = (float)u;
        const float ul = (float)(u - (double)uh);
        const float4 v = make_float4((float)a, (float)W, uh, ul);
        out[c.first[k]] = v;
        if (c.second[k] >= 0) out[c.second[k]] = v;
    }
}

bool in_window(double f, double wc, double ww) { return !(ww > 0) || std::fabs(f - wc) <= 0.5 * ww; }

void asm_axis_table_shifted(const AxisGeo& g, double pitch, double lambda, double z, bool is_x, double shift,
                            double wc, double ww, float4* out) {
    const double K = z / lambda;
    const double c0 = is_x ? frac01(K) : 0.0;
    const double sgn = (is_x && K < 0) ? -1.0 : 1.0;
    const double rt = std::sqrt(std::fabs(K)) * 0.5;
    const double Pd = (double)g.P * pitch;
    const double c1 = z * lambda / (2.0 * Pd * Pd);
    const double c2 = z * lambda * lambda * lambda / (8.0 * Pd * Pd * Pd * Pd);
    for (int i = 0; i < g.P; ++i) {
        const double kt = (double)g.signed_bin(g.freq_of_idx(i));
        const double f = kt / Pd;
        if (!in_window(f, wc, ww)) {
            out[i] = make_float4(2.0f, 0.f, 0.f, 0.f);
            continue;
        }
        const double k2 = kt * kt;
        const double a = lambda * lambda * k2 / (Pd * Pd);
        // the kernel forms psi = -(W_x + W_y) - ...: subtracting frac(shift f) adds shift f cycles
        const double W = frac01(frac01(c1 * k2) + frac01(c2 * k2 * k2) + frac01(-shift * f)) - c0;
        const double u = sgn * rt * a;
        const float uh = (float)u;
        const float ul = (float)(u - (double)uh);
        out[i] = make_float4((float)a, (float)W, uh, ul);
    }
}

void window_bins(const AxisGeo& g, double pitch, double wc, double ww, int* lo, int* hi) {
    const double Pd = (double)g.P * pitch;
    int l = g.P, h = -g.P - 1;
    for (int kt = -g.P / 2; kt < g.P / 2; ++kt)
        if (in_window((double)kt / Pd, wc, ww)) { l = std::min(l, kt); h = std::max(h, kt); }
    *lo = l;
    *hi = h;
}

double band_limit_freq(int p, double pitch, double lambda, double z) {
    const double df = 1.0 / ((double)p * pitch);
    return 1.0 / (lambda * std::sqrt((2.0 * df * z) * (2.0 * df * z) + 1.0));
}


namespace {
float2 unit_cycles(double cyc) {
    const double ph = 2.0 * kPi * frac01(cyc);
    return make_float2((float)std::cos(ph), (float)std::sin(ph));
}
}  // namespace

void shifted_fresnel_axis(int n, double p0, double p1, double o0, double o1, double lambda, double z, cd coeff,
                          float2* f, float2* q, float2* h) {
    const double lz = lambda * z;
    const double S = p0 * p1 / lz;
    for (int a = 0; a < n; ++a) {
        const double m = (double)(a - n / 2);
        const double x0 = m * p0 + o0, x1 = m * p1 + o1;
        const double chirp = frac01(0.5 * S * m * m);
        f[a] = unit_cycles(frac01(x0 * x0 / (2.0 * lz)) + frac01(-m * p0 * o1 / lz) - chirp);
        const double ph = 2.0 * kPi * frac01(frac01(x1 * x1 / (2.0 * lz)) + frac01(-o0 * x1 / lz) - chirp);
        const double cr = std::cos(ph), ci = std::sin(ph);
        q[a] = make_float2((float)(coeff.real() * cr - coeff.imag() * ci), (float)(coeff.real() * ci + coeff.imag() * cr));
    }
    const int P = 2 * n;
    std::vector<cd> hd(P);
    for (int d = 0; d <= P / 2; ++d) {   // exp(i pi S d^2) is even in d
        const double ph = 2.0 * kPi * frac01(0.5 * S * (double)d * (double)d);
        hd[d] = cd(std::cos(ph), std::sin(ph));
        if (d > 0 && d < P / 2) hd[P - d] = hd[d];
    }
    fft64(hd);
    const AxisCache& c = axis_cache(P);
    for (int i = 0; i < P; ++i) {
        const cd v = hd[c.kabs[i]];
        h[i] = make_float2((float)v.real(), (float)v.imag());
    }
}

void fourier_tables(int nx, int ny, double dx, double dy, double lambda, double z, bool literal_scale,
                    float2* pre_x, float2* pre_y, float2* post_x, float2* post_y, int* st_of_col, int* row_of_idx) {
    const double lz = lambda * z;
    for (int m = 0; m < nx; ++m) {
        const double x = (double)(m - nx / 2) * dx;
        pre_x[m] = unit_cycles(x * x / (2.0 * lz));
    }
    for (int n = 0; n < ny; ++n) {
        const double y = (double)(n - ny / 2) * dy;
        pre_y[n] = unit_cycles(y * y / (2.0 * lz));
    }
    // C = exp(i 2 pi z / lambda) / (i lambda z) (times dx dy unless literal), in FP64
    const double cph = 2.0 * kPi * frac01(z / lambda);
    cd C = cd(std::cos(cph), std::sin(cph)) / cd(0.0, lz);
    if (!literal_scale) C *= dx * dy;
    const AxisGeo gx(nx), gy(ny);
    std::vector<int> where(nx);
    for (int i = 0; i < nx; ++i) where[gx.freq_of_idx(i)] = i;
    const double qx = lz / (2.0 * (double)nx * nx * dx * dx);   // cycles per kt^2
    for (int col = 0; col < nx; ++col) {
        const int kt = col - nx / 2;
        const double cyc = frac01(qx * (double)kt * (double)kt) + 0.5 * (double)(kt & 1);
        const double ph = 2.0 * kPi * frac01(cyc);
        const double cr = std::cos(ph), ci = std::sin(ph);
        post_x[col] = make_float2((float)(C.real() * cr - C.imag() * ci), (float)(C.real() * ci + C.imag() * cr));
        st_of_col[col] = where[(kt + nx) % nx];
    }
    const double qy = lz / (2.0 * (double)ny * ny * dy * dy);
    for (int i = 0; i < ny; ++i) {
        const int kt = gy.signed_bin(gy.freq_of_idx(i));
        post_y[i] = unit_cycles(frac01(qy * (double)kt * (double)kt) + 0.5 * (double)(kt & 1));
        row_of_idx[i] = kt + ny / 2;
    }
}

int asm_tail_mode(int px, int py, double dx, double dy, double lambda, double z) {
    (void)px; (void)py;
    const double K = std::fabs(z / lambda);
    const double smax = lambda * lambda * (0.25 / (dx * dx) + 0.25 / (dy * dy));
    if (smax < 0.5 && K * (429.0 / 32768.0) * std::pow(smax, 8) / (1.0 - smax) < 1e-8) return 0;
    if (smax <= 1.0) {
        const double q = std::sqrt(1.0 - smax), d = 1.0 + q;
        const double tail = K * smax * smax * smax * (3.0 + q) / (8.0 * d * d * d);
        if (tail <= 4.0) return 1;
    }
    return 2;
}

void make_h_tables(int px, int py, double dx, double dy, double lambda, double z, bool fresnel,
                   bool literal_scale, float4* ax, float4* ay, float2* hx, float2* hy, float* kf) {
    const AxisGeo gx(px), gy(py);
    if (!fresnel) {
        asm_axis_table(gx, dx, lambda, z, true, ax);
        asm_axis_table(gy, dy, lambda, z, false, ay);
        if (kf) *kf = (float)(z / lambda);
    } else {
        const std::vector<cd> Hx = fresnel_axis_dft(px, dx, lambda, z);
        std::vector<cd> Hy_own;
        if (!(py == px && dy == dx)) Hy_own = fresnel_axis_dft(py, dy, lambda, z);
        const std::vector<cd>& Hy = Hy_own.empty() ? Hx : Hy_own;
        const cd C = fresnel_coeff(dx, dy, lambda, z, literal_scale);
        const double cr = C.real(), ci = C.imag();
        // h_F is even in d (the unpaired sample d = -P/2 contributes (-1)^k, also even), so
        // H[k] = H[P - k]; one representative per pair keeps the float tables exactly even.  The
        // frequencies are walked in natural order and each value is written to the axis indices
        // of +k and -k (reading H in the digit-reversed index order missed the cache on every
        // element: ~10 ns each at P = 8192)
        const AxisCache& cx = axis_cache(px);
        for (int k = 0; k <= px / 2; ++k) {
            const cd h = Hx[k];
            const float2 v = make_float2((float)(cr * h.real() - ci * h.imag()), (float)(cr * h.imag() + ci * h.real()));
            hx[cx.first[k]] = v;
            if (cx.second[k] >= 0) hx[cx.second[k]] = v;
        }
        const AxisCache& cy = axis_cache(py);
        for (int k = 0; k <= py / 2; ++k) {
            const cd h = Hy[k];
            const float2 v = make_float2((float)h.real(), (float)h.imag());
            hy[cy.first[k]] = v;
            if (cy.second[k] >= 0) hy[cy.second[k]] = v;
        }
    }
}

}  // namespace host
}  // namespace cwo
