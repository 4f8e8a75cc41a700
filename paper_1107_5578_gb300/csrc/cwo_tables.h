// cwo_tables.h -- FP64 host computation of the per-plan tables (twiddles, axis permutation,
// transfer-function factors).  Shared by the plan code and the host emulator.
#pragma once
#include <cuda_runtime.h>
#include <complex>
#include <vector>

namespace cwo {
namespace host {

using cd = std::complex<double>;

// Axis geometry, mirrored from the device FFT (cwo_fft.cuh): T = P/16 threads, stages of radix
// 16 followed by one stage of radix RLAST.  Axis index idx = e*T + t <-> DIF position 16 t + e.
struct AxisGeo {
    int P, T, NST, RLAST;
    explicit AxisGeo(int p);
    int radix(int s) const { return s == NST - 1 ? RLAST : 16; }
    int len(int s) const { return P >> (4 * s); }
    int stride(int s) const { return len(s) / radix(s); }
    int tw_off(int s) const { return s <= 0 ? 0 : tw_off(s - 1) + 8 * stride(s - 1); }   // float4 units
    int freq_of_pos(int pos) const;   // bin whose forward DIF output lands at position pos
    int freq_of_idx(int idx) const { return freq_of_pos(16 * (idx % T) + idx / T); }
    int signed_bin(int k) const { return k < P / 2 ? k : k - P; }
};

double frac01(double x);
std::vector<float4> twiddle_table(const AxisGeo& g);
std::vector<int> bin_table(const AxisGeo& g);
// storage columns of the frequencies +k and -k for k = 0 .. P/2 (0 and P/2 pair with themselves)
std::vector<int2> mirror_pairs(const AxisGeo& g);
// Split form of a zero-padded axis of P = 2Q points carrying Q samples x_n: its DFT is the pair of
// Q-point DFTs of x_n (frequencies 2k) and of x_n W_P^n (frequencies 2k + 1).  Split axis index
// i = h Q + idx (h = 0 even, 1 odd; idx a Q-point axis index) holds frequency 2 k(idx) + h.
//   split_axis_index[i]: the P-point axis index (AxisGeo(P)) of the frequency at split index i
//   split_phase[n]:      W_P^n for n < Q, correctly rounded from FP64
std::vector<int> split_axis_index(int P);
std::vector<float2> split_phase(int P);
void fft64(std::vector<cd>& x);
std::vector<cd> fresnel_axis_dft(int P, double pitch, double lambda, double z);
cd fresnel_coeff(double dx, double dy, double lambda, double z, bool literal_scale);
void asm_axis_table(const AxisGeo& g, double pitch, double lambda, double z, bool is_x, float4* out);
// Shifted ASM (Eq. shift_ang2): the phase gains shift * f cycles (f = kt / (P pitch)), and bins
// with |f - wc| > ww / 2 (ww > 0) are outside the Rect window: their entry gets a = 2, which the
// kernel's evanescent test (s > 1) turns into H = 0.  Not symmetric in kt.
void asm_axis_table_shifted(const AxisGeo& g, double pitch, double lambda, double z, bool is_x, double shift,
                            double wc, double ww, float4* out);
// signed-bin interval [lo, hi] of the window |kt / (P pitch) - wc| <= ww / 2 (whole axis if ww <= 0)
void window_bins(const AxisGeo& g, double pitch, double wc, double ww, int* lo, int* hi);
// On-axis band limit of the ASM on a padded grid of P = 2N (Matsushima and Shimobaba, Opt.
// Express 17, 19662 (2009)): |f| <= 1 / (lambda sqrt((2 df z)^2 + 1)), df = 1 / (P pitch).
double band_limit_freq(int p, double pitch, double lambda, double z);
// Fresnel diffraction in Fourier form (Eqs. fre_fourier2, fre_fourier3), unpadded Nx x Ny axes:
//   pre_x[m]     source chirp exp(i pi ((m - Nx/2) dx)^2 / (lambda z))          (natural m)
//   post_x[col]  C exp(i pi x2^2 / (lambda z)) (-1)^kt, kt = col - Nx/2, x2 = kt lambda z / (Nx dx)
//   post_y[i]    exp(i pi y2^2 / (lambda z)) (-1)^kt for axis index i of the column FFT
//   st_of_col    storage column (DIF position) holding the frequency of output column col
//   row_of_idx   output row (kt + Ny/2) of axis index i
// every phase reduced modulo one cycle in FP64; (-1)^kt turns the plain DFT into the centred one
// Shifted Fresnel (Eqs. shift_fre1 to shift_fre3), per axis of n samples (source pitch p0 centred
// at o0, destination pitch p1 centred at o1, m = array index - n/2, S = p0 p1 / (lambda z)):
//   f[a] = exp(i pi x0^2 / (lambda z)) exp(-2 pi i m p0 o1 / (lambda z)) exp(-i pi S m^2)
//   q[a] = exp(i pi x1^2 / (lambda z)) exp(-2 pi i o0 x1 / (lambda z)) exp(-i pi S m^2)  (times coeff)
//   h[i] = DFT over the padded axis (2n) of exp(i pi S d^2), d = i (i < n) else i - 2n, at axis
//          index i (DIF order), made exactly even
// phases reduced modulo one cycle in FP64; coeff multiplies q (pass 1 for the y axis).
void shifted_fresnel_axis(int n, double p0, double p1, double o0, double o1, double lambda, double z, cd coeff,
                          float2* f, float2* q, float2* h);
void fourier_tables(int nx, int ny, double dx, double dy, double lambda, double z, bool literal_scale,
                    float2* pre_x, float2* pre_y, float2* post_x, float2* post_y, int* st_of_col, int* row_of_idx);

// transfer-function tables of one parameter set, in axis-index order
struct HTables {
    std::vector<float4> ax, ay;   // angular spectrum
    std::vector<float2> hx, hy;   // Fresnel (hx includes C)
    float K = 0.f;                // z / lambda (angular spectrum tail term)
};
// Which per-element evaluation of the ASM phase remainder a parameter set needs:
// 0 series tail (truncation < 1e-8 cycle), 1 closed-form tail (tail < 4 cycles, FP32 error
// < 1e-6 cycle), 2 FP64 per element.  s_max = lambda^2 (1/(4 dx^2) + 1/(4 dy^2)) at the Nyquist
// corner of the padded grid.
int asm_tail_mode(int px, int py, double dx, double dy, double lambda, double z);

void make_h_tables(int px, int py, double dx, double dy, double lambda, double z, bool fresnel,
                   bool literal_scale, float4* ax, float4* ay, float2* hx, float2* hy, float* kf);

}  // namespace host
}  // namespace cwo
