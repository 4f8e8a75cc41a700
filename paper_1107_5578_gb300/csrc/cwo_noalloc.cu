// cwo_noalloc.cu -- an angular-spectrum propagation that allocates no memory.
//
// Some callers cannot allocate device memory when they propagate: a host that has handed the
// whole device to its own allocator and forbids side allocations, a real-time loop that must not
// risk the implicit device synchronisation a cudaMalloc may cause, or code that runs where the
// surrounding framework has no allocator to offer.  cwo_propagate_asm_noalloc serves them: the
// caller passes only the input and output fields, and everything else the three passes need --
// the 2Nx-wide intermediate and the per-axis tables -- lives in file-scope __device__ arrays of a
// fixed maximum size that every GPU loading this library keeps until the process exits.
//
// Limits: Nx, Ny <= CWO_NOALLOC_MAX_SIDE (1024), so the intermediate is at most 1024 x 2048
// complex64 (16 MiB).  Every call reuses the same arrays: two calls whose work overlaps on the GPU
// (different streams, or different host threads) race and corrupt each other's results.
// Nothing in the arrays needs to start at zero: each call regenerates every table entry and the
// first pass writes every intermediate element before any later pass reads it.
//
// The tables are generated on the GPU in double precision by a small setup kernel, with the same
// formulas as the host-side plan tables (cwo_tables.cpp), so no host-to-device copy is needed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "../../include/cwo.h"
#include "cwo_fft.cuh"
#include "cwo_internal.h"

#define CWO_NOALLOC_MAX_SIDE 1024

namespace {

constexpr int kMaxP = 2 * CWO_NOALLOC_MAX_SIDE;
constexpr int kMaxTw = cwo::Geo<kMaxP>::TW_WORDS;          // compact per-stage twiddle blocks

static __device__ __align__(256) float2 g_scratch[(size_t)CWO_NOALLOC_MAX_SIDE * kMaxP];
static __device__ __align__(256) float4 g_tw_x[kMaxTw];
static __device__ __align__(256) float4 g_tw_y[kMaxTw];
static __device__ __align__(256) float4 g_ax[kMaxP];
static __device__ __align__(256) float4 g_ay[kMaxP];
static __device__ __align__(256) int g_kb_x[kMaxP];
static __device__ __align__(256) int g_kb_y[kMaxP];
static __device__ __align__(256) int2 g_pairs[kMaxP / 2 + 1];
static __device__ __align__(256) float g_kf[1];
static __device__ __align__(256) int g_status[1];

struct Addrs {
    float2* scratch;
    float4 *tw_x, *tw_y, *ax, *ay;
    int *kb_x, *kb_y;
    int2* pairs;
    float* kf;
    int* status;
};

cwo_status fail(cwo_status st, const char* msg) {
    cwo::set_last_error(msg);   // reported by cwo_last_error()
    return st;
}

// host addresses of the arrays, resolved once per device with that device current
std::mutex g_mu;
bool g_have[64];
Addrs g_addr[64];

cudaError_t resolve(int dev, Addrs* out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!g_have[dev]) {
        Addrs a{};
        cudaError_t e;
        if ((e = cudaGetSymbolAddress((void**)&a.scratch, g_scratch)) ||
            (e = cudaGetSymbolAddress((void**)&a.tw_x, g_tw_x)) || (e = cudaGetSymbolAddress((void**)&a.tw_y, g_tw_y)) ||
            (e = cudaGetSymbolAddress((void**)&a.ax, g_ax)) || (e = cudaGetSymbolAddress((void**)&a.ay, g_ay)) ||
            (e = cudaGetSymbolAddress((void**)&a.kb_x, g_kb_x)) || (e = cudaGetSymbolAddress((void**)&a.kb_y, g_kb_y)) ||
            (e = cudaGetSymbolAddress((void**)&a.pairs, g_pairs)) || (e = cudaGetSymbolAddress((void**)&a.kf, g_kf)) ||
            (e = cudaGetSymbolAddress((void**)&a.status, g_status)))
            return e;
        g_addr[dev] = a;
        g_have[dev] = true;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

// ---- device-side table generation (same formulas as cwo_tables.cpp) ----
__device__ int dev_freq_of_idx(int P, int idx) {
    int lg = 0;
    while ((1 << lg) < P) ++lg;
    const int nst = (lg + 3) / 4, rlast = 1 << (lg - 4 * (nst - 1)), T = P / 16;
    const int pos = 16 * (idx % T) + idx / T;
    int k = 0, below = 1, above = P;
    for (int s = 0; s < nst; ++s) {
        const int r = s == nst - 1 ? rlast : 16;
        above /= r;
        k += ((pos / above) % r) * below;
        below *= r;
    }
    return k;
}

// axis index of frequency k: its DIF position pos, stored at register pos % 16 of thread pos / 16
__device__ int dev_idx_of_freq(int P, int k) {
    int lg = 0;
    while ((1 << lg) < P) ++lg;
    const int nst = (lg + 3) / 4, rlast = 1 << (lg - 4 * (nst - 1)), T = P / 16;
    int pos = 0, below = 1, above = P;
    for (int s = 0; s < nst; ++s) {
        const int r = s == nst - 1 ? rlast : 16;
        above /= r;
        pos += ((k / below) % r) * above;
        below *= r;
    }
    return (pos % 16) * T + pos / 16;
}

__device__ double dev_frac01(double x) { return x - floor(x); }

struct AxisParams {
    int P;
    double pitch;
    bool is_x;
};

__global__ void k_setup(AxisParams ax, AxisParams ay, double lambda, double z, float4* tw_x, float4* tw_y,
                        float4* tax, float4* tay, int* kbx, int* kby, int2* pairs, float* kf, int* status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) status[0] = 0;   // the row passes' bounded waits set it; each call starts clear
    for (int a = 0; a < 2; ++a) {
        const AxisParams g = a == 0 ? ax : ay;
        if (i >= g.P) continue;
        float4* tw = a == 0 ? tw_x : tw_y;
        float4* tab = a == 0 ? tax : tay;
        int* kb = a == 0 ? kbx : kby;
        int lg = 0;
        while ((1 << lg) < g.P) ++lg;
        const int nst = (lg + 3) / 4;
        // twiddles: entry i of each stage block, laid out [kp][j], j = t mod S_s (8 S_s entries)
        for (int s = 0, off = 0; s + 1 < nst; ++s) {
            const int L = g.P >> (4 * s), S = L / 16;
            if (i < 8 * S) {
                const int kp = i / S, j = i % S;
                double re[2], im[2];
                for (int h = 0; h < 2; ++h) {
                    const long long jk = (long long)j * (2 * kp + 1 + h) % L;
                    sincospi(-2.0 * (double)jk / (double)L, &im[h], &re[h]);
                }
                tw[off + i] = make_float4((float)re[0], (float)im[0], (float)re[1], (float)im[1]);
            }
            off += 8 * S;
        }
        const int k = dev_freq_of_idx(g.P, i);
        const int kt = k < g.P / 2 ? k : k - g.P;
        kb[i] = kt;
        // angular-spectrum axis table {a, W (- frac K on x), u_hi, u_lo}
        const double K = z / lambda;
        const double c0 = g.is_x ? dev_frac01(K) : 0.0;
        const double sgn = (g.is_x && K < 0) ? -1.0 : 1.0;
        const double rt = sqrt(fabs(K)) * 0.5;
        const double Pd = (double)g.P * g.pitch;
        const double c1 = z * lambda / (2.0 * Pd * Pd);
        const double c2 = z * lambda * lambda * lambda / (8.0 * Pd * Pd * Pd * Pd);
        const double k2 = (double)kt * (double)kt;
        const double av = lambda * lambda * k2 / (Pd * Pd);
        const double W = dev_frac01(dev_frac01(c1 * k2) + dev_frac01(c2 * k2 * k2)) - c0;
        const double u = sgn * rt * av;
        const float uh = (float)u;
        tab[i] = make_float4((float)av, (float)W, uh, (float)(u - (double)uh));
        if (a == 0 && i <= g.P / 2)     // storage columns of +k and -k, k = i
            pairs[i] = make_int2(dev_idx_of_freq(g.P, i), dev_idx_of_freq(g.P, (g.P - i) % g.P));
        if (a == 0 && i == 0) kf[0] = (float)K;
    }
}

int asm_mode(int px, int py, double dx, double dy, double lambda, double z) {
    const double K = std::fabs(z / lambda);
    const double smax = lambda * lambda * (0.25 / (dx * dx) + 0.25 / (dy * dy));
    if (smax < 0.5 && K * (429.0 / 32768.0) * std::pow(smax, 8) / (1.0 - smax) < 1e-8) return cwo::HMODE_ASM_POLY;
    if (smax <= 1.0) {
        const double q = std::sqrt(1.0 - smax), d = 1.0 + q;
        if (K * smax * smax * smax * (3.0 + q) / (8.0 * d * d * d) <= 4.0) return cwo::HMODE_ASM_EXACT;
    }
    (void)px; (void)py;
    return cwo::HMODE_ASM_FP64;
}

}  // namespace

extern "C" cwo_status cwo_propagate_asm_noalloc(int nx, int ny, double dx, double dy, double lambda, double z,
                                                const void* in_c64, void* out_c64, void* cuda_stream) {
    if (nx < CWO_MIN_SIDE || ny < CWO_MIN_SIDE || (nx & (nx - 1)) || (ny & (ny - 1)))
        return fail(CWO_ERR_INVALID_ARG, "Nx and Ny must be powers of two >= 16");
    if (nx > CWO_NOALLOC_MAX_SIDE || ny > CWO_NOALLOC_MAX_SIDE)
        return fail(CWO_ERR_INVALID_ARG, "cwo_propagate_asm_noalloc: Nx and Ny are limited to 1024 (its fixed scratch)");
    if (!(dx > 0) || !(dy > 0) || !(lambda > 0) || !std::isfinite(dx) || !std::isfinite(dy) || !std::isfinite(lambda) ||
        !std::isfinite(z))
        return fail(CWO_ERR_INVALID_ARG, "pitches and wavelength must be finite and > 0, z finite");
    if (!in_c64 || !out_c64) return fail(CWO_ERR_INVALID_ARG, "input and output must be non-NULL device pointers");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(CWO_ERR_CUDA, cudaGetErrorString(e));
    cwo_status st;
    // both fields must be device memory of the current device, 8-byte aligned and large enough for
    // nx * ny complex64 values inside one allocation (a host pointer or a short buffer would make
    // the passes read or write memory that is not theirs)
    const size_t field_bytes = (size_t)nx * (size_t)ny * 8u;
    if ((st = (cwo_status)cwo::check_device_buffer(in_c64, field_bytes, dev, "input")) ||
        (st = (cwo_status)cwo::check_device_buffer(out_c64, field_bytes, dev, "output")))
        return st;
    Addrs a{};
    if ((e = resolve(dev, &a)) != cudaSuccess) return fail(CWO_ERR_CUDA, cudaGetErrorString(e));
    const int px = 2 * nx, py = 2 * ny;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const unsigned nthreads = 256, nblocks = (unsigned)((std::max(px, py) + nthreads - 1) / nthreads);
    k_setup<<<nblocks, nthreads, 0, s>>>(AxisParams{px, dx, true}, AxisParams{py, dy, false}, lambda, z, a.tw_x, a.tw_y,
                                         a.ax, a.ay, a.kb_x, a.kb_y, a.pairs, a.kf, a.status);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(CWO_ERR_CUDA, cudaGetErrorString(e));
    cwo::HParams hp{};
    hp.mode = asm_mode(px, py, dx, dy, lambda, z);
    hp.ax = a.ax; hp.ay = a.ay; hp.kf = a.kf;
    hp.kbx = a.kb_x; hp.kby = a.kb_y; hp.pairs = a.pairs; hp.npairs = px / 2 + 1;
    hp.K = z / lambda;
    hp.sx = lambda * lambda / ((double)px * dx * (double)px * dx);
    hp.sy = lambda * lambda / ((double)py * dy * (double)py * dy);
    const float2* fin = (const float2*)in_c64;
    float2* fout = (float2*)out_c64;
    const long long field = (long long)nx * ny, wstride = (long long)ny * px;
    const float scale = (float)(1.0 / ((double)px * (double)py));
    CUtensorMap wmap_f, wmap_i;   // host-side descriptions of g_scratch for the TMA copies (no allocation)
    if (cwo::make_intermediate_map(&wmap_f, a.scratch, ny, px, 1, cwo::row_block_rows(px, false)) != cudaSuccess ||
        cwo::make_intermediate_map(&wmap_i, a.scratch, ny, px, 1, cwo::row_block_rows(px, true)) != cudaSuccess)
        return fail(CWO_ERR_CUDA, "tensor map of the fixed scratch");
    if ((e = cwo::launch_row_fwd(px, fin, field, &wmap_f, 0, ny, 1, a.tw_x, a.status, s)) ||
        (e = cwo::launch_col(py, a.scratch, wstride, a.scratch, wstride, px, 1, a.tw_y, hp, s)) ||
        (e = cwo::launch_row_inv(px, &wmap_i, 0, fout, field, ny, 1, scale, a.tw_x, a.status, s)))
        return fail(CWO_ERR_CUDA, cudaGetErrorString(e));
    return CWO_OK;
}
