// cwo_plan.cpp -- host side of libcwo_gb300: plans, FP64 per-axis tables, argument checking,
// scratch management and the C ABI declared in include/cwo.h.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/cwo.h"
#include "../../include/cwo_debug.h"
#include "cwo_internal.h"
#include "cwo_tables.h"

using cd = std::complex<double>;
using namespace cwo::host;

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;
thread_local std::string g_err;

cwo_status fail(cwo_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

cwo_status cuda_fail(cudaError_t e, const char* what) {
    return fail(CWO_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

bool pow2_side(int n) { return n >= CWO_MIN_SIDE && n <= CWO_MAX_SIDE && (n & (n - 1)) == 0; }

// ------------------------------------------------------------------------------------------
// driver entry point for allocation-range checks (avoids a link-time dependency on libcuda)
// ------------------------------------------------------------------------------------------
typedef CUresult (*PFN_memGetAddressRange)(CUdeviceptr*, size_t*, CUdeviceptr);
PFN_memGetAddressRange get_addr_range_fn() {
    static PFN_memGetAddressRange fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_memGetAddressRange)p;
    });
    return fn;
}

// Check that [ptr, ptr + bytes) is device memory of `device` inside one allocation.
cwo_status check_device_range(const void* ptr, size_t bytes, int device, const char* name) {
    if (!ptr) return fail(CWO_ERR_INVALID_ARG, "%s is NULL", name);
    if ((uintptr_t)ptr % 8 != 0) return fail(CWO_ERR_INVALID_ARG, "%s is not 8-byte aligned", name);
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(CWO_ERR_INVALID_ARG, "%s: not a CUDA pointer (%s)", name, cudaGetErrorName(e));
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
        return fail(CWO_ERR_INVALID_ARG, "%s is not device memory", name);
    if (at.type == cudaMemoryTypeDevice && at.device != device)
        return fail(CWO_ERR_INVALID_ARG, "%s lives on device %d, the plan on device %d", name, at.device, device);
    if (PFN_memGetAddressRange fn = get_addr_range_fn()) {
        CUdeviceptr base = 0;
        size_t size = 0;
        if (fn(&base, &size, (CUdeviceptr)(uintptr_t)ptr) == CUDA_SUCCESS) {
            if ((uintptr_t)ptr + bytes > (uintptr_t)base + size)
                return fail(CWO_ERR_INVALID_ARG, "%s: %zu bytes requested but its allocation ends %zu bytes after it",
                            name, bytes, (size_t)((uintptr_t)base + size - (uintptr_t)ptr));
        }
    }
    return CWO_OK;
}

template <typename T>
cwo_status dev_alloc(T** p, size_t count, const char* what) {
    *p = nullptr;
    if (count == 0) return CWO_OK;
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(CWO_ERR_OOM, "cudaMalloc of %zu bytes for %s failed: %s", count * sizeof(T), what, cudaGetErrorName(e));
    }
    return CWO_OK;
}

template <typename T>
cwo_status upload(T* dst, const std::vector<T>& src, const char* what) {
    if (src.empty()) return CWO_OK;
    cudaError_t e = cudaMemcpy(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
    return e == cudaSuccess ? CWO_OK : cuda_fail(e, what);
}

size_t tables_bytes(int nx, int ny) {
    const AxisGeo gx(2 * nx), gy(2 * ny);
    size_t b = 0;
    b += (size_t)(gx.tw_off(gx.NST - 1) + gy.tw_off(gy.NST - 1)) * sizeof(float4);
    b += (size_t)(gx.P + gy.P) * sizeof(int);
    b += (size_t)(gx.P + gy.P) * sizeof(float4) + sizeof(float) * 2;
    return b;
}

}  // namespace

void cwo::set_last_error(const char* msg) { g_err = msg ? msg : ""; }

int cwo::check_device_buffer(const void* ptr, size_t bytes, int device, const char* name) {
    return check_device_range(ptr, bytes, device, name);
}

// ------------------------------------------------------------------------------------------
// plan
// ------------------------------------------------------------------------------------------
// Pinned host staging for per-call tables, K buffers in rotation: a call waits (on the host) only
// for the upload that used its buffer K calls earlier, so preparing the next call's tables
// overlaps the GPU work of the previous ones instead of waiting for it.
struct StagingRing {
    static constexpr int K = 4;
    void* buf[K] = {};
    cudaEvent_t ev[K] = {};
    bool pending[K] = {};
    size_t bytes = 0;
    int next = 0;
    void release() {
        for (int k = 0; k < K; ++k) {
            if (buf[k]) cudaFreeHost(buf[k]);
            if (ev[k]) cudaEventDestroy(ev[k]);
            buf[k] = nullptr; ev[k] = nullptr; pending[k] = false;
        }
        bytes = 0;
        next = 0;
    }
};

struct cwo_plan {
    int nx = 0, ny = 0, px = 0, py = 0;
    double dx = 0, dy = 0, lambda = 0, z = 0;
    cwo_type type = CWO_ANGULAR;
    unsigned flags = 0;
    int device = 0;
    float4* tw_x = nullptr;   // twiddles along x (rows, length px)
    float4* tw_y = nullptr;   // twiddles along y (columns, length py); aliases tw_x if px == py
    int* kb_x = nullptr;
    int* kb_y = nullptr;
    int2* pairs_x = nullptr;   // mirror storage-column pairs along x
    // tables of the plan's own z
    float4* ax = nullptr; float4* ay = nullptr;
    float2* hx = nullptr; float2* hy = nullptr;
    float* kf = nullptr;
    // per-call (per-item z) tables
    int zcap = 0;
    float4* zax = nullptr; float4* zay = nullptr;
    float2* zhx = nullptr; float2* zhy = nullptr;
    float* zkf = nullptr;
    StagingRing zstage;   // pinned staging of the per-item z tables
    std::vector<double> zs_cached;   // distances whose tables the per-item buffers hold
    // mixed-batch (cwo_propagate_items) per-item tables and parameters
    int icap = 0;
    float4* ix = nullptr; float4* iy = nullptr; cwo::ItemParams* iprm = nullptr;
    StagingRing istage;   // pinned staging of the mixed-batch tables
    // scratch intermediate [cap][ny][px]
    float2* scratch = nullptr;
    int scap = 0;
    // optional per-pass timing events (caller-owned)
    cudaEvent_t tev[4] = {nullptr, nullptr, nullptr, nullptr};
    CUtensorMap wmap_f;        // TMA maps of the scratch intermediate [scap][px][ny] for the
    CUtensorMap wmap_i;        // forward and inverse row passes (different box heights)
    CUtensorMap wmap_s;        // Fresnel convolution form: the [scap][nx][ny] intermediate of its
                               // separable line passes
    int* status = nullptr;     // device status word: bounded waits that expired (cwo_plan_check)
    // shifted angular spectrum (CWO_SHIFTED_ANGULAR): shift and Rect windows (Eq. shift_ang1)
    bool shifted = false;
    cwo_shift shift{};
    // Fresnel Fourier form (CWO_FRESNEL_FOURIER): chirps, centring factors, output placement;
    // shifted Fresnel (CWO_SHIFTED_FRESNEL): source factors f (fpre), destination factors q
    // (fpost) and their conjugates for the adjoint (fpre_c = conj q, fpost_c = conj f)
    float2* fpre_x = nullptr; float2* fpre_y = nullptr;
    float2* fpost_x = nullptr; float2* fpost_y = nullptr;
    float2* fpre_cx = nullptr; float2* fpre_cy = nullptr;
    float2* fpost_cx = nullptr; float2* fpost_cy = nullptr;
    int* fst_x = nullptr; int* frow_y = nullptr;
    cwo_shifted_fresnel sfr{};
    // CWO_FLAG_CACHE_H: the ASM transfer function of the plan's own z, [Px/2 + 1 pairs][Py]
    float2* hcache = nullptr;
    // with it at Py = 8192 (split column pass): the 4096-point twiddles, then W_8192^n (float2)
    float4* split_tw = nullptr;
    float2* split_w = nullptr;
};

namespace {

void free_plan(cwo_plan* p) {
    if (!p) return;
    cudaFree(p->tw_x);
    if (p->tw_y != p->tw_x) cudaFree(p->tw_y);
    cudaFree(p->kb_x); cudaFree(p->kb_y); cudaFree(p->pairs_x);
    cudaFree(p->ax); cudaFree(p->ay); cudaFree(p->hx); cudaFree(p->hy); cudaFree(p->kf);
    cudaFree(p->zax); cudaFree(p->zay); cudaFree(p->zhx); cudaFree(p->zhy); cudaFree(p->zkf);
    p->zstage.release();
    cudaFree(p->scratch);
    cudaFree(p->status);
    cudaFree(p->ix); cudaFree(p->iy); cudaFree(p->iprm);
    p->istage.release();
    cudaFree(p->fpre_x); cudaFree(p->fpre_y); cudaFree(p->fpost_x); cudaFree(p->fpost_y);
    cudaFree(p->fst_x); cudaFree(p->frow_y);
    cudaFree(p->fpre_cx); cudaFree(p->fpre_cy); cudaFree(p->fpost_cx); cudaFree(p->fpost_cy);
    cudaFree(p->hcache);
    cudaFree(p->split_tw);
    delete p;
}

cwo_status check_params(int nx, int ny, double dx, double dy, double lambda, double z, int type, unsigned flags) {
    if (!pow2_side(nx) || !pow2_side(ny))
        return fail(CWO_ERR_INVALID_ARG, "Nx=%d, Ny=%d: each side must be a power of two in [%d, %d]", nx, ny, CWO_MIN_SIDE, CWO_MAX_SIDE);
    if (!(dx > 0) || !(dy > 0) || !std::isfinite(dx) || !std::isfinite(dy))
        return fail(CWO_ERR_INVALID_ARG, "pitches must be finite and > 0 (dx=%g, dy=%g)", dx, dy);
    if (!(lambda > 0) || !std::isfinite(lambda)) return fail(CWO_ERR_INVALID_ARG, "wavelength must be finite and > 0 (%g)", lambda);
    if (!std::isfinite(z)) return fail(CWO_ERR_INVALID_ARG, "distance must be finite (%g)", z);
    if (type == CWO_SHIFTED_FRESNEL || type == CWO_SHIFTED_ANGULAR)
        return fail(CWO_ERR_UNSUPPORTED, "diffraction type %d is not provided by cwo_plan_create", type);
    if (type != CWO_ANGULAR && type != CWO_FRESNEL_CONV && type != CWO_FRESNEL_FOURIER)
        return fail(CWO_ERR_INVALID_ARG, "unknown diffraction type %d", type);
    if ((type == CWO_FRESNEL_CONV || type == CWO_FRESNEL_FOURIER) && z == 0.0)
        return fail(CWO_ERR_INVALID_ARG, "Fresnel diffraction needs z != 0");
    if (type == CWO_FRESNEL_FOURIER && (nx < 32 || ny < 32))
        return fail(CWO_ERR_INVALID_ARG, "the Fourier form transforms unpadded axes of at least 32 samples (Nx=%d, Ny=%d)", nx, ny);
    const unsigned known = CWO_FLAG_PHASE_FP32 | CWO_FLAG_PHASE_FP64 | CWO_FLAG_LITERAL_SCALE | CWO_FLAG_CACHE_H;
    if ((flags & CWO_FLAG_CACHE_H) && type != CWO_ANGULAR)
        return fail(CWO_ERR_INVALID_ARG, "CWO_FLAG_CACHE_H applies to CWO_ANGULAR plans only");
    if (flags & ~known) return fail(CWO_ERR_INVALID_ARG, "unknown flag bits 0x%x", flags & ~known);
    if ((flags & CWO_FLAG_PHASE_FP32) && (flags & CWO_FLAG_PHASE_FP64))
        return fail(CWO_ERR_INVALID_ARG, "CWO_FLAG_PHASE_FP32 and CWO_FLAG_PHASE_FP64 are exclusive");
    if ((flags & (CWO_FLAG_PHASE_FP32 | CWO_FLAG_PHASE_FP64)) && type != CWO_ANGULAR)
        return fail(CWO_ERR_INVALID_ARG, "phase-precision flags apply to CWO_ANGULAR only");
    if ((flags & CWO_FLAG_LITERAL_SCALE) && type != CWO_FRESNEL_CONV && type != CWO_FRESNEL_FOURIER)
        return fail(CWO_ERR_INVALID_ARG, "CWO_FLAG_LITERAL_SCALE applies to the Fresnel types only");
    return CWO_OK;
}

// host tables of one parameter set
void host_h_tables(const cwo_plan* p, double z, float4* ax, float4* ay, float2* hx, float2* hy, float* kf) {
    if (p->shifted) {
        asm_axis_table_shifted(AxisGeo(p->px), p->dx, p->lambda, z, true, p->shift.ox, p->shift.cx, p->shift.wx, ax);
        asm_axis_table_shifted(AxisGeo(p->py), p->dy, p->lambda, z, false, p->shift.oy, p->shift.cy, p->shift.wy, ay);
        if (kf) *kf = (float)(z / p->lambda);
        return;
    }
    make_h_tables(p->px, p->py, p->dx, p->dy, p->lambda, z, p->type == CWO_FRESNEL_CONV,
                  (p->flags & CWO_FLAG_LITERAL_SCALE) != 0, ax, ay, hx, hy, kf);
}

cwo_status ensure_scratch(cwo_plan* p, int items) {
    if (items <= p->scap) return CWO_OK;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize before growing scratch");
    cudaFree(p->scratch);
    p->scratch = nullptr;
    p->scap = 0;
    cwo_status st = dev_alloc(&p->scratch, (size_t)items * p->ny * p->px, "scratch");
    if (st != CWO_OK) return st;
    // wmap_s for every type: the mixed batches of any plan run their Fresnel items as line passes
    if ((e = cwo::make_intermediate_map(&p->wmap_f, p->scratch, p->ny, p->px, items, cwo::row_block_rows(p->px, false))) ||
        (e = cwo::make_intermediate_map(&p->wmap_i, p->scratch, p->ny, p->px, items, cwo::row_block_rows(p->px, true))) ||
        (p->type != CWO_FRESNEL_FOURIER &&
         (e = cwo::make_intermediate_map(&p->wmap_s, p->scratch, p->ny, p->nx, items, cwo::line_block_rows(p->px)))))
        return cuda_fail(e, "tensor map of the intermediate");
    p->scap = items;
    return CWO_OK;
}

cwo_status staging_alloc(StagingRing& r, size_t bytes) {
    r.release();
    for (int k = 0; k < StagingRing::K; ++k) {
        cudaError_t e = cudaMallocHost(&r.buf[k], bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            r.buf[k] = nullptr;
            r.release();
            return fail(CWO_ERR_OOM, "pinned staging of %zu bytes failed", bytes);
        }
        if ((e = cudaEventCreateWithFlags(&r.ev[k], cudaEventDisableTiming)) != cudaSuccess) {
            r.release();
            return cuda_fail(e, "cudaEventCreate");
        }
    }
    r.bytes = bytes;
    return CWO_OK;
}

// the next staging buffer, once the upload that last used it has been consumed
cwo_status staging_acquire(StagingRing& r, char** buf, int* slot) {
    const int k = r.next;
    if (r.pending[k]) {
        cudaError_t e = cudaEventSynchronize(r.ev[k]);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
        r.pending[k] = false;
    }
    *buf = (char*)r.buf[k];
    *slot = k;
    r.next = (k + 1) % StagingRing::K;
    return CWO_OK;
}

cwo_status staging_release_after(StagingRing& r, int slot, cudaStream_t s) {
    cudaError_t e = cudaEventRecord(r.ev[slot], s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    r.pending[slot] = true;
    return CWO_OK;
}

cwo_status ensure_ztables(cwo_plan* p, int items) {
    if (items <= p->zcap) return CWO_OK;
    p->zs_cached.clear();
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize before growing tables");
    cudaFree(p->zax); cudaFree(p->zay); cudaFree(p->zhx); cudaFree(p->zhy); cudaFree(p->zkf);
    p->zax = p->zay = nullptr; p->zhx = p->zhy = nullptr; p->zkf = nullptr;
    p->zstage.release();
    p->zcap = 0;
    cwo_status st;
    size_t zbytes = 0;
    const size_t nx4 = (size_t)items * p->px, ny4 = (size_t)items * p->py;
    if (p->type == CWO_ANGULAR) {
        if ((st = dev_alloc(&p->zax, nx4, "per-item x tables")) || (st = dev_alloc(&p->zay, ny4, "per-item y tables")) ||
            (st = dev_alloc(&p->zkf, (size_t)items, "per-item K")))
            return st;
        zbytes = (nx4 + ny4) * sizeof(float4) + items * sizeof(float);
    } else {
        if ((st = dev_alloc(&p->zhx, nx4, "per-item x tables")) || (st = dev_alloc(&p->zhy, ny4, "per-item y tables")))
            return st;
        zbytes = (nx4 + ny4) * sizeof(float2);
    }
    if ((st = staging_alloc(p->zstage, zbytes))) return st;
    p->zcap = items;
    return CWO_OK;
}

cwo_status check_plan_device(const cwo_plan* p) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != p->device) return fail(CWO_ERR_INVALID_ARG, "current device %d differs from the plan's device %d", dev, p->device);
    return CWO_OK;
}

// launch parameters of the transfer function with the plan's own tables: geometry, the shifted
// ASM's shift and windows, and the evaluation mode (for the distances zs, or the plan's z)
cwo::HParams base_hparams(const cwo_plan* p, const double* zs, int batch) {
    cwo::HParams hp{};
    hp.kbx = p->kb_x;
    hp.kby = p->kb_y;
    hp.pairs = p->pairs_x;
    hp.npairs = p->px / 2 + 1;
    hp.K = p->z / p->lambda;
    hp.sx = p->lambda * p->lambda / ((double)p->px * p->dx * (double)p->px * p->dx);
    hp.sy = p->lambda * p->lambda / ((double)p->py * p->dy * (double)p->py * p->dy);
    hp.z = p->z;
    hp.k = 2.0 * kPi / p->lambda;
    hp.dfx = 1.0 / ((double)p->px * p->dx);
    hp.dfy = 1.0 / ((double)p->py * p->dy);
    if (p->shifted) {
        hp.asym = 1;
        hp.shx = p->shift.ox * hp.dfx;
        hp.shy = p->shift.oy * hp.dfy;
        window_bins(AxisGeo(p->px), p->dx, p->shift.cx, p->shift.wx, &hp.wxlo, &hp.wxhi);
        window_bins(AxisGeo(p->py), p->dy, p->shift.cy, p->shift.wy, &hp.wylo, &hp.wyhi);
    }
    if (p->type == CWO_FRESNEL_CONV || p->type == CWO_SHIFTED_FRESNEL) hp.mode = cwo::HMODE_FRESNEL;
    else if (p->flags & CWO_FLAG_PHASE_FP32) hp.mode = cwo::HMODE_ASM_FP32;
    else if (p->flags & CWO_FLAG_PHASE_FP64) hp.mode = cwo::HMODE_ASM_FP64;
    else {
        // the cheapest per-element remainder evaluation that stays within its error budget
        int tm = 0;
        if (zs) for (int i = 0; i < batch; ++i) tm = std::max(tm, asm_tail_mode(p->px, p->py, p->dx, p->dy, p->lambda, zs[i]));
        else tm = asm_tail_mode(p->px, p->py, p->dx, p->dy, p->lambda, p->z);
        hp.mode = tm == 0 ? cwo::HMODE_ASM_POLY : tm == 1 ? cwo::HMODE_ASM_EXACT : cwo::HMODE_ASM_FP64;
    }
    hp.ax = p->ax; hp.ay = p->ay; hp.kf = p->kf; hp.hx = p->hx; hp.hy = p->hy;
    return hp;
}

// prevalidated: the caller (one API call that propagates the same buffers repeatedly) has
// already checked these buffers with this plan
cwo_status run(cwo_plan* p, const void* in, long long in_stride, void* out, int batch,
               const double* zs, void* stream, bool adjoint, const cwo::Epilogue& epi = cwo::Epilogue(),
               bool prevalidated = false) {
    if (!p) return fail(CWO_ERR_INVALID_ARG, "plan is NULL");
    if (batch < 1 || batch > 65535) return fail(CWO_ERR_INVALID_ARG, "batch must be in [1, 65535] (got %d)", batch);
    const long long field = (long long)p->nx * p->ny;
    if (in_stride < 0) return fail(CWO_ERR_INVALID_ARG, "negative input batch stride");
    if (in_stride != 0 && in_stride < field) return fail(CWO_ERR_INVALID_ARG, "input batch stride %lld smaller than one field (%lld)", in_stride, field);
    if (adjoint && in_stride == 0 && batch > 1) return fail(CWO_ERR_INVALID_ARG, "the adjoint takes one input per item (stride > 0)");
    const bool stack = in_stride == 0 && batch > 1;
    if (zs && p->shifted)
        return fail(CWO_ERR_UNSUPPORTED, "per-item distances are not provided for a shifted angular-spectrum plan");
    if (zs) {
        if (p->flags & (CWO_FLAG_PHASE_FP32 | CWO_FLAG_PHASE_FP64))
            return fail(CWO_ERR_UNSUPPORTED, "per-item distances are not provided with the phase-precision study flags");
        for (int i = 0; i < batch; ++i) {
            if (!std::isfinite(zs[i])) return fail(CWO_ERR_INVALID_ARG, "z[%d] is not finite", i);
            if (p->type == CWO_FRESNEL_CONV && zs[i] == 0.0) return fail(CWO_ERR_INVALID_ARG, "z[%d] = 0 with Fresnel", i);
        }
    }
    if (p->type == CWO_SHIFTED_FRESNEL) {
        if (zs) return fail(CWO_ERR_UNSUPPORTED, "per-item distances are not provided for shifted Fresnel plans");
        if (epi.mode != cwo::EPI_NONE) return fail(CWO_ERR_UNSUPPORTED, "output epilogues are not provided for shifted Fresnel plans");
    }
    if (p->type == CWO_FRESNEL_FOURIER) {
        if (adjoint) return fail(CWO_ERR_UNSUPPORTED, "the adjoint is not provided for the Fourier form");
        if (zs) return fail(CWO_ERR_UNSUPPORTED, "per-item distances are not provided for the Fourier form");
        if (stack) return fail(CWO_ERR_UNSUPPORTED, "the shared-source stack is not provided for the Fourier form");
        if (epi.mode != cwo::EPI_NONE) return fail(CWO_ERR_UNSUPPORTED, "output epilogues are not provided for the Fourier form");
    }
    cwo_status st = prevalidated ? CWO_OK : check_plan_device(p);
    if (st) return st;
    const size_t fb = (size_t)field * sizeof(float2);
    const size_t in_bytes = stack ? fb : (size_t)((batch - 1) * (in_stride ? in_stride : field)) * sizeof(float2) + fb;
    if (!prevalidated) {
    if ((st = check_device_range(in, in_bytes, p->device, "input"))) return st;
    if (epi.mode != cwo::EPI_INTENSITY && (st = check_device_range(out, (size_t)batch * fb, p->device, "output"))) return st;
    if (epi.mode != cwo::EPI_NONE) {
        if (stack) return fail(CWO_ERR_INVALID_ARG, "output epilogues take one input per item (stride > 0)");
        const size_t rb = (size_t)batch * field * sizeof(float);
        if (epi.mode == cwo::EPI_AMPLITUDE && (st = check_device_range(epi.amp, rb, p->device, "amplitude"))) return st;
        if (epi.mode == cwo::EPI_INTENSITY && (st = check_device_range(epi.inten, rb, p->device, "intensity"))) return st;
    }
    }
    const int need = stack ? batch + 1 : batch;
    if ((st = ensure_scratch(p, need))) return st;

    cudaStream_t s = (cudaStream_t)stream;
    if (p->type == CWO_FRESNEL_FOURIER) {
        const bool timing = p->tev[0] != nullptr;
        auto mark = [&](int i) { return timing ? cudaEventRecord(p->tev[i], s) : cudaSuccess; };
        const long long wstride = (long long)p->ny * p->px;
        cudaError_t e;
        if ((e = mark(0)) ||
            (e = cwo::launch_fourier_rows(p->px, (const float2*)in, in_stride, &p->wmap_f, p->ny, batch, p->fpre_x,
                                          p->fpre_y, p->tw_x, s)) ||
            (e = mark(1)))
            return cuda_fail(e, "Fourier-form row launch");
        if ((e = cwo::launch_fourier_cols(p->py, p->scratch, wstride, (float2*)out, field, p->nx, batch, p->fst_x, p->frow_y,
                                          p->fpost_x, p->fpost_y, p->tw_y, s)) ||
            (e = mark(2)) || (e = mark(3)))
            return cuda_fail(e, "Fourier-form column launch");
        return CWO_OK;
    }
    cwo::HParams hp = base_hparams(p, zs, batch);
    hp.conj = adjoint ? 1 : 0;
    // FP64 per element with per-item distances: one launch set per item, each with its own K
    const bool per_item_k = zs && hp.mode == cwo::HMODE_ASM_FP64;

    // per-item tables of the same distances as the previous call are reused ("once-calculation")
    const bool ztables_hit = zs && !per_item_k && (int)p->zs_cached.size() == batch &&
                             std::equal(p->zs_cached.begin(), p->zs_cached.end(), zs);
    if (zs && !per_item_k && ztables_hit) {
        if (p->type == CWO_ANGULAR) {
            hp.ax = p->zax; hp.ay = p->zay; hp.kf = p->zkf;
            hp.x_item_stride = p->px; hp.y_item_stride = p->py; hp.kf_item_stride = 1;
        } else {
            hp.hx = p->zhx; hp.hy = p->zhy;
            hp.x_item_stride = p->px; hp.y_item_stride = p->py;
        }
    } else if (zs && !per_item_k) {
        p->zs_cached.clear();
        if ((st = ensure_ztables(p, batch))) return st;
        char* hb = nullptr;
        int zslot = 0;
        if ((st = staging_acquire(p->zstage, &hb, &zslot))) return st;
        if (p->type == CWO_ANGULAR) {
            float4* hax = (float4*)hb;
            float4* hay = hax + (size_t)batch * p->px;
            float* hkf = (float*)(hay + (size_t)batch * p->py);
            for (int i = 0; i < batch; ++i)
                host_h_tables(p, zs[i], hax + (size_t)i * p->px, hay + (size_t)i * p->py, nullptr, nullptr, hkf + i);
            cudaError_t e;
            if ((e = cudaMemcpyAsync(p->zax, hax, (size_t)batch * p->px * sizeof(float4), cudaMemcpyHostToDevice, s)) ||
                (e = cudaMemcpyAsync(p->zay, hay, (size_t)batch * p->py * sizeof(float4), cudaMemcpyHostToDevice, s)) ||
                (e = cudaMemcpyAsync(p->zkf, hkf, (size_t)batch * sizeof(float), cudaMemcpyHostToDevice, s)))
                return cuda_fail(e, "table upload");
            hp.ax = p->zax; hp.ay = p->zay; hp.kf = p->zkf;
            hp.x_item_stride = p->px; hp.y_item_stride = p->py; hp.kf_item_stride = 1;
        } else {
            float2* hhx = (float2*)hb;
            float2* hhy = hhx + (size_t)batch * p->px;
            for (int i = 0; i < batch; ++i)
                host_h_tables(p, zs[i], nullptr, nullptr, hhx + (size_t)i * p->px, hhy + (size_t)i * p->py, nullptr);
            cudaError_t e;
            if ((e = cudaMemcpyAsync(p->zhx, hhx, (size_t)batch * p->px * sizeof(float2), cudaMemcpyHostToDevice, s)) ||
                (e = cudaMemcpyAsync(p->zhy, hhy, (size_t)batch * p->py * sizeof(float2), cudaMemcpyHostToDevice, s)))
                return cuda_fail(e, "table upload");
            hp.hx = p->zhx; hp.hy = p->zhy;
            hp.x_item_stride = p->px; hp.y_item_stride = p->py;
        }
        if ((st = staging_release_after(p->zstage, zslot, s))) return st;
        p->zs_cached.assign(zs, zs + batch);
    } else {
        hp.ax = p->ax; hp.ay = p->ay; hp.kf = p->kf; hp.hx = p->hx; hp.hy = p->hy;
        hp.x_item_stride = 0; hp.y_item_stride = 0; hp.kf_item_stride = 0;
        if (p->hcache) {   // the plan's own z with the transfer function materialised
            hp.mode = cwo::HMODE_TABLE;
            hp.hcache = p->hcache;
            hp.hcache_stride = p->py;
            hp.split_tw = p->split_tw;
            hp.split_w = p->split_w;
        }
    }

    const long long wstride = (long long)p->ny * p->px;
    const bool timing = p->tev[0] != nullptr;
    auto mark = [&](int i) { return timing ? cudaEventRecord(p->tev[i], s) : cudaSuccess; };
    cwo::Prefactor pre;
    cwo::Epilogue ep = epi;
    if (p->type == CWO_SHIFTED_FRESNEL) {   // A = diag(q) conv diag(f);  A^H = diag(f*) conv^H diag(q*)
        pre.fx = adjoint ? p->fpre_cx : p->fpre_x;
        pre.fy = adjoint ? p->fpre_cy : p->fpre_y;
        ep.mode = cwo::EPI_SEPARABLE;
        ep.qx = adjoint ? p->fpost_cx : p->fpost_x;
        ep.qy = adjoint ? p->fpost_cy : p->fpost_y;
    }
    const float2* fin = (const float2*)in;
    float2* fout = (float2*)out;
    cudaError_t e;
    const float scale = (float)(1.0 / ((double)p->px * (double)p->py));
    if (p->type == CWO_FRESNEL_CONV && stack && epi.mode == cwo::EPI_NONE && (uintptr_t)out % 16 == 0 &&
        (uintptr_t)in % 16 == 0 && cwo::line_stack_supported(p->px)) {
        // shared-source stack in the separable form: every source row transformed once and
        // convolved per plane into that plane's intermediate, then every plane's columns
        CUtensorMap omap;
        if ((e = cwo::make_intermediate_map(&omap, out, p->nx, p->ny, batch, cwo::line_block_rows(p->py))))
            return cuda_fail(e, "tensor map of the output");
        if ((e = mark(0)) ||
            (e = cwo::launch_line_stack(p->px, fin, &p->wmap_s, p->ny, batch, hp.hx, hp.x_item_stride, hp.conj,
                                        (float)(1.0 / p->px), p->tw_x, p->status, s)) ||
            (e = mark(1)) ||
            (e = cwo::launch_line_conv(p->py, p->scratch, field, &omap, p->nx, batch, hp.hy, hp.y_item_stride, hp.conj,
                                       (float)(1.0 / p->py), p->tw_y, p->status, nullptr, nullptr, s)) ||
            (e = mark(2)) || (e = mark(3)))
            return cuda_fail(e, "separable Fresnel stack launch");
        return CWO_OK;
    }
    const bool separable = p->type == CWO_FRESNEL_CONV || p->type == CWO_SHIFTED_FRESNEL;
    if (separable && !stack && epi.mode == cwo::EPI_NONE && (uintptr_t)out % 16 == 0) {
        // separable form: a padded line convolution along x into the column-major Nx x Ny
        // intermediate, then one along y into the output (cwo_lines.cu); the shifted form
        // multiplies each pass's input by the source factor and its output by the destination
        // factor of its axis
        const bool sf = p->type == CWO_SHIFTED_FRESNEL;
        const float2* prex = sf ? pre.fx : nullptr;
        const float2* prey = sf ? pre.fy : nullptr;
        const float2* postx = sf ? ep.qx : nullptr;
        const float2* posty = sf ? ep.qy : nullptr;
        CUtensorMap omap;
        if ((e = cwo::make_intermediate_map(&omap, out, p->nx, p->ny, batch, cwo::line_block_rows(p->py))))
            return cuda_fail(e, "tensor map of the output");
        const long long istr = in_stride ? in_stride : field;
        if ((e = mark(0)) ||
            (e = cwo::launch_line_conv(p->px, fin, istr, &p->wmap_s, p->ny, batch, hp.hx, hp.x_item_stride, hp.conj,
                                       (float)(1.0 / p->px), p->tw_x, p->status, prex, postx, s)) ||
            (e = mark(1)) ||
            (e = cwo::launch_line_conv(p->py, p->scratch, field, &omap, p->nx, batch, hp.hy, hp.y_item_stride, hp.conj,
                                       (float)(1.0 / p->py), p->tw_y, p->status, prey, posty, s)) ||
            (e = mark(2)) || (e = mark(3)))
            return cuda_fail(e, "separable Fresnel launch");
        return CWO_OK;
    }
    if (stack) {
        // the shared source: row pass once, then per-plane column and inverse row passes
        float2* w0 = p->scratch;
        float2* wz = p->scratch + wstride;
        if ((e = mark(0)) || (e = cwo::launch_row_fwd(p->px, fin, 0, &p->wmap_f, 0, p->ny, 1, p->tw_x, p->status, s, pre)) || (e = mark(1)))
            return cuda_fail(e, "row forward launch");
        if (per_item_k) {
            for (int i = 0; i < batch; ++i) {
                hp.K = zs[i] / p->lambda;
                if ((e = cwo::launch_col(p->py, w0, 0, wz + i * wstride, 0, p->px, 1, p->tw_y, hp, s)))
                    return cuda_fail(e, "column launch");
            }
            if ((e = mark(2))) return cuda_fail(e, "event");
        } else if ((e = cwo::launch_col_stack(p->py, w0, wz, wstride, p->px, batch, p->tw_y, hp, s)) || (e = mark(2))) {
            return cuda_fail(e, "column launch");
        }
        if ((e = cwo::launch_row_inv(p->px, &p->wmap_i, 1, fout, field, p->ny, batch, scale, p->tw_x, p->status, s, ep)) || (e = mark(3)))
            return cuda_fail(e, "row inverse launch");
    } else {
        const long long istr = in_stride ? in_stride : field;
        if ((e = mark(0)) || (e = cwo::launch_row_fwd(p->px, fin, istr, &p->wmap_f, 0, p->ny, batch, p->tw_x, p->status, s, pre)) || (e = mark(1)))
            return cuda_fail(e, "row forward launch");
        if (per_item_k) {
            for (int i = 0; i < batch; ++i) {
                hp.K = zs[i] / p->lambda;
                float2* wi = p->scratch + i * wstride;
                if ((e = cwo::launch_col(p->py, wi, 0, wi, 0, p->px, 1, p->tw_y, hp, s)))
                    return cuda_fail(e, "column launch");
            }
            if ((e = mark(2))) return cuda_fail(e, "event");
        } else if ((e = cwo::launch_col(p->py, p->scratch, wstride, p->scratch, wstride, p->px, batch, p->tw_y, hp, s)) || (e = mark(2))) {
            return cuda_fail(e, "column launch");
        }
        if ((e = cwo::launch_row_inv(p->px, &p->wmap_i, 0, fout, field, p->ny, batch, scale, p->tw_x, p->status, s, ep)) ||
            (e = mark(3)))
            return cuda_fail(e, "row inverse launch");
    }
    return CWO_OK;
}

cwo_status ensure_itables(cwo_plan* p, int items) {
    if (items <= p->icap) return CWO_OK;
    items = std::max(items, std::min(2 * p->icap, 65535));   // grow geometrically: few reallocations
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize before growing item tables");
    cudaFree(p->ix); cudaFree(p->iy); cudaFree(p->iprm);
    p->ix = p->iy = nullptr; p->iprm = nullptr;
    p->istage.release();
    p->icap = 0;
    cwo_status st;
    const size_t nx4 = (size_t)items * p->px, ny4 = (size_t)items * p->py;
    if ((st = dev_alloc(&p->ix, nx4, "item x tables")) || (st = dev_alloc(&p->iy, ny4, "item y tables")) ||
        (st = dev_alloc(&p->iprm, (size_t)items, "item parameters")))
        return st;
    if ((st = staging_alloc(p->istage, (nx4 + ny4) * sizeof(float4) + (size_t)items * sizeof(cwo::ItemParams)))) return st;
    p->icap = items;
    return CWO_OK;
}

// the tables and scalars of one item of a mixed batch.  lines: a Fresnel item that takes the two
// separable line passes, whose tables are stored as P complex64 values at the start of the item's
// rows (the line pass's layout); otherwise float4 rows (the column pass's layout).
void item_tables(const cwo_plan* p, const cwo_item& it, float4* xt, float4* yt, cwo::ItemParams* prm, bool lines) {
    const AxisGeo gx(p->px), gy(p->py);
    if (it.type == CWO_ANGULAR) {
        asm_axis_table(gx, it.dx, it.lambda, it.z, true, xt);
        asm_axis_table(gy, it.dy, it.lambda, it.z, false, yt);
        const int tm = asm_tail_mode(p->px, p->py, it.dx, it.dy, it.lambda, it.z);
        prm->mode = tm == 0 ? cwo::HMODE_ASM_POLY : tm == 1 ? cwo::HMODE_ASM_EXACT : cwo::HMODE_ASM_FP64;
    } else {
        std::vector<float2> hx(p->px), hy(p->py);
        make_h_tables(p->px, p->py, it.dx, it.dy, it.lambda, it.z, true, (it.flags & CWO_FLAG_LITERAL_SCALE) != 0,
                      nullptr, nullptr, hx.data(), hy.data(), nullptr);
        if (lines) {
            std::copy(hx.begin(), hx.end(), (float2*)xt);
            std::copy(hy.begin(), hy.end(), (float2*)yt);
        } else {
            for (int i = 0; i < p->px; ++i) xt[i] = make_float4(hx[i].x, hx[i].y, 0.f, 0.f);
            for (int i = 0; i < p->py; ++i) yt[i] = make_float4(hy[i].x, hy[i].y, 0.f, 0.f);
        }
        prm->mode = cwo::HMODE_FRESNEL;
    }
    prm->kf = (float)(it.z / it.lambda);
    prm->K = it.z / it.lambda;
    prm->sx = it.lambda * it.lambda / ((double)p->px * it.dx * (double)p->px * it.dx);
    prm->sy = it.lambda * it.lambda / ((double)p->py * it.dy * (double)p->py * it.dy);
}

cwo_status run_items(cwo_plan* p, const void* in, long long in_stride, void* out, int batch, const cwo_item* items,
                     void* stream) {
    if (!p) return fail(CWO_ERR_INVALID_ARG, "plan is NULL");
    if (!items) return fail(CWO_ERR_INVALID_ARG, "items is NULL");
    if (batch < 1 || batch > 65535) return fail(CWO_ERR_INVALID_ARG, "batch must be in [1, 65535] (got %d)", batch);
    const long long field = (long long)p->nx * p->ny;
    if (in_stride < field) return fail(CWO_ERR_INVALID_ARG, "input batch stride %lld smaller than one field (%lld)", in_stride, field);
    for (int i = 0; i < batch; ++i) {
        const cwo_item& it = items[i];
        cwo_status st = check_params(p->nx, p->ny, it.dx, it.dy, it.lambda, it.z, it.type, it.flags);
        if (st) return fail(st, "item %d: %s", i, g_err.c_str());
        if (it.flags & (CWO_FLAG_PHASE_FP32 | CWO_FLAG_PHASE_FP64))
            return fail(CWO_ERR_UNSUPPORTED, "item %d: phase-precision study flags are not provided in mixed batches", i);
    }
    cwo_status st = check_plan_device(p);
    if (st) return st;
    const size_t fb = (size_t)field * sizeof(float2);
    if ((st = check_device_range(in, (size_t)(batch - 1) * in_stride * sizeof(float2) + fb, p->device, "input"))) return st;
    if ((st = check_device_range(out, (size_t)batch * fb, p->device, "output"))) return st;
    if ((st = ensure_scratch(p, batch)) || (st = ensure_itables(p, batch))) return st;
    char* hb = nullptr;
    int islot = 0;
    if ((st = staging_acquire(p->istage, &hb, &islot))) return st;
    float4* hx = (float4*)hb;
    float4* hy = hx + (size_t)batch * p->px;
    cwo::ItemParams* hp_items = (cwo::ItemParams*)(hy + (size_t)batch * p->py);
    // per-item FP64 tables, items spread over host threads when there is enough work
    const size_t work = (size_t)batch * (p->px + p->py);
    const int nthreads = (int)std::min<size_t>((size_t)std::max(1u, std::thread::hardware_concurrency()),
                                               std::min<size_t>((size_t)batch, work / 8192 + 1));
    // Route: a Fresnel convolution item takes the two separable line passes (32 N^2 bytes, as a
    // Fresnel plan does) where the output allows their TMA stores, every other item the three
    // passes; each contiguous run of one route is one sub-batch.  An item's result therefore does
    // not depend on the other items of the batch.
    const bool lines_ok = (uintptr_t)out % 16 == 0;
    auto lines = [&](int i) { return lines_ok && items[i].type == CWO_FRESNEL_CONV; };
    auto worker = [&](int w) {
        for (int i = w; i < batch; i += nthreads)
            item_tables(p, items[i], hx + (size_t)i * p->px, hy + (size_t)i * p->py, hp_items + i, lines(i));
    };
    if (nthreads <= 1) {
        worker(0);
    } else {
        std::vector<std::thread> pool;
        for (int w = 1; w < nthreads; ++w) pool.emplace_back(worker, w);
        worker(0);
        for (auto& th : pool) th.join();
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(p->ix, hx, (size_t)batch * p->px * sizeof(float4), cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(p->iy, hy, (size_t)batch * p->py * sizeof(float4), cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(p->iprm, hp_items, (size_t)batch * sizeof(cwo::ItemParams), cudaMemcpyHostToDevice, s)))
        return cuda_fail(e, "item table upload");
    if ((st = staging_release_after(p->istage, islot, s))) return st;

    const long long wstride = (long long)p->ny * p->px;
    const float scale = (float)(1.0 / ((double)p->px * (double)p->py));
    const bool timing = p->tev[0] != nullptr;
    auto mark = [&](int i) { return timing ? cudaEventRecord(p->tev[i], s) : cudaSuccess; };
    const float2* fin = (const float2*)in;
    float2* fout = (float2*)out;
    if ((e = mark(0))) return cuda_fail(e, "event");
    for (int i0 = 0; i0 < batch;) {
        int i1 = i0 + 1;
        while (i1 < batch && lines(i1) == lines(i0)) ++i1;
        const int n = i1 - i0;
        const bool last = i1 == batch;
        if (lines(i0)) {
            CUtensorMap omap;
            if ((e = cwo::make_intermediate_map(&omap, fout + i0 * field, p->nx, p->ny, n, cwo::line_block_rows(p->py))))
                return cuda_fail(e, "tensor map of the output");
            if ((e = cwo::launch_line_conv(p->px, fin + i0 * in_stride, in_stride, &p->wmap_s, p->ny, n,
                                           (const float2*)(p->ix + (size_t)i0 * p->px), 2LL * p->px, 0,
                                           (float)(1.0 / p->px), p->tw_x, p->status, nullptr, nullptr, s)) ||
                (last && (e = mark(1))) ||
                (e = cwo::launch_line_conv(p->py, p->scratch, field, &omap, p->nx, n,
                                           (const float2*)(p->iy + (size_t)i0 * p->py), 2LL * p->py, 0,
                                           (float)(1.0 / p->py), p->tw_y, p->status, nullptr, nullptr, s)) ||
                (last && (e = mark(2))))
                return cuda_fail(e, "separable Fresnel launch");
        } else {
            cwo::HParams hpar{};
            hpar.mode = cwo::HMODE_ASM_POLY;   // per item, see items
            hpar.ax = p->ix + (size_t)i0 * p->px; hpar.ay = p->iy + (size_t)i0 * p->py; hpar.items = p->iprm + i0;
            hpar.x_item_stride = p->px; hpar.y_item_stride = p->py;
            hpar.kbx = p->kb_x; hpar.kby = p->kb_y; hpar.pairs = p->pairs_x; hpar.npairs = p->px / 2 + 1;
            if ((e = cwo::launch_row_fwd(p->px, fin + i0 * in_stride, in_stride, &p->wmap_f, 0, p->ny, n, p->tw_x,
                                         p->status, s)) ||
                (last && (e = mark(1))))
                return cuda_fail(e, "row forward launch");
            if ((e = cwo::launch_col(p->py, p->scratch, wstride, p->scratch, wstride, p->px, n, p->tw_y, hpar, s)) ||
                (last && (e = mark(2))))
                return cuda_fail(e, "column launch");
            if ((e = cwo::launch_row_inv(p->px, &p->wmap_i, 0, fout + i0 * field, field, p->ny, n, scale, p->tw_x,
                                         p->status, s)))
                return cuda_fail(e, "row inverse launch");
        }
        i0 = i1;
    }
    if ((e = mark(3))) return cuda_fail(e, "event");
    return CWO_OK;
}

}  // namespace

// The GS loop with the field kept in the intermediate between propagations: propagation k of the
// 2I + 1 (+z for even k, the adjoint for odd k) is a column pass between two row passes, and
// the inverse row pass of k with its constraint (phase after +z, amplitude after -z) and the
// forward row pass of k + 1 run as one kernel (launch_row_turn); only the last propagation
// writes the field.  Buffers are checked by the caller.
cwo_status gs_fused(cwo_plan* p, const float* amplitude, float2* u, int batch, int iterations, cudaStream_t s) {
    cwo_status st = ensure_scratch(p, batch);
    if (st) return st;
    cwo::HParams hp = base_hparams(p, nullptr, 1);
    hp.ax = p->ax; hp.ay = p->ay; hp.kf = p->kf; hp.hx = p->hx; hp.hy = p->hy;
    hp.x_item_stride = 0; hp.y_item_stride = 0; hp.kf_item_stride = 0;
    if (p->hcache) {
        hp.mode = cwo::HMODE_TABLE;
        hp.hcache = p->hcache;
        hp.hcache_stride = p->py;
        hp.split_tw = p->split_tw;
        hp.split_w = p->split_w;
    }
    const long long field = (long long)p->nx * p->ny, wstride = (long long)p->ny * p->px;
    const float scale = (float)(1.0 / ((double)p->px * (double)p->py));
    cwo::Epilogue ph, am;
    ph.mode = cwo::EPI_PHASE;
    am.mode = cwo::EPI_AMPLITUDE;
    am.amp = amplitude;
    cudaError_t e = cwo::launch_row_fwd(p->px, u, field, &p->wmap_f, 0, p->ny, batch, p->tw_x, p->status, s);
    if (e) return cuda_fail(e, "row forward launch");
    const int props = 2 * iterations + 1;
    for (int k = 0; k < props; ++k) {
        hp.conj = k & 1;
        if ((e = cwo::launch_col(p->py, p->scratch, wstride, p->scratch, wstride, p->px, batch, p->tw_y, hp, s)))
            return cuda_fail(e, "column launch");
        if (k + 1 < props)
            e = cwo::launch_row_turn(p->px, &p->wmap_f, p->ny, batch, field, scale, p->tw_x, p->status, (k & 1) ? am : ph, s);
        else
            e = cwo::launch_row_inv(p->px, &p->wmap_i, 0, u, field, p->ny, batch, scale, p->tw_x, p->status, s, ph);
        if (e) return cuda_fail(e, "row pass launch");
    }
    return CWO_OK;
}

// ------------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------------
namespace {
cwo_status create_impl(int nx, int ny, double dx, double dy, double lambda, double z, cwo_type type, unsigned flags,
                       const cwo_shift* shift, cwo_plan** out, const cwo_shifted_fresnel* sfr = nullptr) {
    cwo_status st;
    cwo_plan* p = new (std::nothrow) cwo_plan();
    if (!p) return fail(CWO_ERR_OOM, "host allocation failed");
    p->nx = nx; p->ny = ny; p->px = 2 * nx; p->py = 2 * ny;
    if (type == CWO_FRESNEL_FOURIER) { p->px = nx; p->py = ny; }   // one unpadded DFT
    p->dx = dx; p->dy = dy; p->lambda = lambda; p->z = z; p->type = type; p->flags = flags;
    if (shift) {
        p->shifted = true;
        p->shift = *shift;
    }
    if (sfr) p->sfr = *sfr;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) { free_plan(p); return cuda_fail(e, "cudaGetDevice"); }

    const AxisGeo gx(p->px), gy(p->py);
    const std::vector<float4> twx = twiddle_table(gx);
    const std::vector<int> kbx = bin_table(gx), kby = bin_table(gy);
    if ((st = dev_alloc(&p->tw_x, twx.size(), "x twiddles")) || (st = upload(p->tw_x, twx, "x twiddle upload"))) { free_plan(p); return st; }
    if (p->py == p->px) {
        p->tw_y = p->tw_x;
    } else {
        const std::vector<float4> twy = twiddle_table(gy);
        if ((st = dev_alloc(&p->tw_y, twy.size(), "y twiddles")) || (st = upload(p->tw_y, twy, "y twiddle upload"))) { free_plan(p); return st; }
    }
    const std::vector<int2> prs = mirror_pairs(gx);
    if ((st = dev_alloc(&p->pairs_x, prs.size(), "x pairs")) || (st = upload(p->pairs_x, prs, "x pair upload"))) { free_plan(p); return st; }
    if ((st = dev_alloc(&p->kb_x, kbx.size(), "x bins")) || (st = upload(p->kb_x, kbx, "x bin upload")) ||
        (st = dev_alloc(&p->kb_y, kby.size(), "y bins")) || (st = upload(p->kb_y, kby, "y bin upload"))) { free_plan(p); return st; }
    if (type == CWO_SHIFTED_FRESNEL) {
        std::vector<float2> fx(nx), fy(ny), qx(nx), qy(ny), hx(p->px), hy(p->py);
        const double cph = 2.0 * kPi * frac01(z / lambda);
        cd C = cd(std::cos(cph), std::sin(cph)) / cd(0.0, lambda * z);
        if (!(flags & CWO_FLAG_LITERAL_SCALE)) C *= dx * dy;
        shifted_fresnel_axis(nx, dx, p->sfr.dx1, p->sfr.ox0, p->sfr.ox1, lambda, z, C, fx.data(), qx.data(), hx.data());
        shifted_fresnel_axis(ny, dy, p->sfr.dy1, p->sfr.oy0, p->sfr.oy1, lambda, z, cd(1.0, 0.0), fy.data(), qy.data(), hy.data());
        auto conj = [](std::vector<float2> v) { for (auto& a : v) a.y = -a.y; return v; };
        const std::vector<float2> cqx = conj(qx), cqy = conj(qy), cfx = conj(fx), cfy = conj(fy);
        if ((st = dev_alloc(&p->fpre_x, nx, "x source factor")) || (st = upload(p->fpre_x, fx, "upload")) ||
            (st = dev_alloc(&p->fpre_y, ny, "y source factor")) || (st = upload(p->fpre_y, fy, "upload")) ||
            (st = dev_alloc(&p->fpost_x, nx, "x destination factor")) || (st = upload(p->fpost_x, qx, "upload")) ||
            (st = dev_alloc(&p->fpost_y, ny, "y destination factor")) || (st = upload(p->fpost_y, qy, "upload")) ||
            (st = dev_alloc(&p->fpre_cx, nx, "x adjoint factor")) || (st = upload(p->fpre_cx, cqx, "upload")) ||
            (st = dev_alloc(&p->fpre_cy, ny, "y adjoint factor")) || (st = upload(p->fpre_cy, cqy, "upload")) ||
            (st = dev_alloc(&p->fpost_cx, nx, "x adjoint factor")) || (st = upload(p->fpost_cx, cfx, "upload")) ||
            (st = dev_alloc(&p->fpost_cy, ny, "y adjoint factor")) || (st = upload(p->fpost_cy, cfy, "upload")) ||
            (st = dev_alloc(&p->hx, hx.size(), "x table")) || (st = upload(p->hx, hx, "x table upload")) ||
            (st = dev_alloc(&p->hy, hy.size(), "y table")) || (st = upload(p->hy, hy, "y table upload"))) {
            free_plan(p);
            return st;
        }
    } else if (type == CWO_FRESNEL_FOURIER) {
        std::vector<float2> prx(nx), pry(ny), pox(nx), poy(ny);
        std::vector<int> stx(nx), rwy(ny);
        fourier_tables(nx, ny, dx, dy, lambda, z, (flags & CWO_FLAG_LITERAL_SCALE) != 0, prx.data(), pry.data(),
                       pox.data(), poy.data(), stx.data(), rwy.data());
        if ((st = dev_alloc(&p->fpre_x, prx.size(), "x chirp")) || (st = upload(p->fpre_x, prx, "x chirp upload")) ||
            (st = dev_alloc(&p->fpre_y, pry.size(), "y chirp")) || (st = upload(p->fpre_y, pry, "y chirp upload")) ||
            (st = dev_alloc(&p->fpost_x, pox.size(), "x output chirp")) || (st = upload(p->fpost_x, pox, "x output chirp upload")) ||
            (st = dev_alloc(&p->fpost_y, poy.size(), "y output chirp")) || (st = upload(p->fpost_y, poy, "y output chirp upload")) ||
            (st = dev_alloc(&p->fst_x, stx.size(), "x placement")) || (st = upload(p->fst_x, stx, "x placement upload")) ||
            (st = dev_alloc(&p->frow_y, rwy.size(), "y placement")) || (st = upload(p->frow_y, rwy, "y placement upload"))) {
            free_plan(p);
            return st;
        }
    } else if (type == CWO_ANGULAR || type == CWO_SHIFTED_ANGULAR) {
        std::vector<float4> ax(p->px), ay(p->py);
        std::vector<float> kf(1);
        host_h_tables(p, z, ax.data(), ay.data(), nullptr, nullptr, kf.data());
        if ((st = dev_alloc(&p->ax, ax.size(), "x table")) || (st = upload(p->ax, ax, "x table upload")) ||
            (st = dev_alloc(&p->ay, ay.size(), "y table")) || (st = upload(p->ay, ay, "y table upload")) ||
            (st = dev_alloc(&p->kf, kf.size(), "K")) || (st = upload(p->kf, kf, "K upload"))) { free_plan(p); return st; }
    } else {
        std::vector<float2> hx(p->px), hy(p->py);
        host_h_tables(p, z, nullptr, nullptr, hx.data(), hy.data(), nullptr);
        if ((st = dev_alloc(&p->hx, hx.size(), "x table")) || (st = upload(p->hx, hx, "x table upload")) ||
            (st = dev_alloc(&p->hy, hy.size(), "y table")) || (st = upload(p->hy, hy, "y table upload"))) { free_plan(p); return st; }
    }
    if ((st = dev_alloc(&p->status, 1, "status word"))) { free_plan(p); return st; }
    if ((e = cudaMemset(p->status, 0, sizeof(int))) != cudaSuccess) { free_plan(p); return cuda_fail(e, "cudaMemset"); }
    if ((st = ensure_scratch(p, 1))) { free_plan(p); return st; }
    if ((flags & CWO_FLAG_CACHE_H) && type == CWO_ANGULAR) {
        const int npairs = p->px / 2 + 1;
        if ((st = dev_alloc(&p->hcache, (size_t)npairs * p->py, "transfer-function cache"))) { free_plan(p); return st; }
        int* yidx = nullptr;   // the split order of the split column pass
        if (p->py == cwo::kSplitColP) {
            const std::vector<float4> twq = twiddle_table(AxisGeo(p->py / 2));
            const std::vector<float2> wn = split_phase(p->py);
            const std::vector<int> yi = split_axis_index(p->py);
            const size_t n4 = twq.size() + (wn.size() + 1) / 2;
            if ((st = dev_alloc(&p->split_tw, n4, "split twiddles")) || (st = upload(p->split_tw, twq, "split twiddle upload"))) {
                free_plan(p);
                return st;
            }
            p->split_w = reinterpret_cast<float2*>(p->split_tw + twq.size());
            if ((st = upload(p->split_w, wn, "split phase upload")) || (st = dev_alloc(&yidx, yi.size(), "split index")) ||
                (st = upload(yidx, yi, "split index upload"))) {
                cudaFree(yidx);
                free_plan(p);
                return st;
            }
        }
        const cwo::HParams hp = base_hparams(p, nullptr, 1);
        if ((e = cwo::launch_build_hcache(p->hcache, npairs, p->py, hp, nullptr, yidx)) != cudaSuccess ||
            (e = cudaDeviceSynchronize()) != cudaSuccess) {
            cudaFree(yidx);
            free_plan(p);
            return cuda_fail(e, "building the transfer-function cache");
        }
        cudaFree(yidx);
    }
    *out = p;
    return CWO_OK;
}
}  // namespace

extern "C" {

const char* cwo_last_error(void) { return g_err.c_str(); }

int cwo_version(void) { return 1 * 10000 + 0 * 100 + 0; }

cwo_status cwo_plan_device_bytes(int nx, int ny, int batch, size_t* bytes) {
    if (!bytes) return fail(CWO_ERR_INVALID_ARG, "bytes is NULL");
    if (!pow2_side(nx) || !pow2_side(ny)) return fail(CWO_ERR_INVALID_ARG, "Nx=%d, Ny=%d out of range", nx, ny);
    if (batch < 1) return fail(CWO_ERR_INVALID_ARG, "batch must be >= 1");
    *bytes = tables_bytes(nx, ny) + (size_t)batch * ny * (2 * (size_t)nx) * sizeof(float2) +
             (size_t)batch * (2 * (size_t)nx + 2 * (size_t)ny) * sizeof(float4) + (size_t)batch * sizeof(cwo::ItemParams);
    return CWO_OK;
}


cwo_status cwo_plan_create(int nx, int ny, double dx, double dy, double lambda, double z,
                           cwo_type type, unsigned flags, cwo_plan** out) {
    if (!out) return fail(CWO_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (type == CWO_SHIFTED_ANGULAR)
        return fail(CWO_ERR_INVALID_ARG, "create shifted angular-spectrum plans with cwo_plan_create_shifted");
    cwo_status st = check_params(nx, ny, dx, dy, lambda, z, (int)type, flags);
    if (st) return st;
    return create_impl(nx, ny, dx, dy, lambda, z, type, flags, nullptr, out);
}

cwo_status cwo_plan_create_shifted(int nx, int ny, double dx, double dy, double lambda, double z,
                                   const cwo_shift* shift, unsigned flags, cwo_plan** out) {
    if (!out) return fail(CWO_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!shift) return fail(CWO_ERR_INVALID_ARG, "shift is NULL");
    cwo_status st = check_params(nx, ny, dx, dy, lambda, z, (int)CWO_ANGULAR, flags);
    if (st) return st;
    if (flags & CWO_FLAG_PHASE_FP32) return fail(CWO_ERR_UNSUPPORTED, "CWO_FLAG_PHASE_FP32 is not provided with a shift");
    const double v[6] = {shift->ox, shift->oy, shift->cx, shift->wx, shift->cy, shift->wy};
    for (double x : v)
        if (!std::isfinite(x)) return fail(CWO_ERR_INVALID_ARG, "shift and window parameters must be finite");
    int lo, hi;
    window_bins(AxisGeo(2 * nx), dx, shift->cx, shift->wx, &lo, &hi);
    if (lo > hi) return fail(CWO_ERR_INVALID_ARG, "the x window contains no frequency bin");
    window_bins(AxisGeo(2 * ny), dy, shift->cy, shift->wy, &lo, &hi);
    if (lo > hi) return fail(CWO_ERR_INVALID_ARG, "the y window contains no frequency bin");
    return create_impl(nx, ny, dx, dy, lambda, z, CWO_SHIFTED_ANGULAR, flags, shift, out);
}

cwo_status cwo_plan_create_shifted_fresnel(int nx, int ny, double dx0, double dy0, double lambda, double z,
                                           const cwo_shifted_fresnel* sf, unsigned flags, cwo_plan** out) {
    if (!out) return fail(CWO_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!sf) return fail(CWO_ERR_INVALID_ARG, "parameters are NULL");
    cwo_status st = check_params(nx, ny, dx0, dy0, lambda, z, (int)CWO_FRESNEL_CONV, flags);
    if (st) return st;
    if (!(sf->dx1 > 0) || !(sf->dy1 > 0) || !std::isfinite(sf->dx1) || !std::isfinite(sf->dy1))
        return fail(CWO_ERR_INVALID_ARG, "destination pitches must be finite and > 0");
    if (!std::isfinite(sf->ox0) || !std::isfinite(sf->oy0) || !std::isfinite(sf->ox1) || !std::isfinite(sf->oy1))
        return fail(CWO_ERR_INVALID_ARG, "offsets must be finite");
    return create_impl(nx, ny, dx0, dy0, lambda, z, CWO_SHIFTED_FRESNEL, flags, nullptr, out, sf);
}

cwo_status cwo_band_limit(int nx, int ny, double dx, double dy, double lambda, double z, cwo_shift* out) {
    if (!out) return fail(CWO_ERR_INVALID_ARG, "out is NULL");
    cwo_status st = check_params(nx, ny, dx, dy, lambda, z, (int)CWO_ANGULAR, 0);
    if (st) return st;
    *out = cwo_shift{};
    out->wx = 2.0 * band_limit_freq(2 * nx, dx, lambda, z);
    out->wy = 2.0 * band_limit_freq(2 * ny, dy, lambda, z);
    return CWO_OK;
}

cwo_status cwo_plan_destroy(cwo_plan* plan) {
    free_plan(plan);
    return CWO_OK;
}

cwo_status cwo_plan_reserve(cwo_plan* plan, int batch) {
    if (!plan) return fail(CWO_ERR_INVALID_ARG, "plan is NULL");
    if (batch < 1 || batch > 65535) return fail(CWO_ERR_INVALID_ARG, "batch must be in [1, 65535]");
    cwo_status st = check_plan_device(plan);
    if (st) return st;
    if ((st = ensure_scratch(plan, batch + 1))) return st;
    // mixed batches (cwo_propagate_items) also need per-item tables and their pinned staging
    return ensure_itables(plan, batch);
}

cwo_status cwo_propagate(cwo_plan* plan, const void* in_c64, void* out_c64, void* cuda_stream) {
    if (!plan) return fail(CWO_ERR_INVALID_ARG, "plan is NULL");
    return run(plan, in_c64, (long long)plan->nx * plan->ny, out_c64, 1, nullptr, cuda_stream, false);
}

cwo_status cwo_propagate_batch(cwo_plan* plan, const void* in, long long in_batch_stride, void* out,
                               int batch, const double* z_or_null, void* cuda_stream) {
    return run(plan, in, in_batch_stride, out, batch, z_or_null, cuda_stream, false);
}

cwo_status cwo_propagate_items(cwo_plan* plan, const void* in, long long in_batch_stride, void* out, int batch,
                               const cwo_item* items, void* cuda_stream) {
    return run_items(plan, in, in_batch_stride, out, batch, items, cuda_stream);
}

cwo_status cwo_propagate_adjoint(cwo_plan* plan, const void* in_c64, void* out_c64, void* cuda_stream) {
    if (!plan) return fail(CWO_ERR_INVALID_ARG, "plan is NULL");
    return run(plan, in_c64, (long long)plan->nx * plan->ny, out_c64, 1, nullptr, cuda_stream, true);
}

cwo_status cwo_propagate_adjoint_batch(cwo_plan* plan, const void* in, long long in_batch_stride,
                                       void* out, int batch, const double* z_or_null, void* cuda_stream) {
    if (in_batch_stride == 0) return fail(CWO_ERR_INVALID_ARG, "the adjoint takes one input per item (stride > 0)");
    return run(plan, in, in_batch_stride, out, batch, z_or_null, cuda_stream, true);
}

cwo_status cwo_propagate_epilogue(cwo_plan* plan, const void* in_c64, void* out_c64, int batch, int adjoint,
                                  int epilogue, const float* amplitude, float* intensity, void* cuda_stream) {
    if (!plan) return fail(CWO_ERR_INVALID_ARG, "plan is NULL");
    if (epilogue < CWO_EPI_NONE || epilogue > CWO_EPI_INTENSITY) return fail(CWO_ERR_INVALID_ARG, "unknown epilogue %d", epilogue);
    cwo::Epilogue ep;
    ep.mode = epilogue;
    ep.amp = amplitude;
    ep.inten = intensity;
    if (epilogue == CWO_EPI_AMPLITUDE && !amplitude) return fail(CWO_ERR_INVALID_ARG, "the amplitude epilogue needs an amplitude");
    if (epilogue == CWO_EPI_INTENSITY && !intensity) return fail(CWO_ERR_INVALID_ARG, "the intensity epilogue needs an intensity buffer");
    return run(plan, in_c64, (long long)plan->nx * plan->ny, out_c64, batch, nullptr, cuda_stream, adjoint != 0, ep);
}

cwo_status cwo_gs_run(cwo_plan* plan, const float* amplitude, void* field_c64, float* intensity, int batch,
                      int iterations, void* cuda_stream) {
    if (!plan) return fail(CWO_ERR_INVALID_ARG, "plan is NULL");
    if (plan->type != CWO_ANGULAR && plan->type != CWO_SHIFTED_ANGULAR)
        return fail(CWO_ERR_UNSUPPORTED, "the GS iteration uses an angular-spectrum plan");
    if (!amplitude || !field_c64) return fail(CWO_ERR_INVALID_ARG, "amplitude and field are required");
    if (iterations < 0 || iterations > 1000000) return fail(CWO_ERR_INVALID_ARG, "iterations must be in [0, 1e6] (got %d)", iterations);
    const long long f = (long long)plan->nx * plan->ny;
    cwo::Epilogue ph, am, in;
    ph.mode = cwo::EPI_PHASE;
    am.mode = cwo::EPI_AMPLITUDE;
    am.amp = amplitude;
    in.mode = cwo::EPI_INTENSITY;
    in.inten = intensity;
    // every buffer is checked once; the loop then re-propagates the same buffers
    cwo_status st = check_plan_device(plan);
    if (st) return st;
    if (batch < 1 || batch > 65535) return fail(CWO_ERR_INVALID_ARG, "batch must be in [1, 65535] (got %d)", batch);
    const size_t n = (size_t)batch * (size_t)f;
    if ((st = check_device_range(field_c64, n * sizeof(float2), plan->device, "field")) ||
        (st = check_device_range(amplitude, n * sizeof(float), plan->device, "amplitude")) ||
        (intensity && (st = check_device_range(intensity, n * sizeof(float), plan->device, "intensity"))))
        return st;
    if (cwo::row_turn_supported(plan->px)) {
        st = gs_fused(plan, amplitude, (float2*)field_c64, batch, iterations, (cudaStream_t)cuda_stream);
    } else {
        // hologram plane: propagate the object field by +z and keep the phase (the kinoform)
        st = run(plan, field_c64, f, field_c64, batch, nullptr, cuda_stream, false, ph, true);
        for (int i = 0; i < iterations && st == CWO_OK; ++i) {
            // back to the object plane (conj(H) = H(-z)), amplitude constraint; forward, phase constraint
            st = run(plan, field_c64, f, field_c64, batch, nullptr, cuda_stream, true, am, true);
            if (st == CWO_OK) st = run(plan, field_c64, f, field_c64, batch, nullptr, cuda_stream, false, ph, true);
        }
    }
    if (st == CWO_OK && intensity) st = run(plan, field_c64, f, nullptr, batch, nullptr, cuda_stream, true, in, true);
    return st;
}

int cwo_launches_per_call(const cwo_plan* plan) {
    if (!plan) return 0;
    return plan->type == CWO_FRESNEL_FOURIER || plan->type == CWO_FRESNEL_CONV || plan->type == CWO_SHIFTED_FRESNEL ? 2 : 3;
}

cwo_status cwo_plan_check(cwo_plan* plan) {
    if (!plan) return fail(CWO_ERR_INVALID_ARG, "plan is NULL");
    cwo_status st = check_plan_device(plan);
    if (st) return st;
    int word = 0;
    cudaError_t e = cudaMemcpy(&word, plan->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "reading the status word");
    if (word) {
        if ((e = cudaMemset(plan->status, 0, sizeof(int))) != cudaSuccess) return cuda_fail(e, "clearing the status word");
        return fail(CWO_ERR_TIMEOUT, "a bounded wait on an asynchronous copy expired; the affected output was not written");
    }
    return CWO_OK;
}

cwo_status cwo_plan_set_timing_events(cwo_plan* plan, void* const* events) {
    if (!plan) return fail(CWO_ERR_INVALID_ARG, "plan is NULL");
    for (int i = 0; i < 4; ++i) plan->tev[i] = events ? (cudaEvent_t)events[i] : nullptr;
    if (events)
        for (int i = 0; i < 4; ++i)
            if (!plan->tev[i]) { for (auto& ev : plan->tev) ev = nullptr; return fail(CWO_ERR_INVALID_ARG, "events[%d] is NULL", i); }
    return CWO_OK;
}

// ---------------------------------------------------------------- host-only diagnostics
cwo_status cwo_debug_axis_bins(int p, int* bins) {
    if (!bins || p < 32 || p > 8192 || (p & (p - 1))) return fail(CWO_ERR_INVALID_ARG, "bad axis length");
    const AxisGeo g(p);
    for (int i = 0; i < p; ++i) bins[i] = g.freq_of_idx(i);
    return CWO_OK;
}

cwo_status cwo_debug_split_axis(int p, int* index, float* phase_ri) {
    if (p < 64 || p > 8192 || (p & (p - 1))) return fail(CWO_ERR_INVALID_ARG, "bad axis length");
    if (index) {
        const std::vector<int> v = split_axis_index(p);
        std::copy(v.begin(), v.end(), index);
    }
    if (phase_ri) {
        const std::vector<float2> w = split_phase(p);
        for (size_t n = 0; n < w.size(); ++n) { phase_ri[2 * n] = w[n].x; phase_ri[2 * n + 1] = w[n].y; }
    }
    return CWO_OK;
}

cwo_status cwo_debug_fresnel_axis(int p, double pitch, double lambda, double z, double* out_ri) {
    if (!out_ri || p < 2 || (p & (p - 1)) || !(pitch > 0) || !(lambda > 0) || z == 0.0)
        return fail(CWO_ERR_INVALID_ARG, "bad arguments");
    const std::vector<cd> h = fresnel_axis_dft(p, pitch, lambda, z);
    for (int i = 0; i < p; ++i) { out_ri[2 * i] = h[i].real(); out_ri[2 * i + 1] = h[i].imag(); }
    return CWO_OK;
}

cwo_status cwo_debug_twiddles(int p, float* out_ri) {
    if (!out_ri || p < 32 || p > 8192 || (p & (p - 1))) return fail(CWO_ERR_INVALID_ARG, "bad axis length");
    const AxisGeo g(p);
    const std::vector<float4> tw = twiddle_table(g);
    for (size_t i = 0; i < tw.size(); ++i) {
        out_ri[4 * i] = tw[i].x; out_ri[4 * i + 1] = tw[i].y; out_ri[4 * i + 2] = tw[i].z; out_ri[4 * i + 3] = tw[i].w;
    }
    return CWO_OK;
}

cwo_status cwo_debug_asm_axis(int p, double pitch, double lambda, double z, int is_x, float* out4) {
    if (!out4 || p < 32 || p > 8192 || (p & (p - 1)) || !(pitch > 0) || !(lambda > 0))
        return fail(CWO_ERR_INVALID_ARG, "bad arguments");
    const AxisGeo g(p);
    asm_axis_table(g, pitch, lambda, z, is_x != 0, (float4*)out4);
    return CWO_OK;
}

}  // extern "C"
