/*
 * cwo.h -- C ABI of libcwo_gb300.so: FFT-based scalar diffraction on one GB300 GPU.
 *
 * The library computes the two convolution-form diffraction methods of Shimobaba et al.,
 * "Computational wave optics library for C++: CWO++ library":
 *
 *   CWO_ANGULAR       angular spectrum method (Section "Angular spectrum method", Eqs. ang1-ang3)
 *                       u2 = IFFT[ FFT[u1] * H_A ],
 *                       H_A(fx, fy) = exp(i z sqrt(k^2 - 4 pi^2 (fx^2 + fy^2))),  k = 2 pi / lambda
 *   CWO_FRESNEL_CONV  Fresnel diffraction, convolution form (Section "Fresnel diffraction
 *                     (convolution form)", Eqs. fre_conv, fre_conv_fft, fre_conv_prop_d)
 *                       u2 = C * IFFT[ FFT[u1] * FFT[h_F] ],
 *                       h_F(m, n) = exp(i pi ((m dx)^2 + (n dy)^2) / (lambda z)),
 *                       C = dx dy exp(i 2 pi z / lambda) / (i lambda z)
 *
 * Every propagation zero-pads the Nx x Ny source to 2Nx x 2Ny (the source occupies the top-left
 * block), transforms, multiplies by the transfer function, transforms back and keeps the exact
 * Nx x Ny block (Section "Summary of diffraction calculation", Table "Classification of
 * diffraction calculation").  The result equals the linear (not circular) convolution.
 *
 * Conventions the paper leaves open, as this library reads them:
 *   - forward DFT unscaled with exp(-2 pi i k n / P); the inverse carries 1/(Px Py)
 *   - frequency of bin k on the padded grid: f = kt / (P * pitch), kt = k for k < P/2, else k - P
 *   - evanescent bins of H_A (negative radicand) are set to 0
 *   - the Fresnel transfer function is the DFT of h_F sampled on the padded grid (index i maps
 *     to displacement i for i < P/2, i - P otherwise); h_F is separable, so it is formed as the
 *     outer product of two 1-D DFTs computed once per plan in double precision, and the 2-D
 *     padded convolution is computed as a padded 1-D convolution of every row followed by one of
 *     every column (the same linear convolution, up to rounding)
 *   - C includes the area element dx*dy of the discretised integral (CWO_FLAG_LITERAL_SCALE
 *     drops it, which is the paper's printed coefficient)
 *   - defaults (Section "CWO class", paragraph after Eq. norm): wavelength 633 nm, pitch 10 um;
 *     pass CWO_DEFAULT_WAVELENGTH / CWO_DEFAULT_PITCH to use them
 *
 *   CWO_FRESNEL_FOURIER  Fresnel diffraction in Fourier form (Section "The Fresnel diffraction
 *                     (Fourier form)", Eqs. fre_fourier2, fre_fourier3): one UNPADDED Nx x Ny DFT
 *                       u2 = C exp(i pi (x2^2 + y2^2) / (lambda z)) DFT[u1 exp(i pi (x1^2 + y1^2) / (lambda z))]
 *                     with centred coordinates on both planes: x1 = (m - Nx/2) dx and
 *                     x2 = (k - Nx/2) lambda z / (Nx dx) (array element Nx/2 is the axis; the
 *                     destination pitch is lambda z / (Nx dx), as for y), C as above.  Nx, Ny >= 32;
 *                     z != 0; forward only (no adjoint, per-item z, stack or epilogue); two passes.
 *
 * Data layout: fields are complex64 (interleaved float re, im; torch.complex64), row-major
 * [batch][Ny][Nx], contiguous, in DEVICE memory of the current CUDA device.  The caller owns all
 * field buffers; input and output may alias (the input is fully consumed by the first pass before
 * the output is written).  A plan owns its tables and its scratch (the 2N-wide intermediate).
 *
 * Precision: field and FFT arithmetic in FP32; the transfer-function phase (up to ~2e6 cycles for
 * z / lambda at the studied sizes) is range-reduced in FP64 on per-axis tables, leaving an O(1)
 * remainder that is evaluated per element in float-float / FP32 (see cwo_plan_create flags).
 *
 * Ordering: all work is enqueued on the caller's stream (a cudaStream_t passed as void*; NULL is
 * the legacy default stream).  Calls do not synchronise the device, except cwo_plan_create and
 * cwo_plan_reserve (allocation and the upload of the plan's tables).
 *
 * Errors: every entry point returns a cwo_status and never aborts.  Arguments are checked on the
 * host before anything is enqueued; on failure nothing is launched.  cwo_last_error() returns a
 * thread-local message describing the most recent failure on the calling thread.
 *
 * Thread safety: distinct plans may be used concurrently from different threads.  One plan must
 * not be used by two threads at the same time, and calls on one plan that run concurrently on
 * different streams race on the plan's scratch.
 */
#ifndef CWO_H
#define CWO_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CWO_DEFAULT_WAVELENGTH 633e-9
#define CWO_DEFAULT_PITCH 10e-6
#define CWO_MIN_SIDE 16
#define CWO_MAX_SIDE 4096

typedef enum {
    CWO_ANGULAR = 0,          /* angular spectrum method (Eq. ang3)                      */
    CWO_FRESNEL_CONV = 1,     /* Fresnel diffraction, convolution form (Eq. fre_conv_fft) */
    CWO_FRESNEL_FOURIER = 2,  /* Fresnel diffraction, Fourier form (Eq. fre_fourier3; below)  */
    CWO_SHIFTED_FRESNEL = 3,  /* shifted Fresnel (Eqs. shift_fre1-3): plans come from
                                 cwo_plan_create_shifted_fresnel                          */
    CWO_SHIFTED_ANGULAR = 4   /* shifted angular spectrum (Eqs. shift_ang1, shift_ang2): plans come
                                 from cwo_plan_create_shifted                             */
} cwo_type;

typedef enum {
    CWO_OK = 0,
    CWO_ERR_INVALID_ARG = 1,  /* a size, pitch, wavelength, distance, pointer or flag is invalid */
    CWO_ERR_UNSUPPORTED = 2,  /* a diffraction type or mode this library does not provide       */
    CWO_ERR_OOM = 3,          /* device or pinned-host allocation failed                          */
    CWO_ERR_CUDA = 4,         /* a CUDA runtime call or kernel launch failed                      */
    CWO_ERR_TIMEOUT = 5       /* a bounded wait expired                                           */
} cwo_status;

/* plan flags */
#define CWO_FLAG_PHASE_FP32    0x1u  /* precision study: evaluate the whole ASM phase in FP32   */
#define CWO_FLAG_PHASE_FP64    0x2u  /* precision study: literal per-element FP64 ASM phase     */
#define CWO_FLAG_LITERAL_SCALE 0x4u  /* Fresnel: C without the dx*dy area element              */
#define CWO_FLAG_CACHE_H       0x8u  /* ASM: materialise H for the plan's own z at creation
                                        (the paper's "once-calculation", Section "Performance"):
                                        (Nx + 1) x 2Ny complex64 on the device (67 MB at 2048^2);
                                        calls with the plan's z read it instead of evaluating
                                        the phase per element (same values, same results);
                                        calls with per-item distances evaluate as usual       */

typedef struct cwo_plan cwo_plan;

/*
 * Create a plan for Nx x Ny fields (each a power of two in [16, 4096]) with pitches dx, dy (> 0,
 * metres), wavelength lambda (> 0, metres) and distance z (metres; any finite value for
 * CWO_ANGULAR, z = 0 gives the identity; non-zero for CWO_FRESNEL_CONV).  The plan computes
 * its per-axis tables in FP64 on the host ("once-calculation", Section "Performance") and uploads
 * them, and allocates scratch for one field.  *out receives the plan; on failure *out is NULL.
 */
cwo_status cwo_plan_create(int nx, int ny, double dx, double dy, double lambda, double z,
                           cwo_type type, unsigned flags, cwo_plan** out);

/* Shifted angular spectrum parameters (Section "Shifted angular spectrum method",
 * Eqs. shift_ang1 and shift_ang2, the imaginary unit of the shift phase restored):
 *   H_SA = H_A(fx, fy) exp(i 2 pi (ox fx + oy fy)) Rect((fx - cx) / wx) Rect((fy - cy) / wy)
 * ox, oy: shift of the destination window (metres); cx, wx, cy, wy: centre and full width of the
 * band-limit windows (1/metre, on the padded grid's frequencies kt / (2N pitch)); a width <= 0
 * means no window on that axis; Rect(x) = 1 for |x| <= 1/2.  The paper leaves the choice of the
 * windows to the shifted-ASM literature; cwo_band_limit gives the on-axis band limit. */
typedef struct {
    double ox, oy;
    double cx, wx;
    double cy, wy;
} cwo_shift;

/* A CWO_SHIFTED_ANGULAR plan: like cwo_plan_create(..., CWO_ANGULAR, ...) with the shift phase
 * and windows folded into the per-axis FP64 tables.  flags: 0 or CWO_FLAG_PHASE_FP64
 * (CWO_FLAG_PHASE_FP32: CWO_ERR_UNSUPPORTED).  Per-item distances (z_or_null) are not provided
 * for these plans (CWO_ERR_UNSUPPORTED); batches, z-stacks of the plan's z, the adjoint and the
 * epilogues are.  CWO_ERR_INVALID_ARG for non-finite parameters or a window that holds no bin. */
cwo_status cwo_plan_create_shifted(int nx, int ny, double dx, double dy, double lambda, double z,
                                   const cwo_shift* shift, unsigned flags, cwo_plan** out);

/* Shifted Fresnel diffraction (Section "Shifted Fresnel diffraction", Eqs. shift_fre1 to
 * shift_fre3): the Fresnel integral from a source grid of pitch (dx0, dy0) centred at (ox0, oy0)
 * to a destination grid of pitch (dx1, dy1) centred at (ox1, oy1) (metres; off-axis and
 * rescaling).  With x0 = m0 dx0 + ox0, x1 = m1 dx1 + ox1, m = array index - N/2 and
 * S = dx0 dx1 / (lambda z), writing 2 m1 m0 = m1^2 + m0^2 - (m1 - m0)^2 gives
 *   u2[m1] = C q[m1] sum_m0 u1[m0] f[m0] exp(i pi S (m1 - m0)^2)       (per axis, times y)
 *   f = exp(i pi x0^2 / (lambda z)) exp(-2 pi i m0 dx0 ox1 / (lambda z)) exp(-i pi S m0^2)
 *   q = exp(i pi x1^2 / (lambda z)) exp(-2 pi i ox0 x1 / (lambda z)) exp(-i pi S m1^2)
 * C = exp(i 2 pi z / lambda) / (i lambda z) dx0 dy0 (CWO_FLAG_LITERAL_SCALE: without dx0 dy0).
 * The sum is the padded convolution path of CWO_FRESNEL_CONV with H = DFT[exp(i pi S d^2)] per
 * axis; f is applied as the first pass loads the source, q and C as the last pass stores.  The
 * adjoint (destination -> source) is provided; per-item distances and epilogues are not. */
typedef struct {
    double dx1, dy1;   /* destination pitches (> 0)  */
    double ox0, oy0;   /* source-grid centre         */
    double ox1, oy1;   /* destination-grid centre    */
} cwo_shifted_fresnel;

cwo_status cwo_plan_create_shifted_fresnel(int nx, int ny, double dx0, double dy0, double lambda, double z,
                                           const cwo_shifted_fresnel* params, unsigned flags, cwo_plan** out);

/* The on-axis band-limited angular spectrum method (Matsushima and Shimobaba, Opt. Express 17,
 * 19662 (2009)): fills *out with no shift and windows centred on zero of full width 2 u, where
 * u = 1 / (lambda sqrt((2 df z)^2 + 1)), df = 1 / (2N pitch), the frequency beyond which the
 * transfer function's phase is undersampled on the padded grid.  Host only. */
cwo_status cwo_band_limit(int nx, int ny, double dx, double dy, double lambda, double z, cwo_shift* out);

/* Release a plan (NULL is accepted).  The caller must make sure no work using it is pending. */
cwo_status cwo_plan_destroy(cwo_plan* plan);

/* Device bytes a plan for this shape needs to run `batch` fields at once (tables, scratch and
 * per-item tables, i.e. what cwo_plan_reserve(batch) holds), for admission control.  Host-only;
 * touches no device. */
cwo_status cwo_plan_device_bytes(int nx, int ny, int batch, size_t* bytes);

/* Grow the plan's scratch and per-item tables so that batches of up to `batch` fields, z-stacks
 * of up to `batch` planes and mixed batches of up to `batch` items run without allocating (and
 * without the device synchronisation a reallocation needs).  Synchronises the device when it
 * reallocates. */
cwo_status cwo_plan_reserve(cwo_plan* plan, int batch);

/* One propagation of one [Ny][Nx] field with the plan's own parameters (Eq. ang3 or
 * Eq. fre_conv_fft with the padding and crop above). */
cwo_status cwo_propagate(cwo_plan* plan, const void* in_c64, void* out_c64, void* cuda_stream);

/*
 * Batched propagation of `batch` fields in one set of launches.
 *   in_batch_stride  elements (complex64) between consecutive input fields; 0 means that every
 *                    item propagates the SAME source field (3-D stack by stacking 2-D
 *                    diffractions along z, Section "Three-dimensional diffraction calculations"):
 *                    its spectrum is computed once and reused for every plane.
 *   out              [batch][Ny][Nx]
 *   z_or_null        NULL: every item uses the plan's z.  Otherwise a HOST array of `batch`
 *                    distances; the per-item tables are computed in FP64 on the host and uploaded
 *                    stream-ordered.
 * Grows the scratch (synchronising) if `batch` exceeds the reserved size.
 * Any complex64-aligned (8-byte) buffers are accepted; fields whose rows start on 16-byte
 * boundaries take the kernels that move them by bulk and TMA copies (the fastest paths), others
 * take per-thread loads (and, for a Fresnel output, the three-pass method): same results up to
 * rounding.
 */
cwo_status cwo_propagate_batch(cwo_plan* plan, const void* in, long long in_batch_stride,
                               void* out, int batch, const double* z_or_null, void* cuda_stream);

/* One item of a mixed batch: its own diffraction type and parameters (same Nx x Ny as the plan). */
typedef struct {
    double z;         /* distance, metres (non-zero for CWO_FRESNEL_CONV)           */
    double lambda;    /* wavelength, metres (> 0)                                   */
    double dx, dy;    /* sampling pitches, metres (> 0)                             */
    int type;         /* CWO_ANGULAR or CWO_FRESNEL_CONV                            */
    unsigned flags;   /* 0, or CWO_FLAG_LITERAL_SCALE for a Fresnel item            */
} cwo_item;

/*
 * Mixed batch: `batch` fields of the plan's Nx x Ny, item i propagated with items[i] (type,
 * distance, wavelength, pitches) -- the batching step of a serving loop that groups same-size
 * requests.  The plan supplies the shape, the scratch and the FFT tables; its own wavelength,
 * pitches, distance and type are not used.  items is a HOST array; the per-item
 * transfer-function tables are computed in FP64 on the host (in parallel threads) and uploaded
 * stream-ordered.  in_batch_stride as in cwo_propagate_batch but must be > 0.  Each contiguous
 * run of angular-spectrum items is one set of three launches; each contiguous run of Fresnel
 * items, the two separable line passes of a Fresnel plan (three launches instead when out is not
 * on a 16-byte boundary), so a caller that orders its batch by type makes at most five launches.
 * Results are bit-identical to running each item alone (no arithmetic depends on the batch).
 */
cwo_status cwo_propagate_items(cwo_plan* plan, const void* in, long long in_batch_stride, void* out,
                               int batch, const cwo_item* items, void* cuda_stream);

/* Adjoint propagation: the same passes with conj(H) (and conj(C)), i.e. the conjugate
 * transpose of the linear map cwo_propagate applies; for CWO_ANGULAR without evanescent bins
 * it equals back-propagation by -z (Section "Field type", back propagation of List
 * lst:conversion). */
cwo_status cwo_propagate_adjoint(cwo_plan* plan, const void* in_c64, void* out_c64, void* cuda_stream);

/* Batched adjoint, same argument rules as cwo_propagate_batch (in_batch_stride must be > 0). */
cwo_status cwo_propagate_adjoint_batch(cwo_plan* plan, const void* in, long long in_batch_stride,
                                       void* out, int batch, const double* z_or_null,
                                       void* cuda_stream);

/* Output epilogues, fused into the last pass of a propagation (the constraints of the
 * Gerchberg-Saxton iteration, Section "GS algorithm"; w is the propagated value of a pixel):
 *   CWO_EPI_NONE       out = w
 *   CWO_EPI_PHASE      out = w / |w|           phase constraint; a zero pixel becomes 1
 *   CWO_EPI_AMPLITUDE  out = a w / |w|         amplitude constraint with the pixel's a >= 0
 *   CWO_EPI_INTENSITY  intensity = |w|^2       reconstruction; out is not written */
typedef enum { CWO_EPI_NONE = 0, CWO_EPI_PHASE = 1, CWO_EPI_AMPLITUDE = 2, CWO_EPI_INTENSITY = 3 } cwo_epilogue;

/* One propagation of `batch` contiguous fields [batch][ny][nx] (forward, or the adjoint conj(H),
 * which for the angular spectrum method is the propagation by -z), followed by an epilogue.
 * amplitude (CWO_EPI_AMPLITUDE) and intensity (CWO_EPI_INTENSITY) are float [batch][ny][nx]
 * device buffers owned by the caller; out_c64 may be NULL with CWO_EPI_INTENSITY.  in and out may
 * alias.  Errors as cwo_propagate_batch; CWO_ERR_INVALID_ARG for a missing or short buffer. */
cwo_status cwo_propagate_epilogue(cwo_plan* plan, const void* in_c64, void* out_c64, int batch, int adjoint,
                                  int epilogue, const float* amplitude, float* intensity, void* cuda_stream);

/* Gerchberg-Saxton kinoform iteration (Section "GS algorithm") with an angular-spectrum plan of
 * distance z, on `batch` independent fields at once, all stream-ordered on cuda_stream:
 *   field <- phase(ASM(+z) field)                                    (the kinoform)
 *   repeat `iterations` times:
 *     field <- amplitude * phase(ASM(-z) field)                      (amplitude constraint)
 *     field <- phase(ASM(+z) field)                                  (phase constraint)
 *   intensity <- |ASM(-z) field|^2                                   (if intensity != NULL)
 * field_c64 (in: the object field, amplitude times its initial phase; out: the kinoform),
 * amplitude and intensity are [batch][ny][nx] device buffers of the caller.  Each propagation is
 * the three-pass path with the constraint fused into its last pass; up to nx = 1024 the field stays
 * in the plan's intermediate between propagations and one kernel turns from each propagation to
 * the next (inverse row pass, constraint, forward row pass: 4 launches per iteration, the same
 * values bit for bit), above it each propagation reads and writes the field (6 launches).
 * CWO_ERR_UNSUPPORTED for a Fresnel plan, CWO_ERR_INVALID_ARG for bad arguments. */
cwo_status cwo_gs_run(cwo_plan* plan, const float* amplitude, void* field_c64, float* intensity, int batch,
                      int iterations, void* cuda_stream);

/* Number of kernel launches one call of cwo_propagate_batch makes for this plan (for launch
 * accounting in benchmarks): 3 for the angular spectrum types, 2 for the Fresnel Fourier form and
 * for the Fresnel convolution and shifted Fresnel types, whose separable line passes take 2 (3
 * for an output epilogue, an output or a stack source not on a 16-byte boundary, a shifted
 * Fresnel z-stack, or a z-stack of padded rows longer than 4096). */
int cwo_launches_per_call(const cwo_plan* plan);

/* Synchronise the device and report whether any earlier call on this plan had a bounded wait
 * expire (CWO_ERR_TIMEOUT; the affected outputs were not written).  The waits guard asynchronous
 * copies into shared memory; expiry means the device stalled for seconds.  Clears the record. */
cwo_status cwo_plan_check(cwo_plan* plan);

/* Instrumentation: when `events` is non-NULL it must point to 4 cudaEvent_t (passed as void*)
 * created by the caller on the plan's device; every later call records events[0] before the row
 * forward pass, events[1] after it, events[2] after the column pass and events[3] after the row
 * inverse pass, on the call's stream, so that per-pass durations can be read with
 * cudaEventElapsedTime.  NULL switches recording off.  The caller keeps ownership of the events. */
cwo_status cwo_plan_set_timing_events(cwo_plan* plan, void* const* events);

/*
 * Angular-spectrum propagation of one [ny][nx] complex64 field that allocates no memory.
 * The paper has no counterpart: this serves callers that cannot allocate device memory when
 * they propagate -- a host that has given the device to its own allocator and forbids side
 * allocations, a real-time loop that must not risk the device synchronisation cudaMalloc can
 * imply, or code running where no allocator is available.  The caller passes only the input and
 * output fields (device memory of the current device; they may alias); the intermediate and the
 * tables live in file-scope device arrays of this library, which every GPU that loads it keeps
 * until the process exits.  Same method, conventions and accuracy as cwo_propagate with a
 * CWO_ANGULAR plan.
 *   limits   nx, ny powers of two in [16, 1024] (the fixed scratch is 1024 x 2048 complex64,
 *            16 MiB); larger fields return CWO_ERR_INVALID_ARG without launching anything
 *   errors   CWO_ERR_INVALID_ARG, before anything is enqueued, when a field is not 8-byte aligned
 *            device memory of the current device or its allocation ends before nx * ny complex64
 *            values; CWO_ERR_CUDA when a launch fails.  A bounded wait of the row passes that
 *            expires (an asynchronous copy that never lands) is not reported by this entry point:
 *            the output is then incomplete.  Each call clears that record before its passes.
 *   set-up   the first call on a device, with that device current, resolves the arrays'
 *            device addresses (cudaGetSymbolAddress); make that first call before any stream
 *            capture
 *   sharing  all calls use the same arrays, which keep the last call's contents; calls whose
 *            work overlaps on the GPU (other streams or host threads) race and corrupt each
 *            other.  Nothing has to start at zero: each call regenerates every table entry and
 *            writes every intermediate element before it is read.
 *   ordering enqueued on cuda_stream; no host synchronisation; allocates nothing.
 */
cwo_status cwo_propagate_asm_noalloc(int nx, int ny, double dx, double dy, double lambda, double z,
                                     const void* in_c64, void* out_c64, void* cuda_stream);

/* Thread-local description of the most recent failure on this thread ("" if none). */
const char* cwo_last_error(void);

/* Library version, major * 10000 + minor * 100 + patch. */
int cwo_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CWO_H */
