// cwo_internal.h -- structures shared by the host plan code and the kernel launchers.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace cwo {

enum HMode : int {
    HMODE_ASM_POLY = 0,      // ASM, FP64-reduced per-axis phase, float-float cross, series tail
    HMODE_ASM_EXACT = 1,     // ASM, as above with the closed-form tail (larger s)
    HMODE_ASM_FP32 = 2,      // ASM, whole phase in FP32 (precision-study arm)
    HMODE_ASM_FP64 = 3,      // ASM, literal per-element FP64 phase (reference arm, large K s^3)
    HMODE_FRESNEL = 4,       // Fresnel, separable table product
    HMODE_TABLE = 5,         // ASM transfer function materialised per plan ("once-calculation")
};

// Per-item parameters of a mixed batch (cwo_propagate_items): the item's transfer-function mode
// and the scalars its per-element evaluation needs.  Its tables are float4 rows of the per-item
// x/y tables (Fresnel items use .x, .y).
struct ItemParams {
    int mode;                 // HMode of this item
    float kf;                 // K = z / lambda (series / closed-form tail)
    double K, sx, sy;         // FP64 per-element arm
};

// Transfer-function description for the column pass.  Per-axis tables are indexed by the axis
// index idx = e * T + t (register e of thread t in the last forward stage, i.e. DIF position
// 16 t + e); along x the same index is the storage column of the intermediate.
struct HParams {
    int mode;                 // HMode
    int conj;                 // 1: adjoint (conj H)
    // ASM reduced: float4 {a = lambda^2 f^2, W = frac(K(a/2 + a^2/8)) [- frac(K) on x], u_hi, u_lo}
    // with K = z / lambda and u_hi + u_lo = sqrt(K/4) a; K is folded into the tables.
    const float4* ax;
    const float4* ay;
    // Fresnel: float2 per-axis DFTs of the sampled chirp (x table includes C)
    const float2* hx;
    const float2* hy;
    long long x_item_stride;  // elements between items' x tables (0: shared)
    long long y_item_stride;
    const float* kf;          // ASM reduced: K = z / lambda per item (for the O(s^3) tail term)
    long long kf_item_stride; // 0: shared
    double K;                 // z / lambda                       (FP64 arm)
    double sx, sy;            // lambda^2 / (P dx)^2, (P dy)^2    (FP64 arm)
    double z, k;              // distance and wavenumber 2 pi / lambda   (FP32 arm)
    double dfx, dfy;          // frequency pitches 1 / (P dx), 1 / (P dy) (FP32 arm)
    const int* kbx;           // signed bin of each axis index (FP32 / FP64 arms)
    const int* kby;
    // storage-column pairs (st(+kx), st(-kx)) for kx = 0 .. Px/2 (paired column kernel)
    const int2* pairs;
    int npairs;               // Px/2 + 1
    // mixed batch: per-item modes and scalars (nullptr: the launch-wide fields above apply);
    // the tables are then ax / ay (float4) with x_item_stride / y_item_stride for every mode
    const ItemParams* items;
    // shifted ASM: tables not symmetric in kx (single-column kernel); for the per-element FP64
    // evaluation the shift in cycles per signed bin and the signed-bin window [lo, hi]
    int asym;
    double shx, shy;
    int wxlo, wxhi, wylo, wyhi;
    // HMODE_TABLE: H of mirror pair j = |kt_x| at axis index i along y is hcache[j * py + i]
    const float2* hcache;
    long long hcache_stride;
    // HMODE_TABLE at Py = 8192 (k_col_split): the twiddle table of the 4096-point transform and
    // W_8192^n for n < 4096; the hcache rows are then in the split order (index h 4096 + e 256 + t
    // holds frequency 2 k + h, k the 4096-point frequency of register e of thread t)
    const float4* split_tw;
    const float2* split_w;
};

// launchers (return cudaGetLastError() after the launch)
// Record the message returned by cwo_last_error() on this thread.
void set_last_error(const char* msg);
// Check that [ptr, ptr + bytes) is 8-byte aligned device (or managed) memory of `device` inside
// one allocation (cuMemGetAddressRange); returns a cwo_status and sets the error message.
int check_device_buffer(const void* ptr, size_t bytes, int device, const char* name);

// The intermediate is column-major: [items][Px][Ny] complex64 (see cwo_rows.cu).
// The row passes reach the intermediate through rank-3 TMA tensor maps (Ny, Px, items) with
// boxes of row_block_rows(px, inverse) rows x min(256, Px) columns (one map per pass);
// item_off is added to the item index.
int row_block_rows(int px, bool inverse);

// output epilogue of the inverse row pass (see cwo_rows.cu); amp / inten are [items][Ny][Nx]
//   EPI_SEPARABLE: out = w * qx[x] * qy[y] (x, y the output column and row; shifted Fresnel)
enum EpiMode { EPI_NONE = 0, EPI_PHASE = 1, EPI_AMPLITUDE = 2, EPI_INTENSITY = 3, EPI_SEPARABLE = 4 };
struct Epilogue {
    int mode = EPI_NONE;
    const float* amp = nullptr;
    float* inten = nullptr;
    const float2* qx = nullptr;
    const float2* qy = nullptr;
};
// optional separable factor of the source, applied as the forward row pass loads it:
// u(x, y) * fx[x] * fy[y] (shifted Fresnel); both null: none
struct Prefactor {
    const float2* fx = nullptr;
    const float2* fy = nullptr;
};
cudaError_t launch_row_fwd(int px, const float2* in, long long in_item_stride, const CUtensorMap* wmap,
                           int item_off, int ny, int items, const float4* tw, int* status, cudaStream_t st,
                           const Prefactor& pre = Prefactor());
cudaError_t launch_row_inv(int px, const CUtensorMap* wmap, int item_off, float2* out, long long out_item_stride,
                           int ny, int items, float scale, const float4* tw, int* status, cudaStream_t st,
                           const Epilogue& ep = Epilogue());
// The inverse row pass with an EPI_PHASE or EPI_AMPLITUDE constraint followed by the forward row
// pass of the next propagation, in place on the intermediate through `wmap` (the forward pass's
// map); field_item_stride indexes the constraint's amplitude [items][Ny][Nx].  64 <= Px <= 4096 (row_turn_supported: up to 2048).
bool row_turn_supported(int px);
cudaError_t launch_row_turn(int px, const CUtensorMap* wmap, int ny, int items, long long field_item_stride, float scale,
                            const float4* tw, int* status, const Epilogue& ep, cudaStream_t st);
// column pass of a shared-source z-stack: one forward transform per column, `planes` outputs
cudaError_t launch_col_stack(int py, const float2* win, float2* wout, long long wout_item_stride, int px, int planes,
                             const float4* tw, const HParams& hp, cudaStream_t st);
// Materialise the ASM transfer function of hp (modes POLY, EXACT, FP32, FP64 with the plan's
// own tables) for every mirror pair j = 0 .. npairs-1 and axis index i < py: out[j * py + i],
// evaluated by the same device functions as the column pass; with yidx (device, py entries),
// entry i is evaluated at y axis index yidx[i] (the split order of k_col_split).
cudaError_t launch_build_hcache(float2* out, int npairs, int py, const HParams& hp, cudaStream_t st,
                                const int* yidx = nullptr);
// Py of the split column pass (a transfer function cached per plan)
constexpr int kSplitColP = 8192;
// Fresnel diffraction in Fourier form (cwo_fourier.cu): source chirp + row FFT into the
// [items][Px = Nx][Ny] intermediate; column FFT + destination chirp into the centred output
// separable Fresnel line pass (cwo_lines.cu): `lines` lines of P/2 contiguous samples per item,
// optionally multiplied by pre[position], expanded to P, convolved through the axis table h (DIF
// order, P entries per item), scaled, optionally multiplied by post[position], and stored
// transposed through omap (dims: lines, P/2 positions, items; boxes of line_block_rows(P) lines).
// pre and post: both or neither.
int line_block_rows(int p);
// first pass of a shared-source z-stack: `lines` source lines (one item) transformed once and
// stored per plane j (item j of omap) after the multiply by h + j * h_item_stride; 512 <= p <= 4096
// and a 16-byte aligned source
bool line_stack_supported(int p);
cudaError_t launch_line_stack(int p, const float2* in, const CUtensorMap* omap, int lines, int planes, const float2* h,
                              long long h_item_stride, int conj, float scale, const float4* tw, int* status,
                              cudaStream_t st);
cudaError_t launch_line_conv(int p, const float2* in, long long in_item_stride, const CUtensorMap* omap, int lines,
                             int items, const float2* h, long long h_item_stride, int conj, float scale,
                             const float4* tw, int* status, const float2* pre, const float2* post, cudaStream_t st);
cudaError_t launch_fourier_rows(int px, const float2* in, long long in_item_stride, const CUtensorMap* wmap, int ny,
                                int items, const float2* pre_x, const float2* pre_y, const float4* tw, cudaStream_t st);
cudaError_t launch_fourier_cols(int py, const float2* win, long long win_item_stride, float2* out, long long out_item_stride,
                                int nx, int items, const int* st_of_col, const int* row_of_idx, const float2* post_x,
                                const float2* post_y, const float4* tw, cudaStream_t st);
// copy `fields` (<= kCopyMaxFields) fields of `elems` complex64 values from list.src[i] to
// list.dst[i] (device addresses; a NULL address skips item i) -- the serving runtime's gather
// and scatter
constexpr int kCopyMaxFields = 64;
struct CopyList {
    const float2* src[kCopyMaxFields];
    float2* dst[kCopyMaxFields];
};
cudaError_t launch_copy_fields(const CopyList& list, int fields, long long elems, cudaStream_t st);
// Encode the tensor map of an intermediate [cap][px][ny] at base (host only; no allocation).
cudaError_t make_intermediate_map(CUtensorMap* map, void* base, int ny, int px, int cap, int rows);
cudaError_t launch_col(int py, const float2* win, long long win_item_stride, float2* wout,
                       long long wout_item_stride, int px, int items, const float4* tw,
                       const HParams& hp, cudaStream_t st);

}  // namespace cwo
