// cwo_rows.cu -- entry points of the row passes: the tensor maps of the intermediate, the
// forward row pass and the size dispatch of the inverse (cwo_rows_inv_a/b.cu); the kernels are
// in cwo_rows.cuh.
#include "cwo_rows.cuh"

namespace cwo {

#define CWO_P_CASES(X) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096) X(8192)

typedef CUresult (*PFN_tensorMapEncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                              CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                              CUtensorMapFloatOOBfill);

static PFN_tensorMapEncodeTiled encode_fn() {
    static PFN_tensorMapEncodeTiled fn = nullptr;
    static bool tried = false;
    if (!tried) {   // resolved through the runtime: no link-time dependency on libcuda
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_tensorMapEncodeTiled)p;
        tried = true;
    }
    return fn;
}

cudaError_t make_intermediate_map(CUtensorMap* map, void* base, int ny, int px, int cap, int rows) {
    PFN_tensorMapEncodeTiled fn = encode_fn();
    const int R = rows;
    if (!fn || R < 2 || cap < 1 || ny % R) return cudaErrorInvalidValue;
    const cuuint64_t dims[3] = {(cuuint64_t)ny, (cuuint64_t)px, (cuuint64_t)cap};
    const cuuint64_t strides[2] = {(cuuint64_t)ny * sizeof(float2), (cuuint64_t)ny * px * sizeof(float2)};
    const cuuint32_t box[3] = {(cuuint32_t)R, (cuuint32_t)(px < kTmaBoxCols ? px : kTmaBoxCols), 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, base, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

int row_block_rows(int px, bool inverse) {
    switch (px) {
#define CASE(P) case P: return inverse ? rows_inv<P>() : rows_fwd<P>();
        CWO_P_CASES(CASE)
#undef CASE
        default: return 0;
    }
}

cudaError_t launch_row_fwd(int px, const float2* in, long long in_item_stride, const CUtensorMap* wmap,
                           int item_off, int ny, int items, const float4* tw, int* status, cudaStream_t st,
                           const Prefactor& pre) {
    switch (px) {
#define CASE(P) case P: return row_fwd_impl<P>(in, in_item_stride, wmap, item_off, ny, items, tw, status, pre, st);
        CWO_P_CASES(CASE)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_row_inv_a(int px, const CUtensorMap* wmap, int item_off, float2* out, long long out_item_stride,
                             int ny, int items, float scale, const float4* tw, int* status, cudaStream_t st,
                             const Epilogue& ep);
cudaError_t launch_row_inv_b(int px, const CUtensorMap* wmap, int item_off, float2* out, long long out_item_stride,
                             int ny, int items, float scale, const float4* tw, int* status, cudaStream_t st,
                             const Epilogue& ep);

cudaError_t launch_row_inv(int px, const CUtensorMap* wmap, int item_off, float2* out, long long out_item_stride,
                           int ny, int items, float scale, const float4* tw, int* status, cudaStream_t st,
                           const Epilogue& ep) {
    return px <= 1024 ? launch_row_inv_a(px, wmap, item_off, out, out_item_stride, ny, items, scale, tw, status, st, ep)
                      : launch_row_inv_b(px, wmap, item_off, out, out_item_stride, ny, items, scale, tw, status, st, ep);
}


}  // namespace cwo

// ------------------------------------------------------------------------------------------
// Failure-path check of the bounded wait: one thread initialises an mbarrier for one arrival and,
// unless `complete` is set, never arrives, so phase 0 never completes (a flag nothing sets); the
// wait must give up after `limit` polls, set the timeout bit in the status word and return.
// ------------------------------------------------------------------------------------------
namespace {
__global__ void k_debug_bounded_wait(unsigned limit, int complete, int* status) {
    __shared__ __align__(8) uint64_t mbar;
    cwo::mbar_init(&mbar, 1);
    if (complete) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(cwo::smem_u32(&mbar)) : "memory");
    cwo::mbar_wait_bounded(&mbar, 0, status, limit);
}

cwo_status debug_fail(cwo_status st, const char* msg) {
    cwo::set_last_error(msg);
    return st;
}
}  // namespace

extern "C" cwo_status cwo_debug_bounded_wait(unsigned spin_limit, int complete, int* status_out) {
    if (!status_out) return debug_fail(CWO_ERR_INVALID_ARG, "status_out is NULL");
    if (spin_limit < 1 || spin_limit > (1u << 20)) return debug_fail(CWO_ERR_INVALID_ARG, "spin_limit must be in [1, 2^20]");
    int* d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(d, 0, sizeof(int));
    if (e == cudaSuccess) {
        k_debug_bounded_wait<<<1, 1>>>(spin_limit, complete, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(status_out, d, sizeof(int), cudaMemcpyDeviceToHost);
    if (d) cudaFree(d);
    if (e != cudaSuccess) return debug_fail(CWO_ERR_CUDA, cudaGetErrorString(e));
    return CWO_OK;
}
