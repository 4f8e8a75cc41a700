// cwo_tma.cuh -- Tensor Memory Accelerator copies between the column-major intermediate and a
// dense shared-memory tile, and the bounded mbarrier wait that guards them.
//
// The intermediate [items][Px][Ny] complex64 is described by a rank-3 tensor map whose dimensions
// are (Ny, Px, items) innermost first, with 8-byte elements; a box is R rows (inner) by up to 256
// storage columns by 1 item, i.e. R * 8 contiguous bytes per column.  The first box coordinate is
// the row y0, a multiple of R >= 2, so it always starts on a 16-byte boundary, and no coordinate
// is ever negative or out of range.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace cwo {

constexpr int kTmaBoxCols = 256;                 // storage columns per TMA box
constexpr unsigned kMbarSpinLimit = 1u << 24;   // try_wait iterations before a wait gives up
constexpr int kStatusTimeout = 1;               // status-word bit: a bounded wait expired

#ifdef __CUDACC__
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, const void* src, int c0, int c1, int c2) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];"
                 :: "l"(map), "r"(smem_u32(src)), "r"(c0), "r"(c1), "r"(c2) : "memory");
}
__device__ __forceinline__ void tma_store_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the shared-memory sources of every committed store have been read (the tile may be rewritten)
__device__ __forceinline__ void tma_store_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// the same for every committed store but the most recent group
__device__ __forceinline__ void tma_store_wait_read_1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void tma_store_commit_and_drain() {
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// writes of the generic proxy to shared memory become visible to TMA (async proxy) reads
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* mbar, int c0, int c1, int c2) {
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
                 :: "r"(smem_u32(dst)), "l"(map), "r"(smem_u32(mbar)), "r"(c0), "r"(c1), "r"(c2) : "memory");
}
// contiguous global -> shared copy (both addresses 16-byte aligned, bytes a multiple of 16)
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(mbar)) : "memory");
}
// thread-block clusters: rank, addresses in another CTA's shared memory, stores there, barrier
__device__ __forceinline__ unsigned cluster_ctarank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_map(unsigned smem_addr, unsigned rank) {
    unsigned out;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(smem_addr), "r"(rank));
    return out;
}
__device__ __forceinline__ void st_cluster(unsigned addr, float2 v) {
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" :: "r"(addr), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void st_cluster4(unsigned addr, float4 v) {   // addr 16-byte aligned
    asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" :: "r"(addr), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}
// every thread of every CTA of the cluster arrives; release / acquire order the shared-memory
// accesses before and after it across the cluster
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// generic-proxy writes to (any CTA's) shared memory become visible to TMA reads
__device__ __forceinline__ void fence_proxy_async_cluster() { asm volatile("fence.proxy.async.shared::cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* mbar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(mbar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* mbar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_u32(mbar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* mbar, unsigned parity) {
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(smem_u32(mbar)), "r"(parity) : "memory");
    return ok != 0;
}
// Wait for phase `parity` of the barrier with an iteration limit.  On expiry the status word gets
// kStatusTimeout, the thread keeps waiting (again bounded) so that copies still in flight land
// before the block can exit, and false is returned: the caller must not use the data.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* mbar, unsigned parity, int* status,
                                                  unsigned limit = kMbarSpinLimit) {
    for (unsigned i = 0; i < limit; ++i)
        if (mbar_try_wait(mbar, parity)) return true;
    if (status) atomicOr(status, kStatusTimeout);
    for (unsigned i = 0; i < limit; ++i)
        if (mbar_try_wait(mbar, parity)) break;
    return false;
}
#endif  // __CUDACC__

}  // namespace cwo
