// flb_tma.cuh -- tensor-memory-accelerator (TMA) tile loads and mbarrier waits
// for sm_100-class GPUs, written as inline PTX.
//
// A tile load is issued by one thread: cp.async.bulk.tensor copies a box of a
// tiled global tensor (described by a CUtensorMap kernel parameter) into shared
// memory and signals completion of its bytes on an mbarrier; consumers wait on
// the barrier's phase.  Every wait is bounded: after FLB_WAIT_LIMIT polls it
// gives up, records FLB_ETIMEOUT in the caller's status word and reports
// failure, so a lost copy can never hang the GPU.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace flb {

constexpr uint32_t FLB_WAIT_LIMIT = 1u << 20;  // polls of ~0.1-1 us each: about a second at most

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// release the barrier object (before the location is initialised again)
__device__ __forceinline__ void mbar_inval(uint64_t *bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// make barrier initialisation visible to the async (TMA) proxy
__device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// order earlier generic-proxy accesses of shared memory before later TMA writes
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// true once the phase with the given parity has completed
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait; on timeout sets *status (if given) and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *status)
{
    for (uint32_t i = 0; i < FLB_WAIT_LIMIT; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    if (status) atomicExch(status, -5);  // FLB_ETIMEOUT
    return false;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
        "[%2];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z,
                                            int w)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6}], "
        "[%2];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z), "r"(w)
        : "memory");
}

// Host: encode a tiled FP32 tensor map (dims and box innermost first, strides in
// bytes for dims 1..rank-1).  Returns cudaErrorNotSupported if the driver entry
// point is unavailable.
cudaError_t encode_tensor_map_f32(CUtensorMap *map, const void *base, int rank, const uint64_t *dims,
                                  const uint64_t *strides_bytes, const uint32_t *box);

}  // namespace flb
