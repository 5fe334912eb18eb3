// TMA (cp.async.bulk.tensor) and mbarrier helpers in inline PTX, and the
// host-side tensor-map encoder (driver entry point, no libcuda link).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace pcot {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity to complete.  Gives up
// after `timeout_ns` (or at once when the status block already holds an
// error), records kStatusTimeout and returns false; it never spins forever.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity, DevStatus* st, uint64_t timeout_ns,
                                          int where) {
    if (mbar_try_wait(b, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (;;) {
        if (mbar_try_wait(b, parity)) return true;
        const bool failed = *((volatile int*)&st->abort) != 0;
        if (failed || globaltimer_ns() - t0 > timeout_ns) {
            if (atomicCAS(&st->code, 0, kStatusTimeout) == 0) st->info[2] = where;
            atomicExch(&st->abort, 1);
            return false;
        }
    }
}

// 2-D tiled bulk tensor load into shared memory, completion counted in bytes
// on the mbarrier.  x must be a multiple of 16 bytes / element size.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Orders this thread's later async-proxy (TMA) reads of global memory after
// generic-proxy writes it has observed (other CTAs' tile outputs).
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Before the first use of a tensor map that lives in global memory and was
// written through the generic proxy (a copy from the host): makes the
// tensormap proxy observe that content rather than a descriptor cached for
// the same address by an earlier launch.
__device__ __forceinline__ void fence_tensormap_acquire(const void* map) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"((uint64_t)map) : "memory");
}

// Host: encode a 2-D row-major tensor map (innermost dimension first).
// Returns false if the driver entry point is unavailable or encoding fails.
bool encode_tmap_2d(CUtensorMap* map, const void* base, int elem_bytes, uint64_t width, uint64_t height,
                    uint64_t pitch_bytes, uint32_t box_w, uint32_t box_h);

}  // namespace pcot
