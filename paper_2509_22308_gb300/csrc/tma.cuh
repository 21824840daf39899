// Tensor Memory Accelerator (TMA) tile loads into shared memory and the mbarrier waits
// that go with them (inline PTX, sm_90 and later; used here for sm_103a).
//
// A load is one cp.async.bulk.tensor of a box described by a CUtensorMap (built on the
// host by cuTensorMapEncodeTiled); the copy engine signals its completion on an mbarrier
// in shared memory through the transaction count (complete_tx::bytes).  Every wait is
// bounded: it gives up after a number of clock cycles and the caller reports the timeout
// through the handle's error word instead of spinning forever.
#pragma once

#include <cuda.h>
#include <stdint.h>

namespace lbmem {

// About one second at GB300's clocks: far above any healthy wait for one tile.
constexpr long long kWaitCycles = 2000000000LL;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Makes initialised barriers visible to the copy engine (the async proxy).
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders shared-memory accesses of the generic proxy (the block's reads of a buffer,
// made visible to this thread by a barrier) before a later copy into the same buffer.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// A tensor map kept in global memory (a table of them, one per batched instance) is read
// by the copy engine through the tensor-map proxy, which caches descriptors by address: an
// entry left from an earlier map at the same address (a freed and reallocated table) would
// otherwise be used in place of the one the host has since copied there.  The thread that
// issues copies with the map acquires it first; maps passed as __grid_constant__ kernel
// parameters need no fence.
__device__ __forceinline__ void tmap_acquire(const CUtensorMap *map) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"((uint64_t)map) : "memory");
}

// One arrival that also expects `bytes` of transactions in the current phase.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Box of a rank-3 tensor map at element coordinates (x, y, z) into shared memory at dst
// (128-byte aligned), completing on bar.  x * element size must be a multiple of 16
// bytes; coordinates outside the tensor read as zero.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// Box of a rank-2 tensor map at element coordinates (x, y); same rules as tma_load_3d.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// `bytes` contiguous bytes from global memory (16-byte aligned, a multiple of 16) into
// shared memory (16-byte aligned), completing on bar (a non-tensor bulk copy).
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"((uint64_t)src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits until the phase with the given parity has completed; false once about `limit`
// clock cycles have passed without it.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, long long limit = kWaitCycles) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

}  // namespace lbmem
