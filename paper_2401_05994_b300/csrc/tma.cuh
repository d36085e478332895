// Tensor-memory-accelerator (TMA) copies and shared-memory barriers, in
// inline PTX for sm_103a (device side), and the host-side encoding of tensor
// maps.  Used by the strided restriction-and-solve pass to stage tiles of
// lines in shared memory without the threads issuing the copies.
#pragma once

#include <cuda.h>
#include <stdint.h>

#include "common.cuh"

namespace mgb {

__device__ inline uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// A barrier that completes one phase when its single arrival (with the
// expected byte count) and the announced bytes have landed.
__device__ inline void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}

// Make initialized barriers visible to the copy engine.
__device__ inline void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ inline void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// Wait for the phase of parity `parity` to complete, at most `max_iter`
// polls; false if it did not.
__device__ inline bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t max_iter) {
    const uint32_t a = smem_u32(bar);
    for (uint32_t it = 0; it < max_iter; ++it) {
        uint32_t done;
        asm volatile(
            "{\n"
            ".reg .pred p;\n"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n"
            "}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// One box of a 3D tensor map at element coordinates (x, y, z) into shared
// memory, completing on `bar`.  x times the element size must be a multiple
// of 16 bytes; y and z may lie outside the tensor (those elements read 0).
__device__ inline void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                   uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// Host: a tiled 3D tensor map over `base` (dims innermost first, strides in
// bytes of dims 1 and 2, box extents), float or double elements, zero fill
// outside.  MGARD_EINVAL if the driver rejects it (alignment, extents).
mgard_status encode_tensor_map_3d(CUtensorMap* map, const void* base, int elem_bytes,
                                  const uint64_t dims[3], const uint64_t strides[2],
                                  const uint32_t box[3]);

}  // namespace mgb
