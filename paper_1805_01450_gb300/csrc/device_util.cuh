// Device helpers shared by the kernel files: bit-run address maps, leaf restriction,
// shared-memory addresses, bulk asynchronous copies and bounded mbarrier waits.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "device_program.h"

namespace qvx {

__device__ __forceinline__ uint32_t pext_runs(uint32_t c, const DevRun *runs, int n) {
    uint32_t r = 0;
    for (int i = 0; i < n; i++) r |= ((c >> runs[i].src) & ((1u << runs[i].len) - 1u)) << runs[i].dst;
    return r;
}


// First stored entry of `leaf` restricted to this work item (bitstring x, outer slice o).
__device__ __forceinline__ uint32_t leaf_base(const DevLeaf &L, uint64_t x, uint64_t o) {
    uint32_t off = L.data_off;
    for (uint32_t f = 0; f < L.n_fixed; f++) {
        const uint32_t src = L.fixed_src[f];
        const uint64_t bit = src < 64 ? (x >> src) & 1ull : (o >> (src - 64)) & 1ull;
        off += (uint32_t)bit << L.fixed_pos[f];
    }
    return off;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Bulk asynchronous copy (TMA engine) of `bytes` (a multiple of 16, both addresses 16-byte
// aligned) from global to shared memory, completing on the mbarrier at `bar`.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Waits for phase `parity` of the mbarrier, giving up after `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t limit) {
    for (uint32_t i = 0; i < limit; i++) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

}  // namespace qvx
