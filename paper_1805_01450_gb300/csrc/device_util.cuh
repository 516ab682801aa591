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


// A bitstring of up to 128 qubits: bit q is bit q % 64 of word q / 64 (word 1 is zero for
// n_qubits <= 64, whose bitstrings are one word each).
struct Bits {
    uint64_t w0, w1;
};

__device__ __forceinline__ Bits load_bits(const uint64_t *bitstrings, int64_t b, uint32_t words) {
    Bits x;
    x.w0 = bitstrings[b * words];
    x.w1 = words > 1 ? bitstrings[b * words + 1] : 0ull;
    return x;
}

// Nonzero when a qubit without a non-diagonal gate (its output equals its input 0) is 1 in x.
__device__ __forceinline__ bool bits_hit(const Bits &x, uint64_t mask_lo, uint64_t mask_hi) {
    return ((x.w0 & mask_lo) | (x.w1 & mask_hi)) != 0ull;
}

// First stored entry of `leaf` restricted to this work item (bitstring x, outer slice o).
// The leaf is read as five 8-byte words (data offset, fixed-mode count, the packed source
// and position bytes) and the up to 12 fixed modes are applied without a loop-carried branch:
// a source below 64 is a bit of bitstring word 0, below 128 one of word 1, else a bit of o.
__device__ __forceinline__ uint32_t leaf_base(const DevLeaf &L, const Bits &x, uint64_t o) {
    static_assert(sizeof(DevLeaf) == 40 && kMaxFixed == 12, "DevLeaf layout");
    const uint2 *w = reinterpret_cast<const uint2 *>(&L);
    const uint2 w0 = w[0], w1 = w[1], w2 = w[2], w3 = w[3], w4 = w[4];
    const uint32_t srcw[3] = {w2.x, w2.y, w3.x}, posw[3] = {w3.y, w4.x, w4.y};
    const uint32_t nf = w1.x;
    uint32_t off = w0.x;
#pragma unroll
    for (uint32_t f = 0; f < (uint32_t)kMaxFixed; f++) {
        if (f < nf) {
            const uint32_t src = (srcw[f >> 2] >> (8u * (f & 3u))) & 0xffu;
            const uint32_t pos = (posw[f >> 2] >> (8u * (f & 3u))) & 0xffu;
            const uint64_t v = src < 64u ? x.w0 : (src < 128u ? x.w1 : o);
            off += (uint32_t)((v >> (src & 63u)) & 1ull) << pos;
        }
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
