// Dense contractions on the tcgen05 tensor cores (stepwise engine, opts.tensor_cores).
//
// A step C[b, m, n] = sum_k A[b, m, k] B[b, k, n] in complex64 becomes one real GEMM per
// (work item, b): with A = Ar + i Ai and B = Br + i Bi, the rows 2m and 2m + 1 of
//   [Ar  -Ai]        [Br]
//   [Ai   Ar]  times [Bi]
// are Re C[m, :] and Im C[m, :]. Every real operand x is split as x = hi + lo with hi, lo in
// bf16, and the three products hi*hi + hi*lo + lo*hi are taken as one GEMM over a summed
// index three times as long: A' = [Ah | Ah | Al], B' = [Bh ; Bl ; Bh] (the lo*lo term,
// below 2^-16 of the product, is dropped). The pack kernels write A' and B' in the tensor
// cores' K-major core-matrix layout, one tile per (item, b, row or column tile, summed chunk);
// the GEMM kernel copies those tiles into shared memory with bulk asynchronous copies, issues
// tcgen05.mma (bf16 inputs, FP32 accumulator in tensor memory) from one thread, and its four
// warps read the accumulator back with tcgen05.ld and store complex64 C in its own layout.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "device_program.h"
#include "device_util.cuh"
#include "kernels.h"

namespace qvx {
namespace {

constexpr int kGemmRows = 128;      // real rows per tile (64 complex rows)
constexpr int kGemmStages = 3;      // shared-memory ring of summed-index chunks
constexpr uint32_t kGemmPolls = 1u << 22;

__device__ __forceinline__ const float2 *gemm_operand(const LaunchArgs &a, const float2 *arena, uint64_t ref,
                                                      bool leaf, int64_t item) {
    if (!leaf) return arena + ref;
    const unsigned char *img = a.image;
    const DevProgram *P = reinterpret_cast<const DevProgram *>(img);
    const DevLeaf *leaves = reinterpret_cast<const DevLeaf *>(img + P->leaves_off);
    const float2 *ldata = reinterpret_cast<const float2 *>(img + P->leaf_data_off);
    const uint64_t x = a.bitstrings[item / a.o_count];
    const uint64_t o = (uint64_t)(a.o_begin + item % a.o_count);
    return ldata + leaf_base(leaves[ref], x, o);
}

// Byte offset of element (row r, summed index j) inside a tile of `kc` summed entries:
// 8-row x 16-byte core matrices, those of one 8-row group contiguous along j.
__device__ __forceinline__ uint32_t core_offset(uint32_t r, uint32_t j, uint32_t kc) {
    return (r >> 3) * (kc * 16u) + (j >> 3) * 128u + (r & 7u) * 16u;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo_half, float hi_half) {
    const __nv_bfloat16 a = __float2bfloat16_rn(lo_half), b = __float2bfloat16_rn(hi_half);
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// Part `lo` (0: hi, 1: lo) of the bf16 split of v.
__device__ __forceinline__ float split_part(float v, int lo) {
    const float h = __bfloat162float(__float2bfloat16_rn(v));
    return lo ? v - h : h;
}

// A' for items [item0, item0 + n): one thread per 8 consecutive summed entries of one row.
__global__ void pack_a_kernel(LaunchArgs a, GemmStep g, int64_t item0, int64_t n_items, const float2 *arenas,
                              unsigned char *Ap, uint32_t kc) {
    const uint32_t M2 = 2u << g.nm, K = 1u << g.nk, Kp = 6u * K;
    const uint64_t units = (uint64_t)M2 * (Kp / 8u);
    const uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= ((uint64_t)n_items << g.nb) * units) return;
    const uint64_t ib = u / units;                 // (item, b)
    const uint32_t v = (uint32_t)(u - ib * units);
    const uint32_t r = v % M2, q = v / M2;
    const int64_t il = (int64_t)(ib >> g.nb);
    const uint32_t beta = (uint32_t)(ib & ((1u << g.nb) - 1u));
    const uint32_t m = r >> 1, s = r & 1u;
    const uint32_t j0 = 8u * q, seg = j0 / (2u * K), w = j0 % (2u * K), part = w / K, k0 = w % K;
    const float2 *A = gemm_operand(a, arenas + (uint64_t)il * a.arena_elems, g.a_off, g.flags & kStepALeaf,
                                   item0 + il);
    A += pext_runs(beta, g.ab, g.n_ab) + pext_runs(m, g.am, g.n_am);
    float val[8];
#pragma unroll
    for (int t = 0; t < 8; t++) {
        const float2 x = A[pext_runs(k0 + t, g.ak, g.n_ak)];
        const float e = s == 0 ? (part == 0 ? x.x : -x.y) : (part == 0 ? x.y : x.x);
        val[t] = split_part(e, seg == 2);
    }
    const uint32_t n_mt = M2 / kGemmRows, n_kc = Kp / kc;
    const uint64_t tile = ((ib * n_mt + r / kGemmRows) * n_kc + j0 / kc) * (uint64_t)(kGemmRows * kc * 2u);
    uint4 out;
    out.x = pack_bf16x2(val[0], val[1]);
    out.y = pack_bf16x2(val[2], val[3]);
    out.z = pack_bf16x2(val[4], val[5]);
    out.w = pack_bf16x2(val[6], val[7]);
    *reinterpret_cast<uint4 *>(Ap + tile + core_offset(r % kGemmRows, j0 % kc, kc)) = out;
}

// B' for items [item0, item0 + n): one thread per 8 consecutive summed entries of one column.
__global__ void pack_b_kernel(LaunchArgs a, GemmStep g, int64_t item0, int64_t n_items, const float2 *arenas,
                              unsigned char *Bp, uint32_t kc, uint32_t nt_cols) {
    const uint32_t N = 1u << g.nn, K = 1u << g.nk, Kp = 6u * K;
    const uint64_t units = (uint64_t)N * (Kp / 8u);
    const uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= ((uint64_t)n_items << g.nb) * units) return;
    const uint64_t ib = u / units;
    const uint32_t v = (uint32_t)(u - ib * units);
    const uint32_t n = v % N, q = v / N;
    const int64_t il = (int64_t)(ib >> g.nb);
    const uint32_t beta = (uint32_t)(ib & ((1u << g.nb) - 1u));
    const uint32_t j0 = 8u * q, seg = j0 / (2u * K), w = j0 % (2u * K), part = w / K, k0 = w % K;
    const float2 *B = gemm_operand(a, arenas + (uint64_t)il * a.arena_elems, g.b_off, g.flags & kStepBLeaf,
                                   item0 + il);
    B += pext_runs(beta, g.bb, g.n_bb) + pext_runs(n, g.bn, g.n_bn);
    float val[8];
#pragma unroll
    for (int t = 0; t < 8; t++) {
        const float2 x = B[pext_runs(k0 + t, g.bk, g.n_bk)];
        val[t] = split_part(part == 0 ? x.x : x.y, seg == 1);
    }
    const uint32_t n_nt = N / nt_cols, n_kc = Kp / kc;
    const uint64_t tile = ((ib * n_nt + n / nt_cols) * n_kc + j0 / kc) * (uint64_t)(nt_cols * kc * 2u);
    uint4 out;
    out.x = pack_bf16x2(val[0], val[1]);
    out.y = pack_bf16x2(val[2], val[3]);
    out.z = pack_bf16x2(val[4], val[5]);
    out.w = pack_bf16x2(val[6], val[7]);
    *reinterpret_cast<uint4 *>(Bp + tile + core_offset(n % nt_cols, j0 % kc, kc)) = out;
}

// Shared-memory matrix descriptor of a K-major tile without swizzling: start address, the
// byte distance between core matrices along the summed index (lbo) and between 8-row groups
// (sbo), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

struct GemmArgs {
    LaunchArgs a;
    GemmStep g;
    int64_t item0, n_items;
    float2 *arenas;
    const unsigned char *Ap, *Bp;
    uint32_t kc, n_kc, n_mt, n_nt;
};

// One 128 x NT tile of the real GEMM: thread 0 copies summed-index chunks into a ring of
// shared-memory stages, thread 32 issues the MMAs (each chunk's commit frees its stage, the
// last one signals the accumulator), then every warp stores its 32 rows of C.
template <int NT>
__global__ void __launch_bounds__(128) gemm_tc_kernel(GemmArgs ga) {
    constexpr uint32_t kCols = NT < 32 ? 32u : (uint32_t)NT;   // tensor-memory columns (power of 2)
    extern __shared__ __align__(1024) unsigned char gsm[];
    __shared__ __align__(8) uint64_t full_bar[kGemmStages], empty_bar[kGemmStages], acc_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int fail;
    const GemmStep &g = ga.g;
    const uint32_t kc = ga.kc, n_kc = ga.n_kc;
    const uint32_t tile_a = kGemmRows * kc * 2u, tile_b = (uint32_t)NT * kc * 2u;
    uint64_t t = blockIdx.x;
    const uint32_t nt = (uint32_t)(t % ga.n_nt);
    t /= ga.n_nt;
    const uint32_t mt = (uint32_t)(t % ga.n_mt);
    t /= ga.n_mt;
    const uint64_t ib = t;                               // (item, b)
    const int64_t il = (int64_t)(ib >> g.nb);
    const uint32_t beta = (uint32_t)(ib & ((1u << g.nb) - 1u));
    const unsigned char *Ablk = ga.Ap + ((ib * ga.n_mt + mt) * n_kc) * (uint64_t)tile_a;
    const unsigned char *Bblk = ga.Bp + ((ib * ga.n_nt + nt) * n_kc) * (uint64_t)tile_b;
    const uint32_t warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const uint32_t sbase = smem_u32(gsm);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kGemmStages; s++) {
            mbar_init(smem_u32(&full_bar[s]), 1);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        mbar_init(smem_u32(&acc_bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fail = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    if (threadIdx.x == 0) {   // producer
        for (uint32_t c = 0; c < n_kc; c++) {
            const uint32_t s = c % kGemmStages;
            if (c >= (uint32_t)kGemmStages && !mbar_wait(smem_u32(&empty_bar[s]), ((c / kGemmStages) - 1u) & 1u, kGemmPolls)) {
                fail = 1;
                break;
            }
            const uint32_t fb = smem_u32(&full_bar[s]);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(tile_a + tile_b)
                         : "memory");
            const uint32_t sa = sbase + s * (tile_a + tile_b);
            bulk_g2s(sa, Ablk + (uint64_t)c * tile_a, tile_a, fb);
            bulk_g2s(sa + tile_a, Bblk + (uint64_t)c * tile_b, tile_b, fb);
        }
    } else if (threadIdx.x == 32) {   // MMA issuer
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NT >> 3) << 17) |
                               ((uint32_t)(kGemmRows >> 4) << 24);
        const uint32_t sbo = kc * 16u;
        for (uint32_t c = 0; c < n_kc; c++) {
            const uint32_t s = c % kGemmStages;
            if (!mbar_wait(smem_u32(&full_bar[s]), (c / kGemmStages) & 1u, kGemmPolls)) {
                fail = 1;
                break;
            }
            tc_fence_after();
            const uint32_t sa = sbase + s * (tile_a + tile_b), sb = sa + tile_a;
            for (uint32_t i = 0; i < kc / 16u; i++) {
                const uint64_t ad = smem_desc(sa + i * 256u, 128u, sbo), bd = smem_desc(sb + i * 256u, 128u, sbo);
                const uint32_t accumulate = (c | i) != 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&empty_bar[s]))
                         : "memory");
        }
        // always signal the accumulator, so the MMAs issued so far are waited for
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&acc_bar))
                     : "memory");
    }
    __syncwarp();
    const bool ok = mbar_wait(smem_u32(&acc_bar), 0, kGemmPolls);
    tc_fence_after();
    const bool good = __syncthreads_and(ok) && !fail;
    if (good) {
        // row 32 warp + lane of the tile: Re (even lane) or Im (odd lane) of complex row m
        const uint32_t s = lane & 1u;
        const uint32_t m = mt * (kGemmRows / 2) + warp * 16u + (lane >> 1);
        float2 *C = ga.arenas + (uint64_t)il * ga.a.arena_elems + g.c_off + pext_runs(beta, g.cb, g.n_cb) +
                    pext_runs(m, g.cm, g.n_cm);
        const uint32_t taddr = tmem + ((warp * 32u) << 16);
        for (uint32_t j0 = 0; j0 < (uint32_t)NT; j0 += 16) {
            uint32_t r[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                "%13, %14, %15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(taddr + j0));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            // the even lane keeps columns j0..j0+7 and takes Im from its odd neighbour; the
            // odd lane keeps j0+8..j0+15 and takes Re
#pragma unroll
            for (int jj = 0; jj < 8; jj++) {
                const float mine_send = __uint_as_float(s ? r[jj] : r[8 + jj]);
                const float other = __shfl_xor_sync(0xffffffffu, mine_send, 1);
                const uint32_t col = j0 + (s ? 8u : 0u) + (uint32_t)jj;
                const float re = s ? other : __uint_as_float(r[jj]);
                const float im = s ? __uint_as_float(r[8 + jj]) : other;
                C[pext_runs(nt * (uint32_t)NT + col, g.cn, g.n_cn)] = make_float2(re, im);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
    }
    if (!good && threadIdx.x == 0) atomicCAS(ga.a.status, 0u, 4u /* QVX_ETIMEOUT */);
}

template <int NT>
size_t gemm_smem(uint32_t kc) {
    return (size_t)kGemmStages * ((size_t)kGemmRows * kc * 2 + (size_t)NT * kc * 2);
}

}  // namespace

uint32_t gemm_kc(const GemmStep &g) { return ((6u << g.nk) % 64u == 0) ? 64u : 32u; }
uint32_t gemm_nt(const GemmStep &g) { return g.nn >= 7 ? 128u : (1u << g.nn); }

size_t gemm_pack_bytes_per_item(const GemmStep &g) {
    const size_t kp = (size_t)6 << g.nk;
    return ((size_t)1 << g.nb) * kp * 2 * (((size_t)2 << g.nm) + ((size_t)1 << g.nn));
}

template <int NT>
static cudaError_t launch_gemm_nt(const GemmArgs &ga, cudaStream_t s) {
    static int ready[64] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    size_t smem = gemm_smem<NT>(ga.kc);
    // keep the CTAs an SM can hold within its 512 tensor-memory columns
    const int cols = NT < 32 ? 32 : NT;
    const int max_ctas = 512 / cols;
    if (dev < 0 || dev >= 64 || !ready[dev]) {
        if ((e = cudaFuncSetAttribute(gemm_tc_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024)) !=
            cudaSuccess)
            return e;
        if (dev >= 0 && dev < 64) ready[dev] = 1;
    }
    for (;;) {
        int n = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, gemm_tc_kernel<NT>, 128, smem)) != cudaSuccess)
            return e;
        if (n <= max_ctas || smem >= 200 * 1024) break;
        smem += 8 * 1024;
    }
    const uint64_t blocks = ((uint64_t)ga.n_items << ga.g.nb) * ga.n_mt * ga.n_nt;
    if (blocks == 0 || blocks > 0x7fffffffull) return cudaErrorInvalidConfiguration;
    gemm_tc_kernel<NT><<<(unsigned)blocks, 128, smem, s>>>(ga);
    return cudaGetLastError();
}

cudaError_t launch_gemm_step(const LaunchArgs &a, const GemmStep &g, int64_t item0, int64_t n_items, float2 *arenas,
                             unsigned char *pack, cudaStream_t s) {
    if (g.nk < 4 || g.nm < 6 || g.nn < 4 || n_items <= 0) return cudaErrorInvalidConfiguration;
    const uint32_t kc = gemm_kc(g), nt_cols = gemm_nt(g), K = 1u << g.nk, Kp = 6u * K;
    const uint32_t M2 = 2u << g.nm, N = 1u << g.nn;
    const uint64_t ibs = (uint64_t)n_items << g.nb;
    unsigned char *Ap = pack;
    unsigned char *Bp = pack + ibs * (uint64_t)M2 * Kp * 2u;
    cudaError_t e;
    {
        const uint64_t threads = ibs * M2 * (Kp / 8u);
        pack_a_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(a, g, item0, n_items, arenas, Ap, kc);
        if ((e = launch_counted(cudaGetLastError())) != cudaSuccess) return e;
    }
    {
        const uint64_t threads = ibs * N * (Kp / 8u);
        pack_b_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(a, g, item0, n_items, arenas, Bp, kc, nt_cols);
        if ((e = launch_counted(cudaGetLastError())) != cudaSuccess) return e;
    }
    GemmArgs ga;
    ga.a = a;
    ga.g = g;
    ga.item0 = item0;
    ga.n_items = n_items;
    ga.arenas = arenas;
    ga.Ap = Ap;
    ga.Bp = Bp;
    ga.kc = kc;
    ga.n_kc = Kp / kc;
    ga.n_mt = M2 / kGemmRows;
    ga.n_nt = N / nt_cols;
    switch (nt_cols) {
        case 16: e = launch_gemm_nt<16>(ga, s); break;
        case 32: e = launch_gemm_nt<32>(ga, s); break;
        case 64: e = launch_gemm_nt<64>(ga, s); break;
        default: e = launch_gemm_nt<128>(ga, s); break;
    }
    return launch_counted(e);
}

}  // namespace qvx
