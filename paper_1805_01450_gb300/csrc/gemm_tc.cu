// Dense contractions on the tcgen05 tensor cores (stepwise engine, opts.tensor_cores).
//
// A step C[b, m, n] = sum_k A[b, m, k] B[b, k, n] in complex64 becomes one real GEMM per
// (work item, b): with A = Ar + i Ai and B = Br + i Bi, the real rows 2m and 2m + 1 of
//   [Ar  -Ai]        [Br]
//   [Ai   Ar]  times [Bi]
// are Re C[m, :] and Im C[m, :] (the left factor's first column block is "part 0", the
// second "part 1"). Every real operand x is split into three bf16 parts x = h + m + l
// (8 significant bits each: h = rn(x), m = rn(x - h), l = rn(x - h - m)), and the six
// products h*h + h*m + m*h + h*l + l*h + m*m are accumulated in FP32; the dropped terms
// (m*l, l*m, l*l) are below 2^-23 of the product. Two parts with three products (about
// 2^-16 per product) are not accurate enough: on a 64-qubit circuit the amplitude moved by
// 1.2e-5 of its size, above the 1e-5 tolerance.
//
// One CTA computes a tile of 128 real rows (64 complex rows m) by NT columns n for one
// (item, b). Warps 0-3 read the complex64 operands straight from the arena, one chunk of
// 16 summed entries at a time, split them into three bf16 parts and store them in shared
// memory in the tensor cores' K-major core-matrix layout (no separate packing pass: the
// operands cross HBM once, as complex64). Warp 4 allocates the tensor-memory accumulator
// and one of its threads issues the chunk's twelve tcgen05.mma (2 parts x 6 products,
// K = 16 each); the commit of a chunk's MMAs frees its shared-memory stage. Warps 0-3 then read
// the accumulator back with tcgen05.ld and store complex64 C in its own layout.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "device_program.h"
#include "device_util.cuh"
#include "kernels.h"

namespace qvx {
namespace {

constexpr uint32_t kRows = 128;        // real rows per tile (64 complex rows)
constexpr uint32_t kStages = 1;        // shared-memory stages of summed-index chunks (the next
                                       // chunk waits in registers meanwhile)
constexpr uint32_t kKq = 16;           // complex summed entries per chunk (one MMA K-step)
constexpr uint32_t kPitch = 272;       // bytes between 8-row groups: two 128-byte core matrices
                                       // along the summed index and 16 bytes that spread the
                                       // producers' 16-byte stores over all banks
constexpr uint32_t kPolls = 1u << 22;
constexpr uint32_t kThreads = 160;     // warps 0-3: operands and epilogue; warp 4: MMA

__host__ __device__ constexpr uint32_t region_bytes(uint32_t rows) { return rows / 8u * kPitch; }
// One stage: A regions (part 0 h, m, l, part 1 h, m, l), then the same for B.
__host__ __device__ constexpr uint32_t stage_bytes(uint32_t nt) { return 6u * region_bytes(kRows) + 6u * region_bytes(nt); }

__device__ __forceinline__ uint32_t core_offset(uint32_t r, uint32_t g) {
    return (r >> 3) * kPitch + g * 128u + (r & 7u) * 16u;
}

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

// Three-part bf16 split of v as raw 16-bit patterns: h = rn(v), m = rn(v - h),
// l = rn(v - h - m); both differences are exact in FP32.
__device__ __forceinline__ void split_bf16(float v, uint32_t &h, uint32_t &m, uint32_t &l) {
    const __nv_bfloat16 bh = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(bh);
    const __nv_bfloat16 bm = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(bm);
    h = __bfloat16_as_ushort(bh);
    m = __bfloat16_as_ushort(bm);
    l = __bfloat16_as_ushort(__float2bfloat16_rn(r2));
}

__device__ __forceinline__ uint4 pack8(const uint32_t *h) {
    return make_uint4(h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16), h[6] | (h[7] << 16));
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

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// Three bf16 parts (index 0: h, 1: m, 2: l) of the real and imaginary parts of 8 summed
// entries of one operand row or column.
__device__ __forceinline__ void split8(const float2 *v, uint32_t (*re)[8], uint32_t (*im)[8]) {
#pragma unroll
    for (int j = 0; j < 8; j++) {
        split_bf16(v[j].x, re[0][j], re[1][j], re[2][j]);
        split_bf16(v[j].y, im[0][j], im[1][j], im[2][j]);
    }
}

// A rows 2m and 2m+1 of one summed half (8 entries) in the six A regions of a stage
// (region 3p + level): part 0 takes (Ar, Ai), part 1 takes (-Ai, Ar).
__device__ __forceinline__ void store_a(unsigned char *sa, const float2 *v, uint32_t ml, uint32_t h) {
    constexpr uint32_t R = region_bytes(kRows);
    uint32_t re[3][8], im[3][8];
    split8(v, re, im);
    const uint32_t r0 = core_offset(2u * ml, h), r1 = core_offset(2u * ml + 1u, h);
#pragma unroll
    for (uint32_t q = 0; q < 3; q++) {
        *reinterpret_cast<uint4 *>(sa + q * R + r0) = pack8(re[q]);
        *reinterpret_cast<uint4 *>(sa + q * R + r1) = pack8(im[q]);
        *reinterpret_cast<uint4 *>(sa + (3u + q) * R + r1) = pack8(re[q]);
    }
#pragma unroll
    for (uint32_t q = 0; q < 3; q++) {
#pragma unroll
        for (int j = 0; j < 8; j++) im[q][j] ^= 0x8000u;
        *reinterpret_cast<uint4 *>(sa + (3u + q) * R + r0) = pack8(im[q]);
    }
}

// B column n of one summed half in the six B regions: part 0 takes Br, part 1 Bi.
template <int NT>
__device__ __forceinline__ void store_b(unsigned char *sb, const float2 *v, uint32_t nl, uint32_t h) {
    constexpr uint32_t R = region_bytes(NT);
    uint32_t re[3][8], im[3][8];
    split8(v, re, im);
    const uint32_t o = core_offset(nl, h);
#pragma unroll
    for (uint32_t q = 0; q < 3; q++) {
        *reinterpret_cast<uint4 *>(sb + q * R + o) = pack8(re[q]);
        *reinterpret_cast<uint4 *>(sb + (3u + q) * R + o) = pack8(im[q]);
    }
}

// One chunk's operand entries held in registers between their loads and their conversion:
// 8 summed entries of an A row, and of each of the thread's U B columns.
template <uint32_t U>
struct Chunk {
    float2 a[8];
    float2 b[U][8];
};

// Loads of one chunk; ka and kb are the CTA's shared-memory tables of the summed index's
// offsets in A and in B (8 consecutive entries read as two 16-byte words).
template <uint32_t U>
__device__ __forceinline__ void load_chunk(Chunk<U> &ch, uint32_t c, uint32_t h, const float2 *Arow,
                                           const float2 *const *Bcol, const uint32_t *bh, bool b_on,
                                           const uint32_t *ka, const uint32_t *kb) {
    {
        const uint4 o0 = *reinterpret_cast<const uint4 *>(ka + c * kKq + 8u * h);
        const uint4 o1 = *reinterpret_cast<const uint4 *>(ka + c * kKq + 8u * h + 4u);
        const uint32_t o[8] = {o0.x, o0.y, o0.z, o0.w, o1.x, o1.y, o1.z, o1.w};
#pragma unroll
        for (int j = 0; j < 8; j++) ch.a[j] = __ldg(Arow + o[j]);
    }
    if (b_on) {
#pragma unroll
        for (uint32_t i = 0; i < U; i++) {
            const uint4 o0 = *reinterpret_cast<const uint4 *>(kb + c * kKq + 8u * bh[i]);
            const uint4 o1 = *reinterpret_cast<const uint4 *>(kb + c * kKq + 8u * bh[i] + 4u);
            const uint32_t o[8] = {o0.x, o0.y, o0.z, o0.w, o1.x, o1.y, o1.z, o1.w};
#pragma unroll
            for (int j = 0; j < 8; j++) ch.b[i][j] = __ldg(Bcol[i] + o[j]);
        }
    }
}

struct GemmArgs {
    LaunchArgs a;
    GemmStep g;
    int64_t item0, n_items;
    float2 *arenas;
    uint32_t n_chunks, n_mt, n_nt;
};

template <int NT>
__global__ void __launch_bounds__(kThreads, 3) gemm_tc_kernel(GemmArgs ga) {
    constexpr uint32_t kCols = NT < 32 ? 32u : (uint32_t)NT;   // tensor-memory columns (power of 2)
    constexpr uint32_t kRegA = region_bytes(kRows), kStage = stage_bytes(NT);
    constexpr uint32_t kUnits = (2u * (uint32_t)NT + 127u) / 128u;   // B units per producer thread
    using Chunk = qvx::Chunk<kUnits>;
    extern __shared__ __align__(1024) unsigned char gsm[];
    __shared__ __align__(8) uint64_t full_bar[kStages], empty_bar[kStages], acc_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int fail;
    const GemmStep &g = ga.g;
    uint64_t t = blockIdx.x;   // tiles of one (item, b) and column tile run next to each other
    const uint32_t mt = (uint32_t)(t % ga.n_mt);
    t /= ga.n_mt;
    const uint32_t nt = (uint32_t)(t % ga.n_nt);
    t /= ga.n_nt;
    const uint64_t ib = t;
    const int64_t il = (int64_t)(ib >> g.nb);
    const uint32_t beta = (uint32_t)(ib & ((1u << g.nb) - 1u));
    const uint32_t warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const uint32_t sbase = smem_u32(gsm);
    if (threadIdx.x == 0) {
        for (uint32_t s = 0; s < kStages; s++) {
            mbar_init(smem_u32(&full_bar[s]), 128);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        mbar_init(smem_u32(&acc_bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fail = 0;
    }
    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // address tables of this tile (bit-run maps evaluated once per CTA): the summed index's
    // offsets in A and B, and the offsets of the tile's rows and columns in C
    const uint32_t K = ga.n_chunks * kKq;
    uint32_t *tka = reinterpret_cast<uint32_t *>(gsm + kStages * kStage);
    uint32_t *tkb = tka + K, *tcm = tkb + K, *tcn = tcm + 64;
    for (uint32_t i = threadIdx.x; i < K; i += kThreads) {
        tka[i] = pext_runs(i, g.ak, g.n_ak);
        tkb[i] = pext_runs(i, g.bk, g.n_bk);
    }
    for (uint32_t i = threadIdx.x; i < 64u + (uint32_t)NT; i += kThreads)
        tcm[i] = i < 64u ? pext_runs(mt * 64u + i, g.cm, g.n_cm) : pext_runs(nt * (uint32_t)NT + i - 64u, g.cn, g.n_cn);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    float2 *arena = ga.arenas + (uint64_t)il * ga.a.arena_elems;
    if (warp < 4) {
        // producers: A rows m = mt*64 + 32*(warp&1) + lane, summed half h = warp>>1 of the
        // chunk; B units (column, half) strided over the 128 threads. A chunk's loads are
        // all issued before its conversion, and the next chunk's before this one's stores.
        const float2 *A = gemm_operand(ga.a, arena, g.a_off, g.flags & kStepALeaf, ga.item0 + il);
        const float2 *B = gemm_operand(ga.a, arena, g.b_off, g.flags & kStepBLeaf, ga.item0 + il);
        const uint32_t ml = 32u * (warp & 1u) + lane, h = warp >> 1;
        const float2 *Arow = A + pext_runs(beta, g.ab, g.n_ab) + pext_runs(mt * 64u + ml, g.am, g.n_am);
        const float2 *Bcol[kUnits];
        uint32_t bh[kUnits];
#pragma unroll
        for (uint32_t i = 0; i < kUnits; i++) {
            const uint32_t u = threadIdx.x + 128u * i;
            const uint32_t nl = u % (uint32_t)NT;
            bh[i] = u / (uint32_t)NT;
            Bcol[i] = B + pext_runs(beta, g.bb, g.n_bb) + pext_runs(nt * (uint32_t)NT + nl, g.bn, g.n_bn);
        }
        const bool b_on = threadIdx.x < 2u * (uint32_t)NT;   // every unit of a thread shares this
        Chunk cur, nxt;
        load_chunk(cur, 0, h, Arow, Bcol, bh, b_on, tka, tkb);
        for (uint32_t c = 0; c < ga.n_chunks; c++) {
            const uint32_t s = c % kStages;
            if (c + 1 < ga.n_chunks) load_chunk(nxt, c + 1, h, Arow, Bcol, bh, b_on, tka, tkb);
            if (c >= kStages && !mbar_wait(smem_u32(&empty_bar[s]), ((c / kStages) - 1u) & 1u, kPolls)) {
                fail = 1;
                break;
            }
            unsigned char *sa = gsm + s * kStage;
            store_a(sa, cur.a, ml, h);
            if (b_on) {
#pragma unroll
                for (uint32_t i = 0; i < kUnits; i++)
                    store_b<NT>(sa + 6u * kRegA, cur.b[i], (threadIdx.x + 128u * i) % (uint32_t)NT, bh[i]);
            }
            // the generic-proxy stores must be visible to the tensor cores' reads
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&full_bar[s])) : "memory");
            cur = nxt;
        }
    } else if (lane == 0) {   // MMA issuer
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NT >> 3) << 17) |
                               ((kRows >> 4) << 24);
        for (uint32_t c = 0; c < ga.n_chunks; c++) {
            const uint32_t s = c % kStages;
            if (!mbar_wait(smem_u32(&full_bar[s]), (c / kStages) & 1u, kPolls)) {
                fail = 1;
                break;
            }
            tc_fence_after();
            const uint32_t sa = sbase + s * kStage, sb = sa + 6u * kRegA;
            constexpr uint32_t kRegB = region_bytes(NT);
#pragma unroll
            for (uint32_t p = 0; p < 2; p++) {
                uint64_t ad[3], bd[3];
#pragma unroll
                for (uint32_t q = 0; q < 3; q++) {
                    ad[q] = smem_desc(sa + (3u * p + q) * kRegA, 128u, kPitch);
                    bd[q] = smem_desc(sb + (3u * p + q) * kRegB, 128u, kPitch);
                }
                // h*h, h*m, m*h, h*l, l*h, m*m
                mma_bf16(tmem, ad[0], bd[0], idesc, (c | p) != 0u);
                mma_bf16(tmem, ad[0], bd[1], idesc, 1u);
                mma_bf16(tmem, ad[1], bd[0], idesc, 1u);
                mma_bf16(tmem, ad[0], bd[2], idesc, 1u);
                mma_bf16(tmem, ad[2], bd[0], idesc, 1u);
                mma_bf16(tmem, ad[1], bd[1], idesc, 1u);
            }
            mma_commit(smem_u32(&empty_bar[s]));
        }
        // always signal the accumulator, so the MMAs issued so far are waited for
        mma_commit(smem_u32(&acc_bar));
    }
    __syncwarp();
    bool ok = true;
    if (warp < 4) ok = mbar_wait(smem_u32(&acc_bar), 0, kPolls);
    tc_fence_after();
    const bool good = __syncthreads_and(ok) && !fail;
    if (good && warp < 4) {
        // warp w holds tile rows 32w..32w+31, i.e. complex rows m = mt*64 + 16w + lane/2 (Re in
        // the even lane, Im in the odd one). Each block of up to 32 columns goes through a
        // padded shared-memory transpose (the operand stages are free now), so that a warp
        // then stores 32 consecutive columns of one row of C at a time.
        constexpr uint32_t kW = NT < 32 ? (uint32_t)NT : 32u;   // columns per block
        constexpr uint32_t kTPitch = 8u * kW + 8u;               // bytes per row of the transpose
        unsigned char *tb = gsm + warp * 16u * kTPitch;
        const uint32_t s = lane & 1u, mrow = lane >> 1;
        const uint32_t taddr = tmem + ((warp * 32u) << 16);
        float2 *Cb = arena + g.c_off + pext_runs(beta, g.cb, g.n_cb);
        for (uint32_t j0 = 0; j0 < (uint32_t)NT; j0 += kW) {
            uint32_t r[kW];
            if constexpr (kW == 32) {
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                    "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
                    "[%32];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                      "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                      "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
                      "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
                      "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                    : "r"(taddr + j0));
            } else {
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
                    "%12, %13, %14, %15}, [%16];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                      "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                      "=r"(r[14]), "=r"(r[15])
                    : "r"(taddr + j0));
            }
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (uint32_t n = 0; n < kW; n++)
                *reinterpret_cast<uint32_t *>(tb + mrow * kTPitch + n * 8u + s * 4u) = r[n];
            __syncwarp();
            if (lane < kW) {
                const uint32_t coff = tcn[j0 + lane];
#pragma unroll 4
                for (uint32_t i = 0; i < 16; i++) {
                    const float2 v = *reinterpret_cast<const float2 *>(tb + i * kTPitch + lane * 8u);
                    Cb[tcm[warp * 16u + i] + coff] = v;
                }
            }
            __syncwarp();
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 4) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
    }
    if (!good && threadIdx.x == 0) atomicCAS(ga.a.status, 0u, 4u /* QVX_ETIMEOUT */);
}

}  // namespace

uint32_t gemm_nt(const GemmStep &g) { return g.nn >= 7 ? 128u : (1u << g.nn); }

template <int NT>
static cudaError_t launch_gemm_nt(const GemmArgs &ga, cudaStream_t s) {
    static int ready[64] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    size_t smem = (size_t)kStages * stage_bytes(NT) + 4u * (2u * ga.n_chunks * kKq + 64u + (uint32_t)NT);
    constexpr size_t kMaxSmem = 200 * 1024;
    // keep the CTAs an SM can hold within its 512 tensor-memory columns, so that no
    // allocation ever waits for another CTA's columns
    const int cols = NT < 32 ? 32 : NT;
    const int max_ctas = 512 / cols;
    if (dev < 0 || dev >= 64 || !ready[dev]) {
        if ((e = cudaFuncSetAttribute(gemm_tc_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem)) !=
            cudaSuccess)
            return e;
        if (dev >= 0 && dev < 64) ready[dev] = 1;
    }
    for (;;) {
        int n = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, gemm_tc_kernel<NT>, kThreads, smem)) != cudaSuccess)
            return e;
        if (n <= max_ctas) break;
        if (smem >= kMaxSmem) return cudaErrorInvalidConfiguration;
        smem += 8 * 1024;
    }
    const uint64_t blocks = ((uint64_t)ga.n_items << ga.g.nb) * ga.n_mt * ga.n_nt;
    if (blocks == 0 || blocks > 0x7fffffffull) return cudaErrorInvalidConfiguration;
    gemm_tc_kernel<NT><<<(unsigned)blocks, kThreads, smem, s>>>(ga);
    return cudaGetLastError();
}

cudaError_t launch_gemm_step(const LaunchArgs &a, const GemmStep &g, int64_t item0, int64_t n_items, float2 *arenas,
                             cudaStream_t s) {
    if (g.nk < 4 || g.nk > 10 || g.nm < 6 || g.nn < 4 || n_items <= 0) return cudaErrorInvalidConfiguration;
    const uint32_t nt_cols = gemm_nt(g);
    GemmArgs ga;
    ga.a = a;
    ga.g = g;
    ga.item0 = item0;
    ga.n_items = n_items;
    ga.arenas = arenas;
    ga.n_chunks = (1u << g.nk) / kKq;
    ga.n_mt = (2u << g.nm) / kRows;
    ga.n_nt = (1u << g.nn) / nt_cols;
    cudaError_t e;
    switch (nt_cols) {
        case 16: e = launch_gemm_nt<16>(ga, s); break;
        case 32: e = launch_gemm_nt<32>(ga, s); break;
        case 64: e = launch_gemm_nt<64>(ga, s); break;
        default: e = launch_gemm_nt<128>(ga, s); break;
    }
    return launch_counted(e);
}

}  // namespace qvx
