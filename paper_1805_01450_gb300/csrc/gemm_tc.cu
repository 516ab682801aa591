// Dense contractions on the tcgen05 tensor cores (stepwise engine, opts.tensor_cores).
//
// A step C[b, m, n] = sum_k A[b, m, k] B[b, k, n] in complex64 becomes one real GEMM per
// (work item, b): with A = Ar + i Ai and B = Br + i Bi,
//   [Re C[m, n], Im C[m, n]] = [Ar | Ai][m, :]  times  [[Br, Bi], [-Bi, Br]][:, (n, re/im)],
// i.e. the left factor's real summed index is (part p, k) with part 0 = Ar and part 1 = Ai,
// and the right factor has two real columns per complex column n: 2n = (Br; -Bi) and
// 2n + 1 = (Bi; Br). Every real operand x is split into three bf16 parts x = h + m + l (8
// significant bits each: h = rn(x), m = rn(x - h), l = rn(x - h - m)), and the six products
// h*h + h*m + m*h + h*l + l*h + m*m are accumulated in FP32; the dropped terms (m*l, l*m,
// l*l) are below 2^-23 of the product. Two parts with three products (about 2^-16 per
// product) are not accurate enough: on a 64-qubit circuit the amplitude moved by 1.2e-5 of
// its size, above the 1e-5 tolerance.
//
// The row role goes to the operand that holds C's lowest mode, so tensor-memory lane i (row
// m = i of a 128-row tile) holds C entries that are consecutive in memory along the lanes;
// the real columns 2n and 2n + 1 of a lane are Re and Im of C[m, n], so the epilogue stores
// complex64 values straight from the registers tcgen05.ld fills, coalesced across the warp,
// with no transpose. A tile is 128 complex rows by NT real (NT / 2 complex, up to 128)
// columns of one (item, b). The kernel is persistent (one CTA per SM walks the tiles) and
// warp-specialised: producer warps copy the complex64 operands straight from the arena into
// shared memory (cp.async, several chunks of 16 summed entries ahead), split them into
// three bf16 parts and store them in the tensor cores' K-major core-matrix layout in a ring
// of shared-memory stages (no separate packing pass: the operands cross HBM once, as
// complex64); one thread issues each chunk's twelve tcgen05.mma (2 parts x 6 products, K =
// 16 each) into one of two tensor-memory accumulators; epilogue warps store a finished
// accumulator while the next tile's chunks are loaded and multiplied into the other. A step
// with 8 summed entries runs as one chunk whose second half is zeros. Steps with at most two
// chunks and many row tiles per column tile take the B-stationary form (gemm_tc_bs_kernel,
// below): a column tile's split B stays in shared memory for all the row tiles that use it.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "device_program.h"
#include "device_util.cuh"
#include "kernels.h"

namespace qvx {
namespace {

constexpr uint32_t kRows = 128;        // rows per tile (complex rows of C)
constexpr uint32_t kKq = 16;           // complex summed entries per chunk (one MMA K-step)
constexpr uint32_t kPitch = 272;       // bytes between 8-row groups: two 128-byte core matrices
                                       // along the summed index and 16 bytes that spread the
                                       // producers' 16-byte stores over all banks
constexpr uint32_t kPolls = 1u << 22;
constexpr uint32_t kEpiThreads = 256;  // eight epilogue warps, two per tensor-memory lane quarter

__host__ __device__ constexpr uint32_t region_bytes(uint32_t rows) { return rows / 8u * kPitch; }
// One stage: A regions (part 0 h, m, l, part 1 h, m, l), then the same for B.
__host__ __device__ constexpr uint32_t stage_bytes(uint32_t nt) { return 6u * region_bytes(kRows) + 6u * region_bytes(nt); }

// Producer threads: one per operand unit of a chunk (8 summed entries of one A row or one
// complex B column): 128 rows x 2 halves of A and NT / 2 columns x 2 halves of B (threads
// beyond the units, for NT = 16, only take part in the barriers).
template <int NT>
__host__ __device__ constexpr uint32_t producers() { return 256u + ((uint32_t)NT < 32u ? 32u : (uint32_t)NT); }
template <int NT>
__host__ __device__ constexpr uint32_t block_threads() { return producers<NT>() + 32u + kEpiThreads; }
// Operand stages of the shared-memory ring: two for 128- and 256-column tiles (52 and 77 KB),
// three below.
template <int NT>
__host__ __device__ constexpr uint32_t n_stages() { return NT >= 128 ? 2u : 3u; }
// Raw copy slots per producer (chunks in flight): four, two for 256-column tiles (their
// 512 producers' slots and two 77 KB stages fill the shared memory).
template <int NT>
__host__ __device__ constexpr uint32_t raw_depth() { return NT >= 256 ? 2u : 4u; }
// real accumulator columns an epilogue warp reads at a time
template <int NT>
__host__ __device__ constexpr uint32_t epi_cols() { return NT < 32 ? (uint32_t)NT : 32u; }
// raw copy slot: 8 complex64 entries per producer thread, entry j of thread t at j * P + t
template <int NT>
__host__ __device__ constexpr uint32_t raw_slot_bytes() { return 8u * producers<NT>() * 8u; }
template <int NT>
__host__ __device__ constexpr size_t smem_bytes(uint32_t K) {
    return (size_t)n_stages<NT>() * stage_bytes(NT) + (size_t)raw_depth<NT>() * raw_slot_bytes<NT>() + 8u * (size_t)K;
}

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
    const Bits x = load_bits(a.bitstrings, item / a.o_count, a.words);
    const uint64_t o = (uint64_t)(a.o_begin + item % a.o_count);
    return ldata + leaf_base(leaves[ref], x, o);
}

// Three-part bf16 split of two floats at once, as packed pairs (lo in bits 0-15, hi in bits
// 16-31): H = rn(lo, hi), M = rn of the remainders, L = rn of what is left; both remainders
// are exact in FP32. cvt.rn.bf16x2.f32 rounds each half to nearest even.
__device__ __forceinline__ uint32_t cvt_bf16x2(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}
__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

__device__ __forceinline__ void split_pair(float lo, float hi, uint32_t &H, uint32_t &M, uint32_t &L) {
    H = cvt_bf16x2(lo, hi);
    const float rl = lo - bf_lo(H), rh = hi - bf_hi(H);
    M = cvt_bf16x2(rl, rh);
    L = cvt_bf16x2(rl - bf_lo(M), rh - bf_hi(M));
}

// Packed bf16 parts (level 0: h, 1: m, 2: l) of the real and imaginary parts of 8 summed
// entries of one operand row or column: word p holds entries 2p (low) and 2p + 1 (high).
__device__ __forceinline__ void split8(const float2 *v, uint32_t (&re)[3][4], uint32_t (&im)[3][4]) {
#pragma unroll
    for (int p = 0; p < 4; p++) {
        split_pair(v[2 * p].x, v[2 * p + 1].x, re[0][p], re[1][p], re[2][p]);
        split_pair(v[2 * p].y, v[2 * p + 1].y, im[0][p], im[1][p], im[2][p]);
    }
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

// A row m of one summed half (8 entries) in the six A regions of a stage (region 3p +
// level): part 0 takes Ar, part 1 takes Ai.
__device__ __forceinline__ void store_a(unsigned char *sa, const float2 *v, uint32_t m, uint32_t h) {
    constexpr uint32_t R = region_bytes(kRows);
    uint32_t re[3][4], im[3][4];
    split8(v, re, im);
    const uint32_t o = core_offset(m, h);
#pragma unroll
    for (uint32_t q = 0; q < 3; q++) {
        *reinterpret_cast<uint4 *>(sa + q * R + o) = make_uint4(re[q][0], re[q][1], re[q][2], re[q][3]);
        *reinterpret_cast<uint4 *>(sa + (3u + q) * R + o) = make_uint4(im[q][0], im[q][1], im[q][2], im[q][3]);
    }
}

// Complex B column n of one summed half in the six B regions: real column 2n takes Br in
// part 0 and -Bi in part 1, real column 2n + 1 takes Bi in part 0 and Br in part 1.
template <int NT>
__device__ __forceinline__ void store_b(unsigned char *sb, const float2 *v, uint32_t n, uint32_t h) {
    constexpr uint32_t R = region_bytes(NT);
    uint32_t re[3][4], im[3][4];
    split8(v, re, im);
    const uint32_t o0 = core_offset(2u * n, h), o1 = core_offset(2u * n + 1u, h);
#pragma unroll
    for (uint32_t q = 0; q < 3; q++) {
        const uint4 wr = make_uint4(re[q][0], re[q][1], re[q][2], re[q][3]);
        const uint4 wi = make_uint4(im[q][0], im[q][1], im[q][2], im[q][3]);
        const uint4 wn = make_uint4(im[q][0] ^ 0x80008000u, im[q][1] ^ 0x80008000u, im[q][2] ^ 0x80008000u,
                                    im[q][3] ^ 0x80008000u);
        *reinterpret_cast<uint4 *>(sb + q * R + o0) = wr;
        *reinterpret_cast<uint4 *>(sb + (3u + q) * R + o0) = wn;
        *reinterpret_cast<uint4 *>(sb + q * R + o1) = wi;
        *reinterpret_cast<uint4 *>(sb + (3u + q) * R + o1) = wr;
    }
}

__device__ __forceinline__ void cp_async8(uint32_t dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// kW accumulator columns of this warp's 32 tensor-memory lanes into registers (one column
// per register), waited for.
template <uint32_t kW>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, uint32_t (&r)[kW]) {
    if constexpr (kW == 32) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
            "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
            "%30, %31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
              "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
              "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
              "=r"(r[30]), "=r"(r[31])
            : "r"(taddr));
    } else {
        static_assert(kW == 16, "16 or 32 columns");
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
            "%12, %13, %14, %15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
    }
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct GemmArgs {
    LaunchArgs a;
    GemmStep g;
    int64_t item0, n_items;
    float2 *arenas;
    uint32_t n_chunks, n_mt, n_nt;
    uint32_t mt_bits, nt_bits;     // log2 of n_mt and n_nt (every tile count is a power of two)
    uint64_t n_tiles;
};

// Bounded mbarrier wait that also gives up once another role has set the CTA's fail flag.
__device__ __forceinline__ bool wait_or_fail(uint32_t bar, uint32_t parity, volatile int *fail) {
    for (uint32_t i = 0; i < kPolls; i++) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((i & 63u) == 63u && *fail) return false;
    }
    return false;
}

struct TileCoord {
    uint32_t mt, nt, beta;
    int64_t il;
};

// Tile t's row tile, column tile, batch index and work item: row tiles of one (item, b) and
// column tile run next to each other. All counts are powers of two, so shifts and masks.
__device__ __forceinline__ TileCoord tile_coord(uint64_t t, const GemmArgs &ga) {
    TileCoord c;
    c.mt = (uint32_t)t & (ga.n_mt - 1u);
    t >>= ga.mt_bits;
    c.nt = (uint32_t)t & (ga.n_nt - 1u);
    t >>= ga.nt_bits;
    c.il = (int64_t)(t >> ga.g.nb);
    c.beta = (uint32_t)t & ((1u << ga.g.nb) - 1u);
    return c;
}

// Tile order of the B-stationary form: row tiles fastest (one column tile's B serves a run of
// them), then batch index and work item, column tile slowest. The CTAs' contiguous ranges
// then walk the column tiles of one (item, b) at the same time on different SMs, so the
// second column tile's A rows are still in L2 (with the column tile next to the row tiles,
// one CTA read each A tile twice, some 32 row tiles apart, from HBM).
__device__ __forceinline__ TileCoord tile_coord_bs(uint64_t t, const GemmArgs &ga) {
    TileCoord c;
    c.mt = (uint32_t)t & (ga.n_mt - 1u);
    t >>= ga.mt_bits;
    c.beta = (uint32_t)t & ((1u << ga.g.nb) - 1u);
    t >>= ga.g.nb;   // below n_items * n_nt < 2^32: a 32-bit division (a 64-bit one is a
                     // called routine, and the kernel's loops lost a tenth to it)
    const uint32_t q = (uint32_t)t, n = (uint32_t)ga.n_items;
    c.il = (int64_t)(q % n);
    c.nt = q / n;
    return c;
}

// The coordinates of consecutive tiles in that order, advanced without a division (the item
// count need not be a power of two).
struct BsCursor {
    TileCoord c;
    __device__ __forceinline__ void next(const GemmArgs &ga) {
        if (++c.mt < ga.n_mt) return;
        c.mt = 0;
        if (++c.beta < (1u << ga.g.nb)) return;
        c.beta = 0;
        if (++c.il < ga.n_items) return;
        c.il = 0;
        c.nt++;
    }
    // the first row tile of the next column tile
    __device__ __forceinline__ void next_group(const GemmArgs &ga) {
        c.mt = ga.n_mt - 1u;
        next(ga);
    }
};

// Persistent, warp-specialised tensor-core contraction. One CTA per SM walks the tiles
// t = blockIdx.x, blockIdx.x + gridDim.x, ... (128 rows x NT real columns of one (item, b)):
//   producer warps (P threads, one operand unit each): copy the unit's 8
//              complex64 entries of each chunk into a private raw slot with cp.async,
//              kRaw - 1 chunks ahead and across tile boundaries; once a chunk's copies have
//              landed, split it into bf16 parts, store them into the next stage of the ring
//              and arrive on the stage's "full" barrier;
//   one warp   allocates two tensor-memory accumulators; one thread issues each chunk's
//              twelve tcgen05.mma into the tile's accumulator (the tile's first product
//              overwrites it), commits each chunk to the stage's "empty" barrier and the
//              tile's last chunk to the accumulator's "full" barrier;
//   8 warps    epilogue: wait for an accumulator, read it with tcgen05.ld (warp w reads
//              tensor-memory lanes 32 (w mod 4) ..., i.e. rows 32 (w mod 4) + lane; the two
//              warps of a lane quarter take alternate blocks of 32 columns), store each
//              (Re, Im) column pair as one complex64 entry of C and release the accumulator.
//              Four warps left the epilogue about a tenth slower on output-heavy steps: each
//              waits out its tensor-memory reads block by block.
// With two accumulators the epilogue of one tile overlaps the loads and MMAs of the next.
// Every wait is bounded; a wait that runs out sets the CTA's fail flag, the other roles
// leave their loops, the MMA thread waits (bounded) for its issued MMAs before the tensor
// memory is freed, and QVX_ETIMEOUT goes to the status word.
template <int NT>
__global__ void __launch_bounds__(block_threads<NT>(), 1) gemm_tc_kernel(GemmArgs ga) {
    constexpr uint32_t S = n_stages<NT>();
    constexpr uint32_t P = producers<NT>();
    constexpr uint32_t kMmaWarp = P / 32u;
    constexpr uint32_t kCols = NT < 32 ? 32u : (uint32_t)NT;   // columns of one accumulator
    constexpr uint32_t kRegA = region_bytes(kRows), kStage = stage_bytes(NT);
    constexpr uint32_t kW = epi_cols<NT>();
    constexpr uint32_t kNc = (uint32_t)NT / 2u;   // complex columns per tile
    constexpr uint32_t kRawSlot = raw_slot_bytes<NT>();
    constexpr uint32_t kRaw = raw_depth<NT>();
    static_assert(P % 32u == 0u, "producer warps");
    extern __shared__ __align__(1024) unsigned char gsm[];
    __shared__ __align__(8) uint64_t full_bar[S], empty_bar[S], accf_bar[2], acce_bar[2], drain_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int fail;
    const GemmStep &g = ga.g;
    const uint32_t warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const uint32_t sbase = smem_u32(gsm);
    if (threadIdx.x == 0) {
        for (uint32_t s = 0; s < S; s++) {
            mbar_init(smem_u32(&full_bar[s]), P);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        for (uint32_t b = 0; b < 2; b++) {
            mbar_init(smem_u32(&accf_bar[b]), 1);
            mbar_init(smem_u32(&acce_bar[b]), kEpiThreads);
        }
        mbar_init(smem_u32(&drain_bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fail = 0;
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(2u * kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // the summed index's offsets in A and B (bit-run maps evaluated once per CTA)
    const uint32_t K = ga.n_chunks * kKq;
    unsigned char *raw = gsm + S * kStage;
    uint32_t *tka = reinterpret_cast<uint32_t *>(raw + kRaw * kRawSlot);
    uint32_t *tkb = tka + K;
    for (uint32_t i = threadIdx.x; i < K; i += block_threads<NT>()) {
        tka[i] = pext_runs(i, g.ak, g.n_ak);
        tkb[i] = pext_runs(i, g.bk, g.n_bk);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    if (warp < kMmaWarp) {
        // producer: unit u < 256 is A row m = mt*128 + (u & 127), summed half u >> 7; unit
        // u >= 256 is complex B column n = nt*NT/2 + (u - 256) % (NT/2), summed half
        // (u - 256) / (NT/2); threads past the units only take part in the barriers
        const uint32_t u = threadIdx.x;
        const bool is_a = u < 256u;
        const bool active = is_a || u - 256u < (uint32_t)NT;
        const uint32_t row = is_a ? (u & 127u) : (u - 256u) % kNc;
        const uint32_t h = is_a ? (u >> 7) : ((u - 256u) / kNc) & 1u;
        const uint32_t *koff = (is_a ? tka : tkb) + 8u * h;
        // a step with 8 summed entries fills one chunk's first half: the units of the second
        // half load nothing and store zeros, which add nothing to the products
        const bool pad = (1u << g.nk) < kKq && h == 1u;
        const uint32_t raw_mine = smem_u32(raw) + u * 8u;
        // load cursor: the tile and chunk whose copies are issued next
        uint64_t lt = blockIdx.x;
        uint32_t lc = 0;
        const float2 *src = nullptr;
        auto setup = [&](uint64_t t) {
            const TileCoord tc = tile_coord(t, ga);
            const float2 *arena = ga.arenas + (uint64_t)tc.il * ga.a.arena_elems;
            if (is_a)
                src = gemm_operand(ga.a, arena, g.a_off, g.flags & kStepALeaf, ga.item0 + tc.il) +
                      pext_runs(tc.beta, g.ab, g.n_ab) + pext_runs(tc.mt * kRows + row, g.am, g.n_am);
            else
                src = gemm_operand(ga.a, arena, g.b_off, g.flags & kStepBLeaf, ga.item0 + tc.il) +
                      pext_runs(tc.beta, g.bb, g.n_bb) + pext_runs(tc.nt * kNc + row, g.bn, g.n_bn);
        };
        auto issue_next = [&](uint64_t gi) {   // one commit group per chunk, empty past the end
            if (lt < ga.n_tiles && active && !pad) {
                const uint32_t dst = raw_mine + (uint32_t)(gi % kRaw) * kRawSlot;
                const uint4 o0 = *reinterpret_cast<const uint4 *>(koff + lc * kKq);
                const uint4 o1 = *reinterpret_cast<const uint4 *>(koff + lc * kKq + 4u);
                const uint32_t o[8] = {o0.x, o0.y, o0.z, o0.w, o1.x, o1.y, o1.z, o1.w};
#pragma unroll
                for (uint32_t j = 0; j < 8; j++) cp_async8(dst + j * P * 8u, src + o[j]);
            }
            if (lt < ga.n_tiles) {
                if (++lc == ga.n_chunks) {
                    lc = 0;
                    lt += gridDim.x;
                    if (lt < ga.n_tiles && active) setup(lt);
                }
            }
            cp_async_commit();
        };
        if (active) setup(lt);
        const uint64_t my_tiles = (ga.n_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x;
        const uint64_t total = my_tiles * ga.n_chunks;
        for (uint32_t i = 0; i + 1 < kRaw; i++) issue_next(i);
        for (uint64_t gc = 0; gc < total && !fail; gc++) {
            issue_next(gc + kRaw - 1);
            cp_async_wait<kRaw - 1>();   // this thread's copies of chunk gc have landed
            const uint32_t s = (uint32_t)(gc % S);
            if (!wait_or_fail(smem_u32(&empty_bar[s]), (uint32_t)((gc / S) & 1u) ^ 1u, &fail)) {
                fail = 1;
                break;
            }
            if (active) {
                const float2 *rt = reinterpret_cast<const float2 *>(raw + (gc % kRaw) * kRawSlot) + u;
                float2 v[8];
#pragma unroll
                for (uint32_t j = 0; j < 8; j++) v[j] = pad ? make_float2(0.f, 0.f) : rt[j * P];
                unsigned char *sa = gsm + s * kStage;
                if (is_a) store_a(sa, v, row, h);
                else store_b<NT>(sa + 6u * kRegA, v, row, h);
            }
            // the generic-proxy stores must be visible to the tensor cores' reads
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&full_bar[s])) : "memory");
        }
        cp_async_wait<0>();   // no copy may still be landing when the CTA leaves
    } else if (warp == kMmaWarp) {
        if (lane == 0) {   // MMA issuer
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NT >> 3) << 17) |
                                   ((kRows >> 4) << 24);
            constexpr uint32_t kRegB = region_bytes(NT);
            uint64_t gc = 0;
            uint32_t j = 0;
            for (uint64_t t = blockIdx.x; t < ga.n_tiles && !fail; t += gridDim.x, j++) {
                const uint32_t buf = j & 1u;
                if (!wait_or_fail(smem_u32(&acce_bar[buf]), ((j >> 1) & 1u) ^ 1u, &fail)) {
                    fail = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + buf * kCols;
                bool ok = true;
                for (uint32_t c = 0; c < ga.n_chunks; c++, gc++) {
                    const uint32_t s = (uint32_t)(gc % S);
                    if (!wait_or_fail(smem_u32(&full_bar[s]), (uint32_t)((gc / S) & 1u), &fail)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = sbase + s * kStage, sb = sa + 6u * kRegA;
#pragma unroll
                    for (uint32_t p = 0; p < 2; p++) {
                        uint64_t ad[3], bd[3];
#pragma unroll
                        for (uint32_t q = 0; q < 3; q++) {
                            ad[q] = smem_desc(sa + (3u * p + q) * kRegA, 128u, kPitch);
                            bd[q] = smem_desc(sb + (3u * p + q) * kRegB, 128u, kPitch);
                        }
                        // h*h, h*m, m*h, h*l, l*h, m*m
                        mma_bf16(d, ad[0], bd[0], idesc, (c | p) != 0u);
                        mma_bf16(d, ad[0], bd[1], idesc, 1u);
                        mma_bf16(d, ad[1], bd[0], idesc, 1u);
                        mma_bf16(d, ad[0], bd[2], idesc, 1u);
                        mma_bf16(d, ad[2], bd[0], idesc, 1u);
                        mma_bf16(d, ad[1], bd[1], idesc, 1u);
                    }
                    mma_commit(smem_u32(&empty_bar[s]));
                }
                if (!ok) {
                    fail = 1;
                    break;
                }
                mma_commit(smem_u32(&accf_bar[buf]));
            }
            // every MMA issued so far completes before the tensor memory is freed
            mma_commit(smem_u32(&drain_bar));
            if (!mbar_wait(smem_u32(&drain_bar), 0, kPolls)) fail = 1;
        }
        __syncwarp();
    } else {
        // epilogue: warp w reads tensor-memory lanes 32q ... 32q + 31 (q = w mod 4): row
        // m = mt*128 + 32q + lane of the tile, whose real columns 2j and 2j + 1 are Re and Im
        // of C[m, nt*NT/2 + j]. For each column the warp's 32 stores are 32 rows, consecutive
        // in C when its lowest modes are row modes (the planner gives the row role to the
        // operand that holds C's lowest mode).
        const uint32_t q = warp & 3u;
        const uint32_t share = (warp - kMmaWarp - 1u) >> 2;   // the two warps of a lane quarter split its columns
        uint32_t j = 0;
        for (uint64_t t = blockIdx.x; t < ga.n_tiles && !fail; t += gridDim.x, j++) {
            const TileCoord tc = tile_coord(t, ga);
            const uint32_t buf = j & 1u;
            // this lane's row of C and the tile's base, while the MMAs run
            float2 *Crow = ga.arenas + (uint64_t)tc.il * ga.a.arena_elems + g.c_off + pext_runs(tc.beta, g.cb, g.n_cb) +
                           pext_runs(tc.mt * kRows + 32u * q + lane, g.cm, g.n_cm);
            if (!wait_or_fail(smem_u32(&accf_bar[buf]), (j >> 1) & 1u, &fail)) {
                fail = 1;
                break;
            }
            tc_fence_after();
            const uint32_t taddr = tmem + ((q * 32u) << 16) + buf * kCols;
            for (uint32_t j0 = share * kW; j0 < (uint32_t)NT; j0 += 2u * kW) {
                // the column offsets of this block's kW / 2 complex columns, one per lane
                const uint32_t my_col = pext_runs(tc.nt * kNc + j0 / 2u + (lane % (kW / 2u)), g.cn, g.n_cn);
                uint32_t r[kW];
                tmem_ld<kW>(taddr + j0, r);
#pragma unroll
                for (uint32_t i = 0; i < kW / 2u; i++) {
                    const uint32_t coff = __shfl_sync(0xffffffffu, my_col, i);
                    Crow[coff] = make_float2(__uint_as_float(r[2u * i]), __uint_as_float(r[2u * i + 1u]));
                }
            }
            // the accumulator's reads are done: the MMAs of the tile after next may reuse it
            tc_fence_before();
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce_bar[buf])) : "memory");
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2u * kCols) : "memory");
    }
    if (fail && threadIdx.x == 0) atomicCAS(ga.a.status, 0u, 4u /* QVX_ETIMEOUT */);
}

// B-stationary form for steps with at most two chunks of summed entries (K <= 32) and many
// row tiles per column tile: a CTA walks a contiguous range of tiles, row tiles fastest, so
// one column tile's B operand (all its chunks) is split once into resident shared-memory
// regions and serves every row tile of the range that shares it; only A goes through the
// stage ring. The B producers reload when the column tile changes, after the MMAs that read
// the old one have completed. Against the streaming form this removes most of the
// producers' shared-memory traffic on output-heavy steps (B is 4 of the 6 operand values a
// complex entry pair produces).
// A stages (26 KB each) and accumulators: the narrower the column tile, the shorter a tile's
// work against its fixed barrier round trips, so narrow tiles keep more tiles in flight
// (tensor memory holds 512 columns: 2 x 256, 4 x 128, 8 x 64, 8 x 32).
template <int NT>
__host__ __device__ constexpr uint32_t bs_stages() { return NT >= 256 ? 2u : (NT >= 128 ? 3u : 4u); }
template <int NT>
__host__ __device__ constexpr uint32_t bs_cols() { return NT < 32 ? 32u : (uint32_t)NT; }   // one accumulator
template <int NT>
__host__ __device__ constexpr uint32_t bs_accs() { return 512u / bs_cols<NT>() < 8u ? 512u / bs_cols<NT>() : 8u; }
__host__ __device__ constexpr uint32_t bs_stage_bytes() { return 6u * region_bytes(kRows); }
template <int NT>
__host__ __device__ constexpr uint32_t bs_b_bytes() { return 6u * region_bytes(NT); }   // one chunk of B
template <int NT>
__host__ __device__ constexpr uint32_t bs_b_units() { return (uint32_t)NT < 32u ? 32u : (uint32_t)NT; }
template <int NT>
__host__ __device__ constexpr uint32_t bs_raw_depth() { return NT >= 256 ? 3u : 4u; }
template <int NT>
__host__ __device__ constexpr uint32_t bs_threads() { return 256u + bs_b_units<NT>() + 32u + kEpiThreads; }
template <int NT>
__host__ __device__ constexpr size_t bs_smem_bytes() {
    return (size_t)bs_stages<NT>() * bs_stage_bytes() + 2u * (size_t)bs_b_bytes<NT>() +
           (size_t)bs_raw_depth<NT>() * 256u * 64u + (size_t)bs_b_units<NT>() * 64u + 8u * 32u;
}

template <int NT>
__global__ void __launch_bounds__(bs_threads<NT>(), 1) gemm_tc_bs_kernel(GemmArgs ga) {
    constexpr uint32_t S = bs_stages<NT>();
    constexpr uint32_t NA = bs_accs<NT>();
    constexpr uint32_t PA = 256u, PB = bs_b_units<NT>();
    constexpr uint32_t kMmaWarp = (PA + PB) / 32u;
    constexpr uint32_t kCols = NT < 32 ? 32u : (uint32_t)NT;
    constexpr uint32_t kRegA = region_bytes(kRows), kRegB = region_bytes(NT);
    constexpr uint32_t kStage = bs_stage_bytes(), kBChunk = bs_b_bytes<NT>();
    constexpr uint32_t kW = epi_cols<NT>();
    constexpr uint32_t kNc = (uint32_t)NT / 2u;
    constexpr uint32_t kRaw = bs_raw_depth<NT>();
    constexpr uint32_t kRawSlotA = PA * 64u;
    extern __shared__ __align__(1024) unsigned char gsm[];
    __shared__ __align__(8) uint64_t full_bar[S], empty_bar[S], accf_bar[NA], acce_bar[NA], bfull_bar, bempty_bar, drain_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int fail;
    const GemmStep &g = ga.g;
    const uint32_t warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const uint32_t sbase = smem_u32(gsm);
    unsigned char *sB = gsm + S * kStage;                          // resident B, one region set per chunk
    unsigned char *rawA = sB + 2u * kBChunk;
    unsigned char *rawB = rawA + kRaw * kRawSlotA;
    uint32_t *tka = reinterpret_cast<uint32_t *>(rawB + PB * 64u);
    uint32_t *tkb = tka + 2u * kKq;
    // this CTA's contiguous range of tiles
    const uint64_t t0 = (uint64_t)blockIdx.x * ga.n_tiles / gridDim.x;
    const uint64_t t1 = ((uint64_t)blockIdx.x + 1u) * ga.n_tiles / gridDim.x;
    if (threadIdx.x == 0) {
        for (uint32_t s = 0; s < S; s++) {
            mbar_init(smem_u32(&full_bar[s]), PA);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        for (uint32_t b = 0; b < NA; b++) {
            mbar_init(smem_u32(&accf_bar[b]), 1);
            mbar_init(smem_u32(&acce_bar[b]), kEpiThreads);
        }
        mbar_init(smem_u32(&bfull_bar), PB);
        mbar_init(smem_u32(&bempty_bar), 1);
        mbar_init(smem_u32(&drain_bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fail = 0;
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(NA * kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    const uint32_t K = ga.n_chunks * kKq;   // 16 or 32 table entries
    for (uint32_t i = threadIdx.x; i < K; i += bs_threads<NT>()) {
        tka[i] = pext_runs(i, g.ak, g.n_ak);
        tkb[i] = pext_runs(i, g.bk, g.n_bk);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const bool k8 = (1u << g.nk) < kKq;   // 8 summed entries: the second half of the chunk is zero
    if (warp < PA / 32u) {
        // A producers: unit u is row u & 127 of the tile, summed half u >> 7
        const uint32_t u = threadIdx.x;
        const uint32_t row = u & 127u, h = u >> 7;
        const bool pad = k8 && h == 1u;
        const uint32_t *koff = tka + 8u * h;
        const uint32_t raw_mine = smem_u32(rawA) + u * 8u;
        uint64_t lt = t0;
        uint32_t lc = 0;
        const float2 *src = nullptr;
        BsCursor cur;
        cur.c = tile_coord_bs(t0, ga);
        auto setup = [&]() {
            const TileCoord &tc = cur.c;
            const float2 *arena = ga.arenas + (uint64_t)tc.il * ga.a.arena_elems;
            src = gemm_operand(ga.a, arena, g.a_off, g.flags & kStepALeaf, ga.item0 + tc.il) +
                  pext_runs(tc.beta, g.ab, g.n_ab) + pext_runs(tc.mt * kRows + row, g.am, g.n_am);
        };
        auto issue_next = [&](uint64_t gi) {
            if (lt < t1 && !pad) {
                const uint32_t dst = raw_mine + (uint32_t)(gi % kRaw) * kRawSlotA;
                const uint4 o0 = *reinterpret_cast<const uint4 *>(koff + lc * kKq);
                const uint4 o1 = *reinterpret_cast<const uint4 *>(koff + lc * kKq + 4u);
                const uint32_t o[8] = {o0.x, o0.y, o0.z, o0.w, o1.x, o1.y, o1.z, o1.w};
#pragma unroll
                for (uint32_t j = 0; j < 8; j++) cp_async8(dst + j * PA * 8u, src + o[j]);
            }
            if (lt < t1) {
                if (++lc == ga.n_chunks) {
                    lc = 0;
                    if (++lt < t1) {
                        cur.next(ga);
                        setup();
                    }
                }
            }
            cp_async_commit();
        };
        if (t0 < t1) setup();
        const uint64_t total = (t1 - t0) * ga.n_chunks;
        for (uint32_t i = 0; i + 1 < kRaw; i++) issue_next(i);
        for (uint64_t gc = 0; gc < total && !fail; gc++) {
            issue_next(gc + kRaw - 1);
            cp_async_wait<kRaw - 1>();
            const uint32_t s = (uint32_t)(gc % S);
            if (!wait_or_fail(smem_u32(&empty_bar[s]), (uint32_t)((gc / S) & 1u) ^ 1u, &fail)) {
                fail = 1;
                break;
            }
            const float2 *rt = reinterpret_cast<const float2 *>(rawA + (gc % kRaw) * kRawSlotA) + u;
            float2 v[8];
#pragma unroll
            for (uint32_t j = 0; j < 8; j++) v[j] = pad ? make_float2(0.f, 0.f) : rt[j * PA];
            store_a(gsm + s * kStage, v, row, h);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&full_bar[s])) : "memory");
        }
        cp_async_wait<0>();
    } else if (warp < kMmaWarp) {
        // B producers: unit v is complex column v % (NT/2) of the column tile, summed half
        // (v / (NT/2)) & 1; once per column tile of the range, every chunk into its region
        const uint32_t v = threadIdx.x - PA;
        const bool active = v < (uint32_t)NT;
        const uint32_t col = v % kNc, h = (v / kNc) & 1u;
        const bool pad = k8 && h == 1u;
        const uint32_t *koff = tkb + 8u * h;
        const uint32_t raw_mine = smem_u32(rawB) + v * 8u;
        uint32_t gi = 0;
        BsCursor cur;
        cur.c = tile_coord_bs(t0, ga);
        for (uint64_t t = t0; t < t1 && !fail; gi++) {
            const uint64_t grp = t >> ga.mt_bits;
            if (!wait_or_fail(smem_u32(&bempty_bar), (gi & 1u) ^ 1u, &fail)) {
                fail = 1;
                break;
            }
            if (active) {
                const TileCoord &tc = cur.c;
                const float2 *arena = ga.arenas + (uint64_t)tc.il * ga.a.arena_elems;
                const float2 *src = gemm_operand(ga.a, arena, g.b_off, g.flags & kStepBLeaf, ga.item0 + tc.il) +
                                    pext_runs(tc.beta, g.bb, g.n_bb) + pext_runs(tc.nt * kNc + col, g.bn, g.n_bn);
                for (uint32_t c = 0; c < ga.n_chunks; c++) {
                    if (!pad) {
                        const uint4 o0 = *reinterpret_cast<const uint4 *>(koff + c * kKq);
                        const uint4 o1 = *reinterpret_cast<const uint4 *>(koff + c * kKq + 4u);
                        const uint32_t o[8] = {o0.x, o0.y, o0.z, o0.w, o1.x, o1.y, o1.z, o1.w};
#pragma unroll
                        for (uint32_t j = 0; j < 8; j++) cp_async8(raw_mine + j * PB * 8u, src + o[j]);
                    }
                    cp_async_commit();
                    cp_async_wait<0>();
                    const float2 *rt = reinterpret_cast<const float2 *>(rawB) + v;
                    float2 e[8];
#pragma unroll
                    for (uint32_t j = 0; j < 8; j++) e[j] = pad ? make_float2(0.f, 0.f) : rt[j * PB];
                    store_b<NT>(sB + c * kBChunk, e, col, h);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bfull_bar)) : "memory");
            t = (grp + 1u) << ga.mt_bits;   // the next column tile's first row tile
            cur.next_group(ga);
        }
        cp_async_wait<0>();
    } else if (warp == kMmaWarp) {
        if (lane == 0) {
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NT >> 3) << 17) |
                                   ((kRows >> 4) << 24);
            uint64_t gc = 0;
            uint32_t j = 0, gi = 0;
            bool ok = true;
            for (uint64_t t = t0; t < t1 && !fail && ok; t++, j++) {
                const uint64_t grp = t >> ga.mt_bits;
                if (t == t0 || (t & (ga.n_mt - 1u)) == 0u) {   // a new column tile: its B is loaded
                    if (!wait_or_fail(smem_u32(&bfull_bar), gi & 1u, &fail)) {
                        ok = false;
                        break;
                    }
                    gi++;
                }
                const uint32_t buf = j % NA;
                if (!wait_or_fail(smem_u32(&acce_bar[buf]), ((j / NA) & 1u) ^ 1u, &fail)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + buf * kCols;
                for (uint32_t c = 0; c < ga.n_chunks; c++, gc++) {
                    const uint32_t s = (uint32_t)(gc % S);
                    if (!wait_or_fail(smem_u32(&full_bar[s]), (uint32_t)((gc / S) & 1u), &fail)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = sbase + s * kStage, sb = smem_u32(sB) + c * kBChunk;
#pragma unroll
                    for (uint32_t p = 0; p < 2; p++) {
                        uint64_t ad[3], bd[3];
#pragma unroll
                        for (uint32_t q = 0; q < 3; q++) {
                            ad[q] = smem_desc(sa + (3u * p + q) * kRegA, 128u, kPitch);
                            bd[q] = smem_desc(sb + (3u * p + q) * kRegB, 128u, kPitch);
                        }
                        mma_bf16(d, ad[0], bd[0], idesc, (c | p) != 0u);
                        mma_bf16(d, ad[0], bd[1], idesc, 1u);
                        mma_bf16(d, ad[1], bd[0], idesc, 1u);
                        mma_bf16(d, ad[0], bd[2], idesc, 1u);
                        mma_bf16(d, ad[2], bd[0], idesc, 1u);
                        mma_bf16(d, ad[1], bd[1], idesc, 1u);
                    }
                    mma_commit(smem_u32(&empty_bar[s]));
                }
                if (!ok) break;
                mma_commit(smem_u32(&accf_bar[buf]));
                // the column tile's last row tile in this range: its B regions may be reloaded
                // once these MMAs have completed
                if (t + 1u == t1 || ((t + 1u) >> ga.mt_bits) != grp) mma_commit(smem_u32(&bempty_bar));
            }
            if (!ok) fail = 1;
            mma_commit(smem_u32(&drain_bar));
            if (!mbar_wait(smem_u32(&drain_bar), 0, kPolls)) fail = 1;
        }
        __syncwarp();
    } else {
        const uint32_t q = warp & 3u;
        const uint32_t share = (warp - kMmaWarp - 1u) >> 2;
        uint32_t j = 0;
        BsCursor cur;
        cur.c = tile_coord_bs(t0, ga);
        for (uint64_t t = t0; t < t1 && !fail; t++, j++, cur.next(ga)) {
            const TileCoord &tc = cur.c;
            const uint32_t buf = j % NA;
            float2 *Crow = ga.arenas + (uint64_t)tc.il * ga.a.arena_elems + g.c_off + pext_runs(tc.beta, g.cb, g.n_cb) +
                           pext_runs(tc.mt * kRows + 32u * q + lane, g.cm, g.n_cm);
            if (!wait_or_fail(smem_u32(&accf_bar[buf]), (j / NA) & 1u, &fail)) {
                fail = 1;
                break;
            }
            tc_fence_after();
            const uint32_t taddr = tmem + ((q * 32u) << 16) + buf * kCols;
            for (uint32_t j0 = share * kW; j0 < (uint32_t)NT; j0 += 2u * kW) {
                const uint32_t my_col = pext_runs(tc.nt * kNc + j0 / 2u + (lane % (kW / 2u)), g.cn, g.n_cn);
                uint32_t r[kW];
                tmem_ld<kW>(taddr + j0, r);
#pragma unroll
                for (uint32_t i = 0; i < kW / 2u; i++) {
                    const uint32_t coff = __shfl_sync(0xffffffffu, my_col, i);
                    Crow[coff] = make_float2(__uint_as_float(r[2u * i]), __uint_as_float(r[2u * i + 1u]));
                }
            }
            tc_fence_before();
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce_bar[buf])) : "memory");
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NA * kCols) : "memory");
    }
    if (fail && threadIdx.x == 0) atomicCAS(ga.a.status, 0u, 4u /* QVX_ETIMEOUT */);
}

}  // namespace

// real columns of a tile: two per complex column, up to 128 complex columns
uint32_t gemm_nt(const GemmStep &g) { return g.nn >= 7 ? 256u : (2u << g.nn); }

// Grid of a persistent tensor-core kernel: the SM count times the CTAs an SM holds (within
// its 512 tensor-memory columns, so that no allocation ever waits for another CTA's
// columns), queried once per device and kernel (under a lock: host threads may launch on
// several streams at once).
template <int NT, bool kBs>
static cudaError_t gemm_grid(uint64_t n_tiles, uint64_t *grid) {
    static int per_sm[64] = {0}, sms[64] = {0};
    static std::mutex mu;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!per_sm[dev]) {
        const void *fn = kBs ? reinterpret_cast<const void *>(gemm_tc_bs_kernel<NT>)
                             : reinterpret_cast<const void *>(gemm_tc_kernel<NT>);
        const size_t smem = kBs ? bs_smem_bytes<NT>() : smem_bytes<NT>(1024);
        const int threads = kBs ? (int)bs_threads<NT>() : (int)block_threads<NT>();
        if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
        int n = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, smem)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        const int cols = kBs ? (int)(bs_accs<NT>() * bs_cols<NT>()) : 2 * (NT < 32 ? 32 : NT);
        per_sm[dev] = n < 1 ? -1 : std::min(n, 512 / cols);
    }
    if (per_sm[dev] < 1) return cudaErrorInvalidConfiguration;
    *grid = std::min<uint64_t>(n_tiles, (uint64_t)sms[dev] * (uint64_t)per_sm[dev]);
    return cudaSuccess;
}

template <int NT>
static cudaError_t launch_gemm_nt(GemmArgs ga, cudaStream_t s) {
    ga.n_tiles = ((uint64_t)ga.n_items << ga.g.nb) * ga.n_mt * ga.n_nt;
    if (ga.n_tiles == 0) return cudaErrorInvalidConfiguration;
    uint64_t grid = 0;
    cudaError_t e;
    // B-stationary form: at most two chunks of summed entries (B's regions of every chunk
    // stay resident) and at least 4 row tiles per column tile to reuse them over (with 2, the
    // reload between column tiles, which waits for the old tile's MMAs, cost more than the
    // reuse saved; tile coordinates above the row tiles within 32 bits)
    if (ga.n_chunks <= 2u && ga.n_mt >= 4u && (uint64_t)ga.n_items * ga.n_nt < (1ull << 32)) {
        if ((e = gemm_grid<NT, true>(ga.n_tiles, &grid)) != cudaSuccess) return e;
        gemm_tc_bs_kernel<NT><<<(unsigned)grid, bs_threads<NT>(), bs_smem_bytes<NT>(), s>>>(ga);
        return cudaGetLastError();
    }
    // dynamic shared memory: the operand stage ring, the producers' raw copy slots and the
    // summed index tables, sized for the largest summed index (1024 entries)
    if ((e = gemm_grid<NT, false>(ga.n_tiles, &grid)) != cudaSuccess) return e;
    gemm_tc_kernel<NT><<<(unsigned)grid, block_threads<NT>(), smem_bytes<NT>(1024), s>>>(ga);
    return cudaGetLastError();
}

cudaError_t launch_gemm_step(const LaunchArgs &a, const GemmStep &g, int64_t item0, int64_t n_items, float2 *arenas,
                             cudaStream_t s) {
    if (g.nk < 3 || g.nk > 10 || g.nm < 7 || g.nn < 3 || n_items <= 0) return cudaErrorInvalidConfiguration;
    const uint32_t nt_cols = gemm_nt(g);
    GemmArgs ga;
    ga.a = a;
    ga.g = g;
    ga.item0 = item0;
    ga.n_items = n_items;
    ga.arenas = arenas;
    ga.n_chunks = std::max(1u, (1u << g.nk) / kKq);   // 8 summed entries: one half-filled chunk
    ga.n_mt = (1u << g.nm) / kRows;
    ga.n_nt = (2u << g.nn) / nt_cols;
    ga.mt_bits = (uint32_t)__builtin_ctz(ga.n_mt);
    ga.nt_bits = (uint32_t)__builtin_ctz(ga.n_nt);
    ga.n_tiles = 0;
    cudaError_t e;
    switch (nt_cols) {
        case 16: e = launch_gemm_nt<16>(ga, s); break;
        case 32: e = launch_gemm_nt<32>(ga, s); break;
        case 64: e = launch_gemm_nt<64>(ga, s); break;
        case 128: e = launch_gemm_nt<128>(ga, s); break;
        default: e = launch_gemm_nt<256>(ga, s); break;
    }
    return launch_counted(e);
}

}  // namespace qvx
