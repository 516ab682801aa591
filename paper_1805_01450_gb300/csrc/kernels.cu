// Device kernels: the pairwise contraction program (fused and stepwise engines) and the
// exact (fixed-point) sum of the slice terms.
#include <cuda_runtime.h>

#include <algorithm>

#include "device_program.h"
#include "device_util.cuh"
#include "kernels.h"

namespace qvx {
namespace {

__device__ __forceinline__ void cmac(float2 &acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}

// One output entry c of step st.
__device__ __forceinline__ float2 step_entry(const DevStep &st, uint32_t c, const float2 *A,
                                             const float2 *B, bool unary) {
    const uint32_t ia = pext_runs(c, st.runs_a, st.na_runs);
    const uint32_t ib = unary ? 0u : pext_runs(c, st.runs_b, st.nb_runs);
    const uint32_t nab = st.nk_ab, na = st.nk_a;
    const uint32_t nk = nab + na + st.nk_b;
    const uint32_t mask_ka = (1u << (nab + na)) - 1u, mask_ab = (1u << nab) - 1u;
    float2 acc = make_float2(0.f, 0.f);
    for (uint32_t k = 0; k < (1u << nk); k++) {
        const uint32_t ka = k & mask_ka;
        const float2 a = A[ia + (ka << st.a_cb)];
        if (unary) {
            acc.x += a.x;
            acc.y += a.y;
        } else {
            const uint32_t kb = (k & mask_ab) | ((k >> (nab + na)) << nab);
            cmac(acc, a, B[ib + (kb << st.b_cb)]);
        }
    }
    return acc;
}

// ------------------------------------------------------------------ exact sums
// FP64 arithmetic has long latency on this GPU, so the slice terms are added as
// fixed-point integers: a complex64 term t becomes X = t * 2^100 (128-bit, exact for
// 2^-77 <= |t| < 2^27; smaller magnitudes lose only bits below 2^-100), integers add
// exactly and in any order, and each sum is rounded to FP64 once.
struct Fx {
    unsigned long long lo;
    long long hi;
};

constexpr unsigned kStatusRange = 6u;   // QVX_ERANGE

// X = t * 2^100 as a 128-bit integer. A term that is not finite or has |t| >= 2^27 has no
// such form: it contributes nothing and sets `bad`, which the caller reports as QVX_ERANGE.
__device__ __forceinline__ Fx fx_from_float(float f, bool &bad) {
    const uint32_t bits = __float_as_uint(f);
    uint32_t e = (bits >> 23) & 0xffu;
    unsigned long long m = bits & 0x7fffffu;
    Fx r;
    r.lo = 0;
    r.hi = 0;
    if (e >= 154u) {                   // |t| >= 2^27, infinite or NaN
        bad = true;
        return r;
    }
    if (e) m |= 0x800000u;
    else e = 1;
    const int sh = (int)e - 50;        // t = m 2^(e-150), X = m 2^(e-50); sh <= 103
    if (sh >= 64) {
        r.hi = (long long)(m << (sh - 64));
    } else if (sh > 0) {
        r.lo = m << sh;
        r.hi = (long long)(m >> (64 - sh));
    } else if (sh > -64) {
        r.lo = m >> (-sh);
    }
    if (bits >> 31) {                  // two's-complement negation
        r.lo = ~r.lo + 1ull;
        r.hi = (long long)(~(unsigned long long)r.hi + (r.lo == 0 ? 1ull : 0ull));
    }
    return r;
}

// a + b; a sum outside the 128-bit range (|a + b| >= 2^27) sets `bad`: the operands have
// the same sign and the result's sign differs.
__device__ __forceinline__ Fx fx_add(Fx a, Fx b, bool &bad) {
    Fx r;
    r.lo = a.lo + b.lo;
    r.hi = (long long)((unsigned long long)a.hi + (unsigned long long)b.hi + (r.lo < a.lo ? 1ull : 0ull));
    bad |= ((a.hi ^ r.hi) & (b.hi ^ r.hi)) < 0;
    return r;
}

__device__ __forceinline__ Fx fx_shfl_down(Fx a, int d) {
    Fx r;
    r.lo = __shfl_down_sync(0xffffffffu, a.lo, d);
    r.hi = __shfl_down_sync(0xffffffffu, a.hi, d);
    return r;
}

__device__ __forceinline__ double fx_to_double(Fx a) {
    // X = hi 2^64 + lo with lo unsigned; value = X 2^-100
    return __ll2double_rn(a.hi) * 0x1p-36 + __ull2double_rn(a.lo) * 0x1p-100;
}

__device__ __forceinline__ ExactPair fx_pair(Fx re, Fx im) {
    ExactPair p;
    p.re_lo = re.lo;
    p.re_hi = (unsigned long long)re.hi;
    p.im_lo = im.lo;
    p.im_hi = (unsigned long long)im.hi;
    return p;
}

// Block-wide exact sum of the pairs at p[0..n) (written by other CTAs: read through L2),
// rounded to FP64 and times the scalar (sr, si); the result is valid in thread 0. A sum
// outside the exact range sets QVX_ERANGE in the status word; the result is NaN then, and
// also when the status word was already set (an earlier kernel of the call failed).
__device__ double2 block_exact_sum(const ExactPair *p, int64_t n, double sr, double si, unsigned *status) {
    __shared__ Fx red[2][32];
    Fx re = {0ull, 0ll}, im = {0ull, 0ll};
    bool bad = false;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const ulonglong2 a = __ldcg(reinterpret_cast<const ulonglong2 *>(p + i));
        const ulonglong2 b = __ldcg(reinterpret_cast<const ulonglong2 *>(p + i) + 1);
        re = fx_add(re, Fx{a.x, (long long)a.y}, bad);
        im = fx_add(im, Fx{b.x, (long long)b.y}, bad);
    }
    for (int d = 16; d > 0; d >>= 1) {
        re = fx_add(re, fx_shfl_down(re, d), bad);
        im = fx_add(im, fx_shfl_down(im, d), bad);
    }
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
    __syncthreads();
    if (lane == 0) {
        red[0][warp] = re;
        red[1][warp] = im;
    }
    bad = __syncthreads_or(bad) != 0;
    double2 out = make_double2(0.0, 0.0);
    if (threadIdx.x == 0) {
        for (int w = 1; w < nw; w++) {
            re = fx_add(re, red[0][w], bad);
            im = fx_add(im, red[1][w], bad);
        }
        if (bad) atomicCAS(status, 0u, kStatusRange);
        if (bad || *reinterpret_cast<volatile unsigned *>(status) != 0u) {
            out = make_double2(__longlong_as_double(0x7ff8000000000000ll), __longlong_as_double(0x7ff8000000000000ll));
        } else {
            const double r = fx_to_double(re), i = fx_to_double(im);
            out = make_double2(r * sr - i * si, r * si + i * sr);
        }
    }
    return out;
}

// Header fields the item epilogue needs, read once per kernel.
struct FinishInfo {
    uint64_t zero_mask, zero_mask_hi;
    double sr, si;
    uint32_t n_in, present;        // inner slice modes and those present in the final tensor
    uint32_t n_open, open_present; // open output qubits and those present
};

__device__ __forceinline__ FinishInfo finish_info(const DevProgram *P) {
    FinishInfo f;
    f.zero_mask = P->zero_mask;
    f.zero_mask_hi = P->zero_mask_hi;
    f.sr = P->scalar_re;
    f.si = P->scalar_im;
    f.n_in = P->n_inner;
    f.present = P->final_present;
    f.n_open = P->n_open;
    f.open_present = P->open_present;
    return f;
}

__device__ __forceinline__ uint32_t compress_bits(uint32_t v, uint32_t mask, uint32_t n) {
    uint32_t r = 0, bit = 0;
    for (uint32_t j = 0; j < n; j++)
        if ((mask >> j) & 1u) r |= ((v >> j) & 1u) << bit++;
    return r;
}

// For each value j of the open outputs: the exact sum of the inner slice terms of the
// item's final tensor that fall in [s_begin, s_end) (before the plan's scalar), one warp;
// partial of output slot (b, j) for outer slice o. Optionally writes each term (times the
// scalar) at terms[slot * (s_end - s_begin) + s - s_begin].
template <bool CG>
__device__ void finish_item_t(const FinishInfo &P, const LaunchArgs &a, const float2 *fin, int64_t b, uint64_t o,
                              int lane, const Bits &x) {
    const bool zero = bits_hit(x, P.zero_mask, P.zero_mask_hi);
    const uint32_t n_in = P.n_in, present = P.present;
    const uint32_t inner_bits = __popc(present);
    for (uint32_t j = 0; j < (1u << P.n_open); j++) {
        const uint32_t fj = compress_bits(j, P.open_present, P.n_open) << inner_bits;
        const int64_t slot = (b << P.n_open) + j;
        Fx re = {0ull, 0ll}, im = {0ull, 0ll};
        bool bad = false;
        for (uint32_t i = lane; i < (1u << n_in); i += 32) {
            const int64_t s = (int64_t)((o << n_in) | i);
            if (s < a.s_begin || s >= a.s_end) continue;
            const uint32_t fi = compress_bits(i, present, n_in) | fj;
            const float2 t = zero ? make_float2(0.f, 0.f) : (CG ? __ldcg(fin + fi) : fin[fi]);
            re = fx_add(re, fx_from_float(t.x, bad), bad);
            im = fx_add(im, fx_from_float(t.y, bad), bad);
            if (a.terms) {
                const double tr = (double)t.x * P.sr - (double)t.y * P.si;
                const double ti = (double)t.x * P.si + (double)t.y * P.sr;
                a.terms[slot * (a.s_end - a.s_begin) + (s - a.s_begin)] = make_float2((float)tr, (float)ti);
            }
        }
        for (int d = 16; d > 0; d >>= 1) {
            re = fx_add(re, fx_shfl_down(re, d), bad);
            im = fx_add(im, fx_shfl_down(im, d), bad);
        }
        if (bad) atomicCAS(a.status, 0u, kStatusRange);
        if (lane == 0) a.partials[slot * a.o_count + (int64_t)(o - (uint64_t)a.o_begin)] = fx_pair(re, im);
    }
}

__device__ __forceinline__ void finish_item(const FinishInfo &P, const LaunchArgs &a, const float2 *fin, int64_t b,
                                            uint64_t o, int lane, int) {
    finish_item_t<false>(P, a, fin, b, o, lane, load_bits(a.bitstrings, b, a.words));
}

__device__ __forceinline__ void finish_item_cg(const FinishInfo &P, const LaunchArgs &a, const float2 *fin, int64_t b,
                                               uint64_t o, int lane) {
    finish_item_t<true>(P, a, fin, b, o, lane, load_bits(a.bitstrings, b, a.words));
}

// ------------------------------------------------------------------ fused engine
// Each group of `warps_per_item` warps runs the whole program for one work item
// (bitstring b, outer slice o); groups loop over items. Shared memory holds, per CTA, the
// program and the leaf data (when they fit), and per group the item's leaf base offsets
// and its tensor arena.

// One output entry of a fused step: e packs the operands' offsets pext(c); the summed
// index's offsets come from the step's koff tables (nk <= 3) or from its bit counts.
__device__ __forceinline__ float2 fused_entry(const FusedStep &st, uint32_t e, const float2 *__restrict__ A,
                                              const float2 *__restrict__ B, bool unary) {
    const uint32_t ia = e & 0xffffu, ib = e >> 16;
    float2 acc = make_float2(0.f, 0.f);
    if (st.nk <= 3) {
        const uint32_t nk = 1u << st.nk;
#pragma unroll
        for (uint32_t k = 0; k < 8; k++) {   // constant indices keep koff in registers
            if (k < nk) {
                if (unary) {
                    const float2 v = A[ia + st.koff_a[k]];
                    acc.x += v.x;
                    acc.y += v.y;
                } else {
                    cmac(acc, A[ia + st.koff_a[k]], B[ib + st.koff_b[k]]);
                }
            }
        }
        return acc;
    }
    const uint32_t nab = st.nk_ab, na = st.nk_a;
    const uint32_t mask_ka = (1u << (nab + na)) - 1u, mask_ab = (1u << nab) - 1u;
    for (uint32_t k = 0; k < (1u << st.nk); k++) {
        const uint32_t ka = k & mask_ka;
        if (unary) {
            const float2 v = A[ia + (ka << st.a_cb)];
            acc.x += v.x;
            acc.y += v.y;
        } else {
            const uint32_t kb = (k & mask_ab) | ((k >> (nab + na)) << nab);
            cmac(acc, A[ia + (ka << st.a_cb)], B[ib + (kb << st.b_cb)]);
        }
    }
    return acc;
}

// Entries c = sub, sub + cnt, ... < n_out of a two-operand step with 2^NK summed entries
// (NK = 2 or 3), two entries at a time: all operand loads of both are issued before the
// multiply-adds.
template <int NK>
__device__ __forceinline__ void lane_entries_k(const FusedStep &st, uint32_t sub, uint32_t cnt, uint32_t n_out,
                                               const uint32_t *tab, const float2 *__restrict__ A,
                                               const float2 *__restrict__ B, float2 *C) {
    constexpr int K = 1 << NK;
    uint32_t ka[K], kb[K];
#pragma unroll
    for (int k = 0; k < K; k++) {
        ka[k] = st.koff_a[k];
        kb[k] = st.koff_b[k];
    }
    uint32_t c = sub;
    for (; c + cnt < n_out; c += 2 * cnt) {
        const uint32_t e0 = tab[c], e1 = tab[c + cnt];
        const uint32_t ia0 = e0 & 0xffffu, ib0 = e0 >> 16, ia1 = e1 & 0xffffu, ib1 = e1 >> 16;
        float2 p0[K], q0[K], p1[K], q1[K];
#pragma unroll
        for (int k = 0; k < K; k++) {
            p0[k] = A[ia0 + ka[k]];
            q0[k] = B[ib0 + kb[k]];
            p1[k] = A[ia1 + ka[k]];
            q1[k] = B[ib1 + kb[k]];
        }
        float2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < K; k++) {
            cmac(acc0, p0[k], q0[k]);
            cmac(acc1, p1[k], q1[k]);
        }
        C[c] = acc0;
        C[c + cnt] = acc1;
    }
    if (c < n_out) {
        const uint32_t e = tab[c], ia = e & 0xffffu, ib = e >> 16;
        float2 p[K], q[K];
#pragma unroll
        for (int k = 0; k < K; k++) {
            p[k] = A[ia + ka[k]];
            q[k] = B[ib + kb[k]];
        }
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < K; k++) cmac(acc, p[k], q[k]);
        C[c] = acc;
    }
}

constexpr uint32_t kWaitPolls = 1u << 20;

// The work of one lane in one phase: its step, operand bases and entry stride.
struct LaneWork {
    const FusedStep *stp;          // the step (its summed-index tables, for nk >= 2)
    const float2 *A, *B;
    float2 *C;
    const uint32_t *tab;
    uint32_t sub, cnt;
    uint32_t info;                 // bits 0-7: output rank, 8-15: summed modes, 16: one operand
    uint32_t k1;                   // offsets of summed entry 1 in A (low 16 bits) and B (high)
    bool active;
};

template <bool STAGED>
__device__ __forceinline__ LaneWork lane_work(uint32_t m, const FusedStep *steps, const uint32_t *tabs,
                                              const float2 *ldata, const uint32_t *lbase, float2 *arena) {
    LaneWork w;
    w.active = m != 0xffffffffu;
    if (!w.active) return w;
    // 16-byte shared-memory loads of the fields used here; summed entry 0 is at offset 0 in
    // both operands, entry 1's offsets ride along, the rest stay in the step
    w.stp = steps + (m & 0xfffu);
    const uint4 *src = reinterpret_cast<const uint4 *>(w.stp);
    const uint4 v0 = src[0], v1 = src[1], v2 = src[2], v3 = src[3];
    const uint32_t a_off = v0.x, b_off = v0.y, c_off = v0.z, tab_off = v0.w, flags = v1.x;
    w.info = (v1.y & 0xffu) | (((v1.z >> 16) & 0xffu) << 8) | ((flags & kStepUnary) << 16);
    w.k1 = (v2.x >> 16) | (v3.x & 0xffff0000u);
    w.sub = (m >> 12) & 0x3ffu;
    w.cnt = m >> 22;
    w.A = (flags & kStepALeaf) ? ldata + lbase[a_off] : arena + a_off;
    w.B = (flags & kStepUnary) ? w.A : ((flags & kStepBLeaf) ? ldata + lbase[b_off] : arena + b_off);
    w.C = arena + c_off;
    w.tab = tabs + tab_off;
    return w;
}

// The lane's entries of its step, with the summed-index loop unrolled by case.
__device__ __forceinline__ void run_lane_work(const LaneWork &w) {
    const uint32_t n_out = 1u << (w.info & 0xffu), nk = (w.info >> 8) & 0xffu;
    const bool unary = (w.info >> 16) & 1u;
    const float2 *__restrict__ A = w.A;
    const float2 *__restrict__ B = w.B;
    const uint32_t ka1 = w.k1 & 0xffffu, kb1 = w.k1 >> 16;
    // two entries per iteration: independent loads and FMA chains overlap
    if (!unary && nk == 0) {
        uint32_t c = w.sub;
        for (; c + w.cnt < n_out; c += 2 * w.cnt) {
            const uint32_t e0 = w.tab[c], e1 = w.tab[c + w.cnt];
            const float2 a0 = A[e0 & 0xffffu], b0 = B[e0 >> 16];
            const float2 a1 = A[e1 & 0xffffu], b1 = B[e1 >> 16];
            w.C[c] = make_float2(a0.x * b0.x - a0.y * b0.y, a0.x * b0.y + a0.y * b0.x);
            w.C[c + w.cnt] = make_float2(a1.x * b1.x - a1.y * b1.y, a1.x * b1.y + a1.y * b1.x);
        }
        if (c < n_out) {
            const uint32_t e = w.tab[c];
            const float2 a = A[e & 0xffffu], b = B[e >> 16];
            w.C[c] = make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
        }
    } else if (!unary && nk == 1) {
        uint32_t c = w.sub;
        for (; c + 3 * w.cnt < n_out; c += 4 * w.cnt) {   // four entries: loads of all issued first
            uint32_t e[4];
            float2 p[4], q[4], r[4], t[4];
#pragma unroll
            for (int u = 0; u < 4; u++) e[u] = w.tab[c + u * w.cnt];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const uint32_t ia = e[u] & 0xffffu, ib = e[u] >> 16;
                p[u] = A[ia];
                q[u] = B[ib];
                r[u] = A[ia + ka1];
                t[u] = B[ib + kb1];
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                float2 acc = make_float2(0.f, 0.f);
                cmac(acc, p[u], q[u]);
                cmac(acc, r[u], t[u]);
                w.C[c + u * w.cnt] = acc;
            }
        }
        for (; c + w.cnt < n_out; c += 2 * w.cnt) {
            const uint32_t e0 = w.tab[c], e1 = w.tab[c + w.cnt];
            const uint32_t ia0 = e0 & 0xffffu, ib0 = e0 >> 16, ia1 = e1 & 0xffffu, ib1 = e1 >> 16;
            const float2 p0 = A[ia0], q0 = B[ib0], p1 = A[ia0 + ka1], q1 = B[ib0 + kb1];
            const float2 r0 = A[ia1], s0 = B[ib1], r1 = A[ia1 + ka1], s1 = B[ib1 + kb1];
            float2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
            cmac(acc0, p0, q0);
            cmac(acc1, r0, s0);
            cmac(acc0, p1, q1);
            cmac(acc1, r1, s1);
            w.C[c] = acc0;
            w.C[c + w.cnt] = acc1;
        }
        if (c < n_out) {
            const uint32_t e = w.tab[c], ia = e & 0xffffu, ib = e >> 16;
            const float2 a0 = A[ia], b0 = B[ib], a1 = A[ia + ka1], b1 = B[ib + kb1];
            float2 acc = make_float2(0.f, 0.f);
            cmac(acc, a0, b0);
            cmac(acc, a1, b1);
            w.C[c] = acc;
        }
    } else if (!unary && nk == 2) {
        lane_entries_k<2>(*w.stp, w.sub, w.cnt, n_out, w.tab, A, B, w.C);
    } else if (!unary && nk == 3) {
        lane_entries_k<3>(*w.stp, w.sub, w.cnt, n_out, w.tab, A, B, w.C);
    } else {
        for (uint32_t c = w.sub; c < n_out; c += w.cnt) w.C[c] = fused_entry(*w.stp, w.tab[c], A, B, unary);
    }
}

// STAGED: the fused steps with their tables and lane maps, the leaf data and the leaf
// table are copied into shared memory once per CTA by the TMA engine, and every operand
// access is a shared-memory access; otherwise the program is read from global memory.
// Header fields are read once into registers. Each phase's lane work is prepared one
// phase ahead, so a phase's critical path is its operand loads, FMAs, store and barrier.
template <bool STAGED>
__global__ void __launch_bounds__(512) fused_program_kernel(LaunchArgs a, int warps_per_item) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ __align__(8) uint64_t stage_bar;
    const unsigned char *img = a.image;
    const DevProgram *P = reinterpret_cast<const DevProgram *>(img);
    const uint64_t steps_off = a.fused_steps_off, tab_off = a.fused_tab_off, map_off = a.fused_lane_map_off;
    const uint32_t n_phases = a.n_fused_phases, n_leaves = a.n_leaves;
    const uint64_t final_off = a.final_off;
    const DevLeaf *leaves = reinterpret_cast<const DevLeaf *>(img + a.leaves_off);
    const FusedStep *steps = reinterpret_cast<const FusedStep *>(img + steps_off);
    const uint32_t *tabs = reinterpret_cast<const uint32_t *>(img + tab_off);
    const uint32_t *lane_map = reinterpret_cast<const uint32_t *>(img + map_off);
    const float2 *ldata = reinterpret_cast<const float2 *>(img + a.leaf_data_off);
    unsigned char *cur = smem;
    // the first item's bitstring is read while the program is being staged
    const int groups0 = blockDim.x / (32 * warps_per_item);
    const int64_t item0 = (int64_t)blockIdx.x * groups0 + threadIdx.x / (32 * warps_per_item);
    Bits x_next = item0 < a.batch * a.o_count ? load_bits(a.bitstrings, item0 / a.o_count, a.words) : Bits{0ull, 0ull};
    bool staged_ok = true;
    if (STAGED) {
        const uint32_t s1 = a.smem_steps_bytes, s2 = s1 + a.smem_leaf_bytes, s3 = s2 + a.smem_leaves_bytes;
        const uint32_t bar = smem_u32(&stage_bar);
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(s3) : "memory");
            if (s1) bulk_g2s(smem_u32(smem), steps, s1, bar);
            if (a.smem_leaf_bytes) bulk_g2s(smem_u32(smem + s1), ldata, a.smem_leaf_bytes, bar);
            if (a.smem_leaves_bytes) bulk_g2s(smem_u32(smem + s2), leaves, a.smem_leaves_bytes, bar);
        }
        __syncthreads();
        const bool ok = mbar_wait(bar, 0, a.selftest_stage_timeout ? 0u : kWaitPolls);
        if (__syncthreads_or(!ok)) {
            // the copy never completed: report it, give the copies in flight a last bounded
            // wait, skip the work items and still take this CTA's ticket below, so that the
            // last CTA runs (it writes NaN amplitudes and resets the counter)
            if (threadIdx.x == 0) atomicCAS(a.status, 0u, 4u /* QVX_ETIMEOUT */);
            mbar_wait(bar, 0, kWaitPolls);
            staged_ok = false;
        } else {
            steps = reinterpret_cast<const FusedStep *>(smem);
            tabs = reinterpret_cast<const uint32_t *>(smem + (tab_off - steps_off));
            lane_map = reinterpret_cast<const uint32_t *>(smem + (map_off - steps_off));
            ldata = reinterpret_cast<const float2 *>(smem + s1);
            leaves = reinterpret_cast<const DevLeaf *>(smem + s2);
            cur = smem + s3;
        }
    } else {
        __syncthreads();
    }
    const FinishInfo fin = finish_info(P);
    if (staged_ok) {
        const int lanes = 32 * warps_per_item;
        const int group = threadIdx.x / lanes;
        const int lane = threadIdx.x % lanes;
        const int groups = blockDim.x / lanes;
        unsigned char *mine = cur + (size_t)group * a.group_bytes;
        uint32_t *lbase = reinterpret_cast<uint32_t *>(mine);
        float2 *arena = reinterpret_cast<float2 *>(mine + a.leaf_table_bytes);
        const int64_t n_items = a.batch * a.o_count;
        const unsigned bar_id = 1 + group;
        for (int64_t item = (int64_t)blockIdx.x * groups + group; item < n_items;
             item += (int64_t)gridDim.x * groups) {
            const int64_t b = item / a.o_count;
            const uint64_t o = (uint64_t)(a.o_begin + item % a.o_count);
            const Bits x = x_next;
            const int64_t item_next = item + (int64_t)gridDim.x * groups;
            if (item_next < n_items) x_next = load_bits(a.bitstrings, item_next / a.o_count, a.words);
            for (uint32_t l = lane; l < n_leaves; l += lanes) lbase[l] = leaf_base(leaves[l], x, o);
            if (warps_per_item == 1) __syncwarp();
            else asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(lanes));
            LaneWork w = lane_work<STAGED>(n_phases ? lane_map[lane] : 0xffffffffu, steps, tabs, ldata, lbase, arena);
            for (uint32_t ph = 0; ph < n_phases; ph++) {
                const uint32_t m_next =
                    ph + 1 < n_phases ? lane_map[(ph + 1) * (uint32_t)lanes + (uint32_t)lane] : 0xffffffffu;
                const LaneWork next = lane_work<STAGED>(m_next, steps, tabs, ldata, lbase, arena);
                if (w.active) run_lane_work(w);
                if (warps_per_item == 1) __syncwarp();
                else asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(lanes));
                w = next;
            }
            if (lane < 32) finish_item_t<false>(fin, a, arena + final_off, b, o, lane, x);
            if (warps_per_item == 1) __syncwarp();
            else asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(lanes));
        }
    }
    if (a.amps == nullptr) return;
    // the last CTA to finish adds every bitstring's item partials (NaN when a kernel of this
    // call set the status word) and resets the counter for the next call
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned ticket = atomicAdd(a.counter, 1u);
        last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    // every other CTA fenced its partials before counting itself, and the loads below
    // depend on the count: they read the partials through L2
    for (int64_t slot = 0; slot < (a.batch << fin.n_open); slot++) {
        const double2 r = block_exact_sum(a.partials + slot * a.o_count, a.o_count, fin.sr, fin.si, a.status);
        if (threadIdx.x == 0) {
            a.amps[2 * slot] = r.x;
            a.amps[2 * slot + 1] = r.y;
        }
    }
    if (threadIdx.x == 0) *a.counter = 0u;
}

// ------------------------------------------------------------------ stepwise engine
__global__ void step_kernel(LaunchArgs a, uint32_t s_idx, int64_t item_begin, int64_t n_items,
                            float2 *arenas) {
    const unsigned char *img = a.image;
    const DevProgram *P = reinterpret_cast<const DevProgram *>(img);
    const DevStep &st = reinterpret_cast<const DevStep *>(img + P->steps_off)[s_idx];
    const uint64_t per = 1ull << st.rc;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= per * (uint64_t)n_items) return;
    const int64_t il = (int64_t)(tid >> st.rc);
    const uint32_t c = (uint32_t)(tid & (per - 1));
    const int64_t item = item_begin + il;
    const int64_t b = item / a.o_count;
    const uint64_t o = (uint64_t)(a.o_begin + item % a.o_count);
    const Bits x = load_bits(a.bitstrings, b, a.words);
    float2 *arena = arenas + (uint64_t)il * a.arena_elems;
    const bool unary = st.flags & kStepUnary;
    const DevLeaf *leaves = reinterpret_cast<const DevLeaf *>(img + P->leaves_off);
    const float2 *ldata = reinterpret_cast<const float2 *>(img + P->leaf_data_off);
    const float2 *A = (st.flags & kStepALeaf) ? ldata + leaf_base(leaves[st.a_off], x, o) : arena + st.a_off;
    const float2 *B = unary ? A
                            : ((st.flags & kStepBLeaf) ? ldata + leaf_base(leaves[st.b_off], x, o) : arena + st.b_off);
    arena[st.c_off + c] = step_entry(st, c, A, B, unary);
}

__global__ void step_group_kernel(LaunchArgs a, StepGroup g, int64_t item_begin, int64_t n_items, float2 *arenas) {
    uint32_t j = 0;
    while (j + 1 < g.n && blockIdx.x >= g.first_block[j + 1]) j++;
    const unsigned char *img = a.image;
    const DevProgram *P = reinterpret_cast<const DevProgram *>(img);
    const DevStep &st = reinterpret_cast<const DevStep *>(img + P->steps_off)[g.step[j]];
    const uint64_t per = 1ull << st.rc;
    const uint64_t tid = (uint64_t)(blockIdx.x - g.first_block[j]) * blockDim.x + threadIdx.x;
    if (tid >= per * (uint64_t)n_items) return;
    const int64_t il = (int64_t)(tid >> st.rc);
    const uint32_t c = (uint32_t)(tid & (per - 1));
    float2 *arena = arenas + (uint64_t)il * a.arena_elems;
    const bool unary = st.flags & kStepUnary;
    const DevLeaf *leaves = reinterpret_cast<const DevLeaf *>(img + P->leaves_off);
    const float2 *ldata = reinterpret_cast<const float2 *>(img + P->leaf_data_off);
    Bits x = {0ull, 0ull};
    uint64_t o = 0;
    if (st.flags & (kStepALeaf | kStepBLeaf)) {
        const int64_t item = item_begin + il;
        x = load_bits(a.bitstrings, item / a.o_count, a.words);
        o = (uint64_t)(a.o_begin + item % a.o_count);
    }
    const float2 *A = (st.flags & kStepALeaf) ? ldata + leaf_base(leaves[st.a_off], x, o) : arena + st.a_off;
    const float2 *B = unary ? A
                            : ((st.flags & kStepBLeaf) ? ldata + leaf_base(leaves[st.b_off], x, o) : arena + st.b_off);
    arena[st.c_off + c] = step_entry(st, c, A, B, unary);
}

// ------------------------------------------------------------------ persistent engine
constexpr uint32_t kBarrierPolls = 1u << 24;   // x ~64 ns sleeps: about a second

// Grid-wide barrier of a cooperative launch: thread 0 of each CTA arrives on a counter; the
// last arrival resets it and advances the generation, the others poll the generation with
// a bounded wait. False (and QVX_ETIMEOUT in the status word) if the wait ran out.
__device__ bool grid_sync(unsigned *count, unsigned *gen, unsigned nblocks, unsigned *status) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = gen;
        const unsigned g = *vgen;
        __threadfence();
        int ok = 1;
        if (atomicAdd(count, 1u) == nblocks - 1) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            unsigned i = 0;
            while (*vgen == g) {
                if (++i > kBarrierPolls) { ok = 0; break; }
                __nanosleep(64);
            }
        }
        __threadfence();
        if (!ok) atomicCAS(status, 0u, 4u /* QVX_ETIMEOUT */);
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// One output entry of a generic step. Arena tensors are written once per launch into
// regions of their own (no cache line is ever reused), so plain cached loads see them;
// leaf operands go through the read-only path.
__device__ __forceinline__ float2 persistent_entry(const DevStep &st, uint32_t c, const float2 *A, bool a_arena,
                                                   const float2 *B, bool b_arena, bool unary) {
    const uint32_t ia = pext_runs(c, st.runs_a, st.na_runs);
    const uint32_t ib = unary ? 0u : pext_runs(c, st.runs_b, st.nb_runs);
    const uint32_t nab = st.nk_ab, na = st.nk_a;
    const uint32_t nk = nab + na + st.nk_b;
    const uint32_t mask_ka = (1u << (nab + na)) - 1u, mask_ab = (1u << nab) - 1u;
    float2 acc = make_float2(0.f, 0.f);
    for (uint32_t k = 0; k < (1u << nk); k++) {
        const uint32_t ka = k & mask_ka;
        const float2 *pa = A + ia + (ka << st.a_cb);
        const float2 a = a_arena ? *pa : __ldg(pa);
        if (unary) {
            acc.x += a.x;
            acc.y += a.y;
        } else {
            const uint32_t kb = (k & mask_ab) | ((k >> (nab + na)) << nab);
            const float2 *pb = B + ib + (kb << st.b_cb);
            cmac(acc, a, b_arena ? *pb : __ldg(pb));
        }
    }
    return acc;
}

// All contractions of a chunk of work items in one cooperative launch: phase by phase;
// within a phase the CTAs sweep each step's (item, entry) space with a grid-stride loop
// (the step's descriptor staged once in shared memory), a grid barrier separates phases,
// then each item's final tensor is summed into its partial.
__global__ void __launch_bounds__(256) persistent_program_kernel(LaunchArgs a, int64_t item_begin, int64_t n_items,
                                                                 float2 *arenas, unsigned *bar_count, unsigned *bar_gen) {
    __shared__ __align__(16) DevStep sd;
    const unsigned char *img = a.image;
    const DevProgram *P = reinterpret_cast<const DevProgram *>(img);
    const DevStep *steps = reinterpret_cast<const DevStep *>(img + P->steps_off);
    const DevLeaf *leaves = reinterpret_cast<const DevLeaf *>(img + P->leaves_off);
    const float2 *ldata = reinterpret_cast<const float2 *>(img + P->leaf_data_off);
    const uint32_t *phase_first = reinterpret_cast<const uint32_t *>(img + P->level_phases_off);
    const uint32_t n_phases = P->n_level_phases;
    const uint64_t arena_elems = a.arena_elems;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint32_t ph = 0; ph < n_phases; ph++) {
        const uint32_t s0 = phase_first[ph], s1 = phase_first[ph + 1];
        for (uint32_t s = s0; s < s1; s++) {
            __syncthreads();   // the previous step's readers are done with sd
            if (threadIdx.x < sizeof(DevStep) / 8)
                reinterpret_cast<uint64_t *>(&sd)[threadIdx.x] = reinterpret_cast<const uint64_t *>(steps + s)[threadIdx.x];
            __syncthreads();
            const uint32_t rc = sd.rc, flags = sd.flags;
            const bool unary = flags & kStepUnary;
            const bool a_leaf = flags & kStepALeaf, b_leaf = flags & kStepBLeaf;
            const uint64_t total = (uint64_t)n_items << rc;
            // rotate the start so that small steps of one phase land on different CTAs
            const uint64_t first = (((uint64_t)blockIdx.x + (uint64_t)(s - s0) * 37u) % gridDim.x) * blockDim.x + threadIdx.x;
            for (uint64_t w = first; w < total; w += stride) {
                const int64_t il = (int64_t)(w >> rc);
                const uint32_t c = (uint32_t)(w & ((1ull << rc) - 1));
                const int64_t item = item_begin + il;
                const int64_t b = item / a.o_count;
                const uint64_t o = (uint64_t)(a.o_begin + item % a.o_count);
                float2 *arena = arenas + (uint64_t)il * arena_elems;
                const float2 *A, *B;
                if (a_leaf || (!unary && b_leaf)) {
                    const Bits x = load_bits(a.bitstrings, b, a.words);
                    A = a_leaf ? ldata + leaf_base(leaves[sd.a_off], x, o) : arena + sd.a_off;
                    B = unary ? A : (b_leaf ? ldata + leaf_base(leaves[sd.b_off], x, o) : arena + sd.b_off);
                } else {
                    A = arena + sd.a_off;
                    B = unary ? A : arena + sd.b_off;
                }
                arena[sd.c_off + c] = persistent_entry(sd, c, A, !a_leaf, B, !b_leaf, unary);
            }
        }
        if (!grid_sync(bar_count, bar_gen, gridDim.x, a.status)) return;
    }
    const FinishInfo fin = finish_info(P);
    const int warps = blockDim.x / 32, warp = threadIdx.x / 32;
    for (int64_t il = (int64_t)blockIdx.x * warps + warp; il < n_items; il += (int64_t)gridDim.x * warps) {
        const int64_t item = item_begin + il;
        const int64_t b = item / a.o_count;
        const uint64_t o = (uint64_t)(a.o_begin + item % a.o_count);
        // the final tensor was written by other CTAs: read it through L2
        const float2 *fsrc = arenas + (uint64_t)il * arena_elems + P->final_off;
        finish_item_cg(fin, a, fsrc, b, o, threadIdx.x % 32);
    }
}

// ------------------------------------------------------------------ register-tiled contraction
// One thread per 2^RM x 2^RN output entries of a two-operand step (RegTileStep): per summed
// index it loads 2^RM entries of A and 2^RN of B and forms all their products, so each
// loaded entry serves several outputs from registers. Tiles of up to 4 x 4 run 256 threads
// per CTA with the summed-index loop unrolled four deep (more loads in flight per thread);
// the 8-wide tiles of compute-heavy steps hold 2 x 64 accumulator registers and run 128
// threads per CTA, two CTAs per SM, with the loop unrolled twice.
template <int RM, int RN>
struct RegTileShape {
    static constexpr bool kWide = RM + RN >= 5;
    static constexpr int kThreads = kWide ? 128 : 256;
    static constexpr int kMinBlocks = kWide ? 2 : 4;
};

template <int RM, int RN>
__global__ void __launch_bounds__(RegTileShape<RM, RN>::kThreads, RegTileShape<RM, RN>::kMinBlocks)
    regtile_step_kernel(LaunchArgs a, RegTileStep rs, int64_t item_begin, int64_t n_items, float2 *arenas) {
    constexpr int TM = 1 << RM, TN = 1 << RN;
    const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ((uint64_t)n_items << rs.nt)) return;
    const int64_t il = (int64_t)(g >> rs.nt);
    const uint32_t t = (uint32_t)(g & ((1ull << rs.nt) - 1ull));
    float2 *arena = arenas + (uint64_t)il * a.arena_elems;
    const float2 *A, *B;
    {
        const unsigned char *img = a.image;
        const DevProgram *P = reinterpret_cast<const DevProgram *>(img);
        const DevLeaf *leaves = reinterpret_cast<const DevLeaf *>(img + P->leaves_off);
        const float2 *ldata = reinterpret_cast<const float2 *>(img + P->leaf_data_off);
        Bits x = {0ull, 0ull};
        uint64_t o = 0;
        if (rs.flags & (kStepALeaf | kStepBLeaf)) {
            const int64_t item = item_begin + il;
            x = load_bits(a.bitstrings, item / a.o_count, a.words);
            o = (uint64_t)(a.o_begin + item % a.o_count);
        }
        A = (rs.flags & kStepALeaf) ? ldata + leaf_base(leaves[rs.a_off], x, o) : arena + rs.a_off;
        B = (rs.flags & kStepBLeaf) ? ldata + leaf_base(leaves[rs.b_off], x, o) : arena + rs.b_off;
    }
    const uint32_t c0 = pext_runs(t, rs.free_runs, rs.n_free);
    A += pext_runs(c0, rs.runs_a, rs.na_runs);
    B += pext_runs(c0, rs.runs_b, rs.nb_runs);
    const uint32_t nab = rs.nk_ab, na = rs.nk_a;
    const uint32_t nk = nab + na + rs.nk_b;
    const uint32_t mask_ka = (1u << (nab + na)) - 1u, mask_ab = (1u << nab) - 1u;
    uint32_t am[TM], bn[TN];
#pragma unroll
    for (int i = 0; i < TM; i++) am[i] = rs.a_m[i];
#pragma unroll
    for (int j = 0; j < TN; j++) bn[j] = rs.b_n[j];
    float2 acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; i++)
#pragma unroll
        for (int j = 0; j < TN; j++) acc[i][j] = make_float2(0.f, 0.f);
    constexpr int kUnroll = RegTileShape<RM, RN>::kWide ? 2 : 4;
#pragma unroll kUnroll
    for (uint32_t k = 0; k < (1u << nk); k++) {
        const uint32_t ka = k & mask_ka;
        const uint32_t kb = (k & mask_ab) | ((k >> (nab + na)) << nab);
        const float2 *Ak = A + (ka << rs.a_cb), *Bk = B + (kb << rs.b_cb);
        float2 av[TM], bv[TN];
#pragma unroll
        for (int i = 0; i < TM; i++) av[i] = Ak[am[i]];
#pragma unroll
        for (int j = 0; j < TN; j++) bv[j] = Bk[bn[j]];
#pragma unroll
        for (int i = 0; i < TM; i++)
#pragma unroll
            for (int j = 0; j < TN; j++) cmac(acc[i][j], av[i], bv[j]);
    }
    float2 *C = arena + rs.c_off + c0;
#pragma unroll
    for (int i = 0; i < TM; i++)
#pragma unroll
        for (int j = 0; j < TN; j++) C[rs.c_m[i] + rs.c_n[j]] = acc[i][j];
}

// A contraction with many summed entries and few outputs: 32 consecutive outputs per CTA,
// the summed index split over the 8 warps, partial sums added through shared memory.
__global__ void __launch_bounds__(256) splitk_step_kernel(LaunchArgs a, uint32_t s_idx, int64_t item_begin,
                                                          int64_t n_items, float2 *arenas) {
    __shared__ float2 part[8][33];
    __shared__ __align__(16) DevStep sd;
    const unsigned char *img = a.image;
    const DevProgram *P = reinterpret_cast<const DevProgram *>(img);
    if (threadIdx.x < sizeof(DevStep) / 8)
        reinterpret_cast<uint64_t *>(&sd)[threadIdx.x] =
            reinterpret_cast<const uint64_t *>(reinterpret_cast<const DevStep *>(img + P->steps_off) + s_idx)[threadIdx.x];
    __syncthreads();
    const uint32_t lane = threadIdx.x % 32, warp = threadIdx.x / 32;
    const uint64_t w = (uint64_t)blockIdx.x * 32 + lane;
    const bool valid = w < ((uint64_t)n_items << sd.rc);
    float2 acc = make_float2(0.f, 0.f);
    uint32_t c = 0;
    float2 *arena = nullptr;
    if (valid) {
        const int64_t il = (int64_t)(w >> sd.rc);
        c = (uint32_t)(w & ((1ull << sd.rc) - 1));
        const int64_t item = item_begin + il;
        arena = arenas + (uint64_t)il * a.arena_elems;
        const DevLeaf *leaves = reinterpret_cast<const DevLeaf *>(img + P->leaves_off);
        const float2 *ldata = reinterpret_cast<const float2 *>(img + P->leaf_data_off);
        Bits x = {0ull, 0ull};
        uint64_t o = 0;
        if (sd.flags & (kStepALeaf | kStepBLeaf)) {
            x = load_bits(a.bitstrings, item / a.o_count, a.words);
            o = (uint64_t)(a.o_begin + item % a.o_count);
        }
        const bool unary = sd.flags & kStepUnary;
        const float2 *A = (sd.flags & kStepALeaf) ? ldata + leaf_base(leaves[sd.a_off], x, o) : arena + sd.a_off;
        const float2 *B = unary ? A : ((sd.flags & kStepBLeaf) ? ldata + leaf_base(leaves[sd.b_off], x, o) : arena + sd.b_off);
        const uint32_t ia = pext_runs(c, sd.runs_a, sd.na_runs);
        const uint32_t ib = unary ? 0u : pext_runs(c, sd.runs_b, sd.nb_runs);
        const uint32_t nab = sd.nk_ab, na = sd.nk_a, nk = nab + na + sd.nk_b;
        const uint32_t mask_ka = (1u << (nab + na)) - 1u, mask_ab = (1u << nab) - 1u;
        if (unary) {
            for (uint32_t k = warp; k < (1u << nk); k += 8) {
                const float2 av = A[ia + ((k & mask_ka) << sd.a_cb)];
                acc.x += av.x;
                acc.y += av.y;
            }
        } else {
#pragma unroll 4
            for (uint32_t k = warp; k < (1u << nk); k += 8) {
                const uint32_t kb = (k & mask_ab) | ((k >> (nab + na)) << nab);
                cmac(acc, A[ia + ((k & mask_ka) << sd.a_cb)], B[ib + (kb << sd.b_cb)]);
            }
        }
    }
    part[warp][lane] = acc;
    __syncthreads();
    if (warp == 0 && valid) {
        float2 s = part[0][lane];
        for (int j = 1; j < 8; j++) {
            s.x += part[j][lane].x;
            s.y += part[j][lane].y;
        }
        arena[sd.c_off + c] = s;
    }
}

__global__ void finish_kernel(LaunchArgs a, int64_t item_begin, int64_t n_items, const float2 *arenas) {
    const DevProgram *P = reinterpret_cast<const DevProgram *>(a.image);
    const int64_t il = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    if (il >= n_items) return;
    const int64_t item = item_begin + il;
    const int64_t b = item / a.o_count;
    const uint64_t o = (uint64_t)(a.o_begin + item % a.o_count);
    finish_item(finish_info(P), a, arenas + (uint64_t)il * a.arena_elems + P->final_off, b, o, threadIdx.x % 32, 32);
}

// ------------------------------------------------------------------ slice sum
__global__ void slice_sum_kernel(const unsigned char *img, const ExactPair *partials, int64_t o_count, double *amps,
                                 unsigned *status) {
    const DevProgram *P = reinterpret_cast<const DevProgram *>(img);
    const int64_t b = blockIdx.x;
    const double2 r = block_exact_sum(partials + b * o_count, o_count, P->scalar_re, P->scalar_im, status);
    if (threadIdx.x == 0) {
        amps[2 * b] = r.x;
        amps[2 * b + 1] = r.y;
    }
}

// ------------------------------------------------------------------ gradient program
__device__ __forceinline__ uint32_t runs_pdep(uint32_t v, const DevRun *runs, uint32_t n) {
    uint32_t r = 0;
    for (uint32_t i = 0; i < n; i++) r |= ((v >> runs[i].src) & ((1u << runs[i].len) - 1u)) << runs[i].dst;
    return r;
}

// Parametrised leaf entries from the angles: U = cos(t/2) I - i sin(t/2) (cos(phi) X +
// sin(phi) Y) and dU/dtheta = -sin(t/2)/2 I - (i/2) cos(t/2) (cos(phi) X + sin(phi) Y).
__global__ void set_params_kernel(unsigned char *img, const double *thetas) {
    const DevProgram *P = reinterpret_cast<const DevProgram *>(img);
    const ParamLeaf &pl = reinterpret_cast<const ParamLeaf *>(img + P->params_off)[blockIdx.x];
    const DevLeaf &L = reinterpret_cast<const DevLeaf *>(img + P->leaves_off)[pl.leaf];
    const uint8_t *codes = img + P->codes_off + pl.code_off;
    float2 *data = reinterpret_cast<float2 *>(img + P->leaf_data_off) + L.data_off;
    float2 *deriv = reinterpret_cast<float2 *>(img + P->deriv_data_off) + L.data_off;
    const double th = thetas ? thetas[pl.param] : reinterpret_cast<const double *>(img + P->thetas_off)[pl.param];
    double s, c, sp, cp;
    sincos(0.5 * th, &s, &c);
    sincos(pl.phi, &sp, &cp);
    for (uint32_t e = threadIdx.x; e < pl.n_stored; e += blockDim.x) {
        const uint32_t code = codes[e];
        const uint32_t row = code >> 1, col = code & 1u;
        double ur, ui, dr, di;
        if (row == col) {
            ur = c; ui = 0; dr = -0.5 * s; di = 0;
        } else {
            // off-diagonal: -i s e^{-i phi} (row 0) or -i s e^{+i phi} (row 1)
            const double sg = row == 0 ? -1.0 : 1.0;
            ur = sg * s * sp;  ui = -s * cp;          // -i s (cp + i sg sp)
            dr = sg * 0.5 * c * sp; di = -0.5 * c * cp;
        }
        data[e] = make_float2((float)ur, (float)ui);
        deriv[e] = make_float2((float)dr, (float)di);
    }
}

__device__ __forceinline__ const float2 *gen_base(const GenOperand &op, const DevProgram *P,
                                                  const unsigned char *img, float2 *arena, const Bits &x,
                                                  uint64_t o) {
    if (op.kind == kOpArena) return arena + op.off;
    if (op.kind == kOpOne) return nullptr;
    const DevLeaf &L = reinterpret_cast<const DevLeaf *>(img + P->leaves_off)[op.off];
    const uint64_t data = op.kind == kOpLeaf ? P->leaf_data_off : P->deriv_data_off;
    return reinterpret_cast<const float2 *>(img + data) + leaf_base(L, x, o);
}

__global__ void __launch_bounds__(256) grad_program_kernel(GradArgs g) {
    const unsigned char *img = g.image;
    const DevProgram *P = reinterpret_cast<const DevProgram *>(img);
    const GenStep *steps = reinterpret_cast<const GenStep *>(img + P->grad_steps_off);
    float2 *arena = g.arenas + (uint64_t)blockIdx.x * g.arena_elems;
    const int64_t n_items = g.batch * g.o_count;
    const uint32_t npl = P->n_param_leaves;
    const uint32_t n_phases = P->n_grad_phases;
    const uint32_t *phase_first = reinterpret_cast<const uint32_t *>(img + P->grad_phases_off);
    const uint32_t *elem_off = reinterpret_cast<const uint32_t *>(img + P->grad_elem_off_off);
    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int64_t b = item / g.o_count;
        const uint64_t o = (uint64_t)(item % g.o_count);
        const Bits x = load_bits(g.bitstrings, b, g.words);
        // phase by phase: the entries of all steps of a phase are spread over the CTA
        for (uint32_t ph = 0; ph < n_phases; ph++) {
            const uint32_t s0 = phase_first[ph], s1 = phase_first[ph + 1];
            const uint32_t total = elem_off[s1 - 1] + (1u << steps[s1 - 1].ro);
            for (uint32_t e = threadIdx.x; e < total; e += blockDim.x) {
                uint32_t lo = s0, hi = s1 - 1;   // the last step whose first entry is <= e
                while (lo < hi) {
                    const uint32_t mid = (lo + hi + 1) >> 1;
                    if (elem_off[mid] <= e) lo = mid;
                    else hi = mid - 1;
                }
                const GenStep &st = steps[lo];
                const uint32_t oi = e - elem_off[lo];
                const float2 *X = gen_base(st.x, P, img, arena, x, o);
                const float2 *Y = gen_base(st.y, P, img, arena, x, o);
                const uint32_t ox = runs_pdep(oi, st.x.oruns, st.x.n_oruns);
                const uint32_t oy = runs_pdep(oi, st.y.oruns, st.y.n_oruns);
                float2 acc = make_float2(0.f, 0.f);
                for (uint32_t k = 0; k < (1u << st.nk); k++) {
                    const float2 av = X ? X[ox + runs_pdep(k, st.x.kruns, st.x.n_kruns)] : make_float2(1.f, 0.f);
                    const float2 bv = Y ? Y[oy + runs_pdep(k, st.y.kruns, st.y.n_kruns)] : make_float2(1.f, 0.f);
                    cmac(acc, av, bv);
                }
                arena[st.out_off + oi] = acc;
            }
            __syncthreads();
        }
        // amplitude partial: exact sum of the final tensor over the inner slice modes
        const bool zero = bits_hit(x, P->zero_mask, P->zero_mask_hi);
        if (threadIdx.x < 32) {
            const float2 *fin = arena + P->final_fwd_off;
            Fx re = {0ull, 0ll}, im = {0ull, 0ll};
            bool bad = false;
            const uint32_t n_in = P->n_inner, present = P->final_present;
            for (uint32_t i = threadIdx.x; i < (1u << n_in); i += 32) {
                uint32_t fi = 0, bit = 0;
                for (uint32_t j = 0; j < n_in; j++)
                    if ((present >> j) & 1u) fi |= ((i >> j) & 1u) << bit++;
                const float2 t = zero ? make_float2(0.f, 0.f) : fin[fi];
                re = fx_add(re, fx_from_float(t.x, bad), bad);
                im = fx_add(im, fx_from_float(t.y, bad), bad);
            }
            for (int d = 16; d > 0; d >>= 1) {
                re = fx_add(re, fx_shfl_down(re, d), bad);
                im = fx_add(im, fx_shfl_down(im, d), bad);
            }
            if (bad) atomicCAS(g.status, 0u, kStatusRange);
            if (threadIdx.x == 0) g.partials[item] = fx_pair(re, im);
        }
        for (uint32_t lp = threadIdx.x; lp < npl; lp += blockDim.x) {
            const float2 t = zero ? make_float2(0.f, 0.f) : arena[P->gslot_off + lp];
            bool bad = false;
            const Fx tr = fx_from_float(t.x, bad), ti = fx_from_float(t.y, bad);
            if (bad) atomicCAS(g.status, 0u, kStatusRange);
            g.gpart[(uint64_t)item * npl + lp] = fx_pair(tr, ti);
        }
        __syncthreads();
    }
}

// One output entry of the gradient program from its record: sum over the summed index of
// X * Y, where an operand is the shared-memory arena, a restricted leaf (base in lbase), its
// derivative, or the constant one.
__device__ __forceinline__ float2 grad_record_value(const uint4 rv, const float2 *arena, const uint32_t *lbase,
                                                    const float2 *ldata, const float2 *ddata,
                                                    const uint32_t *ktab) {
    const uint32_t meta = rv.x >> 16;
    const uint32_t xr = rv.y & 0xffffu, xo = rv.y >> 16, yr = rv.z & 0xffffu, yo = rv.z >> 16;
    const uint32_t xk = meta & 3u, yk = (meta >> 2) & 3u, nk = (meta >> 4) & 15u;
    const float2 *X = xk == kOpArena ? arena + xr : xk == kOpLeaf ? ldata + lbase[xr] : xk == kOpDeriv ? ddata + lbase[xr] : nullptr;
    const float2 *Y = yk == kOpArena ? arena + yr : yk == kOpLeaf ? ldata + lbase[yr] : yk == kOpDeriv ? ddata + lbase[yr] : nullptr;
    const float2 one = make_float2(1.f, 0.f);
    if (X) X += xo;
    if (Y) Y += yo;
    float2 acc = make_float2(0.f, 0.f);
    if (nk == 2) {   // the three offset pairs first, so the six operand loads are independent
        const uint32_t k1 = ktab[rv.w], k2 = ktab[rv.w + 1], k3 = ktab[rv.w + 2];
        const float2 x0 = X ? X[0] : one, y0 = Y ? Y[0] : one;
        const float2 x1 = X ? X[k1 & 0xffffu] : one, y1 = Y ? Y[k1 >> 16] : one;
        const float2 x2 = X ? X[k2 & 0xffffu] : one, y2 = Y ? Y[k2 >> 16] : one;
        const float2 x3 = X ? X[k3 & 0xffffu] : one, y3 = Y ? Y[k3 >> 16] : one;
        cmac(acc, x0, y0);
        cmac(acc, x1, y1);
        cmac(acc, x2, y2);
        cmac(acc, x3, y3);
        return acc;
    }
    cmac(acc, X ? X[0] : one, Y ? Y[0] : one);
    if (nk == 1) {
        cmac(acc, X ? X[rv.w & 0xffffu] : one, Y ? Y[rv.w >> 16] : one);
    } else if (nk > 2) {
#pragma unroll 4
        for (uint32_t k = 1; k < (1u << nk); k++) {
            const uint32_t kp = ktab[rv.w + k - 1];
            cmac(acc, X ? X[kp & 0xffffu] : one, Y ? Y[kp >> 16] : one);
        }
    }
    return acc;
}

constexpr int kGradPrefetch = 4;   // records per thread loaded one phase ahead

// The gradient program with the work item's arena in shared memory: the records of each
// level phase are spread over the CTA's threads, one barrier per phase, and each thread
// loads its first record of the next phase before the barrier of the current one.
// STAGED: the leaf data, the derivative data and the summed-index table are first copied
// into shared memory (after the arena and the leaf table) by bulk asynchronous copies on one
// mbarrier with a bounded wait, so the operand reads of every phase stay on chip.
template <bool STAGED>
__global__ void __launch_bounds__(256) grad_smem_kernel(GradArgs g) {
    extern __shared__ float4 gsm[];
    __shared__ __align__(8) uint64_t stage_bar;
    const unsigned char *img = g.image;
    const DevProgram *P = reinterpret_cast<const DevProgram *>(img);
    float2 *arena = reinterpret_cast<float2 *>(gsm);
    uint32_t *lbase = reinterpret_cast<uint32_t *>(arena + P->grad_arena_elems);
    const uint4 *rec = reinterpret_cast<const uint4 *>(img + P->gentry_off);
    const uint32_t *ktab = reinterpret_cast<const uint32_t *>(img + P->gktab_off);
    const uint32_t *pe = reinterpret_cast<const uint32_t *>(img + P->gphase_entry_off);
    const DevLeaf *leaves = reinterpret_cast<const DevLeaf *>(img + P->leaves_off);
    const float2 *ldata = reinterpret_cast<const float2 *>(img + P->leaf_data_off);
    const float2 *ddata = reinterpret_cast<const float2 *>(img + P->deriv_data_off);
    const uint32_t n_phases = P->n_grad_phases, n_leaves = P->n_leaves, npl = P->n_param_leaves;
    if (STAGED) {
        const size_t head = ((size_t)P->grad_arena_elems * 8 + (size_t)n_leaves * 4 + 15) & ~size_t(15);
        unsigned char *st = reinterpret_cast<unsigned char *>(gsm) + head;
        const uint32_t bar = smem_u32(&stage_bar);
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                         "r"(g.stage_ldata + g.stage_ddata + g.stage_ktab)
                         : "memory");
            bulk_g2s(smem_u32(st), ldata, g.stage_ldata, bar);
            bulk_g2s(smem_u32(st + g.stage_ldata), ddata, g.stage_ddata, bar);
            if (g.stage_ktab) bulk_g2s(smem_u32(st + g.stage_ldata + g.stage_ddata), ktab, g.stage_ktab, bar);
        }
        __syncthreads();
        const bool ok = mbar_wait(bar, 0, kWaitPolls);
        if (__syncthreads_or(!ok)) {          // the copy never completed: report and leave
            if (threadIdx.x == 0) atomicCAS(g.status, 0u, 4u /* QVX_ETIMEOUT */);
            mbar_wait(bar, 0, kWaitPolls);
            return;
        }
        ldata = reinterpret_cast<const float2 *>(st);
        ddata = reinterpret_cast<const float2 *>(st + g.stage_ldata);
        ktab = reinterpret_cast<const uint32_t *>(st + g.stage_ldata + g.stage_ddata);
    }
    const int64_t n_items = g.batch * g.o_count;
    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int64_t b = item / g.o_count;
        const uint64_t o = (uint64_t)(item % g.o_count);
        const Bits x = load_bits(g.bitstrings, b, g.words);
        for (uint32_t l = threadIdx.x; l < n_leaves; l += blockDim.x) lbase[l] = leaf_base(leaves[l], x, o);
        // a thread's first kGradPrefetch records of a phase are loaded during the phase before
        uint4 cur[kGradPrefetch];
#pragma unroll
        for (int j = 0; j < kGradPrefetch; j++) {
            const uint32_t e = pe[0] + threadIdx.x + j * blockDim.x;
            cur[j] = n_phases > 0 && e < pe[1] ? rec[e] : make_uint4(0u, 0u, 0u, 0u);
        }
        __syncthreads();
        for (uint32_t ph = 0; ph < n_phases; ph++) {
            const uint32_t e0 = pe[ph], e1 = pe[ph + 1];
            uint4 nxt[kGradPrefetch];
#pragma unroll
            for (int j = 0; j < kGradPrefetch; j++) {
                const uint32_t e = e1 + threadIdx.x + j * blockDim.x;
                nxt[j] = ph + 1 < n_phases && e < pe[ph + 2] ? rec[e] : make_uint4(0u, 0u, 0u, 0u);
            }
#pragma unroll
            for (int j = 0; j < kGradPrefetch; j++)
                if (e0 + threadIdx.x + j * blockDim.x < e1)
                    arena[cur[j].x & 0xffffu] = grad_record_value(cur[j], arena, lbase, ldata, ddata, ktab);
            for (uint32_t e = e0 + threadIdx.x + kGradPrefetch * blockDim.x; e < e1; e += blockDim.x) {
                const uint4 rv = rec[e];
                arena[rv.x & 0xffffu] = grad_record_value(rv, arena, lbase, ldata, ddata, ktab);
            }
#pragma unroll
            for (int j = 0; j < kGradPrefetch; j++) cur[j] = nxt[j];
            __syncthreads();
        }
        const bool zero = bits_hit(x, P->zero_mask, P->zero_mask_hi);
        if (threadIdx.x < 32) {
            const float2 *fin = arena + P->final_fwd_off;
            Fx re = {0ull, 0ll}, im = {0ull, 0ll};
            bool bad = false;
            const uint32_t n_in = P->n_inner, present = P->final_present;
            for (uint32_t i = threadIdx.x; i < (1u << n_in); i += 32) {
                uint32_t fi = 0, bit = 0;
                for (uint32_t j = 0; j < n_in; j++)
                    if ((present >> j) & 1u) fi |= ((i >> j) & 1u) << bit++;
                const float2 t = zero ? make_float2(0.f, 0.f) : fin[fi];
                re = fx_add(re, fx_from_float(t.x, bad), bad);
                im = fx_add(im, fx_from_float(t.y, bad), bad);
            }
            for (int d = 16; d > 0; d >>= 1) {
                re = fx_add(re, fx_shfl_down(re, d), bad);
                im = fx_add(im, fx_shfl_down(im, d), bad);
            }
            if (bad) atomicCAS(g.status, 0u, kStatusRange);
            if (threadIdx.x == 0) g.partials[item] = fx_pair(re, im);
        }
        for (uint32_t lp = threadIdx.x; lp < npl; lp += blockDim.x) {
            const float2 t = zero ? make_float2(0.f, 0.f) : arena[P->gslot_off + lp];
            bool bad = false;
            const Fx tr = fx_from_float(t.x, bad), ti = fx_from_float(t.y, bad);
            if (bad) atomicCAS(g.status, 0u, kStatusRange);
            g.gpart[(uint64_t)item * npl + lp] = fx_pair(tr, ti);
        }
        __syncthreads();
    }
}

// One block per (bitstring, parameter): exact sum over the work items and over the
// parameter's leaves (CSR lists in the image), rounded once and times the plan's scalar.
__global__ void grad_sum_kernel(const unsigned char *img, const ExactPair *gpart, int64_t o_count, uint32_t npl,
                                uint32_t n_params, double *grad, unsigned *status) {
    __shared__ Fx red[2][32];
    const DevProgram *P = reinterpret_cast<const DevProgram *>(img);
    const uint32_t *csr = reinterpret_cast<const uint32_t *>(img + P->param_csr_off);
    const int64_t b = blockIdx.x / n_params;
    const uint32_t p = blockIdx.x % n_params;
    const uint32_t first = csr[p], last = csr[p + 1];
    const uint32_t *list = csr + n_params + 1;
    Fx re = {0ull, 0ll}, im = {0ull, 0ll};
    bool bad = false;
    const int64_t n = (int64_t)(last - first) * o_count;
    for (int64_t t = threadIdx.x; t < n; t += blockDim.x) {
        const uint32_t lp = list[first + t / o_count];
        const int64_t o = t % o_count;
        const ExactPair v = gpart[((uint64_t)(b * o_count + o)) * npl + lp];
        re = fx_add(re, Fx{v.re_lo, (long long)v.re_hi}, bad);
        im = fx_add(im, Fx{v.im_lo, (long long)v.im_hi}, bad);
    }
    for (int d = 16; d > 0; d >>= 1) {
        re = fx_add(re, fx_shfl_down(re, d), bad);
        im = fx_add(im, fx_shfl_down(im, d), bad);
    }
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
    if (lane == 0) {
        red[0][warp] = re;
        red[1][warp] = im;
    }
    bad = __syncthreads_or(bad) != 0;
    if (threadIdx.x == 0) {
        for (int w = 1; w < nw; w++) {
            re = fx_add(re, red[0][w], bad);
            im = fx_add(im, red[1][w], bad);
        }
        if (bad) atomicCAS(status, 0u, kStatusRange);
        double gr, gi;
        if (bad || *reinterpret_cast<volatile unsigned *>(status) != 0u) {   // no valid sum: NaN
            gr = gi = __longlong_as_double(0x7ff8000000000000ll);
        } else {
            const double r = fx_to_double(re), i = fx_to_double(im);
            gr = r * P->scalar_re - i * P->scalar_im;
            gi = r * P->scalar_im + i * P->scalar_re;
        }
        grad[2 * (b * n_params + p)] = gr;
        grad[2 * (b * n_params + p) + 1] = gi;
    }
}

// Self-test of the bounded waits: a grid barrier for two CTAs run by one, and an mbarrier
// whose phase never completes. Each wait must give up after `polls` polls; the kernel
// records which did in out[0] (barrier) and out[1] (mbarrier) and sets the status word.
__global__ void wait_selftest_kernel(unsigned *words, unsigned *status, uint32_t polls, unsigned *out) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    // grid barrier: one arrival of two, the generation never advances
    unsigned *count = words, *gen = words + 1;
    *count = 0;
    const unsigned g = *(volatile unsigned *)gen;
    atomicAdd(count, 1u);
    unsigned i = 0;
    bool gave_up = false;
    while (*(volatile unsigned *)gen == g) {
        if (++i > polls) { gave_up = true; break; }
        __nanosleep(64);
    }
    out[0] = gave_up ? 1u : 0u;
    atomicExch(count, 0u);
    // mbarrier expecting one arrival that never comes
    const uint32_t b = smem_u32(&bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
    out[1] = mbar_wait(b, 0, polls) ? 0u : 1u;
    if (out[0] && out[1]) atomicCAS(status, 0u, 4u /* QVX_ETIMEOUT */);
}

thread_local uint64_t t_launches = 0;   // kernels this host thread has launched

cudaError_t counted(cudaError_t e) {
    if (e == cudaSuccess) t_launches++;
    return e;
}

}  // namespace

uint64_t launches_issued() { return t_launches; }

cudaError_t launch_counted(cudaError_t e) { return counted(e); }

cudaError_t launch_wait_selftest(unsigned *words, unsigned *status, uint32_t polls, unsigned *out, cudaStream_t s) {
    wait_selftest_kernel<<<1, 32, 0, s>>>(words, status, polls, out);
    return counted(cudaGetLastError());
}

cudaError_t launch_set_params(unsigned char *image, uint32_t n_param_leaves, const double *thetas, cudaStream_t s) {
    if (n_param_leaves == 0) return cudaSuccess;
    set_params_kernel<<<n_param_leaves, 32, 0, s>>>(image, thetas);
    return counted(cudaGetLastError());
}

cudaError_t launch_grad_program(const GradArgs &g, int grid, cudaStream_t s) {
    grad_program_kernel<<<grid, 256, 0, s>>>(g);
    return counted(cudaGetLastError());
}

size_t grad_smem_bytes(const DevProgram *h) {
    if (!h->gentry_off) return 0;
    return ((size_t)h->grad_arena_elems * 8 + (size_t)h->n_leaves * 4 + 15) & ~size_t(15);
}

size_t grad_stage_bytes(const DevProgram *h, GradArgs *g) {
    auto r16 = [](size_t x) { return (x + 15) & ~size_t(15); };
    const size_t ld = r16((size_t)h->n_leaf_entries * 8);
    const size_t kt = h->gphase_entry_off > h->gktab_off ? r16(h->gphase_entry_off - h->gktab_off) : 0;
    g->stage_ldata = (uint32_t)ld;
    g->stage_ddata = (uint32_t)ld;
    g->stage_ktab = (uint32_t)kt;
    return 2 * ld + kt;
}

int grad_smem_blocks_per_sm(size_t smem_bytes, bool staged) {
    static bool raised[64] = {false};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (dev >= 0 && dev < 64 && !raised[dev]) {
        int optin = 0;
        if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, grad_smem_kernel<true>) != cudaSuccess) return 0;
        const int limit = optin - (int)fa.sharedSizeBytes;
        if (cudaFuncSetAttribute(grad_smem_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit) != cudaSuccess ||
            cudaFuncSetAttribute(grad_smem_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit) != cudaSuccess)
            return 0;
        raised[dev] = true;
    }
    int n = 0;
    if ((staged ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, grad_smem_kernel<true>, 256, smem_bytes)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, grad_smem_kernel<false>, 256, smem_bytes)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t launch_grad_smem(const GradArgs &g, int grid, size_t smem_bytes, cudaStream_t s) {
    if (g.stage_ldata) grad_smem_kernel<true><<<grid, 256, smem_bytes, s>>>(g);
    else grad_smem_kernel<false><<<grid, 256, smem_bytes, s>>>(g);
    return counted(cudaGetLastError());
}

cudaError_t launch_grad_sum(const unsigned char *image, const ExactPair *gpart, int64_t batch, int64_t o_count,
                            uint32_t n_param_leaves, uint32_t n_params, double *grad, unsigned *status, cudaStream_t s) {
    if (n_params == 0 || batch == 0) return cudaSuccess;
    grad_sum_kernel<<<(unsigned)(batch * n_params), 256, 0, s>>>(image, gpart, o_count, n_param_leaves, n_params, grad,
                                                                 status);
    return counted(cudaGetLastError());
}

// The dynamic shared-memory limit is an attribute of the kernel function, shared by every
// plan: raise it once per device to the most the device allows, never lower it.
cudaError_t fused_prepare(size_t smem_bytes) {
    static bool raised[64] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && raised[dev]) return cudaSuccess;
    int optin = 0;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, fused_program_kernel<true>)) != cudaSuccess) return e;
    const int limit = optin - (int)fa.sharedSizeBytes;
    if ((size_t)limit < smem_bytes) return cudaErrorInvalidValue;
    if ((e = cudaFuncSetAttribute(fused_program_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(fused_program_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit)) != cudaSuccess)
        return e;
    if (dev >= 0 && dev < 64) raised[dev] = true;
    return cudaSuccess;
}

int fused_blocks_per_sm(int threads, size_t smem_bytes, bool staged) {
    int n = 0;
    cudaError_t e = staged ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fused_program_kernel<true>, threads, smem_bytes)
                           : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fused_program_kernel<false>, threads, smem_bytes);
    return e == cudaSuccess ? n : 0;
}

bool fused_shape(const DevProgram *h, uint64_t arena_elems, int warps_per_item, LaunchArgs *a, size_t *shared,
                 size_t *group, int *max_ipc) {
    auto r16 = [](size_t x) { return (x + 15) & ~size_t(15); };
    const size_t kBudget = 220u << 10;   // dynamic shared memory per CTA
    *group = r16((size_t)h->n_leaves * 4) + (size_t)arena_elems * 8;
    if (h->fused_lanes != (uint32_t)(32 * warps_per_item)) return false;
    const size_t steps_b = r16((size_t)(h->fused_lane_map_off - h->fused_steps_off) +
                               (size_t)h->n_fused_phases * h->fused_lanes * 4);
    const size_t leaf_b = r16((size_t)h->n_leaf_entries * 8);
    const size_t leaves_b = r16((size_t)h->n_leaves * sizeof(DevLeaf));
    size_t sh = steps_b + leaf_b + leaves_b;
    if (sh + *group > kBudget) sh = 0;    // the program stays in global memory
    if (sh + *group > kBudget) return false;
    a->smem_steps_bytes = sh ? (uint32_t)steps_b : 0;
    a->smem_leaf_bytes = sh ? (uint32_t)leaf_b : 0;
    a->smem_leaves_bytes = sh ? (uint32_t)leaves_b : 0;
    a->leaf_table_bytes = (uint32_t)r16((size_t)h->n_leaves * 4);
    a->group_bytes = (uint32_t)*group;
    a->fused_steps_off = h->fused_steps_off;
    a->fused_tab_off = h->fused_tab_off;
    a->fused_lane_map_off = h->fused_lane_map_off;
    a->leaves_off = h->leaves_off;
    a->leaf_data_off = h->leaf_data_off;
    a->final_off = h->final_off;
    a->n_fused_phases = h->n_fused_phases;
    a->n_leaves = h->n_leaves;
    *shared = sh;
    *max_ipc = (int)std::max<size_t>(1, std::min<size_t>(std::max(1, 8 / warps_per_item), (kBudget - sh) / *group));
    return true;
}

cudaError_t launch_fused(const LaunchArgs &a, int warps_per_item, int items_per_cta, int grid,
                         size_t smem_bytes, cudaStream_t s) {
    const int threads = 32 * warps_per_item * items_per_cta;
    if (a.smem_steps_bytes) fused_program_kernel<true><<<grid, threads, smem_bytes, s>>>(a, warps_per_item);
    else fused_program_kernel<false><<<grid, threads, smem_bytes, s>>>(a, warps_per_item);
    return counted(cudaGetLastError());
}

cudaError_t launch_step(const LaunchArgs &a, uint32_t step, int64_t item_begin, int64_t n_items,
                        float2 *arenas, uint32_t rc, cudaStream_t s) {
    const uint64_t total = (uint64_t)n_items << rc;
    const int threads = 256;
    const uint64_t blocks = (total + threads - 1) / threads;
    step_kernel<<<(unsigned)blocks, threads, 0, s>>>(a, step, item_begin, n_items, arenas);
    return counted(cudaGetLastError());
}

cudaError_t launch_step_group(const LaunchArgs &a, const StepGroup &g, int64_t item_begin, int64_t n_items,
                              float2 *arenas, cudaStream_t s) {
    if (g.n == 0 || g.n > (uint32_t)kMaxGroupSteps || g.first_block[g.n] == 0) return cudaErrorInvalidConfiguration;
    step_group_kernel<<<g.first_block[g.n], 256, 0, s>>>(a, g, item_begin, n_items, arenas);
    return counted(cudaGetLastError());
}

cudaError_t launch_splitk_step(const LaunchArgs &a, uint32_t step, int64_t item_begin, int64_t n_items,
                               float2 *arenas, uint32_t rc, cudaStream_t s) {
    const uint64_t blocks = (((uint64_t)n_items << rc) + 31) / 32;
    if (blocks > 0x7fffffffull) return cudaErrorInvalidConfiguration;
    splitk_step_kernel<<<(unsigned)blocks, 256, 0, s>>>(a, step, item_begin, n_items, arenas);
    return counted(cudaGetLastError());
}

template <int RM, int RN>
static void launch_regtile_t(const LaunchArgs &a, const RegTileStep &rs, int64_t item_begin, int64_t n_items,
                             float2 *arenas, cudaStream_t s) {
    constexpr int kThreads = RegTileShape<RM, RN>::kThreads;
    const uint64_t blocks = (((uint64_t)n_items << rs.nt) + kThreads - 1) / kThreads;
    regtile_step_kernel<RM, RN><<<(unsigned)blocks, kThreads, 0, s>>>(a, rs, item_begin, n_items, arenas);
}

cudaError_t launch_regtile_step(const LaunchArgs &a, const RegTileStep &rs, int64_t item_begin, int64_t n_items,
                                float2 *arenas, cudaStream_t s) {
    const uint64_t blocks = (((uint64_t)n_items << rs.nt) + 127) / 128;
    if (blocks > 0x7fffffffull || rs.rm > 3 || rs.rn > 3 || rs.rm + rs.rn == 0) return cudaErrorInvalidConfiguration;
    switch (rs.rm * 4 + rs.rn) {
        case 1: launch_regtile_t<0, 1>(a, rs, item_begin, n_items, arenas, s); break;
        case 2: launch_regtile_t<0, 2>(a, rs, item_begin, n_items, arenas, s); break;
        case 3: launch_regtile_t<0, 3>(a, rs, item_begin, n_items, arenas, s); break;
        case 4: launch_regtile_t<1, 0>(a, rs, item_begin, n_items, arenas, s); break;
        case 5: launch_regtile_t<1, 1>(a, rs, item_begin, n_items, arenas, s); break;
        case 6: launch_regtile_t<1, 2>(a, rs, item_begin, n_items, arenas, s); break;
        case 7: launch_regtile_t<1, 3>(a, rs, item_begin, n_items, arenas, s); break;
        case 8: launch_regtile_t<2, 0>(a, rs, item_begin, n_items, arenas, s); break;
        case 9: launch_regtile_t<2, 1>(a, rs, item_begin, n_items, arenas, s); break;
        case 10: launch_regtile_t<2, 2>(a, rs, item_begin, n_items, arenas, s); break;
        case 11: launch_regtile_t<2, 3>(a, rs, item_begin, n_items, arenas, s); break;
        case 12: launch_regtile_t<3, 0>(a, rs, item_begin, n_items, arenas, s); break;
        case 13: launch_regtile_t<3, 1>(a, rs, item_begin, n_items, arenas, s); break;
        case 14: launch_regtile_t<3, 2>(a, rs, item_begin, n_items, arenas, s); break;
        default: launch_regtile_t<3, 3>(a, rs, item_begin, n_items, arenas, s); break;
    }
    return counted(cudaGetLastError());
}

int persistent_blocks_per_sm() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, persistent_program_kernel, 256, 0) != cudaSuccess) return 0;
    return n;
}

cudaError_t launch_persistent(const LaunchArgs &a, int64_t item_begin, int64_t n_items, float2 *arenas,
                              unsigned *bar_count, unsigned *bar_gen, int grid, cudaStream_t s) {
    LaunchArgs aa = a;
    void *args[] = {&aa, &item_begin, &n_items, &arenas, &bar_count, &bar_gen};
    return counted(cudaLaunchCooperativeKernel((const void *)persistent_program_kernel, dim3(grid), dim3(256), args, 0, s));
}

cudaError_t launch_finish_items(const LaunchArgs &a, int64_t item_begin, int64_t n_items,
                                const float2 *arenas, cudaStream_t s) {
    const int per_block = 8;
    const int64_t blocks = (n_items + per_block - 1) / per_block;
    finish_kernel<<<(unsigned)blocks, 32 * per_block, 0, s>>>(a, item_begin, n_items, arenas);
    return counted(cudaGetLastError());
}

cudaError_t launch_slice_sum(const unsigned char *image, const ExactPair *partials, int64_t batch, int64_t o_count,
                             double *amps, unsigned *status, cudaStream_t s) {
    slice_sum_kernel<<<(unsigned)batch, 256, 0, s>>>(image, partials, o_count, amps, status);
    return counted(cudaGetLastError());
}

}  // namespace qvx
