// Device kernels: the pairwise contraction program (fused and stepwise engines) and the
// FP64 compensated sum of the slice terms.
#include <cuda_runtime.h>

#include "device_program.h"
#include "kernels.h"

namespace qvx {
namespace {

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

__device__ __forceinline__ double2 warp_sum(double2 v) {
    for (int d = 16; d > 0; d >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, d);
        v.y += __shfl_down_sync(0xffffffffu, v.y, d);
    }
    return v;
}

// Sum of the inner slice terms of the item's final tensor that fall in [s_begin, s_end)
// (FP64), times the plan's scalar; optionally writes each term.
__device__ void finish_item(const DevProgram *P, const LaunchArgs &a, const float2 *fin, int64_t b,
                            uint64_t o, int lane, int lanes) {
    const uint64_t x = a.bitstrings[b];
    const bool zero = (x & P->zero_mask) != 0;
    const double sr = P->scalar_re, si = P->scalar_im;
    double2 acc = make_double2(0.0, 0.0);
    const uint32_t n_in = P->n_inner, present = P->final_present;
    for (uint32_t i = lane; i < (1u << n_in); i += lanes) {
        const int64_t s = (int64_t)((o << n_in) | i);
        if (s < a.s_begin || s >= a.s_end) continue;
        uint32_t fi = 0, bit = 0;
        for (uint32_t j = 0; j < n_in; j++)
            if ((present >> j) & 1u) fi |= ((i >> j) & 1u) << bit++;
        const float2 t = zero ? make_float2(0.f, 0.f) : fin[fi];
        const double tr = (double)t.x * sr - (double)t.y * si;
        const double ti = (double)t.x * si + (double)t.y * sr;
        acc.x += tr;
        acc.y += ti;
        if (a.terms) a.terms[b * (a.s_end - a.s_begin) + (s - a.s_begin)] = make_float2((float)tr, (float)ti);
    }
    if (lanes == 32) {
        acc = warp_sum(acc);
        if (lane == 0) a.partials[b * a.o_count + (int64_t)(o - (uint64_t)a.o_begin)] = acc;
    }
}

// ------------------------------------------------------------------ compensated sums
// Neumaier's compensated addition, and Knuth's exact two-sum to merge (sum, compensation)
// pairs, so partial sums from many threads combine without losing the compensation.
__device__ __forceinline__ void neumaier_add(double &s, double &c, double v) {
    const double t = s + v;
    if (fabs(s) >= fabs(v)) c += (s - t) + v;
    else c += (v - t) + s;
    s = t;
}

__device__ __forceinline__ void merge_pair(double &s, double &c, double s2, double c2) {
    const double t = s + s2;
    const double bp = t - s;
    const double err = (s - (t - bp)) + (s2 - bp);
    s = t;
    c = c + c2 + err;
}

// Block-wide compensated sum of partials[0..n) (stride 1, double2): result in thread 0.
__device__ double2 block_compensated_sum(const double2 *partials, int64_t n) {
    __shared__ double red[4][32];
    double sr = 0, cr = 0, si = 0, ci = 0;
    for (int64_t o = threadIdx.x; o < n; o += blockDim.x) {
        const double2 v = __ldcg(partials + o);   // written by other CTAs: read from L2
        neumaier_add(sr, cr, v.x);
        neumaier_add(si, ci, v.y);
    }
    for (int d = 16; d > 0; d >>= 1) {
        const double a = __shfl_down_sync(0xffffffffu, sr, d), b = __shfl_down_sync(0xffffffffu, cr, d);
        const double e = __shfl_down_sync(0xffffffffu, si, d), f = __shfl_down_sync(0xffffffffu, ci, d);
        merge_pair(sr, cr, a, b);
        merge_pair(si, ci, e, f);
    }
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
    __syncthreads();
    if (lane == 0) {
        red[0][warp] = sr; red[1][warp] = cr; red[2][warp] = si; red[3][warp] = ci;
    }
    __syncthreads();
    double2 out = make_double2(0.0, 0.0);
    if (threadIdx.x == 0) {
        double s0 = red[0][0], c0 = red[1][0], s1 = red[2][0], c1 = red[3][0];
        for (int w = 1; w < nw; w++) {
            merge_pair(s0, c0, red[0][w], red[1][w]);
            merge_pair(s1, c1, red[2][w], red[3][w]);
        }
        out = make_double2(s0 + c0, s1 + c1);
    }
    return out;
}

// ------------------------------------------------------------------ fused engine
// Each group of `warps_per_item` warps runs the whole program for one work item
// (bitstring b, outer slice o); groups loop over items. Shared memory holds, per CTA, the
// step descriptors and the leaf data (when they fit), and per group the item's leaf base
// offsets and its tensor arena.
__device__ __forceinline__ void copy_to_smem(void *dst, const void *src, size_t bytes) {
    uint4 *d = reinterpret_cast<uint4 *>(dst);
    const uint4 *s = reinterpret_cast<const uint4 *>(src);
    for (size_t i = threadIdx.x; i < bytes / 16; i += blockDim.x) d[i] = __ldg(s + i);
}

// One output entry of a fused step: e packs the operands' offsets pext(c).
__device__ __forceinline__ float2 fused_entry(const FusedStep &st, uint32_t e, const float2 *__restrict__ A,
                                              const float2 *__restrict__ B, bool unary) {
    const uint32_t ia = e & 0xffffu, ib = e >> 16;
    const uint32_t nab = st.nk_ab, na = st.nk_a;
    const uint32_t nk = nab + na + st.nk_b;
    const uint32_t mask_ka = (1u << (nab + na)) - 1u, mask_ab = (1u << nab) - 1u;
    float2 acc = make_float2(0.f, 0.f);
    if (unary) {
        for (uint32_t k = 0; k < (1u << nk); k++) {
            const float2 v = A[ia + (k << st.a_cb)];
            acc.x += v.x;
            acc.y += v.y;
        }
        return acc;
    }
#pragma unroll 2
    for (uint32_t k = 0; k < (1u << nk); k++) {
        const uint32_t ka = k & mask_ka;
        const uint32_t kb = (k & mask_ab) | ((k >> (nab + na)) << nab);
        cmac(acc, A[ia + (ka << st.a_cb)], B[ib + (kb << st.b_cb)]);
    }
    return acc;
}

__global__ void __launch_bounds__(256) fused_program_kernel(LaunchArgs a, int warps_per_item) {
    extern __shared__ __align__(16) unsigned char smem[];
    const unsigned char *img = a.image;
    const DevProgram *P = reinterpret_cast<const DevProgram *>(img);
    const DevLeaf *leaves = reinterpret_cast<const DevLeaf *>(img + P->leaves_off);
    const FusedStep *steps = reinterpret_cast<const FusedStep *>(img + P->fused_steps_off);
    const uint32_t *tabs = reinterpret_cast<const uint32_t *>(img + P->fused_tab_off);
    const float2 *ldata = reinterpret_cast<const float2 *>(img + P->leaf_data_off);
    unsigned char *cur = smem;
    if (a.smem_steps_bytes) {
        // fused steps and their tables are contiguous in the image
        copy_to_smem(cur, steps, a.smem_steps_bytes);
        const size_t tab_rel = P->fused_tab_off - P->fused_steps_off;
        steps = reinterpret_cast<const FusedStep *>(cur);
        tabs = reinterpret_cast<const uint32_t *>(cur + tab_rel);
        cur += a.smem_steps_bytes;
    }
    if (a.smem_leaf_bytes) {
        copy_to_smem(cur, ldata, a.smem_leaf_bytes);
        ldata = reinterpret_cast<const float2 *>(cur);
        cur += a.smem_leaf_bytes;
    }
    __syncthreads();
    const int lanes = 32 * warps_per_item;
    const int group = threadIdx.x / lanes;
    const int lane = threadIdx.x % lanes;
    const int groups = blockDim.x / lanes;
    unsigned char *mine = cur + (size_t)group * a.group_bytes;
    uint32_t *lbase = reinterpret_cast<uint32_t *>(mine);
    float2 *arena = reinterpret_cast<float2 *>(mine + a.leaf_table_bytes);
    const int64_t n_items = a.batch * a.o_count;
    const unsigned bar_id = 1 + group;
    const uint32_t n_leaves = P->n_leaves;
    for (int64_t item = (int64_t)blockIdx.x * groups + group; item < n_items;
         item += (int64_t)gridDim.x * groups) {
        const int64_t b = item / a.o_count;
        const uint64_t o = (uint64_t)(a.o_begin + item % a.o_count);
        const uint64_t x = a.bitstrings[b];
        for (uint32_t l = lane; l < n_leaves; l += lanes) lbase[l] = leaf_base(leaves[l], x, o);
        if (warps_per_item == 1) __syncwarp();
        else asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(lanes));
        for (uint32_t s = 0; s < a.n_steps; s++) {
            const FusedStep st = steps[s];
            const uint32_t flags = st.flags;
            const bool unary = flags & kStepUnary;
            const float2 *A = (flags & kStepALeaf) ? ldata + lbase[st.a_off] : arena + st.a_off;
            const float2 *B = unary ? A : ((flags & kStepBLeaf) ? ldata + lbase[st.b_off] : arena + st.b_off);
            float2 *C = arena + st.c_off;
            const uint32_t *tab = tabs + st.tab_off;
            for (uint32_t c = lane; c < (1u << st.rc); c += lanes) C[c] = fused_entry(st, tab[c], A, B, unary);
            if (warps_per_item == 1) __syncwarp();
            else asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(lanes));
        }
        if (lane < 32) finish_item(P, a, arena + P->final_off, b, o, lane, 32);
        if (warps_per_item == 1) __syncwarp();
        else asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(lanes));
    }
    if (a.amps == nullptr) return;
    // the last CTA to finish adds every bitstring's item partials
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned ticket = atomicAdd(a.counter, 1u);
        last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int64_t b = 0; b < a.batch; b++) {
        const double2 r = block_compensated_sum(a.partials + b * a.o_count, a.o_count);
        if (threadIdx.x == 0) {
            a.amps[2 * b] = r.x;
            a.amps[2 * b + 1] = r.y;
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
    const uint64_t x = a.bitstrings[b];
    float2 *arena = arenas + (uint64_t)il * a.arena_elems;
    const bool unary = st.flags & kStepUnary;
    const DevLeaf *leaves = reinterpret_cast<const DevLeaf *>(img + P->leaves_off);
    const float2 *ldata = reinterpret_cast<const float2 *>(img + P->leaf_data_off);
    const float2 *A = (st.flags & kStepALeaf) ? ldata + leaf_base(leaves[st.a_off], x, o) : arena + st.a_off;
    const float2 *B = unary ? A
                            : ((st.flags & kStepBLeaf) ? ldata + leaf_base(leaves[st.b_off], x, o) : arena + st.b_off);
    arena[st.c_off + c] = step_entry(st, c, A, B, unary);
}

__global__ void finish_kernel(LaunchArgs a, int64_t item_begin, int64_t n_items, const float2 *arenas) {
    const DevProgram *P = reinterpret_cast<const DevProgram *>(a.image);
    const int64_t il = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    if (il >= n_items) return;
    const int64_t item = item_begin + il;
    const int64_t b = item / a.o_count;
    const uint64_t o = (uint64_t)(a.o_begin + item % a.o_count);
    finish_item(P, a, arenas + (uint64_t)il * a.arena_elems + P->final_off, b, o, threadIdx.x % 32, 32);
}

// ------------------------------------------------------------------ slice sum
__global__ void slice_sum_kernel(const double2 *partials, int64_t o_count, double *amps) {
    const int64_t b = blockIdx.x;
    const double2 r = block_compensated_sum(partials + b * o_count, o_count);
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
                                                  const unsigned char *img, float2 *arena, uint64_t x,
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
    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int64_t b = item / g.o_count;
        const uint64_t o = (uint64_t)(item % g.o_count);
        const uint64_t x = g.bitstrings[b];
        for (uint32_t s = 0; s < P->n_grad_steps; s++) {
            const GenStep &st = steps[s];
            const float2 *X = gen_base(st.x, P, img, arena, x, o);
            const float2 *Y = gen_base(st.y, P, img, arena, x, o);
            float2 *out = arena + st.out_off;
            for (uint32_t oi = threadIdx.x; oi < (1u << st.ro); oi += blockDim.x) {
                const uint32_t ox = runs_pdep(oi, st.x.oruns, st.x.n_oruns);
                const uint32_t oy = runs_pdep(oi, st.y.oruns, st.y.n_oruns);
                float2 acc = make_float2(0.f, 0.f);
                for (uint32_t k = 0; k < (1u << st.nk); k++) {
                    const float2 a = X ? X[ox + runs_pdep(k, st.x.kruns, st.x.n_kruns)] : make_float2(1.f, 0.f);
                    const float2 v = Y ? Y[oy + runs_pdep(k, st.y.kruns, st.y.n_kruns)] : make_float2(1.f, 0.f);
                    cmac(acc, a, v);
                }
                out[oi] = acc;
            }
            __syncthreads();
        }
        // amplitude partial: sum of the final tensor over the inner slice modes
        const bool zero = (x & P->zero_mask) != 0;
        if (threadIdx.x < 32) {
            const float2 *fin = arena + P->final_fwd_off;
            double2 acc = make_double2(0.0, 0.0);
            const uint32_t n_in = P->n_inner, present = P->final_present;
            for (uint32_t i = threadIdx.x; i < (1u << n_in); i += 32) {
                uint32_t fi = 0, bit = 0;
                for (uint32_t j = 0; j < n_in; j++)
                    if ((present >> j) & 1u) fi |= ((i >> j) & 1u) << bit++;
                const float2 t = fin[fi];
                acc.x += (double)t.x * P->scalar_re - (double)t.y * P->scalar_im;
                acc.y += (double)t.x * P->scalar_im + (double)t.y * P->scalar_re;
            }
            acc = warp_sum(acc);
            if (threadIdx.x == 0) g.partials[item] = zero ? make_double2(0.0, 0.0) : acc;
        }
        for (uint32_t lp = threadIdx.x; lp < npl; lp += blockDim.x) {
            const float2 t = arena[P->gslot_off + lp];
            const double2 v = make_double2((double)t.x * P->scalar_re - (double)t.y * P->scalar_im,
                                           (double)t.x * P->scalar_im + (double)t.y * P->scalar_re);
            g.gpart[(uint64_t)item * npl + lp] = zero ? make_double2(0.0, 0.0) : v;
        }
        __syncthreads();
    }
}

// One block per (bitstring, parameter): compensated sum over the work items and over the
// parameter's leaves (CSR lists in the image).
__global__ void grad_sum_kernel(const unsigned char *img, const double2 *gpart, int64_t o_count, uint32_t npl,
                                uint32_t n_params, double *grad) {
    __shared__ double red[4][32];
    const DevProgram *P = reinterpret_cast<const DevProgram *>(img);
    const uint32_t *csr = reinterpret_cast<const uint32_t *>(img + P->param_csr_off);
    const int64_t b = blockIdx.x / n_params;
    const uint32_t p = blockIdx.x % n_params;
    const uint32_t first = csr[p], last = csr[p + 1];
    const uint32_t *list = csr + n_params + 1;
    double sr = 0, cr = 0, si = 0, ci = 0;
    const int64_t n = (int64_t)(last - first) * o_count;
    for (int64_t t = threadIdx.x; t < n; t += blockDim.x) {
        const uint32_t lp = list[first + t / o_count];
        const int64_t o = t % o_count;
        const double2 v = gpart[((uint64_t)(b * o_count + o)) * npl + lp];
        neumaier_add(sr, cr, v.x);
        neumaier_add(si, ci, v.y);
    }
    for (int d = 16; d > 0; d >>= 1) {
        const double a = __shfl_down_sync(0xffffffffu, sr, d), bb = __shfl_down_sync(0xffffffffu, cr, d);
        const double e = __shfl_down_sync(0xffffffffu, si, d), f = __shfl_down_sync(0xffffffffu, ci, d);
        merge_pair(sr, cr, a, bb);
        merge_pair(si, ci, e, f);
    }
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
    if (lane == 0) {
        red[0][warp] = sr; red[1][warp] = cr; red[2][warp] = si; red[3][warp] = ci;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = red[0][0], c0 = red[1][0], s1 = red[2][0], c1 = red[3][0];
        for (int w = 1; w < nw; w++) {
            merge_pair(s0, c0, red[0][w], red[1][w]);
            merge_pair(s1, c1, red[2][w], red[3][w]);
        }
        grad[2 * (b * n_params + p)] = s0 + c0;
        grad[2 * (b * n_params + p) + 1] = s1 + c1;
    }
}

}  // namespace

cudaError_t launch_set_params(unsigned char *image, uint32_t n_param_leaves, const double *thetas, cudaStream_t s) {
    if (n_param_leaves == 0) return cudaSuccess;
    set_params_kernel<<<n_param_leaves, 32, 0, s>>>(image, thetas);
    return cudaGetLastError();
}

cudaError_t launch_grad_program(const GradArgs &g, int grid, cudaStream_t s) {
    grad_program_kernel<<<grid, 256, 0, s>>>(g);
    return cudaGetLastError();
}

cudaError_t launch_grad_sum(const unsigned char *image, const double2 *gpart, int64_t batch, int64_t o_count,
                            uint32_t n_param_leaves, uint32_t n_params, double *grad, cudaStream_t s) {
    if (n_params == 0 || batch == 0) return cudaSuccess;
    grad_sum_kernel<<<(unsigned)(batch * n_params), 256, 0, s>>>(image, gpart, o_count, n_param_leaves, n_params, grad);
    return cudaGetLastError();
}

cudaError_t fused_prepare(size_t smem_bytes) {
    return cudaFuncSetAttribute(fused_program_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_bytes);
}

int fused_blocks_per_sm(int threads, size_t smem_bytes) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fused_program_kernel, threads, smem_bytes) != cudaSuccess)
        return 0;
    return n;
}

cudaError_t launch_fused(const LaunchArgs &a, int warps_per_item, int items_per_cta, int grid,
                         size_t smem_bytes, cudaStream_t s) {
    const int threads = 32 * warps_per_item * items_per_cta;
    fused_program_kernel<<<grid, threads, smem_bytes, s>>>(a, warps_per_item);
    return cudaGetLastError();
}

cudaError_t launch_step(const LaunchArgs &a, uint32_t step, int64_t item_begin, int64_t n_items,
                        float2 *arenas, uint32_t rc, cudaStream_t s) {
    const uint64_t total = (uint64_t)n_items << rc;
    const int threads = 256;
    const uint64_t blocks = (total + threads - 1) / threads;
    step_kernel<<<(unsigned)blocks, threads, 0, s>>>(a, step, item_begin, n_items, arenas);
    return cudaGetLastError();
}

cudaError_t launch_finish_items(const LaunchArgs &a, int64_t item_begin, int64_t n_items,
                                const float2 *arenas, cudaStream_t s) {
    const int per_block = 8;
    const int64_t blocks = (n_items + per_block - 1) / per_block;
    finish_kernel<<<(unsigned)blocks, 32 * per_block, 0, s>>>(a, item_begin, n_items, arenas);
    return cudaGetLastError();
}

cudaError_t launch_slice_sum(const double2 *partials, int64_t batch, int64_t o_count, double *amps,
                             cudaStream_t s) {
    slice_sum_kernel<<<(unsigned)batch, 256, 0, s>>>(partials, o_count, amps);
    return cudaGetLastError();
}

}  // namespace qvx
