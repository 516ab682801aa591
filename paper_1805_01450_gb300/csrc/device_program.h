// Layout of a plan's device image: plain structs read by the kernels and written by the
// host serializer. All offsets are counted from the start of the image.
#pragma once
#include <stdint.h>

namespace qvx {

constexpr int kMaxRuns = 12;       // contiguous bit runs per operand address map
constexpr int kMaxFixed = 12;      // modes of one leaf fixed per work item
constexpr uint32_t kStepUnary = 1;  // the step has no second operand
constexpr uint32_t kStepALeaf = 2;  // operand A is a leaf: a_off is its leaf index
constexpr uint32_t kStepBLeaf = 4;  // operand B is a leaf: b_off is its leaf index

// out[c] = sum_k A[pext(c, runs_a) + (ka << a_cb)] * B[pext(c, runs_b) + (kb << b_cb)]
// where the summed index k = [k_ab | k_a | k_b] (low to high),
// ka = k & ((1 << (nk_ab + nk_a)) - 1), kb = (k & ((1 << nk_ab) - 1)) | ((k >> (nk_ab + nk_a)) << nk_ab).
struct DevRun {
    uint8_t src, len, dst, pad;    // ((c >> src) & ((1 << len) - 1)) << dst
};

struct DevStep {
    uint64_t a_off, b_off, c_off;  // arena offsets (complex64 entries) or leaf indices (flags)
    uint8_t rc;                    // output rank
    uint8_t nk_ab, nk_a, nk_b;     // summed modes shared by A and B, in A only, in B only
    uint8_t a_cb, b_cb;            // number of output modes held by A, by B
    uint8_t na_runs, nb_runs;
    uint32_t flags;
    uint32_t pad;
    DevRun runs_a[kMaxRuns];
    DevRun runs_b[kMaxRuns];
};

// A leaf is read in its consumer's layout: entry e of the restricted leaf is stored entry
// elem_map[elem_off + e] + (sum over fixed modes of value << fixed_pos) after data_off.
struct DevLeaf {
    uint32_t data_off;             // first stored entry (complex64 units) in the leaf data
    uint32_t elem_off;             // first entry of this leaf in the element map
    uint32_t n_elem;               // entries after restriction (2^consumer rank)
    uint32_t n_fixed;              // modes fixed per work item
    uint8_t fixed_src[kMaxFixed];  // < 64: bit of the bitstring; >= 64: bit (src-64) of the outer slice number
    uint8_t fixed_pos[kMaxFixed];  // bit position of that mode in the stored leaf
};

struct DevProgram {
    uint32_t magic;
    uint32_t n_steps, n_leaves, n_leaf_elems;
    uint64_t arena_elems;          // complex64 entries of one work item's arena
    uint64_t final_off;            // arena offset of the final tensor (over the inner slice modes)
    uint32_t n_inner;              // inner (open) sliced variables
    uint32_t final_present;        // inner bits that are modes of the final tensor, low to high
    uint64_t zero_mask;            // amplitude is 0 when x & zero_mask != 0
    double scalar_re, scalar_im;   // constant prefactor
    uint64_t n_outer;              // work items per bitstring = 2^(sliced - inner)
    uint64_t steps_off, leaves_off, elem_map_off, leaf_data_off;  // byte offsets
    uint64_t image_bytes;
};

constexpr uint32_t kProgramMagic = 0x51565831u;  // "QVX1"

}  // namespace qvx
