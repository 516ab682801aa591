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

// A leaf is stored with its consumer's modes in the low bits (in the consumer's order)
// and the modes fixed per work item above them. Entry e of the restricted leaf is stored
// entry data_off + e + sum over fixed modes f of value_f << fixed_pos[f].
struct DevLeaf {
    uint32_t data_off;             // first stored entry (complex64 units) in the leaf data
    uint32_t n_elem;               // entries after restriction (2^consumer rank)
    uint32_t n_fixed;              // modes fixed per work item
    uint32_t pad;
    uint8_t fixed_src[kMaxFixed];  // < 128: bit src of the bitstring (word src / 64, bit src % 64);
                                   // >= 128: bit (src - 128) of the outer slice number
    uint8_t fixed_pos[kMaxFixed];  // bit position of that mode in the stored leaf
};

// The fused engine's form of a step: operand offsets and a per-step table holding, for
// each output entry c, the operands' offsets pext(c) for A (low 16 bits) and B (high 16).
// Steps are grouped into phases of independent steps; lane_map[phase * lanes + lane] gives
// the step a lane of a work item's group works on (bits 0-11), the lane's index among the
// step's lanes (bits 12-21) and their count (bits 22-31), or 0xffffffff for none.
struct alignas(16) FusedStep {
    uint32_t a_off, b_off, c_off;  // arena offsets, or leaf indices (flags as in DevStep)
    uint32_t tab_off;              // first table entry of this step
    uint32_t flags;
    uint8_t rc, nk_ab, nk_a, nk_b;
    uint8_t a_cb, b_cb, nk, pad1;
    uint32_t pad2;
    uint16_t koff_a[8], koff_b[8]; // offsets of summed index k (nk <= 3) in A and B
};

// Gradient program: out[o] = sum_k X(o, k) * Y(o, k), each operand addressed through bit
// runs of the output index o and of the summed index k. Operand kinds: arena tensor, leaf
// data or leaf derivative data (restricted like a leaf), or the constant one.
constexpr uint32_t kOpArena = 0, kOpLeaf = 1, kOpDeriv = 2, kOpOne = 3;

struct GenOperand {
    uint64_t off;                  // arena offset, or device leaf index
    uint32_t kind;
    uint8_t n_oruns, n_kruns, pad0, pad1;
    DevRun oruns[kMaxRuns];        // output-index bits -> operand bits
    DevRun kruns[kMaxRuns];        // summed-index bits -> operand bits
};

struct GenStep {
    GenOperand x, y;
    uint64_t out_off;              // arena offset of the output
    uint32_t ro, nk;               // output rank, summed bits
};

// Tabulated form of the gradient program for the shared-memory gradient kernel: one record
// per output entry of every gradient step, in step order (so each level phase is one
// contiguous range of records). Operand v (X or Y) of the entry is base(kind, vr) + vo:
// the arena at offset vr, or the restricted leaf (or its derivative) vr of the work item.
struct GradEntry {
    uint16_t c;                    // arena offset of the output entry
    uint16_t meta;                 // X kind (bits 0-1), Y kind (bits 2-3), summed bits nk (bits 4-7)
    uint16_t xr, xo, yr, yo;
    uint32_t k1;                   // nk == 1: X and Y offsets of summed index 1 (low / high 16 bits);
                                   // nk >= 2: first of the 2^nk - 1 such pairs (index 1, 2, ...) in the k table
};

// A leaf that is one parametrised gate exp(-i theta (cos phi X + sin phi Y) / 2): its
// stored entry e is matrix element code[e] (bit 1: row, bit 0: column) of U or dU/dtheta.
struct ParamLeaf {
    uint32_t leaf;                 // device leaf index
    uint32_t param;                // index into the angle vector
    uint32_t n_stored;             // stored entries
    uint32_t code_off;             // first entry in the code array
    double phi;
};

// Register-tiled form of a two-operand step (global-arena engines). Each thread computes
// 2^rm x 2^rn output entries (rm, rn <= 3) that differ only in rm modes held by A alone and
// rn modes held by B alone, so every operand entry it loads serves 2^rn (from A) or 2^rm (from B) of its
// outputs. Thread t of a work item owns the entries c0 + c_m[i] + c_n[j], where
// c0 = pext-style move of t's bits by free_runs; its operand entries are
// A[pext(c0, runs_a) + a_m[i] + (ka << a_cb)] and B[pext(c0, runs_b) + b_n[j] + (kb << b_cb)]
// with ka, kb split from the summed index as in DevStep.
struct RegTileStep {
    uint64_t a_off, b_off, c_off;  // arena offsets or leaf indices (flags as in DevStep)
    uint32_t flags;
    uint8_t rc, nt, rm, rn;        // output rank, thread bits (rc - rm - rn), tile bits in A / B
    uint8_t nk_ab, nk_a, nk_b, a_cb, b_cb, n_free, na_runs, nb_runs;
    DevRun free_runs[6];           // thread index -> output entry with the tile bits zero
    DevRun runs_a[kMaxRuns], runs_b[kMaxRuns];
    uint32_t a_m[8], b_n[8], c_m[8], c_n[8];
};

// Tensor-core form of a dense two-operand step C[b, m, n] = sum_k A[b, m, k] B[b, k, n]
// (stepwise engine): b are the output modes held by A and B, m those held by A alone, n those
// held by B alone, k the summed modes (all held by both). A group's compact index (its modes
// in C's order; k in A's order) moves into an operand's entry index by bit runs. nk = 0:
// the step has no tensor-core form.
constexpr int kGroupRuns = 8;
struct GemmStep {
    uint64_t a_off, b_off, c_off;  // arena offsets or leaf indices (flags as in DevStep)
    uint32_t flags;
    uint8_t nb, nm, nn, nk;        // group sizes in bits
    uint8_t n_ab, n_am, n_ak, n_bb, n_bn, n_bk, n_cb, n_cm, n_cn, pad[3];
    DevRun ab[kGroupRuns], am[kGroupRuns], ak[kGroupRuns];   // A: b, m, k
    DevRun bb[kGroupRuns], bn[kGroupRuns], bk[kGroupRuns];   // B: b, n, k
    DevRun cb[kGroupRuns], cm[kGroupRuns], cn[kGroupRuns];   // C: b, m, n
};

struct DevProgram {
    uint32_t magic;
    uint32_t n_steps, n_leaves, pad0;
    uint64_t n_leaf_entries;       // complex64 entries of all stored leaves
    uint64_t arena_elems;          // complex64 entries of one work item's arena
    uint64_t final_off;            // arena offset of the final tensor (over the inner slice modes)
    uint32_t n_inner;              // inner (open) sliced variables
    uint32_t final_present;        // inner bits that are modes of the final tensor, low to high
    uint64_t zero_mask;            // amplitude is 0 when x & zero_mask != 0 (bitstring word 0;
                                   // word 1 against zero_mask_hi)
    double scalar_re, scalar_im;   // constant prefactor
    uint64_t n_outer;              // work items per bitstring = 2^(sliced - inner)
    uint64_t steps_off, leaves_off, leaf_data_off;  // byte offsets
    uint64_t fused_steps_off, fused_tab_off;        // byte offsets (0 if the fused form is absent)
    uint64_t n_tab_entries;
    uint64_t fused_lane_map_off;                    // byte offset, right after the tables
    uint32_t n_fused_phases, fused_lanes;
    // gradient program (zero when absent)
    uint64_t grad_steps_off, params_off, codes_off, deriv_data_off, thetas_off, param_csr_off;
    uint32_t n_grad_steps, n_param_leaves, n_params, grad_pad;
    uint64_t grad_arena_elems;
    uint64_t final_fwd_off;        // gradient arena offset of the final tensor
    uint64_t gslot_off;            // gradient arena offset of the per-leaf derivative slots
    uint64_t level_phases_off;     // byte offset of n_level_phases + 1 step indices (phase starts)
    uint32_t n_level_phases, n_grad_phases;
    uint64_t grad_phases_off;      // n_grad_phases + 1 gradient-step indices (phase starts)
    uint64_t grad_elem_off_off;    // per gradient step: its first entry inside its phase
    uint32_t n_open;               // open output qubits (2^n_open amplitudes per bitstring)
    uint32_t open_present;         // open qubits that are modes of the final tensor, low to high
    uint64_t regtile_off;          // byte offset of n_steps RegTileStep (0 if absent; rm + rn = 0: none)
    uint64_t gentry_off;           // byte offset of the GradEntry records (0 if absent)
    uint64_t gktab_off;            // byte offset of the k table (pairs of 16-bit offsets)
    uint64_t gphase_entry_off;     // byte offset of n_grad_phases + 1 record indices (phase starts)
    uint64_t gemm_off;             // byte offset of n_steps GemmStep (0 if absent)
    uint64_t image_bytes;
    uint64_t zero_mask_hi;         // qubits 64..127 of the zero mask
};

constexpr uint32_t kProgramMagic = 0x51565831u;  // "QVX1"

}  // namespace qvx

namespace qvx {
static_assert(sizeof(DevStep) == 136, "DevStep layout");
static_assert(sizeof(DevLeaf) == 40, "DevLeaf layout");
static_assert(sizeof(DevProgram) == 328, "DevProgram layout");
static_assert(sizeof(GemmStep) == 336, "GemmStep layout");
static_assert(sizeof(GradEntry) == 16, "GradEntry layout");
static_assert(sizeof(RegTileStep) == 288, "RegTileStep layout");
static_assert(sizeof(GenOperand) == 112, "GenOperand layout");
static_assert(sizeof(GenStep) == 240, "GenStep layout");
static_assert(sizeof(ParamLeaf) == 24, "ParamLeaf layout");
static_assert(sizeof(FusedStep) == 64, "FusedStep layout");
}  // namespace qvx
