// Launchers of the device kernels (kernels.cu). All take the caller's stream and return
// the cudaError_t of the launch.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "device_program.h"

namespace qvx {

// An exact partial sum of complex slice terms: real and imaginary parts each a 128-bit
// two's-complement integer X standing for X * 2^-100 (every complex64 term with magnitude
// between 2^-77 and 2^27 converts without rounding and sums exactly).
struct ExactPair {
    unsigned long long re_lo, re_hi, im_lo, im_hi;
};

struct LaunchArgs {
    const unsigned char *image;     // device image (DevProgram first)
    const uint64_t *bitstrings;     // device, batch x words entries
    int64_t batch;
    uint32_t words;                 // 64-bit words per bitstring (1: up to 64 qubits, 2: up to 128)
    int64_t o_begin, o_count;       // outer slice numbers of this call
    int64_t s_begin, s_end;         // slice range summed / written
    uint64_t arena_elems;
    uint32_t n_steps, n_inner;
    ExactPair *partials;            // batch * o_count exact item sums (before the plan's scalar)
    float2 *terms;                  // optional: batch * (s_end - s_begin) slice terms
    unsigned int *status;           // device status word
    unsigned int *counter;          // CTAs finished (fused engine's final sum); zero between calls
    double *amps;                   // optional: 2 * batch FP64 amplitudes written by the fused engine
    // fused engine shared-memory layout: [steps][leaf data][leaf table][per group: leaf bases, arena]
    uint32_t smem_steps_bytes;      // 0: the program is read from global memory
    uint32_t smem_leaf_bytes;
    uint32_t smem_leaves_bytes;
    uint32_t leaf_table_bytes;      // per group, 16-byte multiple
    uint32_t group_bytes;           // per group: leaf table + arena
    // fused engine: the image header fields it needs before staging (passed as arguments so
    // the copies start without a round trip to the header in device memory)
    uint64_t fused_steps_off, fused_tab_off, fused_lane_map_off, leaves_off, leaf_data_off, final_off;
    uint32_t n_fused_phases, n_leaves;
    // self-test of the fused kernel's failure path: 1 makes the first staging wait give up at
    // once (the copies then get the normal bounded wait before the CTA moves on); 0 normally
    uint32_t selftest_stage_timeout;
};

// Fused engine: one warp group per work item, every tensor in shared memory. When
// a.amps is set, the last CTA to finish also adds the item partials (exactly).
cudaError_t launch_fused(const LaunchArgs &a, int warps_per_item, int items_per_cta, int grid,
                         size_t smem_bytes, cudaStream_t s);
int fused_blocks_per_sm(int threads, size_t smem_bytes, bool staged);
cudaError_t fused_prepare(size_t smem_bytes);
// Shared-memory layout of a fused launch: fills a's smem fields, the bytes shared by the
// CTA, the bytes per work-item group and the most groups a CTA can hold; false if one
// group's arena does not fit.
bool fused_shape(const DevProgram *h, uint64_t arena_elems, int warps_per_item, LaunchArgs *a, size_t *shared,
                 size_t *group, int *max_ipc);

// Stepwise engine: one launch per program step over `n_items` work items, tensors in a
// global-memory arena per item.
cudaError_t launch_step(const LaunchArgs &a, uint32_t step, int64_t item_begin, int64_t n_items,
                        float2 *arenas, uint32_t rc, cudaStream_t s);
// Several independent small steps (of one level phase) in one launch: step j takes the CTAs
// [first_block[j], first_block[j + 1]), one thread per output entry of each work item.
constexpr int kMaxGroupSteps = 24;
struct StepGroup {
    uint32_t n;
    uint32_t step[kMaxGroupSteps];
    uint32_t first_block[kMaxGroupSteps + 1];
};
cudaError_t launch_step_group(const LaunchArgs &a, const StepGroup &g, int64_t item_begin, int64_t n_items,
                              float2 *arenas, cudaStream_t s);
// Contraction with many summed entries: 32 outputs per CTA, the summed index split over warps.
cudaError_t launch_splitk_step(const LaunchArgs &a, uint32_t step, int64_t item_begin, int64_t n_items,
                               float2 *arenas, uint32_t rc, cudaStream_t s);
// Register-tiled form of a two-operand step (2^rm x 2^rn outputs per thread, rm, rn <= 2).
cudaError_t launch_regtile_step(const LaunchArgs &a, const RegTileStep &rs, int64_t item_begin, int64_t n_items,
                                float2 *arenas, cudaStream_t s);
// Persistent engine: one cooperative launch per chunk of work items (grid <= co-resident CTAs).
int persistent_blocks_per_sm();
cudaError_t launch_persistent(const LaunchArgs &a, int64_t item_begin, int64_t n_items, float2 *arenas,
                              unsigned *bar_count, unsigned *bar_gen, int grid, cudaStream_t s);
cudaError_t launch_finish_items(const LaunchArgs &a, int64_t item_begin, int64_t n_items,
                                const float2 *arenas, cudaStream_t s);

// Gradient program (one CTA per work item, arenas in global memory).
struct GradArgs {
    unsigned char *image;           // workspace copy of the image (its parametrised leaves are rewritten)
    const uint64_t *bitstrings;     // batch x words entries
    uint32_t words;
    int64_t batch, o_count;
    float2 *arenas;                 // slots * grad_arena_elems
    uint64_t arena_elems;
    int64_t slots;
    ExactPair *partials;            // batch * o_count amplitude partials
    ExactPair *gpart;               // batch * o_count * n_param_leaves derivative partials
    unsigned int *status;           // device status word
    // staged form of the shared-memory kernel: bytes of the leaf data, derivative data and
    // summed-index table copied into shared memory after the arena and leaf table (0: read
    // from the image in device memory)
    uint32_t stage_ldata, stage_ddata, stage_ktab;
};
// Rewrites the parametrised leaves (U and dU/dtheta) from thetas (device, or the image's own).
cudaError_t launch_set_params(unsigned char *image, uint32_t n_param_leaves, const double *thetas, cudaStream_t s);
cudaError_t launch_grad_program(const GradArgs &g, int grid, cudaStream_t s);
// The same program from its per-entry records with the work item's arena in shared memory:
// the bytes a CTA needs (0 if the plan has no records), how many CTAs fit on an SM (0: none;
// raises the kernel's shared-memory limit once per device), and the launch.
size_t grad_smem_bytes(const DevProgram *h);
// Bytes the staged form adds (leaf data, derivative data and summed-index table, each rounded
// to 16), and the matching GradArgs fields.
size_t grad_stage_bytes(const DevProgram *h, GradArgs *g);
int grad_smem_blocks_per_sm(size_t smem_bytes, bool staged);
cudaError_t launch_grad_smem(const GradArgs &g, int grid, size_t smem_bytes, cudaStream_t s);
// d alpha / d theta_p = exact sum over work items and the parameter's leaves.
// A sum outside the exact range sets QVX_ERANGE; NaN is written when the status word is set.
cudaError_t launch_grad_sum(const unsigned char *image, const ExactPair *gpart, int64_t batch, int64_t o_count,
                            uint32_t n_param_leaves, uint32_t n_params, double *grad, unsigned *status, cudaStream_t s);

// Kernels the calling host thread has launched through these launchers (successful launches);
// launch_counted(e) counts one launch if e is cudaSuccess and returns e.
uint64_t launches_issued();
cudaError_t launch_counted(cudaError_t e);
// Tensor-core form of a dense step (gemm_tc.cu): the column tile size, and the launch for
// items [item0, item0 + n_items) whose arenas start at `arenas` (operands are read from the
// arenas as complex64 and split into bf16 parts inside the kernel).
uint32_t gemm_nt(const GemmStep &g);
cudaError_t launch_gemm_step(const LaunchArgs &a, const GemmStep &g, int64_t item0, int64_t n_items, float2 *arenas,
                             cudaStream_t s);
// Self-test of the bounded waits (grid barrier and mbarrier that can never complete).
cudaError_t launch_wait_selftest(unsigned *words, unsigned *status, uint32_t polls, unsigned *out, cudaStream_t s);

// Exact sum of the item partials of every bitstring (Section 3.B.2: the slice terms are
// added), rounded once to FP64 and times the plan's scalar. A sum outside the exact range
// sets QVX_ERANGE in the status word; an amplitude is written as NaN when the status word is
// set (by this kernel or an earlier one of the call).
cudaError_t launch_slice_sum(const unsigned char *image, const ExactPair *partials, int64_t batch, int64_t o_count,
                             double *amps, unsigned *status, cudaStream_t s);

}  // namespace qvx
