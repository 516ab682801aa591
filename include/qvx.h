/* qvx: single amplitudes <x|C|0...0> of quantum circuits by variable elimination on the
 * circuit's undirected graphical model, with sliced variables, on one GB300 (sm_103a).
 *
 * Method (arXiv:1805.01450):
 *   - the amplitude is the Feynman path sum of Eq. (1);
 *   - every distinct path variable is a vertex of an undirected graph; diagonal gates
 *     (T, CZ) add no variable, non-diagonal single-qubit gates start a new one
 *     (Section 3.A, Fig. 3); input and output vertices are fixed and removed (Section 3.B.2);
 *   - variables are summed one at a time in an elimination order (Section 3.B.1), whose
 *     cost is the sum over steps of 2^deg(v) (Section 3.B.1, last paragraph);
 *   - k chosen variables are fixed ("sliced"), which splits the sum into 2^k independent
 *     terms that are added at the end (Section 3.B.2); they are chosen greedily by the cost
 *     under a first ordering, and the graph is then re-ordered (Section 3.B.3).
 *
 * Conventions for every entry point:
 *   - Ownership: the caller owns every buffer it passes. A plan copies what it needs from
 *     the circuit and the lists; it is owned by the library until qvx_plan_destroy.
 *   - Device memory: the library never allocates device memory. The caller passes a
 *     workspace of at least qvx_workspace_size bytes (256-byte aligned); it holds the
 *     plan's device image, the intermediate tensors and a device status word.
 *   - Streams: all device work is enqueued on the caller's stream; calls return without
 *     synchronising unless stated.
 *   - Bitstrings: W = ceil(n_qubits / 64) uint64_t words per bitstring (n_qubits <= 128, so
 *     W is 1 or 2), bitstring b at words [b*W, b*W + W): the value of qubit q is bit q % 64
 *     of word q / 64. With up to 64 qubits a bitstring is one uint64_t, bit q = qubit q.
 *   - Amplitudes: complex128, interleaved (re, im).
 *   - Errors: every call returns a qvx_status; qvx_last_error() gives a message for the
 *     calling thread's last failure. Failures inside kernels (a bounded wait that ran out, a
 *     slice term or exact sum outside the exact range) set the device status word, read by
 *     qvx_workspace_status; every amplitude written while it is set is NaN. Device indices
 *     need no run-time check: every offset a kernel forms is a bit-run map of an index below
 *     2^rank of the tensor it addresses, fixed when the plan is built.
 */
#ifndef QVX_H
#define QVX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    QVX_OK = 0,
    QVX_EINVAL = 1,        /* bad argument: sizes, ids, a bitstring with bits >= n_qubits */
    QVX_ENOMEM = 2,        /* host allocation failed, or a workspace/plan exceeds a limit */
    QVX_ECUDA = 3,         /* a CUDA runtime call failed (message in qvx_last_error) */
    QVX_ETIMEOUT = 4,      /* a bounded device wait ran out (device status word) */
    QVX_EUNSUPPORTED = 5,  /* a gate, rank or size outside what the plan can run */
    QVX_ERANGE = 6         /* a slice term or an exact partial sum was not finite or had magnitude
                              2^27 or more, outside the 128-bit fixed-point sum (device status word) */
} qvx_status;

/* Gate kinds (matrices indexed [output, input]):
 *   H       [[1,1],[1,-1]]/sqrt(2)
 *   T       diag(1, e^{i pi/4})
 *   SQRT_X  (1/2)[[1+i, 1-i],[1-i, 1+i]]     (principal square root of X)
 *   SQRT_Y  (1/2)[[1+i, -1-i],[1+i, 1+i]]    (principal square root of Y)
 *   CZ      diag(1,1,1,-1) on (q0, q1)
 *   RXY     exp(-i theta (cos(phi) X + sin(phi) Y)/2), parametrised by theta
 *   U1      any 2x2 matrix u[8] = (re, im) row-major; treated as non-diagonal */
typedef enum {
    QVX_GATE_H = 0,
    QVX_GATE_T = 1,
    QVX_GATE_SQRT_X = 2,
    QVX_GATE_SQRT_Y = 3,
    QVX_GATE_CZ = 4,
    QVX_GATE_RXY = 5,
    QVX_GATE_U1 = 6
} qvx_gate_kind;

typedef struct {
    int32_t kind;          /* qvx_gate_kind */
    int32_t q0, q1;        /* q1 = -1 for single-qubit gates */
    int32_t param_index;   /* RXY: index into a theta vector for gradients, or -1 */
    double theta, phi;     /* RXY angles */
    double u[8];           /* U1 matrix */
} qvx_gate;

typedef struct {
    int32_t n_qubits;      /* 1..128 */
    int32_t reserved;
    int64_t n_gates;
    const qvx_gate *gates; /* in time order */
} qvx_circuit;

/* FUSED: one warp group per work item, every tensor in shared memory (small programs).
 * STEPWISE: one kernel launch per contraction over all work items in flight (global arenas).
 * PERSISTENT: one cooperative launch per chunk of work items that walks the contractions
 * level by level, with a grid-wide barrier (bounded wait) between levels (global arenas).
 * AUTO: FUSED when a work item's tensors fit in shared memory, else PERSISTENT. */
typedef enum { QVX_ENGINE_AUTO = 0, QVX_ENGINE_FUSED = 1, QVX_ENGINE_STEPWISE = 2, QVX_ENGINE_PERSISTENT = 3 } qvx_engine;

typedef struct {
    int32_t n_slices;          /* sliced variables when the planner picks them; -1: as many as
                                  the memory budget needs (0 if none) */
    int32_t order_restarts;    /* randomised min-fill orderings tried (best kept), >= 1 */
    uint64_t order_seed;       /* seed of the ordering's random tie-breaks */
    int64_t mem_budget_bytes;  /* per-work-item tensor budget of the stepwise engine */
    int32_t engine;            /* qvx_engine */
    int32_t inner_slices;      /* sliced variables kept open inside one work item; -1 auto */
    int32_t max_rank;          /* largest tensor rank a plan may create (<= 30) */
    int32_t warps_per_item;    /* fused engine: warps sharing one work item (1, 2, 4, 8 or 16) */
    int32_t host_merge_rank;   /* two leaves whose product has at most this many modes (modes
                                  fixed per work item included) are contracted on the host in
                                  FP64 at plan time; 0 keeps every contraction on the device */
    int32_t gradient;          /* 1: the plan also serves qvx_amplitude_grad (every gate with
                                  param_index >= 0 stays a tensor of its own) */
    int32_t slice_rule;        /* how the planner picks sliced variables: 0 the greedy rule of
                                  Section 3.B.2 (cost under the first ordering); 1 the same with
                                  the graph re-ordered after every removal (Section 6's larger
                                  circuits); 2 only candidates that sit on two or more CZ gates
                                  (the observation of Section 6), then the greedy rule */
    int32_t n_open_qubits;     /* 0..16: qubits whose output stays open, so one contraction gives
                                  2^n_open_qubits amplitudes per bitstring (Section 6: batches of
                                  amplitudes). Not with gradient plans. */
    int32_t open_qubits[16];   /* the open qubits; amplitude j of a bitstring sets open_qubits[i]
                                  to bit i of j (the bitstring's own bits there are ignored) */
    int32_t tensor_cores;      /* stepwise engine: 1 runs the dense contractions (16 to 1024
                                  summed entries, 64 output entries of one operand's own and 16 of
                                  the other's, 12 or more flops per algorithmic byte) as complex
                                  GEMMs on the tcgen05 tensor cores, each FP32 operand split into
                                  three bf16 parts (six products, FP32 accumulation: about 2^-23
                                  relative error per product); 0 keeps them on FP32 SIMT kernels */
    int32_t plan_trials;       /* 1 ... 65536 independent planning trials (ordering, slice choice and
                                  re-ordering, each from its own seed; trial 0 from order_seed);
                                  the plan with the smallest bandwidth-weighted contraction
                                  estimate is kept. Ignored when both order and slices are given */
} qvx_plan_opts;

typedef struct {
    int32_t n_qubits, n_vars, n_edges, n_sliced, n_inner, n_steps, n_leaves, max_rank;
    int32_t engine, warps_per_item;
    int64_t n_items_per_bitstring;   /* 2^(n_sliced - n_inner) */
    double log2_cost;                /* log2 of sum over steps of 2^deg(v), per slice */
    double log2_cost_unsliced;       /* the same for the first ordering, nothing sliced */
    double flops_per_amplitude;      /* algorithmic real flops: 8 * 2^|S_A u S_B| per step, all items */
    double bytes_per_amplitude;      /* algorithmic tensor bytes read + written, all items */
    int64_t arena_bytes;             /* tensor memory of one work item */
    int64_t device_image_bytes;      /* program, leaves and tables */
    int32_t n_params;                /* 1 + largest param_index (gradient plans), else 0 */
    int32_t n_grad_steps;            /* contractions of the gradient program (0 if none) */
    int64_t grad_arena_bytes;        /* gradient program memory of one work item */
    double grad_flops_per_amplitude; /* algorithmic real flops of the gradient program, all items */
    double grad_bytes_per_amplitude; /* its algorithmic tensor bytes, all items */
    int32_t n_tiled_steps;           /* contractions with a register-tiled form (global-arena engines) */
    int32_t n_phases;                /* levels of mutually independent contractions */
    int32_t n_open_qubits;           /* amplitudes per bitstring = 2^n_open_qubits */
    int32_t n_gemm_steps;            /* contractions run on the tensor cores (opts.tensor_cores) */
    int32_t grad_smem_bytes;         /* shared memory per work item of the gradient kernel's on-chip
                                        form (0: absent; larger than the device allows: global memory) */
    int32_t grad_recomputed;         /* gradient plans: forward contractions recomputed in the
                                        backward pass because one work item's gradient arena would
                                        exceed opts.mem_budget_bytes with every forward value kept */
    double est_bytes_per_amplitude;  /* the planner's ranking of planning trials: per contraction
                                        max(algorithmic bytes, flops / 12), all items */
} qvx_plan_info;

typedef struct qvx_plan qvx_plan;

/* Fills *opts with defaults: n_slices -1, 8 restarts, seed 1, 1 GiB budget, auto engine,
 * auto inner slices, max_rank 30, 1 warp per item, host_merge_rank 8. */
void qvx_plan_opts_default(qvx_plan_opts *opts);

/* The graphical model of Section 3.A with output and input vertices removed.
 * Variable v (canonical id, 0 <= v < n_vars) is the value of qubit var_qubit[v] after its
 * var_ordinal[v]-th non-diagonal single-qubit gate; ids run in order of (qubit, ordinal).
 * Pass NULL arrays to query the counts; otherwise var_qubit/var_ordinal hold n_vars
 * entries and edges holds 2*edges_cap int32 (pairs a < b, sorted). */
qvx_status qvx_graph_export(const qvx_circuit *circuit, int32_t *n_vars, int32_t *var_qubit,
                            int32_t *var_ordinal, int64_t *n_edges, int32_t *edges,
                            int64_t edges_cap);

/* Builds a plan on the host (no device work). order: n_order canonical ids (every
 * variable not sliced, each once) or n_order = 0 for the planner's ordering. slices:
 * n_slices ids, or n_slices = -1 to let the planner choose opts->n_slices of them by the
 * greedy rule of Section 3.B.2. opts may be NULL for defaults. */
qvx_status qvx_plan_create(const qvx_circuit *circuit, const int32_t *order, int32_t n_order,
                           const int32_t *slices, int32_t n_slices, const qvx_plan_opts *opts,
                           qvx_plan **out);

void qvx_plan_destroy(qvx_plan *plan);

qvx_status qvx_plan_get_info(const qvx_plan *plan, qvx_plan_info *info);

/* The plan's elimination order (n_vars - n_sliced ids) and slice list (n_sliced ids).
 * Slice number s assigns bit i of s to slices[i]; the first n_inner entries are the ones
 * kept open inside a work item. Either pointer may be NULL. */
qvx_status qvx_plan_get_order(const qvx_plan *plan, int32_t *order, int32_t *slices);

/* The plan's device image (program, leaves, maps; layout in csrc/device_program.h) as the
 * plan holds it on the host: *data stays valid until qvx_plan_destroy. For inspection and
 * for host-side checks of the program. */
qvx_status qvx_plan_get_image(const qvx_plan *plan, const void **data, size_t *bytes);

/* Workspace bytes for calls of up to `batch` bitstrings. */
qvx_status qvx_workspace_size(const qvx_plan *plan, int64_t batch, size_t *bytes);

/* Copies the plan's device image into the head of the workspace and clears the device
 * status word; synchronises `stream`. Call once per (plan, workspace) before the amplitude
 * calls, and again if the workspace memory was used for anything else in between. */
qvx_status qvx_workspace_init(const qvx_plan *plan, void *workspace_dev, size_t workspace_bytes,
                              void *stream);

/* alpha_b = <x_b|C|0> for b < batch. bitstrings_dev: batch uint64 on the device;
 * amps_dev: 2*batch doubles on the device (2*batch*2^n_open_qubits with open qubits:
 * amplitude j of bitstring b at amps_dev[2*(b*2^n_open + j)]); bitstrings_dev holds batch*W
 * words (W per bitstring, see the conventions). Slice terms are computed in complex64 and
 * added exactly (128-bit fixed point, scale 2^-100), then rounded once to FP64. */
qvx_status qvx_amplitude(qvx_plan *plan, const uint64_t *bitstrings_dev, int64_t batch,
                         double *amps_dev, void *workspace_dev, size_t workspace_bytes,
                         void *stream);

/* qvx_amplitude with the bitstrings and amplitudes in HOST memory; returns once the
 * amplitudes are in amps_host (it synchronises `stream`). Page-locked buffers
 * (cudaHostAlloc/cudaHostRegister, e.g. torch's pin_memory) are read and written by the
 * kernels directly, with no separate copy; pageable buffers are staged through the
 * workspace with cudaMemcpyAsync. Bitstrings with bits at or above n_qubits: QVX_EINVAL. */
qvx_status qvx_amplitude_host(qvx_plan *plan, const uint64_t *bitstrings_host, int64_t batch, double *amps_host,
                              void *workspace_dev, size_t workspace_bytes, void *stream);

/* Sum of the slice terms s in [slice_begin, slice_begin + slice_count) only: the share of
 * one rank when the slices are split over several processes (Section 3.B.2). */
qvx_status qvx_amplitude_slices(qvx_plan *plan, const uint64_t *bitstrings_dev, int64_t batch,
                                int64_t slice_begin, int64_t slice_count, double *amps_dev,
                                void *workspace_dev, size_t workspace_bytes, void *stream);

/* The individual slice terms beta_s (complex64, interleaved) for s in
 * [slice_begin, slice_begin + slice_count): terms_dev holds 2*batch*slice_count floats,
 * bitstring-major. For checking and for callers that sum the terms themselves. */
qvx_status qvx_slice_terms(qvx_plan *plan, const uint64_t *bitstrings_dev, int64_t batch,
                           int64_t slice_begin, int64_t slice_count, float *terms_dev,
                           void *workspace_dev, size_t workspace_bytes, void *stream);

/* The paper has no counterpart to this entry point; it serves callers that cannot
 * allocate device memory: code that runs where the allocator is off limits (inside another
 * library's callback, a real-time loop that must not block on an allocation, a process whose
 * device memory is all reserved up front) and so cannot provide a workspace.
 * alpha_b = <x_b|C|0> for b < batch, like qvx_amplitude, but without a workspace: the
 * library keeps this call's scratch (the plan's device image, a status word and the
 * per-work-item partial sums) in one fixed device array of 4 MiB that every GPU loading the
 * library holds until the process exits. bitstrings_dev and amps_dev are the caller's device
 * buffers as for qvx_amplitude. Fused-engine plans only (QVX_EUNSUPPORTED otherwise); a plan
 * and batch whose scratch exceeds 4 MiB are rejected with QVX_EINVAL. The scratch holds 256
 * bytes of status words, the plan's device image rounded up to 256 bytes, and 32 bytes per
 * (bitstring, open-output value, outer work item). The first call on a device also looks up
 * the array's device address (cudaGetSymbolAddress). All calls share the one array and each
 * call overwrites it: calls that overlap on the GPU (other streams, other threads) race and
 * must be serialised by the caller. The array's status word records a kernel failure
 * (QVX_ETIMEOUT, QVX_ERANGE) and is not cleared by the next call: read it with
 * qvx_noalloc_status; while it is set, amplitudes are written as NaN. */
qvx_status qvx_amplitude_noalloc(qvx_plan *plan, const uint64_t *bitstrings_dev, int64_t batch,
                                 double *amps_dev, void *stream);

/* Companion of qvx_amplitude_noalloc (no paper counterpart): synchronises `stream`, returns
 * the status word of the current device's fixed array (QVX_OK if it is clear or no call has
 * run on the device yet) and clears it. Allocates nothing. */
qvx_status qvx_noalloc_status(void *stream);

/* alpha_b = <x_b|C|0> and its derivatives d alpha_b / d theta_p with respect to the angles
 * of the RXY gates (adjoint of the pairwise contractions: each gate's environment tensor
 * contracted with dU/dtheta; the per-slice terms are added exactly in 128-bit fixed point).
 * The plan must have been created with opts.gradient = 1. thetas_dev: n_thetas doubles on
 * the device that replace the circuit's angles (gate g takes thetas_dev[g.param_index]),
 * or NULL to keep them; n_thetas must then be 0 or the plan's n_params. amps_dev: 2*batch
 * doubles; grad_dev: 2*batch*n_params doubles, complex d alpha_b / d theta_p at
 * grad_dev[2*(b*n_params + p)]. The workspace holds the gradient program's arenas
 * (qvx_workspace_size covers them for gradient plans). */
qvx_status qvx_amplitude_grad(qvx_plan *plan, const uint64_t *bitstrings_dev, int64_t batch,
                              const double *thetas_dev, int32_t n_thetas, double *amps_dev,
                              double *grad_dev, void *workspace_dev, size_t workspace_bytes,
                              void *stream);

/* Self-test of the library's bounded device waits (the paper has no counterpart): runs a
 * one-CTA kernel whose grid-barrier wait and mbarrier wait can never complete, so both give
 * up after `polls` polls (1..2^20) and report QVX_ETIMEOUT in the workspace status word.
 * Returns QVX_ETIMEOUT when both waits reported it (as designed), QVX_OK otherwise; the
 * status word is cleared again. Uses two scratch words of the workspace's status block. */
qvx_status qvx_selftest_wait_timeout(const qvx_plan *plan, void *workspace_dev, size_t workspace_bytes,
                                     uint32_t polls, void *stream);

/* Self-test of the fused kernel's failure path (the paper has no counterpart): runs
 * qvx_amplitude for a fused-engine plan whose program is staged in shared memory, with the
 * first staging wait of every CTA giving up at once, as a wait that ran out would. Each CTA
 * then reports QVX_ETIMEOUT in the workspace status word, waits (bounded) for its staging
 * copies to land, skips its work items and still counts itself, so the last CTA writes the
 * amplitudes as NaN and resets the finished-CTA counter: the next call on the workspace,
 * after qvx_workspace_status has cleared the word, computes normally. Nothing faults or
 * hangs. QVX_EUNSUPPORTED for other plans. */
qvx_status qvx_selftest_fused_timeout(qvx_plan *plan, const uint64_t *bitstrings_dev, int64_t batch, double *amps_dev,
                                      void *workspace_dev, size_t workspace_bytes, void *stream);

/* Synchronises `stream` and returns the device status word kept in the workspace
 * (QVX_OK, QVX_ETIMEOUT or QVX_ERANGE), then clears it. */
qvx_status qvx_workspace_status(const qvx_plan *plan, void *workspace_dev, void *stream);

/* Message for the calling thread's last failed call ("" if none). */
const char *qvx_last_error(void);

/* Kernels of the library, as named in qvx_launch_record.kernel. */
typedef enum {
    QVX_KERNEL_FUSED = 0,       /* fused_program_kernel: whole program per work item, shared memory */
    QVX_KERNEL_PERSISTENT = 1,  /* persistent_program_kernel */
    QVX_KERNEL_STEP = 2,        /* step_kernel: one thread per output entry */
    QVX_KERNEL_STEP_GROUP = 3,  /* step_group_kernel: several small steps of one level */
    QVX_KERNEL_SPLITK = 4,      /* splitk_step_kernel */
    QVX_KERNEL_REGTILE = 5,     /* regtile_step_kernel: register-tiled SIMT contraction */
    QVX_KERNEL_GEMM_TC = 6,     /* gemm_tc_kernel: tcgen05 tensor-core contraction */
    QVX_KERNEL_FINISH = 7,      /* finish_kernel: exact sums of the items' final tensors */
    QVX_KERNEL_SLICE_SUM = 8    /* slice_sum_kernel: exact sum over the slice terms */
} qvx_kernel_id;

/* One kernel launch of a profiled call. */
typedef struct {
    int32_t kernel;        /* qvx_kernel_id */
    int32_t step;          /* program step of a single-step launch, else -1 */
    int64_t items;         /* work items the launch processed (sums: partials added) */
    double flops;          /* algorithmic real flops of the launch (8 per complex MAC) */
    double bytes;          /* algorithmic bytes of the launch: each operand read and each
                              output written once (complex64; 32-byte exact partials) */
    float ms;              /* device time between CUDA events recorded on the call's stream
                              just before and just after the launch */
    int32_t pad;
} qvx_launch_record;

/* qvx_amplitude_slices with a CUDA event recorded on `stream` just before and just after
 * every kernel launch, for measuring each kernel against its roofline. The launches are
 * appended to the plan's launch log; nothing is synchronised. No paper counterpart:
 * instrumentation of this implementation. The events belong to the plan (created on first
 * use on the current device, freed by qvx_plan_destroy); the log holds at most about 2^20
 * launches (QVX_ENOMEM beyond: read it first). */
qvx_status qvx_amplitude_profiled(qvx_plan *plan, const uint64_t *bitstrings_dev, int64_t batch, int64_t slice_begin,
                                  int64_t slice_count, double *amps_dev, void *workspace_dev, size_t workspace_bytes,
                                  void *stream);

/* Waits for the logged launches' events, then records[i] (i < cap) describes logged launch i
 * in issue order (its ms filled in), *n_records is the number of logged launches (which may
 * exceed cap), and the log is emptied. With cap = 0 only *n_records is set and the log stays. */
qvx_status qvx_profile_read(qvx_plan *plan, qvx_launch_record *records, int64_t cap, int64_t *n_records);

/* The name of kernel id `kernel` (a qvx_kernel_id value), or "" if unknown. */
const char *qvx_kernel_name(int32_t kernel);

/* Kernels the calling host thread has launched through the library so far (successful
 * launches only; a count, not device work). Reading it before and after a call gives that
 * call's launches. No paper counterpart: instrumentation of this implementation. */
uint64_t qvx_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* QVX_H */
