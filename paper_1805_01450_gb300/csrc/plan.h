// Host-side plan: graphical model, elimination order, slices and the pairwise program.
#pragma once
#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/qvx.h"
#include "device_program.h"

namespace qvx {

using cplx = std::complex<double>;

// A tensor over binary variables: bit j of an entry's index is the value of modes[j].
struct HostTensor {
    std::vector<int> modes;
    std::vector<cplx> data;
    // a parametrised gate kept as its own tensor (gradient plans): entry e is element
    // code[e] of its 2x2 matrix (bit 1 row, bit 0 column)
    int param = -1;
    double theta = 0, phi = 0;
    std::vector<uint8_t> code;
};

// Variable ids inside a plan: [0, n_vars) are the summed variables (canonical ids);
// n_vars + q is the output variable of qubit q, fixed to x_q per bitstring.
struct Model {
    int n_qubits = 0, n_vars = 0;
    std::vector<int> var_qubit, var_ordinal;
    uint64_t zero_mask[2] = {0, 0};   // qubits with no non-diagonal gate (output equals input 0):
                                      // bit q of word q / 64
    std::vector<int> cz_count;     // per summed variable: CZ gates acting on it
    cplx scalar = 1.0;
    std::vector<HostTensor> tensors;
    std::vector<std::pair<int, int>> edges;   // a < b, sorted, summed variables only
};

// One pairwise contraction of the program.
struct PStep {
    int a = -1, b = -1, c = -1;                 // tensor ids; b = -1 for a one-operand sum
    std::vector<int> k_ab, k_a, k_b;            // summed modes
};

// A tensor of the program: a restricted leaf or a step's output.
struct PTensor {
    std::vector<int> modes;                     // layout, set from the consumer
    int leaf = -1;                              // index in Plan::leaves, or -1
    int producer = -1, consumer = -1;           // step ids (-1: leaf / final)
    int64_t offset = 0;                         // arena offset (complex64 entries)
};

struct Plan {
    qvx_plan_opts opts{};
    Model model;
    std::vector<int> order;                     // elimination order (non-sliced ids)
    std::vector<int> slices;                    // inner slices first, then outer
    std::vector<int> open_qubits;               // outputs kept open (amplitude batches)
    int n_inner = 0;
    double log2_cost = 0, log2_cost_unsliced = 0;
    int width = 0;
    // program
    std::vector<HostTensor> leaves;             // stored leaves (may hold fixed modes)
    std::vector<PTensor> tensors;
    std::vector<PStep> steps;
    std::vector<std::pair<int, int>> phases;    // [first, last) step ranges of independent steps
    int final_tensor = -1;
    int64_t arena_elems = 0;
    int max_rank = 0;
    double flops_per_item = 0, bytes_per_item = 0;
    cplx prog_scalar = 1.0;                     // model scalar times the program's own factors
    int engine = QVX_ENGINE_FUSED;
    int warps_per_item = 1;
    std::vector<unsigned char> image;          // device image (DevProgram first)
    std::vector<RegTileStep> regtile;          // per step, global-arena engines: register-tiled form (rm + rn > 0)
    std::vector<GemmStep> gemm;                // per step, stepwise engine with tensor cores: GEMM form (nk > 0)
    // gradient program
    int n_params = 0;
    std::vector<GenStep> grad_steps;
    int64_t grad_arena_elems = 0;
    int64_t grad_final_off = 0, grad_gslot_off = 0;
    std::vector<int> grad_param_leaves;        // leaf indices of the parametrised leaves
    double grad_flops_per_item = 0, grad_bytes_per_item = 0;
    std::vector<uint32_t> grad_phase_first;    // phases of independent gradient steps (+ end)
    std::vector<uint32_t> grad_elem_off;       // per gradient step: first entry inside its phase
    int grad_recomputed = 0;                   // forward steps recomputed in the backward pass
};

// planner.cpp
bool build_model(const qvx_circuit *c, Model *m, std::string *err, bool keep_params = false);
qvx_status make_plan(const qvx_circuit *c, const int32_t *order, int32_t n_order,
                     const int32_t *slices, int32_t n_slices, const qvx_plan_opts &opts,
                     Plan *p, std::string *err);
double plan_estimate(const Plan &p);   // bandwidth-weighted contraction estimate, all items
// Algorithmic flops (8 per complex MAC) and bytes (every operand read and the output
// written once, complex64) of step s for one work item.
void step_cost(const Plan &p, size_t s, double *flops, double *bytes);

}  // namespace qvx
