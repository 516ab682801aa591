// The C interface of include/qvx.h: plans, workspaces and the amplitude entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <string>

#include "kernels.h"
#include "plan.h"
#include "plan_handle.h"

namespace {

thread_local std::string g_err;

qvx_status fail(qvx_status s, const std::string &msg) {
    g_err = msg;
    return s;
}

qvx_status cuda_fail(cudaError_t e, const char *where) {
    return fail(QVX_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// 64-bit words per bitstring: bit q of a bitstring is bit q % 64 of its word q / 64.
uint32_t words_of(const qvx::Plan &p) { return (uint32_t)((p.model.n_qubits + 63) / 64); }

// Workspace layout: [device image][status word, CTA counter][host staging: bitstrings,
// amplitudes][item partials][stepwise arenas], and for gradient plans [derivative
// partials][gradient arenas]
struct WsLayout {
    size_t image, status, stage_bits, stage_amps, partials, arenas, total;
    int64_t items_in_flight;
    size_t grad_partials = 0, grad_arenas = 0;
    int64_t grad_slots = 0;
};

WsLayout layout_of(const qvx::Plan &p, int64_t batch) {
    WsLayout w{};
    const int64_t n_outer = int64_t(1) << ((int)p.slices.size() - p.n_inner);
    w.image = 0;
    w.status = align256(p.image.size());
    w.stage_bits = w.status + 256;
    const size_t slots = (size_t)std::max<int64_t>(batch, 1) << p.open_qubits.size();   // amplitudes per call
    w.stage_amps = align256(w.stage_bits + (size_t)std::max<int64_t>(batch, 1) * 8 * words_of(p));
    w.partials = align256(w.stage_amps + slots * 16);
    w.arenas = align256(w.partials + slots * (size_t)n_outer * sizeof(qvx::ExactPair));
    w.items_in_flight = 0;
    if (p.engine == QVX_ENGINE_STEPWISE || p.engine == QVX_ENGINE_PERSISTENT) {
        const int64_t arena_bytes = std::max<int64_t>(p.arena_elems, 4) * 8;
        const int64_t total_items = std::max<int64_t>(batch, 1) * n_outer;
        int64_t fit = std::max<int64_t>(1, p.opts.mem_budget_bytes / arena_bytes);
        w.items_in_flight = std::min(total_items, fit);
    }
    w.total = align256(w.arenas + (size_t)w.items_in_flight * (size_t)std::max<int64_t>(p.arena_elems, 4) * 8);
    if (p.opts.gradient) {
        const qvx::DevProgram *h = reinterpret_cast<const qvx::DevProgram *>(p.image.data());
        const int64_t total_items = std::max<int64_t>(batch, 1) * n_outer;
        const int64_t arena_bytes = std::max<int64_t>(p.grad_arena_elems, 4) * 8;
        w.grad_partials = w.total;
        w.grad_arenas = align256(w.grad_partials + (size_t)total_items * h->n_param_leaves * sizeof(qvx::ExactPair));
        w.grad_slots = std::min(total_items, std::max<int64_t>(1, p.opts.mem_budget_bytes / arena_bytes));
        w.total = align256(w.grad_arenas + (size_t)w.grad_slots * (size_t)arena_bytes);
    }
    return w;
}

struct DeviceCaps {
    int sms = 0, device = -1;
};

qvx_status device_caps(DeviceCaps *c) {
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    return QVX_OK;
}

qvx_status check_ws(const qvx_plan *plan, int64_t batch, void *ws, size_t ws_bytes, WsLayout *w) {
    if (!plan) return fail(QVX_EINVAL, "null plan");
    if (batch < 0) return fail(QVX_EINVAL, "negative batch");
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255)) return fail(QVX_EINVAL, "workspace must be 256-byte aligned");
    *w = layout_of(plan->p, batch);
    if (ws_bytes < w->total)
        return fail(QVX_EINVAL, "workspace too small: need " + std::to_string(w->total) + " bytes");
    return QVX_OK;
}

// Per-launch CUDA events of profiled calls (qvx_amplitude_profiled): an event before and
// after every launch on the call's stream, with the launch's kernel, step, work items and
// algorithmic work appended to the plan's launch log; qvx_profile_read waits for the events
// and turns them into durations.
struct Profiler {
    qvx_plan *plan;
    cudaStream_t st;
    cudaError_t err = cudaSuccess;

    cudaEvent_t event(size_t i) {
        while (plan->prof_events.size() <= i) {
            cudaEvent_t ev;
            cudaError_t e = cudaEventCreate(&ev);
            if (e != cudaSuccess) {
                err = e;
                return nullptr;
            }
            plan->prof_events.push_back(ev);
        }
        return plan->prof_events[i];
    }
    void begin() {
        cudaEvent_t ev = event(2 * plan->prof_log.size());
        if (ev && err == cudaSuccess) err = cudaEventRecord(ev, st);
    }
    void end(int kernel, int step, int64_t items, double flops, double bytes) {
        cudaEvent_t ev = event(2 * plan->prof_log.size() + 1);
        if (ev && err == cudaSuccess) err = cudaEventRecord(ev, st);
        qvx_launch_record r{};
        r.kernel = kernel;
        r.step = step;
        r.items = items;
        r.flops = flops;
        r.bytes = bytes;
        plan->prof_log.push_back(r);
    }
};

struct PStepShape {
    int nk;
};
PStepShape shape_of(const qvx::Plan &p, size_t s) {
    const qvx::PStep &st = p.steps[s];
    return PStepShape{(int)(st.k_ab.size() + st.k_a.size() + st.k_b.size())};
}

// Runs the program over outer slices [o_begin, o_begin + o_count) for every bitstring,
// leaving exact item sums in the workspace partials (and slice terms if requested).
// With the fused engine and amps != nullptr the same launch also writes the amplitudes.
qvx_status run_items(qvx_plan *plan, const uint64_t *bits, int64_t batch, int64_t s_begin,
                     int64_t s_end, float *terms, double *amps, void *ws, const WsLayout &w,
                     cudaStream_t st, int64_t *o_count_out, Profiler *prof = nullptr,
                     bool selftest_stage_timeout = false) {
    const qvx::Plan &p = plan->p;
    const int n_inner = p.n_inner;
    const int64_t o_begin = s_begin >> n_inner;
    const int64_t o_end = ((s_end - 1) >> n_inner) + 1;
    qvx::LaunchArgs a{};
    unsigned char *base = static_cast<unsigned char *>(ws);
    a.image = base + w.image;
    a.bitstrings = bits;
    a.words = words_of(p);
    a.batch = batch;
    a.o_begin = o_begin;
    a.o_count = o_end - o_begin;
    a.s_begin = s_begin;
    a.s_end = s_end;
    a.arena_elems = (uint64_t)std::max<int64_t>(p.arena_elems, 4);
    a.n_steps = (uint32_t)p.steps.size();
    a.n_inner = (uint32_t)n_inner;
    a.partials = reinterpret_cast<qvx::ExactPair *>(base + w.partials);
    a.terms = reinterpret_cast<float2 *>(terms);
    a.status = reinterpret_cast<unsigned int *>(base + w.status);
    a.counter = reinterpret_cast<unsigned int *>(base + w.status) + 1;
    a.amps = p.engine == QVX_ENGINE_FUSED ? amps : nullptr;
    a.selftest_stage_timeout = selftest_stage_timeout ? 1u : 0u;
    *o_count_out = a.o_count;
    const int64_t n_items = batch * a.o_count;
    if (n_items == 0) return QVX_OK;
    cudaError_t e;
    if (p.engine == QVX_ENGINE_FUSED) {
        const int wpi = p.warps_per_item;
        const qvx::DevProgram *h = reinterpret_cast<const qvx::DevProgram *>(p.image.data());
        size_t shared = 0, group = 0;
        int max_ipc = 1;
        if (!qvx::fused_shape(h, a.arena_elems, wpi, &a, &shared, &group, &max_ipc))
            return fail(QVX_EUNSUPPORTED, "fused kernel: arena exceeds shared memory");
        const bool staged = a.smem_steps_bytes != 0;
        int dev = -1;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
        if (dev != plan->launch_device) {
            DeviceCaps caps;
            qvx_status s = device_caps(&caps);
            if (s != QVX_OK) return s;
            if ((e = qvx::fused_prepare(shared + (size_t)max_ipc * group)) != cudaSuccess)
                return cuda_fail(e, "fused kernel attributes");
            for (int ipc = 1; ipc <= 8; ipc++)
                plan->ctas_per_sm[ipc] =
                    ipc <= max_ipc ? qvx::fused_blocks_per_sm(32 * wpi * ipc, shared + ipc * group, staged) : 0;
            plan->sms = caps.sms;
            plan->launch_device = dev;
        }
        // spread the items over every SM first, then stack up to 8 warps per CTA
        const int ipc = (int)std::max<int64_t>(1, std::min<int64_t>(max_ipc, (n_items + plan->sms - 1) / plan->sms));
        if (plan->ctas_per_sm[ipc] < 1) return fail(QVX_EUNSUPPORTED, "fused kernel: no CTA fits on an SM");
        const int64_t ctas_needed = (n_items + ipc - 1) / ipc;
        const int grid = (int)std::min<int64_t>(ctas_needed, (int64_t)plan->sms * plan->ctas_per_sm[ipc]);
        if (prof) prof->begin();
        if ((e = qvx::launch_fused(a, wpi, ipc, grid, shared + (size_t)ipc * group, st)) != cudaSuccess)
            return cuda_fail(e, "fused kernel launch");
        if (prof) prof->end(QVX_KERNEL_FUSED, -1, n_items, p.flops_per_item * (double)n_items, p.bytes_per_item * (double)n_items);
        return QVX_OK;
    }
    float2 *arenas = reinterpret_cast<float2 *>(base + w.arenas);
    if (p.engine == QVX_ENGINE_PERSISTENT) {
        int dev = -1;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
        if (dev != plan->persist_device) {
            DeviceCaps caps;
            qvx_status s = device_caps(&caps);
            if (s != QVX_OK) return s;
            const int per_sm = qvx::persistent_blocks_per_sm();
            if (per_sm < 1) return fail(QVX_EUNSUPPORTED, "persistent kernel: no CTA fits on an SM");
            plan->persist_grid = caps.sms * std::min(per_sm, 4);
            plan->persist_device = dev;
        }
        unsigned *bar = reinterpret_cast<unsigned *>(base + w.status) + 2;   // [count, generation]
        for (int64_t ib = 0; ib < n_items; ib += w.items_in_flight) {
            const int64_t n = std::min<int64_t>(w.items_in_flight, n_items - ib);
            if (prof) prof->begin();
            if ((e = qvx::launch_persistent(a, ib, n, arenas, bar, bar + 1, plan->persist_grid, st)) != cudaSuccess)
                return cuda_fail(e, "persistent kernel launch");
            if (prof) prof->end(QVX_KERNEL_PERSISTENT, -1, n, p.flops_per_item * (double)n, p.bytes_per_item * (double)n);
        }
        return QVX_OK;
    }
    auto cost = [&](size_t s, int64_t n, double *fl, double *by) {
        qvx::step_cost(p, s, fl, by);
        *fl *= (double)n;
        *by *= (double)n;
    };
    // one launch of a single step s (its kind chosen as below), timed when profiling
    auto single = [&](int s, int kind, int64_t ib, int64_t n) -> cudaError_t {
        const uint32_t rc = (uint32_t)p.tensors[p.steps[s].c].modes.size();
        if (prof) prof->begin();
        cudaError_t r;
        if (kind == QVX_KERNEL_GEMM_TC) r = qvx::launch_gemm_step(a, p.gemm[s], ib, n, arenas, st);
        else if (kind == QVX_KERNEL_SPLITK) r = qvx::launch_splitk_step(a, (uint32_t)s, ib, n, arenas, rc, st);
        else if (kind == QVX_KERNEL_REGTILE) r = qvx::launch_regtile_step(a, p.regtile[s], ib, n, arenas, st);
        else r = qvx::launch_step(a, (uint32_t)s, ib, n, arenas, rc, st);
        if (prof && r == cudaSuccess) {
            double fl, by;
            cost((size_t)s, n, &fl, &by);
            prof->end(kind, s, n, fl, by);
        }
        return r;
    };
    for (int64_t ib = 0; ib < n_items; ib += w.items_in_flight) {
        const int64_t n = std::min<int64_t>(w.items_in_flight, n_items - ib);
        for (const auto &ph : p.phases) {
            // the phase's small steps (under 2^18 outputs over the items in flight) share one
            // launch; the others get their own. Split-K takes the steps with many summed
            // entries and few outputs (it gives each output 8 warps' share of the sum).
            qvx::StepGroup grp{};
            for (int s = ph.first; s < ph.second; s++) {
                const uint32_t rc = (uint32_t)p.tensors[p.steps[s].c].modes.size();
                const PStepShape sh = shape_of(p, s);
                const uint64_t threads = (uint64_t)n << rc;
                const bool splitk = sh.nk >= 5 && rc <= 12;
                if (!p.gemm.empty() && p.gemm[s].nk > 0) {   // tensor cores
                    if ((e = single(s, QVX_KERNEL_GEMM_TC, ib, n)) != cudaSuccess)
                        return cuda_fail(e, "tensor-core step launch");
                    continue;
                }
                if (threads < (1u << 18) && !splitk && grp.n < (uint32_t)qvx::kMaxGroupSteps) {
                    grp.step[grp.n] = (uint32_t)s;
                    grp.first_block[grp.n + 1] = grp.first_block[grp.n] + (uint32_t)((threads + 255) / 256);
                    grp.n++;
                    continue;
                }
                const int kind = splitk ? QVX_KERNEL_SPLITK
                                        : (p.regtile[s].rm + p.regtile[s].rn > 0 ? QVX_KERNEL_REGTILE : QVX_KERNEL_STEP);
                if ((e = single(s, kind, ib, n)) != cudaSuccess) return cuda_fail(e, "step kernel launch");
            }
            if (grp.n == 1) {
                const int s = (int)grp.step[0];
                const int kind = p.regtile[s].rm + p.regtile[s].rn > 0 ? QVX_KERNEL_REGTILE : QVX_KERNEL_STEP;
                if ((e = single(s, kind, ib, n)) != cudaSuccess) return cuda_fail(e, "step kernel launch");
            } else if (grp.n > 1) {
                if (prof) prof->begin();
                if ((e = qvx::launch_step_group(a, grp, ib, n, arenas, st)) != cudaSuccess)
                    return cuda_fail(e, "step group launch");
                if (prof) {
                    double fl = 0, by = 0;
                    for (uint32_t j = 0; j < grp.n; j++) {
                        double f1, b1;
                        cost(grp.step[j], n, &f1, &b1);
                        fl += f1;
                        by += b1;
                    }
                    prof->end(QVX_KERNEL_STEP_GROUP, -1, n, fl, by);
                }
            }
        }
        if (prof) prof->begin();
        if ((e = qvx::launch_finish_items(a, ib, n, arenas, st)) != cudaSuccess)
            return cuda_fail(e, "finish kernel launch");
        if (prof) {
            const double fin = std::ldexp(8.0, (int)p.tensors[p.final_tensor].modes.size());
            prof->end(QVX_KERNEL_FINISH, -1, n, 0.0,
                      (double)n * (fin + (double)sizeof(qvx::ExactPair) * std::ldexp(1.0, (int)p.open_qubits.size())));
        }
    }
    return QVX_OK;
}

qvx_status check_range(const qvx_plan *plan, int64_t s_begin, int64_t s_count) {
    const int64_t total = int64_t(1) << plan->p.slices.size();
    if (s_begin < 0 || s_count < 0 || s_begin + s_count > total)
        return fail(QVX_EINVAL, "slice range outside [0, 2^n_sliced)");
    return QVX_OK;
}

}  // namespace

extern "C" {

void qvx_plan_opts_default(qvx_plan_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->n_slices = -1;
    o->order_restarts = 8;
    o->order_seed = 1;
    o->mem_budget_bytes = int64_t(1) << 30;
    o->engine = QVX_ENGINE_AUTO;
    o->inner_slices = -1;
    o->max_rank = 30;
    o->warps_per_item = 1;
    o->host_merge_rank = 8;
    o->gradient = 0;
    o->slice_rule = 0;
    o->plan_trials = 1;
}

qvx_status qvx_graph_export(const qvx_circuit *circuit, int32_t *n_vars, int32_t *var_qubit,
                            int32_t *var_ordinal, int64_t *n_edges, int32_t *edges, int64_t edges_cap) {
    qvx::Model m;
    std::string err;
    try {
        if (!qvx::build_model(circuit, &m, &err)) return fail(QVX_EINVAL, err);
    } catch (const std::bad_alloc &) {
        return fail(QVX_ENOMEM, "out of host memory");
    }
    if (n_vars) *n_vars = m.n_vars;
    if (n_edges) *n_edges = (int64_t)m.edges.size();
    if (var_qubit)
        for (int v = 0; v < m.n_vars; v++) var_qubit[v] = m.var_qubit[v];
    if (var_ordinal)
        for (int v = 0; v < m.n_vars; v++) var_ordinal[v] = m.var_ordinal[v];
    if (edges) {
        if (edges_cap < (int64_t)m.edges.size()) return fail(QVX_EINVAL, "edges: capacity too small");
        for (size_t i = 0; i < m.edges.size(); i++) {
            edges[2 * i] = m.edges[i].first;
            edges[2 * i + 1] = m.edges[i].second;
        }
    }
    return QVX_OK;
}

qvx_status qvx_plan_create(const qvx_circuit *circuit, const int32_t *order, int32_t n_order,
                           const int32_t *slices, int32_t n_slices, const qvx_plan_opts *opts,
                           qvx_plan **out) {
    if (!out) return fail(QVX_EINVAL, "null output pointer");
    *out = nullptr;
    qvx_plan_opts o;
    if (opts) o = *opts;
    else qvx_plan_opts_default(&o);
    if (n_order < 0) return fail(QVX_EINVAL, "n_order < 0");
    if (o.order_restarts < 1 || o.max_rank < 1 || o.mem_budget_bytes < 64)
        return fail(QVX_EINVAL, "opts: restarts >= 1, max_rank >= 1, budget >= 64 bytes");
    if (o.slice_rule < 0 || o.slice_rule > 2) return fail(QVX_EINVAL, "opts: slice_rule must be 0, 1 or 2");
    if (o.plan_trials < 1 || o.plan_trials > 65536) return fail(QVX_EINVAL, "opts: plan_trials must be in [1, 65536]");
    if (o.tensor_cores < 0 || o.tensor_cores > 1) return fail(QVX_EINVAL, "opts: tensor_cores must be 0 or 1");
    if (o.host_merge_rank < 0 || o.host_merge_rank > 16)
        return fail(QVX_EINVAL, "opts: host_merge_rank must be in [0, 16]");
    if (o.warps_per_item < 1 || o.warps_per_item > 16 || (o.warps_per_item & (o.warps_per_item - 1)))
        return fail(QVX_EINVAL, "opts: warps_per_item must be 1, 2, 4, 8 or 16");
    qvx_plan *plan = nullptr;
    try {
        plan = new qvx_plan();
        std::string err;
        qvx_status s = qvx::make_plan(circuit, order, n_order, slices, n_slices, o, &plan->p, &err);
        if (s != QVX_OK) {
            delete plan;
            return fail(s, err);
        }
    } catch (const std::bad_alloc &) {
        delete plan;
        return fail(QVX_ENOMEM, "out of host memory");
    }
    *out = plan;
    return QVX_OK;
}

void qvx_plan_destroy(qvx_plan *plan) { delete plan; }

qvx_status qvx_plan_get_info(const qvx_plan *plan, qvx_plan_info *info) {
    if (!plan || !info) return fail(QVX_EINVAL, "null argument");
    const qvx::Plan &p = plan->p;
    std::memset(info, 0, sizeof(*info));
    info->n_qubits = p.model.n_qubits;
    info->n_vars = p.model.n_vars;
    info->n_edges = (int32_t)p.model.edges.size();
    info->n_sliced = (int32_t)p.slices.size();
    info->n_inner = p.n_inner;
    info->n_steps = (int32_t)p.steps.size();
    info->n_leaves = (int32_t)reinterpret_cast<const qvx::DevProgram *>(p.image.data())->n_leaves;
    info->max_rank = p.max_rank;
    info->engine = p.engine;
    info->warps_per_item = p.warps_per_item;
    info->n_items_per_bitstring = int64_t(1) << ((int)p.slices.size() - p.n_inner);
    info->log2_cost = p.log2_cost;
    info->log2_cost_unsliced = p.log2_cost_unsliced;
    info->flops_per_amplitude = p.flops_per_item * (double)info->n_items_per_bitstring;
    info->bytes_per_amplitude = p.bytes_per_item * (double)info->n_items_per_bitstring;
    info->arena_bytes = p.arena_elems * 8;
    info->device_image_bytes = (int64_t)p.image.size();
    info->n_params = p.n_params;
    info->n_grad_steps = (int32_t)p.grad_steps.size();
    info->grad_arena_bytes = p.grad_arena_elems * 8;
    info->grad_flops_per_amplitude = p.grad_flops_per_item * (double)info->n_items_per_bitstring;
    info->n_tiled_steps = 0;
    for (const qvx::RegTileStep &r : p.regtile) info->n_tiled_steps += r.rm + r.rn > 0 ? 1 : 0;
    info->n_phases = (int32_t)p.phases.size();
    info->n_open_qubits = (int32_t)p.open_qubits.size();
    info->n_gemm_steps = 0;
    for (const qvx::GemmStep &g : p.gemm) info->n_gemm_steps += g.nk > 0 ? 1 : 0;
    info->grad_recomputed = p.grad_recomputed;
    info->est_bytes_per_amplitude = qvx::plan_estimate(p);
    info->grad_smem_bytes = p.opts.gradient
        ? (int32_t)qvx::grad_smem_bytes(reinterpret_cast<const qvx::DevProgram *>(p.image.data())) : 0;
    info->grad_bytes_per_amplitude = p.grad_bytes_per_item * (double)info->n_items_per_bitstring;
    return QVX_OK;
}

qvx_status qvx_plan_get_order(const qvx_plan *plan, int32_t *order, int32_t *slices) {
    if (!plan) return fail(QVX_EINVAL, "null plan");
    if (order)
        for (size_t i = 0; i < plan->p.order.size(); i++) order[i] = plan->p.order[i];
    if (slices)
        for (size_t i = 0; i < plan->p.slices.size(); i++) slices[i] = plan->p.slices[i];
    return QVX_OK;
}

qvx_status qvx_plan_get_image(const qvx_plan *plan, const void **data, size_t *bytes) {
    if (!plan || !data || !bytes) return fail(QVX_EINVAL, "null argument");
    *data = plan->p.image.data();
    *bytes = plan->p.image.size();
    return QVX_OK;
}

qvx_status qvx_workspace_size(const qvx_plan *plan, int64_t batch, size_t *bytes) {
    if (!plan || !bytes || batch < 0) return fail(QVX_EINVAL, "bad argument");
    *bytes = layout_of(plan->p, batch).total;
    return QVX_OK;
}

qvx_status qvx_workspace_init(const qvx_plan *plan, void *ws, size_t ws_bytes, void *stream) {
    WsLayout w;
    qvx_status s = check_ws(plan, 0, ws, ws_bytes, &w);
    if (s != QVX_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char *base = static_cast<unsigned char *>(ws);
    cudaError_t e = cudaMemcpyAsync(base + w.image, plan->p.image.data(), plan->p.image.size(),
                                    cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "image upload");
    if ((e = cudaMemsetAsync(base + w.status, 0, 256, st)) != cudaSuccess) return cuda_fail(e, "status clear");
    // the upload reads pageable host memory owned by the plan: finish it before returning
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "image upload sync");
    return QVX_OK;
}

}  // extern "C"

namespace {
qvx_status amplitude_slices_impl(qvx_plan *plan, const uint64_t *bitstrings_dev, int64_t batch, int64_t slice_begin,
                                 int64_t slice_count, double *amps_dev, void *ws, size_t ws_bytes, void *stream,
                                 Profiler *prof) {
    WsLayout w;
    qvx_status s = check_ws(plan, batch, ws, ws_bytes, &w);
    if (s != QVX_OK) return s;
    if ((s = check_range(plan, slice_begin, slice_count)) != QVX_OK) return s;
    if (batch == 0) return QVX_OK;
    if (!bitstrings_dev || !amps_dev) return fail(QVX_EINVAL, "null device buffer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (slice_count == 0) {
        if ((e = cudaMemsetAsync(amps_dev, 0, ((size_t)batch << plan->p.open_qubits.size()) * 16, st)) != cudaSuccess)
            return cuda_fail(e, "memset");
        return QVX_OK;
    }
    int64_t o_count = 0;
    s = run_items(plan, bitstrings_dev, batch, slice_begin, slice_begin + slice_count, nullptr, amps_dev, ws, w,
                  st, &o_count, prof);
    if (s != QVX_OK) return s;
    if (plan->p.engine == QVX_ENGINE_FUSED) return QVX_OK;   // the fused launch wrote the sums
    unsigned char *base = static_cast<unsigned char *>(ws);
    const int64_t slots = batch << plan->p.open_qubits.size();
    if (prof) prof->begin();
    if ((e = qvx::launch_slice_sum(base + w.image, reinterpret_cast<const qvx::ExactPair *>(base + w.partials),
                                   batch << plan->p.open_qubits.size(), o_count,
                                   amps_dev, reinterpret_cast<unsigned *>(base + w.status), st)) != cudaSuccess)
        return cuda_fail(e, "slice sum launch");
    if (prof)
        prof->end(QVX_KERNEL_SLICE_SUM, -1, slots * o_count, 0.0,
                  (double)slots * ((double)o_count * (double)sizeof(qvx::ExactPair) + 16.0));
    return QVX_OK;
}
}  // namespace

extern "C" {

qvx_status qvx_amplitude_slices(qvx_plan *plan, const uint64_t *bitstrings_dev, int64_t batch,
                                int64_t slice_begin, int64_t slice_count, double *amps_dev,
                                void *ws, size_t ws_bytes, void *stream) {
    return amplitude_slices_impl(plan, bitstrings_dev, batch, slice_begin, slice_count, amps_dev, ws, ws_bytes, stream,
                                 nullptr);
}

qvx_status qvx_amplitude_profiled(qvx_plan *plan, const uint64_t *bitstrings_dev, int64_t batch, int64_t slice_begin,
                                  int64_t slice_count, double *amps_dev, void *ws, size_t ws_bytes, void *stream) {
    if (!plan) return fail(QVX_EINVAL, "null plan");
    if (plan->prof_log.size() > (size_t(1) << 20)) return fail(QVX_ENOMEM, "launch log full: read it first");
    Profiler prof{plan, static_cast<cudaStream_t>(stream)};
    qvx_status s = amplitude_slices_impl(plan, bitstrings_dev, batch, slice_begin, slice_count, amps_dev, ws, ws_bytes,
                                         stream, &prof);
    if (s != QVX_OK) return s;
    if (prof.err != cudaSuccess) return cuda_fail(prof.err, "profiling event");
    return QVX_OK;
}

qvx_status qvx_profile_read(qvx_plan *plan, qvx_launch_record *records, int64_t cap, int64_t *n_records) {
    if (!plan) return fail(QVX_EINVAL, "null plan");
    if (cap < 0 || (cap > 0 && !records)) return fail(QVX_EINVAL, "records: null with a positive capacity");
    if (cap == 0) {   // the count only; the log stays
        if (n_records) *n_records = (int64_t)plan->prof_log.size();
        return QVX_OK;
    }
    std::vector<qvx_launch_record> log;
    log.swap(plan->prof_log);
    cudaError_t e;
    for (size_t i = 0; i < log.size(); i++) {
        if ((e = cudaEventSynchronize(plan->prof_events[2 * i + 1])) != cudaSuccess)
            return cuda_fail(e, "cudaEventSynchronize");
        float ms = 0.f;
        if ((e = cudaEventElapsedTime(&ms, plan->prof_events[2 * i], plan->prof_events[2 * i + 1])) != cudaSuccess)
            return cuda_fail(e, "cudaEventElapsedTime");
        log[i].ms = ms;
        if ((int64_t)i < cap) records[i] = log[i];
    }
    if (n_records) *n_records = (int64_t)log.size();
    return QVX_OK;
}

const char *qvx_kernel_name(int32_t kernel) {
    switch (kernel) {
        case QVX_KERNEL_FUSED: return "fused_program_kernel";
        case QVX_KERNEL_PERSISTENT: return "persistent_program_kernel";
        case QVX_KERNEL_STEP: return "step_kernel";
        case QVX_KERNEL_STEP_GROUP: return "step_group_kernel";
        case QVX_KERNEL_SPLITK: return "splitk_step_kernel";
        case QVX_KERNEL_REGTILE: return "regtile_step_kernel";
        case QVX_KERNEL_GEMM_TC: return "gemm_tc_kernel";
        case QVX_KERNEL_FINISH: return "finish_kernel";
        case QVX_KERNEL_SLICE_SUM: return "slice_sum_kernel";
        default: return "";
    }
}

namespace {
// Device-accessible address of a page-locked host buffer, or nullptr for pageable memory.
const void *pinned_device_ptr(const void *host) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, host) != cudaSuccess) {
        cudaGetLastError();   // pageable memory may report an error on older drivers: clear it
        return nullptr;
    }
    if (at.type != cudaMemoryTypeHost || !at.devicePointer) return nullptr;
    return at.devicePointer;
}
}  // namespace

qvx_status qvx_amplitude_host(qvx_plan *plan, const uint64_t *bitstrings_host, int64_t batch, double *amps_host,
                              void *ws, size_t ws_bytes, void *stream) {
    WsLayout w;
    qvx_status s = check_ws(plan, batch, ws, ws_bytes, &w);
    if (s != QVX_OK) return s;
    if (batch == 0) return QVX_OK;
    if (!bitstrings_host || !amps_host) return fail(QVX_EINVAL, "null host buffer");
    const int n = plan->p.model.n_qubits;
    const uint32_t W = words_of(plan->p);
    for (int64_t b = 0; b < batch; b++)
        for (uint32_t wd = 0; wd < W; wd++) {
            const int valid = n - 64 * (int)wd;   // bits of this word that are qubits
            if (valid < 64 && (bitstrings_host[b * W + wd] >> valid) != 0)
                return fail(QVX_EINVAL, "bitstring has bits at or above n_qubits");
        }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char *base = static_cast<unsigned char *>(ws);
    cudaError_t e;
    const uint64_t *bits_dev = static_cast<const uint64_t *>(pinned_device_ptr(bitstrings_host));
    if (!bits_dev) {
        bits_dev = reinterpret_cast<const uint64_t *>(base + w.stage_bits);
        if ((e = cudaMemcpyAsync(base + w.stage_bits, bitstrings_host, (size_t)batch * 8 * W, cudaMemcpyHostToDevice, st)) !=
            cudaSuccess)
            return cuda_fail(e, "bitstring upload");
    }
    double *amps_dev = static_cast<double *>(const_cast<void *>(pinned_device_ptr(amps_host)));
    const bool stage_out = amps_dev == nullptr;
    if (stage_out) amps_dev = reinterpret_cast<double *>(base + w.stage_amps);
    s = qvx_amplitude(plan, bits_dev, batch, amps_dev, ws, ws_bytes, stream);
    if (s != QVX_OK) return s;
    if (stage_out && (e = cudaMemcpyAsync(amps_host, amps_dev, ((size_t)batch << plan->p.open_qubits.size()) * 16,
                                          cudaMemcpyDeviceToHost, st)) !=
                         cudaSuccess)
        return cuda_fail(e, "amplitude download");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "stream synchronize");
    return QVX_OK;
}

qvx_status qvx_amplitude(qvx_plan *plan, const uint64_t *bitstrings_dev, int64_t batch, double *amps_dev,
                         void *ws, size_t ws_bytes, void *stream) {
    if (!plan) return fail(QVX_EINVAL, "null plan");
    return qvx_amplitude_slices(plan, bitstrings_dev, batch, 0, int64_t(1) << plan->p.slices.size(),
                                amps_dev, ws, ws_bytes, stream);
}

qvx_status qvx_slice_terms(qvx_plan *plan, const uint64_t *bitstrings_dev, int64_t batch,
                           int64_t slice_begin, int64_t slice_count, float *terms_dev, void *ws,
                           size_t ws_bytes, void *stream) {
    WsLayout w;
    qvx_status s = check_ws(plan, batch, ws, ws_bytes, &w);
    if (s != QVX_OK) return s;
    if ((s = check_range(plan, slice_begin, slice_count)) != QVX_OK) return s;
    if (batch == 0 || slice_count == 0) return QVX_OK;
    if (!bitstrings_dev || !terms_dev) return fail(QVX_EINVAL, "null device buffer");
    int64_t o_count = 0;
    return run_items(plan, bitstrings_dev, batch, slice_begin, slice_begin + slice_count, terms_dev, nullptr,
                     ws, w, static_cast<cudaStream_t>(stream), &o_count);
}

qvx_status qvx_amplitude_grad(qvx_plan *plan, const uint64_t *bitstrings_dev, int64_t batch, const double *thetas_dev,
                              int32_t n_thetas, double *amps_dev, double *grad_dev, void *ws, size_t ws_bytes,
                              void *stream) {
    WsLayout w;
    qvx_status s = check_ws(plan, batch, ws, ws_bytes, &w);
    if (s != QVX_OK) return s;
    const qvx::Plan &p = plan->p;
    if (!p.opts.gradient) return fail(QVX_EUNSUPPORTED, "plan was created without opts.gradient");
    if (thetas_dev ? n_thetas != p.n_params : n_thetas != 0)
        return fail(QVX_EINVAL, "n_thetas must equal the plan's n_params (" + std::to_string(p.n_params) + ")");
    if (batch == 0) return QVX_OK;
    if (!bitstrings_dev || !amps_dev || (p.n_params > 0 && !grad_dev)) return fail(QVX_EINVAL, "null device buffer");
    const qvx::DevProgram *h = reinterpret_cast<const qvx::DevProgram *>(p.image.data());
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char *base = static_cast<unsigned char *>(ws);
    cudaError_t e;
    if ((e = qvx::launch_set_params(base + w.image, h->n_param_leaves, thetas_dev, st)) != cudaSuccess)
        return cuda_fail(e, "parameter kernel launch");
    const int64_t n_outer = int64_t(1) << ((int)p.slices.size() - p.n_inner);
    qvx::GradArgs g{};
    g.image = base + w.image;
    g.bitstrings = bitstrings_dev;
    g.words = words_of(p);
    g.batch = batch;
    g.o_count = n_outer;
    g.arenas = reinterpret_cast<float2 *>(base + w.grad_arenas);
    g.arena_elems = (uint64_t)std::max<int64_t>(p.grad_arena_elems, 4);
    g.slots = w.grad_slots;
    g.partials = reinterpret_cast<qvx::ExactPair *>(base + w.partials);
    g.gpart = reinterpret_cast<qvx::ExactPair *>(base + w.grad_partials);
    g.status = reinterpret_cast<unsigned int *>(base + w.status);
    const size_t gsm = qvx::grad_smem_bytes(h);
    qvx::GradArgs staged_args = g;
    const size_t gsm_staged = gsm ? gsm + qvx::grad_stage_bytes(h, &staged_args) : 0;
    if (gsm) {
        int dev = -1;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
        if (dev != plan->grad_device) {
            DeviceCaps caps;
            qvx_status s = device_caps(&caps);
            if (s != QVX_OK) return s;
            plan->grad_sms = caps.sms;
            plan->grad_ctas_per_sm = qvx::grad_smem_blocks_per_sm(gsm, false);
            plan->grad_staged_ctas_per_sm = qvx::grad_smem_blocks_per_sm(gsm_staged, true);
            plan->grad_device = dev;
        }
    }
    // the staged form (leaf data and tables on chip too) when every work item still gets its
    // own CTA at once; it holds more shared memory, so fewer CTAs fit on an SM
    const int64_t n_items = batch * n_outer;
    if (gsm && plan->grad_staged_ctas_per_sm > 0 && n_items <= (int64_t)plan->grad_sms * plan->grad_staged_ctas_per_sm) {
        if ((e = qvx::launch_grad_smem(staged_args, (int)n_items, gsm_staged, st)) != cudaSuccess)
            return cuda_fail(e, "gradient kernel launch");
    } else if (gsm && plan->grad_ctas_per_sm > 0) {
        const int grid = (int)std::min<int64_t>(batch * n_outer, (int64_t)plan->grad_sms * plan->grad_ctas_per_sm);
        if ((e = qvx::launch_grad_smem(g, grid, gsm, st)) != cudaSuccess) return cuda_fail(e, "gradient kernel launch");
    } else {
        const int grid = (int)std::min<int64_t>(batch * n_outer, w.grad_slots);
        if ((e = qvx::launch_grad_program(g, grid, st)) != cudaSuccess) return cuda_fail(e, "gradient kernel launch");
    }
    if ((e = qvx::launch_slice_sum(base + w.image, g.partials, batch, n_outer, amps_dev, g.status, st)) != cudaSuccess)
        return cuda_fail(e, "slice sum launch");
    if ((e = qvx::launch_grad_sum(base + w.image, g.gpart, batch, n_outer, h->n_param_leaves, (uint32_t)p.n_params,
                                  grad_dev, g.status, st)) != cudaSuccess)
        return cuda_fail(e, "gradient sum launch");
    return QVX_OK;
}

qvx_status qvx_selftest_wait_timeout(const qvx_plan *plan, void *ws, size_t ws_bytes, uint32_t polls, void *stream) {
    WsLayout w;
    qvx_status s = check_ws(plan, 0, ws, ws_bytes, &w);
    if (s != QVX_OK) return s;
    if (polls < 1 || polls > (1u << 20)) return fail(QVX_EINVAL, "polls must be in [1, 2^20]");
    unsigned char *base = static_cast<unsigned char *>(ws);
    unsigned *status = reinterpret_cast<unsigned *>(base + w.status);
    unsigned *words = status + 4;   // [count, generation] of the test barrier
    unsigned *out = status + 6;     // which waits gave up
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if ((e = cudaMemsetAsync(status + 4, 0, 4 * sizeof(unsigned), st)) != cudaSuccess) return cuda_fail(e, "memset");
    if ((e = qvx::launch_wait_selftest(words, status, polls, out, st)) != cudaSuccess)
        return cuda_fail(e, "self-test launch");
    unsigned h[2] = {0, 0}, word = 0;
    if ((e = cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return cuda_fail(e, "read");
    if ((e = cudaMemcpyAsync(&word, status, sizeof(word), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(e, "read");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "stream synchronize");
    if ((e = cudaMemset(status, 0, 8 * sizeof(unsigned))) != cudaSuccess) return cuda_fail(e, "status clear");
    if (h[0] && h[1] && word == (unsigned)QVX_ETIMEOUT) return fail(QVX_ETIMEOUT, "both bounded waits gave up as designed");
    return QVX_OK;
}

qvx_status qvx_selftest_fused_timeout(qvx_plan *plan, const uint64_t *bitstrings_dev, int64_t batch, double *amps_dev,
                                      void *ws, size_t ws_bytes, void *stream) {
    WsLayout w;
    qvx_status s = check_ws(plan, batch, ws, ws_bytes, &w);
    if (s != QVX_OK) return s;
    if (batch <= 0 || !bitstrings_dev || !amps_dev) return fail(QVX_EINVAL, "need a batch and device buffers");
    const qvx::Plan &p = plan->p;
    if (p.engine != QVX_ENGINE_FUSED) return fail(QVX_EUNSUPPORTED, "the self-test runs fused-engine plans");
    {
        qvx::LaunchArgs probe{};
        size_t shared = 0, group = 0;
        int max_ipc = 1;
        if (!qvx::fused_shape(reinterpret_cast<const qvx::DevProgram *>(p.image.data()),
                              (uint64_t)std::max<int64_t>(p.arena_elems, 4), p.warps_per_item, &probe, &shared, &group,
                              &max_ipc) ||
            probe.smem_steps_bytes == 0)
            return fail(QVX_EUNSUPPORTED, "the plan's program is not staged in shared memory");
    }
    int64_t o_count = 0;
    return run_items(plan, bitstrings_dev, batch, 0, int64_t(1) << p.slices.size(), nullptr, amps_dev, ws, w,
                     static_cast<cudaStream_t>(stream), &o_count, nullptr, true);
}

qvx_status qvx_workspace_status(const qvx_plan *plan, void *ws, void *stream) {
    WsLayout w;
    qvx_status s = check_ws(plan, 0, ws, (size_t)-1, &w);
    if (s != QVX_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned int word = 0;
    unsigned char *base = static_cast<unsigned char *>(ws);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    if ((e = cudaMemcpy(&word, base + w.status, sizeof(word), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "status read");
    if (word != 0) {
        if ((e = cudaMemset(base + w.status, 0, sizeof(word))) != cudaSuccess) return cuda_fail(e, "status clear");
        return fail((qvx_status)word, "device status word set by a kernel");
    }
    return QVX_OK;
}

const char *qvx_last_error(void) { return g_err.c_str(); }

uint64_t qvx_kernel_launches(void) { return qvx::launches_issued(); }

}  // extern "C"

namespace qvx {
// Sets the calling thread's qvx_last_error message (for entry points in other files).
void set_last_error(const std::string &msg) { g_err = msg; }
}  // namespace qvx
