// The opaque qvx_plan handle of include/qvx.h.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "plan.h"

struct qvx_plan {
    qvx::Plan p;
    // fused-engine launch shape, cached for the device it was computed on
    int launch_device = -1;
    int sms = 0;
    int ctas_per_sm[9] = {0};   // by work items per CTA
    // persistent-engine grid, cached for the device it was computed on
    int persist_device = -1, persist_grid = 0;
    // shared-memory gradient kernel: CTAs per SM (0: the global-memory kernel runs), CTAs per
    // SM of its staged form (leaf data and tables in shared memory too; 0: does not fit), SMs
    int grad_device = -1, grad_ctas_per_sm = 0, grad_staged_ctas_per_sm = 0, grad_sms = 0;
    // launch log of qvx_amplitude_profiled and its timing events (two per logged launch,
    // created on first use and reused after qvx_profile_read empties the log)
    std::vector<qvx_launch_record> prof_log;
    std::vector<cudaEvent_t> prof_events;

    ~qvx_plan() {
        for (cudaEvent_t e : prof_events) cudaEventDestroy(e);
    }
};
