// qvx_amplitude_noalloc: the amplitude call for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc or hand us a workspace: code that runs where the
// allocator is off limits (inside another library's callback, a real-time loop that must
// not block on the allocator, or a process whose memory is fully reserved up front). This
// entry point keeps its scratch memory — the plan's device image, the status word, the
// finished-CTA counter and the per-work-item partial sums — in one fixed array of
// kNoAllocScratchBytes bytes that lives in the library's own device globals. Every GPU
// that loads the library holds that array until the process exits. Nothing here calls
// cudaMalloc, cudaFree or any allocating routine.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "device_program.h"
#include "kernels.h"
#include "plan_handle.h"

namespace qvx {
void set_last_error(const std::string &msg);
}

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(4) << 20;   // 4 MiB per device
constexpr int kMaxDevices = 64;
constexpr size_t kStatusBytes = 256;                       // [status word, CTA counter], padded

// The scratch array. In host code `g_noalloc_scratch` names a host-side stand-in, not the
// device memory: its device address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mutex;
void *g_scratch_ptr[kMaxDevices] = {nullptr};
int g_sms[kMaxDevices] = {0};

qvx_status fail(qvx_status s, const std::string &msg) {
    qvx::set_last_error(msg);
    return s;
}

qvx_status cuda_fail(cudaError_t e, const char *where) {
    return fail(QVX_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Once per device, with that device current: the device address of the scratch array.
qvx_status scratch_for_device(int dev, void **ptr) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (dev < 0 || dev >= kMaxDevices) return fail(QVX_EUNSUPPORTED, "device index above 63");
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
        if (reinterpret_cast<uintptr_t>(p) & 255) return fail(QVX_ECUDA, "no-allocation scratch is not 256-byte aligned");
        int sms = 0;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return cuda_fail(e, "cudaDeviceGetAttribute");
        g_sms[dev] = sms;
        g_scratch_ptr[dev] = p;
    }
    *ptr = g_scratch_ptr[dev];
    return QVX_OK;
}

size_t r256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" qvx_status qvx_amplitude_noalloc(qvx_plan *plan, const uint64_t *bitstrings_dev, int64_t batch,
                                            double *amps_dev, void *stream) {
    if (!plan) return fail(QVX_EINVAL, "null plan");
    if (batch < 0) return fail(QVX_EINVAL, "negative batch");
    if (batch == 0) return QVX_OK;
    if (!bitstrings_dev || !amps_dev) return fail(QVX_EINVAL, "null device buffer");
    const qvx::Plan &p = plan->p;
    if (p.engine != QVX_ENGINE_FUSED)
        return fail(QVX_EUNSUPPORTED, "the no-allocation entry point runs fused-engine plans only");
    const qvx::DevProgram *h = reinterpret_cast<const qvx::DevProgram *>(p.image.data());
    const int64_t n_outer = int64_t(1) << ((int)p.slices.size() - p.n_inner);
    // scratch layout: [status word, CTA counter][plan image][partials]; the status word sits
    // at a fixed offset so that qvx_noalloc_status can find it without a plan
    const size_t image_off = kStatusBytes;
    const size_t partials_off = image_off + r256(p.image.size());
    const size_t need = partials_off + ((size_t)batch << p.open_qubits.size()) * (size_t)n_outer * sizeof(qvx::ExactPair);
    if (need > kNoAllocScratchBytes)
        return fail(QVX_EINVAL, "no-allocation scratch too small: this plan and batch need " + std::to_string(need) +
                                    " bytes, the fixed array holds " + std::to_string(kNoAllocScratchBytes));
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    void *scratch = nullptr;
    qvx_status s = scratch_for_device(dev, &scratch);
    if (s != QVX_OK) return s;
    unsigned char *base = static_cast<unsigned char *>(scratch);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the array keeps the previous call's contents: load this plan's image and zero the
    // finished-CTA counter before the launch. The status word is left as it is: a failure of
    // an earlier call stays visible to qvx_noalloc_status until it is read (and the amplitudes
    // of every call made while it is set are written as NaN).
    if ((e = cudaMemcpyAsync(base + image_off, p.image.data(), p.image.size(), cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
        return cuda_fail(e, "image copy into the no-allocation scratch");
    if ((e = cudaMemsetAsync(base + sizeof(unsigned), 0, sizeof(unsigned), st)) != cudaSuccess)
        return cuda_fail(e, "scratch clear");

    qvx::LaunchArgs a{};
    a.image = base + image_off;
    a.bitstrings = bitstrings_dev;
    a.words = (uint32_t)((p.model.n_qubits + 63) / 64);
    a.batch = batch;
    a.o_begin = 0;
    a.o_count = n_outer;
    a.s_begin = 0;
    a.s_end = int64_t(1) << p.slices.size();
    a.arena_elems = (uint64_t)std::max<int64_t>(p.arena_elems, 4);
    a.n_steps = (uint32_t)p.steps.size();
    a.n_inner = (uint32_t)p.n_inner;
    a.partials = reinterpret_cast<qvx::ExactPair *>(base + partials_off);
    a.terms = nullptr;
    a.status = reinterpret_cast<unsigned int *>(base);
    a.counter = a.status + 1;
    a.amps = amps_dev;
    // shared-memory layout and grid, chosen as for the workspace entry points
    const int wpi = p.warps_per_item;
    size_t shared = 0, group = 0;
    int max_ipc = 1;
    if (!qvx::fused_shape(h, a.arena_elems, wpi, &a, &shared, &group, &max_ipc))
        return fail(QVX_EUNSUPPORTED, "fused kernel: arena exceeds shared memory");
    const int64_t n_items = batch * n_outer;
    const int ipc = (int)std::max<int64_t>(1, std::min<int64_t>(max_ipc, (n_items + g_sms[dev] - 1) / g_sms[dev]));
    if ((e = qvx::fused_prepare(shared + (size_t)max_ipc * group)) != cudaSuccess)
        return cuda_fail(e, "fused kernel attributes");
    const int per_sm = qvx::fused_blocks_per_sm(32 * wpi * ipc, shared + ipc * group, a.smem_steps_bytes != 0);
    if (per_sm < 1) return fail(QVX_EUNSUPPORTED, "fused kernel: no CTA fits on an SM");
    const int64_t ctas_needed = (n_items + ipc - 1) / ipc;
    const int grid = (int)std::min<int64_t>(ctas_needed, (int64_t)g_sms[dev] * per_sm);
    if ((e = qvx::launch_fused(a, wpi, ipc, grid, shared + (size_t)ipc * group, st)) != cudaSuccess)
        return cuda_fail(e, "fused kernel launch");
    return QVX_OK;
}

extern "C" qvx_status qvx_noalloc_status(void *stream) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (dev >= 0 && dev < kMaxDevices) scratch = g_scratch_ptr[dev];
    }
    if (!scratch) return QVX_OK;   // no call has run on this device
    if ((e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream))) != cudaSuccess)
        return cuda_fail(e, "stream synchronize");
    unsigned word = 0;
    if ((e = cudaMemcpy(&word, scratch, sizeof(word), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "status read");
    if (word == 0) return QVX_OK;
    if ((e = cudaMemset(scratch, 0, sizeof(word))) != cudaSuccess) return cuda_fail(e, "status clear");
    return fail((qvx_status)word, "device status word of the no-allocation scratch set by a kernel");
}
