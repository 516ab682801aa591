#!/usr/bin/env python
"""Throughput of single amplitudes <x|C|0> by sliced variable elimination on one GB300.

Default workload: the 6 x 6 random grid circuit of depth 25 (Section 4 rules, circuit seed
2001), one seeded bitstring (seed 2002) per step, 12 sliced variables (4096 slice terms)
chosen greedily (Section 3.B.2), slice terms in complex64 and their sum in FP64. A step is
one amplitude: every slice term, every pairwise contraction and the compensated sum.

Prints one JSON line. Timing: CUDA events on the launching stream around each step, W
warm-up steps first, L2 flushed (a 256 MiB write) before every timed step, max over ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl qvx|reference]
  torchrun --nproc-per-node N bench.py --gpus N ...   (each rank: its own bitstrings)
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import circuitgen as cg  # noqa: E402

WORKLOADS = {
    # name: (kind, rows, cols, depth, circuit seed, bitstring seed, sliced variables, bitstrings per step)
    "grid6x6d25-k12": ("grid", 6, 6, 25, 2001, 2002, 12, 1),
    "grid4x4d10": ("grid", 4, 4, 10, 1001, 1002, 0, 1),
    "grid7x7d30-b1024": ("grid", 7, 7, 30, 3001, 3002, 4, 1024),
    "rot5x5d20-grad": ("rotation", 5, 5, 20, 4001, 4002, 8, 1),
    "grid8x8d40": ("grid", 8, 8, 40, 5001, 5002, 10, 1),
}
# workloads whose plan variant the autotuner also picks the slice count and engine for,
# and the arena memory the global-arena engines may use there (MiB)
TUNE = {"grid6x6d25-k12": dict(trial_counts=(1, 16, 256)),
        "grid7x7d30-b1024": dict(slice_counts=(0, 2, 4, 6, 8), engines=("stepwise",), budget_s=90.0),
        "grid8x8d40": dict(slice_counts=(10, 12), engines=("stepwise", "stepwise-tc"), inner=(4,), trial_counts=(1, 16, 256),
                           budget_s=120.0)}
MEM_BUDGET_MB = {"grid7x7d30-b1024": 32768, "grid8x8d40": 65536}
# independent planning trials (ordering + slice choice from distinct seeds, the best by the
# planner's bandwidth-weighted estimate kept); planning is outside the timed region
PLAN_TRIALS = {"grid6x6d25-k12": 64, "grid7x7d30-b1024": 64, "grid8x8d40": 64}
DEFAULT_WORKLOAD = "grid6x6d25-k12"
METRIC = "amplitudes/s and complex TFLOP/s (% of GB300 peak) at |Δα|≤1e-5·2^-N/2 vs FP64"
L2_FLUSH_BYTES = 256 << 20
# dram__bytes_read.sum + dram__bytes_write.sum per launch of the dominant kernel (fused
# program kernel; gradient kernel for the gradient workload), from one ncu capture of the
# workload with the current kernels (profiles/ holds the summaries). Keyed by the plan it was
# taken on (its device image size): another plan of the workload reports no traffic.
NCU_TRAFFIC = {("grid6x6d25-k12", 1, 92416): 147968.0, ("rot5x5d20-grad", 1, 1793024): 509184.0}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["qvx", "reference"], default="qvx")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--batch", type=int, default=None, help="bitstrings per step (workload default)")
    ap.add_argument("--inner-slices", type=int, default=None, help="fix the plan variant instead of autotuning")
    ap.add_argument("--mem-budget-mb", type=int, default=None,
                    help="arena memory of the global-arena engines (work items in flight; workload default)")
    ap.add_argument("--warps-per-item", type=int, default=None)
    ap.add_argument("--host-merge-rank", type=int, default=8, help="fixed plan variant: leaf products contracted at plan time")
    ap.add_argument("--tensor-cores", action="store_true",
                    help="stepwise engine: dense contractions as bf16 hi/lo GEMMs on the tensor cores")
    ap.add_argument("--engine", default="auto")
    ap.add_argument("--sliced", type=int, default=None, help="override the workload's sliced-variable count")
    ap.add_argument("--plan-trials", type=int, default=None, help="planning trials (workload default)")
    ap.add_argument("--circuit-seed", type=int, default=None, help="override the workload's circuit seed")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="CPU-baseline sample budget")
    return ap.parse_args()


def workload(name, batch, rank, circuit_seed=None):
    kind, r, c, d, cseed, bseed, k, b0 = WORKLOADS[name]
    batch = b0 if batch is None else batch
    cseed = cseed if circuit_seed is None else circuit_seed
    circ = cg.grid_circuit(r, c, d, cseed) if kind == "grid" else cg.rotation_circuit(r, c, d, cseed)
    bits = cg.random_bitstrings(r * c, batch * (rank + 1), bseed)[batch * rank:]
    return circ, bits, k


def is_grad(name):
    return name.endswith("-grad")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            out, _ = self.proc.communicate(timeout=10)
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        if not self.lines:
            return None
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            try:
                sm.append(float(f[0]))
                mx = max(mx, float(f[1]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(circ, bits, k, plan_order, plan_slices, budget_s):
    """The oracle (C bucket elimination, all host cores) on whole amplitudes of the same
    workload, repeated until about `budget_s` seconds of work."""
    from oracle import ve as VE
    threads = os.cpu_count() or 1
    VE.build_library()
    done, t0 = 0, time.perf_counter()
    while True:
        VE.ve_amplitude(circ, bits[done % len(bits)], plan_order, plan_slices, threads=threads)
        done += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": "amplitudes/s", "cores": threads, "kind": "oracle",
            "sample": f"{done} whole amplitudes (all {1 << k} slice terms each) of the same circuit, "
                      f"complex128 bucket elimination in the plan's order, OpenMP over slices"}


REFERENCE_SLICES_PER_STEP = 256


def run_reference(args, rank, world):
    """The oracle as the reference arm: each step evaluates a bounded sample of one
    amplitude (REFERENCE_SLICES_PER_STEP of its slice terms, cycling through them), so the
    rate in amplitudes/s is slice terms per second / slice terms per amplitude."""
    if rank != 0:
        return
    import numpy as np
    from oracle import ve as VE
    circ, bits, k = workload(args.workload, args.batch, 0, args.circuit_seed)
    if args.sliced is not None:
        k = args.sliced
    args.batch = len(bits)
    import paper_1805_01450_gb300 as q
    trials = args.plan_trials if args.plan_trials is not None else PLAN_TRIALS.get(args.workload, 1)
    # host planner only: the oracle takes its order and slices
    plan = q.Plan(circ, n_slices=k, plan_trials=1 if is_grad(args.workload) else trials)
    threads = os.cpu_count() or 1
    VE.build_library()
    total = 1 << k
    per = min(REFERENCE_SLICES_PER_STEP, total)

    def one(i):
        ids = (np.arange(per, dtype=np.int64) + i * per) % total
        for x in bits:
            VE.slice_terms(circ, x, plan.order, plan.slices, slice_ids=ids, threads=threads)

    for i in range(args.warmup):
        one(i)
    t0 = time.perf_counter()
    for i in range(args.steps):
        one(i)
    dt = time.perf_counter() - t0
    v = args.steps * per * len(bits) / total / dt
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "amplitudes/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
           "data": "synthetic", "config": {"workload": args.workload, "bitstrings_per_step": args.batch,
                                           "sliced": k},
           "cpu_baseline": {"value": v, "unit": "amplitudes/s", "cores": threads, "kind": "oracle",
                            "sample": f"{per} of the {total} slice terms of one amplitude per step, "
                                      f"{args.steps} steps, complex128 bucket elimination"},
           "e2e": {"value": v, "unit": "amplitudes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import paper_1805_01450_gb300 as q
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    circ, bits_host, k = workload(args.workload, args.batch, rank, args.circuit_seed)
    if args.plan_trials is None:
        args.plan_trials = 1 if is_grad(args.workload) else PLAN_TRIALS.get(args.workload, 1)
    if args.sliced is not None:
        k = args.sliced
    if args.mem_budget_mb is None:
        args.mem_budget_mb = MEM_BUDGET_MB.get(args.workload, 1024)
    budget = args.mem_budget_mb << 20
    dev = torch.device("cuda", local)
    grad = is_grad(args.workload)
    tuning = None
    if args.inner_slices is None and args.warps_per_item is None and args.engine == "auto" and not grad:
        from paper_1805_01450_gb300.autotune import autotune
        tune = dict(TUNE.get(args.workload, {})) if args.sliced is None else {}
        plan, tuning = autotune(circ, bits_host, n_slices=k, device=dev, mem_budget_bytes=budget,
                                plan_trials=args.plan_trials, **tune)
        if plan is None:
            raise SystemExit(f"autotune: no plan variant of {args.workload} could be built or timed")
    else:
        # gradient workload: one sliced variable open inside a work item (128 items, each on a
        # CTA of the staged shared-memory kernel at once)
        inner = args.inner_slices if args.inner_slices is not None else (1 if grad else -1)
        plan = q.Plan(circ, n_slices=k, inner_slices=inner,
                      warps_per_item=args.warps_per_item or 1, engine=args.engine, gradient=grad,
                      mem_budget_bytes=budget, tensor_cores=args.tensor_cores, plan_trials=args.plan_trials,
                      host_merge_rank=args.host_merge_rank)
    info = plan.info
    B = len(bits_host)
    bits = plan._bits(bits_host, dev)
    ws = plan.workspace(B, dev)
    out = torch.empty(2 * B, dtype=torch.float64, device=dev)
    gout = torch.empty(2 * B * max(info["n_params"], 1), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    L = q.lib()
    sptr = q._stream_ptr(stream)

    def step():
        if grad:   # amplitude and every d alpha / d theta (one qvx_amplitude_grad call)
            q._check(L.qvx_amplitude_grad(plan._h, q.ctypes.c_void_p(bits.data_ptr()), B, None, 0,
                                          q.ctypes.c_void_p(out.data_ptr()), q.ctypes.c_void_p(gout.data_ptr()),
                                          q.ctypes.c_void_p(ws.data_ptr()), ws.numel(), sptr))
        else:
            plan.amplitude(bits, workspace=ws, out=out, validate=False, stream=stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    plan.check_status(ws)

    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    with ClockSampler(torch.cuda.current_device()) as clocks:
        barrier()
        torch.cuda.synchronize()
        launches0 = L.qvx_kernel_launches()
        for i in range(K):
            flush.zero_()
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        barrier()
    launches = L.qvx_kernel_launches() - launches0   # this library's kernels in the timed region
    dev_ms = sum(a.elapsed_time(b) for a, b in ev)
    plan.check_status(ws)

    # end to end through the public call: pinned host bitstrings in, amplitudes (and
    # gradients) out
    h_bits = torch.tensor([b - (1 << 64) if b >= 1 << 63 else b for b in bits_host], dtype=torch.int64).pin_memory()
    h_out = torch.empty(2 * B, dtype=torch.float64).pin_memory()
    h_gout = torch.empty(gout.numel(), dtype=torch.float64).pin_memory()
    e2e_s = 0.0
    barrier()
    torch.cuda.synchronize()
    if grad:
        ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        for i in range(K):
            flush.zero_()
            ev2[i][0].record(stream)
            bits.copy_(h_bits, non_blocking=True)
            step()
            h_out.copy_(out, non_blocking=True)
            h_gout.copy_(gout, non_blocking=True)
            ev2[i][1].record(stream)
        torch.cuda.synchronize()
        e2e_s = sum(a.elapsed_time(b) for a, b in ev2) / 1e3
    else:
        # the blocking host-buffer call: the kernel reads the pinned bitstrings and writes
        # the pinned amplitudes itself; host wall clock around each call
        hb, ho = q.ctypes.c_void_p(h_bits.data_ptr()), q.ctypes.c_void_p(h_out.data_ptr())
        wsp = q.ctypes.c_void_p(ws.data_ptr())
        for i in range(K):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            q._check(L.qvx_amplitude_host(plan._h, hb, B, ho, wsp, ws.numel(), sptr))
            e2e_s += time.perf_counter() - t0
    barrier()
    e2e_ms = 1e3 * e2e_s

    # parity of what was timed, against the oracle's slice terms (first bitstring), when
    # the oracle finishes in seconds
    from oracle import ve as VE
    n = circ.n_qubits
    err = None
    if info["log2_cost"] + len(plan.slices) <= 26:
        ref = VE.exact_sum(VE.slice_terms(circ, bits_host[0], plan.order, plan.slices))
        got = complex(h_out[0].item(), h_out[1].item())
        err = abs(got - ref)

    t = torch.tensor([dev_ms, e2e_ms], dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dev_ms, e2e_ms = float(t[0]), float(t[1])
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    amps = K * B * world
    value = amps / (dev_ms / 1e3)
    e2e = amps / (e2e_ms / 1e3)
    ms_step = dev_ms / K
    flops = (info["grad_flops_per_amplitude"] if grad else info["flops_per_amplitude"]) * B
    algo_bytes = (info["grad_bytes_per_amplitude"] if grad else info["bytes_per_amplitude"]) * B
    peak, peak_kind = measured_peaks()
    achieved = algo_bytes / (ms_step / 1e3) / 1e9
    fused = info["engine"] == "fused" and not grad
    if grad:
        kernel = "grad_smem_kernel" if 0 < info["grad_smem_bytes"] <= 232448 else "grad_program_kernel"
    elif fused:
        kernel = "fused_program_kernel"
    elif info["engine"] == "persistent":
        kernel = "persistent_program_kernel"
    else:
        kernel = "regtile_step_kernel"
    res = {
        "metric": METRIC, "value": value, "unit": "amplitudes/s", "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64", "data": "synthetic",
        "config": {"workload": args.workload, "circuit_seed": WORKLOADS[args.workload][4]
                   if args.circuit_seed is None else args.circuit_seed,
                   "qubits": n, "depth": circ.depth, "sliced": len(plan.slices),
                   "inner_slices": info["n_inner"], "bitstrings_per_step": B, "engine": info["engine"],
                   "warps_per_item": info["warps_per_item"], "mem_budget_mb": args.mem_budget_mb,
                   "tensor_core_steps": info["n_gemm_steps"], "plan_trials": plan.plan_trials,
                   "l2": "flushed (256 MiB write) before each step",
                   "parallelism": f"bitstrings per rank x {world}"},
        "complex_tflops": flops / (ms_step / 1e3) / 1e12,
        "abs_err": err, "err_bound": 1e-5 * 2.0 ** (-n / 2),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": NCU_TRAFFIC.get((args.workload, B, info["device_image_bytes"])),
                     "peak_source": peak_kind,
                     "kernel": kernel,
                     "algorithmic_bytes_per_launch": algo_bytes},
        "e2e": {"value": e2e, "unit": "amplitudes/s", "h2d_bytes_per_step": 8 * B,
                "d2h_bytes_per_step": 16 * B + (8 * gout.numel() if grad else 0)},
        "gpu_launches": launches,
        "clocks": clocks.summary(),
        "autotune": None if tuning is None else [list(t) for t in tuning],
        "gradients_per_amplitude": info["n_params"] if grad else 0,
        "plan": {"n_vars": info["n_vars"], "n_steps": info["n_steps"], "log2_cost": info["log2_cost"],
                 "log2_cost_unsliced": info["log2_cost_unsliced"], "max_rank": info["max_rank"],
                 "arena_bytes": info["arena_bytes"]},
    }
    if world == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(circ, bits_host, k, plan.order, plan.slices, args.cpu_seconds)
    print(json.dumps(res), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
