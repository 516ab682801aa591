#!/usr/bin/env python
"""Throughput of single amplitudes <x|C|0> by sliced variable elimination on one GB300.

Default workload: the 8 x 8 random grid circuit of depth 40 (64 qubits, Section 4 rules,
circuit seed 5001), one seeded bitstring (seed 5002) per step, 10 sliced variables (1024
slice terms, 5 of the variables kept open inside a work item: 32 work items), the plan
variant kept for this circuit (recorded below: the ordering and sliced variables of 16384
planning trials, stored in paper_1805_01450_gb300/orderings/; --autotune re-runs the
autotuner instead). A
step is one whole amplitude: every slice term, every pairwise contraction (the dense ones
on the tcgen05 tensor cores as three-part bf16 GEMMs, the rest as FP32 SIMT kernels) and
the exact sum of the slice terms.

Prints one JSON line. Timing: CUDA events on the launching stream around each step, W
warm-up steps first, L2 flushed (a 256 MiB write) before every timed step, max over ranks.
Inside the timed region every kernel launch is bracketed by CUDA events too (the library's
launch log), which gives each kernel's duration for its roofline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl qvx|reference] [--workload W]
  torchrun --nproc-per-node N bench.py --gpus N ...                 (each rank: its own bitstrings)
  torchrun --nproc-per-node N bench.py --gpus N --shard slices ...  (the ranks share the slices)
"""
import argparse
import json
import math
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
    "grid8x8d40": ("grid", 8, 8, 40, 5001, 5002, 10, 1),
    "grid6x6d25-k12": ("grid", 6, 6, 25, 2001, 2002, 12, 1),
    "grid4x4d10": ("grid", 4, 4, 10, 1001, 1002, 0, 1),
    "grid7x7d30-b1024": ("grid", 7, 7, 30, 3001, 3002, 4, 1024),
    "rot5x5d20-grad": ("rotation", 5, 5, 20, 4001, 4002, 8, 1),
    "grid9x9d40": ("grid", 9, 9, 40, 9001, 9002, 20, 1),
}
# workloads timed on a contiguous sample of each amplitude's slice terms (slice terms per
# step); their amplitude rate is extrapolated: steps x sample / 2^k / time
SLICE_SAMPLE = {"grid9x9d40": 1 << 10}
DEFAULT_WORKLOAD = "grid8x8d40"
# The plan variant kept for each circuit seed of a workload, from timing (L2 flushed, CUDA
# events) the stepwise tensor-core engine at 10 sliced variables over planning-trial counts
# 16 ... 4096 (trials ranked by the planner's kernel-rate estimate) and 4, 5 or 6 sliced
# variables open inside a work item. The timed plan, its parity tests
# (tests/test_gpu_8x8x40.py) and its ncu traffic are keyed by these. 9x9x40 (20 sliced):
# 8, 512 and 2048 trials gave 278, 75 and 36 ms per 1024 slice terms (the 2048 trials take
# about two minutes on 16 host cores).
RECORDED_PLANS = {
    ("grid8x8d40", 5001): dict(n_slices=10, inner_slices=5, engine="stepwise", tensor_cores=True, plan_trials=16384,
                               ordering=True),
    ("grid8x8d40", 5002): dict(n_slices=10, inner_slices=6, engine="stepwise", tensor_cores=True, plan_trials=16384,
                               ordering=True),
    ("grid8x8d40", 5003): dict(n_slices=10, inner_slices=6, engine="stepwise", tensor_cores=True, plan_trials=16384,
                               ordering=True),
    ("grid9x9d40", 9001): dict(n_slices=20, inner_slices=5, engine="stepwise", tensor_cores=True, plan_trials=2048),
}
# autotuner search of the workloads without a recorded plan
TUNE = {"grid6x6d25-k12": dict(trial_counts=(1, 16, 256)),
        "grid7x7d30-b1024": dict(slice_counts=(0, 2, 4, 6, 8), engines=("stepwise",), budget_s=90.0),
        "grid8x8d40": dict(slice_counts=(10, 12), engines=("stepwise", "stepwise-tc"), inner=(4,),
                           trial_counts=(1, 16, 64, 256), budget_s=120.0)}
MEM_BUDGET_MB = {"grid7x7d30-b1024": 32768, "grid8x8d40": 65536, "grid9x9d40": 65536}
# independent planning trials (ordering + slice choice from distinct seeds, the best by the
# planner's bandwidth-weighted estimate kept); planning is outside the timed region
PLAN_TRIALS = {"grid6x6d25-k12": 64, "grid7x7d30-b1024": 64, "grid8x8d40": 64}
METRIC = "amplitudes/s and complex TFLOP/s (% of GB300 peak) at |Δα|≤1e-5·2^-N/2 vs FP64"
L2_FLUSH_BYTES = 256 << 20
# dram__bytes_read.sum + dram__bytes_write.sum per launch of the dominant kernel, averaged
# over its launches in one ncu launch list of the workload's timed plan (profiles/ holds
# the summaries and commands). Keyed by (workload, circuit seed, kernel, device image bytes
# of the plan): another plan, or a kernel changed since the capture, reports null.
NCU_TRAFFIC = {("grid8x8d40", 5001, "gemm_tc_kernel", 241664): 10230352774.4,
               ("grid8x8d40", 5001, "regtile_step_kernel", 241664): 1338227991.4}
# FP32 SIMT peak for the "alu" bound: 152 SMs x 128 FP32 lanes x 2 flops (FMA) x 2.07 GHz
FP32_SIMT_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# the tensor-core contraction spends 48 bf16 flops per complex multiply-add (4 real MACs of
# the real block form, each as 6 products of three-part bf16 splits) against 8 algorithmic
# flops, so its algorithmic peak is 8/48 of the bf16 rate
TC_ALGO_PER_BF16 = 8.0 / 48.0


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["qvx", "reference"], default="qvx")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--batch", type=int, default=None, help="bitstrings per step (workload default)")
    ap.add_argument("--autotune", action="store_true", help="re-run the autotuner instead of the recorded plan")
    ap.add_argument("--inner-slices", type=int, default=None, help="fix the plan variant instead of autotuning")
    ap.add_argument("--mem-budget-mb", type=int, default=None,
                    help="arena memory of the global-arena engines (work items in flight; workload default)")
    ap.add_argument("--warps-per-item", type=int, default=None)
    ap.add_argument("--host-merge-rank", type=int, default=8, help="fixed plan variant: leaf products contracted at plan time")
    ap.add_argument("--tensor-cores", action="store_true",
                    help="stepwise engine: dense contractions as three-part bf16 GEMMs on the tensor cores")
    ap.add_argument("--engine", default="auto")
    ap.add_argument("--sliced", type=int, default=None, help="override the workload's sliced-variable count")
    ap.add_argument("--plan-trials", type=int, default=None, help="planning trials (workload default)")
    ap.add_argument("--circuit-seed", type=int, default=None, help="override the workload's circuit seed")
    ap.add_argument("--shard", choices=["bitstrings", "slices"], default="bitstrings",
                    help="under torchrun: each rank its own bitstrings, or the ranks share every amplitude's slices")
    ap.add_argument("--slice-sample", type=int, default=None,
                    help="slice terms per step (a contiguous range; the amplitude rate is extrapolated); 0: all")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32-forms", action="store_true", help="skip timing the plain FP32 forms of the plan")
    ap.add_argument("--cpu-seconds", type=float, default=20.0, help="CPU-baseline sample budget")
    ap.add_argument("--plan-json", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--record-ordering", action="store_true",
                    help="run the planner for the workload's recorded variant and store its ordering")
    ap.add_argument("--record-trial", type=int, default=None,
                    help="with --record-ordering: store this planning trial instead of the estimate's first")
    ap.add_argument("--selected-by", default="chosen by timing", help=argparse.SUPPRESS)
    return ap.parse_args(argv)


def workload(name, batch, rank, circuit_seed=None):
    kind, r, c, d, cseed, bseed, k, b0 = WORKLOADS[name]
    batch = b0 if batch is None else batch
    cseed = cseed if circuit_seed is None else circuit_seed
    circ = cg.grid_circuit(r, c, d, cseed) if kind == "grid" else cg.rotation_circuit(r, c, d, cseed)
    bits = cg.random_bitstrings(r * c, batch * (rank + 1), bseed)[batch * rank:]
    return circ, bits, k


def is_grad(name):
    return name.endswith("-grad")


def circuit_seed(args):
    return WORKLOADS[args.workload][4] if args.circuit_seed is None else args.circuit_seed


def recorded_plan(args):
    """The recorded plan variant for this run, or None (overrides and --autotune disable it)."""
    if args.autotune or args.sliced is not None or args.plan_trials is not None or args.inner_slices is not None \
            or args.engine != "auto" or args.warps_per_item is not None or args.tensor_cores:
        return None
    return RECORDED_PLANS.get((args.workload, circuit_seed(args)))


# Recorded orderings: the planning trials are the slow part of planning (16384 trials of the
# 64-qubit circuit take minutes on the host cores), so a variant marked `ordering` stores the
# winning trial's elimination order and sliced variables (written by `bench.py
# --record-ordering`, which runs the planner); the plan's program is rebuilt from them in
# about a second. Without the file the planner runs the trials itself.
ORDERINGS = os.path.join(ROOT, "paper_1805_01450_gb300", "orderings")


def ordering_path(workload_name, seed):
    return os.path.join(ORDERINGS, f"{workload_name}-s{seed}.json")


def recorded_plan_kwargs(workload_name, seed):
    """Plan keyword arguments of a recorded variant, with its recorded ordering if there is
    one: (kwargs, planning trials it stands for, where the ordering came from)."""
    rec = dict(RECORDED_PLANS[(workload_name, seed)])
    trials = rec["plan_trials"]
    if rec.pop("ordering", False) and os.path.exists(ordering_path(workload_name, seed)):
        with open(ordering_path(workload_name, seed)) as f:
            d = json.load(f)
        rec.pop("plan_trials")
        rec.pop("n_slices")
        rec["order"], rec["slices"] = d["order"], d["slices"]
        if "trial" in d:
            return rec, trials, f"recorded (trial {d['trial']} of {trials} planning trials, {d['selected_by']})"
        return rec, trials, f"recorded ({trials} planning trials)"
    return rec, trials, "planned in this run"


# planning trial t runs from order seed 1 + t * TRIAL_SEED_STEP (mod 2^64), as in the planner
TRIAL_SEED_STEP = 0xD1B54A32D192ED03


def record_ordering(args):
    """Runs the planner for the workload's recorded variant and stores its ordering. With
    --record-trial T it stores trial T of the search instead of the one the planner's
    estimate ranks first (the trial a timing of the estimate's best-ranked trials kept)."""
    import paper_1805_01450_gb300 as q
    seed = circuit_seed(args)
    rec = dict(RECORDED_PLANS[(args.workload, seed)])
    rec.pop("ordering", None)
    if args.plan_trials is not None:
        rec["plan_trials"] = args.plan_trials
    circ = workload(args.workload, None, 0, args.circuit_seed)[0]
    budget = (args.mem_budget_mb or MEM_BUDGET_MB.get(args.workload, 1024)) << 20
    t0 = time.perf_counter()
    extra = {}
    if args.record_trial is not None:
        one = dict(rec, plan_trials=1, order_seed=(1 + args.record_trial * TRIAL_SEED_STEP) % (1 << 64))
        plan = q.Plan(circ, mem_budget_bytes=budget, **one)
        extra = {"trial": args.record_trial, "selected_by": args.selected_by}
    else:
        plan = q.Plan(circ, mem_budget_bytes=budget, **rec)
    out = {"workload": args.workload, "circuit_seed": seed, "variant": rec, **extra, "mem_budget_mb": budget >> 20,
           "planner_seconds": time.perf_counter() - t0, "host_threads": min(os.cpu_count() or 1, 16),
           "bytes_per_amplitude": plan.info["bytes_per_amplitude"], "device_image_bytes": plan.info["device_image_bytes"],
           "order": [int(v) for v in plan.order], "slices": [int(v) for v in plan.slices]}
    os.makedirs(ORDERINGS, exist_ok=True)
    with open(ordering_path(args.workload, seed), "w") as f:
        json.dump(out, f)
        f.write("\n")
    print(json.dumps({k: v for k, v in out.items() if k not in ("order", "slices")}))


def measured_peaks():
    """(HBM GB/s, bf16 dense TFLOP/s burst, source) from MEASURED_PEAKS.json, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), float(pk["bf16_tflops"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, 1900.0, "fallback"


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


def sample_slice_ids(total, count, seed):
    """`count` seeded slice numbers in [0, total): distinct while count <= total."""
    import numpy as np
    rng = np.random.default_rng(seed)
    if count <= total:
        return [int(v) for v in rng.choice(total, size=count, replace=False)]
    return [int(v) for v in rng.integers(0, total, size=count)]


def oracle_terms(circ, x, order, slices, ids, threads):
    """The oracle's slice terms beta_s (complex128) for slice numbers `ids`, OpenMP over them."""
    import numpy as np
    from oracle import ve as VE
    return VE.slice_terms(circ, x, order, slices, slice_ids=np.asarray(ids, dtype=np.int64), threads=threads)


def cpu_baseline(circ, x, order, slices, budget_s, seed):
    """The oracle (C bucket elimination, complex128, OpenMP over slice terms on all host cores)
    on a seeded sample of the amplitude's slice terms, in rounds of growing size until about
    `budget_s` seconds of wall time (at least one term per core). The amplitude rate is
    extrapolated: sampled terms per second / slice terms per amplitude. Returns the baseline
    dict and the sampled (ids, terms) for the parity figures."""
    from oracle import ve as VE
    threads = os.cpu_count() or 1
    VE.build_library()
    total = 1 << len(slices)
    pool = sample_slice_ids(total, min(total, 1 << 16), seed)
    ids, terms, done, n, dt = [], [], 0, threads, 0.0
    while True:
        chunk = [pool[(done + i) % len(pool)] for i in range(n)]
        t0 = time.perf_counter()
        out = oracle_terms(circ, x, order, slices, chunk, threads)
        dt += time.perf_counter() - t0
        ids += chunk
        terms += list(out)
        done += n
        if dt >= budget_s or done >= 1 << 20:
            break
        n = min(2 * n, max(threads, int(n * budget_s / max(dt, 1e-3))))
    rate = done / dt / total
    base = {"value": rate, "unit": "amplitudes/s", "cores": threads, "kind": "oracle",
            "sample": f"{done} seeded slice terms of the {total} of one amplitude, complex128 bucket elimination "
                      f"in the plan's order, OpenMP over the terms, {dt:.1f} s; amplitude rate extrapolated "
                      f"(terms per second / {total})",
            "extrapolated": done < total}
    return base, ids, terms


def slice_parity(plan, x, ids, ref_terms, n_qubits, dev, ws):
    """GPU slice terms (qvx_slice_terms over the whole slice range) against the oracle's on
    the sampled slice numbers: max and rms of |d beta|, and the aggregate sqrt(2^k) rms."""
    import numpy as np
    got = plan.slice_terms(plan._bits([x], dev), workspace=ws).cpu().numpy()[0]
    d = np.abs(got[np.asarray(ids)] - np.asarray(ref_terms))
    rms = float(np.sqrt(np.mean(d * d)))
    c13 = math.sqrt(plan.n_slice_terms) * rms
    return {"sampled": len(ids), "max": float(np.max(d)), "rms": rms, "c13": c13,
            "bound": 1e-5 * 2.0 ** (-n_qubits / 2), "pass": c13 <= 1e-5 * 2.0 ** (-n_qubits / 2)}


def build_plan(args, circ, k, budget, dev, bits_host, need_timing=True):
    """The plan for this run and how it was chosen: (plan, tuning results or None, plan seconds)."""
    import paper_1805_01450_gb300 as q
    grad = is_grad(args.workload)
    rec = recorded_plan(args)
    t0 = time.perf_counter()
    if rec is not None:
        kw, trials, args.ordering_source = recorded_plan_kwargs(args.workload, circuit_seed(args))
        plan = q.Plan(circ, mem_budget_bytes=budget, **kw)
        plan.plan_trials = trials
        return plan, None, time.perf_counter() - t0
    trials = args.plan_trials if args.plan_trials is not None else (1 if grad else PLAN_TRIALS.get(args.workload, 1))
    if need_timing and args.inner_slices is None and args.warps_per_item is None and args.engine == "auto" and not grad:
        from paper_1805_01450_gb300.autotune import autotune
        tune = dict(TUNE.get(args.workload, {})) if args.sliced is None else {}
        plan, tuning = autotune(circ, bits_host, n_slices=k, device=dev, mem_budget_bytes=budget,
                                plan_trials=trials, **tune)
        if plan is None:
            raise SystemExit(f"autotune: no plan variant of {args.workload} could be built or timed")
        return plan, tuning, time.perf_counter() - t0
    # gradient workload: one sliced variable open inside a work item (128 items, each on a CTA
    # of the staged shared-memory kernel at once)
    inner = args.inner_slices if args.inner_slices is not None else (1 if grad else -1)
    plan = q.Plan(circ, n_slices=k, inner_slices=inner, warps_per_item=args.warps_per_item or 1, engine=args.engine,
                  gradient=grad, mem_budget_bytes=budget, tensor_cores=args.tensor_cores, plan_trials=trials,
                  host_merge_rank=args.host_merge_rank)
    return plan, None, time.perf_counter() - t0


def run_config(args, circ, plan, world, B):
    info = plan.info
    return {"workload": args.workload, "circuit_seed": circuit_seed(args), "qubits": circ.n_qubits,
            "depth": circ.depth, "sliced": len(plan.slices), "inner_slices": info["n_inner"],
            "bitstrings_per_step": B, "engine": info["engine"], "warps_per_item": info["warps_per_item"],
            "mem_budget_mb": args.mem_budget_mb, "tensor_core_steps": info["n_gemm_steps"],
            "plan_trials": plan.plan_trials, "ordering": getattr(args, "ordering_source", "planned in this run"),
            "l2": "flushed (256 MiB write) before each step",
            "parallelism": (f"slices split over {world} ranks" if args.shard == "slices" and world > 1
                            else f"bitstrings per rank x {world}"),
            **({"slice_sample": slice_sample(args, plan), "extrapolated": True} if slice_sample(args, plan) else {})}


def slice_sample(args, plan):
    """Slice terms per step when the run samples each amplitude's slices, else 0."""
    n = SLICE_SAMPLE.get(args.workload, 0) if args.slice_sample is None else args.slice_sample
    return min(n, plan.n_slice_terms) if n and n < plan.n_slice_terms else 0


def plan_json(args):
    """--plan-json: the run's plan (order, slices) and config, for the reference arm, which
    takes them from this separate process so that its own process loads only the oracle."""
    circ, bits_host, k = workload(args.workload, args.batch, 0, args.circuit_seed)
    if args.sliced is not None:
        k = args.sliced
    if args.mem_budget_mb is None:
        args.mem_budget_mb = MEM_BUDGET_MB.get(args.workload, 1024)
    plan, _, _ = build_plan(args, circ, k, args.mem_budget_mb << 20, None, bits_host, need_timing=False)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    print(json.dumps({"order": plan.order, "slices": plan.slices, "log2_cost": plan.info["log2_cost"],
                      "config": run_config(args, circ, plan, world, len(bits_host))}), flush=True)


def run_reference(args, rank, world):
    """The oracle as the reference arm, on the same workload, plan order and slices as the
    GPU arm: the W warm-up steps and then the K timed steps each evaluate a bounded sample of
    one amplitude's slice terms (one term per step on the 64-qubit circuit, up to 256 on the
    small ones); the timed steps' terms run in one OpenMP call over the host cores, and the
    rate in amplitudes/s is slice terms per second / slice terms per amplitude."""
    if rank != 0:
        return
    cmd = [sys.executable, os.path.abspath(__file__), "--plan-json", "--workload", args.workload]
    if args.shard != "bitstrings":
        cmd += ["--shard", args.shard]
    for flag, v in (("--batch", args.batch), ("--sliced", args.sliced), ("--plan-trials", args.plan_trials),
                    ("--circuit-seed", args.circuit_seed), ("--inner-slices", args.inner_slices),
                    ("--mem-budget-mb", args.mem_budget_mb), ("--warps-per-item", args.warps_per_item)):
        if v is not None:
            cmd += [flag, str(v)]
    if args.engine != "auto":
        cmd += ["--engine", args.engine]
    if args.tensor_cores:
        cmd.append("--tensor-cores")
    pj = json.loads([l for l in subprocess.run(cmd, check=True, capture_output=True, text=True).stdout.splitlines()
                     if l.startswith("{")][-1])
    from oracle import ve as VE
    circ, bits, k = workload(args.workload, args.batch, 0, args.circuit_seed)
    threads = os.cpu_count() or 1
    VE.build_library()
    total = 1 << len(pj["slices"])
    per = int(min(total, 256, max(1, 2 ** (22 - pj["log2_cost"]))))
    ids = sample_slice_ids(total, min(total, (args.warmup + args.steps) * per), 7)
    ids = [ids[i % len(ids)] for i in range((args.warmup + args.steps) * per)]
    warm, timed = ids[:args.warmup * per], ids[args.warmup * per:]
    if warm:
        for x in bits:
            oracle_terms(circ, x, pj["order"], pj["slices"], warm, threads)
    t0 = time.perf_counter()
    for x in bits:
        oracle_terms(circ, x, pj["order"], pj["slices"], timed, threads)
    dt = time.perf_counter() - t0
    v = args.steps * per * len(bits) / total / dt
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "amplitudes/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
           "data": "synthetic", "config": pj["config"],
           "cpu_baseline": {"value": v, "unit": "amplitudes/s", "cores": threads, "kind": "oracle",
                            "sample": f"{per} of the {total} slice terms of one amplitude per step "
                                      f"({args.steps} steps' terms in one OpenMP call), complex128 bucket "
                                      f"elimination in the GPU arm's plan order",
                            "extrapolated": True},
           "e2e": {"value": v, "unit": "amplitudes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def kernel_roofline(records, hbm_gbs, bf16_tflops):
    """Per-kernel totals of the timed launch log and the dominant kernel's roofline. Each
    launch's roofline time is max(bytes / HBM, flops / compute peak), the compute peak being
    the FP32 SIMT rate, or the tensor cores' algorithmic rate for the GEMM kernel."""
    per = {}
    for r in records:
        peak = bf16_tflops * TC_ALGO_PER_BF16 if r["kernel"] == "gemm_tc_kernel" else FP32_SIMT_TFLOPS
        t_mem = r["bytes"] / (hbm_gbs * 1e9)
        t_cmp = r["flops"] / (peak * 1e12)
        d = per.setdefault(r["kernel"], {"launches": 0, "ms": 0.0, "bytes": 0.0, "flops": 0.0, "t_mem": 0.0,
                                         "t_cmp": 0.0, "t_roof": 0.0, "peak_tflops": peak})
        d["launches"] += 1
        d["ms"] += r["ms"]
        d["bytes"] += r["bytes"]
        d["flops"] += r["flops"]
        d["t_mem"] += t_mem
        d["t_cmp"] += t_cmp
        d["t_roof"] += max(t_mem, t_cmp)
    total = sum(d["ms"] for d in per.values()) or 1.0
    summary = {k: {"launches": d["launches"], "ms": d["ms"], "share": d["ms"] / total,
                   "gbs": d["bytes"] / (d["ms"] / 1e3) / 1e9 if d["ms"] else None,
                   "tflops": d["flops"] / (d["ms"] / 1e3) / 1e12 if d["ms"] else None,
                   "roofline_time_frac": d["t_roof"] / (d["ms"] / 1e3) if d["ms"] else None}
               for k, d in per.items()}
    name = max(per, key=lambda k: per[k]["ms"])
    d = per[name]
    sec = d["ms"] / 1e3
    if d["t_mem"] >= d["t_cmp"]:
        bound, achieved, peak, unit = "hbm", d["bytes"] / sec / 1e9, hbm_gbs, "GB/s"
    else:
        bound = "tensor" if name == "gemm_tc_kernel" else "alu"
        achieved, peak, unit = d["flops"] / sec / 1e12, d["peak_tflops"], "TFLOP/s"
    roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
            "kernel": name, "launches": d["launches"],
            "algorithmic_bytes_per_launch": d["bytes"] / d["launches"],
            "algorithmic_flops_per_launch": d["flops"] / d["launches"],
            "mean_launch_ms": d["ms"] / d["launches"],
            "roofline_time_frac": d["t_roof"] / sec}
    return roof, summary


def time_form(plan, bits, reps, flush, stream):
    """Mean device ms per amplitude call of `plan` (one warm-up call; L2 flushed before each)."""
    import torch
    n = bits.numel() // plan.words
    ws = plan.workspace(n, bits.device)
    out = torch.empty(2 * n << plan.n_open, dtype=torch.float64, device=bits.device)
    plan.amplitude(bits, workspace=ws, out=out, validate=False)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for e0, e1 in evs:
        flush.zero_()
        e0.record(stream)
        plan.amplitude(bits, workspace=ws, out=out, validate=False)
        e1.record(stream)
    torch.cuda.synchronize()
    plan.check_status(ws)
    return sum(a.elapsed_time(b) for a, b in evs) / reps


def main():
    args = parse()
    if args.plan_json:
        return plan_json(args)
    if args.record_ordering:
        return record_ordering(args)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch
    import paper_1805_01450_gb300 as q
    from paper_1805_01450_gb300.distributed import compensated_sum, slice_range
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    shard = args.shard == "slices" and world > 1
    circ, bits_host, k = workload(args.workload, args.batch, 0 if shard else rank, args.circuit_seed)
    if args.sliced is not None:
        k = args.sliced
    if args.mem_budget_mb is None:
        args.mem_budget_mb = MEM_BUDGET_MB.get(args.workload, 1024)
    budget = args.mem_budget_mb << 20
    dev = torch.device("cuda", local)
    grad = is_grad(args.workload)
    plan, tuning, plan_s = build_plan(args, circ, k, budget, dev, bits_host)
    info = plan.info
    B = len(bits_host)
    bits = plan._bits(bits_host, dev)
    ws = plan.workspace(B, dev)
    out = torch.empty(2 * B << plan.n_open, dtype=torch.float64, device=dev)
    gout = torch.empty(2 * B * max(info["n_params"], 1), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    L = q.lib()
    sptr = q._stream_ptr(stream)
    sample = slice_sample(args, plan)
    s_begin, s_end = slice_range(plan.n_slice_terms, rank, world) if shard else (0, sample or plan.n_slice_terms)
    partial = shard or bool(sample)
    gathered = torch.empty(world * 2 * B, dtype=torch.float64, device=dev) if shard else None

    def step(profiled=False):
        if grad:   # amplitude and every d alpha / d theta (one qvx_amplitude_grad call)
            q._check(L.qvx_amplitude_grad(plan._h, q.ctypes.c_void_p(bits.data_ptr()), B, None, 0,
                                          q.ctypes.c_void_p(out.data_ptr()), q.ctypes.c_void_p(gout.data_ptr()),
                                          q.ctypes.c_void_p(ws.data_ptr()), ws.numel(), sptr))
        elif profiled:
            plan.amplitude_profiled(bits, ws, out, stream, slice_begin=s_begin, slice_count=s_end - s_begin)
        elif partial:   # this rank's (or the sample's) slice range
            plan.amplitude(bits, workspace=ws, out=out, validate=False, stream=stream, slice_begin=s_begin,
                           slice_count=s_end - s_begin)
        else:
            plan.amplitude(bits, workspace=ws, out=out, validate=False, stream=stream)
        if shard:   # one all_gather of the B complex128 partials
            dist.all_gather_into_tensor(gathered, out)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    plan.check_status(ws)
    plan.read_profile()

    K = args.steps
    profiled = not grad
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    with ClockSampler(torch.cuda.current_device()) as clocks:
        barrier()
        torch.cuda.synchronize()
        launches0 = L.qvx_kernel_launches()
        for i in range(K):
            flush.zero_()
            ev[i][0].record(stream)
            step(profiled)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        barrier()
    launches = L.qvx_kernel_launches() - launches0   # this library's kernels in the timed region
    dev_ms = sum(a.elapsed_time(b) for a, b in ev)
    plan.check_status(ws)
    records = plan.read_profile() if profiled else []

    # end to end through the public call: pinned host bitstrings in, amplitudes (and
    # gradients) out
    h_bits = torch.tensor(q.bitstring_words(bits_host, plan.words), dtype=torch.int64).pin_memory()
    h_out = torch.empty(2 * B << plan.n_open, dtype=torch.float64).pin_memory()
    h_gout = torch.empty(gout.numel(), dtype=torch.float64).pin_memory()
    h_gath = torch.empty(gathered.numel(), dtype=torch.float64).pin_memory() if shard else None
    e2e_s = 0.0
    barrier()
    torch.cuda.synchronize()
    if grad or partial:
        ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        for i in range(K):
            flush.zero_()
            ev2[i][0].record(stream)
            bits.copy_(h_bits, non_blocking=True)
            step()
            if shard:   # every rank's partials (combined on the host in rank order)
                h_gath.copy_(gathered, non_blocking=True)
            else:
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

    amp = None
    if shard:   # the ranks' partials in rank order, compensated
        g = gathered.view(world, B, 2).cpu().numpy()
        amp = compensated_sum(g[..., 0] + 1j * g[..., 1])[0]
    elif not grad:
        amp = complex(h_out[0].item(), h_out[1].item())

    t = torch.tensor([dev_ms, e2e_ms], dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dev_ms, e2e_ms = float(t[0]), float(t[1])
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    n = circ.n_qubits
    amps = K * B * (1 if shard else world) * ((s_end - s_begin) / plan.n_slice_terms if sample else 1)
    value = amps / (dev_ms / 1e3)
    e2e = amps / (e2e_ms / 1e3)
    ms_step = dev_ms / K
    flops = (info["grad_flops_per_amplitude"] if grad else info["flops_per_amplitude"]) * B
    algo_bytes = (info["grad_bytes_per_amplitude"] if grad else info["bytes_per_amplitude"]) * B
    hbm, bf16, peak_kind = measured_peaks()
    if records:
        roof, kernels = kernel_roofline(records, hbm, bf16)
    else:   # gradient and slice-sharded runs: the whole step against the HBM roofline
        if grad:
            kname = "grad_smem_kernel" if 0 < info["grad_smem_bytes"] <= 232448 else "grad_program_kernel"
        else:
            kname = {"fused": "fused_program_kernel", "persistent": "persistent_program_kernel"}.get(
                info["engine"], "regtile_step_kernel")
        ach = algo_bytes / (ms_step / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm, "kernel": kname,
                "algorithmic_bytes_per_launch": algo_bytes}
        kernels = None
    roof["traffic"] = NCU_TRAFFIC.get((args.workload, circuit_seed(args), roof["kernel"], info["device_image_bytes"]))
    roof["peak_source"] = peak_kind
    res = {
        "metric": METRIC, "value": value, "unit": "amplitudes/s", "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "strong" if shard else "weak",
        "vs_baseline": None, "dtype": "c64", "data": "synthetic",
        "config": run_config(args, circ, plan, world, B),
        "complex_tflops": flops / (ms_step / 1e3) / 1e12,
        "roofline": roof,
        "kernels": kernels,
        "e2e": {"value": e2e, "unit": "amplitudes/s", "h2d_bytes_per_step": 8 * B * plan.words,
                "d2h_bytes_per_step": (16 * B * world if shard else 16 * (B << plan.n_open))
                + (8 * gout.numel() if grad else 0)},
        "gpu_launches": launches,
        "clocks": clocks.summary(),
        "plan_seconds": plan_s,
        "autotune": None if tuning is None else [list(t) for t in tuning],
        "gradients_per_amplitude": info["n_params"] if grad else 0,
        "plan": {"n_vars": info["n_vars"], "n_steps": info["n_steps"], "log2_cost": info["log2_cost"],
                 "log2_cost_unsliced": info["log2_cost_unsliced"], "max_rank": info["max_rank"],
                 "arena_bytes": info["arena_bytes"], "device_image_bytes": info["device_image_bytes"],
                 "algorithmic_bytes_per_amplitude": info["bytes_per_amplitude"],
                 "algorithmic_flops_per_amplitude": info["flops_per_amplitude"]},
        "abs_err": None, "err_bound": 1e-5 * 2.0 ** (-n / 2),
    }
    if world == 1 and not grad and not sample:
        # parity of what was timed: against the oracle's whole amplitude when it finishes in
        # seconds, else (and always for the timing baseline) on seeded sampled slice terms
        from oracle import ve as VE
        x = bits_host[0]
        if info["log2_cost"] + len(plan.slices) <= 26 and not plan.n_open:
            ref = VE.exact_sum(VE.slice_terms(circ, x, plan.order, plan.slices))
            res["abs_err"] = abs(amp - ref)
            res["err_kind"] = "whole amplitude vs the oracle"
        if not args.no_cpu_baseline:
            base, ids, ref_terms = cpu_baseline(circ, x, plan.order, plan.slices, args.cpu_seconds, seed=11)
            res["cpu_baseline"] = base
            if not plan.n_open:
                sp = slice_parity(plan, x, ids, ref_terms, n, dev, ws)
                res["slice_err"] = sp
                if res["abs_err"] is None:
                    res["abs_err"] = sp["c13"]
                    res["err_kind"] = (f"sqrt(2^k) x rms |d beta| over {sp['sampled']} sampled slice terms vs the "
                                       f"oracle (random-phase estimate of |d alpha|)")
        if not args.no_fp32_forms:
            # the plain FP32 forms of the same plan (order and slices): per-slice (one slice per
            # work item, one launch per contraction, SIMT) and, for tensor-core plans, the
            # batched SIMT form with the same open slices
            forms = {}
            base_kw = dict(order=plan.order, slices=plan.slices, engine="stepwise", mem_budget_bytes=budget,
                           plan_trials=plan.plan_trials)
            variants = [("fp32_per_slice", dict(inner_slices=0))]
            if info["n_gemm_steps"]:
                variants.append(("fp32_batched_simt", dict(inner_slices=info["n_inner"])))
            for name, kw in variants:
                try:
                    p2 = q.Plan(circ, **base_kw, **kw)
                    ms = time_form(p2, bits, 3, flush, stream)
                    forms[name] = {"ms_per_amplitude": ms / B, "amplitudes/s": 1e3 * B / ms,
                                   "timed_form_speedup": ms / ms_step}
                    del p2
                except Exception as e:   # the form does not fit this device
                    forms[name] = {"error": str(e)[:200]}
            res["fp32_forms"] = forms
    elif shard:
        res["amplitude_sharded"] = [amp.real, amp.imag]
    print(json.dumps(res), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
