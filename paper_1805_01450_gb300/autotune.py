"""Launch-shape autotuner: picks the plan variant with the lowest measured time.

For a circuit and a slice count it builds plans that differ in how many sliced variables
stay open inside one work item (inner slices: more sharing of work between slices, fewer
and longer items) and in how many warps share one item, times each through the library
with CUDA events on the caller's stream, and returns the fastest. Every timed call is the
library's own amplitude entry point; the tuner only chooses among plans.
"""
from __future__ import annotations

import time

from . import Plan


def autotune(circ, bitstrings, n_slices=-1, slices=None, order=None, inner=None, warps=(1, 2, 4, 8, 16),
             merges=(8, 10), reps=20, warmup=3, budget_s=30.0, device=None, verbose=False, **plan_kw):
    """Returns (best_plan, results) with results = [(inner, warps, host_merge_rank,
    us_per_call), ...]. host_merge_rank is the largest leaf product contracted at plan time."""
    import torch
    dev = torch.device(device if device is not None else "cuda")
    base = Plan(circ, order=order, slices=slices, n_slices=n_slices, **plan_kw)
    k = len(base.slices)
    if inner is None:
        inner = range(0, min(k, 7) + 1)
    order, slices = base.order, base.slices
    bits = Plan._bits(bitstrings, dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    results, best, best_t = [], None, None
    t_start = time.perf_counter()
    for n_in, w, m in [(n_in, w, m) for m in merges for n_in in inner for w in warps]:
        if time.perf_counter() - t_start > budget_s:
            break
        try:
            p = Plan(circ, order=order, slices=slices, inner_slices=n_in, warps_per_item=w,
                     host_merge_rank=m, **plan_kw)
        except Exception:      # a variant the engine cannot run (shared memory)
            continue
        if p.info["engine"] != "fused" and w != warps[0]:
            continue
        ws = p.workspace(bits.numel(), dev)
        out = torch.empty(2 * bits.numel(), dtype=torch.float64, device=dev)
        for _ in range(warmup):
            p.amplitude(bits, workspace=ws, out=out, validate=False)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for e0, e1 in evs:
            flush.zero_()
            e0.record(stream)
            p.amplitude(bits, workspace=ws, out=out, validate=False)
            e1.record(stream)
        torch.cuda.synchronize()
        us = 1e3 * sorted(e0.elapsed_time(e1) for e0, e1 in evs)[reps // 2]
        results.append((n_in, w, m, us))
        if verbose:
            print(f"autotune: inner={n_in} warps={w} merge={m} {us:.1f} us", flush=True)
        if best_t is None or us < best_t:
            best, best_t = p, us
    return best, results
