"""Launch-shape autotuner: picks the plan variant with the lowest measured time.

For a circuit it builds plans that differ in how many variables are sliced (more slices:
smaller tensors and more, shorter work items, but more total work), how many sliced
variables stay open inside one work item (inner slices: more sharing of work between
slices, fewer and longer items), the engine (fused shared-memory program or stepwise
global-memory launches) and, for the fused engine, how many warps share one item and how
large the leaf products contracted at plan time are. Each variant is timed through the
library's own amplitude entry point with CUDA events on the caller's stream; the tuner only
chooses among plans.
"""
from __future__ import annotations

import time

from . import Plan, bits_tensor


def _time_plan(p, bits, flush, stream, reps, warmup):
    import torch
    n = bits.numel() // p.words
    ws = p.workspace(n, bits.device)
    out = torch.empty(2 * n << p.n_open, dtype=torch.float64, device=bits.device)
    for _ in range(warmup):
        p.amplitude(bits, workspace=ws, out=out, validate=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    p.amplitude(bits, workspace=ws, out=out, validate=False)
    torch.cuda.synchronize()
    if time.perf_counter() - t0 > 0.01:    # long calls: fewer repetitions
        reps = max(3, min(reps, 5))
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for e0, e1 in evs:
        flush.zero_()
        e0.record(stream)
        p.amplitude(bits, workspace=ws, out=out, validate=False)
        e1.record(stream)
    torch.cuda.synchronize()
    del ws
    # mean of the middle half: single event intervals are quantised to about a microsecond
    ts = sorted(e0.elapsed_time(e1) for e0, e1 in evs)
    mid = ts[len(ts) // 4:len(ts) - len(ts) // 4] or ts
    return 1e3 * sum(mid) / len(mid)


def autotune(circ, bitstrings, n_slices=-1, slices=None, order=None, inner=None, warps=(1, 2, 4, 8, 16),
             merges=(8, 10), reps=20, warmup=3, budget_s=30.0, device=None, verbose=False,
             slice_counts=None, engines=("fused",), order_seeds=(), trial_counts=(), **plan_kw):
    """Returns (best_plan, results) with results = [(n_sliced, inner, engine, warps,
    host_merge_rank, us_per_call), ...]. host_merge_rank is the largest leaf product
    contracted at plan time. slice_counts (a list of k) replaces n_slices when given;
    engines lists the engines tried ("fused", "stepwise", "persistent"). order_seeds: after
    the search, the best variant is rebuilt with each of these seeds of the randomised
    ordering (another order, and the slices chosen under it; the same amplitude) and timed;
    their results carry the seed as a seventh field. trial_counts: likewise, the best variant
    is rebuilt with each of these numbers of planning trials (the planner ranks trials by an
    estimate; timing decides between the plans it keeps), carried as "plan_trials=T"."""
    import torch
    dev = torch.device(device if device is not None else "cuda")
    bits = bits_tensor(bitstrings, (circ.n_qubits + 63) // 64, dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    results, best, best_t = [], None, None
    t_start = time.perf_counter()
    ks = [n_slices] if slice_counts is None else list(slice_counts)
    for k in ks:
        base = Plan(circ, order=order, slices=slices, n_slices=k, **plan_kw)
        kk = len(base.slices)
        inners = range(0, min(kk, 7) + 1) if inner is None else [i for i in inner if i <= kk]
        variants = []
        for eng in engines:
            if eng == "fused":
                variants += [(n_in, eng, w, m) for m in merges for n_in in inners for w in warps]
            else:
                variants += [(n_in, eng, 1, merges[0]) for n_in in inners]
        for n_in, eng, w, m in variants:
            if time.perf_counter() - t_start > budget_s:
                break
            try:
                tc = eng.endswith("-tc")   # the stepwise engine with tensor-core contractions
                p = Plan(circ, order=base.order, slices=base.slices, inner_slices=n_in, warps_per_item=w,
                         host_merge_rank=m, engine=eng[:-3] if tc else eng, tensor_cores=tc, **plan_kw)
                if tc and p.info["n_gemm_steps"] == 0:
                    continue
            except Exception:      # a variant the engine cannot run (shared memory)
                continue
            us = _time_plan(p, bits, flush, stream, reps, warmup)
            results.append((kk, n_in, eng, w, m, us))
            if verbose:
                print(f"autotune: k={kk} inner={n_in} engine={eng} warps={w} merge={m} {us:.1f} us", flush=True)
            if best_t is None or us < best_t:
                best, best_t = p, us
                best_kw = dict(inner_slices=n_in, warps_per_item=w, host_merge_rank=m,
                               engine=eng[:-3] if tc else eng, tensor_cores=tc, n_slices=kk)
                best_key = (kk, n_in, eng, w, m)
            else:
                del p
    if best is not None and trial_counts and order is None and slices is None:
        # the stepwise engine's two forms are both re-timed: another plan may have dense
        # steps that the tensor cores take
        kw = {k: v for k, v in plan_kw.items() if k != "plan_trials"}
        forms = [best_key[2]]
        if best_key[2] in ("stepwise", "stepwise-tc"):
            forms += [e for e in ("stepwise", "stepwise-tc") if e in engines and e != best_key[2]]
        for tr in trial_counts:
            if tr == plan_kw.get("plan_trials", 1) or time.perf_counter() - t_start > budget_s + 30.0:
                continue
            picked = {}   # the trials' order and slices, planned once per trial count
            for eng in forms:
                tc = eng.endswith("-tc")
                try:
                    p = Plan(circ, plan_trials=tr, **picked,
                             **dict(best_kw, engine=eng[:-3] if tc else eng, tensor_cores=tc), **kw)
                    picked = dict(order=p.order, slices=p.slices)
                    if tc and p.info["n_gemm_steps"] == 0:
                        continue
                except Exception:
                    continue
                us = _time_plan(p, bits, flush, stream, reps, warmup)
                results.append(best_key[:2] + (eng,) + best_key[3:] + (us, f"plan_trials={tr}"))
                if us < best_t:
                    best, best_t = p, us
                else:
                    del p
    if best is not None and order_seeds and order is None and slices is None:
        for seed in order_seeds:
            if time.perf_counter() - t_start > budget_s + 30.0:
                break
            try:
                p = Plan(circ, order_seed=seed, **best_kw, **plan_kw)
            except Exception:
                continue
            us = _time_plan(p, bits, flush, stream, reps, warmup)
            results.append(best_key + (us, seed))
            if us < best_t:
                best, best_t = p, us
            else:
                del p
    return best, results
