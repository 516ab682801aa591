"""Recorded orderings (bench.py --record-ordering): the planner's winning trial is stored as
its elimination order and sliced variables, and the plan rebuilt from them is the planner's
plan, byte for byte (device image), so timing the recorded ordering times the planned
contraction. Also checks the committed headline ordering against the workload it names."""
import argparse
import json
import os

import pytest

import bench

q = pytest.importorskip("paper_1805_01450_gb300")


def test_recorded_ordering_rebuilds_the_planned_program(tmp_path, monkeypatch):
    key = ("grid6x6d25-k12", 2001)
    variant = dict(n_slices=6, inner_slices=2, engine="stepwise", tensor_cores=True, plan_trials=6, ordering=True)
    monkeypatch.setattr(bench, "ORDERINGS", str(tmp_path))
    monkeypatch.setitem(bench.RECORDED_PLANS, key, variant)
    args = argparse.Namespace(workload=key[0], circuit_seed=None, plan_trials=None, mem_budget_mb=256,
                              record_trial=None, selected_by="")
    bench.record_ordering(args)
    path = bench.ordering_path(*key)
    with open(path) as f:
        rec = json.load(f)
    assert rec["variant"]["plan_trials"] == 6 and rec["circuit_seed"] == 2001
    circ = bench.workload(key[0], None, 0, None)[0]
    planned = q.Plan(circ, mem_budget_bytes=256 << 20, n_slices=6, inner_slices=2, engine="stepwise",
                     tensor_cores=True, plan_trials=6)
    kw, trials, source = bench.recorded_plan_kwargs(*key)
    assert trials == 6 and source.startswith("recorded") and "plan_trials" not in kw
    rebuilt = q.Plan(circ, mem_budget_bytes=256 << 20, **kw)
    assert rebuilt.order == planned.order and rebuilt.slices == planned.slices
    assert rebuilt.image() == planned.image()
    # a chosen trial instead of the estimate's first: trial 3's own seed, one trial
    args.record_trial, args.selected_by = 3, "chosen by timing"
    bench.record_ordering(args)
    kw, trials, source = bench.recorded_plan_kwargs(*key)
    assert trials == 6 and "trial 3 of 6" in source
    third = q.Plan(circ, mem_budget_bytes=256 << 20, n_slices=6, inner_slices=2, engine="stepwise",
                   tensor_cores=True, plan_trials=1, order_seed=(1 + 3 * bench.TRIAL_SEED_STEP) % (1 << 64))
    assert q.Plan(circ, mem_budget_bytes=256 << 20, **kw).image() == third.image()
    # without the file the variant plans in the run
    os.remove(path)
    kw, _, source = bench.recorded_plan_kwargs(*key)
    assert source == "planned in this run" and kw["plan_trials"] == 6 and "order" not in kw


def test_committed_headline_ordering_matches_its_workload():
    for (name, seed), variant in bench.RECORDED_PLANS.items():
        if not variant.get("ordering"):
            continue
        with open(bench.ordering_path(name, seed)) as f:
            rec = json.load(f)
        assert rec["workload"] == name and rec["circuit_seed"] == seed
        assert rec["variant"]["plan_trials"] == variant["plan_trials"]
        assert rec["variant"]["n_slices"] == len(rec["slices"]) == variant["n_slices"]
        circ = bench.workload(name, None, 0, seed)[0]
        # the order eliminates every path variable of the circuit that is not sliced
        n_vars = len(q.graph_export(circ)[0])
        assert sorted(rec["order"] + rec["slices"]) == list(range(n_vars))
