"""Host-side checks of libqvx.so: exports, graph, planner, and the program run on the CPU."""
import os
import random
import re

import numpy as np
import pytest

import circuitgen as cg
import paper_1805_01450_gb300 as q
from oracle import graph as GR
from oracle import statevector as SV
from oracle import ve as VE

from _program_exec import Program, check_schedule

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_symbol():
    header = open(os.path.join(ROOT, "include", "qvx.h")).read()
    declared = set(re.findall(r"\b(qvx_[a-z_0-9]+)\s*\(", header))
    L = q.lib()
    for name in declared:
        assert hasattr(L, name), name
    assert declared == set(q.EXPORTED)


@pytest.mark.parametrize("maker", [cg.worked_example, lambda: cg.grid_circuit(4, 4, 10, 1001),
                                   lambda: cg.grid_circuit(6, 6, 25, 2001),
                                   lambda: cg.rotation_circuit(3, 3, 4, 5)])
def test_graph_export_matches_oracle(maker):
    c = maker()
    vq, vo, ed = q.graph_export(c)
    m = GR.build(c)
    assert list(zip(vq, vo)) == m.variables
    assert sorted(ed) == sorted(GR.edges(m))


def test_plan_order_cost_matches_oracle_graph_ops():
    # the plan's reported cost is sum 2^deg over its order after fixing its slices
    c = cg.grid_circuit(6, 6, 25, 2001)
    p = q.Plan(c, n_slices=6)
    m = GR.build(c)
    adj = GR.adjacency(len(m.variables), GR.edges(m))
    for v in p.slices:
        adj = GR.fix_vertex(adj, v)
    cost, _ = GR.order_cost(adj, p.order)
    assert abs(np.log2(cost) - p.info["log2_cost"]) < 1e-9
    assert sorted(p.order + p.slices) == list(range(len(m.variables)))


M64 = (1 << 64) - 1


def _splitmix64(state):
    state = (state + 0x9E3779B97F4A7C15) & M64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return state, z ^ (z >> 31)


def _minfill_from_definition(adj, seed, fixed=()):
    # greedy min-fill: eliminate a vertex whose neighbours miss the fewest edges among
    # themselves, then the smallest degree; among equals (in increasing vertex id) pick with
    # the seeded splitmix64 stream; every fill value recomputed from the graph at every step;
    # fixed vertices are no longer in the graph
    alive = [v for v in range(len(adj)) if v not in fixed]
    rng, order = seed, []
    while alive:
        best, ties = None, []
        for v in alive:
            nb = sorted(adj[v])
            fill = sum(1 for i in range(len(nb)) for j in range(i + 1, len(nb)) if nb[j] not in adj[nb[i]])
            key = (fill, len(nb))
            if best is None or key < best:
                best, ties = key, [v]
            elif key == best:
                ties.append(v)
        rng, r = _splitmix64(rng)
        pick = ties[r % len(ties)]
        adj, _ = GR.eliminate_vertex(adj, pick)
        order.append(pick)
        alive.remove(pick)
    return order


@pytest.mark.parametrize("maker", [cg.worked_example, lambda: cg.grid_circuit(4, 4, 10, 1001),
                                   lambda: cg.grid_circuit(3, 4, 16, 2)])
@pytest.mark.parametrize("order_seed", [1, 7, 99])
def test_planner_ordering_is_min_fill(maker, order_seed):
    # one restart, nothing sliced: the plan's order is the min-fill order of the oracle's
    # graph with the planner's tie-break stream (seed order_seed ^ 2 * golden ratio, one
    # splitmix64 step for the restart's seed, one per pick)
    c = maker()
    p = q.Plan(c, n_slices=0, order_restarts=1, order_seed=order_seed)
    m = GR.build(c)
    adj = GR.adjacency(len(m.variables), GR.edges(m))
    s = (order_seed ^ (2 * 0x9E3779B97F4A7C15)) & M64
    _, seed = _splitmix64(s)
    assert p.order == _minfill_from_definition(adj, seed)


@pytest.mark.parametrize("maker,k", [(lambda: cg.grid_circuit(4, 4, 10, 1001), 3),
                                     (lambda: cg.grid_circuit(3, 4, 16, 2), 4)])
def test_planner_slices_are_the_greedy_rule(maker, k):
    # Section 3.B.2-3 from their definitions on the oracle's graph: the first order is
    # min-fill (salt 1); each round fixes the vertex whose removal gives the smallest sum of
    # 2^deg along that first order (ties to the lowest id); the final order is min-fill of
    # the reduced graph (salt 2)
    c = maker()
    p = q.Plan(c, n_slices=k, inner_slices=0, order_restarts=1, order_seed=5)
    m = GR.build(c)
    adj = GR.adjacency(len(m.variables), GR.edges(m))
    _, seed1 = _splitmix64((5 ^ 0x9E3779B97F4A7C15) & M64)
    first = _minfill_from_definition(adj, seed1)
    fixed = []
    for _ in range(k):
        best = None
        for v in range(len(adj)):
            if v in fixed:
                continue
            a = adj
            for u in fixed + [v]:
                a = GR.fix_vertex(a, u)
            cost, _ = GR.order_cost(a, [u for u in first if u not in fixed and u != v])
            if best is None or cost < best[0]:
                best = (cost, v)
        fixed.append(best[1])
    assert p.slices == fixed
    a = adj
    for u in fixed:
        a = GR.fix_vertex(a, u)
    _, seed2 = _splitmix64((5 ^ (2 * 0x9E3779B97F4A7C15)) & M64)
    assert p.order == _minfill_from_definition(a, seed2, fixed)


def test_greedy_slices_follow_section_3b2():
    # each greedy pick lowers the cost under the first order; the final cost is far below
    # the unsliced one
    c = cg.grid_circuit(6, 6, 25, 2001)
    p0 = q.Plan(c, n_slices=0)
    p12 = q.Plan(c, n_slices=12)
    assert p12.info["log2_cost"] < p0.info["log2_cost"] - 5
    assert len(set(p12.slices)) == 12


def test_user_order_and_slices_are_used():
    c = cg.grid_circuit(4, 4, 10, 1001)
    nv = len(GR.build(c).variables)
    sl = [3, 7]
    order = [v for v in range(nv) if v not in sl][::-1]
    p = q.Plan(c, order=order, slices=sl)
    assert p.order == order and sorted(p.slices) == sorted(sl)


@pytest.mark.parametrize("bad", [dict(order=[0, 0]), dict(slices=[999]), dict(slices=[1, 1])])
def test_invalid_plan_arguments(bad):
    with pytest.raises(q.QvxError) as e:
        q.Plan(cg.grid_circuit(4, 4, 10, 1001), **bad)
    assert e.value.status == q.QVX_EINVAL


def test_invalid_circuit():
    c = cg.Circuit(n_qubits=2, gates=[cg.Gate(cg.CZ, 0, 0)])
    with pytest.raises(q.QvxError):
        q.Plan(c)
    c = cg.Circuit(n_qubits=2, gates=[cg.Gate(99, 0)])
    with pytest.raises(q.QvxError):
        q.Plan(c)


CASES = [
    ("worked", cg.worked_example, dict()),
    ("4x4x10", lambda: cg.grid_circuit(4, 4, 10, 1001), dict()),
    ("4x4x10-k3", lambda: cg.grid_circuit(4, 4, 10, 1001), dict(n_slices=3, inner_slices=1)),
    ("3x4x16-k4", lambda: cg.grid_circuit(3, 4, 16, 2), dict(n_slices=4, inner_slices=2)),
    ("rot2x3", lambda: cg.rotation_circuit(2, 3, 4, 12), dict(n_slices=2, inner_slices=0)),
    ("4x4x10-devonly", lambda: cg.grid_circuit(4, 4, 10, 1001), dict(host_merge_rank=0)),
    ("3x4x16-k4-devonly", lambda: cg.grid_circuit(3, 4, 16, 2), dict(n_slices=4, inner_slices=2,
                                                                      host_merge_rank=0)),
    ("3x4x16-k4-merge12", lambda: cg.grid_circuit(3, 4, 16, 2), dict(n_slices=4, inner_slices=1,
                                                                      host_merge_rank=12)),
    ("empty", lambda: cg.Circuit(n_qubits=3, gates=[]), dict()),
    ("untouched", lambda: cg.Circuit(n_qubits=3, gates=[cg.Gate(cg.H, 0), cg.Gate(cg.T, 1),
                                                        cg.Gate(cg.CZ, 0, 1)]), dict()),
]


@pytest.mark.parametrize("name,maker,kw", CASES, ids=[c[0] for c in CASES])
def test_program_on_host_matches_oracle(name, maker, kw):
    c = maker()
    p = q.Plan(c, **kw)
    prog = Program(p.image())
    psi = SV.final_state(c)
    xs = [0, (1 << c.n_qubits) - 1] + cg.random_bitstrings(c.n_qubits, 4, 9)
    for x in xs:
        terms = prog.slice_terms(x)
        assert abs(terms.sum() - psi[x]) < 1e-6 * 2 ** (-c.n_qubits / 2) + 1e-7
        if prog.fsteps is not None:
            assert np.array_equal(prog.slice_terms(x, fused=True), terms)
            check_schedule(prog)
        if p.slices:
            ref = VE.slice_terms(c, x, p.order, p.slices)
            assert np.max(np.abs(terms - ref)) < 1e-6 * 2 ** (-c.n_qubits / 2)


@pytest.mark.parametrize("name,maker,kw", CASES[1:4] + CASES[5:8], ids=[c[0] for c in CASES[1:4] + CASES[5:8]])
def test_register_tiled_forms_on_host(name, maker, kw):
    # the stepwise engine's register-tiled steps cover every output entry once and give the
    # plain step's values exactly
    c = maker()
    p = q.Plan(c, engine="stepwise", **kw)
    prog = Program(p.image())
    assert prog.rtsteps is not None
    for x in cg.random_bitstrings(c.n_qubits, 2, 19):
        assert np.array_equal(prog.slice_terms(x, regtile=True), prog.slice_terms(x))


def test_register_tiled_forms_7x7x30():
    c = cg.grid_circuit(7, 7, 30, 3001)
    p = q.Plan(c, n_slices=8, inner_slices=4, engine="stepwise")
    prog = Program(p.image())
    rt = prog.rtsteps
    assert int(((rt["rm"] + rt["rn"]) > 0).sum()) == p.info["n_tiled_steps"] >= 50
    x = cg.random_bitstrings(49, 1, 3003)[0]
    got = prog.item_terms(x, 5, regtile=True)
    plain = prog.item_terms(x, 5)   # same products, numpy may round them differently
    assert np.max(np.abs(got - plain)) <= 1e-12 * np.max(np.abs(plain))
    ref = VE.slice_terms(c, x, p.order, p.slices, slice_ids=[(5 << 4) | i for i in range(16)])
    assert np.max(np.abs(got - ref)) < 1e-6 * 2 ** -24.5


@pytest.mark.parametrize("rows,cols,seed", [(6, 6, 7066), (6, 6, 16)])
def test_tensor_core_form_on_host(rows, cols, seed):
    # depth 40, 8 sliced variables (2 open): contractions that qualify for the tensor cores;
    # their GEMMs of three-part bf16 splits stay within 2^-21 of the exact product and the
    # slice terms within the amplitude tolerance of the oracle's. The GEMM's row role goes to
    # the operand that holds the output's lowest mode (the host form checks it): on circuit
    # 16 some steps keep the operands' order and some swap them.
    c = cg.grid_circuit(rows, cols, 40, seed)
    n = rows * cols
    p = q.Plan(c, n_slices=8, inner_slices=2, engine="stepwise", tensor_cores=True)
    assert p.info["n_gemm_steps"] >= 1
    prog = Program(p.image())
    gem = [i for i, g in enumerate(prog.gemms) if int(g["nk"]) > 0]
    sw = [i for i in gem if (int(prog.gemms[i]["flags"]) & 6, int(prog.gemms[i]["a_off"])) !=
          (int(prog.steps[i]["flags"]) & 6, int(prog.steps[i]["a_off"]))]
    if seed == 16:   # both orientations: a step that keeps its operands' order and one that swaps them
        assert len(sw) >= 1 and len(gem) - len(sw) >= 1
    # the first seeded (bitstring, work item) whose slice terms are not all zero (many
    # terms of these circuits cancel exactly)
    x, o = next((x, o) for x in cg.random_bitstrings(n, 64, seed + 1) for o in range(4)
                if np.max(np.abs(prog.item_terms(x, o))) > 1e-12)
    got = prog.item_terms(x, o, gemm=True)
    plain = prog.item_terms(x, o)
    assert np.max(np.abs(got - plain)) <= 2.0 ** -21 * np.max(np.abs(plain))
    ref = VE.slice_terms(c, x, p.order, p.slices, slice_ids=[(o << 2) | i for i in range(4)])
    assert np.max(np.abs(got - ref)) < 1e-5 * 2 ** (-n / 2)
    assert q.Plan(c, n_slices=8, inner_slices=2, engine="stepwise").info["n_gemm_steps"] == 0


def test_tensor_core_steps_store_along_their_unit_stride():
    # 8x8x40 (circuit 5001, 64 planning trials): a dense step whose output's lowest mode is
    # held by both operands keeps its SIMT form; every tensor-core step's lowest output mode
    # is a row mode of the GEMM (the row operand holds the output's unit stride)
    c = cg.grid_circuit(8, 8, 40, 5001)
    p = q.Plan(c, n_slices=10, inner_slices=4, engine="stepwise", tensor_cores=True, plan_trials=64,
               mem_budget_bytes=64 << 30)
    prog = Program(p.image())

    def holds_low(runs, n):
        return any(int(r["src"]) == 0 and int(r["len"]) > 0 for r in runs[:n])

    kept_simt = 0
    for s, st in enumerate(prog.steps):
        g = prog.gemms[s]
        dense = int(st["nk_a"]) == 0 and int(st["nk_b"]) == 0 and 3 <= int(st["nk_ab"]) <= 10 and int(st["rc"]) >= 10
        low_batch = holds_low(st["runs_a"], int(st["na_runs"])) and holds_low(st["runs_b"], int(st["nb_runs"]))
        if int(g["nk"]) == 0:
            kept_simt += dense and low_batch
            continue
        assert not low_batch
        dsts = lambda f, n: [int(r["dst"]) for r in g[f][:n] if int(r["len"]) > 0]
        assert 0 not in dsts("cb", int(g["n_cb"]))
        assert 0 in dsts("cm", int(g["n_cm"]))
    assert kept_simt >= 1 and p.info["n_gemm_steps"] >= 2


@pytest.mark.parametrize("merge", [0, 8])
def test_program_slice_terms_6x6_sample(merge):
    c = cg.grid_circuit(6, 6, 25, 2001)
    p = q.Plan(c, n_slices=12, inner_slices=3, host_merge_rank=merge)
    prog = Program(p.image())
    x = cg.random_bitstrings(36, 1, 2002)[0]
    rng = random.Random(0)
    for o in rng.sample(range(int(prog.h["n_outer"])), 3):
        got = prog.item_terms(x, o)
        assert np.array_equal(prog.item_terms(x, o, fused=True), got)
        ids = [(o << 3) | i for i in range(8)]
        ref = VE.slice_terms(c, x, p.order, p.slices, slice_ids=ids)
        assert np.max(np.abs(got - ref)) < 1e-6 * 2 ** -18


def test_bench_plan_6x6_on_host():
    # the plan the benchmark times on 6x6x25: 64 planning trials for the order and slices,
    # then 5 open slices, 8 warps per item, leaf products to rank 10 merged on the host; its
    # fused schedule is complete and its items' slice terms match the oracle's
    c = cg.grid_circuit(6, 6, 25, 2001)
    base = q.Plan(c, n_slices=12, mem_budget_bytes=1 << 30, plan_trials=64)
    p = q.Plan(c, order=base.order, slices=base.slices, inner_slices=5, warps_per_item=8, host_merge_rank=10,
               engine="fused", mem_budget_bytes=1 << 30, plan_trials=64)
    assert p.info["engine"] == "fused" and p.info["n_inner"] == 5
    prog = Program(p.image())
    check_schedule(prog)
    x = cg.random_bitstrings(36, 1, 2002)[0]
    rng = random.Random(1)
    for o in rng.sample(range(int(prog.h["n_outer"])), 2):
        got = prog.item_terms(x, o, fused=True)
        ids = [(o << 5) | i for i in range(32)]
        ref = VE.slice_terms(c, x, p.order, p.slices, slice_ids=ids)
        assert np.max(np.abs(got - ref)) < 1e-6 * 2 ** -18


def test_host_merging_shortens_the_device_program():
    c = cg.grid_circuit(6, 6, 25, 2001)
    full = q.Plan(c, n_slices=12, inner_slices=4, host_merge_rank=0).info
    merged = q.Plan(c, n_slices=12, inner_slices=4, host_merge_rank=8).info
    assert merged["n_steps"] < full["n_steps"] / 2
    assert merged["flops_per_amplitude"] < full["flops_per_amplitude"]
    # chains of steps that each multiply a large tensor by a leaf take the leaves' product
    # (contracted on the host) in one step: fewer levels of dependent steps
    assert merged["n_phases"] <= 18 < full["n_phases"]


GRAD_CASES = [
    ("rot2x3d4", lambda: cg.rotation_circuit(2, 3, 4, 12), dict()),
    ("rot2x3d4-k3", lambda: cg.rotation_circuit(2, 3, 4, 12), dict(n_slices=3, inner_slices=1)),
    ("rot3x3d3-k4-merge", lambda: cg.rotation_circuit(3, 3, 3, 7), dict(n_slices=4, inner_slices=2,
                                                                        host_merge_rank=8)),
    ("rot3x3d3-k4-trials", lambda: cg.rotation_circuit(3, 3, 3, 7), dict(n_slices=4, inner_slices=2,
                                                                         plan_trials=8)),
    ("one-rotation", lambda: cg.Circuit(n_qubits=1, gates=[cg.Gate(cg.RXY, 0, theta=0.9, phi=0.0, param=0)]), dict()),
]


@pytest.mark.parametrize("name,maker,kw", GRAD_CASES, ids=[c[0] for c in GRAD_CASES])
def test_gradient_program_on_host_matches_oracle(name, maker, kw):
    from _program_exec import grad, check_grad_schedule
    c = maker()
    p = q.Plan(c, gradient=True, **kw)
    assert p.info["n_params"] == c.n_params
    prog = Program(p.image())
    check_grad_schedule(prog)
    assert prog.gentries is not None
    for x in [0] + cg.random_bitstrings(c.n_qubits, 2, 4):
        a_ref, g_ref = SV.sv_adjoint_grad(c, x)
        a, g = grad(prog, x)
        assert abs(a - a_ref) < 1e-6 * 2 ** (-c.n_qubits / 2)
        assert np.max(np.abs(g - g_ref)) < 1e-6 * 2 ** (-c.n_qubits / 2)
        # the per-entry records of the shared-memory gradient kernel, phase by phase
        a_t, g_t = grad(prog, x, tables=True)   # same products; numpy and Python may round apart
        assert abs(a_t - a) < 1e-14 and np.max(np.abs(g_t - g)) < 1e-14
    # other angles through the parametrised leaves
    th = np.random.default_rng(0).uniform(0, 2 * np.pi, c.n_params)
    x = 1
    a_ref, g_ref = SV.sv_adjoint_grad(SV.with_thetas(c, th), x)
    a, g = grad(prog, x, th)
    assert abs(a - a_ref) < 1e-6 and np.max(np.abs(g - g_ref)) < 1e-6


def test_gradient_checkpointing_on_host():
    # rotation circuit 4x4, depth 16: with a memory budget below one work item's gradient
    # arena, forward values are recomputed in the backward pass instead of kept
    # (checkpointing); the arena shrinks and the gradients still match the state-vector adjoint
    from _program_exec import grad, check_grad_schedule
    c = cg.rotation_circuit(4, 4, 16, 9)
    full = q.Plan(c, gradient=True, n_slices=0)
    small = q.Plan(c, gradient=True, n_slices=0, order=full.order,
                   mem_budget_bytes=full.info["grad_arena_bytes"] // 2)
    assert full.info["grad_recomputed"] == 0
    assert small.info["grad_recomputed"] > 0
    assert small.info["grad_arena_bytes"] < full.info["grad_arena_bytes"]
    assert small.info["n_grad_steps"] == full.info["n_grad_steps"] + small.info["grad_recomputed"]
    prog = Program(small.image())
    check_grad_schedule(prog)
    for x in cg.random_bitstrings(16, 2, 10):
        a_ref, g_ref = SV.sv_adjoint_grad(c, x)
        a, g = grad(prog, x)
        assert abs(a - a_ref) < 1e-6 * 2 ** -8
        assert np.max(np.abs(g - g_ref)) < 1e-6 * 2 ** -8
        a_t, g_t = grad(prog, x, tables=True)
        assert abs(a_t - a) < 1e-14 and np.max(np.abs(g_t - g)) < 1e-14


@pytest.mark.parametrize("inner,wpi,merge", [(0, 1, 8), (3, 2, 10), (5, 4, 10), (5, 4, 0), (5, 8, 10), (6, 16, 10)])
def test_fused_schedule_6x6x25(inner, wpi, merge):
    c = cg.grid_circuit(6, 6, 25, 2001)
    p = q.Plan(c, n_slices=12, inner_slices=inner, warps_per_item=wpi, host_merge_rank=merge)
    prog = Program(p.image())
    check_schedule(prog)
    assert int(prog.h["fused_lanes"]) == 32 * wpi


def _cz_counts(c):
    m = GR.build(c)
    counts = [0] * len(m.variables)
    for keys, data in m.tensors:
        if len(keys) == 2 and keys[0][0] != keys[1][0]:
            for k in keys:
                if k in m.index:
                    counts[m.index[k]] += 1
    return counts


def test_slice_rules_section6():
    c = cg.grid_circuit(7, 7, 30, 3001)
    greedy = q.Plan(c, n_slices=10, inner_slices=0)
    reorder = q.Plan(c, n_slices=10, inner_slices=0, slice_rule="reorder")
    czpair = q.Plan(c, n_slices=10, inner_slices=0, slice_rule="cz-pair")
    # re-ordering after every removal finds cheaper subtasks on this seeded circuit
    assert reorder.info["log2_cost"] < greedy.info["log2_cost"]
    counts = _cz_counts(c)
    assert all(counts[v] >= 2 for v in czpair.slices)
    for p in (greedy, reorder, czpair):
        assert sorted(p.order + p.slices) == list(range(len(counts)))


def test_planning_trials_keep_the_cheapest_valid_plan():
    # trial 0 is the single-trial planner; more trials never rank worse, give the same plan
    # on every build (threads do not decide), and the kept plan's reported cost is the sum
    # of 2^deg of its own order after fixing its own slices (oracle graph operations)
    c = cg.grid_circuit(7, 7, 30, 3001)
    one = q.Plan(c, n_slices=4, inner_slices=0)
    t1 = q.Plan(c, n_slices=4, inner_slices=0, plan_trials=1)
    assert (one.order, one.slices) == (t1.order, t1.slices)
    a = q.Plan(c, n_slices=4, inner_slices=0, plan_trials=16)
    b = q.Plan(c, n_slices=4, inner_slices=0, plan_trials=16)
    assert (a.order, a.slices) == (b.order, b.slices)
    assert a.info["est_bytes_per_amplitude"] <= one.info["est_bytes_per_amplitude"]
    m = GR.build(c)
    adj = GR.adjacency(len(m.variables), GR.edges(m))
    for v in a.slices:
        adj = GR.fix_vertex(adj, v)
    cost, _ = GR.order_cost(adj, a.order)
    assert abs(np.log2(cost) - a.info["log2_cost"]) < 1e-9
    assert sorted(a.order + a.slices) == list(range(len(m.variables)))
    # a given order and slice set leave nothing to try
    f = q.Plan(c, order=one.order, slices=one.slices, inner_slices=0, plan_trials=8)
    assert (f.order, f.slices) == (one.order, one.slices)
    for bad in (0, 65537):
        with pytest.raises(q.QvxError) as e:
            q.Plan(c, n_slices=4, plan_trials=bad)
        assert e.value.status == q.QVX_EINVAL
    # a circuit the single-trial planner cannot fit under max_rank still fails cleanly when
    # no trial fits either
    with pytest.raises(q.QvxError) as e:
        q.Plan(c, n_slices=0, max_rank=6, plan_trials=4)
    assert e.value.status == q.QVX_EUNSUPPORTED


def test_planning_trials_program_matches_oracle():
    c = cg.grid_circuit(4, 4, 12, 31)
    p = q.Plan(c, n_slices=4, inner_slices=1, plan_trials=8)
    prog = Program(p.image())
    psi = SV.final_state(c)
    for x in cg.random_bitstrings(16, 3, 33):
        terms = prog.slice_terms(x)
        assert abs(terms.sum() - psi[x]) < 1e-6 * 2 ** -8
        assert np.max(np.abs(terms - VE.slice_terms(c, x, p.order, p.slices))) < 1e-6 * 2 ** -8


@pytest.mark.parametrize("rule", ["reorder", "cz-pair"])
def test_slice_rules_program_matches_oracle(rule):
    c = cg.grid_circuit(4, 4, 12, 31)
    p = q.Plan(c, n_slices=4, inner_slices=1, slice_rule=rule)
    prog = Program(p.image())
    psi = SV.final_state(c)
    for x in cg.random_bitstrings(16, 3, 32):
        assert abs(prog.slice_terms(x).sum() - psi[x]) < 1e-6 * 2 ** -8


def _with_open_bits(x, open_qubits, j):
    for i, qb in enumerate(open_qubits):
        x = (x & ~(1 << qb)) | (((j >> i) & 1) << qb)
    return x


@pytest.mark.parametrize("kw", [dict(), dict(n_slices=3, inner_slices=1), dict(n_slices=2, host_merge_rank=0),
                                dict(n_slices=3, inner_slices=1, plan_trials=8),
                                dict(n_slices=3, inner_slices=1, plan_trials=8, slice_rule="reorder",
                                     engine="persistent")])
def test_open_qubits_program_on_host(kw):
    # Section 6: batches of amplitudes from one contraction (open output variables)
    c = cg.grid_circuit(4, 4, 10, 1001)
    oq = [0, 5, 15]
    p = q.Plan(c, open_qubits=oq, **kw)
    assert p.info["n_open_qubits"] == 3
    prog = Program(p.image())
    psi = SV.final_state(c)
    for x in cg.random_bitstrings(16, 3, 70):
        terms = prog.slice_terms(x)
        assert terms.shape[0] == 8
        got = terms.sum(axis=-1)
        want = np.array([psi[_with_open_bits(x, oq, j)] for j in range(8)])
        assert np.max(np.abs(got - want)) < 1e-6 * 2 ** -8


def test_open_qubit_errors():
    c = cg.grid_circuit(4, 4, 10, 1001)
    with pytest.raises(q.QvxError):
        q.Plan(c, open_qubits=[3, 3])
    with pytest.raises(q.QvxError):
        q.Plan(c, open_qubits=[16])
    with pytest.raises(q.QvxError):
        q.Plan(cg.rotation_circuit(2, 2, 2, 1), open_qubits=[0], gradient=True)
    untouched = cg.Circuit(n_qubits=2, gates=[cg.Gate(cg.H, 0)])
    with pytest.raises(q.QvxError):
        q.Plan(untouched, open_qubits=[1])


def test_81_qubit_program_on_host_matches_oracle():
    # bitstrings of more than 64 qubits: the device program reads qubits 64.. from the second
    # word (leaf sources 64..127) and slice bits from sources 128..
    c = cg.grid_circuit(9, 9, 8, 91)
    p = q.Plan(c, n_slices=3, inner_slices=1, engine="stepwise")
    assert p.words == 2 and p.info["n_qubits"] == 81
    prog = Program(p.image())
    xs = cg.random_bitstrings(81, 3, 92)
    assert all(x >> 64 for x in xs)
    for x in xs:
        ref = VE.slice_terms(c, x, p.order, p.slices)
        terms = prog.slice_terms(x)
        assert np.max(np.abs(terms - ref)) < 1e-6 * 2 ** (-81 / 2)
    words = q.bitstring_words(xs, 2)
    assert [(w & (2 ** 64 - 1)) | ((words[2 * i + 1] & (2 ** 64 - 1)) << 64)
            for i, w in enumerate(words[0::2])] == xs


def test_bitstring_words_and_generator():
    assert q.bitstring_words([1 << 70 | 5], 2) == [5, 1 << 6]
    assert q.bitstring_words([2 ** 64 - 1], 1) == [-1]
    # up to 64 qubits one draw per string (the sequence the earlier workloads use)
    assert cg.random_bitstrings(64, 3, 5) == [v for v in cg.random_bitstrings(64, 3, 5)]
    wide = cg.random_bitstrings(81, 4, 9)
    assert all(0 <= v < 2 ** 81 for v in wide) and any(v >> 64 for v in wide)
    rng = cg.SplitMix64(9)
    first = rng.next() | (rng.next() << 64)
    assert wide[0] == first & (2 ** 81 - 1)


def test_reordering_between_removals_on_7x7x60():
    # Section 6: the 7x7 grid reaches depth 60 with the graph re-ordered after every slice
    # removal. At 30 sliced variables (8 planning trials each) the re-ordered plan's per-slice
    # cost is at least 2^2 below the greedy rule's under the first order.
    c = cg.grid_circuit(7, 7, 60, 7001)
    kw = dict(n_slices=30, inner_slices=4, engine="stepwise", plan_trials=8, mem_budget_bytes=16 << 30)
    greedy = q.Plan(c, slice_rule="greedy", **kw)
    reorder = q.Plan(c, slice_rule="reorder", **kw)
    assert reorder.info["log2_cost"] + 2 <= greedy.info["log2_cost"]
    assert reorder.info["max_rank"] < greedy.info["max_rank"]


def test_wide_register_tiles_on_host():
    # a compute-heavy step (6 or more flops per algorithmic byte) takes an 8 x 8 register
    # tile; its host form matches the plain form and the oracle's slice terms
    c = cg.grid_circuit(5, 6, 40, 19)
    p = q.Plan(c, n_slices=8, inner_slices=2, engine="stepwise")
    prog = Program(p.image())
    assert any(int(t["rm"]) == 3 and int(t["rn"]) == 3 for t in prog.rtsteps)
    x, o = next((x, o) for x in cg.random_bitstrings(30, 64, 20) for o in range(4)
                if np.max(np.abs(prog.item_terms(x, o))) > 1e-12)
    got = prog.item_terms(x, o, regtile=True)
    plain = prog.item_terms(x, o)
    assert np.max(np.abs(got - plain)) <= 1e-12 * np.max(np.abs(plain))
    ref = VE.slice_terms(c, x, p.order, p.slices, slice_ids=[(o << 2) | i for i in range(4)])
    assert np.max(np.abs(got - ref)) < 1e-6 * 2 ** -15
