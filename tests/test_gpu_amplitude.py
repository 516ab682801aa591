"""GPU parity: amplitudes and slice terms from libqvx.so against the FP64 oracle.

Tolerance (stated for the FP32 path): |d alpha| <= 1e-5 * 2^{-N/2}. Slice terms carry
the per-term bound of the same size.
"""
import random

import numpy as np
import pytest

import circuitgen as cg
from oracle import statevector as SV
from oracle import ve as VE

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
q = pytest.importorskip("paper_1805_01450_gb300")


def tol(n):
    return 1e-5 * 2.0 ** (-n / 2)


def _amps(plan, xs):
    a = plan.amplitude(xs)
    return a.cpu().numpy()


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    q.lib()


@pytest.mark.parametrize("engine", ["fused", "stepwise", "persistent"])
def test_worked_example_all_bitstrings(engine):
    c = cg.worked_example()
    psi = SV.final_state(c)
    p = q.Plan(c, engine=engine)
    got = _amps(p, list(range(16)))
    assert np.max(np.abs(got - psi)) < tol(4)


@pytest.mark.parametrize("engine,wpi", [("fused", 1), ("fused", 2), ("fused", 4), ("fused", 8), ("fused", 16),
                                        ("stepwise", 1), ("persistent", 1)])
def test_4x4x10_batch(engine, wpi):
    c = cg.grid_circuit(4, 4, 10, 1001)
    psi = SV.final_state(c)
    xs = [0] + cg.random_bitstrings(16, 200, 1002)
    p = q.Plan(c, engine=engine, warps_per_item=wpi)
    got = _amps(p, xs)
    assert np.max(np.abs(got - psi[xs])) < tol(16)


@pytest.mark.parametrize("inner,wpi,engine,merge", [(-1, 1, "fused", 8), (0, 1, "fused", 8),
                                                    (2, 2, "fused", 8), (6, 4, "fused", 8),
                                                    (3, 1, "stepwise", 8), (4, 1, "fused", 0),
                                                    (2, 1, "stepwise", 0), (4, 1, "persistent", 8),
                                                    (0, 1, "persistent", 0),
                                                    # the bench's autotuned launch configurations
                                                    (5, 8, "fused", 10), (5, 8, "fused", 8)])
def test_6x6x25_k12_full(inner, wpi, engine, merge):
    c = cg.grid_circuit(6, 6, 25, 2001)
    x = cg.random_bitstrings(36, 1, 2002)[0]
    p = q.Plan(c, n_slices=12, inner_slices=inner, warps_per_item=wpi, engine=engine,
               host_merge_rank=merge)
    ref_terms = VE.slice_terms(c, x, p.order, p.slices)
    ref = VE.exact_sum(ref_terms)
    got = _amps(p, [x])[0]
    assert abs(got - ref) < tol(36)
    terms = p.slice_terms([x]).cpu().numpy()[0]
    assert terms.shape == (4096,)
    assert np.max(np.abs(terms - ref_terms)) < tol(36)
    ws = p._ws_for(1, torch.device("cuda"))
    p.check_status(ws)


def test_6x6x25_k12_bench_plan():
    # the plan the benchmark times: order and slices from 64 planning trials (engine and
    # open slices left to the planner, as the autotuner's base plan), then 5 open slices,
    # 8 warps per item, host merging to rank 10 on the fused engine
    c = cg.grid_circuit(6, 6, 25, 2001)
    x = cg.random_bitstrings(36, 1, 2002)[0]
    base = q.Plan(c, n_slices=12, mem_budget_bytes=1 << 30, plan_trials=64)
    p = q.Plan(c, order=base.order, slices=base.slices, inner_slices=5, warps_per_item=8, host_merge_rank=10,
               engine="fused", mem_budget_bytes=1 << 30, plan_trials=64)
    ref_terms = VE.slice_terms(c, x, p.order, p.slices)
    assert abs(_amps(p, [x])[0] - VE.exact_sum(ref_terms)) < tol(36)
    terms = p.slice_terms([x]).cpu().numpy()[0]
    assert np.max(np.abs(terms - ref_terms)) < tol(36)
    p.check_status(p._ws_for(1, torch.device("cuda")))


def test_6x6x25_ragged_slice_ranges_and_batch():
    c = cg.grid_circuit(6, 6, 25, 2001)
    xs = cg.random_bitstrings(36, 5, 77)
    p = q.Plan(c, n_slices=12, inner_slices=3)
    refs = [VE.slice_terms(c, x, p.order, p.slices) for x in xs]
    rng = random.Random(3)
    for _ in range(4):
        s0 = rng.randrange(4096)
        cnt = rng.randrange(1, 4096 - s0 + 1)
        got = p.amplitude(xs, slice_begin=s0, slice_count=cnt).cpu().numpy()
        for g, r in zip(got, refs):
            assert abs(g - VE.exact_sum(r[s0:s0 + cnt])) < tol(36)
    got = p.amplitude(xs, slice_begin=100, slice_count=0).cpu().numpy()
    assert np.all(got == 0)


def test_rotation_circuit_stepwise_and_fused():
    c = cg.rotation_circuit(3, 3, 6, 4001)
    psi = SV.final_state(c)
    xs = cg.random_bitstrings(9, 40, 5)
    for engine in ("fused", "stepwise", "persistent"):
        p = q.Plan(c, n_slices=3, engine=engine)
        assert np.max(np.abs(_amps(p, xs) - psi[xs])) < tol(9)


@pytest.mark.parametrize("engine", ["stepwise", "persistent"])
def test_5x5x20_global_arena_engines_unsliced(engine):
    c = cg.grid_circuit(5, 5, 20, 4001)
    xs = cg.random_bitstrings(25, 8, 6)
    p = q.Plan(c, n_slices=0, engine=engine)
    got = _amps(p, xs)
    for g, x in zip(got, xs):
        assert abs(g - VE.ve_amplitude(c, x, p.order)) < tol(25)


def test_7x7x30_persistent_chunks_and_sampled_slices():
    # rank-17 tensors, 16 work items per bitstring, a memory budget that forces several
    # chunks of items in flight; slice terms checked on a seeded sample of slices
    c = cg.grid_circuit(7, 7, 30, 3001)
    xs = cg.random_bitstrings(49, 3, 3002)
    p = q.Plan(c, n_slices=8, inner_slices=4, engine="persistent", mem_budget_bytes=12 << 20)
    assert p.info["max_rank"] >= 16
    terms = p.slice_terms(xs).cpu().numpy()
    ids = np.random.default_rng(5).choice(256, 12, replace=False)
    for i, x in enumerate(xs):
        ref = VE.slice_terms(c, x, p.order, p.slices, slice_ids=ids)
        assert np.max(np.abs(terms[i, ids] - ref)) < tol(49)
    amps = _amps(p, xs)
    assert np.max(np.abs(amps - terms.sum(axis=1))) < tol(49)
    ws = p._ws_for(3, torch.device("cuda"))
    p.check_status(ws)


def test_degenerate_circuits():
    empty = cg.Circuit(n_qubits=3, gates=[])
    p = q.Plan(empty)
    assert np.allclose(_amps(p, [0, 1, 5]), [1, 0, 0])
    partial = cg.Circuit(n_qubits=3, gates=[cg.Gate(cg.H, 0), cg.Gate(cg.T, 1), cg.Gate(cg.CZ, 0, 1)])
    psi = SV.final_state(partial)
    assert np.max(np.abs(_amps(q.Plan(partial), list(range(8))) - psi)) < 1e-7
    hh = cg.Circuit(n_qubits=2, gates=[cg.Gate(cg.H, 0), cg.Gate(cg.H, 1)])
    assert np.allclose(_amps(q.Plan(hh), [0, 1, 2, 3]), [0.5] * 4)


def test_empty_batch_and_bad_bitstring():
    p = q.Plan(cg.grid_circuit(3, 3, 8, 1))
    assert p.amplitude(torch.zeros(0, dtype=torch.int64, device="cuda")).numel() == 0
    with pytest.raises(q.QvxError):
        p.amplitude([1 << 9])


def test_repeated_calls_reuse_workspace():
    c = cg.grid_circuit(6, 6, 25, 2001)
    x = cg.random_bitstrings(36, 1, 2002)[0]
    p = q.Plan(c, n_slices=12)
    first = _amps(p, [x])[0]
    for _ in range(5):
        assert _amps(p, [x])[0] == first


def test_plans_with_different_shared_memory_interleave():
    # the kernel's shared-memory limit is per function: a small plan launched between two
    # launches of a large one must not shrink it
    c = cg.grid_circuit(6, 6, 25, 2001)
    x = cg.random_bitstrings(36, 1, 2002)[0]
    ref = VE.exact_sum(VE.slice_terms(c, x, q.Plan(c, n_slices=12).order, q.Plan(c, n_slices=12).slices))
    big = q.Plan(c, n_slices=12, inner_slices=7, warps_per_item=1)
    small = q.Plan(c, n_slices=12, inner_slices=0, warps_per_item=16)
    for p in (big, small, big, small):
        assert abs(_amps(p, [x])[0] - ref) < tol(36)


@pytest.mark.parametrize("pin_in,pin_out", [(True, True), (False, False), (True, False), (False, True)])
def test_host_buffer_entry_point(pin_in, pin_out):
    c = cg.grid_circuit(6, 6, 25, 2001)
    p = q.Plan(c, n_slices=12)
    xs = cg.random_bitstrings(36, 3, 55)
    ref = p.amplitude(xs).cpu().numpy()
    h = torch.tensor(xs, dtype=torch.int64)
    out = torch.full((6,), float("nan"), dtype=torch.float64)
    if pin_in:
        h = h.pin_memory()
    if pin_out:
        out = out.pin_memory()
    for _ in range(2):
        got = p.amplitude_host(h, out=out)
        assert np.max(np.abs(got - ref)) < tol(36)
    with pytest.raises(q.QvxError):
        p.amplitude_host([1 << 40])


@pytest.mark.parametrize("engine", ["fused", "stepwise", "persistent"])
def test_cuda_graph_capture_and_replay(engine):
    c = cg.grid_circuit(5, 5, 14, 9)
    p = q.Plan(c, n_slices=4, engine=engine)
    xs = cg.random_bitstrings(25, 2, 10)
    bits = torch.tensor(xs, dtype=torch.int64, device="cuda")
    replay, out = p.graphed(bits)
    ref = lambda zs: np.array([VE.ve_amplitude(c, z, p.order, p.slices) for z in zs])
    replay()
    torch.cuda.synchronize()
    assert np.max(np.abs(out.cpu().numpy() - ref(xs))) < tol(25)
    ys = cg.random_bitstrings(25, 2, 11)
    bits.copy_(torch.tensor(ys, dtype=torch.int64, device="cuda"))
    replay()
    torch.cuda.synchronize()
    assert np.max(np.abs(out.cpu().numpy() - ref(ys))) < tol(25)


@pytest.mark.parametrize("engine", ["stepwise", "persistent"])
def test_7x7x30_large_contractions(engine):
    # rank-17 outputs: the stepwise engine runs most contractions in register-tiled form
    c = cg.grid_circuit(7, 7, 30, 3001)
    xs = cg.random_bitstrings(49, 2, 3003)
    p = q.Plan(c, n_slices=8, inner_slices=4, engine=engine, mem_budget_bytes=40 << 20)
    if engine == "stepwise":
        assert p.info["n_tiled_steps"] >= 50
    ids = np.random.default_rng(6).choice(256, 8, replace=False)
    terms = p.slice_terms(xs).cpu().numpy()
    for i, x in enumerate(xs):
        ref = VE.slice_terms(c, x, p.order, p.slices, slice_ids=ids)
        assert np.max(np.abs(terms[i, ids] - ref)) < tol(49)


@pytest.mark.parametrize("rule", ["reorder", "cz-pair"])
def test_slice_rules_on_device(rule):
    c = cg.grid_circuit(6, 6, 25, 2001)
    x = cg.random_bitstrings(36, 1, 2002)[0]
    p = q.Plan(c, n_slices=12, slice_rule=rule)
    ref = VE.exact_sum(VE.slice_terms(c, x, p.order, p.slices))
    assert abs(_amps(p, [x])[0] - ref) < tol(36)


def _with_open_bits(x, open_qubits, j):
    for i, qb in enumerate(open_qubits):
        x = (x & ~(1 << qb)) | (((j >> i) & 1) << qb)
    return x


@pytest.mark.parametrize("engine", ["fused", "stepwise", "persistent"])
def test_open_qubits_batches_of_amplitudes(engine):
    c = cg.grid_circuit(4, 4, 10, 1001)
    oq = [2, 7, 9, 14]
    psi = SV.final_state(c)
    xs = cg.random_bitstrings(16, 5, 71)
    p = q.Plan(c, n_slices=3, open_qubits=oq, engine=engine)
    got = p.amplitude(xs).cpu().numpy()
    assert got.shape == (5, 16)
    want = np.array([[psi[_with_open_bits(x, oq, j)] for j in range(16)] for x in xs])
    assert np.max(np.abs(got - want)) < tol(16)
    terms = p.slice_terms(xs).cpu().numpy()
    assert terms.shape == (5, 16, 8)
    assert np.max(np.abs(terms.sum(axis=-1) - want)) < tol(16)
    host = p.amplitude_host(xs)
    assert np.max(np.abs(host - want)) < tol(16)


def test_open_qubits_6x6x25_k12():
    c = cg.grid_circuit(6, 6, 25, 2001)
    oq = [0, 35]
    x = cg.random_bitstrings(36, 1, 2002)[0]
    p = q.Plan(c, n_slices=12, open_qubits=oq)
    got = p.amplitude([x]).cpu().numpy()[0]
    for j in range(4):
        xj = _with_open_bits(x, oq, j)
        assert abs(got[j] - VE.ve_amplitude(c, xj, p.order, p.slices)) < tol(36)
