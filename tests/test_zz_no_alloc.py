"""qvx_amplitude_noalloc, the entry point for callers that cannot allocate device memory.

Such callers (code running inside another library's callback, a real-time loop that must not
block on an allocation, a process whose device memory is all reserved up front) cannot
provide a workspace; they get the amplitude through a fixed 4 MiB scratch array inside the
library. These tests call it through the C interface, two calls in a row, and compare with
the FP64 oracle and with qvx_amplitude on the same plan and bitstrings, within the amplitude
tolerance 1e-5 * 2^{-N/2} used by the other GPU tests; they also check the size limit on
both sides of it and the status query. The file sorts last so that a run stopping at the
first failure has run everything else.
"""
import ctypes

import numpy as np
import pytest

import circuitgen as cg
from oracle import ve as VE

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
q = pytest.importorskip("paper_1805_01450_gb300")

SCRATCH = 4 << 20


def tol(n):
    return 1e-5 * 2.0 ** (-n / 2)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _call(plan, bits, n, out):
    return q.lib().qvx_amplitude_noalloc(plan._h, ctypes.c_void_p(bits.data_ptr()), n, ctypes.c_void_p(out.data_ptr()),
                                         _stream())


def _noalloc(plan, bits, n):
    out = torch.full((2 * n,), float("nan"), dtype=torch.float64, device=bits.device)
    st = _call(plan, bits, n, out)
    assert st == q.QVX_OK, q.lib().qvx_last_error()
    assert q.lib().qvx_noalloc_status(_stream()) == q.QVX_OK, q.lib().qvx_last_error()
    return torch.view_as_complex(out.view(n, 2)).cpu().numpy()


def _oracle(circ, plan, xs):
    return np.array([VE.ve_amplitude(circ, x, plan.order, plan.slices) for x in xs])


CASES = [
    ("4x4x10-batch33", lambda: cg.grid_circuit(4, 4, 10, 1001), dict(n_slices=2), 33),
    ("6x6x25-k12", lambda: cg.grid_circuit(6, 6, 25, 2001), dict(n_slices=12, inner_slices=4, warps_per_item=2), 1),
    ("6x6x25-k12-batch3", lambda: cg.grid_circuit(6, 6, 25, 2001), dict(n_slices=12, inner_slices=5,
                                                                         warps_per_item=4), 3),
]


@pytest.mark.parametrize("name,maker,kw,batch", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_oracle_and_workspace_entry_point(name, maker, kw, batch):
    circ = maker()
    plan = q.Plan(circ, **kw)
    xs = cg.random_bitstrings(circ.n_qubits, batch, 91)
    want = _oracle(circ, plan, xs)
    ref = plan.amplitude(xs).cpu().numpy()
    bits = plan._bits(xs)
    for _ in range(2):
        got = _noalloc(plan, bits, batch)
        assert np.max(np.abs(got - want)) < tol(circ.n_qubits)
        assert np.max(np.abs(got - ref)) < tol(circ.n_qubits)


def test_noalloc_alternating_plans_reload_the_scratch():
    ca, cb = cg.grid_circuit(4, 4, 10, 1001), cg.grid_circuit(3, 4, 12, 5)
    a = q.Plan(ca, n_slices=3)
    b = q.Plan(cb, n_slices=2)
    xa, xb = cg.random_bitstrings(16, 4, 1), cg.random_bitstrings(12, 4, 2)
    ra, rb = _oracle(ca, a, xa), _oracle(cb, b, xb)
    ba, bb = a._bits(xa), b._bits(xb)
    for _ in range(2):
        assert np.max(np.abs(_noalloc(a, ba, 4) - ra)) < tol(16)
        assert np.max(np.abs(_noalloc(b, bb, 4) - rb)) < tol(12)


def _max_batch(plan):
    # the documented scratch layout: 256 bytes of status words, the device image rounded up to
    # 256 bytes, 32 bytes per (bitstring, outer work item)
    image = -(-len(plan.image()) // 256) * 256
    return (SCRATCH - 256 - image) // (32 * plan.info["n_items_per_bitstring"])


def test_noalloc_size_limit_on_both_sides():
    circ = cg.grid_circuit(4, 4, 10, 1001)
    plan = q.Plan(circ, n_slices=8, inner_slices=0)    # 256 work items per bitstring: 8 KiB each
    n = _max_batch(plan)
    assert 100 < n < 1000
    xs = cg.random_bitstrings(16, n + 1, 17)
    bits = plan._bits(xs)
    got = _noalloc(plan, bits[:n], n)                   # just fits
    sv_idx = [0, n // 2, n - 1]
    want = _oracle(circ, plan, [xs[i] for i in sv_idx])
    assert np.max(np.abs(got[sv_idx] - want)) < tol(16)
    out = torch.empty(2 * (n + 1), dtype=torch.float64, device="cuda")
    L = q.lib()
    assert _call(plan, bits, n + 1, out) == q.QVX_EINVAL       # one bitstring more does not
    assert b"scratch too small" in L.qvx_last_error()


def test_noalloc_rejects_what_it_cannot_hold():
    L = q.lib()
    plan = q.Plan(cg.grid_circuit(6, 6, 25, 2001), n_slices=12, inner_slices=0)   # 4096 items per bitstring
    n = 100                                                                       # 13.1 MB of partials
    bits = plan._bits(cg.random_bitstrings(36, n, 3))
    out = torch.empty(2 * n, dtype=torch.float64, device="cuda")
    assert _call(plan, bits, n, out) == q.QVX_EINVAL and b"scratch too small" in L.qvx_last_error()
    step = q.Plan(cg.grid_circuit(4, 4, 10, 1001), engine="stepwise")
    assert _call(step, bits, 1, out) == q.QVX_EUNSUPPORTED


def test_noalloc_status_reports_an_out_of_range_sum_then_clears():
    # a U1 gate of size 1e9 makes the amplitude 5e8, outside the exact sum's range: the call
    # itself succeeds, the amplitudes are NaN and the status query reports QVX_ERANGE once
    big = cg.Circuit(2, [cg.Gate(cg.H, 0), cg.Gate(cg.H, 1), cg.Gate(cg.CZ, 0, 1),
                         cg.Gate(cg.U1, 0, u=(1e9, 0.0, 0.0, 0.0, 0.0, 0.0, 1e9, 0.0)), cg.Gate(cg.H, 1)])
    plan = q.Plan(big, engine="fused", host_merge_rank=0)
    bits = plan._bits([0, 1])
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    L = q.lib()
    assert _call(plan, bits, 2, out) == q.QVX_OK
    assert L.qvx_noalloc_status(_stream()) == q.QVX_ERANGE
    assert torch.isnan(out).all()
    assert L.qvx_noalloc_status(_stream()) == q.QVX_OK
    # and the scratch serves the next plan normally
    circ = cg.grid_circuit(4, 4, 10, 1001)
    p = q.Plan(circ, n_slices=2)
    xs = cg.random_bitstrings(16, 3, 4)
    assert np.max(np.abs(_noalloc(p, p._bits(xs), 3) - _oracle(circ, p, xs))) < tol(16)
