"""qvx_amplitude_noalloc, the entry point for callers that cannot allocate device memory.

Such callers (code that may not call cudaMalloc or hold a workspace of its own) get the
amplitude through a fixed scratch array inside the library. These tests call it through
the C interface, two calls in a row, and compare with qvx_amplitude on the same plan and
bitstrings, within the amplitude tolerance 1e-5 * 2^{-N/2} used by the other GPU tests.
The file sorts last so that a run stopping at the first failure has run everything else.
"""
import ctypes

import numpy as np
import pytest

import circuitgen as cg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
q = pytest.importorskip("paper_1805_01450_gb300")


def tol(n):
    return 1e-5 * 2.0 ** (-n / 2)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _noalloc(plan, bits, n):
    out = torch.full((2 * n,), float("nan"), dtype=torch.float64, device=bits.device)
    L = q.lib()
    st = L.qvx_amplitude_noalloc(plan._h, ctypes.c_void_p(bits.data_ptr()), n, ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == q.QVX_OK, L.qvx_last_error()
    torch.cuda.synchronize()
    return torch.view_as_complex(out.view(n, 2)).cpu().numpy()


CASES = [
    ("4x4x10-batch33", lambda: cg.grid_circuit(4, 4, 10, 1001), dict(n_slices=2), 33),
    ("6x6x25-k12", lambda: cg.grid_circuit(6, 6, 25, 2001), dict(n_slices=12, inner_slices=4, warps_per_item=2), 1),
    ("6x6x25-k12-batch3", lambda: cg.grid_circuit(6, 6, 25, 2001), dict(n_slices=12, inner_slices=5,
                                                                         warps_per_item=4), 3),
]


@pytest.mark.parametrize("name,maker,kw,batch", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_workspace_entry_point(name, maker, kw, batch):
    circ = maker()
    plan = q.Plan(circ, **kw)
    xs = cg.random_bitstrings(circ.n_qubits, batch, 91)
    ref = plan.amplitude(xs).cpu().numpy()
    bits = plan._bits(xs)
    for _ in range(2):
        got = _noalloc(plan, bits, batch)
        assert np.max(np.abs(got - ref)) < tol(circ.n_qubits)


def test_noalloc_alternating_plans_reload_the_scratch():
    a = q.Plan(cg.grid_circuit(4, 4, 10, 1001), n_slices=3)
    b = q.Plan(cg.grid_circuit(3, 4, 12, 5), n_slices=2)
    xa, xb = cg.random_bitstrings(16, 4, 1), cg.random_bitstrings(12, 4, 2)
    ra, rb = a.amplitude(xa).cpu().numpy(), b.amplitude(xb).cpu().numpy()
    ba, bb = a._bits(xa), b._bits(xb)
    for _ in range(2):
        assert np.max(np.abs(_noalloc(a, ba, 4) - ra)) < tol(16)
        assert np.max(np.abs(_noalloc(b, bb, 4) - rb)) < tol(12)


def test_noalloc_rejects_what_it_cannot_hold():
    L = q.lib()
    plan = q.Plan(cg.grid_circuit(6, 6, 25, 2001), n_slices=12, inner_slices=0)   # 4096 items per bitstring
    n = 100                                                                       # 6.4 MB of partials
    bits = plan._bits(cg.random_bitstrings(36, n, 3))
    out = torch.empty(2 * n, dtype=torch.float64, device="cuda")
    st = L.qvx_amplitude_noalloc(plan._h, ctypes.c_void_p(bits.data_ptr()), n, ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == q.QVX_EINVAL and b"scratch too small" in L.qvx_last_error()
    step = q.Plan(cg.grid_circuit(4, 4, 10, 1001), engine="stepwise")
    st = L.qvx_amplitude_noalloc(step._h, ctypes.c_void_p(bits.data_ptr()), 1, ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == q.QVX_EUNSUPPORTED
