"""Bounded device waits and a full-size statistical property.

The waits of the library's kernels (the TMA staging wait of the fused kernel, the grid
barrier of the persistent kernel) are bounded: the self-test runs both forms on waits that
can never complete and checks that they give up and report QVX_ETIMEOUT without losing the
context. The 7x7x30 workload with 1024 bitstrings is checked at full size against the
Porter-Thomas moments of 2^N |alpha|^2 (mean 1, second moment 2) and on sampled
amplitudes against the oracle.
"""
import ctypes

import numpy as np
import pytest

import circuitgen as cg
from oracle import ve as VE

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
q = pytest.importorskip("paper_1805_01450_gb300")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_bounded_waits_time_out_and_report():
    c = cg.grid_circuit(4, 4, 10, 1001)
    p = q.Plan(c, n_slices=2)
    ws = p.workspace(4)
    L = q.lib()
    st = L.qvx_selftest_wait_timeout(p._h, ctypes.c_void_p(ws.data_ptr()), ws.numel(), 4096,
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == q.QVX_ETIMEOUT, L.qvx_last_error()
    p.check_status(ws)                      # cleared again
    # the context and the workspace still work
    from oracle import statevector as SV
    psi = SV.final_state(c)
    xs = cg.random_bitstrings(16, 4, 3)
    assert np.max(np.abs(p.amplitude(xs, workspace=ws).cpu().numpy() - psi[xs])) < 1e-5 * 2 ** -8


@pytest.mark.parametrize("k", [8, 4])   # 4 sliced, all open: the bench's autotuned configuration
def test_7x7x30_1024_bitstrings_porter_thomas_and_samples(k):
    c = cg.grid_circuit(7, 7, 30, 3001)
    xs = cg.random_bitstrings(49, 1024, 3002)
    p = q.Plan(c, n_slices=k, inner_slices=4, engine="stepwise", mem_budget_bytes=32 << 30)
    amps = p.amplitude(xs).cpu().numpy()
    pt = (2.0 ** 49) * np.abs(amps) ** 2
    assert abs(pt.mean() - 1.0) < 0.15
    assert abs((pt ** 2).mean() - 2.0) < 0.6
    for i in (0, 511, 1023):
        ref = VE.ve_amplitude(c, xs[i], p.order, p.slices)
        assert abs(amps[i] - ref) < 1e-5 * 2.0 ** (-49 / 2)
