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


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def test_fused_kernel_staging_timeout_writes_nan_and_the_workspace_recovers():
    # every CTA's first staging wait gives up at once (the copies still land before the CTA
    # moves on): QVX_ETIMEOUT, NaN amplitudes, and the finished-CTA counter is reset, so the
    # next call on the same workspace computes correct amplitudes
    from oracle import statevector as SV
    c = cg.grid_circuit(4, 4, 10, 1001)
    p = q.Plan(c, n_slices=4, inner_slices=1, engine="fused")
    xs = cg.random_bitstrings(16, 6, 77)
    bits = p._bits(xs)
    ws = p.workspace(len(xs))
    out = torch.zeros(2 * len(xs), dtype=torch.float64, device="cuda")
    L = q.lib()
    for _ in range(2):
        st = L.qvx_selftest_fused_timeout(p._h, ctypes.c_void_p(bits.data_ptr()), len(xs),
                                          ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(ws.data_ptr()),
                                          ws.numel(), _stream())
        assert st == q.QVX_OK, L.qvx_last_error()
        torch.cuda.synchronize()
        assert torch.isnan(out).all()
        with pytest.raises(q.QvxError) as e:
            p.check_status(ws)
        assert e.value.status == q.QVX_ETIMEOUT
        want = SV.final_state(c)[xs]
        got = p.amplitude(xs, workspace=ws).cpu().numpy()
        assert np.max(np.abs(got - want)) < 1e-5 * 2 ** -8
        p.check_status(ws)


def _huge_gate_circuit(scale):
    # H on both qubits, then a U1 gate scale * identity on qubit 0 (non-diagonal kind): the
    # amplitude is scale / 2, far outside the exact sum's range when scale is large
    c = cg.Circuit(2, [cg.Gate(cg.H, 0), cg.Gate(cg.H, 1), cg.Gate(cg.CZ, 0, 1),
                       cg.Gate(cg.U1, 0, u=(scale, 0.0, 0.0, 0.0, 0.0, 0.0, scale, 0.0)), cg.Gate(cg.H, 1)])
    return c


@pytest.mark.parametrize("engine", ["fused", "stepwise"])
def test_exact_sum_out_of_range_is_reported_not_wrapped(engine):
    from oracle import statevector as SV
    small = _huge_gate_circuit(3.0)
    p = q.Plan(small, engine=engine, host_merge_rank=0)   # every contraction on the device
    got = p.amplitude([0, 1, 2, 3]).cpu().numpy()
    assert np.max(np.abs(got - SV.final_state(small)[[0, 1, 2, 3]])) < 1e-6
    big = _huge_gate_circuit(1e9)           # |alpha| = 5e8 >= 2^27
    p = q.Plan(big, engine=engine, host_merge_rank=0)
    ws = p.workspace(2)
    a = p.amplitude([0, 1], workspace=ws).cpu().numpy()
    assert np.isnan(a).all()
    with pytest.raises(q.QvxError) as e:
        p.check_status(ws)
    assert e.value.status == q.QVX_ERANGE
    p.check_status(ws)                      # cleared


@pytest.mark.parametrize("engine,kw", [("fused", dict(n_slices=6, inner_slices=2)),
                                       ("stepwise", dict(n_slices=4, inner_slices=2)),
                                       ("stepwise", dict(n_slices=8, inner_slices=2, tensor_cores=True))])
def test_profiled_call_logs_every_launch(engine, kw):
    c = cg.grid_circuit(6, 6, 25, 2001) if not kw.get("tensor_cores") else cg.grid_circuit(5, 6, 40, 19)
    p = q.Plan(c, engine=engine, **kw)
    xs = cg.random_bitstrings(c.n_qubits, 3, 5)
    bits = p._bits(xs)
    ws = p.workspace(3)
    out = torch.empty(6, dtype=torch.float64, device="cuda")
    want = p.amplitude(bits, workspace=ws).cpu().numpy()
    L = q.lib()
    n0 = L.qvx_kernel_launches()
    for _ in range(2):
        p.amplitude_profiled(bits, ws, out)
    launches = L.qvx_kernel_launches() - n0
    recs = p.read_profile()
    assert len(recs) == launches and p.read_profile() == []
    assert np.array_equal(torch.view_as_complex(out.view(3, 2)).cpu().numpy(), want)
    assert all(r["ms"] > 0 for r in recs)
    # the contraction launches carry the plan's algorithmic work exactly (both calls)
    contr = [r for r in recs if r["kernel"] not in ("finish_kernel", "slice_sum_kernel")]
    assert sum(r["bytes"] for r in contr) == pytest.approx(2 * 3 * p.info["bytes_per_amplitude"], rel=1e-12)
    assert sum(r["flops"] for r in contr) == pytest.approx(2 * 3 * p.info["flops_per_amplitude"], rel=1e-12)
    if kw.get("tensor_cores"):
        assert p.info["n_gemm_steps"] > 0 and any(r["kernel"] == "gemm_tc_kernel" for r in recs)
    if engine == "fused":
        assert [r["kernel"] for r in recs] == ["fused_program_kernel"] * 2


def test_checkpointed_amplitude_resumes_on_the_gpu(tmp_path):
    # ranges of 1000 of the 4096 slice terms (the last one ragged); an interrupted run
    # resumes from its journal to the oracle's amplitudes
    from paper_1805_01450_gb300.checkpoint import amplitude_resumable
    c = cg.grid_circuit(6, 6, 25, 2001)
    p = q.Plan(c, n_slices=12, inner_slices=3, plan_trials=4)
    xs = cg.random_bitstrings(36, 2, 2002)
    path = str(tmp_path / "journal.jsonl")
    assert amplitude_resumable(p, xs, path, 1000, stop_after=2) is None
    got = amplitude_resumable(p, xs, path, 1000)
    want = [VE.exact_sum(VE.slice_terms(c, x, p.order, p.slices)) for x in xs]
    assert np.max(np.abs(got - np.array(want))) < 1e-5 * 2.0 ** -18
    assert np.max(np.abs(got - p.amplitude(xs).cpu().numpy())) < 1e-5 * 2.0 ** -18
