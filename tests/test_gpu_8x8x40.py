"""GPU parity at the full size of the 8x8 grid circuit of depth 40 (64 qubits, 525 path
variables, 10 sliced of which 4 stay open inside a work item, tensors up to rank 27), in
the stepwise engine with the dense contractions on the tensor cores, for the three seeded
circuits whose median time per amplitude is reported (planned with 64 planning trials, as
the benchmark does): slice terms of one seeded work item against the FP64 oracle on a
seeded sample of its slices (the oracle takes tens of seconds per slice term here), and
the whole amplitude of the tensor-core form against the FP32 SIMT form of the same plan.

Tolerance: |d beta| <= 1e-5 * 2^{-N/2} per slice term and |d alpha| of the same size for the
amplitude. Each slice term is far smaller than 2^{-N/2}, so the terms are also held to a
relative error of 1e-4 (the three-part bf16 split leaves about 2^-23 relative error per
product).
"""
import numpy as np
import pytest

import circuitgen as cg
from oracle import ve as VE

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
q = pytest.importorskip("paper_1805_01450_gb300")

N = 64
TOL = 1e-5 * 2.0 ** (-N / 2)
BUDGET = 16 << 30


@pytest.fixture(scope="module", params=[5001, 5002, 5003])
def circuit(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return cg.grid_circuit(8, 8, 40, request.param), cg.random_bitstrings(N, 1, 5002)[0]


@pytest.fixture(scope="module")
def tc_plan(circuit):
    c, _ = circuit
    p = q.Plan(c, n_slices=10, inner_slices=4, engine="stepwise", tensor_cores=True, mem_budget_bytes=BUDGET,
               plan_trials=64)
    # circuit 5002's one dense step stores along a batch mode and keeps its SIMT form
    assert p.info["n_gemm_steps"] >= (0 if c.name.endswith("s5002") else 1) and p.info["max_rank"] >= 24
    return p


def test_8x8x40_tensor_core_slice_terms_vs_oracle(circuit, tc_plan):
    c, x = circuit
    rng = np.random.default_rng(5003)
    o = int(rng.integers(0, 64))                 # work item o: slices 16 o ... 16 o + 15
    terms = tc_plan.slice_terms([x], slice_begin=16 * o, slice_count=16).cpu().numpy()[0]
    local = sorted(int(i) for i in rng.choice(16, 2, replace=False))
    ref = VE.slice_terms(c, x, tc_plan.order, tc_plan.slices, slice_ids=[16 * o + i for i in local], threads=2)
    got = terms[local]
    assert np.max(np.abs(got - ref)) < TOL
    assert np.max(np.abs(got - ref)) < 1e-4 * np.max(np.abs(ref))
    tc_plan.check_status(tc_plan._ws_for(1, torch.device("cuda")))


def test_8x8x40_amplitude_tensor_cores_vs_simt(circuit, tc_plan):
    c, x = circuit
    simt = q.Plan(c, order=tc_plan.order, slices=tc_plan.slices, inner_slices=4, engine="stepwise",
                  mem_budget_bytes=BUDGET)
    assert simt.info["n_gemm_steps"] == 0
    a = tc_plan.amplitude([x]).cpu().numpy()
    b = simt.amplitude([x]).cpu().numpy()
    assert np.all(np.isfinite(a)) and abs(b[0]) > 0
    assert np.max(np.abs(a - b)) < TOL
