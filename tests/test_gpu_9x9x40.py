"""GPU parity on the 9 x 9 grid of depth 40 (81 qubits, 701 path variables), the largest
circuit class of the paper's Section 6 results: bitstrings take two 64-bit words, and the
slice terms of a seeded work item are compared element by element with the FP64 oracle.

28 variables are sliced (4 kept open inside a work item), so one slice term costs about
2^27 complex multiply-adds and the oracle finishes a term in seconds; the amplitude itself
needs all 2^28 terms (its time is extrapolated by bench.py --workload grid9x9d40 from a
sample of slices, with the plan that slices fewer variables). Pass condition as for the
8 x 8 circuits: sqrt(2^k) * rms |d beta| <= 1e-5 * 2^{-N/2}, and each term within 1e-4 of
its size.
"""
import math
import os

import numpy as np
import pytest

import circuitgen as cg
from oracle import ve as VE

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
q = pytest.importorskip("paper_1805_01450_gb300")

N = 81
TOL = 1e-5 * 2.0 ** (-N / 2)


@pytest.fixture(scope="module")
def case():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = cg.grid_circuit(9, 9, 40, 9001)
    x = cg.random_bitstrings(N, 1, 9002)[0]
    p = q.Plan(c, n_slices=28, inner_slices=4, engine="stepwise", tensor_cores=True, plan_trials=16,
               mem_budget_bytes=16 << 30)
    return c, x, p


def test_9x9x40_slice_terms_vs_oracle(case):
    c, x, p = case
    assert x >> 64 and p.words == 2 and p.info["n_qubits"] == N
    assert p.info["n_gemm_steps"] >= 1 and p.info["n_sliced"] == 28
    rng = np.random.default_rng(9003)
    o = int(rng.integers(0, p.info["n_items_per_bitstring"]))   # work item o: slices 16 o ... 16 o + 15
    got = p.slice_terms([x], slice_begin=16 * o, slice_count=16).cpu().numpy()[0]
    p.check_status(p._ws_for(1, torch.device("cuda")))
    local = sorted(int(i) for i in rng.choice(16, 4, replace=False))
    ref = VE.slice_terms(c, x, p.order, p.slices, slice_ids=[16 * o + i for i in local],
                         threads=min(4, os.cpu_count() or 1))
    d = np.abs(got[local] - ref)
    assert math.sqrt(p.n_slice_terms) * math.sqrt(np.mean(d * d)) <= TOL
    assert np.max(d) <= 1e-4 * np.max(np.abs(ref))


def test_9x9x40_high_word_bits_matter(case):
    # flipping a qubit of the second word changes the item's slice terms (the output
    # variables of qubits 64..80 are read from word 1)
    c, x, p = case
    y = x ^ (1 << 70)
    a = p.slice_terms([x, y], slice_begin=0, slice_count=16).cpu().numpy()
    assert np.max(np.abs(a[0] - a[1])) > 1e-3 * np.max(np.abs(a[0]))
    ref = VE.slice_terms(c, y, p.order, p.slices, slice_ids=[3], threads=1)
    assert abs(a[1][3] - ref[0]) <= 1e-4 * abs(ref[0])
