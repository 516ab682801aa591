"""GPU parity of the tensor-core form of the dense contractions (three-part bf16 GEMM on
tcgen05, FP32 accumulation) against the FP64 oracle and against the FP32 SIMT kernels."""
import numpy as np
import pytest

import circuitgen as cg
from oracle import ve as VE

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
q = pytest.importorskip("paper_1805_01450_gb300")


def tol(n):
    return 1e-5 * 2.0 ** (-n / 2)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


CASES = [
    # (rows, cols, depth, seed, sliced, inner)
    (6, 6, 40, 7066, 8, 2),
    (7, 8, 32, 7078, 6, 2),
    (5, 6, 40, 19, 8, 2),      # the step's second operand takes the GEMM's row role
]


@pytest.mark.parametrize("r,c_,d,seed,k,inner", CASES)
def test_tensor_core_slice_terms_vs_oracle(r, c_, d, seed, k, inner):
    c = cg.grid_circuit(r, c_, d, seed)
    n = r * c_
    p = q.Plan(c, n_slices=k, inner_slices=inner, engine="stepwise", tensor_cores=True)
    assert p.info["n_gemm_steps"] >= 1
    xs = cg.random_bitstrings(n, 2, seed + 1)
    terms = p.slice_terms(xs).cpu().numpy()
    ids = np.random.default_rng(seed).choice(1 << k, 6, replace=False)
    for i, x in enumerate(xs):
        ref = VE.slice_terms(c, x, p.order, p.slices, slice_ids=ids)
        assert np.max(np.abs(terms[i, ids] - ref)) < tol(n)


@pytest.mark.parametrize("r,c_,d,seed,k,inner", CASES)
def test_tensor_core_amplitudes_match_simt(r, c_, d, seed, k, inner):
    c = cg.grid_circuit(r, c_, d, seed)
    n = r * c_
    xs = cg.random_bitstrings(n, 3, seed + 2)
    tc = q.Plan(c, n_slices=k, inner_slices=inner, engine="stepwise", tensor_cores=True)
    simt = q.Plan(c, order=tc.order, slices=tc.slices, inner_slices=inner, engine="stepwise")
    assert simt.info["n_gemm_steps"] == 0
    a = tc.amplitude(xs).cpu().numpy()
    b = simt.amplitude(xs).cpu().numpy()
    assert np.max(np.abs(a - b)) < tol(n)


def test_tensor_core_item_batches():
    # a memory budget that fits the operand tiles of a single work item at a time
    c = cg.grid_circuit(6, 6, 40, 7066)
    xs = cg.random_bitstrings(36, 2, 7068)
    big = q.Plan(c, n_slices=8, inner_slices=2, engine="stepwise", tensor_cores=True)
    small = q.Plan(c, order=big.order, slices=big.slices, inner_slices=2, engine="stepwise", tensor_cores=True,
                   mem_budget_bytes=8 << 20)
    a = big.amplitude(xs).cpu().numpy()
    b = small.amplitude(xs).cpu().numpy()
    assert np.max(np.abs(a - b)) < tol(36)


def test_wide_register_tiles_vs_oracle():
    # the SIMT form of a compute-heavy step: an 8 x 8 register tile per thread
    c = cg.grid_circuit(5, 6, 40, 19)
    p = q.Plan(c, n_slices=8, inner_slices=2, engine="stepwise")
    xs = cg.random_bitstrings(30, 2, 21)
    terms = p.slice_terms(xs).cpu().numpy()
    ids = np.random.default_rng(19).choice(1 << 8, 6, replace=False)
    for i, x in enumerate(xs):
        ref = VE.slice_terms(c, x, p.order, p.slices, slice_ids=ids)
        assert np.max(np.abs(terms[i, ids] - ref)) < tol(30)


# 6x7x40 plans whose tensor-core steps take the B-stationary form (at most 32 summed entries,
# at least 4 row tiles of 128 per column tile), one case per column-tile width and summed
# size: (rows, cols, depth, seed, sliced, inner, real columns NT, summed-index bits)
BS_CASES = [
    (6, 7, 40, 1, 8, 2, 32, 3),
    (6, 7, 40, 14, 10, 2, 64, 3),
    (6, 7, 40, 3, 8, 2, 128, 5),
    (6, 7, 40, 5, 10, 2, 128, 3),
    (6, 7, 40, 2, 10, 2, 256, 3),
    (6, 7, 40, 12, 10, 2, 32, 4),
]


@pytest.mark.parametrize("r,c_,d,seed,k,inner,nt,nk", BS_CASES)
def test_b_stationary_form_vs_oracle(r, c_, d, seed, k, inner, nt, nk):
    import os
    from _program_exec import Program
    c = cg.grid_circuit(r, c_, d, seed)
    n = r * c_
    p = q.Plan(c, n_slices=k, inner_slices=inner, engine="stepwise", tensor_cores=True)
    shapes = [(int(g["nm"]), int(g["nn"]), int(g["nk"])) for g in Program(p.image()).gemms if int(g["nk"]) > 0]
    # the launcher's choice: B-stationary when the summed index fills at most two chunks of 16
    # and there are at least 4 row tiles; the case's step is among them
    assert any((256 if nn >= 7 else 2 << nn) == nt and kk == nk and max(1, (1 << kk) // 16) <= 2 and (1 << nm) // 128 >= 4
               for nm, nn, kk in shapes), shapes
    xs = cg.random_bitstrings(n, 1, seed + 1)
    terms = p.slice_terms(xs).cpu().numpy()
    ids = np.random.default_rng(seed).choice(1 << k, 4, replace=False)
    ref = VE.slice_terms(c, xs[0], p.order, p.slices, slice_ids=ids, threads=min(4, os.cpu_count() or 1))
    assert np.max(np.abs(terms[0, ids] - ref)) < tol(n)
