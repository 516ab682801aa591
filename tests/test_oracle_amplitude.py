"""Oracle amplitudes pinned to closed forms, brute force and invariants (Eq. 1, Section 3.B)."""
import math
import random

import numpy as np
import pytest

import circuitgen as cg
from oracle import graph as GR
from oracle import statevector as SV
from oracle import ve as VE


def _circ(n, gates):
    return cg.Circuit(n_qubits=n, gates=gates)


@pytest.mark.parametrize("x", [0, 1, 6, 7])
def test_empty_circuit_is_delta(x):
    c = _circ(3, [])
    want = 1.0 if x == 0 else 0.0
    assert SV.sv_amplitude(c, x) == want
    assert VE.ve_amplitude(c, x) == want


def test_hadamard_layer_is_uniform():
    n = 6
    c = _circ(n, [cg.Gate(cg.H, q) for q in range(n)])
    for x in (0, 5, 63):
        assert abs(SV.sv_amplitude(c, x) - 2 ** (-n / 2)) < 1e-15
        assert abs(VE.ve_amplitude(c, x) - 2 ** (-n / 2)) < 1e-15


def test_hadamard_then_diagonal_closed_form():
    # H layer then CZ and T only: alpha_x = 2^{-N/2} prod_CZ (-1)^{x_a x_b} prod_T e^{i pi x_q/4}
    rng = random.Random(5)
    n = 7
    gates = [cg.Gate(cg.H, q) for q in range(n)]
    for _ in range(25):
        if rng.random() < 0.5:
            a, b = rng.sample(range(n), 2)
            gates.append(cg.Gate(cg.CZ, a, b))
        else:
            gates.append(cg.Gate(cg.T, rng.randrange(n)))
    c = _circ(n, gates)
    for x in range(1 << n):
        want = 2 ** (-n / 2)
        for g in gates[n:]:
            if g.kind == cg.CZ and (x >> g.q0) & 1 and (x >> g.q1) & 1:
                want *= -1
            if g.kind == cg.T and (x >> g.q0) & 1:
                want *= complex(math.cos(math.pi / 4), math.sin(math.pi / 4))
        assert abs(SV.sv_amplitude(c, x) - want) < 1e-14
        assert abs(VE.ve_amplitude(c, x) - want) < 1e-14


def test_double_hadamard_is_identity():
    n = 4
    c = _circ(n, [cg.Gate(cg.H, q) for q in range(n)] * 2)
    for x in range(1 << n):
        assert abs(VE.ve_amplitude(c, x) - (1.0 if x == 0 else 0.0)) < 1e-15


def test_single_qubit_closed_forms():
    # sqrt(X)|0> = ((1+i)|0> + (1-i)|1>)/2; sqrt(Y)|0> = ((1+i)|0> + (1+i)|1>)/2
    for kind, a0, a1 in ((cg.SQRT_X, 0.5 + 0.5j, 0.5 - 0.5j), (cg.SQRT_Y, 0.5 + 0.5j, 0.5 + 0.5j)):
        c = _circ(1, [cg.Gate(kind, 0)])
        assert abs(VE.ve_amplitude(c, 0) - a0) < 1e-15 and abs(VE.ve_amplitude(c, 1) - a1) < 1e-15
        c2 = _circ(1, [cg.Gate(kind, 0), cg.Gate(kind, 0)])   # squares to X or Y: |0> -> |1>
        want = 1.0 if kind == cg.SQRT_X else 1j
        assert abs(VE.ve_amplitude(c2, 1) - want) < 1e-15 and abs(VE.ve_amplitude(c2, 0)) < 1e-15
    th = 0.7
    c = _circ(1, [cg.Gate(cg.RXY, 0, theta=th, phi=math.pi / 2, param=0)])
    assert abs(VE.ve_amplitude(c, 0) - math.cos(th / 2)) < 1e-15
    assert abs(VE.ve_amplitude(c, 1) - math.sin(th / 2)) < 1e-15   # -i sin * e^{i pi/2} = sin


def test_worked_example_sv_vs_ve_all_x():
    c = cg.worked_example()
    psi = SV.final_state(c)
    for x in range(16):
        assert abs(VE.ve_amplitude(c, x) - psi[x]) < 1e-15


@pytest.mark.parametrize("rows,cols,depth,seed", [(3, 3, 8, 1), (4, 4, 10, 1001), (3, 4, 16, 2)])
def test_ve_matches_state_vector(rows, cols, depth, seed):
    c = cg.grid_circuit(rows, cols, depth, seed)
    psi = SV.final_state(c)
    for x in cg.random_bitstrings(c.n_qubits, 12, seed + 1) + [0]:
        assert abs(VE.ve_amplitude(c, x) - psi[x]) < 1e-14


def test_normalisation_by_elimination():
    # sum over all x of |alpha_x|^2 = 1, each alpha from its own elimination
    c = cg.grid_circuit(3, 3, 12, 4)
    tot = sum(abs(VE.ve_amplitude(c, x)) ** 2 for x in range(1 << 9))
    assert abs(tot - 1.0) < 1e-13
    c4 = cg.grid_circuit(4, 4, 10, 1001)
    assert abs(np.sum(np.abs(SV.final_state(c4)) ** 2) - 1.0) < 1e-12


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_order_and_slice_invariance(seed):
    c = cg.grid_circuit(4, 4, 12, 40 + seed)
    m = GR.build(c)
    nv = len(m.variables)
    x = cg.random_bitstrings(16, 1, seed)[0]
    ref = SV.sv_amplitude(c, x)
    rng = random.Random(seed)
    for k in (0, 1, 3):
        sl = rng.sample(range(nv), k)
        order = [v for v in range(nv) if v not in sl]
        rng.shuffle(order)
        terms = VE.slice_terms(c, x, order, sl, model=m)
        assert len(terms) == 1 << k
        assert abs(VE.exact_sum(terms) - ref) < 1e-14


def test_slice_terms_are_restricted_sums():
    # a slice term equals the amplitude with that variable's value forced (Section 3.B.2):
    # here the sliced variable is the only summed one of a 1-qubit H-H-H circuit
    c = _circ(1, [cg.Gate(cg.H, 0), cg.Gate(cg.H, 0)])
    t = VE.slice_terms(c, 0, [], [0])
    assert np.allclose(t, [0.5, 0.5])
    t1 = VE.slice_terms(c, 1, [], [0])
    assert np.allclose(t1, [0.5, -0.5])


def test_numpy_einsum_third_path():
    c = cg.grid_circuit(3, 3, 10, 8)
    m = GR.build(c)
    letters = "abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ"
    for x in (0, 77, 300):
        tens, scalar = GR.restricted_tensors(m, x)
        assert len(m.variables) <= len(letters)
        spec = ",".join("".join(letters[v] for v in ids) for ids, _ in tens) + "->"
        val = scalar * np.einsum(spec, *[d for _, d in tens], optimize="greedy")
        assert abs(val - VE.ve_amplitude(c, x)) < 1e-14


def test_porter_thomas_moments():
    # a deep random circuit: 2^N |alpha|^2 has mean 1 (exactly, by normalisation) and second
    # moment close to 2 (exponential distribution)
    c = cg.grid_circuit(4, 4, 40, 77)
    p = (1 << 16) * np.abs(SV.final_state(c)) ** 2
    assert abs(p.mean() - 1.0) < 1e-10
    assert abs((p ** 2).mean() - 2.0) < 0.15
