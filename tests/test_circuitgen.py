"""The workload generator against the circuit rules of Section 4 and Fig. 7."""
import os

import pytest

import circuitgen as cg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fig7_cz_layouts.txt")


def _fig7():
    out = {c: set() for c in range(1, 9)}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        c, r1, c1, r2, c2 = map(int, line.split())
        out[c].add((r1 * 7 + c1, r2 * 7 + c2))
    return out


def test_layouts_match_fig7():
    fig = _fig7()
    assert sum(len(v) for v in fig.values()) == 97
    for c in range(1, 9):
        assert set(cg.layout_pairs(8, 7, c)) == fig[c], c


@pytest.mark.parametrize("rows,cols", [(4, 4), (5, 5), (6, 6), (7, 7), (8, 8), (3, 9), (9, 2)])
def test_layouts_cover_each_edge_once(rows, cols):
    seen = {}
    for c in range(1, 9):
        for a, b in cg.layout_pairs(rows, cols, c):
            assert (a, b) not in seen
            seen[(a, b)] = c
        busy = [q for p in cg.layout_pairs(rows, cols, c) for q in p]
        assert len(busy) == len(set(busy)), "a qubit carries two CZs in one layout"
    assert len(seen) == (rows - 1) * cols + rows * (cols - 1)


@pytest.mark.parametrize("rows,cols,depth", [(4, 4, 8), (6, 6, 24), (7, 7, 32), (8, 8, 40), (5, 7, 16)])
def test_two_qubit_count_section5(rows, cols, depth):
    # g2 = d/8 ((m-1)n + m(n-1)), exact when 8 divides d (Section 5)
    _, g2 = cg.count_gates(cg.grid_circuit(rows, cols, depth, 7))
    assert g2 == depth // 8 * ((rows - 1) * cols + rows * (cols - 1))


@pytest.mark.parametrize("rows,cols,depth", [(6, 6, 25), (7, 7, 30), (8, 8, 40)])
def test_single_qubit_count_near_section5(rows, cols, depth):
    g1, _ = cg.count_gates(cg.grid_circuit(rows, cols, depth, 11))
    est = depth / 8 * (3 * rows * cols - (rows + cols + 1)) - rows * cols / 4
    assert abs(g1 - est) <= 0.05 * est


def test_rules_3a_3b():
    circ = cg.grid_circuit(6, 6, 25, 2001)
    n = circ.n_qubits
    cz_in = [set() for _ in range(26)]
    for g in circ.gates:
        if g.kind == cg.CZ:
            cz_in[g.cycle] |= {g.q0, g.q1}
    first = {}
    for g in circ.gates:
        if g.cycle == 0:
            assert g.kind == cg.H
            continue
        if g.kind == cg.CZ:
            continue
        assert g.q0 not in cz_in[g.cycle]                   # idle slot
        assert g.q0 in cz_in[g.cycle - 1]                   # rule 3.A
        first.setdefault(g.q0, g.kind)
    assert all(k == cg.T for k in first.values())           # rule 3.B
    assert sum(1 for g in circ.gates if g.cycle == 0) == n
    kinds = {g.kind for g in circ.gates if g.cycle > 0 and g.kind != cg.CZ}
    assert kinds == {cg.T, cg.SQRT_X, cg.SQRT_Y}


def test_all_idle_rule():
    circ = cg.grid_circuit(4, 4, 10, 3, rule="all-idle")
    for t in range(1, 11):
        busy = {q for g in circ.gates if g.cycle == t and g.kind == cg.CZ for q in (g.q0, g.q1)}
        single = {g.q0 for g in circ.gates if g.cycle == t and g.kind != cg.CZ}
        assert busy | single == set(range(16)) and not (busy & single)


def test_splitmix64_reference_values():
    # published splitmix64 outputs for seed 0
    r = cg.SplitMix64(0)
    assert r.next() == 0xE220A8397B1DCDAF
    assert r.next() == 0x6E789E6AA1B965F4
    assert r.next() == 0x06C45D188009454F


def test_seeded_and_deterministic():
    a = cg.grid_circuit(5, 5, 12, 99)
    b = cg.grid_circuit(5, 5, 12, 99)
    c = cg.grid_circuit(5, 5, 12, 100)
    key = lambda ci: [(g.kind, g.q0, g.q1) for g in ci.gates]
    assert key(a) == key(b) and key(a) != key(c)
    bs = cg.random_bitstrings(49, 1000, 3002)
    assert all(0 <= x < (1 << 49) for x in bs) and len(set(bs)) == 1000
    mean_bits = sum(bin(x).count("1") for x in bs) / len(bs)
    assert abs(mean_bits - 24.5) < 0.5


def test_rotation_circuit_counts():
    circ = cg.rotation_circuit(5, 5, 20, 4001)
    rots = [g for g in circ.gates if g.kind == cg.RXY]
    assert len(rots) == 1000 == circ.n_params
    assert sorted(g.param for g in rots) == list(range(1000))
    assert all(0 <= g.theta < 6.2832 and g.phi in (0.0, 1.5707963267948966) for g in rots)
