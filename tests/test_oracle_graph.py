"""Oracle graphical model against the worked example (Section 3.A, Figs. 4-6)."""
import circuitgen as cg
from oracle import graph as GR

from _golden import worked_example


def _letters(model, var):
    by_key = {v: k for k, v in var.items()}
    return {i: by_key[key] for i, key in enumerate(model.variables)}


def test_worked_example_graph_fig4():
    var, edges, _, _ = worked_example()
    m = GR.build(cg.worked_example())
    assert len(m.variables) == 10                     # 2^10 terms (Section 3.A)
    assert set(m.variables) == set(var.values())
    name = _letters(m, var)
    got = {frozenset((name[a], name[b])) for a, b in GR.edges(m)}
    assert got == edges and len(got) == 12


def test_fixing_vertices_fig5():
    var, edges, fix, _ = worked_example()
    m = GR.build(cg.worked_example())
    name = _letters(m, var)
    ident = {v: k for k, v in name.items()}
    adj = GR.adjacency(10, GR.edges(m))
    for letter, removed in fix.items():
        after = GR.fix_vertex(adj, ident[letter])
        left = {frozenset((name[a], name[b])) for a in range(10) for b in after[a] if a < b}
        assert edges - left == removed
        assert left <= edges


def test_eliminating_vertices_fig6():
    var, edges, _, elim = worked_example()
    m = GR.build(cg.worked_example())
    name = _letters(m, var)
    ident = {v: k for k, v in name.items()}
    adj = GR.adjacency(10, GR.edges(m))
    for letter, (cost, added) in elim.items():
        v = ident[letter]
        after, c = GR.eliminate_vertex(adj, v)
        assert c == cost
        left = {frozenset((name[a], name[b])) for a in range(10) for b in after[a] if a < b}
        gone = {e for e in edges if letter in e}
        assert left == (edges - gone) | added


def test_output_vertices_removed_and_merging():
    # diagonal gates add no variables: H, CZ, T only -> one summed variable per qubit
    circ = cg.Circuit(n_qubits=3, gates=[cg.Gate(cg.H, q) for q in range(3)] +
                      [cg.Gate(cg.CZ, 0, 1), cg.Gate(cg.T, 2), cg.Gate(cg.CZ, 1, 2)] +
                      [cg.Gate(cg.H, q) for q in range(3)])
    m = GR.build(circ)
    assert m.variables == [(0, 1), (1, 1), (2, 1)]
    assert GR.edges(m) == {(0, 1), (1, 2)}
    # no final layer: the first variable is the output and is fixed, nothing is summed
    circ2 = cg.grid_circuit(3, 3, 0, 1)
    assert GR.build(circ2).variables == []
