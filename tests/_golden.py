"""Readers for the text fixtures under tests/golden/."""
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def worked_example():
    """Letters -> (qubit 0-based, ordinal); edges; fix and eliminate expectations (Figs. 4-6)."""
    var, edges, fix, elim = {}, set(), {}, {}
    for line in open(os.path.join(GOLDEN, "worked_example_graph.txt")):
        w = line.split()
        if not w or w[0].startswith("#"):
            continue
        if w[0] == "var":
            var[w[1]] = (int(w[2]) - 1, int(w[3]))
        elif w[0] == "edge":
            edges.add(frozenset(w[1:3]))
        elif w[0] == "fix":
            fix[w[1]] = {frozenset(p.split("-")) for p in w[3:]}
        elif w[0] == "eliminate":
            elim[w[1]] = (int(w[3]), {frozenset(p.split("-")) for p in w[5:]})
    return var, edges, fix, elim
