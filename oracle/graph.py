"""The undirected graphical model of Section 3.A (test infrastructure only).

Walking the circuit in time order, every qubit carries a current variable. A diagonal
gate (T, CZ) adds no variable: it becomes a tensor on the current variable(s). A
non-diagonal single-qubit gate U ends the current variable i and starts a new one j; it
becomes the rank-2 tensor tau[i, j] = U[j, i] (Fig. 3). Variable (q, 0) is the input
value of qubit q, fixed to 0; the last variable of qubit q is its output, fixed to x_q
(Section 3.B.2: output vertices are removed for free; the footnote there allows removing
the input vertices too).

Canonical variable naming: the summed variables are the pairs (q, j) with
0 < j < last(q), numbered 0, 1, ... in order of (q, j). Orders and slice sets are lists
of these numbers.

Also the graph operations the paper draws: fixing a vertex (Fig. 5) and eliminating one
(Section 3.B.1 step 4, Fig. 6), with the step cost 2^deg(v).
"""
from dataclasses import dataclass, field
import numpy as np

import circuitgen as cg
from . import gates as G


@dataclass
class Model:
    n_qubits: int
    last: list                        # last ordinal per qubit (its output variable)
    tensors: list                     # (keys tuple of (q, j), complex128 ndarray with one axis per key)
    variables: list = field(default_factory=list)   # canonical id -> (q, j)
    index: dict = field(default_factory=dict)       # (q, j) -> canonical id


def build(circ) -> Model:
    n = circ.n_qubits
    cur = [0] * n
    tensors = []
    for g in circ.gates:
        if g.kind == cg.CZ:
            tensors.append((((g.q0, cur[g.q0]), (g.q1, cur[g.q1])), G.CZ_DIAG.copy()))
        elif g.kind == cg.T:
            tensors.append((((g.q0, cur[g.q0]),), G.T_DIAG.copy()))
        else:
            q = g.q0
            i, j = (q, cur[q]), (q, cur[q] + 1)
            tensors.append(((i, j), G.matrix(g).T.copy()))   # tau[i, j] = U[j, i]
            cur[q] += 1
    variables = [(q, j) for q in range(n) for j in range(1, cur[q])]
    index = {v: k for k, v in enumerate(variables)}
    return Model(n, cur, tensors, variables, index)


def fixed_values(model: Model, x: int) -> dict:
    """(q, j) -> value for the inputs (0) and outputs (x_q). A qubit with no
    non-diagonal gate has one variable that is both; its consistency is a separate factor."""
    vals = {}
    for q in range(model.n_qubits):
        vals[(q, 0)] = 0
        if model.last[q] > 0:
            vals[(q, model.last[q])] = (x >> q) & 1
    return vals


def restricted_tensors(model: Model, x: int):
    """Tensors with inputs and outputs substituted: list of (canonical ids, ndarray), and a
    scalar prefactor (0 if some untouched qubit has x_q = 1)."""
    vals = fixed_values(model, x)
    scalar = 1.0 + 0j
    for q in range(model.n_qubits):
        if model.last[q] == 0 and (x >> q) & 1:
            scalar = 0.0 + 0j
    out = []
    for keys, data in model.tensors:
        sel = tuple(vals[k] if k in vals else slice(None) for k in keys)
        sub = data[sel]
        ids = tuple(model.index[k] for k in keys if k not in vals)
        if len(ids) == 0:
            scalar *= complex(sub)
        else:
            out.append((ids, np.ascontiguousarray(sub)))
    return out, scalar


def edges(model: Model) -> set:
    """Edge set of G over canonical ids: two summed variables joined by a common tensor."""
    es = set()
    for keys, _ in model.tensors:
        ids = sorted({model.index[k] for k in keys if k in model.index})
        for a in range(len(ids)):
            for b in range(a + 1, len(ids)):
                es.add((ids[a], ids[b]))
    return es


def adjacency(n_vars: int, es) -> list:
    adj = [set() for _ in range(n_vars)]
    for a, b in es:
        adj[a].add(b)
        adj[b].add(a)
    return adj


def fix_vertex(adj: list, v: int) -> list:
    """Fixing v's value removes the vertex and its edges; no tensor is added (Section 3.B.2)."""
    out = [set(a) for a in adj]
    for u in out[v]:
        out[u].discard(v)
    out[v] = set()
    return out


def eliminate_vertex(adj: list, v: int):
    """Step 4 of Section 3.B.1: join every two neighbours of v, then remove v.
    Returns (new adjacency, step cost 2^deg(v)) with the cost of Section 3.B.1."""
    nb = set(adj[v])
    out = [set(a) for a in adj]
    for u in nb:
        out[u] |= nb
        out[u].discard(u)
        out[u].discard(v)
    out[v] = set()
    return out, 2 ** len(nb)


def order_cost(adj: list, order) -> tuple:
    """(sum of 2^deg over the order's steps, largest degree met); vertices already
    fixed (absent from the adjacency's live set) are skipped by the caller."""
    cost, width = 0, 0
    for v in order:
        width = max(width, len(adj[v]))
        adj, c = eliminate_vertex(adj, v)
        cost += c
    return cost, width
