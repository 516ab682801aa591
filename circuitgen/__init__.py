"""Seeded synthetic workloads: random 2-D grid circuits, rotation circuits and bitstrings.

This module only *describes* circuits (gate kinds, qubits, angles) and draws random
bitstrings. It holds none of the simulation arithmetic: no gate matrix, no graph, no
contraction. Both the CPU oracle and the GPU library consume its output, each with its
own gate matrices and its own graph construction.

Circuit family (Section 4, rules 1-3 and Fig. 7):
  * cycle 0 is a layer of Hadamards on every qubit (rule 1);
  * cycles t = 1..depth place CZ gates in the 8 staggered nearest-neighbour layouts of
    Fig. 7, layout ((t-1) mod 8) + 1 in cycle t (rule 2);
  * a qubit idle in cycle t receives a single-qubit gate only if it took part in a CZ in
    cycle t-1 (rule 3.A); its first such gate is T (rule 3.B); later ones are drawn
    uniformly from {sqrt(X), sqrt(Y), T} (rule 3).
"depth" counts the CZ cycles after the Hadamard cycle, which makes the two-qubit gate
count d/8 * ((m-1)n + m(n-1)) of Section 5 exact whenever 8 divides d.

Qubit q of an R x C grid sits at row q // C, column q % C; bit q of an integer bitstring
is the value of qubit q.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

# Gate kinds. The integer codes are the ones the C interface uses (include/qvx.h).
H, T, SQRT_X, SQRT_Y, CZ, RXY, U1 = range(7)
KIND_NAMES = {H: "H", T: "T", SQRT_X: "sqrtX", SQRT_Y: "sqrtY", CZ: "CZ", RXY: "Rxy", U1: "U1"}
SINGLE_QUBIT = (H, T, SQRT_X, SQRT_Y, RXY, U1)
MASK64 = (1 << 64) - 1


@dataclass
class Gate:
    kind: int
    q0: int
    q1: int = -1
    theta: float = 0.0
    phi: float = 0.0
    param: int = -1          # index into an angle vector, or -1 for a fixed gate
    u: tuple = ()            # U1 only: 2x2 complex matrix as 8 doubles (re, im) row-major
    cycle: int = 0


@dataclass
class Circuit:
    n_qubits: int
    gates: list = field(default_factory=list)
    rows: int = 0
    cols: int = 0
    depth: int = 0
    name: str = ""

    @property
    def n_params(self) -> int:
        return 1 + max((g.param for g in self.gates), default=-1)

    def thetas(self) -> list:
        out = [0.0] * self.n_params
        for g in self.gates:
            if g.param >= 0:
                out[g.param] = g.theta
        return out


class SplitMix64:
    """splitmix64 (Steele, Lea, Flood 2014): state += 0x9E3779B97F4A7C15, then two xor-shift-multiply rounds."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next() >> 11) * (1.0 / (1 << 53))


def cz_layout_of_edge(r: int, c: int, vertical: bool) -> int:
    """Fig. 7 configuration (1..8) that holds the grid edge anchored at (r, c).

    A horizontal edge joins (r, c)-(r, c+1); a vertical one joins (r, c)-(r+1, c). The
    rule below reproduces every drawn pair of Fig. 7 on its 8 x 7 lattice and extends
    the same stagger to any grid.
    """
    if not vertical:
        return {2: 1, 0: 2, 3: 5, 1: 6}[(c + 2 * r) % 4]
    return {3: 3, 1: 4, 0: 7, 2: 8}[(r + 2 * c) % 4]


def layout_pairs(rows: int, cols: int, config: int) -> list:
    """Qubit pairs (a, b), a < b, that carry a CZ in Fig. 7 configuration `config`."""
    out = []
    for r in range(rows):
        for c in range(cols):
            if c + 1 < cols and cz_layout_of_edge(r, c, False) == config:
                out.append((r * cols + c, r * cols + c + 1))
            if r + 1 < rows and cz_layout_of_edge(r, c, True) == config:
                out.append((r * cols + c, (r + 1) * cols + c))
    return out


def grid_circuit(rows: int, cols: int, depth: int, seed: int, rule: str = "paper") -> Circuit:
    """Random supremacy circuit of Section 4 on a rows x cols grid with `depth` CZ cycles.

    rule="paper": rules 3.A/3.B as stated. rule="all-idle": every idle qubit of cycles
    1..depth gets a gate drawn uniformly from {sqrt(X), sqrt(Y), T}.
    Draws: one splitmix64 value per random gate, cycles ascending, qubits ascending;
    value mod 3 selects sqrt(X), sqrt(Y), T in that order.
    """
    if rule not in ("paper", "all-idle"):
        raise ValueError(f"unknown gate rule {rule!r}")
    n = rows * cols
    rng = SplitMix64(seed)
    circ = Circuit(n_qubits=n, rows=rows, cols=cols, depth=depth,
                   name=f"grid{rows}x{cols}d{depth}s{seed}{'' if rule == 'paper' else '-' + rule}")
    for q in range(n):
        circ.gates.append(Gate(H, q, cycle=0))
    prev_busy = [False] * n          # took part in a CZ in the previous cycle
    had_single = [False] * n         # has received a single-qubit gate after the H cycle
    for t in range(1, depth + 1):
        pairs = layout_pairs(rows, cols, (t - 1) % 8 + 1)
        busy = [False] * n
        for a, b in pairs:
            busy[a] = busy[b] = True
        for a, b in pairs:
            circ.gates.append(Gate(CZ, a, b, cycle=t))
        for q in range(n):
            if busy[q]:
                continue
            if rule == "paper":
                if not prev_busy[q]:
                    continue
                if not had_single[q]:
                    kind = T
                else:
                    kind = (SQRT_X, SQRT_Y, T)[rng.next() % 3]
            else:
                kind = (SQRT_X, SQRT_Y, T)[rng.next() % 3]
            had_single[q] = True
            circ.gates.append(Gate(kind, q, cycle=t))
        prev_busy = busy
    return circ


def rotation_circuit(rows: int, cols: int, depth: int, seed: int) -> Circuit:
    """Parametrised grid circuit: every single-qubit gate is R(theta, phi).

    R(theta, phi) = exp(-i theta (cos(phi) X + sin(phi) Y) / 2). Each of the `depth` cycles
    holds a rotation layer on all qubits, the cycle's CZ layout (Fig. 7 order) and a second
    rotation layer, so the circuit carries 2 * rows * cols * depth angles. theta is uniform
    in [0, 2 pi) and phi is 0 or pi/2, both from one splitmix64 stream.
    """
    n = rows * cols
    rng = SplitMix64(seed)
    circ = Circuit(n_qubits=n, rows=rows, cols=cols, depth=depth,
                   name=f"rot{rows}x{cols}d{depth}s{seed}")
    p = 0

    def layer(t):
        nonlocal p
        for q in range(n):
            theta = 2.0 * math.pi * rng.uniform()
            phi = 0.0 if (rng.next() & 1) == 0 else math.pi / 2
            circ.gates.append(Gate(RXY, q, theta=theta, phi=phi, param=p, cycle=t))
            p += 1

    for t in range(1, depth + 1):
        layer(t)
        for a, b in layout_pairs(rows, cols, (t - 1) % 8 + 1):
            circ.gates.append(Gate(CZ, a, b, cycle=t))
        layer(t)
    return circ


def worked_example() -> Circuit:
    """The 4-qubit, 8-cycle circuit of Section 3.A (Fig. 2), qubits 1..4 mapped to 0..3."""
    c = Circuit(n_qubits=4, rows=1, cols=4, depth=8, name="worked-example")
    seq = [
        [(H, 0), (H, 1), (H, 2), (H, 3)],
        [(CZ, 0, 1), (SQRT_X, 2), (SQRT_Y, 3)],
        [(T, 0), (T, 1), (CZ, 2, 3)],
        [(CZ, 0, 2), (SQRT_X, 3)],
        [(CZ, 1, 3), (SQRT_X, 0)],
        [(CZ, 1, 2), (SQRT_Y, 0), (SQRT_Y, 3)],
        [(CZ, 0, 3)],
        [(H, 0), (H, 1), (H, 2), (H, 3)],
    ]
    for t, cyc in enumerate(seq):
        for g in cyc:
            c.gates.append(Gate(g[0], g[1], g[2] if len(g) > 2 else -1, cycle=t))
    return c


def random_bitstrings(n_qubits: int, count: int, seed: int) -> list:
    """`count` uniform n-bit strings (bit q = qubit q) from splitmix64(seed): one draw per
    string up to 64 qubits; above that, one draw per 64 bits, lowest word first."""
    rng = SplitMix64(seed)
    mask = (1 << n_qubits) - 1
    words = (n_qubits + 63) // 64
    out = []
    for _ in range(count):
        v = 0
        for w in range(words):
            v |= rng.next() << (64 * w)
        out.append(v & mask)
    return out


def count_gates(circ: Circuit) -> tuple:
    """(single-qubit gates after the first cycle, two-qubit gates): g1 and g2 of Section 5."""
    g1 = sum(1 for g in circ.gates if g.kind in SINGLE_QUBIT and g.cycle > 0)
    g2 = sum(1 for g in circ.gates if g.kind == CZ)
    return g1, g2
