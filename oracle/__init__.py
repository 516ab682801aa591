"""CPU oracle for single-amplitude simulation (TEST INFRASTRUCTURE ONLY).

This package is the independent, plain, slow and obviously correct reference that the
GPU library is checked against. It shares no code with the GPU path: its gate matrices,
graph construction and elimination loop are written here from the paper's definitions.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import it. The
product path never does.

Contents
  gates        gate matrices (the readings of sqrt(X), sqrt(Y), T, H, CZ, R(theta, phi))
  statevector  complex128 state-vector simulation of Eq. (1) and its adjoint gradient
  graph        the undirected graphical model of Section 3.A and its vertex operations
  ve           bucket (variable) elimination of Section 3.B.1 with the slicing of 3.B.2,
               complex128, loops written out in C (ve.c) and driven from Python

Parity pins (tests/test_oracle_*.py): the worked example's graph (Fig. 4), the graph
operations of Figs. 5-6, closed-form amplitudes, normalisation, state vector vs
elimination, order and slice invariance, finite differences for the gradient. The
absolute phase convention of sqrt(X) and sqrt(Y) is a reading, not a paper value:
"parity unpinned" for that phase only (|amplitude| is pinned).
"""
from . import gates, graph, statevector, ve  # noqa: F401
