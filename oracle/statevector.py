"""State-vector simulation of Eq. (1) in complex128 (test infrastructure only).

<x|C|0...0> is evaluated as the definition reads: start from |0...0>, apply the gates in
time order to the 2^N amplitudes, read entry x. Basis index bit q is the value of qubit q.
Also the adjoint gradient d<x|C|0>/d theta_g for parametrised gates R(theta, phi).
Usable up to N of about 28 (2^28 complex128 = 4 GiB).
"""
import numpy as np

import circuitgen as cg
from . import gates as G


def _apply_1q(psi: np.ndarray, u: np.ndarray, q: int, n: int) -> np.ndarray:
    v = psi.reshape(1 << (n - q - 1), 2, 1 << q)
    return np.einsum("ij,ajb->aib", u, v).reshape(-1)


def _apply_cz(psi: np.ndarray, a: int, b: int, n: int) -> np.ndarray:
    idx = np.arange(1 << n, dtype=np.int64)
    both = ((idx >> a) & 1) & ((idx >> b) & 1)
    out = psi.copy()
    out[both == 1] *= -1.0
    return out


def apply_gate(psi: np.ndarray, g, n: int, u=None) -> np.ndarray:
    if g.kind == cg.CZ:
        return _apply_cz(psi, g.q0, g.q1, n)
    return _apply_1q(psi, G.matrix(g) if u is None else u, g.q0, n)


def final_state(circ) -> np.ndarray:
    n = circ.n_qubits
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    for g in circ.gates:
        psi = apply_gate(psi, g, n)
    return psi


def sv_amplitude(circ, x: int) -> complex:
    """<x|C|0...0> by direct state-vector evolution."""
    return complex(final_state(circ)[x])


def sv_adjoint_grad(circ, x: int):
    """(alpha, grad) with grad[p] = d alpha / d theta_p over the gates with param p >= 0.

    alpha = <x| U_G ... U_1 |0>. For gate g, d alpha / d theta_g = <lambda_g| dU_g |psi_{g-1}>
    with psi_{g-1} = U_{g-1} ... U_1 |0> and <lambda_g| = <x| U_G ... U_{g+1}. The sweep walks
    the gates backwards, undoing each U_g on psi and moving lambda through U_g^dagger.
    Gates sharing one parameter index add their contributions.
    """
    n = circ.n_qubits
    psi = final_state(circ)
    alpha = complex(psi[x])
    lam = np.zeros(1 << n, dtype=np.complex128)
    lam[x] = 1.0                       # lam holds the ket (U_G...U_{g+1})^dagger |x>
    grad = np.zeros(circ.n_params, dtype=np.complex128)
    for g in reversed(circ.gates):
        if g.kind == cg.CZ:
            psi = _apply_cz(psi, g.q0, g.q1, n)          # CZ is its own inverse
            lam = _apply_cz(lam, g.q0, g.q1, n)
            continue
        u = G.matrix(g)
        psi = _apply_1q(psi, u.conj().T, g.q0, n)         # psi_{g-1}
        if g.param >= 0:
            du = G.drxy_dtheta(g.theta, g.phi)
            grad[g.param] += np.vdot(lam, _apply_1q(psi, du, g.q0, n))
        lam = _apply_1q(lam, u.conj().T, g.q0, n)
    return alpha, grad


def with_thetas(circ, thetas):
    """Copy of `circ` whose parametrised gates take angles from `thetas`."""
    out = cg.Circuit(n_qubits=circ.n_qubits, rows=circ.rows, cols=circ.cols,
                     depth=circ.depth, name=circ.name)
    for g in circ.gates:
        h = cg.Gate(g.kind, g.q0, g.q1, g.theta, g.phi, g.param, g.u, g.cycle)
        if g.param >= 0:
            h.theta = float(thetas[g.param])
        out.gates.append(h)
    return out
