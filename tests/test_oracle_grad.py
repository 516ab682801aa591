"""Oracle gradient: adjoint sweep vs closed forms and central differences."""
import math

import numpy as np

import circuitgen as cg
from oracle import gates as G
from oracle import statevector as SV
from oracle import ve as VE


def test_gate_matrix_identities():
    for u in (G.H, G.T, G.SQRT_X, G.SQRT_Y, G.rxy(1.3, 0.0), G.rxy(2.1, math.pi / 2)):
        assert np.allclose(u.conj().T @ u, np.eye(2), atol=1e-15)
    assert np.allclose(G.SQRT_X @ G.SQRT_X, G.X, atol=1e-15)
    assert np.allclose(G.SQRT_Y @ G.SQRT_Y, G.Y, atol=1e-15)
    assert np.allclose(G.T @ G.T, np.diag([1, 1j]), atol=1e-15)
    assert np.allclose(G.rxy(math.pi, 0.0), -1j * G.X, atol=1e-15)
    assert np.allclose(G.rxy(math.pi, math.pi / 2), -1j * G.Y, atol=1e-15)
    for th, ph in ((0.3, 0.0), (2.5, math.pi / 2)):
        h = 1e-6
        fd = (G.rxy(th + h, ph) - G.rxy(th - h, ph)) / (2 * h)
        assert np.allclose(fd, G.drxy_dtheta(th, ph), atol=1e-9)


def test_single_rotation_closed_form():
    th = 0.9
    c = cg.Circuit(n_qubits=1, gates=[cg.Gate(cg.RXY, 0, theta=th, phi=0.0, param=0)])
    a0, g0 = SV.sv_adjoint_grad(c, 0)
    a1, g1 = SV.sv_adjoint_grad(c, 1)
    assert abs(a0 - math.cos(th / 2)) < 1e-15 and abs(g0[0] + 0.5 * math.sin(th / 2)) < 1e-15
    assert abs(a1 + 1j * math.sin(th / 2)) < 1e-15 and abs(g1[0] + 0.5j * math.cos(th / 2)) < 1e-15


def test_adjoint_matches_central_differences():
    c = cg.rotation_circuit(2, 3, 4, 12)
    x = 0b101101
    alpha, grad = SV.sv_adjoint_grad(c, x)
    th = np.array(c.thetas())
    h = 1e-4
    for p in range(len(th)):
        tp, tm = th.copy(), th.copy()
        tp[p] += h
        tm[p] -= h
        fd = (VE.ve_amplitude(SV.with_thetas(c, tp), x) -
              VE.ve_amplitude(SV.with_thetas(c, tm), x)) / (2 * h)
        assert abs(fd - grad[p]) < 1e-8, p
    assert abs(alpha - VE.ve_amplitude(c, x)) < 1e-14
