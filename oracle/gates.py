"""Gate matrices of the oracle (test infrastructure only).

The paper names the gates H, T, CZ, sqrt(X) and sqrt(Y) (Section 3.A, Eq. 2; Section 4,
rule 3) without writing their matrices. The readings used here:
  H       = [[1, 1], [1, -1]] / sqrt(2)
  T       = diag(1, exp(i pi/4))
  CZ      = diag(1, 1, 1, -1)
  sqrt(X) = principal square root of X = (1/2) [[1+i, 1-i], [1-i, 1+i]]
  sqrt(Y) = principal square root of Y = (1/2) [[1+i, -1-i], [1+i, 1+i]]
  R(theta, phi) = exp(-i theta (cos phi X + sin phi Y) / 2)
               = cos(theta/2) I - i sin(theta/2) (cos phi X + sin phi Y)
Matrices are indexed [output, input].
"""
import math
import numpy as np

import circuitgen as cg

SQ2 = 1.0 / math.sqrt(2.0)
H = np.array([[SQ2, SQ2], [SQ2, -SQ2]], dtype=np.complex128)
T_DIAG = np.array([1.0, np.exp(1j * math.pi / 4)], dtype=np.complex128)
T = np.diag(T_DIAG)
SQRT_X = 0.5 * np.array([[1 + 1j, 1 - 1j], [1 - 1j, 1 + 1j]], dtype=np.complex128)
SQRT_Y = 0.5 * np.array([[1 + 1j, -1 - 1j], [1 + 1j, 1 + 1j]], dtype=np.complex128)
CZ_DIAG = np.array([[1.0, 1.0], [1.0, -1.0]], dtype=np.complex128)  # [bit a, bit b]
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
I2 = np.eye(2, dtype=np.complex128)


def rxy(theta: float, phi: float) -> np.ndarray:
    """exp(-i theta (cos phi X + sin phi Y) / 2), written as cos/sin of theta/2."""
    gen = math.cos(phi) * X + math.sin(phi) * Y
    return math.cos(theta / 2) * I2 - 1j * math.sin(theta / 2) * gen


def drxy_dtheta(theta: float, phi: float) -> np.ndarray:
    """d/dtheta of rxy: -(1/2) sin(theta/2) I - (i/2) cos(theta/2) (cos phi X + sin phi Y)."""
    gen = math.cos(phi) * X + math.sin(phi) * Y
    return -0.5 * math.sin(theta / 2) * I2 - 0.5j * math.cos(theta / 2) * gen


def is_diagonal(kind: int) -> bool:
    return kind in (cg.T, cg.CZ)


def matrix(g) -> np.ndarray:
    """2x2 matrix [out, in] of a single-qubit gate record."""
    if g.kind == cg.H:
        return H
    if g.kind == cg.T:
        return T
    if g.kind == cg.SQRT_X:
        return SQRT_X
    if g.kind == cg.SQRT_Y:
        return SQRT_Y
    if g.kind == cg.RXY:
        return rxy(g.theta, g.phi)
    if g.kind == cg.U1:
        u = g.u
        return np.array([[u[0] + 1j * u[1], u[2] + 1j * u[3]],
                         [u[4] + 1j * u[5], u[6] + 1j * u[7]]], dtype=np.complex128)
    raise ValueError(f"not a single-qubit gate kind: {g.kind}")
