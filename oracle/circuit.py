"""Gate matrices and ordered gate lists (oracle; test infrastructure only).

Qubit k is pixel (r, c) = (k // p, k % p): the p x p image is flattened
row-major onto a chain (Sec. II.B).  A gate list is a list of tuples

    ("1q", k, U)   U a 2x2 unitary acting on qubit k
    ("2q", k, G)   G a 4x4 unitary on qubits (k, k+1); basis index 2*s_k + s_{k+1}

applied in list order.

Two ansaetze:

* ``ladder`` (the benchmark circuit): R_Y(pi x_k) on every qubit once, then
  L layers of [R_Y(alpha_{l,k}) then R_Z(beta_{l,k}) on every qubit, then
  CNOT(k -> k+1) for k = 0, 1, ..., n-2 in that order].
* ``paper`` (Sec. II.B, Eq. 2): L repetitions of [H on every qubit, then
  R_Y(phi_k) with phi_k = 2 pi x_k - pi (Eq. 2), then nearest-neighbour CNOTs
  in a staggered pattern: bonds (0,1), (2,3), ... in ascending order, then
  bonds (1,2), (3,4), ... in ascending order].  The paper fixes neither the
  CNOT direction nor the order inside a staggered sub-layer; here the control
  is the lower chain index and both sub-layers run in ascending order.
"""
from __future__ import annotations

import numpy as np


def ry(theta: float) -> np.ndarray:
    """R_Y(theta) = exp(-i theta Y / 2)."""
    c, s = np.cos(theta / 2.0), np.sin(theta / 2.0)
    return np.array([[c, -s], [s, c]], dtype=np.complex128)


def rz(theta: float) -> np.ndarray:
    """R_Z(theta) = exp(-i theta Z / 2)."""
    return np.array([[np.exp(-0.5j * theta), 0.0], [0.0, np.exp(0.5j * theta)]],
                    dtype=np.complex128)


HADAMARD = np.array([[1.0, 1.0], [1.0, -1.0]], dtype=np.complex128) / np.sqrt(2.0)

# CNOT with the control on the first qubit of the pair: |a, b> -> |a, b xor a>.
CNOT = np.zeros((4, 4), dtype=np.complex128)
for _a in range(2):
    for _b in range(2):
        CNOT[2 * _a + (_b ^ _a), 2 * _a + _b] = 1.0


def ladder_circuit(x: np.ndarray, L: int, params: np.ndarray) -> list:
    """Benchmark ansatz for one image: x ``[n]`` in [0,1], params ``[L][>=n][2]``."""
    n = len(x)
    ops = [("1q", k, ry(np.pi * x[k])) for k in range(n)]
    for layer in range(L):
        for k in range(n):
            ops.append(("1q", k, ry(params[layer][k][0])))
            ops.append(("1q", k, rz(params[layer][k][1])))
        for k in range(n - 1):
            ops.append(("2q", k, CNOT))
    return ops


def paper_circuit(x: np.ndarray, L: int) -> list:
    """Paper ansatz for one image (Sec. II.B, Eq. 2), L encoding-entangling layers."""
    n = len(x)
    ops = []
    for _ in range(L):
        for k in range(n):
            ops.append(("1q", k, HADAMARD))
        for k in range(n):
            ops.append(("1q", k, ry(2.0 * np.pi * x[k] - np.pi)))
        for k in range(0, n - 1, 2):
            ops.append(("2q", k, CNOT))
        for k in range(1, n - 1, 2):
            ops.append(("2q", k, CNOT))
    return ops


def build_circuit(ansatz: str, x: np.ndarray, L: int, params=None) -> list:
    if ansatz == "ladder":
        return ladder_circuit(x, L, params)
    if ansatz == "paper":
        return paper_circuit(x, L)
    raise ValueError(f"unknown ansatz {ansatz!r}")
