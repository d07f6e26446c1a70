"""Dense statevector simulator, n <= 20 qubits (oracle; test infrastructure only).

The state is a complex128 array of shape [2]*n; axis k is qubit k, so in the
flat 2^n vector qubit k is bit (n-1-k) of the index.  Gates are applied by
contracting their matrix with the qubit axes.  This is the "statevector
simulation" backend the paper compares against (Sec. I, Sec. III).
"""
from __future__ import annotations

import numpy as np

PAULI = [
    np.eye(2, dtype=np.complex128),
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
]

MAX_QUBITS = 20


def zero_state(n: int) -> np.ndarray:
    if n > MAX_QUBITS:
        raise ValueError(f"statevector oracle limited to {MAX_QUBITS} qubits, got {n}")
    psi = np.zeros([2] * n, dtype=np.complex128)
    psi[(0,) * n] = 1.0
    return psi


def apply_1q(psi: np.ndarray, k: int, U: np.ndarray) -> np.ndarray:
    out = np.tensordot(U, psi, axes=([1], [k]))
    return np.moveaxis(out, 0, k)


def apply_2q(psi: np.ndarray, k: int, G: np.ndarray) -> np.ndarray:
    G4 = G.reshape(2, 2, 2, 2)
    out = np.tensordot(G4, psi, axes=([2, 3], [k, k + 1]))
    return np.moveaxis(out, [0, 1], [k, k + 1])


def run(n: int, ops: list) -> np.ndarray:
    psi = zero_state(n)
    for kind, k, M in ops:
        psi = apply_1q(psi, k, M) if kind == "1q" else apply_2q(psi, k, M)
    return psi


def expectation(psi: np.ndarray, ops_on_qubits: dict) -> complex:
    """<psi| O |psi> / <psi|psi> for O a tensor product of 2x2 operators."""
    phi = psi
    for k, M in ops_on_qubits.items():
        phi = apply_1q(phi, k, M)
    return np.vdot(psi, phi) / np.vdot(psi, psi)


def pair_paulis(psi: np.ndarray, pairs: list) -> np.ndarray:
    """Pauli cache ``[m][16]`` (Eq. 5): entry 4a+b = <P_a on i (x) P_b on j>.

    Computed by the definition: apply P_b to qubit j and P_a to qubit i, take
    the inner product with psi.  Index order I, X, Y, Z = 0..3.
    """
    out = np.zeros((len(pairs), 16))
    for q, (i, j) in enumerate(pairs):
        for a in range(4):
            for b in range(4):
                v = expectation(psi, {i: PAULI[a], j: PAULI[b]})
                out[q, 4 * a + b] = v.real
    return out


def schmidt_values(psi: np.ndarray, cut: int) -> np.ndarray:
    """Singular values of psi across the cut between qubits cut and cut+1."""
    n = psi.ndim
    return np.linalg.svd(psi.reshape(2 ** (cut + 1), 2 ** (n - cut - 1)), compute_uv=False)
