"""Adaptive non-local observables and the linear layer (oracle; test infrastructure only).

Sec. II.A: each observable acts on a pair e_q and is a 4x4 Hermitian matrix
H_q built from real parameter sets A_q (real off-diagonal), B_q (imaginary
off-diagonal) and D_q (diagonal).  Parameter layout per pair, 16 reals:

    A[0..5]  Re H[k][l] for (k,l) = (0,1),(0,2),(0,3),(1,2),(1,3),(2,3)
    B[0..5]  Im H[k][l] for the same (k,l); H[l][k] = conj(H[k][l])
    D[0..3]  H[k][k]

Eq. 4: H_q = sum_alpha c_{q,alpha} P_alpha with c_{q,alpha} = 2^-k Tr(H_q P_alpha),
k = 2, P_alpha = P_a (x) P_b, alpha = 4a + b, I,X,Y,Z = 0..3, P_a on the first
qubit of the pair.  Eq. 5: <H_q> = sum_alpha c_{q,alpha} <P_alpha>.  Eq. 1 is
the same value computed directly as Tr(rho_q H_q).  Eq. 6: y = W q + b.
"""
from __future__ import annotations

import numpy as np

from .statevector import PAULI

UPPER = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]


def hermitian(abd: np.ndarray) -> np.ndarray:
    H = np.zeros((4, 4), dtype=np.complex128)
    for k in range(4):
        H[k, k] = abd[12 + k]
    for u, (k, l) in enumerate(UPPER):
        H[k, l] = abd[u] + 1j * abd[6 + u]
        H[l, k] = np.conj(H[k, l])
    return H


def pauli2(alpha: int) -> np.ndarray:
    return np.kron(PAULI[alpha // 4], PAULI[alpha % 4])


def coefficients(abd: np.ndarray) -> np.ndarray:
    """c_{q,alpha} = 2^-2 Tr(H_q P_alpha) (Eq. 4), real because H_q is Hermitian."""
    H = hermitian(abd)
    c = np.array([np.trace(H @ pauli2(a)) for a in range(16)]) / 4.0
    return c.real


def features(pauli_cache: np.ndarray, abd: np.ndarray) -> np.ndarray:
    """q_q = sum_alpha c_{q,alpha} <P_alpha> (Eq. 5) for one image: [m][16] -> [m]."""
    return np.array([coefficients(abd[q]) @ pauli_cache[q] for q in range(len(pauli_cache))])


def feature_direct(rho: np.ndarray, abd: np.ndarray) -> float:
    """q = Tr(rho H) (Eq. 1) for a 4x4 two-qubit reduced density matrix rho."""
    return float(np.trace(rho @ hermitian(abd)).real)


def rho_from_paulis(p16: np.ndarray) -> np.ndarray:
    """Two-qubit reduced density matrix rebuilt from its 16 Pauli expectations."""
    return sum(p16[a] * pauli2(a) for a in range(16)) / 4.0


def linear(W: np.ndarray, q: np.ndarray, b: np.ndarray) -> np.ndarray:
    """y = W q + b (Eq. 6)."""
    return W @ q + b
