"""Per-image oracle pipeline (test infrastructure only).

image x -> gate list (Sec. II.B, Eq. 2) -> state (statevector for n <= 20, or
MPS with truncation to chi, Eq. 3) -> Pauli cache over image-local pairs
(Sec. II.C, Eq. 5) -> ANO features (Eq. 4-5) -> linear layer (Eq. 6).
"""
from __future__ import annotations

import numpy as np

from . import ano, circuit, mps, pairs, statevector


def pauli_cache(x, p: int, L: int, chi: int, ansatz: str = "ladder", params=None,
                diagonals: bool = False, backend: str = "mps", return_state: bool = False):
    """Pauli cache ``[m][16]`` of one p x p image (x: ``[p*p]`` in [0,1])."""
    x = np.asarray(x, dtype=np.float64)
    n = p * p
    if x.shape != (n,):
        raise ValueError("x must hold p*p pixels")
    ops = circuit.build_circuit(ansatz, x, L, params)
    prs = pairs.image_pairs(p, diagonals)
    if backend == "statevector":
        psi = statevector.run(n, ops)
        out = statevector.pair_paulis(psi, prs)
        return (out, psi) if return_state else out
    state = mps.simulate(ops, n, chi)
    out = state.pair_paulis(prs)
    return (out, state) if return_state else out


def features(cache: np.ndarray, abd: np.ndarray) -> np.ndarray:
    return ano.features(cache, abd)


def reconstruct(cache: np.ndarray, abd: np.ndarray, W: np.ndarray, b: np.ndarray):
    q = ano.features(cache, abd)
    return q, ano.linear(W, q, b)


def _worker(args):
    x, p, L, chi, ansatz, params = args
    return pauli_cache(x, p, L, chi, ansatz, params)


def pauli_cache_batch(X, p: int, L: int, chi: int, ansatz: str = "ladder", params=None,
                      processes: int = 1):
    """Pauli caches for a batch ``[B][p*p]`` -> ``[B][m][16]``.

    With processes > 1 the images are spread over a ``spawn`` process pool
    (one BLAS thread per worker is the caller's responsibility).
    """
    jobs = [(np.asarray(x), p, L, chi, ansatz, params) for x in X]
    if processes <= 1:
        return np.stack([_worker(j) for j in jobs])
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(processes) as pool:
        return np.stack(pool.map(_worker, jobs, chunksize=1))
