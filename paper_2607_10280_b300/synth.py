"""Seeded synthetic inputs shared by the CUDA path, its tests and the oracle.

This module holds input generation only: pixel images, circuit rotation
parameters, observable parameters, linear-layer weights and serving arrivals.
It contains none of the method's arithmetic (no gates, no contractions, no
Pauli algebra), so both the CUDA path and the oracle may import it.

The paper trains on Fashion-MNIST 7x7 inputs (Sec. II.B, Sec. II.D).  The
dataset is not available here; ``garment_pixels`` is a synthetic stand-in with
the same shape and value range: a zero background with one to three Gaussian
blobs whose amplitudes lie in [0.3, 1], clipped to [0, 1].

Seeds (one PCG64 stream per role): pixels 0, circuit parameters 1, observable
parameters 2, linear layer 3, serving arrivals 4.
"""
from __future__ import annotations

import numpy as np

SEED_PIXELS = 0
SEED_PARAMS = 1
SEED_ABD = 2
SEED_LINEAR = 3
SEED_ARRIVALS = 4


def _rng(seed: int, *salt: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([int(seed), *[int(s) for s in salt]]))


def uniform_pixels(batch: int, p: int, seed: int = SEED_PIXELS) -> np.ndarray:
    """i.i.d. U[0,1] pixels, float64 ``[batch][p*p]`` in row-major pixel order."""
    return _rng(seed, p).random((batch, p * p))


def garment_pixels(batch: int, p: int, seed: int = SEED_PIXELS) -> np.ndarray:
    """Garment-like p x p images, float64 ``[batch][p*p]`` row-major.

    Per image: K ~ U{1,2,3} isotropic Gaussian blobs with centre ~ U[0,p)^2,
    width ~ U[0.15p, 0.35p] and amplitude ~ U[0.3,1], summed on a zero
    background and clipped to [0,1].
    """
    rng = _rng(seed, p, 1)
    rr, cc = np.meshgrid(np.arange(p), np.arange(p), indexing="ij")
    out = np.zeros((batch, p * p))
    for b in range(batch):
        img = np.zeros((p, p))
        for _ in range(int(rng.integers(1, 4))):
            cy, cx = rng.uniform(0, p, size=2)
            w = rng.uniform(0.15 * p, 0.35 * p)
            a = rng.uniform(0.3, 1.0)
            img += a * np.exp(-((rr - cy) ** 2 + (cc - cx) ** 2) / (2.0 * w * w))
        out[b] = np.clip(img, 0.0, 1.0).reshape(-1)
    return out


def circuit_params(L: int, n: int, seed: int = SEED_PARAMS) -> np.ndarray:
    """Rotation angles ``[L][n][2]`` ~ U[0, 2pi): (alpha for R_Y, beta for R_Z).

    One draw per (layer, qubit), shared by every image of a batch.  An image
    with n_i <= n qubits and L_i <= L layers uses the leading entries.
    """
    return _rng(seed, L, n).uniform(0.0, 2.0 * np.pi, size=(L, n, 2))


def observable_params(m: int, seed: int = SEED_ABD) -> np.ndarray:
    """Observable parameters ``[m][16]`` ~ N(0,1): A (6 real off-diagonal),
    B (6 imaginary off-diagonal), D (4 diagonal), per image-local pair."""
    return _rng(seed, m).standard_normal((m, 16))


def linear_params(out_dim: int, m: int, seed: int = SEED_LINEAR):
    """Linear layer W ``[out_dim][m]`` ~ N(0, 1/m) and bias ``[out_dim]``.

    The bias is drawn ~ N(0, 0.01) so that tests exercise it; benchmarks may
    zero it.
    """
    rng = _rng(seed, out_dim, m)
    W = rng.standard_normal((out_dim, m)) / np.sqrt(m)
    b = 0.1 * rng.standard_normal(out_dim)
    return W, b


def uneven_sizes(batch: int, lo: int = 4, hi: int = 16, seed: int = SEED_PIXELS) -> np.ndarray:
    """Image side lengths p ~ U{lo..hi}, int32 ``[batch]``."""
    return _rng(seed, lo, hi, 7).integers(lo, hi + 1, size=batch).astype(np.int32)


def uneven_pixels(sizes, seed: int = SEED_PIXELS) -> list:
    """Garment-like pixels for a batch of mixed sizes: list of float64 arrays."""
    out = []
    for i, p in enumerate(np.asarray(sizes).tolist()):
        out.append(garment_pixels(1, int(p), seed=seed * 1000003 + i)[0])
    return out


def serving_requests(count: int, rate_hz: float = 2000.0,
                     p_choices=tuple(range(6, 17)), L_choices=(1, 2, 3, 4),
                     chi_choices=(4, 8, 16, 32), seed: int = SEED_ARRIVALS):
    """Poisson arrivals of single-image requests with a uniform (p, L, chi) mix.

    Returns a list of dicts with keys ``t`` (arrival time in seconds from 0),
    ``p``, ``L``, ``chi`` and ``pixels`` (float64 ``[p*p]``).
    """
    rng = _rng(seed, count)
    gaps = rng.exponential(1.0 / rate_hz, size=count)
    t = np.cumsum(gaps) - gaps[0]
    reqs = []
    for i in range(count):
        p = int(rng.choice(p_choices))
        reqs.append({
            "id": i,
            "t": float(t[i]),
            "p": p,
            "L": int(rng.choice(L_choices)),
            "chi": int(rng.choice(chi_choices)),
            "pixels": garment_pixels(1, p, seed=seed * 7919 + i)[0],
        })
    return reqs
