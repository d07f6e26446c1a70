"""Matrix-product-state simulator with SVD truncation (oracle; test infrastructure only).

State (Sec. II.B, Eq. 3):

    |psi> = sum_s A[0]^{s_0} A[1]^{s_1} ... A[n-1]^{s_{n-1}} |s_0 ... s_{n-1}>

stored as a list of complex128 site tensors A[k] of shape (D_left, 2, D_right),
with D_left of site 0 and D_right of site n-1 equal to 1.

One-qubit gates update their site tensor; a nearest-neighbour two-qubit gate
updates the two adjacent tensors and is followed by bond truncation to chi
(Sec. II.B).  The paper does not state the truncation rule; the reading used
here is the standard optimal one, in this order for every two-qubit gate on
sites (k, k+1):

  1. move the orthogonality centre to site k by exact QR / LQ factorisations;
  2. theta = A[k] A[k+1], reshaped to a (2 D_{k-1}) x (2 D_{k+1}) matrix;
  3. apply the 4x4 gate to the two physical indices;
  4. theta = U diag(sigma) V^H (full SVD, numpy / LAPACK);
  5. keep the largest min(chi, 2 D_{k-1}, 2 D_{k+1}) singular values and
     rescale the kept ones to unit 2-norm (renormalisation);
  6. A[k] = U_kept, A[k+1] = diag(sigma_kept) V^H_kept; the centre is now k+1.

No singular-value cutoff is applied.  The discarded weight sum(sigma_dropped^2)
/ sum(sigma^2) of every step is recorded.  Because each truncation happens at
the orthogonality centre, the truncated state equals the truncation of the full
state's Schmidt decomposition across cut k, whatever gauge is used elsewhere.

Expectations (Eq. 5) are contracted with explicit left and right environments
and divided by <psi|psi>, so no canonical form is assumed.
"""
from __future__ import annotations

import numpy as np

from .statevector import PAULI


class MPS:
    def __init__(self, n: int):
        self.n = n
        self.A = []
        for _ in range(n):
            t = np.zeros((1, 2, 1), dtype=np.complex128)
            t[0, 0, 0] = 1.0
            self.A.append(t)
        self.centre = 0  # every site of a product state is both left- and right-orthonormal
        self.discarded = []  # per two-qubit gate: relative discarded weight
        self.min_gap = float("inf")  # smallest (sigma_keep - sigma_keep+1) / sigma_1 at a real cut

    # ---- bonds -------------------------------------------------------------
    def bond_dims(self) -> list:
        """D_k between sites k and k+1, k = 0..n-2."""
        return [self.A[k].shape[2] for k in range(self.n - 1)]

    # ---- gauge moves (exact) ----------------------------------------------
    def _shift_right(self):
        c = self.centre
        Dl, _, Dr = self.A[c].shape
        Q, R = np.linalg.qr(self.A[c].reshape(Dl * 2, Dr))
        self.A[c] = Q.reshape(Dl, 2, Q.shape[1])
        self.A[c + 1] = np.einsum("ab,bsr->asr", R, self.A[c + 1])
        self.centre = c + 1

    def _shift_left(self):
        c = self.centre
        Dl, _, Dr = self.A[c].shape
        # LQ of the Dl x (2 Dr) matrix via QR of its conjugate transpose.
        Q, R = np.linalg.qr(self.A[c].reshape(Dl, 2 * Dr).conj().T)
        self.A[c] = Q.conj().T.reshape(Q.shape[1], 2, Dr)
        self.A[c - 1] = np.einsum("lsa,ab->lsb", self.A[c - 1], R.conj().T)
        self.centre = c - 1

    def move_centre(self, k: int):
        while self.centre < k:
            self._shift_right()
        while self.centre > k:
            self._shift_left()

    # ---- gates ---------------------------------------------------------------
    def apply_1q(self, k: int, U: np.ndarray):
        self.A[k] = np.einsum("st,ltr->lsr", U, self.A[k])

    def apply_2q(self, k: int, G: np.ndarray, chi: int):
        self.move_centre(k)
        a, b = self.A[k], self.A[k + 1]
        Dl, Dr = a.shape[0], b.shape[2]
        theta = np.einsum("lsm,mtr->lstr", a, b)
        theta = np.einsum("stuv,luvr->lstr", G.reshape(2, 2, 2, 2), theta)
        M = theta.reshape(2 * Dl, 2 * Dr)
        U, S, Vh = np.linalg.svd(M, full_matrices=False)
        keep = min(chi, 2 * Dl, 2 * Dr)
        total = float(np.sum(S ** 2))
        kept = S[:keep]
        if len(S) > keep and S[keep] > 1e-13 * S[0]:
            self.min_gap = min(self.min_gap, float((S[keep - 1] - S[keep]) / S[0]))
        self.discarded.append(float(np.sum(S[keep:] ** 2)) / total if total > 0 else 0.0)
        kept = kept / np.linalg.norm(kept)
        self.A[k] = U[:, :keep].reshape(Dl, 2, keep)
        self.A[k + 1] = (kept[:, None] * Vh[:keep, :]).reshape(keep, 2, Dr)
        self.centre = k + 1

    def run(self, ops: list, chi: int):
        for kind, k, M in ops:
            if kind == "1q":
                self.apply_1q(k, M)
            else:
                self.apply_2q(k, M, chi)
        return self

    # ---- contraction ---------------------------------------------------------
    def to_statevector(self) -> np.ndarray:
        v = self.A[0].reshape(2, -1)
        for k in range(1, self.n):
            v = np.einsum("xa,asr->xsr", v, self.A[k]).reshape(-1, self.A[k].shape[2])
        return v.reshape([2] * self.n)

    def _left_envs(self) -> list:
        """left[i] = contraction of sites < i with their conjugates, (bra, ket)."""
        left = [np.ones((1, 1), dtype=np.complex128)]
        for k in range(self.n):
            A = self.A[k]
            left.append(np.einsum("lsr,lm,msq->rq", A.conj(), left[-1], A))
        return left

    def _right_envs(self) -> list:
        """right[j] = contraction of sites > j with their conjugates, (bra, ket)."""
        right = [None] * self.n
        right[self.n - 1] = np.ones((1, 1), dtype=np.complex128)
        for k in range(self.n - 1, 0, -1):
            A = self.A[k]
            right[k - 1] = np.einsum("lsr,rq,msq->lm", A.conj(), right[k], A)
        return right

    def pair_paulis(self, pairs: list, return_imag: bool = False):
        """Pauli cache ``[m][16]`` (Eq. 5), entry 4a+b = <P_a(i) P_b(j)>, i < j."""
        left = self._left_envs()
        right = self._right_envs()
        norm = left[self.n][0, 0].real
        out = np.zeros((len(pairs), 16))
        imag = np.zeros((len(pairs), 16))
        for q, (i, j) in enumerate(pairs):
            if not i < j:
                raise ValueError("pairs must satisfy i < j")
            Ai, Aj = self.A[i], self.A[j]
            for a in range(4):
                E = np.einsum("lsr,lm,st,mtq->rq", Ai.conj(), left[i], PAULI[a], Ai, optimize=True)
                for k in range(i + 1, j):
                    Ak = self.A[k]
                    E = np.einsum("lsr,lm,msq->rq", Ak.conj(), E, Ak, optimize=True)
                for b in range(4):
                    v = np.einsum("lm,lsr,st,mtq,rq->", E, Aj.conj(), PAULI[b], Aj, right[j], optimize=True)
                    out[q, 4 * a + b] = v.real / norm
                    imag[q, 4 * a + b] = v.imag / norm
        return (out, imag) if return_imag else out

    def norm_sq(self) -> float:
        return self._left_envs()[self.n][0, 0].real


def simulate(ops: list, n: int, chi: int) -> MPS:
    return MPS(n).run(ops, chi)
