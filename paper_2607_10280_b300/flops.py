"""Algorithmic flop counts of the CUDA kernels, per image, from the bond schedule.

Real flops; a complex multiply-add counts 8.  The counts follow the work each
kernel performs on the true bond dimensions (no padding, no idle lanes):

circuit  per two-qubit step on theta = (2 Dl) x (2 Dr) with inner bond Dm:
           one-qubit gate on the loaded site      8 * 4 * Dm * Dr
           theta = A_k A_{k+1}                    8 * M * N * Dm       (M = 2 Dl, N = 2 Dr)
           exact split, N <= M (Householder QR and explicit Q)
                                                  2 * 8 * (M N^2 - N^3 / 3)
           exact split, M < N                     0                    (A_k = identity)
           truncated split (K = min(M, N) > chi)  Gram 4 K^2 max(M, N), Jacobi
                                                  48 K per rotation over the measured
                                                  sweeps (6 assumed), U^H theta 8 chi M N
         per centre move of a (2 Dl) x Dm site     QR + Q + R * next site
renv     per site                                 8 * (2 Dl Dr^2 + 2 Dl^2 Dr)
pauli    per column unit: E_a and closings at its sites, the carried closing
         matrices through p - 1 sites per row     3 * 8 * (2 Dl Dr^2 + 2 Dl^2 Dr)
sweep    per site of the per-image sweep (sweep_flops): E_a once, the closing sums,
         and one stacked transfer of R and every carried (M, C_Z) pair

Circuits without truncation and 2^L <= min(chi, padding, 16) take the
operator-product path (ladder_mpo.cu): bond 2^L at every inner cut, the circuit
only applies one-qubit gates (32 Dl Dr per site and layer; the CNOT ladder copies
entries), the environment launch adds left environments at the cost of the right
ones, and each E_a of the Pauli kernel first forms L A (8 * 2 Dl^2 Dr).  For the
ladder every site but the last is half-structured (A[2l+s][r] = 0 unless r is in
half s of the right bond), and the transfers, right closings and right-environment
steps contract half of it.
"""
from __future__ import annotations

from functools import lru_cache


def _qr_flops(M: int, N: int) -> float:
    K = min(M, N)
    # complex Householder QR of M x N with K reflectors, plus forming the M x K factor
    return 8.0 * (M * N * K - (M + N) * K * K / 2 + K ** 3 / 3) * 2


@lru_cache(maxsize=None)
def circuit_schedule(n: int, L: int, chi: int, ansatz: str = "ladder") -> tuple:
    """Steps of the circuit kernel: tuples (kind, Dl, Dm, Dr, new_bond), kind in
    {'gate', 'move', 'lq'}; plus the final bond dimensions."""
    bd = [1] * (n + 1)
    steps = []

    def run_pass(first: int, stride: int, fresh: bool):
        trunc = False
        dl = bd[first]
        for k in range(first, n - 1):
            if (k - first) % stride == 0:
                mn = min(2 * dl, 2 * bd[k + 2])
                trunc |= mn > chi
                dl = min(mn, chi)
            else:
                dl = min(2 * dl, bd[k + 1])
        if trunc and not fresh:
            for k in range(n - 1, first, -1):
                nb = min(bd[k], 2 * bd[k + 1])
                steps.append(("lq", bd[k - 1], bd[k], bd[k + 1], nb))
                bd[k] = nb
        for k in range(first, n - 1):
            if (k - first) % stride == 0:
                M, N = 2 * bd[k], 2 * bd[k + 2]
                nb = min(chi, M, N)
                steps.append(("gate", bd[k], bd[k + 1], bd[k + 2], nb))
            else:
                nb = min(2 * bd[k], bd[k + 1])
                steps.append(("move", bd[k], bd[k + 1], bd[k + 2], nb))
            bd[k + 1] = nb

    for layer in range(L):
        if ansatz == "ladder":
            run_pass(0, 1, layer == 0)
        else:
            run_pass(0, 2, layer == 0)
            if n > 2:
                run_pass(1, 2, False)
    return tuple(steps), tuple(bd)


def _jacobi_flops(K: int, sweeps: float) -> float:
    """Cyclic Jacobi on a K x K Hermitian matrix: per rotation two columns of G and of
    V and two rows of G (6 K complex rotation updates, 8 real flops each)."""
    return sweeps * (K * (K - 1) / 2) * 48.0 * K


def circuit_flops_by_pipe(n: int, L: int, chi: int, ansatz: str = "ladder", chain: str = "c64",
                          jacobi_sweeps: float = 6.0, refine_sweeps: float = 2.0) -> dict:
    """Flops of the sequential circuit kernel per image, split by the pipe that runs
    them: {"fp32": ..., "fp64": ...}.

    chain "c64": complex64 state (MPS_MIXED_FAST, and the exact-regime sequential
    kernel of MPS_MIXED): gates, theta, QR/LQ in FP32; inside a truncation the Gram
    matrix, U (re-orthogonalised by an FP64 QR) and U^H theta in FP64, the Jacobi
    eigensolver in FP32.
    chain "fp64": complex128 state (a truncating chain of MPS_MIXED, and MPS_FP64):
    everything in FP64 except, up to bond 16, the FP32 Jacobi that starts the
    eigen-decomposition, which then costs an FP64 Cholesky QR of the K x K vectors
    (4 K^3), the transform W^H G W (16 K^3) and `refine_sweeps` rotating FP64 sweeps."""
    steps, _ = circuit_schedule(n, L, chi, ansatz)
    f32 = f64 = 0.0
    state64 = chain == "fp64"
    for kind, Dl, Dm, Dr, nb in steps:
        if kind == "gate":
            M, N = 2 * Dl, 2 * Dr
            g = 32.0 * Dm * Dr + 8.0 * M * N * Dm
            if min(M, N) <= chi:
                if N <= M:
                    g += _qr_flops(M, N)
                if state64:
                    f64 += g
                else:
                    f32 += g
            else:
                K = min(M, N)
                gram = 4.0 * K * K * max(M, N)
                uht = 8.0 * chi * M * N
                right = 8.0 * M * chi * N + _qr_flops(M, chi) if M > N else 0.0
                if state64:
                    f64 += g + gram + uht + right
                    if K <= 32:   # bond <= 16: FP32 Jacobi, then the FP64 refinement
                        f32 += _jacobi_flops(K, jacobi_sweeps)
                        f64 += 4.0 * K ** 3 + 16.0 * K ** 3 + _jacobi_flops(K, refine_sweeps)
                    else:
                        f64 += _jacobi_flops(K, jacobi_sweeps)
                else:
                    f32 += g + _jacobi_flops(K, jacobi_sweeps)
                    f64 += gram + uht + right + (0.0 if M > N else _qr_flops(M, chi))
        elif kind == "move":
            M, N = 2 * Dl, Dm
            g = _qr_flops(M, N) + 8.0 * nb * Dm * 2 * Dr
            if state64:
                f64 += g
            else:
                f32 += g
        else:  # lq of site (Dl x 2 Dr) and site_{k-1} * L
            g = _qr_flops(2 * Dr, Dm) + 8.0 * 2 * Dl * Dm * nb
            if state64:
                f64 += g
            else:
                f32 += g
    return {"fp32": f32, "fp64": f64}


def circuit_flops(n: int, L: int, chi: int, ansatz: str = "ladder", jacobi_sweeps: int = 6) -> float:
    """All flops of the complex64-state sequential circuit kernel per image."""
    d = circuit_flops_by_pipe(n, L, chi, ansatz, "c64", jacobi_sweeps)
    return d["fp32"] + d["fp64"]


def lossy(p: int, L: int, chi: int) -> bool:
    """Whether a ladder circuit truncates lossily (its exact bond min(2^L, 2^floor(n/2))
    exceeds chi), so that MPS_MIXED runs it on a complex128 state."""
    n = p * p
    return min(1 << min(L, 30), 1 << min(n // 2, 30)) > chi


HALF_SPLIT_MIN = 8   # pauli.cuh: split contractions of half-structured sites from this bond on


def renv_flops(bonds, half: bool = False) -> float:
    """half: every site but the last is half-structured (its contractions over the
    right index run over half of it from bond HALF_SPLIT_MIN on, pauli.cuh times_site_t)."""
    n = len(bonds) - 1
    return sum(_transfer(bonds[j], bonds[j + 1], half and j < n - 1 and bonds[j + 1] >= HALF_SPLIT_MIN)
               for j in range(n))


def _transfer(Dl: int, Dr: int, half: bool = False, diag_out: bool = False) -> float:
    """One matrix through a site: C A^T (Dr x 2Dl x Dr) then sum_s conj(A^s) (C A^T)^s
    (Dl x Dl x 2Dr); on a half-structured site only the diagonal blocks of C enter the
    first product (a quarter) and half of the right index the second (a half);
    diag_out: only the diagonal blocks of the result are formed (half the second)."""
    return 8.0 * (2 * Dl * Dr * Dr * (0.25 if half else 1.0)
                  + 2 * Dl * Dl * Dr * (0.5 if half else 1.0) * (0.5 if diag_out else 1.0))


def pauli_flops(p: int, bonds, lenv: bool = False, half: bool = False) -> float:
    """Flops of the Pauli kernel for one image (all p column units); lenv: the image
    brings left environments (each E_a first forms L A); half: every site but the last
    is half-structured (transfers and right closings contract half the right index)."""
    f = 0.0
    n = len(bonds) - 1

    def hf(k):
        return 0.5 if half and k < n - 1 and bonds[k + 1] >= HALF_SPLIT_MIN else 1.0

    def hq(k):   # E_a of a half-structured site: one compact Dr x Dr block product
        return 0.25 if half and k < n - 1 else 1.0

    def env_a(Dl, Dr):
        return 8.0 * 2 * Dl * Dl * Dr if lenv else 0.0

    def transfer(Dl, Dr, k, last):  # C <- sum_s conj(A^s) C A^{sT} through site k
        dout = half and not last and bonds[k] >= HALF_SPLIT_MIN   # next: through site k - 1
        return _transfer(Dl, Dr, half and k < n - 1 and Dr >= HALF_SPLIT_MIN, dout)

    for c in range(p):
        for row in range(p - 1, -1, -1):
            j = row * p + c
            Dl, Dr = bonds[j], bonds[j + 1]
            f += (3 * 8.0 * Dr * Dr * 2 * Dl + env_a(Dl, Dr)) * hq(j)   # E_a
            f += 3 * 8.0 * Dr * Dr                   # <E_a, R>
            if row < p - 1:
                f += 9 * 8.0 * Dr * Dr               # vertical closing
            f += 8.0 * (2 * Dl * Dr * Dr + 3 * Dl * Dl * Dr) * hf(j)   # right closings
            if c == 0 and row == 0:
                break
            k0 = j - 1
            if c > 0:
                D0 = bonds[k0]
                f += (3 * 8.0 * Dl * Dl * 2 * D0 + env_a(D0, Dl)) * hq(k0) + 12 * 8.0 * Dl * Dl
            if row == 0:
                break
            for k in range(k0, j - p, -1):
                # two carried matrices: M = C_X + i C_Y and C_Z
                f += 2 * transfer(bonds[k], bonds[k + 1], k, k == j - p + 1)
    return f


def sweep_flops(p: int, bonds, lenv: bool = False, half: bool = False, diag: bool = False) -> float:
    """Flops of the per-image sweep Pauli kernel (pauli_sweep.cuh) for one image, step by
    step as it runs: left blocks E_a of each site once (with L_k first when lenv; stored
    by the left chain at half-structured sites), the closing sums, and the stacked
    transfer of R and of every carried closing matrix (M, C_Z), with the closings of the
    site formed from the R rows."""
    n = p * p
    ns = p + (1 if diag else 0)

    def half_tr(i):
        return half and i < n - 1 and bonds[i + 1] >= HALF_SPLIT_MIN

    def half_at(i):
        return half and i < n - 1 and bonds[i + 1] >= 2

    def uses(o):
        r, c = divmod(o, p)
        u = []
        if c >= 1:
            u.append(o - 1)
        if r >= 1:
            u.append(o - p)
        if diag and r >= 1 and c <= p - 2:
            u.append(o - p + 1)
        if diag and r >= 1 and c >= 1:
            u.append(o - p - 1)
        return u

    f = 0.0
    for k in range(n - 1, -1, -1):
        Dl, Dr = bonds[k], bonds[k + 1]
        row, col = divmod(k, p)
        if half_at(k):
            # compact F' (Dr x Dr over Dl): with left environments the left chain stores it
            # on its way (lenv_flops), else formed here
            f += 0.0 if lenv else 8.0 * Dr * Dr * Dl
        else:            # the four blocks F_ss' (2Dr x 2Dr over Dl), after T = L A
            f += 8.0 * 4 * Dr * Dr * Dl + (8.0 * Dl * Dl * 2 * Dr if lenv else 0.0)
        sets = (col < p - 1) + (row < p - 1) + (diag and row < p - 1 and col < p - 1) + \
            (diag and row < p - 1 and col >= 1)
        f += 4.0 * Dr * Dr * (3 + 12 * sets)          # Re(E_a Y) sums
        htr = half_tr(k)
        K1 = Dr // 2 if htr else Dr
        dg = k >= 1 and half_tr(k - 1) and Dl % 2 == 0
        carried = [o for o in range(k + 1, min(k + ns - 1, n - 1) + 1) if uses(o) and min(uses(o)) < k]
        f += 8.0 * 2 * (Dr + 2 * len(carried) * K1) * Dl * K1          # first product, both planes
        f += 8.0 * Dl * Dl * 2 * K1                                      # R_{k-1}
        for o in carried:
            full = (not dg) or (k - 1) in uses(o)
            f += 2 * 8.0 * Dl * Dl * (1.0 if full else 0.5) * 2 * K1
        if k >= 1 and uses(k):
            f += 8.0 * Dl * Dl * K1 + 8.0 * Dl * Dl * 2 * K1              # M_k, C_Z,k
    return f


def lenv_flops(bonds, half: bool = False) -> float:
    """Left-environment chain of one image (lenv_image).  half: at a half-structured site
    (right bond >= 2, not the last) each product contracts one half of the site, and once
    the site before was half-structured too, L_k is block diagonal and the first product
    sums over half of the left bond."""
    n = len(bonds) - 1
    tot = 0.0
    for j in range(n):
        dl, dr = bonds[j], bonds[j + 1]
        if half and j < n - 1 and dr >= 2:
            first = dl * dl * dr * (0.5 if j >= 1 and dl >= 2 else 1.0)
            tot += 8.0 * (first + dl * dr * dr)
        else:
            tot += 8.0 * (2 * dl * dl * dr + 2 * dl * dr * dr)
    return tot


def padding(p: int, chi: int) -> int:
    """Site padding of an image (the library's layout rule)."""
    n = p * p
    cap = 1
    while cap < chi and cap < (1 << min(n // 2, 20)):
        cap <<= 1
    cap = min(cap, chi, 32)
    ld = 4
    while ld < cap:
        ld <<= 1
    return ld


def operator_product_path(p: int, L: int, chi: int, ansatz: str = "ladder") -> bool:
    """Whether the library runs the circuit (either ansatz) as an operator product
    (ladder_mpo.cu)."""
    # 2^L <= chi: no cut ever needs more (each layer crosses a cut with one CNOT)
    return 1 <= L <= 4 and (1 << L) <= min(padding(p, chi), chi, 16)


def image_flops(p: int, L: int, chi: int, ansatz: str = "ladder", dense: bool = False,
                kernel: str = "sweep") -> dict:
    """dense: count the operator-product path's contractions without the half-structure.
    kernel: the Pauli-cache kernel ("sweep": the per-image sweep, which forms the right
    environments itself, so the environment launch runs only the left chains; "column":
    the column walk after the right and left chains)."""
    n = p * p
    if operator_product_path(p, L, chi, ansatz):
        D = 1 << L
        bonds = [1] + [D] * (n - 1) + [1]
        circ = 0.0
        for k in range(n):
            dl = dr = 1
            for _ in range(L):
                circ += 32.0 * dl * dr
                dl = dl if k == 0 else 2 * dl
                dr = dr if k == n - 1 else 2 * dr
        half = ansatz == "ladder" and not dense
        # left chain: L A on the needed half, block-diagonal result (half the dense work)
        lenv = lenv_flops(bonds, half)
        if kernel == "sweep":
            return {"circuit": circ, "renv": lenv, "pauli": sweep_flops(p, bonds, lenv=True, half=half)}
        return {"circuit": circ, "renv": renv_flops(bonds, half) + lenv,
                "pauli": pauli_flops(p, bonds, lenv=True, half=half)}
    _, bonds = circuit_schedule(n, L, chi, ansatz)
    if kernel == "sweep":
        return {"circuit": circuit_flops(n, L, chi, ansatz), "renv": 0.0, "pauli": sweep_flops(p, bonds)}
    return {"circuit": circuit_flops(n, L, chi, ansatz), "renv": renv_flops(bonds), "pauli": pauli_flops(p, bonds)}
