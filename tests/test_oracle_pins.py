"""Pins for the CPU oracle: each check compares the oracle with something other
than itself -- values printed in the paper, closed forms, brute-force Kronecker
products, Clifford conjugation, the Schmidt truncation of the dense state, and
mathematical invariants.  CPU only.
"""
import itertools
import os

import numpy as np
import pytest
import scipy.linalg

from oracle import ano, circuit, mps, pairs, pipeline
from oracle import statevector as sv
from paper_2607_10280_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# Literal Pauli matrices and CNOT, written out here independently of the oracle.
P_I = np.eye(2, dtype=complex)
P_X = np.array([[0, 1], [1, 0]], dtype=complex)
P_Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
P_Z = np.array([[1, 0], [0, -1]], dtype=complex)
PAULIS = [P_I, P_X, P_Y, P_Z]
CNOT_LIT = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=complex)


def golden_facts():
    facts = {}
    with open(os.path.join(GOLDEN, "paper_facts.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                key, val, _cite = line.split()
                facts[key] = float(val)
    return facts


def expm_ry(t):
    return scipy.linalg.expm(-0.5j * t * P_Y)


def expm_rz(t):
    return scipy.linalg.expm(-0.5j * t * P_Z)


# ---------------------------------------------------------------- gates ----

def test_gate_matrices_match_exponentials():
    for t in (0.0, 0.37, 1.9, -2.6, 5.5):
        assert np.allclose(circuit.ry(t), expm_ry(t), atol=1e-15)
        assert np.allclose(circuit.rz(t), expm_rz(t), atol=1e-15)
    assert np.allclose(circuit.HADAMARD, (P_X + P_Z) / np.sqrt(2), atol=1e-15)
    assert np.array_equal(circuit.CNOT, CNOT_LIT)


# ------------------------------------------------------- brute force SV ----

def kron_embed(n, k, U):
    """Full 2^n operator of U acting on qubits k.. (qubit 0 = most significant bit)."""
    w = int(round(np.log2(U.shape[0])))
    return np.kron(np.kron(np.eye(2 ** k), U), np.eye(2 ** (n - k - w)))


def brute_state(n, ops):
    psi = np.zeros(2 ** n, dtype=complex)
    psi[0] = 1
    for _kind, k, M in ops:
        psi = kron_embed(n, k, M) @ psi
    return psi


def brute_pair(psi, n, i, j, a, b):
    O = np.eye(1)
    for k in range(n):
        O = np.kron(O, PAULIS[a] if k == i else PAULIS[b] if k == j else P_I)
    return np.vdot(psi, O @ psi).real


@pytest.mark.parametrize("ansatz", ["ladder", "paper"])
@pytest.mark.parametrize("n,L", [(2, 1), (3, 2), (5, 1), (6, 2)])
def test_statevector_matches_kronecker_brute_force(ansatz, n, L):
    x = synth.uniform_pixels(1, n, seed=11)[0][:n] if n * n >= n else None
    x = np.random.default_rng(n * 10 + L).random(n)
    params = synth.circuit_params(L, n, seed=5)
    ops = circuit.build_circuit(ansatz, x, L, params)
    psi = sv.run(n, ops).reshape(-1)
    ref = brute_state(n, ops)
    assert np.allclose(psi, ref, atol=1e-13)
    prs = [(i, j) for i in range(n) for j in range(i + 1, n)]
    cache = sv.pair_paulis(psi.reshape([2] * n), prs)
    for q, (i, j) in enumerate(prs):
        for a in range(4):
            for b in range(4):
                assert abs(cache[q, 4 * a + b] - brute_pair(ref, n, i, j, a, b)) < 1e-13


# ----------------------------------------------------- golden examples ----

def test_bell_pair_golden():
    data = np.loadtxt(os.path.join(GOLDEN, "bell_pair.txt"))
    expect = np.zeros(16)
    expect[data[:, 0].astype(int)] = data[:, 1]
    x = np.array([0.5, 0.0])
    ops = circuit.ladder_circuit(x, 1, np.zeros((1, 2, 2)))
    psi = sv.run(2, ops)
    assert np.allclose(sv.pair_paulis(psi, [(0, 1)])[0], expect, atol=1e-14)
    st = mps.simulate(ops, 2, chi=2)
    assert np.allclose(st.pair_paulis([(0, 1)])[0], expect, atol=1e-14)


def test_pair_counts_match_paper():
    facts = golden_facts()
    assert len(pairs.image_pairs(7, diagonals=True)) == facts["pairs_7x7_hvd"]
    assert len(list(itertools.combinations(range(49), 2))) == facts["pairs_7x7_all"]
    for p in range(2, 17):
        prs = pairs.image_pairs(p)
        assert len(prs) == 2 * p * (p - 1)
        assert len(set(prs)) == len(prs)
        for i, j in pairs.image_pairs(p, diagonals=True):
            assert i < j
            (ri, ci), (rj, cj) = divmod(i, p), divmod(j, p)
            assert (abs(ri - rj), abs(ci - cj)) in {(0, 1), (1, 0), (1, 1)}


# --------------------------------------------------------- closed forms ----

@pytest.mark.parametrize("backend", ["statevector", "mps"])
def test_encoding_only_closed_form(backend):
    """L = 0: product state R_Y(pi x)|0>; <X> = sin(pi x), <Y> = 0, <Z> = cos(pi x),
    and every pair expectation factorises."""
    p = 3
    x = synth.uniform_pixels(1, p, seed=3)[0]
    cache = pipeline.pauli_cache(x, p, 0, 2, "ladder", np.zeros((0, p * p, 2)), backend=backend)
    single = np.stack([np.ones_like(x), np.sin(np.pi * x), np.zeros_like(x), np.cos(np.pi * x)], 1)
    for q, (i, j) in enumerate(pairs.image_pairs(p)):
        expect = np.outer(single[i], single[j]).reshape(16)
        assert np.allclose(cache[q], expect, atol=1e-14)


def test_paper_encoding_block_closed_form():
    """One paper block on one qubit, H then R_Y(2 pi x - pi) (Eq. 2):
    <X> = -cos(2 pi x), <Z> = sin(2 pi x), <Y> = 0."""
    for x in (0.0, 0.13, 0.5, 0.77, 1.0):
        psi = sv.run(1, circuit.paper_circuit(np.array([x]), 1))
        got = [sv.expectation(psi, {0: P}).real for P in (P_X, P_Y, P_Z)]
        assert np.allclose(got, [-np.cos(2 * np.pi * x), 0.0, np.sin(2 * np.pi * x)], atol=1e-14)


def cnot_conjugate(a, b):
    M = CNOT_LIT @ np.kron(PAULIS[a], PAULIS[b]) @ CNOT_LIT
    for a2 in range(4):
        for b2 in range(4):
            c = np.trace(M @ np.kron(PAULIS[a2], PAULIS[b2]).conj().T) / 4
            if abs(c) > 0.5:
                return c.real, a2, b2
    raise AssertionError


def clifford_closed_form(phis, cnot_bonds, i, j, a, b):
    """<P_a(i) P_b(j)> after CNOTs on bonds (applied in the given order) acting on
    the product state prod_k phis[k]: conjugate the Pauli string backwards through
    the CNOTs, then multiply single-qubit expectations."""
    string = [0] * len(phis)
    string[i], string[j] = a, b
    sign = 1.0
    for k in reversed(cnot_bonds):
        s, string[k], string[k + 1] = cnot_conjugate(string[k], string[k + 1])
        sign *= s
    val = sign
    for k, ph in enumerate(phis):
        val *= np.vdot(ph, PAULIS[string[k]] @ ph).real
    return val


@pytest.mark.parametrize("ansatz,p", [("ladder", 4), ("ladder", 7), ("paper", 4), ("paper", 7)])
def test_single_layer_clifford_closed_form(ansatz, p):
    """L = 1: the rotations give a product state and the CNOTs are Clifford, so every
    pair Pauli has a closed form; rank <= 2 makes chi = 2 exact at any size."""
    n = p * p
    x = synth.garment_pixels(1, p, seed=8)[0]
    params = synth.circuit_params(1, n, seed=9)
    e0 = np.array([1, 0], dtype=complex)
    if ansatz == "ladder":
        phis = [expm_rz(params[0][k][1]) @ expm_ry(params[0][k][0]) @ expm_ry(np.pi * x[k]) @ e0
                for k in range(n)]
        bonds = list(range(n - 1))
    else:
        Hd = (P_X + P_Z) / np.sqrt(2)
        phis = [expm_ry(2 * np.pi * x[k] - np.pi) @ Hd @ e0 for k in range(n)]
        bonds = list(range(0, n - 1, 2)) + list(range(1, n - 1, 2))
    cache = pipeline.pauli_cache(x, p, 1, 2, ansatz, params)
    for q, (i, j) in enumerate(pairs.image_pairs(p)):
        for a in range(4):
            for b in range(4):
                ref = clifford_closed_form(phis, bonds, i, j, a, b)
                assert abs(cache[q, 4 * a + b] - ref) < 1e-12, (q, a, b)


# ------------------------------------------------- truncated regime pin ----

def schmidt_truncated_paulis(n, ops, chi, prs):
    """Dense state, truncated to chi Schmidt values across cut k after every
    two-qubit gate on (k, k+1), renormalised.  Returns the pair Paulis and the
    smallest relative gap sigma_chi - sigma_{chi+1} met at a cut."""
    psi = np.zeros(2 ** n, dtype=complex)
    psi[0] = 1
    min_gap = np.inf
    for _kind, k, M in ops:
        psi = kron_embed(n, k, M) @ psi
        if M.shape[0] == 4:
            U, S, Vh = np.linalg.svd(psi.reshape(2 ** (k + 1), -1), full_matrices=False)
            if len(S) > chi and S[chi] > 1e-13 * S[0]:
                min_gap = min(min_gap, (S[chi - 1] - S[chi]) / S[0])
                psi = (U[:, :chi] * S[:chi]) @ Vh[:chi]
                psi = psi.reshape(-1) / np.linalg.norm(psi)
    out = np.array([[brute_pair(psi, n, i, j, a, b) for a in range(4) for b in range(4)]
                    for (i, j) in prs])
    return out, min_gap


@pytest.mark.parametrize("ansatz", ["ladder", "paper"])
@pytest.mark.parametrize("L,chi", [(2, 1), (2, 3), (3, 2), (3, 3)])
def test_mps_truncation_equals_schmidt_truncation(ansatz, L, chi):
    p = 3
    n = p * p
    x = synth.uniform_pixels(1, p, seed=21)[0]
    params = synth.circuit_params(L, n, seed=22)
    ops = circuit.build_circuit(ansatz, x, L, params)
    prs = pairs.image_pairs(p)
    ref, gap = schmidt_truncated_paulis(n, ops, chi, prs)
    assert gap > 1e-6, "seeded case has a near-tie at the cut"
    st = mps.simulate(ops, n, chi)
    got, imag = st.pair_paulis(prs, return_imag=True)
    assert np.max(np.abs(got - ref)) < 1e-10
    assert np.max(np.abs(imag)) < 1e-12
    assert abs(st.norm_sq() - 1.0) < 1e-12
    assert max(st.bond_dims()) <= chi


@pytest.mark.parametrize("ansatz", ["ladder", "paper"])
def test_mps_exact_when_chi_reaches_schmidt_bound(ansatz):
    """Every layer crosses every cut with one CNOT, so the Schmidt rank is <= 2^L and
    chi = 2^L reproduces the dense state."""
    p = 4
    n = p * p
    for L in (1, 2, 3):
        x = synth.garment_pixels(1, p, seed=30 + L)[0]
        params = synth.circuit_params(L, n, seed=31)
        ops = circuit.build_circuit(ansatz, x, L, params)
        psi = sv.run(n, ops)
        for cut in range(n - 1):
            s = sv.schmidt_values(psi, cut)
            assert np.sum(s > 1e-12) <= 2 ** L
        st = mps.simulate(ops, n, 2 ** L)
        v = st.to_statevector().reshape(-1)
        ov = abs(np.vdot(v, psi.reshape(-1)))
        assert abs(ov - 1.0) < 1e-12
        prs = pairs.image_pairs(p)
        assert np.max(np.abs(st.pair_paulis(prs) - sv.pair_paulis(psi, prs))) < 1e-12


@pytest.mark.parametrize("ansatz", ["ladder", "paper"])
def test_truncation_error_within_discarded_weight_bound(ansatz):
    """Truncated regime (Sec. II.B; chi < 2^L): a renormalised truncation that drops
    the relative weight eps moves the unit state by sqrt(2 - 2 sqrt(1 - eps)) <=
    sqrt(2 eps), and the gates are unitary, so by the triangle inequality
    ||psi_exact - psi_chi|| <= sum_k sqrt(2 eps_k) over the oracle's steps, and every
    Pauli expectation moves by at most twice that.  Checked against the dense state
    at 16 qubits with the oracle's own per-step discarded weights, so keeping the
    wrong singular values or misreporting what was dropped fails."""
    p = 4
    n = p * p
    prs = pairs.image_pairs(p)
    worst = 0.0
    for L, chi in ((2, 1), (2, 3), (3, 2), (3, 5)):
        for seed in (70, 71):
            x = synth.garment_pixels(1, p, seed=seed)[0]
            params = synth.circuit_params(L, n, seed=seed + 10)
            ops = circuit.build_circuit(ansatz, x, L, params)
            psi = sv.run(n, ops)
            st = mps.simulate(ops, n, chi)
            bound = float(np.sum(np.sqrt(2.0 * np.asarray(st.discarded))))
            dist = float(np.linalg.norm(st.to_statevector().reshape(-1) - psi.reshape(-1)))
            assert dist <= bound + 1e-12, (L, chi, seed, dist, bound)
            err = float(np.max(np.abs(st.pair_paulis(prs) - sv.pair_paulis(psi, prs))))
            assert err <= 2.0 * dist + 1e-12, (L, chi, seed, err, dist)
            worst = max(worst, err)
    assert worst > 1e-3, "the seeded cases must actually truncate"


@pytest.mark.parametrize("ansatz", ["ladder", "paper"])
def test_each_truncation_keeps_overlap_sqrt_one_minus_discarded(ansatz):
    """One truncating step (Sec. II.B) is the projection onto the kept Schmidt
    vectors followed by renormalisation, so the states just before and just after
    it have overlap sqrt(1 - eps) exactly, eps being the weight the oracle reports
    as dropped at that step.  Pins the reported discarded weights step by step
    (the discarded-weight bound above is too loose to catch a misreported eps);
    which vectors are kept is pinned by the dense Schmidt truncation test."""
    import copy
    p, L, chi = 3, 3, 3
    n = p * p
    x = synth.garment_pixels(1, p, seed=90)[0]
    params = synth.circuit_params(L, n, seed=91)
    ops = circuit.build_circuit(ansatz, x, L, params)
    st = mps.MPS(n)
    truncating = 0
    for kind, k, M in ops:
        if kind == "1q":
            st.apply_1q(k, M)
            continue
        exact = copy.deepcopy(st)
        exact.apply_2q(k, M, 1 << 20)
        st.apply_2q(k, M, chi)
        eps = st.discarded[-1]
        ov = np.vdot(exact.to_statevector().reshape(-1), st.to_statevector().reshape(-1))
        assert abs(ov - np.sqrt(1.0 - eps)) < 1e-12, (k, eps, ov)
        truncating += eps > 1e-8
    assert truncating >= 3


def test_mae_falls_with_chi():
    """MAE against the exact state over a fixed set of images falls as chi grows and
    vanishes at chi = 2^L (Sec. III reports the same trend).  Not a theorem for
    sequential truncation, so this pins the trend on the seeded set only."""
    p, L = 4, 3
    n = p * p
    prs = pairs.image_pairs(p)
    X = synth.garment_pixels(4, p, seed=80)
    params = synth.circuit_params(L, n, seed=81)
    maes = []
    for chi in (1, 2, 4, 8):
        errs = []
        for x in X:
            ops = circuit.build_circuit("ladder", x, L, params)
            ref = sv.pair_paulis(sv.run(n, ops), prs)
            errs.append(np.abs(mps.simulate(ops, n, chi).pair_paulis(prs) - ref))
        maes.append(float(np.mean(errs)))
    assert all(a > b for a, b in zip(maes, maes[1:])), maes
    assert maes[-1] < 1e-13 and maes[0] > 1e-2, maes


def test_ladder_bond_dimensions():
    n, L, chi = 49, 3, 16
    x = synth.garment_pixels(1, 7, seed=40)[0]
    st = mps.simulate(circuit.ladder_circuit(x, L, synth.circuit_params(L, n)), n, chi)
    expect = [min(chi, 2 ** L, 2 ** (k + 1), 2 ** (n - k - 1)) for k in range(n - 1)]
    assert st.bond_dims() == expect


# ------------------------------------------------ paper's printed sweep ----

@pytest.mark.slow
@pytest.mark.parametrize("ansatz", ["paper", "ladder"])
def test_first_near_exact_bond_dimension_7x7(ansatz):
    """Sec. III: at 7 x 7 the first near-exact chi (MAE <= 1e-12, Eq. 7) is 2^L for
    L = 1..4, and for L = 4 the MAE falls as chi grows.  Reference: chi = 64."""
    facts = golden_facts()
    thr = facts["near_exact_mae"]
    p = 7
    x = synth.garment_pixels(1, p, seed=0)[0]
    for L in (1, 2, 3, 4):
        params = synth.circuit_params(L, p * p)
        ref = pipeline.pauli_cache(x, p, L, 64, ansatz, params)
        mae = {}
        chis = (1, 2, 4, 8, 16) if L == 4 else (2 ** (L - 1), 2 ** L)
        for chi in chis:
            mae[chi] = np.mean(np.abs(pipeline.pauli_cache(x, p, L, chi, ansatz, params) - ref))
        first = facts[f"first_near_exact_chi_L{L}"]
        assert mae[int(first)] <= thr
        assert mae[int(first) // 2] > thr
        if L == 4:
            seq = [mae[c] for c in (2, 4, 8, 16)]
            assert all(seq[i] > seq[i + 1] for i in range(3)), seq


# ----------------------------------------------------------- invariants ----

def _operator_product_sites(ansatz, x, L, params):
    """Site tensors [Dl][2][Dr] of a circuit whose CNOT layers act as operators, from
    the decomposition CNOT = sum_c P_c (x) X^c: every layer applies its one-qubit gates,
    then each site gets, for its left and right bond bits (a, b), the physical operator
    P_b X^a (left CNOT first: the ladder, odd sites of the brick-wall) or X^a P_b
    (right CNOT first: even sites of the brick-wall), placed at bond indices
    (l + Dl a, r + Dr b).  Written here from that derivation alone."""
    n = len(x)
    X = np.array([[0, 1], [1, 0]], dtype=complex)
    P = [np.diag([1.0, 0.0]).astype(complex), np.diag([0.0, 1.0]).astype(complex)]
    sites = []
    for k in range(n):
        t = np.zeros((1, 2, 1), dtype=complex)
        if ansatz == "ladder":
            t[0, :, 0] = expm_ry(np.pi * x[k]) @ np.array([1.0, 0.0])
        else:
            t[0, 0, 0] = 1.0
        for layer in range(L):
            if ansatz == "ladder":
                G = expm_rz(params[layer][k][1]) @ expm_ry(params[layer][k][0])
            else:
                G = expm_ry(2 * np.pi * x[k] - np.pi) @ ((P_X + P_Z) / np.sqrt(2))
            t = np.einsum("st,ltr->lsr", G, t)
            Dl, _, Dr = t.shape
            has_l, has_r = k > 0, k < n - 1
            u = np.zeros((2 * Dl if has_l else Dl, 2, 2 * Dr if has_r else Dr), dtype=complex)
            right_first = ansatz == "paper" and k % 2 == 0
            for a in range(2 if has_l else 1):
                for b in range(2 if has_r else 1):
                    Xa = np.linalg.matrix_power(X, a) if has_l else np.eye(2)
                    Pb = P[b] if has_r else np.eye(2)
                    O = Xa @ Pb if right_first else Pb @ Xa
                    u[a * Dl:(a + 1) * Dl, :, b * Dr:(b + 1) * Dr] = np.einsum("st,ltr->lsr", O, t)
            t = u
        sites.append(t)
    return sites


@pytest.mark.parametrize("ansatz,p,L", [("ladder", 3, 3), ("ladder", 4, 2), ("paper", 3, 3), ("paper", 4, 2)])
def test_cnot_layers_as_bond_two_operators(ansatz, p, L):
    """The construction behind the GPU's operator-product path (Sec. II.B as operator
    products): contracting the site tensors gives the dense statevector of the circuit,
    every inner bond is 2^L, and the sites that path treats as half-structured (all but
    the last for the ladder) vanish outside half s of their right bond."""
    n = p * p
    x = synth.garment_pixels(1, p, seed=160 + L)[0]
    params = synth.circuit_params(L, n, seed=161) if ansatz == "ladder" else None
    sites = _operator_product_sites(ansatz, x, L, params)
    psi = sites[0][0]
    for t in sites[1:]:
        psi = np.einsum("...a,asb->...sb", psi, t)
    psi = psi.reshape(-1)
    ref = sv.run(n, circuit.build_circuit(ansatz, x, L, params)).reshape(-1)
    assert np.max(np.abs(psi - ref)) < 1e-12
    assert [t.shape[2] for t in sites[:-1]] == [2 ** L] * (n - 1)
    for k, t in enumerate(sites[:-1]):
        if ansatz == "paper" and k % 2 == 0 and k > 0:
            continue   # even brick-wall sites: output bit a xor b, not half-structured
        h = t.shape[2] // 2
        for s in range(2):
            assert np.all(t[:, s, (1 - s) * h:(2 - s) * h] == 0), (k, s)


def test_state_invariants_truncated():
    p, L, chi = 4, 3, 3
    n = p * p
    x = synth.garment_pixels(1, p, seed=50)[0]
    params = synth.circuit_params(L, n, seed=51)
    for ansatz in ("ladder", "paper"):
        cache, st = pipeline.pauli_cache(x, p, L, chi, ansatz, params, return_state=True)
        assert np.allclose(cache[:, 0], 1.0, atol=1e-13)           # <I (x) I> = 1
        assert np.all(np.abs(cache) <= 1 + 1e-12)
        for q in range(len(cache)):
            rho = ano.rho_from_paulis(cache[q])
            assert abs(np.trace(rho) - 1) < 1e-13
            assert np.min(np.linalg.eigvalsh(rho)) > -1e-12          # PSD
        # single-site terms agree across every pair that contains the site
        single = {}
        for q, (i, j) in enumerate(pairs.image_pairs(p)):
            for site, vals in ((i, cache[q, [4, 8, 12]]), (j, cache[q, [1, 2, 3]])):
                if site in single:
                    assert np.allclose(single[site], vals, atol=1e-12)
                single[site] = vals
        # canonical form: sites left of the centre left-orthonormal, right of it right-orthonormal
        for k, A in enumerate(st.A):
            if k < st.centre:
                G = np.einsum("lsr,lsq->rq", A.conj(), A)
                assert np.allclose(G, np.eye(G.shape[0]), atol=1e-12)
            elif k > st.centre:
                G = np.einsum("lsr,msr->lm", A, A.conj())
                assert np.allclose(G, np.eye(G.shape[0]), atol=1e-12)
        if ansatz == "paper":
            # H, R_Y and CNOT are real, so the state is real and every Pauli string
            # with an odd number of Y factors has zero expectation.
            odd_y = [4 * a + b for a in range(4) for b in range(4) if ((a == 2) + (b == 2)) % 2]
            assert np.max(np.abs(cache[:, odd_y])) < 1e-13


# ------------------------------------------------------------------ ANO ----

def test_pauli_coefficients_complete_basis():
    facts = golden_facts()
    assert facts["pauli_norm_k"] == 2
    abd = synth.observable_params(5)
    for q in range(5):
        H = ano.hermitian(abd[q])
        assert np.allclose(H, H.conj().T)
        assert H[0, 1] == abd[q][0] + 1j * abd[q][6] and H[2, 3] == abd[q][5] + 1j * abd[q][11]
        assert np.allclose(np.diag(H).real, abd[q][12:16])
        c = ano.coefficients(abd[q])
        rebuilt = sum(c[a] * np.kron(PAULIS[a // 4], PAULIS[a % 4]) for a in range(16))
        assert np.allclose(rebuilt, H, atol=1e-14)


def test_feature_pauli_route_equals_direct_trace():
    """Eq. 5 (sum_alpha c <P_alpha>) equals Eq. 1 (Tr rho H) with rho from a partial trace."""
    p, L = 3, 2
    n = p * p
    x = synth.garment_pixels(1, p, seed=60)[0]
    ops = circuit.ladder_circuit(x, L, synth.circuit_params(L, n, seed=61))
    psi = sv.run(n, ops)
    prs = pairs.image_pairs(p)
    cache = sv.pair_paulis(psi, prs)
    abd = synth.observable_params(len(prs))
    q_pauli = ano.features(cache, abd)
    for q, (i, j) in enumerate(prs):
        rest = [k for k in range(n) if k not in (i, j)]
        M = np.transpose(psi, [i, j] + rest).reshape(4, -1)
        rho = M @ M.conj().T
        assert np.allclose(ano.rho_from_paulis(cache[q]), rho, atol=1e-14)
        assert abs(q_pauli[q] - ano.feature_direct(rho, abd[q])) < 1e-13


def test_linear_layer_special_cases():
    q = np.arange(5.0)
    b = np.ones(5)
    assert np.allclose(ano.linear(np.eye(5), q, b), q + 1)
    assert np.allclose(ano.linear(np.zeros((3, 5)), q, np.arange(3.0)), np.arange(3.0))


@pytest.mark.parametrize("ansatz", ["ladder", "paper"])
def test_schmidt_rank_at_most_two_to_the_cnots_across_the_cut(ansatz):
    """A CNOT has operator Schmidt rank 2 and one-qubit gates have rank 1, so after c
    CNOTs have crossed a cut the state's Schmidt rank there is at most 2^c.  Checked on
    the dense state after every gate (3x3 and 4x4 images, L = 3 and 2): the GPU splits
    keep at most min(chi, 2^c) values on this ground."""
    from oracle import circuit as circ, statevector as sv
    for p, L in ((3, 3), (4, 2)):
        n = p * p
        rng = np.random.default_rng(7)
        x = rng.random(n)
        params = rng.uniform(0, 2 * np.pi, size=(L, n, 2))
        ops = circ.build_circuit(ansatz, x, L, params if ansatz == "ladder" else None)
        psi = sv.zero_state(n)
        crossed = np.zeros(n - 1, dtype=int)
        for kind, k, M in ops:
            if kind == "1q":
                psi = sv.apply_1q(psi, k, M)
                continue
            psi = sv.apply_2q(psi, k, M)
            crossed[k] += 1
            for cut in range(n - 1):
                s = sv.schmidt_values(psi, cut)
                assert np.sum(s > 1e-10 * s[0]) <= 2 ** crossed[cut]
