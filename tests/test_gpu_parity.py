"""Parity of the CUDA path against the CPU oracle (GPU tests).

Tolerances: the FP64 path must match the oracle within 1e-10 per Pauli entry and
the mixed paths within 1e-5 absolute, flat.  The mixed paths keep a complex64
state wherever nothing is truncated lossily and run a truncating circuit on a
complex128 state, so the truncated regime meets the same bound.  Cases where the
oracle meets a near-tie at a truncation cut (relative gap below 1e-6) have no
unique answer and are skipped; the seeds used here are checked to avoid them.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import ano as o_ano          # noqa: E402
from oracle import circuit as o_circ     # noqa: E402
from oracle import mps as o_mps          # noqa: E402
from oracle import pairs as o_pairs      # noqa: E402
from oracle import statevector as o_sv   # noqa: E402
from paper_2607_10280_b300 import synth  # noqa: E402

TOL = {"fp64": 1e-10, "mixed": 1e-5, "mixed_orth64": 1e-5}
TIE_GAP = 1e-6   # relative singular-value gap below which a truncation has no unique answer


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_10280_b300 import build
    build.build()


def oracle_cache(x, p, L, chi, ansatz="ladder", params=None, backend="mps"):
    n = p * p
    ops = o_circ.build_circuit(ansatz, np.asarray(x), L, params)
    prs = o_pairs.image_pairs(p)
    if backend == "statevector":
        return o_sv.pair_paulis(o_sv.run(n, ops), prs), np.inf
    st = o_mps.simulate(ops, n, chi)
    return st.pair_paulis(prs), st.min_gap


def run_gpu(pixels_list, ps, L, chi, precision, ansatz="ladder", params=None, shape=None, pipeline=True):
    from paper_2607_10280_b300.api import Batch
    px = torch.tensor(np.concatenate([np.asarray(x) for x in pixels_list]), dtype=torch.float64, device="cuda")
    pr = None if params is None else torch.tensor(params, dtype=torch.float64, device="cuda").contiguous()
    b = Batch(np.asarray(ps, dtype=np.int32), chi, precision)
    if shape:
        b.set_launch_shape(*shape)
    b.set_layer_pipeline(pipeline)
    b.apply_circuit(px, L, ansatz, pr)
    out = b.pauli_cache()
    b.sync()
    res = out.double().cpu().numpy()
    offs = b.pair_offsets
    bonds = b.bond_dims()
    disc = b.discarded_weight()
    b.close()
    return [res[offs[i]:offs[i + 1]] for i in range(len(ps))], bonds, disc


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_orth64"])
def test_tiny_4x4_vs_statevector(precision):
    """4x4 image (16 qubits), batch 8, U[0,1] pixels, L = 1, chi = 4 (plain method, tiny)."""
    p, B, L, chi = 4, 8, 1, 4
    X = synth.uniform_pixels(B, p)
    params = synth.circuit_params(L, p * p)
    got, _, _ = run_gpu(list(X), [p] * B, L, chi, precision, params=params)
    for i in range(B):
        ref, _ = oracle_cache(X[i], p, L, chi, params=params, backend="statevector")
        assert got[i].shape == (24, 16)
        assert np.max(np.abs(got[i] - ref)) < TOL[precision], (i, np.max(np.abs(got[i] - ref)))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("p,L,chi", [(3, 2, 1), (3, 3, 2), (3, 3, 3), (4, 2, 2), (4, 3, 3), (4, 4, 4), (5, 3, 4)])
def test_truncated_regime_vs_oracle_mps(precision, p, L, chi):
    B = 4
    X = synth.uniform_pixels(B, p, seed=100 + p)
    params = synth.circuit_params(L, p * p, seed=101)
    got, _, disc = run_gpu(list(X), [p] * B, L, chi, precision, params=params)
    for i in range(B):
        st = o_mps.simulate(o_circ.build_circuit("ladder", X[i], L, params), p * p, chi)
        ref, gap = st.pair_paulis(o_pairs.image_pairs(p)), st.min_gap
        if gap < TIE_GAP:
            continue
        assert np.max(np.abs(got[i] - ref)) < TOL[precision], (i, gap, np.max(np.abs(got[i] - ref)))
        # the discarded weight summed over the steps (the truncation error's budget);
        # both precisions truncate on an FP64 state
        ref_disc = float(np.sum(st.discarded))
        assert abs(disc[i] - ref_disc) <= 1e-10, (i, disc[i], ref_disc)
    assert np.all(disc >= 0)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_uneven_batch_ragged_sizes(precision):
    ps = [2, 5, 3, 4, 2, 6, 3]
    L, chi = 2, 4
    params = synth.circuit_params(L, 36, seed=7)
    X = [synth.garment_pixels(1, p, seed=200 + i)[0] for i, p in enumerate(ps)]
    got, _, _ = run_gpu(X, ps, L, chi, precision, params=params)
    for i, p in enumerate(ps):
        ref, gap = oracle_cache(X[i], p, L, chi, params=params)
        assert gap >= 1e-6
        assert np.max(np.abs(got[i] - ref)) < TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_paper_ansatz_vs_statevector(precision):
    p, B, L, chi = 4, 4, 2, 16
    X = synth.garment_pixels(B, p, seed=5)
    got, _, _ = run_gpu(list(X), [p] * B, L, chi, precision, ansatz="paper")
    for i in range(B):
        ref, _ = oracle_cache(X[i], p, L, chi, ansatz="paper", backend="statevector")
        assert np.max(np.abs(got[i] - ref)) < TOL[precision]


def test_paper_ansatz_truncated_vs_oracle_mps():
    p, B, L, chi = 3, 4, 3, 2
    X = synth.uniform_pixels(B, p, seed=9)
    got, _, _ = run_gpu(list(X), [p] * B, L, chi, "fp64", ansatz="paper")
    for i in range(B):
        ref, gap = oracle_cache(X[i], p, L, chi, ansatz="paper")
        if gap < 1e-6:
            continue
        assert np.max(np.abs(got[i] - ref)) < 1e-10


def test_encoding_only_and_chi_one():
    """L = 0 gives the product state (closed form of the encoding); chi = 1 forces
    every two-qubit step through the SVD branch."""
    p = 3
    X = synth.uniform_pixels(2, p, seed=3)
    got, bonds, _ = run_gpu(list(X), [p, p], 0, 2, "fp64", params=np.zeros((1, 9, 2)))
    for i in range(2):
        s = np.stack([np.ones(9), np.sin(np.pi * X[i]), np.zeros(9), np.cos(np.pi * X[i])], 1)
        for q, (a, b) in enumerate(o_pairs.image_pairs(p)):
            assert np.allclose(got[i][q], np.outer(s[a], s[b]).reshape(16), atol=1e-12)
    params = synth.circuit_params(2, 9, seed=4)
    got, bonds, disc = run_gpu(list(X), [p, p], 2, 1, "fp64", params=params)
    assert all(max(bd) == 1 for bd in bonds)
    for i in range(2):
        ref, gap = oracle_cache(X[i], p, 2, 1, params=params)
        assert np.max(np.abs(got[i] - ref)) < 1e-10
    assert np.all(disc > 0)


def _ld(p, chi):
    """Site padding of an image (the library's layout rule): the bond cap rounded up
    to a power of two, at least 4."""
    n = p * p
    cap = 1
    while cap < chi and cap < (1 << min(n // 2, 20)):
        cap <<= 1
    cap = min(cap, chi, 32)
    ld = 4
    while ld < cap:
        ld <<= 1
    return ld


def _operator_product_path(p, L, chi):
    """Whether the library runs an image as an operator product (bond 2^L)."""
    return 1 <= L <= 4 and (1 << L) <= min(_ld(p, chi), chi, 16)


def test_ladder_bond_dimensions_7x7():
    """Sequential sweep: canonical bonds min(chi, 2^L, 2^(k+1), 2^(n-k-1)); the
    operator-product path (Sec. II.B as a CNOT-ladder product, no factorisation): 2^L
    at every inner cut."""
    n, L, chi = 49, 3, 16
    X = synth.garment_pixels(2, 7, seed=40)
    params = synth.circuit_params(L, n)
    _, bonds, _ = run_gpu(list(X), [7, 7], L, chi, "mixed", params=params, pipeline=False)
    expect = [1] + [min(chi, 2 ** L, 2 ** (k + 1), 2 ** (n - k - 1)) for k in range(n - 1)] + [1]
    assert bonds[0] == expect and bonds[1] == expect
    _, bonds, _ = run_gpu(list(X), [7, 7], L, chi, "mixed", params=params, pipeline=True)
    assert _operator_product_path(7, L, chi)
    assert list(bonds[0]) == [1] + [2 ** L] * (n - 1) + [1] and list(bonds[1]) == list(bonds[0])


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_headline_7x7_L4_chi16_sampled(precision):
    """7x7 images (49 qubits), L = 4, chi = 16: the benchmark workload shape, run at
    batch 64 with the same launch configuration; sampled images vs the oracle."""
    p, L, chi, B = 7, 4, 16, 64
    X = synth.garment_pixels(B, p)
    params = synth.circuit_params(L, p * p)
    got, _, disc = run_gpu(list(X), [p] * B, L, chi, precision, params=params)
    for i in (0, 17, 63):
        ref, _ = oracle_cache(X[i], p, L, chi, params=params)
        err = np.max(np.abs(got[i] - ref))
        assert err < TOL[precision], (i, err)
    assert np.max(disc) == 0.0   # chi = 2^L: nothing is truncated


def test_headline_full_batch_sampled():
    """The benchmark workload itself: 1024 garment-like 7x7 images (pixel seed 0),
    L = 4, chi = 16, mixed, default launch shape (the operator-product circuit path,
    since nothing truncates at chi = 2^L); the first, a middle and the last image vs
    the oracle."""
    p, L, chi, B = 7, 4, 16, 1024
    X = synth.garment_pixels(B, p)
    params = synth.circuit_params(L, p * p)
    got, _, disc = run_gpu(list(X), [p] * B, L, chi, "mixed", params=params)
    for i in (0, 511, 1023):
        ref, _ = oracle_cache(X[i], p, L, chi, params=params)
        assert np.max(np.abs(got[i] - ref)) < TOL["mixed"], i
    assert np.max(disc) == 0.0


def test_truncated_full_batch_sampled_within_discarded_bound():
    """Truncated regime at full size (1024 7x7 images, L = 4, chi = 4, mixed, as in the
    chi x L sweep): sampled images vs the oracle at the same chi (gap-aware bound),
    the reported discarded weight vs the oracle's, and the distance to the exact
    result (oracle at chi = 2^L) within 2 sum_k sqrt(2 eps_k) <= 2 sqrt(2 T sum_k eps_k),
    T = L (n - 1) two-qubit steps, with the GPU's own discarded weights."""
    p, L, chi, B = 7, 4, 4, 1024
    n = p * p
    X = synth.garment_pixels(B, p)
    params = synth.circuit_params(L, n)
    got, _, disc = run_gpu(list(X), [p] * B, L, chi, "mixed", params=params)
    prs = o_pairs.image_pairs(p)
    worst = 0.0
    for i in (0, 511, 1023):
        st = o_mps.simulate(o_circ.build_circuit("ladder", X[i], L, params), n, chi)
        ref, gap = st.pair_paulis(prs), st.min_gap
        if gap >= TIE_GAP:
            assert np.max(np.abs(got[i] - ref)) < TOL["mixed"], (i, gap)
        ref_disc = float(np.sum(st.discarded))
        assert abs(disc[i] - ref_disc) <= 1e-10, (i, disc[i], ref_disc)
        exact, _ = oracle_cache(X[i], p, L, 2 ** L, params=params)
        err = np.max(np.abs(got[i] - exact))
        assert err <= 2.0 * np.sqrt(2.0 * L * (n - 1) * disc[i]) + 1e-5, (i, err, disc[i])
        worst = max(worst, err)
    assert worst > 1e-3   # the sampled images are truncated for real


def test_large_16x16_and_uneven_mix():
    """Maximum image size (256 qubits) and an uneven mix up to it, L = 2."""
    ps = [16, 4, 11, 16, 7]
    L, chi = 2, 32
    params = synth.circuit_params(L, 256, seed=12)
    X = [synth.garment_pixels(1, p, seed=300 + i)[0] for i, p in enumerate(ps)]
    got, _, _ = run_gpu(X, ps, L, chi, "mixed", params=params)
    for i in (0, 1, 2):
        ref, _ = oracle_cache(X[i], ps[i], L, chi, params=params)
        assert np.max(np.abs(got[i] - ref)) < 1e-5


def test_launch_shapes_agree():
    p, L, chi, B = 5, 3, 8, 11
    X = synth.garment_pixels(B, p, seed=77)
    params = synth.circuit_params(L, 25, seed=78)
    base, _, _ = run_gpu(list(X), [p] * B, L, chi, "mixed", params=params, shape=(1, 32, 32))
    for shape in ((2, 32, 64), (4, 32, 128), (8, 32, 32), (3, 32, 64)):
        got, _, _ = run_gpu(list(X), [p] * B, L, chi, "mixed", params=params, shape=shape)
        for i in range(B):
            assert np.array_equal(got[i], base[i])   # these knobs keep every bit
    # wider circuit teams change the QR summation order only
    for shape in ((1, 64, 64), (1, 128, 128)):   # bucket 8: runs one warp per image
        got, _, _ = run_gpu(list(X), [p] * B, L, chi, "mixed", params=params, shape=shape)
        for i in range(B):
            assert np.max(np.abs(got[i] - base[i])) < 2e-6
    p2, L2, chi2, B2 = 7, 4, 16, 6    # bucket 16, where the wider teams are compiled
    X2 = synth.garment_pixels(B2, p2, seed=79)
    params2 = synth.circuit_params(L2, 49, seed=80)
    base2, _, _ = run_gpu(list(X2), [p2] * B2, L2, chi2, "mixed", params=params2, shape=(2, 32, 64))
    for shape in ((1, 64, 64), (1, 128, 128)):
        got, _, _ = run_gpu(list(X2), [p2] * B2, L2, chi2, "mixed", params=params2, shape=shape)
        for i in range(B2):
            assert np.max(np.abs(got[i] - base2[i])) < 2e-6


def test_ano_features_and_linear_vs_oracle():
    from paper_2607_10280_b300.api import ano_features
    p, B = 7, 5
    m = 2 * p * (p - 1)
    X = synth.garment_pixels(B, p, seed=90)
    params = synth.circuit_params(2, 49, seed=91)
    caches = np.stack([oracle_cache(X[i], p, 2, 8, params=params)[0] for i in range(B)])
    abd = synth.observable_params(m)
    W, bias = synth.linear_params(784, m)
    for dt in (torch.float32, torch.float64):
        P = torch.tensor(caches.reshape(B * m, 16), dtype=dt, device="cuda")
        feats, out = ano_features(P, m, torch.tensor(abd, dtype=torch.float32, device="cuda"),
                                  torch.tensor(W, dtype=torch.float32, device="cuda"),
                                  torch.tensor(bias, dtype=torch.float32, device="cuda"))
        torch.cuda.synchronize()
        f = feats.double().cpu().numpy()
        y = out.double().cpu().numpy()
        abd32 = abd.astype(np.float32).astype(np.float64)
        W32 = W.astype(np.float32).astype(np.float64)
        b32 = bias.astype(np.float32).astype(np.float64)
        for i in range(B):
            ref_q = o_ano.features(caches[i], abd32)
            scale_q = np.array([np.sum(np.abs(o_ano.coefficients(abd32[q]) * caches[i][q])) for q in range(m)])
            assert np.all(np.abs(f[i] - ref_q) <= 1e-5 * (1 + scale_q))
            ref_y = o_ano.linear(W32, ref_q, b32)
            scale_y = np.abs(W32) @ np.abs(ref_q) + np.abs(b32)
            assert np.all(np.abs(y[i] - ref_y) <= 1e-5 * (1 + scale_y))


def test_linear_layer_tensor_cores_partial_tiles():
    """y = W q + b (Eq. 6) for the 16x16 pair count (480 features) into 1000 outputs
    and 300 images: partial 128 x 128 tiles in both directions and a K tail."""
    from paper_2607_10280_b300 import _lib
    from paper_2607_10280_b300.api import ano_features
    rng = np.random.default_rng(5)
    B, m, O = 300, 480, 1000
    P = rng.uniform(-1, 1, size=(B * m, 16)).astype(np.float32)
    P[:, 0] = 1.0
    abd = synth.observable_params(m)
    W = (rng.standard_normal((O, m)) / np.sqrt(m)).astype(np.float32)
    bias = rng.standard_normal(O).astype(np.float32)
    feats, out = ano_features(torch.tensor(P, device="cuda"), m, torch.tensor(abd, dtype=torch.float32, device="cuda"),
                              torch.tensor(W, device="cuda"), torch.tensor(bias, device="cuda"))
    _lib.check(_lib.lib().ano_status())
    q = feats.double().cpu().numpy()
    ref = q @ W.astype(np.float64).T + bias.astype(np.float64)
    scale = np.abs(q) @ np.abs(W.astype(np.float64)).T + np.abs(bias)
    assert np.all(np.abs(out.double().cpu().numpy() - ref) <= 1e-5 * (1 + scale))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("ansatz,p,L,chi", [("ladder", 2, 1, 2), ("ladder", 3, 2, 4), ("ladder", 4, 3, 8),
                                             ("ladder", 7, 2, 4), ("paper", 4, 2, 16), ("ladder", 5, 3, 3)])
def test_diagonal_pairs_vs_oracle(precision, ansatz, p, L, chi):
    """The paper's full pair set (Sec. II.C): horizontal, vertical and both diagonals
    (156 pairs at 7x7); the H+V block equals the H+V-only cache bit for bit."""
    from paper_2607_10280_b300.api import Batch
    B = 3
    X = synth.garment_pixels(B, p, seed=60 + p)
    params = synth.circuit_params(L, p * p, seed=61) if ansatz == "ladder" else None
    b = Batch(np.full(B, p, np.int32), chi, precision)
    px = torch.tensor(X.reshape(-1), dtype=torch.float64, device="cuda")
    pr = None if params is None else torch.tensor(params, dtype=torch.float64, device="cuda")
    b.apply_circuit(px, L, ansatz, pr)
    full = b.pauli_cache(pair_set="hvd")
    hv = b.pauli_cache(pair_set="hv")
    b.sync()
    full = full.double().cpu().numpy()
    hv = hv.double().cpu().numpy()
    mh, md = 2 * p * (p - 1), 2 * p * (p - 1) + 2 * (p - 1) ** 2
    assert full.shape[0] == B * md and (p != 7 or md == 156)
    prs = o_pairs.image_pairs(p, diagonals=True)
    for i in range(B):
        blk = full[i * md:(i + 1) * md]
        assert np.array_equal(blk[:mh], hv[i * mh:(i + 1) * mh])
        ops = o_circ.build_circuit(ansatz, X[i], L, params)
        st = o_mps.simulate(ops, p * p, chi)
        if st.min_gap < 1e-6:
            continue
        ref = st.pair_paulis(prs)
        assert np.max(np.abs(blk - ref)) < TOL[precision], (st.min_gap, np.max(np.abs(blk - ref)))


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_orth64"])
def test_layer_pipeline_equals_sequential_sweep(precision):
    """The fast paths for ladder circuits without truncation (L <= 4) against the
    sequential sweep: the layer-pipelined kernel runs every two-qubit step on the same
    inputs with the same operations (same bonds); the operator-product path (2^L within
    chi and the padding) builds the same state without factorisation, with bond 2^L at
    every inner cut.  Pauli caches equal to rounding (1e-12 FP64, 5e-6 mixed: complex64
    rounding of different but exact operation sequences, up to 255 steps per layer of
    a 16x16 image); an ordering or synchronisation error would show in FP64."""
    cases = [([7] * 6, 4, 16), ([5] * 5, 3, 8), ([4, 9, 6, 16, 5], 2, 16), ([6] * 4, 1, 2),
             ([3, 2, 8, 7], [4, 0, 3, 2], 32)]
    bound = 1e-12 if precision == "fp64" else 5e-6
    for ci, (ps, L, chi) in enumerate(cases):
        X = [synth.garment_pixels(1, p, seed=60 + 7 * ci + i)[0] for i, p in enumerate(ps)]
        params = synth.circuit_params(int(np.max(L)), max(ps) ** 2, seed=70 + ci)
        seq, b_seq, d_seq = run_gpu(X, ps, L, chi, precision, params=params, pipeline=False)
        pip, b_pip, d_pip = run_gpu(X, ps, L, chi, precision, params=params, pipeline=True)
        for i, p in enumerate(ps):
            Li = int(np.atleast_1d(L)[i]) if np.ndim(L) else L
            if _operator_product_path(p, Li, chi):
                assert list(b_pip[i]) == [1] + [2 ** Li] * (p * p - 1) + [1], (ci, i)
            else:
                assert np.array_equal(b_seq[i], b_pip[i]), (ci, i)
        assert np.all(d_pip == 0.0) and np.all(d_seq == 0.0)
        for i in range(len(ps)):
            err = np.max(np.abs(seq[i] - pip[i]))
            assert err <= bound, (ci, i, err)
    # the sample of the pipelined path also matches the oracle
    ref, _ = oracle_cache(X[0], ps[0], int(L[0]), chi, params=params)
    assert np.max(np.abs(pip[0] - ref)) < TOL[precision]


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_half_structured_contractions_are_bit_identical(precision):
    """Ladder circuits built as operator products: every site but the last vanishes
    outside half s of its right bond, and the environment and Pauli kernels contract
    over that half only.  The skipped terms are exact zeros, so the Pauli caches (H+V
    and with diagonals) equal the dense contractions bit for bit, at L = 4 (bond 16,
    split products) and L = 2 (bond 4, compact left blocks only)."""
    from paper_2607_10280_b300.api import Batch
    for p, L, chi in ((7, 4, 16), (5, 2, 8)):
        X = synth.garment_pixels(3, p, seed=150 + L)
        params = torch.tensor(synth.circuit_params(L, p * p, seed=151), dtype=torch.float64, device="cuda")
        px = torch.tensor(X.reshape(-1), dtype=torch.float64, device="cuda")
        caches = []
        for half in (True, False):
            b = Batch(np.full(3, p, np.int32), chi, precision)
            b.set_half_structure(half)
            b.apply_circuit(px, L, "ladder", params)
            hv, hvd = b.pauli_cache(), b.pauli_cache(pair_set="hvd")
            b.sync()
            caches.append((hv.cpu().numpy(), hvd.cpu().numpy()))
            b.close()
        assert np.array_equal(caches[0][0], caches[1][0]) and np.array_equal(caches[0][1], caches[1][1]), (p, L)
        ref, _ = oracle_cache(X[0], p, L, chi, params=params.cpu().numpy())
        assert np.max(np.abs(caches[0][0][:len(ref)] - ref)) < TOL[precision]


def test_layer_pipeline_falls_back_when_a_step_truncates():
    """chi < 2^L (a truncating pass): the sequential sweep runs whatever the switch."""
    p, L, chi = 5, 3, 4
    X = synth.garment_pixels(3, p, seed=91)
    params = synth.circuit_params(L, p * p, seed=92)
    a, ba, da = run_gpu(list(X), [p] * 3, L, chi, "mixed", params=params, pipeline=False)
    b, bb, db = run_gpu(list(X), [p] * 3, L, chi, "mixed", params=params, pipeline=True)
    assert all(np.array_equal(u, v) for u, v in zip(ba, bb)) and np.array_equal(da, db)
    for i in range(3):
        assert np.array_equal(a[i], b[i])


@pytest.mark.parametrize("overlap", [True, False])
def test_pipeline_overlapped_steps_keep_their_results(overlap):
    """Pipeline.submit/result with two buffer sets: steps whose copies (and, with
    overlap, kernels on a compute stream and batch per buffer set) overlap the next
    step's return exactly what each step gives when run alone."""
    from paper_2607_10280_b300 import api
    p, B, L, chi = 5, 16, 2, 4
    m = api.pair_count(p)
    params = torch.tensor(synth.circuit_params(L, p * p, seed=101), dtype=torch.float64, device="cuda")
    abd = torch.tensor(synth.observable_params(m, seed=102), dtype=torch.float32, device="cuda")
    W, b = synth.linear_params(40, m, seed=103)
    W = torch.tensor(W, dtype=torch.float32, device="cuda")
    b = torch.tensor(b, dtype=torch.float32, device="cuda")
    pipe = api.Pipeline(np.full(B, p, np.int32), chi, L, "mixed", params, abd, W, b, overlap=overlap)
    assert len(pipe.batches) == (2 if overlap else 1)
    host = [torch.tensor(synth.garment_pixels(B, p, seed=110 + s).reshape(-1), dtype=torch.float64).pin_memory()
            for s in range(3)]
    alone = [[t.clone() for t in pipe.run(h)] for h in host]
    k0 = pipe.submit(host[0])
    k1 = pipe.submit(host[1])
    r0 = [t.clone() for t in pipe.result(k0)]
    k2 = pipe.submit(host[2])
    r1 = [t.clone() for t in pipe.result(k1)]
    r2 = [t.clone() for t in pipe.result(k2)]
    for got, ref in zip((r0, r1, r2), alone):
        for g, r in zip(got, ref):
            assert torch.equal(g, r)
    assert not torch.equal(r0[0], r1[0])
    pipe.sync()


def test_bond_caps_above_the_exact_bond_change_nothing():
    """Sec. III sweeps chi up to 2048 at 7x7: bonds never exceed 2^L there, so every cap
    chi >= 2^L gives the same state (same bonds, same Pauli cache to the last bit)."""
    p, L = 7, 3
    X = list(synth.garment_pixels(4, p, seed=120))
    params = synth.circuit_params(L, p * p, seed=121)
    base, b0, _ = run_gpu(X, [p] * 4, L, 8, "mixed", params=params)
    for chi in (9, 64, 2048):
        got, bb, _ = run_gpu(X, [p] * 4, L, chi, "mixed", params=params)
        assert all(np.array_equal(u, v) for u, v in zip(b0, bb))
        for i in range(4):
            assert np.array_equal(got[i], base[i]), chi
    ref, _ = oracle_cache(X[0], p, L, 2048, params=params)
    assert np.max(np.abs(base[0] - ref)) < TOL["mixed"]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_paper_ansatz_exact_regime_rank_revealing_splits(precision):
    """Paper ansatz (Sec. II.B), 7x7, L = 3 at chi = 8 = 2^L and chi = 64.  Sequential
    sweep: the odd-bond sub-layer's theta has twice the rows and columns of its rank
    bound 2^c, and the pivoted-QR split keeps exactly the rank (bonds <= 2^L) while the
    oracle keeps the zero singular values.  Operator-product path (the brick-wall CNOTs
    as bond-2 operators): bond 2^L at every inner cut.  Both match the exact oracle."""
    p, L = 7, 3
    X = list(synth.garment_pixels(3, p, seed=130))
    ref = [oracle_cache(X[i], p, L, 64, ansatz="paper")[0] for i in range(3)]
    for pipeline in (False, True):
        for chi in (8, 64):
            got, bonds, disc = run_gpu(X, [p] * 3, L, chi, precision, ansatz="paper", pipeline=pipeline)
            if pipeline:
                assert all(list(b) == [1] + [2 ** L] * (p * p - 1) + [1] for b in bonds)
            else:
                assert all(max(b) <= 2 ** L for b in bonds)
            assert np.all(np.asarray(disc) == 0.0)          # nothing lossy
            for i in range(3):
                assert np.max(np.abs(got[i] - ref[i])) < TOL[precision], (pipeline, chi, i)


def test_mixed_batch_routes_each_image_by_its_own_circuit():
    """A batch mixing images the layer-pipelined kernel can run (chi >= 2^L) with images
    that truncate: every image gives the same bits as in a batch of its own."""
    p = 6
    X = list(synth.garment_pixels(6, p, seed=140))
    params = synth.circuit_params(3, p * p, seed=141)
    chis = np.array([8, 4, 16, 2, 8, 4], dtype=np.int32)       # L = 3: exact, lossy, ...
    from paper_2607_10280_b300.api import Batch
    px = torch.tensor(np.concatenate(X), dtype=torch.float64, device="cuda")
    pr = torch.tensor(params, dtype=torch.float64, device="cuda")
    b = Batch(np.full(6, p, np.int32), chis, "mixed")
    b.apply_circuit(px, 3, "ladder", pr)
    mixed = b.pauli_cache().cpu().numpy()
    b.close()
    m = 2 * p * (p - 1)
    for i in range(6):
        alone, _, _ = run_gpu([X[i]], [p], 3, int(chis[i]), "mixed", params=params)
        assert np.array_equal(mixed[i * m:(i + 1) * m], alone[0]), i


def test_failed_calls_leave_no_stale_state():
    """Error paths of the batch handle: a circuit refused after its argument checks
    (a bond above the largest the kernels hold) leaves no circuit for the Pauli cache to read;
    the next good circuit gives the oracle's values; refused reshape arguments leave
    the batch and its circuit as they were; a reshape asks for a new circuit."""
    from paper_2607_10280_b300._lib import MpsError
    from paper_2607_10280_b300.api import Batch
    p, chi = 5, 4096        # bond above the largest the kernels hold (128) at L = 8
    X = synth.garment_pixels(2, p, seed=31)
    params = synth.circuit_params(8, p * p, seed=32)
    px = torch.tensor(np.concatenate(X), dtype=torch.float64, device="cuda")
    pr = torch.tensor(params, dtype=torch.float64, device="cuda").contiguous()
    b = Batch(np.array([p, p], dtype=np.int32), chi, "mixed")
    b.apply_circuit(px, [2, 2], "ladder", pr)
    first = b.pauli_cache().clone()
    with pytest.raises(MpsError) as e:
        b.apply_circuit(px, [3, 8], "ladder", pr)      # bond 256 > 128 at image 1
    assert e.value.status == 5
    with pytest.raises(MpsError) as e:
        b.pauli_cache()
    assert e.value.status == 6
    b.apply_circuit(px, [2, 2], "ladder", pr)
    again = b.pauli_cache()
    b.sync()
    assert torch.equal(first, again)
    res = again.double().cpu().numpy()
    for i in range(2):
        ref, _ = oracle_cache(X[i], p, 2, chi, params=params)
        got = res[b.pair_offsets[i]:b.pair_offsets[i + 1]]
        assert np.max(np.abs(got - ref)) < TOL["mixed"]
    with pytest.raises(MpsError) as e:
        b.reshape([1], chi)                           # p = 1 refused: nothing changes
    assert e.value.status == 1
    assert torch.equal(b.pauli_cache(), first)
    b.reshape([3], chi)
    with pytest.raises(MpsError) as e:
        b.pauli_cache()
    assert e.value.status == 6
    b.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("L", [5, 6])
def test_largest_bond_bucket_32(precision, L):
    """Bonds at the largest compiled size, 32, on 5x5 images: L = 5 reaches it
    exactly (2^L), L = 6 truncates a bond of 64 to chi = 32 at the middle cuts, on
    a complex128 state for both precisions (its FP64 workspace, about 205 KB,
    shares the block's shared memory with the site buffers)."""
    p, chi, B = 5, 32, 2
    n = p * p
    X = synth.garment_pixels(B, p, seed=70 + L)
    params = synth.circuit_params(L, n, seed=71)
    got, bonds, disc = run_gpu(list(X), [p] * B, L, chi, precision, params=params)
    expect = [1] + [min(chi, 2 ** L, 2 ** (k + 1), 2 ** (n - k - 1)) for k in range(n - 1)] + [1]
    for i in range(B):
        assert list(bonds[i]) == expect
        st = o_mps.simulate(o_circ.build_circuit("ladder", X[i], L, params), n, chi)
        ref, gap = st.pair_paulis(o_pairs.image_pairs(p)), st.min_gap
        if gap < TIE_GAP:
            continue
        assert np.max(np.abs(got[i] - ref)) < TOL[precision], (i, gap, np.max(np.abs(got[i] - ref)))
        if L == 5:
            assert float(np.sum(st.discarded)) < 1e-20
        else:
            assert abs(disc[i] - float(np.sum(st.discarded))) <= 1e-10
    assert max(expect) == 32


@pytest.mark.parametrize("L,chi", [(4, 2), (4, 4), (3, 2), (2, 2)])
def test_truncated_full_batch_mixed_within_1e5_of_fp64(L, chi):
    """The chi x L sweep's truncated points at full size (1024 garment-like 7x7
    images, pixel seed 0): every Pauli entry of every image on the mixed path
    within 1e-5 of the FP64 path (itself pinned to the oracle at 1e-10 above), and
    sampled images of both against the oracle.  A complex64 state through these
    truncation chains gave up to 4e-3."""
    p, B = 7, 1024
    X = synth.garment_pixels(B, p)
    params = synth.circuit_params(L, p * p)
    mixed, _, _ = run_gpu(list(X), [p] * B, L, chi, "mixed", params=params)
    fp64, _, _ = run_gpu(list(X), [p] * B, L, chi, "fp64", params=params)
    err = max(float(np.max(np.abs(a - b))) for a, b in zip(mixed, fp64))
    assert err <= 1e-5, err
    for i in (0, 777):
        st = o_mps.simulate(o_circ.build_circuit("ladder", X[i], L, params), p * p, chi)
        if st.min_gap < TIE_GAP:
            continue
        ref = st.pair_paulis(o_pairs.image_pairs(p))
        assert np.max(np.abs(fp64[i] - ref)) < TOL["fp64"]
        assert np.max(np.abs(mixed[i] - ref)) < TOL["mixed"]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("L,chi", [(6, 64), (7, 128)])
def test_large_bonds_exact_vs_statevector(precision, L, chi):
    """Bonds of 64 and 128 (the paper's large-chi sweep): 4x4 images (16 qubits) at
    L = 6 and 7 reach bond 2^L at the middle cuts, held exactly at chi = 2^L; the
    kernels run with their workspaces in global memory.  Against the dense
    statevector."""
    p, B = 4, 2
    X = synth.garment_pixels(B, p, seed=80 + L)
    params = synth.circuit_params(L, p * p, seed=81)
    got, bonds, disc = run_gpu(list(X), [p] * B, L, chi, precision, params=params)
    n = p * p
    expect = [1] + [min(chi, 2 ** L, 2 ** (k + 1), 2 ** (n - k - 1)) for k in range(n - 1)] + [1]
    assert max(expect) == chi
    for i in range(B):
        assert list(bonds[i]) == expect
        ref, _ = oracle_cache(X[i], p, L, chi, params=params, backend="statevector")
        assert np.max(np.abs(got[i] - ref)) < TOL[precision], (i, np.max(np.abs(got[i] - ref)))
    assert np.max(disc) < 1e-12


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_bond_64_truncated_vs_oracle_mps(precision):
    """A truncation at bond 64: 5x5 images (25 qubits), L = 7, chi = 64, where the
    middle cuts would reach 128 (theta of 128 x 128, a 128 x 128 Gram matrix); both
    precisions truncate on a complex128 state.  Against the oracle MPS at the same chi,
    with the discarded weight."""
    p, L, chi, B = 5, 7, 64, 1
    X = synth.garment_pixels(B, p, seed=90)
    params = synth.circuit_params(L, p * p, seed=91)
    got, bonds, disc = run_gpu(list(X), [p] * B, L, chi, precision, params=params)
    st = o_mps.simulate(o_circ.build_circuit("ladder", X[0], L, params), p * p, chi)
    assert max(bonds[0]) == 64 and float(np.sum(st.discarded)) > 1e-8   # the cut binds
    assert abs(disc[0] - float(np.sum(st.discarded))) <= 1e-10
    if st.min_gap >= TIE_GAP:
        ref = st.pair_paulis(o_pairs.image_pairs(p))
        assert np.max(np.abs(got[0] - ref)) < TOL[precision], np.max(np.abs(got[0] - ref))


def test_large_bonds_refuse_the_diagonal_pair_set():
    from paper_2607_10280_b300._lib import MpsError
    from paper_2607_10280_b300.api import Batch
    p, L, chi = 4, 6, 64
    X = synth.garment_pixels(1, p, seed=3)
    b = Batch(np.array([p], np.int32), chi, "mixed")
    b.apply_circuit(torch.tensor(X.reshape(-1), dtype=torch.float64, device="cuda"), L, "ladder",
                    torch.tensor(synth.circuit_params(L, p * p), dtype=torch.float64, device="cuda"))
    with pytest.raises(MpsError) as e:
        b.pauli_cache(pair_set="hvd")
    assert e.value.status == 5
    b.close()


@pytest.mark.parametrize("pair_set", ["hv", "hvd"])
def test_paper_ansatz_real_kernels(pair_set):
    """The paper ansatz (H, R_Y(2 pi x - pi), CNOT: all real) gives a real state; the
    mixed path then runs real-element environment and Pauli kernels.  Against the
    complex kernels (set_real_arithmetic(False)) to rounding, against the oracle within
    1e-5, and every Pauli with one Y exactly zero."""
    from paper_2607_10280_b300.api import Batch
    p, B, chi = 5, 6, 16
    X = synth.garment_pixels(B, p, seed=61)
    px = torch.tensor(X.reshape(-1), dtype=torch.float64, device="cuda")
    for L in (2, 3):      # operator-product path (2^L <= chi), then rank-bounded splits
        res = {}
        for real in (True, False):
            b = Batch(np.full(B, p, np.int32), chi, "mixed")
            b.set_real_arithmetic(real)
            b.set_layer_pipeline(L == 2)
            b.apply_circuit(px, L, "paper")
            out = b.pauli_cache(pair_set=pair_set)
            b.sync()
            res[real] = out.double().cpu().numpy().reshape(B, -1, 16)
            b.close()
        assert np.max(np.abs(res[True] - res[False])) < 1e-6
        one_y = [4 * a + b for a in range(4) for b in range(4) if (a == 2) != (b == 2)]
        assert np.all(res[True][:, :, one_y] == 0.0)
        for i in (0, B - 1):
            ref = o_mps.simulate(o_circ.build_circuit("paper", X[i], L), p * p, chi).pair_paulis(
                o_pairs.image_pairs(p, pair_set == "hvd"))
            assert np.max(np.abs(res[True][i] - ref)) < TOL["mixed"], (L, i)


def test_fp64_chain_team_widths_agree():
    """The complex128 truncation chain on one warp per image and on 128-thread teams
    (mps_set_launch_shape circuit_threads = 128): the same FP64 arithmetic in another
    summation order, so the two agree to FP64 rounding, and both match the oracle."""
    p, L, chi, B = 5, 4, 4, 8
    X = synth.garment_pixels(B, p, seed=95)
    params = synth.circuit_params(L, p * p, seed=96)
    a, _, da = run_gpu(list(X), [p] * B, L, chi, "mixed", params=params, shape=(0, 32, 0))
    b, _, db = run_gpu(list(X), [p] * B, L, chi, "mixed", params=params, shape=(0, 128, 0))
    f, _, _ = run_gpu(list(X), [p] * B, L, chi, "fp64", params=params, shape=(0, 128, 0))
    for i in range(B):
        st = o_mps.simulate(o_circ.build_circuit("ladder", X[i], L, params), p * p, chi)
        if st.min_gap < TIE_GAP:
            continue
        ref = st.pair_paulis(o_pairs.image_pairs(p))
        assert np.max(np.abs(a[i] - b[i])) < 1e-6
        assert np.max(np.abs(b[i] - ref)) < TOL["mixed"]
        assert np.max(np.abs(f[i] - ref)) < TOL["fp64"]
        assert abs(da[i] - db[i]) < 1e-12
