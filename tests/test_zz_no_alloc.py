"""The no-allocation entry point (mps_pauli_cache_noalloc) against the allocating
one (mps_create_batch + mps_apply_circuit + mps_pauli_cache) and against the CPU
oracle, two calls in a row per case.

Some callers cannot allocate device memory: a plug-in inside an application that
owns the GPU's memory through its own allocator, a process whose framework
reserved the whole device at start-up, a serving loop that must not stall on
cudaMalloc.  This entry point keeps all its working memory in a fixed array
inside the library and reports its device-side checks through a caller-owned
status word.  The file sorts last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5   # the mixed-path tolerance used by the other parity tests


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_10280_b300 import _lib, build
    build.build()
    return _lib.lib()


def allocating_path(X, p, chi, L, params):
    from paper_2607_10280_b300.api import Batch
    b = Batch(np.full(len(X), p, np.int32), chi, "mixed")
    b.apply_circuit(torch.tensor(X.reshape(-1), dtype=torch.float64, device="cuda"), L, "ladder", params)
    out = b.pauli_cache()
    b.sync()
    res = out.cpu().numpy().reshape(len(X), -1, 16)
    b.close()
    return res


def noalloc_path(lib, X, p, chi, L, params):
    """One call; returns the Pauli cache and the call's device status word."""
    B = len(X)
    m = 2 * p * (p - 1)
    px = torch.tensor(X.reshape(-1), dtype=torch.float64, device="cuda")
    out = torch.full((B * m, 16), float("nan"), dtype=torch.float32, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    pr = ctypes.c_void_p(params.data_ptr()) if params is not None else None
    pn = params.shape[1] if params is not None else 0
    st = lib.mps_pauli_cache_noalloc(B, p, chi, L, ctypes.c_void_p(px.data_ptr()), pr, pn,
                                     ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(status.data_ptr()),
                                     ctypes.c_void_p(stream.cuda_stream))
    assert st == 0, lib.mps_last_error()
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(B, m, 16), int(status.item())


def oracle(x, p, chi, L, params_np):
    from oracle import pipeline as o_pipe
    ref, st = o_pipe.pauli_cache(x, p, L, chi, "ladder", params_np, return_state=True)
    return ref, st.min_gap


# (p, chi, L, images, seed): exact regime; truncating (complex128 chain); the largest
# image count at bond 16 (62 x 49 x 2 x 16^2 x 8 B <= 12 MiB); a truncation at bond 32
CASES = [(7, 16, 4, 12, 0), (5, 3, 3, 20, 1), (7, 16, 4, 62, 2), (6, 32, 6, 2, 3)]


@pytest.mark.parametrize("p,chi,L,B,seed", CASES)
def test_noalloc_matches_allocating_entry_point_and_oracle_twice(lib, p, chi, L, B, seed):
    from paper_2607_10280_b300 import synth
    X = synth.garment_pixels(B, p, seed=40 + seed)
    params_np = synth.circuit_params(L, p * p, seed=41 + seed)
    params = torch.tensor(params_np, dtype=torch.float64, device="cuda")
    ref = allocating_path(X, p, chi, L, params)
    for call in range(2):
        got, status = noalloc_path(lib, X, p, chi, L, params)
        assert status == 0, (call, status)
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref)) <= TOL, (call, p, chi, L, np.max(np.abs(got - ref)))
    for i in sorted({0, B - 1}):
        o, gap = oracle(X[i], p, chi, L, params_np)
        if gap < 1e-6:
            continue   # near-tie at a truncation cut: no unique answer
        assert np.max(np.abs(got[i] - o)) <= TOL, (i, np.max(np.abs(got[i] - o)))


def test_noalloc_encoding_only_closed_form_after_a_larger_call(lib):
    """L = 0 (no gate table, no two-qubit gate) right after a large call: the product
    state's closed form <X> = sin(pi x), <Y> = 0, <Z> = cos(pi x), pairs factorised."""
    from oracle import pairs as o_pairs
    from paper_2607_10280_b300 import synth
    big = synth.garment_pixels(62, 7, seed=9)
    params = torch.tensor(synth.circuit_params(4, 49, seed=9), dtype=torch.float64, device="cuda")
    _, status = noalloc_path(lib, big, 7, 16, 4, params)
    assert status == 0
    p, B = 4, 8
    X = synth.uniform_pixels(B, p, seed=11)
    for call in range(2):
        got, status = noalloc_path(lib, X, p, 4, 0, None)
        assert status == 0
        for i in range(B):
            single = np.stack([np.ones(p * p), np.sin(np.pi * X[i]), np.zeros(p * p), np.cos(np.pi * X[i])], 1)
            ref = np.array([np.outer(single[a], single[b]).reshape(16) for a, b in o_pairs.image_pairs(p)])
            assert np.max(np.abs(got[i] - ref)) <= TOL, (call, i)


def test_noalloc_small_call_after_large_one_matches_alone(lib):
    """Per-call state is cleared: a small truncating call after a large exact one
    gives what the allocating path gives."""
    from paper_2607_10280_b300 import synth
    big = synth.garment_pixels(62, 7, seed=21)
    pb = torch.tensor(synth.circuit_params(4, 49, seed=21), dtype=torch.float64, device="cuda")
    X = synth.garment_pixels(3, 3, seed=22)
    ps = torch.tensor(synth.circuit_params(2, 9, seed=22), dtype=torch.float64, device="cuda")
    ref = allocating_path(X, 3, 2, 2, ps)
    for _ in range(2):
        noalloc_path(lib, big, 7, 16, 4, pb)
        got, status = noalloc_path(lib, X, 3, 2, 2, ps)
        assert status == 0
        assert np.max(np.abs(got - ref)) <= TOL


def test_noalloc_rejects_oversized_requests(lib):
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    outp = torch.zeros(1, dtype=torch.float32, device="cuda")
    args = (ctypes.c_void_p(dummy.data_ptr()), ctypes.c_void_p(dummy.data_ptr()), 256,
            ctypes.c_void_p(outp.data_ptr()), None, None)
    assert lib.mps_pauli_cache_noalloc(65, 7, 16, 4, *args) == 1
    assert b"n_images" in lib.mps_last_error()
    assert lib.mps_pauli_cache_noalloc(64, 16, 32, 4, *args) == 1   # 64 x 256 qubits at bond 16
    assert b"limit" in lib.mps_last_error()
    assert lib.mps_pauli_cache_noalloc(63, 7, 16, 4, *args) == 1    # one image above the site storage
    assert b"limit" in lib.mps_last_error()
