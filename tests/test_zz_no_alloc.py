"""The no-allocation entry point (mps_pauli_cache_noalloc) against the allocating
one (mps_create_batch + mps_apply_circuit + mps_pauli_cache), two calls in a row.

Some callers cannot allocate device memory (a plug-in inside an application that
owns the GPU's memory, a process whose framework reserved the whole device, a
serving loop that must not stall on cudaMalloc); this entry point keeps all its
working memory in a fixed array inside the library.  The file sorts last so that
a run stopping at the first failure has already run every other test.
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
    B = len(X)
    m = 2 * p * (p - 1)
    px = torch.tensor(X.reshape(-1), dtype=torch.float64, device="cuda")
    out = torch.full((B * m, 16), float("nan"), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    st = lib.mps_pauli_cache_noalloc(B, p, chi, L, ctypes.c_void_p(px.data_ptr()),
                                     ctypes.c_void_p(params.data_ptr()), params.shape[1],
                                     ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert st == 0, lib.mps_last_error()
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(B, m, 16)


def test_noalloc_matches_allocating_entry_point_twice(lib):
    from paper_2607_10280_b300 import synth
    cases = [(7, 16, 4, 12, 0), (5, 3, 3, 20, 1)]   # (p, chi, L, images, seed): exact, then truncating
    for p, chi, L, B, seed in cases:
        X = synth.garment_pixels(B, p, seed=40 + seed)
        params = torch.tensor(synth.circuit_params(L, p * p, seed=41 + seed), dtype=torch.float64, device="cuda")
        ref = allocating_path(X, p, chi, L, params)
        got = noalloc_path(lib, X, p, chi, L, params)
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref)) <= TOL, (p, chi, L, np.max(np.abs(got - ref)))


def test_noalloc_rejects_oversized_requests(lib):
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    outp = torch.zeros(1, dtype=torch.float32, device="cuda")
    args = (ctypes.c_void_p(dummy.data_ptr()), ctypes.c_void_p(dummy.data_ptr()), 256,
            ctypes.c_void_p(outp.data_ptr()), None)
    assert lib.mps_pauli_cache_noalloc(65, 7, 16, 4, *args) == 1
    assert b"n_images" in lib.mps_last_error()
    assert lib.mps_pauli_cache_noalloc(64, 16, 32, 4, *args) == 1   # 64 x 256 qubits at bond 16
    assert b"limit" in lib.mps_last_error()
