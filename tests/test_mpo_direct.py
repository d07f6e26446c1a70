"""Circuits as operator products: the closed-form site kernel against the
layer-by-layer one, ladder and brick-wall (GPU tests).

Both build the exact MPS of L ladder layers (Sec. II.B) with bond 2^L; the closed form
computes every site element as one product of gate entries and rounds it in the order
the layered kernel does, so the two must give the same site tensors, hence the same
Pauli caches bit for bit, and both must match the oracle.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import pipeline as o_pipe    # noqa: E402
from paper_2607_10280_b300 import synth  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_10280_b300 import build
    build.build()


def run(X, p, L, chi, precision, params, layered, ansatz="ladder"):
    from paper_2607_10280_b300.api import Batch
    old = os.environ.get("MPSANO_MPO")
    if layered:
        os.environ["MPSANO_MPO"] = "layered"
    else:
        os.environ.pop("MPSANO_MPO", None)
    try:
        px = torch.tensor(np.concatenate(list(X)), dtype=torch.float64, device="cuda")
        pr = None if params is None else torch.tensor(params, dtype=torch.float64, device="cuda").contiguous()
        b = Batch(np.full(len(X), p, np.int32), chi, precision)
        b.apply_circuit(px, L, ansatz, pr)
        out = b.pauli_cache()
        b.sync()
        res = out.double().cpu().numpy().reshape(len(X), -1, 16)
        bonds = b.bond_dims()
        b.close()
    finally:
        if old is None:
            os.environ.pop("MPSANO_MPO", None)
        else:
            os.environ["MPSANO_MPO"] = old
    return res, bonds


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("p,L,chi", [(2, 1, 4), (3, 2, 4), (4, 3, 8), (7, 4, 16), (5, 4, 32)])
def test_closed_form_matches_layered_kernel(precision, p, L, chi):
    B = 5
    X = synth.garment_pixels(B, p, seed=400 + p + L)
    params = synth.circuit_params(L, p * p, seed=401)
    direct, bd = run(X, p, L, chi, precision, params, layered=False)
    layered, bl = run(X, p, L, chi, precision, params, layered=True)
    assert [list(x) for x in bd] == [list(x) for x in bl]
    assert np.array_equal(direct, layered)
    tol = 1e-10 if precision == "fp64" else 1e-5
    for i in (0, B - 1):
        ref = o_pipe.pauli_cache(X[i], p, L, chi, "ladder", params)
        assert np.max(np.abs(direct[i] - ref)) < tol, (i, np.max(np.abs(direct[i] - ref)))


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("p,L,chi", [(3, 1, 4), (4, 2, 4), (5, 3, 8), (7, 4, 16)])
def test_closed_form_matches_layered_kernel_paper_ansatz(precision, p, L, chi):
    """The paper's brick-wall circuit (H, R_Y(2 pi x - pi) every layer, CNOTs on the even
    then the odd bonds): even sites take the CNOT on their right bond first."""
    B = 4
    X = synth.garment_pixels(B, p, seed=500 + p + L)
    direct, bd = run(X, p, L, chi, precision, None, layered=False, ansatz="paper")
    layered, bl = run(X, p, L, chi, precision, None, layered=True, ansatz="paper")
    assert [list(x) for x in bd] == [list(x) for x in bl]
    assert np.array_equal(direct, layered)
    tol = 1e-10 if precision == "fp64" else 1e-5
    for i in (0, B - 1):
        ref = o_pipe.pauli_cache(X[i], p, L, chi, "paper")
        assert np.max(np.abs(direct[i] - ref)) < tol, (i, np.max(np.abs(direct[i] - ref)))
