"""FP64 truncation: the block solve against the full eigen-decomposition (GPU tests).

A truncation at the orthogonality centre (Sec. II.B) keeps the span of the chi largest
eigenvectors of theta's Gram matrix; the basis inside that span is a gauge of the new
bond.  Where the cut lies in a clear gap the FP64 Jacobi step only decouples the kept
from the dropped directions (mps_set_block_truncation, on by default).  These tests run
the same truncating circuits with the block solve on and off: the Pauli caches and the
discarded weights must agree to FP64 rounding, and both must match the oracle MPS.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import circuit as o_circ     # noqa: E402
from oracle import mps as o_mps          # noqa: E402
from oracle import pairs as o_pairs      # noqa: E402
from paper_2607_10280_b300 import synth  # noqa: E402

TIE_GAP = 1e-6


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_10280_b300 import build
    build.build()


def run(X, p, L, chi, precision, params, block, threads=None):
    from paper_2607_10280_b300.api import Batch
    px = torch.tensor(np.concatenate(list(X)), dtype=torch.float64, device="cuda")
    pr = torch.tensor(params, dtype=torch.float64, device="cuda").contiguous()
    b = Batch(np.full(len(X), p, np.int32), chi, precision)
    b.set_block_truncation(block)
    if threads:
        b.set_launch_shape(0, threads, 0)
    b.apply_circuit(px, L, "ladder", pr)
    out = b.pauli_cache()
    b.sync()
    res = out.double().cpu().numpy().reshape(len(X), -1, 16)
    disc = b.discarded_weight()
    b.close()
    return res, disc


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("p,L,chi,threads", [(5, 3, 2, None), (6, 4, 4, None), (6, 4, 8, 128), (7, 4, 4, None)])
def test_block_solve_matches_full_eigendecomposition(precision, p, L, chi, threads):
    n = p * p
    B = 6
    X = synth.garment_pixels(B, p, seed=300 + p + L)
    params = synth.circuit_params(L, n, seed=301)
    blk, dblk = run(X, p, L, chi, precision, params, True, threads)
    full, dfull = run(X, p, L, chi, precision, params, False, threads)
    prs = o_pairs.image_pairs(p)
    tol = 1e-10 if precision == "fp64" else 1e-5
    checked = 0
    for i in range(B):
        st = o_mps.simulate(o_circ.build_circuit("ladder", X[i], L, params), n, chi)
        assert abs(dblk[i] - dfull[i]) <= 1e-12, (i, dblk[i], dfull[i])
        if st.min_gap < TIE_GAP:
            continue
        ref = st.pair_paulis(prs)
        # both solves give the same truncated state: their caches agree to FP64 rounding
        # (the complex64 rounding of the final state on the mixed path comes on top)
        assert np.max(np.abs(blk[i] - full[i])) <= (1e-11 if precision == "fp64" else 1e-6), i
        assert np.max(np.abs(blk[i] - ref)) < tol, (i, np.max(np.abs(blk[i] - ref)))
        assert np.max(np.abs(full[i] - ref)) < tol, (i, np.max(np.abs(full[i] - ref)))
        checked += 1
    assert checked >= B // 2
    assert np.max(dblk) > 1e-8   # the circuits truncate for real
