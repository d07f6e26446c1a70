"""The per-image sweep Pauli kernel against the column-walk kernel (GPU tests).

Both accumulate every product and every closing sum in the same order, so the caches
must agree bit for bit, over the kernel variants the sweep has: half-structured
operator-product images (with left environments), left-canonical images from the
truncating circuit kernel, dense operator-product images, real elements (paper ansatz),
the diagonal pair sets, and batches of mixed image sizes (slots sized by the largest
side).  The parity tests against the oracle run through the sweep by default.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import circuit as o_circ     # noqa: E402
from oracle import mps as o_mps          # noqa: E402
from oracle import pairs as o_pairs      # noqa: E402
from paper_2607_10280_b300 import synth  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_10280_b300 import build
    build.build()


def _caches(ps, L, chi, ansatz="ladder", pair_set="hv", seed=0, half=True, real=True, pipeline=True):
    from paper_2607_10280_b300.api import Batch
    from paper_2607_10280_b300._lib import lib
    X = [synth.garment_pixels(1, p, seed=seed + i)[0] for i, p in enumerate(ps)]
    px = torch.tensor(np.concatenate(X), dtype=torch.float64, device="cuda")
    params = None
    if ansatz == "ladder":
        params = torch.tensor(synth.circuit_params(L, max(ps) ** 2, seed=seed), dtype=torch.float64,
                              device="cuda").contiguous()
    res = {}
    for sweep in (True, False):
        b = Batch(np.asarray(ps, dtype=np.int32), chi, "mixed")
        b.set_half_structure(half)
        b.set_real_arithmetic(real)
        b.set_layer_pipeline(pipeline)
        b.set_pauli_sweep(sweep)
        b.apply_circuit(px, L, ansatz, params)
        n0 = lib().mps_launch_count()
        out = b.pauli_cache(pair_set=pair_set)
        b.sync()
        res[sweep] = (out.double().cpu().numpy(), list(b.pair_offsets_for(pair_set)),
                      lib().mps_launch_count() - n0)
        b.close()
    return X, res


def _check_equal(res):
    a, offs, _ = res[True]
    c, _, _ = res[False]
    assert a.shape == c.shape
    assert np.isfinite(a).all()
    assert np.array_equal(a, c), float(np.max(np.abs(a - c)))
    return a, offs


@pytest.mark.parametrize("pair_set", ["hv", "hvd"])
def test_sweep_half_structured_headline_shape(pair_set):
    """7x7, L = 4, chi = 16: operator-product images, every site half-structured, left
    environments; the sweep launches the left-environment chains and itself."""
    X, res = _caches([7] * 24, 4, 16, pair_set=pair_set, seed=3)
    a, offs = _check_equal(res)
    assert res[True][2] <= 2
    for i in (0, 23):
        ref = o_mps.simulate(o_circ.build_circuit("ladder", X[i], 4, synth.circuit_params(4, 49, seed=3)), 49,
                             16).pair_paulis(o_pairs.image_pairs(7, pair_set == "hvd"))
        assert np.max(np.abs(a[offs[i]:offs[i + 1]] - ref)) < 1e-5


@pytest.mark.parametrize("pair_set", ["hv", "hvd"])
def test_sweep_left_canonical_truncated_images(pair_set):
    """6x6, L = 4, chi = 4: lossy truncation (complex128 chain, rounded), left-canonical
    sites, no left environments, dense contractions."""
    _check_equal(_caches([6] * 12, 4, 4, pair_set=pair_set, seed=11)[1])


@pytest.mark.parametrize("pair_set", ["hv", "hvd"])
def test_sweep_dense_operator_product_images(pair_set):
    """Operator-product images with the half structure switched off (the dense kernel
    variant with left environments), chi = 8 at L = 3."""
    _check_equal(_caches([5] * 10, 3, 8, pair_set=pair_set, seed=21, half=False)[1])


@pytest.mark.parametrize("pair_set", ["hv", "hvd"])
def test_sweep_mixed_image_sizes(pair_set):
    """Sides 2 .. 7 in one batch: the slots are sized for the largest side, every image
    walks its own chain."""
    _check_equal(_caches([3, 7, 5, 2, 4, 6, 7, 3], 3, 8, pair_set=pair_set, seed=31)[1])
    _check_equal(_caches([4, 6, 5, 7], 2, 4, pair_set=pair_set, seed=37)[1])


@pytest.mark.parametrize("pair_set", ["hv", "hvd"])
@pytest.mark.parametrize("real", [True, False])
def test_sweep_paper_ansatz(pair_set, real):
    """The paper ansatz at 5x5: real elements (and the complex kernels), operator
    product (L = 2) and rank-bounded splits (L = 3)."""
    for L in (2, 3):
        _check_equal(_caches([5] * 8, L, 16, ansatz="paper", pair_set=pair_set, seed=41 + L, real=real,
                             pipeline=L == 2)[1])
