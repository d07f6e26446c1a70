"""Training on cached Paulis on the GPU (ano_train_step) against the FP64 oracle:
loss, gradients, the Adam update, a short run, reproducibility and checkpoints."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import train as o_train      # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_10280_b300 import build
    build.build()


def _problem(B, m, O, seed):
    rng = np.random.default_rng(seed)
    pauli = rng.uniform(-1, 1, size=(B, m, 16))
    pauli[:, :, 0] = 1.0
    abd = rng.normal(size=(m, 16))
    W = rng.normal(size=(O, m)) / np.sqrt(m)
    b = 0.1 * rng.normal(size=O)
    Y = rng.uniform(0, 1, size=(B, O))
    return pauli, abd, W, b, Y


def _trainer(pauli, abd, W, b, m, **hp):
    from paper_2607_10280_b300.api import Trainer
    dev = torch.device("cuda")
    pt = torch.tensor(pauli.reshape(-1, 16), dtype=torch.float32, device=dev)
    t = Trainer(pt, m, torch.tensor(abd, dtype=torch.float32, device=dev),
                torch.tensor(W, dtype=torch.float32, device=dev), torch.tensor(b, dtype=torch.float32, device=dev),
                **hp)
    return t


def _f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def test_one_step_loss_gradients_and_adam_vs_oracle():
    """B = 300, m = 40, out = 200: several 128-row tiles with ragged tails."""
    B, m, O = 300, 40, 200
    pauli, abd, W, b, Y = _problem(B, m, O, 5)
    hp = dict(lr_abd=1e-2, lr_linear=1e-3, mse_weight=0.3)
    tr = _trainer(pauli, abd, W, b, m, **hp)
    loss = tr.step(torch.tensor(Y, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    from paper_2607_10280_b300.api import _lib, lib
    assert lib().ano_status() == _lib.MPS_OK
    # the oracle sees the same (float32-rounded) inputs
    ref_loss, g_abd, g_W, g_b = o_train.loss_and_grads(_f32(pauli), _f32(abd), _f32(W), _f32(b), _f32(Y), 0.3)
    assert abs(loss.item() - ref_loss) <= 1e-5 * ref_loss
    ga, gw, gb = (g.double().cpu().numpy() for g in tr.gradients())
    for got, ref in ((ga, g_abd), (gw, g_W), (gb, g_b)):
        assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref)), np.max(np.abs(got - ref))
    # Adam applied to the GPU's own gradients: the update arithmetic alone
    for got, theta, g, lr in ((tr.abd, abd, ga, 1e-2), (tr.W, W, gw, 1e-3), (tr.bias, b, gb, 1e-3)):
        want, _, _ = o_train.adam_update(_f32(theta), g, 0.0, 0.0, 1, lr)
        assert np.max(np.abs(got.double().cpu().numpy() - want)) <= 1e-6 * max(1.0, np.max(np.abs(want)))


def test_short_run_tracks_the_oracle_and_reproduces():
    B, m, O = 128, 24, 64
    pauli, abd, W, b, Y = _problem(B, m, O, 7)
    steps, lr_abd, lr_lin = 15, 3e-3, 3e-3
    *_, ref_losses = o_train.train(_f32(pauli), _f32(abd), _f32(W), _f32(b), _f32(Y), steps, lr_abd, lr_lin)
    runs = []
    for _ in range(2):
        tr = _trainer(pauli, abd, W, b, m, lr_abd=lr_abd, lr_linear=lr_lin)
        y = torch.tensor(Y, dtype=torch.float32, device="cuda")
        losses = [tr.step(y).item() for _ in range(steps)]
        runs.append((losses, tr.abd.cpu().clone(), tr.W.cpu().clone()))
    losses = runs[0][0]
    assert np.allclose(losses, ref_losses, rtol=1e-4), (losses[-1], ref_losses[-1])
    assert losses[-1] < losses[0]
    assert runs[0][0] == runs[1][0]                                   # bit-reproducible
    assert torch.equal(runs[0][1], runs[1][1]) and torch.equal(runs[0][2], runs[1][2])


def test_checkpoint_resume_and_cache_round_trip(tmp_path):
    from paper_2607_10280_b300 import api
    B, m, O = 64, 12, 30
    pauli, abd, W, b, Y = _problem(B, m, O, 9)
    y = torch.tensor(Y, dtype=torch.float32, device="cuda")
    full = _trainer(pauli, abd, W, b, m)
    for _ in range(6):
        full.step(y)
    part = _trainer(pauli, abd, W, b, m)
    for _ in range(3):
        part.step(y)
    sd = part.state_dict()
    path = str(tmp_path / "cache.npz")
    api.save_pauli_cache(path, part.pauli, {"p": 4, "L": 2, "chi": 8})
    cache = api.load_pauli_cache(path, "cuda")
    assert torch.equal(cache, part.pauli)
    resumed = api.Trainer(cache, m, torch.empty_like(part.abd), torch.empty_like(part.W),
                          torch.empty_like(part.bias))
    resumed.load_state_dict(sd)
    for _ in range(3):
        resumed.step(y)
    assert torch.equal(resumed.W, full.W) and torch.equal(resumed.abd, full.abd)
    assert torch.equal(resumed.bias, full.bias)
