"""Pins of the training oracle (CPU): hand-derived Pauli coefficients of the
parameter map, central-difference gradients, Adam's closed form under a constant
gradient, and a realisable fit whose loss falls."""
import numpy as np
import pytest

from oracle import ano, train


def _problem(B=3, m=4, O=5, seed=0):
    rng = np.random.default_rng(seed)
    pauli = rng.uniform(-1, 1, size=(B, m, 16))
    pauli[:, :, 0] = 1.0
    abd = rng.normal(size=(m, 16))
    W = rng.normal(size=(O, m)) / np.sqrt(m)
    b = 0.1 * rng.normal(size=O)
    Y = rng.uniform(0, 1, size=(B, O))
    return pauli, abd, W, b, Y


def test_coefficient_map_hand_derived_entries():
    """Tr(H P)/4 worked out by hand from the Pauli matrices:
    c_II = (D0+D1+D2+D3)/4, c_ZZ = (D0-D1-D2+D3)/4, c_IZ = (D0-D1+D2-D3)/4,
    c_XX = (A03 + A12)/2, c_YY = (A12 - A03)/2, c_XI = (A02 + A13)/2,
    c_IY = -(B01 + B23)/2 (upper pairs (0,1),(0,2),(0,3),(1,2),(1,3),(2,3))."""
    M = train.coefficient_map()
    A = lambda u: u           # noqa: E731  parameter index of Re H[k][l]
    Bi = lambda u: 6 + u      # noqa: E731  parameter index of Im H[k][l]
    D = lambda k: 12 + k      # noqa: E731
    expect = {
        0: {D(0): .25, D(1): .25, D(2): .25, D(3): .25},            # II
        15: {D(0): .25, D(1): -.25, D(2): -.25, D(3): .25},         # ZZ
        3: {D(0): .25, D(1): -.25, D(2): .25, D(3): -.25},          # IZ
        5: {A(2): .5, A(3): .5},                                    # XX
        10: {A(3): .5, A(2): -.5},                                  # YY
        4: {A(1): .5, A(4): .5},                                    # XI
        2: {Bi(0): -.5, Bi(5): -.5},                                # IY
    }
    for alpha, row in expect.items():
        want = np.zeros(16)
        for k, v in row.items():
            want[k] = v
        assert np.allclose(M[alpha], want, atol=1e-15), alpha
    rng = np.random.default_rng(1)
    x = rng.normal(size=16)
    assert np.allclose(M @ x, ano.coefficients(x), atol=1e-14)       # the map is linear


def test_gradients_match_central_differences():
    pauli, abd, W, b, Y = _problem()
    lam = 0.3
    loss, g_abd, g_W, g_b = train.loss_and_grads(pauli, abd, W, b, Y, lam)
    h = 1e-6

    def fd(arr, idx):
        old = arr[idx]
        arr[idx] = old + h
        lp = train.loss_and_grads(pauli, abd, W, b, Y, lam)[0]
        arr[idx] = old - h
        lm = train.loss_and_grads(pauli, abd, W, b, Y, lam)[0]
        arr[idx] = old
        return (lp - lm) / (2 * h)

    for arr, g in ((abd, g_abd), (W, g_W), (b, g_b)):
        for idx in np.ndindex(arr.shape):
            assert abs(fd(arr, idx) - g[idx]) < 1e-8 * max(1.0, abs(g[idx])), idx


def test_loss_is_weighted_mean_squared_error():
    pauli, abd, W, b, Y = _problem(seed=2)
    f, y_hat = train.forward(pauli, abd, W, b)
    for i in range(pauli.shape[0]):                                   # Eq. 5 and Eq. 6 per image
        assert np.allclose(f[i], ano.features(pauli[i], abd), atol=1e-13)
        assert np.allclose(y_hat[i], ano.linear(W, f[i], b), atol=1e-13)
    l1 = train.loss_and_grads(pauli, abd, W, b, Y, 1.0)
    l3 = train.loss_and_grads(pauli, abd, W, b, Y, 0.3)
    assert np.isclose(l1[0], np.mean((y_hat - Y) ** 2))
    assert np.isclose(l3[0], 0.3 * l1[0])
    for a, c in zip(l1[1:], l3[1:]):
        assert np.allclose(c, 0.3 * a)


@pytest.mark.parametrize("g", [0.5, -2.0, 1e-3])
def test_adam_constant_gradient_closed_form(g):
    """Under a constant gradient the bias-corrected moments are exactly g and g^2, so
    every step moves the parameter by lr * g / (|g| + eps)."""
    theta, m, v = np.array([1.0]), np.zeros(1), np.zeros(1)
    lr, eps = 0.01, 1e-8
    for t in range(1, 6):
        new, m, v = train.adam_update(theta, np.array([g]), m, v, t, lr, 0.9, 0.999, eps)
        assert np.isclose(theta - new, lr * g / (abs(g) + eps), rtol=1e-12, atol=0)[0]
        theta = new


def test_realisable_fit_loss_falls():
    rng = np.random.default_rng(3)
    B, m, O = 64, 6, 10
    pauli = rng.uniform(-1, 1, size=(B, m, 16))
    pauli[:, :, 0] = 1.0
    abd_true, W_true, b_true = rng.normal(size=(m, 16)), rng.normal(size=(O, m)), rng.normal(size=O)
    Y = train.forward(pauli, abd_true, W_true, b_true)[1]
    abd0 = abd_true + 0.5 * rng.normal(size=(m, 16))
    W0 = W_true + 0.5 * rng.normal(size=(O, m))
    *_, losses = train.train(pauli, abd0, W0, np.zeros(O), Y, 300, 0.01, 0.01)
    assert losses[-1] < 0.05 * losses[0]
