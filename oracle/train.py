"""Training on cached Pauli expectations (oracle; test infrastructure only).

Sec. II.C: the Pauli expectations depend on the image only, so they are computed
once and cached; training then updates the observable parameters (A, B, D) and
the linear layer (W, b) of Eq. 5 and Eq. 6.  Sec. II.D, Eq. 7: the loss weights
MSE and LPIPS; only the MSE term is built here (LPIPS needs a pretrained network),
L = lambda_MSE * mean_{i,o} (y_hat[i][o] - y[i][o])^2.  Two separate Adam
optimizers update (A, B, D) and (W, b) (Sec. II.D; Adam as defined by Kingma and
Ba, 2015, Algorithm 1, with the bias corrections).

Everything is FP64 numpy and follows the chain rule term by term:
  c[q] = M abd[q]                       (Eq. 4, M[alpha][k] = Tr(H(e_k) P_alpha) / 4)
  f[i][q] = sum_alpha c[q][alpha] P[i][q][alpha]                        (Eq. 5)
  y_hat[i] = W f[i] + b                                                 (Eq. 6)
  g_yhat = 2 lambda / (B O) (y_hat - y)
  g_W = g_yhat^T f,  g_b = sum_i g_yhat[i],  g_f = g_yhat W
  g_c[q][alpha] = sum_i g_f[i][q] P[i][q][alpha],  g_abd[q] = M^T g_c[q]
"""
from __future__ import annotations

import numpy as np

from . import ano


def coefficient_map() -> np.ndarray:
    """M [16][16]: column k holds the Pauli coefficients of the unit parameter e_k."""
    M = np.zeros((16, 16))
    for k in range(16):
        e = np.zeros(16)
        e[k] = 1.0
        M[:, k] = ano.coefficients(e)
    return M


def forward(pauli: np.ndarray, abd: np.ndarray, W: np.ndarray, b: np.ndarray):
    """pauli [B][m][16], abd [m][16], W [O][m], b [O] -> (features [B][m], y_hat [B][O])."""
    c = np.stack([ano.coefficients(abd[q]) for q in range(abd.shape[0])])      # [m][16]
    f = np.einsum("qa,iqa->iq", c, pauli)
    return f, f @ W.T + b


def loss_and_grads(pauli, abd, W, b, Y, mse_weight: float = 1.0):
    """Loss and its gradients with respect to abd, W and b (all FP64)."""
    pauli = np.asarray(pauli, dtype=np.float64)
    f, y_hat = forward(pauli, abd, W, b)
    B, O = y_hat.shape
    r = y_hat - Y
    loss = mse_weight * float(np.mean(r * r))
    g_yhat = 2.0 * mse_weight / (B * O) * r
    g_W = g_yhat.T @ f
    g_b = g_yhat.sum(axis=0)
    g_f = g_yhat @ W
    g_c = np.einsum("iq,iqa->qa", g_f, pauli)
    g_abd = g_c @ coefficient_map()
    return loss, g_abd, g_W, g_b


def adam_update(theta, grad, m, v, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
                eps: float = 1e-8):
    """One Adam step (Kingma and Ba, Algorithm 1): returns (theta, m, v) updated."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    return theta - lr * m_hat / (np.sqrt(v_hat) + eps), m, v


def train(pauli, abd, W, b, Y, steps: int, lr_abd: float, lr_linear: float, mse_weight: float = 1.0,
          beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """`steps` full-batch steps; returns (abd, W, b, losses) with losses[t] before step t+1."""
    abd, W, b = (np.array(x, dtype=np.float64) for x in (abd, W, b))
    state = {k: (np.zeros_like(x), np.zeros_like(x)) for k, x in (("abd", abd), ("W", W), ("b", b))}
    losses = []
    for t in range(1, steps + 1):
        loss, g_abd, g_W, g_b = loss_and_grads(pauli, abd, W, b, Y, mse_weight)
        losses.append(loss)
        abd, *state["abd"] = adam_update(abd, g_abd, *state["abd"], t, lr_abd, beta1, beta2, eps)
        W, *state["W"] = adam_update(W, g_W, *state["W"], t, lr_linear, beta1, beta2, eps)
        b, *state["b"] = adam_update(b, g_b, *state["b"], t, lr_linear, beta1, beta2, eps)
    return abd, W, b, losses
