"""Oracle: conditional flow matching loss, its gradient and AdamW, in FP64
(test infrastructure only).

Eq. 9: L(theta) = E_{t ~ U[0,1], x0, x1} || v_theta(x_t, t) - dx_t/dt ||^2 with
the linear (conditional optimal transport) path x_t = (1 - t) x0 + t x1, so
dx_t/dt = x1 - x0. The expectation over a batch of B rows is the batch mean of
the squared Euclidean norm over the 4 state components:
    L = (1/B) sum_b sum_d (v_bd - (x1_bd - x0_bd))^2.
Here x1 is the standardized exit state y of a training transmission, x0 a
standard normal draw, t a uniform draw and c the standardized condition, all
passed in as inputs.

The gradient is the hand-derived reverse pass through the network of
`oracle.mlp` (linear layers and SiLU, silu'(z) = sig(z) (1 + z (1 - sig(z)))).

AdamW is the decoupled-weight-decay Adam of Loshchilov & Hutter: with bias
corrections m_hat = m / (1 - b1^k), v_hat = v / (1 - b2^k),
    p <- p (1 - lr wd) - lr m_hat / (sqrt(v_hat) + eps),
applied to every weight and bias.
"""
import numpy as np

from .mlp import time_embedding


def _sig(z):
    return 1.0 / (1.0 + np.exp(-z))


def forward_cache(W, b, cn, x, t):
    """Forward pass keeping pre-activations; returns (v, cache)."""
    h = np.concatenate([cn, x, time_embedding(t)], axis=1)
    acts, pres = [h], []
    for l in range(4):
        z = h @ W[l].T + b[l]
        pres.append(z)
        h = z * _sig(z)
        acts.append(h)
    v = h @ W[4].T + b[4]
    return v, (acts, pres)


def cfm_loss_grad(W, b, cn, x1, x0, t):
    """Returns (loss, gW list, gb list) for one batch (all arrays FP64).

    cn [B,5] standardized conditions, x1 [B,4] standardized targets,
    x0 [B,4] noise, t [B] flow times.
    """
    W = [np.asarray(w, np.float64) for w in W]
    b = [np.asarray(v, np.float64) for v in b]
    B = x1.shape[0]
    t = np.asarray(t, dtype=np.float64)
    xt = (1.0 - t)[:, None] * x0 + t[:, None] * x1
    target = x1 - x0
    v, (acts, pres) = forward_cache(W, b, cn, xt, t)
    r = v - target
    loss = float(np.sum(r * r) / B)
    gW = [None] * 5
    gb = [None] * 5
    d = 2.0 * r / B
    gW[4] = d.T @ acts[4]
    gb[4] = d.sum(axis=0)
    da = d @ W[4]
    for l in range(3, -1, -1):
        z = pres[l]
        s = _sig(z)
        dz = da * (s * (1.0 + z * (1.0 - s)))
        gW[l] = dz.T @ acts[l]
        gb[l] = dz.sum(axis=0)
        da = dz @ W[l]
    return loss, gW, gb


def adamw_step(p, g, m, v, k, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, wd=0.01):
    """One AdamW update at step k >= 1; returns new (p, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    m_hat = m / (1.0 - b1 ** k)
    v_hat = v / (1.0 - b2 ** k)
    p = p * (1.0 - lr * wd) - lr * m_hat / (np.sqrt(v_hat) + eps)
    return p, m, v
