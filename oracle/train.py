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
For the residual-modulated network (the reading in `oracle.mlp`: blocks
a' = a + SiLU(g z), z = W a + b + M c, g = 1 + G[0] c_3 + G[1] c_4) the
reverse pass of a block, with da the gradient reaching a', is
    dp = da silu'(g z),  dz = dp g,  dW = dz^T a,  db = sum dz,  dM = dz^T c,
    dG[0] = sum (dp z c_3),  dG[1] = sum (dp z c_4),  da <- da + dz W
(the residual path carries da through unchanged).

AdamW is the decoupled-weight-decay Adam of Loshchilov & Hutter: with bias
corrections m_hat = m / (1 - b1^k), v_hat = v / (1 - b2^k),
    p <- p (1 - lr wd) - lr m_hat / (sqrt(v_hat) + eps),
applied to every weight and bias.
"""
import numpy as np

from .mlp import network_input


def _sig(z):
    return 1.0 / (1.0 + np.exp(-z))


def forward_cache(W, b, cn, x, t):
    """Forward pass keeping pre-activations; returns (v, cache)."""
    h = network_input(cn, x, t)
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

    cn [B,5] standardized conditions ([B,6] for rectangular cells: W[0]
    then has 26 columns), x1 [B,4] standardized targets,
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


def forward_cache_rm(P, cn, x, t):
    """Forward pass of the residual-modulated network (P: dict of W, b, M, G
    as oracle.mlp.Net holds them) keeping every block's input, z and g."""
    h = network_input(cn, x, t)
    z1 = h @ P["W"][0].T + P["b"][0]
    a = z1 * _sig(z1)
    blocks = []
    for j in range(3):
        z = a @ P["W"][j + 1].T + P["b"][j + 1] + cn @ P["M"][j].T
        g = 1.0 + cn[:, 3:4] * P["G"][j][0][None, :] + cn[:, 4:5] * P["G"][j][1][None, :]
        blocks.append((a, z, g))
        p = g * z
        a = a + p * _sig(p)
    v = a @ P["W"][4].T + P["b"][4]
    return v, (h, z1, blocks, a)


def cfm_loss_grad_rm(P, cn, x1, x0, t):
    """Loss and gradient of Eq. 9 for the residual-modulated network: returns
    (loss, grads) with grads a dict of W, b (lists of 5), M and G (lists of 3)."""
    P = {"W": [np.asarray(w, np.float64) for w in P["W"]],
         "b": [np.asarray(v, np.float64) for v in P["b"]],
         "M": [np.asarray(m, np.float64) for m in P["M"]],
         "G": [np.asarray(q, np.float64) for q in P["G"]]}
    B = x1.shape[0]
    t = np.asarray(t, dtype=np.float64)
    xt = (1.0 - t)[:, None] * x0 + t[:, None] * x1
    v, (h, z1, blocks, a4) = forward_cache_rm(P, cn, xt, t)
    r = v - (x1 - x0)
    loss = float(np.sum(r * r) / B)
    gW, gb, gM, gG = [None] * 5, [None] * 5, [None] * 3, [None] * 3
    d = 2.0 * r / B
    gW[4] = d.T @ a4
    gb[4] = d.sum(axis=0)
    da = d @ P["W"][4]
    for j in range(2, -1, -1):
        a_in, z, g = blocks[j]
        p = g * z
        s = _sig(p)
        dp = da * (s * (1.0 + p * (1.0 - s)))
        dz = dp * g
        dg = dp * z
        gW[j + 1] = dz.T @ a_in
        gb[j + 1] = dz.sum(axis=0)
        gM[j] = dz.T @ cn
        gG[j] = np.stack([(dg * cn[:, 3:4]).sum(axis=0), (dg * cn[:, 4:5]).sum(axis=0)])
        da = da + dz @ P["W"][j + 1]
    s = _sig(z1)
    dz1 = da * (s * (1.0 + z1 * (1.0 - s)))
    gW[0] = dz1.T @ h
    gb[0] = dz1.sum(axis=0)
    return loss, {"W": gW, "b": gb, "M": gM, "G": gG}
