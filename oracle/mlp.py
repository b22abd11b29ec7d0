"""FP64 reference of the work-estimator network -- TEST INFRASTRUCTURE ONLY.

Same definition the engine documents in include/mce.h: input log2(1 + raw
feature), standardised by (x - mean) / std; 16 -> 64 (ReLU) -> 64 (ReLU) -> 1;
every weight rounded to bfloat16 (round to nearest, ties to even) before use;
biases unrounded. Loss: mean squared error; gradients with respect to the
unrounded weights (the rounding passes gradients straight through). Training
step: Adam (Kingma and Ba, 2015) with bias correction on every trained entry
(all but the standardisation's mean and std).
Everything here is float64 so that it can check the GPU's float32 arithmetic.
"""
import numpy as np

F, H = 16, 64
OW1, OB1 = 0, H * F
OW2 = OB1 + H
OB2 = OW2 + H * H
OW3 = OB2 + H
OB3 = OW3 + H
OMEAN = OB3 + 1
OSTD = OMEAN + F
NPARAMS = OSTD + F


def bf16_round(x):
    """float32 values rounded to bfloat16 (nearest, ties to even), as float64."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    bias = 0x7FFF + ((u >> 16) & 1)
    r = ((u + bias) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def unpack(params, rounded=True):
    p = np.asarray(params, dtype=np.float64)
    # rounded: the float32 master weight as the engine stores it, then bfloat16
    rnd = (lambda z: bf16_round(z.astype(np.float32))) if rounded else (lambda z: z)
    return {
        "W1": rnd(p[OW1:OB1]).reshape(H, F),
        "b1": p[OB1:OW2],
        "W2": rnd(p[OW2:OB2]).reshape(H, H),
        "b2": p[OB2:OW3],
        "W3": rnd(p[OW3:OB3]),
        "b3": p[OB3],
        "mean": p[OMEAN:OSTD],
        "std": p[OSTD:NPARAMS],
    }


def forward(params, feat, rounded=True):
    """Predictions y[B] and the cached activations."""
    q = unpack(params, rounded)
    x = (np.asarray(feat, np.float64) - q["mean"]) / q["std"]
    z1 = x @ q["W1"].T + q["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ q["W2"].T + q["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ q["W3"] + q["b3"]
    return y, (q, x, z1, h1, z2, h2)


def loss_and_grad(params, feat, label, rounded=True):
    """(mean squared error, gradient vector in the parameter layout)."""
    y, (q, x, z1, h1, z2, h2) = forward(params, feat, rounded)
    t = np.asarray(label, np.float64)
    B = len(t)
    loss = float(np.mean((y - t) ** 2))
    dy = 2.0 * (y - t) / B
    g = np.zeros(NPARAMS)
    g[OW3:OB3] = dy @ h2
    g[OB3] = dy.sum()
    d2 = np.outer(dy, q["W3"]) * (z2 > 0)
    g[OW2:OB2] = (d2.T @ h1).ravel()
    g[OB2:OW3] = d2.sum(0)
    d1 = (d2 @ q["W2"]) * (z1 > 0)
    g[OW1:OB1] = (d1.T @ x).ravel()
    g[OB1:OW2] = d1.sum(0)
    return loss, g


ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-8


def adam_step(params, grad, m, v, t, lr):
    """One Adam step (t = 1, 2, ...) in float64: the moment estimates
    m <- b1 m + (1 - b1) g and v <- b2 v + (1 - b2) g^2, their bias-corrected
    forms m / (1 - b1^t) and v / (1 - b2^t), and the update
    theta <- theta - lr * m_hat / (sqrt(v_hat) + eps) on the trained entries.
    Returns new (params, m, v); the inputs are not modified."""
    p = np.array(params, dtype=np.float64)
    g = np.asarray(grad, dtype=np.float64)[:OMEAN]
    m = ADAM_B1 * np.asarray(m, np.float64) + (1.0 - ADAM_B1) * g
    v = ADAM_B2 * np.asarray(v, np.float64) + (1.0 - ADAM_B2) * g * g
    m_hat = m / (1.0 - ADAM_B1 ** t)
    v_hat = v / (1.0 - ADAM_B2 ** t)
    p[:OMEAN] -= lr * m_hat / (np.sqrt(v_hat) + ADAM_EPS)
    return p, m, v
