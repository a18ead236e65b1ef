"""Oracle of the warm-start network (test infrastructure only: the product
path never imports it).  Plain numpy in float64 of what the device computes:
72 -> 128 -> 128 -> 1 with ReLU, weight matrices rounded to bf16, biases as
given, features rounded to bf16; loss sum(mask (y - t)^2) / n and its
gradient by the chain rule.  Parameter layout: W1[72][128], b1[128],
W2[128][128], b2[128], w3[128], b3.  Pinned against central finite
differences in tests/test_oracle_pins.py."""
import numpy as np

NIN, NH = 72, 128
OFF_W1 = 0
OFF_B1 = OFF_W1 + NIN * NH
OFF_W2 = OFF_B1 + NH
OFF_B2 = OFF_W2 + NH * NH
OFF_W3 = OFF_B2 + NH
OFF_B3 = OFF_W3 + NH
NPARAMS = OFF_B3 + 1


def bf16(x):
    """Round float32 values to bfloat16 (nearest, ties to even), as float64."""
    a = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    lsb = (a >> 16) & 1
    r = ((a + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(p, round_weights=True):
    p = np.asarray(p, np.float32)
    rw = bf16 if round_weights else (lambda v: np.asarray(v, np.float64))
    W1 = rw(p[OFF_W1:OFF_B1]).reshape(NIN, NH)
    b1 = p[OFF_B1:OFF_W2].astype(np.float64)
    W2 = rw(p[OFF_W2:OFF_B2]).reshape(NH, NH)
    b2 = p[OFF_B2:OFF_W3].astype(np.float64)
    w3 = rw(p[OFF_W3:OFF_B3])
    b3 = float(p[OFF_B3])
    return W1, b1, W2, b2, w3, b3


def forward(p, feats, round_inputs=True):
    W1, b1, W2, b2, w3, b3 = unpack(p, round_inputs)
    x = bf16(feats) if round_inputs else np.asarray(feats, np.float64)
    h1 = np.maximum(x @ W1 + b1, 0.0)
    h2 = np.maximum(h1 @ W2 + b2, 0.0)
    return h2 @ w3 + b3, (x, h1, h2)


def loss_grad(p, feats, target, mask=None, round_inputs=True):
    """(loss, gradient) with the layout of the parameter vector."""
    W1, b1, W2, b2, w3, b3 = unpack(p, round_inputs)
    y, (x, h1, h2) = forward(p, feats, round_inputs)
    n = len(y)
    m = np.ones(n) if mask is None else np.asarray(mask, np.float64)
    e = y - np.asarray(target, np.float64)
    loss = float(np.sum(m * e * e) / n)
    d3 = 2.0 * m * e / n
    g = np.zeros(NPARAMS)
    g[OFF_W3:OFF_B3] = h2.T @ d3
    g[OFF_B3] = d3.sum()
    d2 = np.outer(d3, w3) * (h2 > 0)
    g[OFF_W2:OFF_B2] = (h1.T @ d2).ravel()
    g[OFF_B2:OFF_W3] = d2.sum(0)
    d1 = (d2 @ W2.T) * (h1 > 0)
    g[OFF_W1:OFF_B1] = (x.T @ d1).ravel()
    g[OFF_B1:OFF_W2] = d1.sum(0)
    return loss, g
