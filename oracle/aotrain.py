"""Oracle of one training step of the learned AO surrogate (TEST
INFRASTRUCTURE ONLY: used by the tests, never by the library).

Not part of the paper: the surrogate stands in for the traced density AO of
Sec. 5.3. Float64 numpy, written from the model definition (reading L1 in
aomlp.c) and the chain rule:

Training forward pass (the model with bfloat16 operands; the per-voxel part
of layer 1 is not rounded separately here, unlike inference):
    Z1 = q(X) q(W1)^T + b1,  H1 = q(ReLU(Z1))
    Z2 = H1 q(W2)^T + b2,    H2 = q(ReLU(Z2))
    Z3 = H2 q(W3)^T + b3,    H3 = q(ReLU(Z3))
    y  = sigmoid(H3 . q(W4) + b4),  loss = mean_r (y_r - t_r)^2
with q = round to bfloat16 (through float32, nearest even).

Backward pass: the rounding q is passed through unchanged (straight-through),
the ReLU derivative is [Z > 0], and the gradients of the hidden layers enter
the products as bfloat16 (q(dZ)), as the weights and activations do:
    dz4 = 2 (y - t) / R * y (1 - y);  db4 = sum dz4;  dW4 = H3^T dz4
    dZ3 = (dz4 q(W4)^T) [Z3 > 0];     db3 = colsum dZ3;  dW3 = q(dZ3)^T H2
    dZ2 = (q(dZ3) q(W3)) [Z2 > 0];    db2 = colsum dZ2;  dW2 = q(dZ2)^T H1
    dZ1 = (q(dZ2) q(W2)) [Z1 > 0];    db1 = colsum dZ1;  dW1 = q(dZ1)^T q(X)
With rnd=False every q is the identity and the gradient is the exact
derivative of the float64 loss.

Adam (Kingma and Ba, Algorithm 1): m <- b1 m + (1 - b1) g,
v <- b2 v + (1 - b2) g^2, p <- p - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
"""
from __future__ import annotations

import numpy as np

NIN, NH = 400, 64
NHIT, VOFF = 15, 16          # per-hit inputs 0..14; per-voxel inputs from 16
OW1 = 0
OB1 = OW1 + NH * NIN
OW2 = OB1 + NH
OB2 = OW2 + NH * NH
OW3 = OB2 + NH
OB3 = OW3 + NH * NH
OW4 = OB3 + NH
OB4 = OW4 + NH
NPARAM = OB4 + 1


def bf16(a):
    """float64 -> float32 (nearest) -> bfloat16 (nearest even), as float64."""
    f = np.asarray(a, np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    finite = (u & 0x7F800000) != 0x7F800000
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    u = np.where(finite, r, u).astype(np.uint32)
    return u.view(np.float32).astype(np.float64)


def unpack(p):
    p = np.asarray(p, np.float64)
    return (p[OW1:OB1].reshape(NH, NIN), p[OB1:OW2], p[OW2:OB2].reshape(NH, NH), p[OB2:OW3],
            p[OW3:OB3].reshape(NH, NH), p[OB3:OW4], p[OW4:OB4], p[OB4])


def forward(p, X, rnd=True):
    q = bf16 if rnd else (lambda a: np.asarray(a, np.float64))
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(p)
    Xq = q(X)
    Z1 = Xq @ q(W1).T + b1
    H1 = q(np.maximum(Z1, 0.0))
    Z2 = H1 @ q(W2).T + b2
    H2 = q(np.maximum(Z2, 0.0))
    Z3 = H2 @ q(W3).T + b3
    H3 = q(np.maximum(Z3, 0.0))
    y = 1.0 / (1.0 + np.exp(-(H3 @ q(W4) + b4)))
    return dict(Xq=Xq, Z1=Z1, H1=H1, Z2=Z2, H2=H2, Z3=Z3, H3=H3, y=y)


def loss(p, X, t, rnd=True) -> float:
    y = forward(p, X, rnd)["y"]
    return float(np.mean((y - np.asarray(t, np.float64)) ** 2))


def loss_and_grad(p, X, t, rnd=True):
    """(loss, gradient float64 [NPARAM]) of the batch (X [R][NIN], t [R])."""
    q = bf16 if rnd else (lambda a: np.asarray(a, np.float64))
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(p)
    f = forward(p, X, rnd)
    t = np.asarray(t, np.float64)
    R = len(t)
    y = f["y"]
    g = np.zeros(NPARAM)
    dz4 = 2.0 * (y - t) / R * y * (1.0 - y)
    g[OB4] = dz4.sum()
    g[OW4:OB4] = f["H3"].T @ dz4
    dZ3 = np.outer(dz4, q(W4)) * (f["Z3"] > 0)
    g[OB3:OW4] = dZ3.sum(0)
    g[OW3:OB3] = (q(dZ3).T @ f["H2"]).reshape(-1)
    dZ2 = (q(dZ3) @ q(W3)) * (f["Z2"] > 0)
    g[OB2:OW3] = dZ2.sum(0)
    g[OW2:OB2] = (q(dZ2).T @ f["H1"]).reshape(-1)
    dZ1 = (q(dZ2) @ q(W2)) * (f["Z1"] > 0)
    g[OB1:OW2] = dZ1.sum(0)
    g[OW1:OB1] = (q(dZ1).T @ f["Xq"]).reshape(-1)
    return float(np.mean((y - t) ** 2)), g


def adam(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step = 1, 2, ...); returns new (p, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
