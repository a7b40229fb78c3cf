"""FP64 reference of the learned reorder proposal's network (oracle; test
infrastructure only).  Not from the paper: the paper's reordering is the
greedy Eq. 18 cost; the network is this project's proposal, kept only
where it is no worse than the greedy order.

Network: F = 12 features -> 64 -> 64 -> 1 with ReLU; parameters flattened as
W1[64][12], b1[64], W2[64][64], b2[64], w3[64], b3.  With bf16=True the
matrix-product inputs are rounded to bfloat16 (round to nearest even on the
float32 value) exactly where the GPU kernels round them: features, weights
W1, W2, w3, and the activations h1, h2 after ReLU; biases stay unrounded.
Rounding is treated as the identity in the backward pass (its derivative is
zero almost everywhere, the kernels and this reference both pass the
gradient straight through).

Loss: for each step s with rows R_s and target row t_s,
    L_s = -log softmax(-score)[t_s] = score[t_s] + logsumexp(-score[R_s]),
averaged over steps.
"""
from __future__ import annotations

import numpy as np

NF, NH = 12, 64
P_W1 = 0
P_B1 = P_W1 + NH * NF
P_W2 = P_B1 + NH
P_B2 = P_W2 + NH * NH
P_W3 = P_B2 + NH
P_B3 = P_W3 + NH
NPARAM = P_B3 + 1


def bf16(x):
    """Round to bfloat16 (nearest even) via the float32 bit pattern."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(params):
    p = np.asarray(params, dtype=np.float64)
    W1 = p[P_W1:P_B1].reshape(NH, NF)
    b1 = p[P_B1:P_W2]
    W2 = p[P_W2:P_B2].reshape(NH, NH)
    b2 = p[P_B2:P_W3]
    w3 = p[P_W3:P_B3]
    b3 = p[P_B3]
    return W1, b1, W2, b2, w3, b3


def forward(params, X, bf: bool = True):
    W1, b1, W2, b2, w3, b3 = unpack(params)
    r = bf16 if bf else (lambda a: np.asarray(a, dtype=np.float64))
    x = r(X)
    W1r, W2r, w3r = r(W1), r(W2), r(w3)
    a1 = x @ W1r.T + b1
    h1 = r(np.maximum(a1, 0.0))
    a2 = h1 @ W2r.T + b2
    h2 = r(np.maximum(a2, 0.0))
    score = h2 @ w3r + b3
    return score, (x, W1r, W2r, w3r, a1, h1, a2, h2)


def loss_and_grad(params, X, step_first, target_row, bf: bool = True):
    """Mean softmax cross-entropy over steps and its gradient (FP64)."""
    score, (x, W1r, W2r, w3r, a1, h1, a2, h2) = forward(params, X, bf)
    nsteps = len(target_row)
    ds = np.zeros_like(score)
    loss = 0.0
    for s in range(nsteps):
        a, b, t = int(step_first[s]), int(step_first[s + 1]), int(target_row[s])
        z = -score[a:b]
        m = z.max()
        e = np.exp(z - m)
        p = e / e.sum()
        loss += score[t] + m + np.log(e.sum())
        ds[a:b] = -p
        ds[t] += 1.0
    loss /= nsteps
    ds /= nsteps
    g = np.zeros(NPARAM, dtype=np.float64)
    g[P_W3:P_B3] = h2.T @ ds
    g[P_B3] = ds.sum()
    d2 = np.outer(ds, w3r) * (a2 > 0)
    g[P_W2:P_B2] = (d2.T @ h1).reshape(-1)
    g[P_B2:P_W3] = d2.sum(axis=0)
    d1 = (d2 @ W2r) * (a1 > 0)
    g[P_W1:P_B1] = (d1.T @ x).reshape(-1)
    g[P_B1:P_W2] = d1.sum(axis=0)
    return loss, g
