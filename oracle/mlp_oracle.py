"""FP64 numpy oracle of the learned cell-patch preconditioner.

TEST INFRASTRUCTURE ONLY (tests, smoke, the benchmark's baseline legs).  It
shares no code with the CUDA library.  Definitions (the paper has no learned
component; these are the layer's own definitions):

    MLP(u)  = W2 relu(W1 u + b1) + b2          W1: 128 x n3, W2: n3 x 128
    loss    = mean over all entries of (MLP(U) - T)^2
    z       = D^-1 r + sum_e R_e^T ( w_e * s_e * MLP(R_e r / s_e) ),
              s_e = ||R_e r||, w_e = 1 / (cells sharing the node),
              Dirichlet nodes read and written as 0.

``precond(..., bf16=True)`` rounds the patch inputs, the weights and the
hidden activations to bfloat16 (round to nearest, ties to even) exactly where
the tensor-core kernel does, and does everything else in FP64.
"""
from __future__ import annotations

import numpy as np

from . import oracle as orc


def bf16_round(x: np.ndarray) -> np.ndarray:
    """float -> nearest bfloat16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(W1, b1, W2, b2, U):
    Hpre = U @ W1.T + b1
    H = np.maximum(Hpre, 0.0)
    return Hpre, H, H @ W2.T + b2


def loss_and_grads(W1, b1, W2, b2, U, T):
    """Mean squared error and its gradients, written out by the chain rule."""
    Hpre, H, Y = forward(W1, b1, W2, b2, U)
    R = Y - T
    N = R.size
    loss = np.sum(R * R) / N
    dY = 2.0 * R / N
    gW2 = dY.T @ H
    gb2 = dY.sum(axis=0)
    dH = dY @ W2
    dHpre = dH * (Hpre > 0)
    gW1 = dHpre.T @ U
    gb1 = dHpre.sum(axis=0)
    return loss, gW1, gb1, gW2, gb2


def partition_weights(mesh: orc.Mesh, p: int) -> np.ndarray:
    """w[e, i] = 1 / (number of cells sharing local node i of cell e)."""
    n = orc.num_dofs(mesh, p)
    count = np.zeros(n)
    dofs = np.stack([orc.cell_dofs(mesh, p, e) for e in range(mesh.num_cells)])
    np.add.at(count, dofs.reshape(-1), 1.0)
    return 1.0 / count[dofs], dofs


def precond(mesh: orc.Mesh, p: int, r: np.ndarray, dinv: np.ndarray, W1, b1, W2, b2, bf16: bool = True):
    r = np.asarray(r, dtype=np.float64)
    con = orc.constrained_mask(mesh, p)
    w, dofs = partition_weights(mesh, p)
    z = dinv[:, None] * r
    if bf16:
        W1, W2 = bf16_round(W1), bf16_round(W2)
    rr = r.copy()
    rr[con] = 0.0
    for e in range(mesh.num_cells):
        patch = rr[dofs[e]].T                       # columns x n3
        s = np.sqrt(np.sum(np.float32(patch) ** 2, axis=1))
        inv = np.where(s > 0, 1.0 / np.where(s > 0, s, 1.0), 0.0)
        u = bf16_round(patch) if bf16 else patch
        h = np.maximum((u @ W1.T) * inv[:, None] + b1, 0.0)
        if bf16:
            h = bf16_round(h)
        y = (h @ W2.T + b2) * s[:, None] * w[e][None, :]
        y[:, con[dofs[e]]] = 0.0
        np.add.at(z, dofs[e], y.T)
    return z
