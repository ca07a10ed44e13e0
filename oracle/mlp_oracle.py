"""FP64 numpy oracle of the learned cell-patch preconditioner.

TEST INFRASTRUCTURE ONLY (tests, smoke, the benchmark's baseline legs).  It
shares no code with the CUDA library.  Definitions (the paper has no learned
component; these are the layer's own definitions):

    MLP(u)  = W2 relu(W1 u + b1) + b2          W1: 128 x n3, W2: n3 x 128
    loss    = mean over all entries of (MLP(U) - T)^2
    z       = D^-1 r + sum_e R_e^T ( w_e * s_e * MLP(R_e r / s_e) ),
              s_e = ||R_e r||, w_e = 1 / (cells sharing the node),
              Dirichlet nodes read and written as 0.
    energy objective on one snapshot (r_k, x_k) of a solve with solution x*:
              c_j = 1 / sqrt((x* - x_k)_j . r_j)   (1 / ||r_j|| if that is <= 0)
              r' = c r,  e' = c (x* - x_k),  z = z(r'),
              loss = (1 / n_col) sum_j (z - e')_j^T A (z - e')_j.

``precond(..., bf16=True)`` rounds the patch inputs, the weights and the
hidden activations to bfloat16 (round to nearest, ties to even) exactly where
the tensor-core kernel does, and does everything else in FP64 (the patch
norms s_e included).
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
        s = np.sqrt(np.sum(patch ** 2, axis=1))
        inv = np.where(s > 0, 1.0 / np.where(s > 0, s, 1.0), 0.0)
        u = bf16_round(patch) if bf16 else patch
        h = np.maximum((u @ W1.T) * inv[:, None] + b1, 0.0)
        if bf16:
            h = bf16_round(h)
        y = (h @ W2.T + b2) * s[:, None] * w[e][None, :]
        y[:, con[dofs[e]]] = 0.0
        np.add.at(z, dofs[e], y.T)
    return z


def _patches(mesh: orc.Mesh, p: int, r: np.ndarray):
    """Rows (cell-major, column-minor) of unit patches R_e r / s_e, their norms
    s_e, and the cells' DoFs, partition weights and constrained flags."""
    con = orc.constrained_mask(mesh, p)
    w, dofs = partition_weights(mesh, p)
    rr = np.array(r, dtype=np.float64)
    rr[con] = 0.0
    nv = rr.shape[1]
    U, S = [], []
    for e in range(mesh.num_cells):
        patch = rr[dofs[e]].T                      # columns x n3
        s = np.sqrt(np.sum(patch ** 2, axis=1))
        U.append(patch / np.where(s > 0, s, 1.0)[:, None])
        S.append(s)
    return np.concatenate(U), np.concatenate(S), dofs, w, con, nv


def energy_loss_and_grads(mesh: orc.Mesh, p: int, A, dinv: np.ndarray, W1, b1, W2, b2, r, xk, xstar):
    """The energy objective on one snapshot and its gradients, in FP64.

    A: the operator as a scipy sparse matrix (P A P on a Dirichlet box), dinv:
    the Jacobi weights 1 / diag(A).  Steps in the order of the definition:
    column scaling, the preconditioner z(r') (network applied to every
    cell's unit patch, outputs scaled by s_e and the partition weights and
    summed into the nodes), the residual of the error g = z - e', the loss
    g^T A g / n_col; then the chain rule back to the weights: dL/dz = 2 A g /
    n_col, per patch entry dL/dy = s_e w_i (dL/dz)_dof (0 at Dirichlet
    nodes), and the two layers.  Returns loss, gW1, gb1, gW2, gb2."""
    r = np.asarray(r, dtype=np.float64)
    err = np.asarray(xstar, dtype=np.float64) - np.asarray(xk, dtype=np.float64)
    er = np.sum(err * r, axis=0)
    rn = np.sqrt(np.sum(r * r, axis=0))
    c = np.where(er > 0, 1.0 / np.sqrt(np.where(er > 0, er, 1.0)), np.where(rn > 0, 1.0 / np.where(rn > 0, rn, 1.0), 0.0))
    r1 = r * c[None, :]
    e1 = err * c[None, :]
    U, S, dofs, w, con, nv = _patches(mesh, p, r1)
    Hpre, H, Y = forward(W1, b1, W2, b2, U)
    z = dinv[:, None] * r1
    n3 = dofs.shape[1]
    for e in range(mesh.num_cells):
        y = Y[e * nv:(e + 1) * nv] * S[e * nv:(e + 1) * nv, None] * w[e][None, :]
        y[:, con[dofs[e]]] = 0.0
        np.add.at(z, dofs[e], y.T)
    g = z - e1
    q = A @ g
    loss = float(np.sum(g * q)) / nv
    dz = 2.0 * q / nv
    dY = np.zeros_like(Y)
    for e in range(mesh.num_cells):
        d = dz[dofs[e]].T * S[e * nv:(e + 1) * nv, None] * w[e][None, :]
        d[:, con[dofs[e]]] = 0.0
        dY[e * nv:(e + 1) * nv] = d
    gW2 = dY.T @ H
    gb2 = dY.sum(axis=0)
    dHpre = (dY @ W2) * (Hpre > 0)
    gW1 = dHpre.T @ U
    gb1 = dHpre.sum(axis=0)
    assert gW1.shape == (W1.shape[0], n3)
    return loss, gW1, gb1, gW2, gb2
