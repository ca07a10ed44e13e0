"""Pins of the learned-preconditioner oracle (CPU): finite-difference
gradients, the zero-network case (Jacobi), positive homogeneity, and the
bfloat16 rounding against torch's own conversion."""
import numpy as np
import pytest

from oracle import mlp_oracle as mo
from oracle import oracle as orc


def _weights(n3, rng, scale=0.3):
    return (rng.normal(0, scale, (128, n3)), rng.normal(0, 0.1, 128),
            rng.normal(0, scale, (n3, 128)), rng.normal(0, 0.1, n3))


def test_gradients_by_finite_differences():
    rng = np.random.default_rng(0)
    n3 = 8
    W1, b1, W2, b2 = _weights(n3, rng)
    U = rng.normal(size=(5, n3))
    T = rng.normal(size=(5, n3))
    loss, gW1, gb1, gW2, gb2 = mo.loss_and_grads(W1, b1, W2, b2, U, T)
    h = 1e-6
    params = [W1, b1, W2, b2]
    grads = [gW1, gb1, gW2, gb2]
    for P, G in zip(params, grads):
        flat = P.reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = mo.loss_and_grads(W1, b1, W2, b2, U, T)[0]
            flat[idx] = old - h
            lm = mo.loss_and_grads(W1, b1, W2, b2, U, T)[0]
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - G.reshape(-1)[idx]) < 1e-6 * max(1.0, abs(fd)), (fd, G.reshape(-1)[idx])


def test_zero_network_is_jacobi_and_homogeneous():
    p = 2
    mesh = orc.Mesh(2, 2, 2)
    n = orc.num_dofs(mesh, p)
    rng = np.random.default_rng(1)
    r = rng.normal(size=(n, 3))
    r[orc.constrained_mask(mesh, p)] = 0
    dinv = rng.uniform(0.5, 2, n)
    z = mo.precond(mesh, p, r, dinv, np.zeros((128, 27)), np.zeros(128), np.zeros((27, 128)), np.zeros(27),
                   bf16=False)
    np.testing.assert_allclose(z, dinv[:, None] * r)
    W1, b1, W2, b2 = _weights(27, rng)
    z1 = mo.precond(mesh, p, r, dinv, W1, b1, W2, b2, bf16=False)
    z2 = mo.precond(mesh, p, 2.0 * r, dinv, W1, b1, W2, b2, bf16=False)
    np.testing.assert_allclose(z2, 2.0 * z1, rtol=1e-12, atol=1e-12)
    w, dofs = mo.partition_weights(mesh, p)
    # the weights of each node sum to one over the cells that share it
    acc = np.zeros(n)
    np.add.at(acc, dofs.reshape(-1), w.reshape(-1))
    np.testing.assert_allclose(acc, 1.0)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(2).normal(size=10000).astype(np.float32) * 10 ** np.random.default_rng(3).uniform(-3, 3, 10000)
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mo.bf16_round(x), ref)


def _snapshot(mesh, p, nv, seed):
    """A consistent snapshot: random x* and x_k (Dirichlet rows 0), r = A (x* - x_k)."""
    rng = np.random.default_rng(seed)
    n = orc.num_dofs(mesh, p)
    con = orc.constrained_mask(mesh, p)
    A = orc.assemble(mesh, p, p + 2, Vq=np.full(mesh.num_cells * (p + 2) ** 3, 0.7))
    xs, xk = rng.normal(size=(n, nv)), rng.normal(size=(n, nv))
    xs[con] = 0.0
    xk[con] = 0.0
    return A, A @ (xs - xk), xk, xs, con


def test_energy_gradients_by_finite_differences():
    p, mesh = 2, orc.Mesh(2, 2, 2)
    A, r, xk, xs, con = _snapshot(mesh, p, 3, 4)
    rng = np.random.default_rng(5)
    dinv = 1.0 / np.where(con, 1.0, A.diagonal())
    W1, b1, W2, b2 = _weights(27, rng)
    loss, *grads = mo.energy_loss_and_grads(mesh, p, A, dinv, W1, b1, W2, b2, r, xk, xs)
    h = 1e-6
    for P, G in zip([W1, b1, W2, b2], grads):
        flat = P.reshape(-1)
        for idx in rng.choice(flat.size, size=min(8, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = mo.energy_loss_and_grads(mesh, p, A, dinv, W1, b1, W2, b2, r, xk, xs)[0]
            flat[idx] = old - h
            lm = mo.energy_loss_and_grads(mesh, p, A, dinv, W1, b1, W2, b2, r, xk, xs)[0]
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - G.reshape(-1)[idx]) < 1e-6 * max(1.0, abs(fd)), (fd, G.reshape(-1)[idx])


def test_energy_loss_special_cases():
    """z = 0 leaves the whole error: with r = A e and columns scaled to unit
    energy norm, every column contributes e'^T A e' = 1.  On a mesh with one
    free node, Jacobi is the exact inverse, so z = e' and the loss is 0.
    Scaling a column of r and e by the same factor changes nothing."""
    p, mesh = 2, orc.Mesh(2, 2, 2)
    A, r, xk, xs, con = _snapshot(mesh, p, 4, 6)
    zero = (np.zeros((128, 27)), np.zeros(128), np.zeros((27, 128)), np.zeros(27))
    loss = mo.energy_loss_and_grads(mesh, p, A, np.zeros(A.shape[0]), *zero, r, xk, xs)[0]
    assert abs(loss - 1.0) < 1e-12
    W = _weights(27, np.random.default_rng(7))
    dinv = 1.0 / np.where(con, 1.0, A.diagonal())
    a = mo.energy_loss_and_grads(mesh, p, A, dinv, *W, r, xk, xs)
    f = np.array([0.5, 3.0, 1.0, 10.0])
    b = mo.energy_loss_and_grads(mesh, p, A, dinv, *W, r * f, xk * f, xs * f)
    assert abs(a[0] - b[0]) < 1e-12 * abs(a[0])
    for ga, gb in zip(a[1:], b[1:]):
        np.testing.assert_allclose(gb, ga, rtol=1e-10, atol=1e-12)
    m1 = orc.Mesh(2, 2, 2)
    A1, r1, xk1, xs1, con1 = _snapshot(m1, 1, 2, 8)
    assert np.count_nonzero(~con1) == 1
    d1 = 1.0 / np.where(con1, 1.0, A1.diagonal())
    z8 = (np.zeros((128, 8)), np.zeros(128), np.zeros((8, 128)), np.zeros(8))
    assert abs(mo.energy_loss_and_grads(m1, 1, A1, d1, *z8, r1, xk1, xs1)[0]) < 1e-14
