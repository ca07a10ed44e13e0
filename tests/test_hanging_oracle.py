"""Pins of the hanging-node oracle (oracle/hanging_oracle.py): the
structured operator when nothing is refined, exact reproduction of
polynomials by the constraints, the Galerkin identity K u = M f for a
polynomial u in the constrained space, symmetry, and the Laplacian's
smallest eigenvalue."""
import numpy as np
import pytest

from oracle import hanging_oracle as ho
from oracle import oracle as orc
from paper_2208_07129_gb300 import inputs


def _xyz(m):
    H = np.array([(m.hi[d] - m.lo[d]) / n for d, n in enumerate((m.nx, m.ny, m.nz))])
    return np.array(m.lo)[None, :] + m.values * (H / 4.0)[None, :]


def test_no_refinement_is_the_structured_operator():
    p, nq = 3, 5
    m = ho.build(3, 2, 2, (0, 0, 0), (0, 0, 0), p)
    mesh = orc.Mesh(3, 2, 2)
    assert len(m.slaves) == 0
    V = inputs.gaussian_potential(orc.quad_points(mesh, p, nq), 3, False)
    A = ho.operator(m, nq, Vq=V).toarray()
    B = orc.assemble(mesh, p, nq, Vq=V).toarray()
    assert np.abs(A - B).max() <= 1e-14 * np.abs(B).max()


@pytest.mark.parametrize("p", [2, 3, 4])
def test_hanging_counts_and_partition_of_unity(p):
    m = ho.build(3, 3, 3, (1, 1, 1), (2, 2, 2), p)
    # the refined cell's surface carries (2p+1)^3 - (2p-1)^3 fine nodes; the ones at coarse
    # node positions (8 corners, plus the face/edge midpoints for even p) are shared
    surf = (2 * p + 1) ** 3 - (2 * p - 1) ** 3
    shared = 3 ** 3 - 1 if p % 2 == 0 else 8
    assert len(m.slaves) == surf - shared
    for s, ms in m.slaves.items():
        assert abs(sum(w for _, w in ms) - 1.0) <= 1e-13


@pytest.mark.parametrize("p,box", [(2, ((1, 1, 0), (3, 2, 2))), (3, ((0, 1, 1), (2, 3, 2))), (4, ((1, 1, 1), (2, 2, 2)))])
def test_constraints_reproduce_polynomials(p, box):
    """A polynomial of degree <= p per direction that vanishes on the
    boundary lies in the constrained space: the slave values computed from
    the free ones equal the polynomial at the slave nodes."""
    m = ho.build(4, 3, 3, box[0], box[1], p)
    x = _xyz(m)
    u = x[:, 0] * (1 - x[:, 0]) * x[:, 1] * (1 - x[:, 1]) * x[:, 2] * (1 - x[:, 2])
    if p >= 3:
        u = u * (0.3 + x[:, 0] - 0.5 * x[:, 2])
    C = ho.constraint_matrix(m)
    free = ho.free_mask(m)
    uf = np.where(free, u, 0.0)
    rec = C @ uf
    s = np.array(sorted(m.slaves))
    np.testing.assert_allclose(rec[s], u[s], rtol=0, atol=1e-13 * np.abs(u).max())


@pytest.mark.parametrize("p", [2, 3])
def test_galerkin_identity_with_hanging_nodes(p):
    """u = x(1-x) y(1-y) z(1-z) (times a linear factor for p >= 3) is in the
    constrained space and f = -1/2 lap u is in Q_p; with quadrature exact for
    these integrands, (C^T K C u)_I = (C^T M C f)_I at every free row."""
    m = ho.build(3, 3, 2, (1, 0, 0), (3, 2, 1), p)
    nq = p + 2
    x = _xyz(m)
    X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
    a, b, c = X * (1 - X), Y * (1 - Y), Z * (1 - Z)
    if p >= 3:
        L = 0.3 + X - 0.5 * Z
        u = a * b * c * L
        # -1/2 lap(a b c L) with L linear: a'' = -2, (aL)'' = -2L + 2 a' L_x, a' = 1 - 2X
        f = -0.5 * ((-2 * L + 2 * (1 - 2 * X) * 1.0) * b * c + a * (-2) * c * L +
                    a * b * (-2 * L + 2 * (1 - 2 * Z) * (-0.5)))
    else:
        u = a * b * c
        f = -0.5 * (-2 * b * c - 2 * a * c - 2 * a * b)
    free = ho.free_mask(m)
    K = ho.operator(m, nq, mu=0.5, Vq=None)
    E = len(m.cells)
    lhs = K @ np.where(free, u, 0.0)
    # f does not vanish on the boundary: the right-hand side tests the full
    # interpolant of f (boundary values included) against the free basis
    C = ho.constraint_matrix(m)
    D = np.diag(free.astype(float))
    Mfull = ho.assemble_full(m, nq, mu=0.0, Vq=np.ones((E, nq ** 3)))
    rhs = D @ (C.T @ (Mfull @ f))
    assert np.abs(lhs - rhs)[free].max() <= 1e-11 * np.abs(rhs).max()


def test_symmetry():
    m = ho.build(3, 2, 3, (1, 0, 1), (2, 2, 3), 3)
    nq = 5
    V = inputs.gaussian_potential(ho.quad_points(m, nq), 4, False)
    A = ho.operator(m, nq, Vq=V)
    assert abs(A - A.T).max() <= 1e-14 * abs(A).max()


def test_laplacian_smallest_eigenvalue():
    import scipy.linalg as sla
    p, nq = 3, 5
    m = ho.build(2, 2, 2, (0, 0, 0), (1, 1, 1), p)
    E = len(m.cells)
    free = ho.free_mask(m)
    K = ho.operator(m, nq, mu=0.5).toarray()[free][:, free]
    M = ho.operator(m, nq, mu=0.0, Vq=np.ones((E, nq ** 3))).toarray()[free][:, free]
    lam = sla.eigh(K, M, eigvals_only=True, subset_by_index=(0, 0))[0]
    assert abs(lam - 1.5 * np.pi ** 2) <= 2e-3 * 1.5 * np.pi ** 2
