"""Pins of the FP64 oracle to facts that do not come from the oracle itself.

Each test checks the oracle against a closed form, an invariant, a textbook
value, an independent brute-force construction (numpy's Gauss rule and a
monomial basis) or a number printed in the paper, chosen so that a dropped
term, a wrong sign or index or a transposed operand in the oracle fails one
of them.  CPU only.
"""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import oracle as orc
from paper_2208_07129_gb300 import inputs


# --------------------------------------------------------------------------
# P1  quadrature (Sec. 2.2: tensor n_q-point rule; GLL nodes of the basis)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", range(1, 13))
def test_gauss_exactness(n):
    x, w = orc.gauss(n)
    for k in range(0, 2 * n):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.sum(w * x ** k) - exact) < 1e-14 * max(1.0, 4 ** 0)
    # degree 2n is NOT integrated exactly (the rule is not of higher order)
    assert abs(np.sum(w * x ** (2 * n)) - 2.0 / (2 * n + 1)) > 1e-8


@pytest.mark.parametrize("n", range(2, 13))
def test_gll_exactness(n):
    x, w = orc.gll(n)
    assert x[0] == -1.0 and x[-1] == 1.0
    for k in range(0, 2 * n - 2):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.sum(w * x ** k) - exact) < 1e-14


def test_textbook_rules():
    x, w = orc.gauss(2)
    np.testing.assert_allclose(x, [-1 / math.sqrt(3), 1 / math.sqrt(3)], rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, [1, 1], atol=1e-15)
    x, w = orc.gauss(3)
    np.testing.assert_allclose(x, [-math.sqrt(0.6), 0, math.sqrt(0.6)], atol=1e-15)
    np.testing.assert_allclose(w, [5 / 9, 8 / 9, 5 / 9], atol=1e-15)
    x, w = orc.gll(3)
    np.testing.assert_allclose(x, [-1, 0, 1], atol=1e-15)
    np.testing.assert_allclose(w, [1 / 3, 4 / 3, 1 / 3], atol=1e-15)
    x, w = orc.gll(4)
    np.testing.assert_allclose(x, [-1, -1 / math.sqrt(5), 1 / math.sqrt(5), 1], atol=1e-15)
    np.testing.assert_allclose(w, [1 / 6, 5 / 6, 5 / 6, 1 / 6], atol=1e-15)
    x, w = orc.gll(5)
    np.testing.assert_allclose(x, [-1, -math.sqrt(3 / 7), 0, math.sqrt(3 / 7), 1], atol=1e-15)
    np.testing.assert_allclose(w, [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10], atol=1e-15)


def test_against_numpy_leggauss():
    for n in range(1, 16):
        x, w = orc.gauss(n)
        xr, wr = np.polynomial.legendre.leggauss(n)
        np.testing.assert_allclose(x, xr, atol=2e-15)
        np.testing.assert_allclose(w, wr, atol=2e-15)


# --------------------------------------------------------------------------
# P2  1D Lagrange basis on GLL nodes (Sec. 2.2, tensor-product basis)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("p", range(1, 10))
def test_lagrange_basis(p):
    nodes, _ = orc.gll(p + 1)
    for j, xj in enumerate(nodes):
        phi, _ = orc.lagrange(nodes, xj)
        np.testing.assert_allclose(phi, np.eye(p + 1)[j], atol=1e-15)
    rng = np.random.default_rng(p)
    for t in list(rng.uniform(-1, 1, 7)) + list(nodes):
        phi, dphi = orc.lagrange(nodes, t)
        assert abs(phi.sum() - 1) < 1e-13
        assert abs(dphi.sum()) < 1e-11
        for k in range(p + 1):   # reproduces monomials of degree <= p and their derivatives
            assert abs(np.dot(phi, nodes ** k) - t ** k) < 1e-13
            dk = k * t ** (k - 1) if k > 0 else 0.0
            assert abs(np.dot(dphi, nodes ** k) - dk) < 1e-11


# --------------------------------------------------------------------------
# helpers: node coordinates of a uniform box mesh, written out independently
# --------------------------------------------------------------------------

def node_coords_uniform(mesh, p):
    """Physical coordinates of every global node of a uniform box mesh."""
    lx = np.polynomial.legendre.Legendre.basis(p).deriv().roots() if p > 1 else np.array([])
    gll = np.concatenate([[-1.0], np.sort(lx.real), [1.0]])
    n = orc.num_dofs(mesh, p)
    xyz = np.zeros((n, 3))
    h = [(mesh.hi[d] - mesh.lo[d]) / [mesh.nx, mesh.ny, mesh.nz][d] for d in range(3)]
    for e in range(mesh.num_cells):
        cx, cy, cz = e % mesh.nx, (e // mesh.nx) % mesh.ny, e // (mesh.nx * mesh.ny)
        dofs = orc.cell_dofs(mesh, p, e)
        for i3 in range(p + 1):
            for i2 in range(p + 1):
                for i1 in range(p + 1):
                    I = i1 + (p + 1) * (i2 + (p + 1) * i3)
                    xyz[dofs[I]] = [mesh.lo[0] + h[0] * (cx + (1 + gll[i1]) / 2),
                                    mesh.lo[1] + h[1] * (cy + (1 + gll[i2]) / 2),
                                    mesh.lo[2] + h[2] * (cz + (1 + gll[i3]) / 2)]
    return xyz


# --------------------------------------------------------------------------
# P3  polynomial reproduction: (K u)_I = (M f)_I, f = -mu lap u, u in Q_p
# --------------------------------------------------------------------------

@pytest.mark.parametrize("p,nq", [(2, 3), (3, 5), (4, 6)])
def test_polynomial_reproduction(p, nq):
    mesh = orc.Mesh(2, 3, 2, periodic=False, lo=(0.0, -0.5, 0.25), hi=(1.0, 1.5, 0.75))
    mu = 0.5
    K = orc.assemble(mesh, p, nq, mu=mu, Vq=None, constrain=False)
    E = mesh.num_cells
    ones = np.ones((E, nq ** 3))
    M = orc.assemble(mesh, p, nq, mu=0.0, Vq=ones, constrain=False)
    xyz = node_coords_uniform(mesh, p)
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    # u = x^p y^(p-1) z + 3 x y^p - z^p  (degree <= p per direction)
    u = x ** p * y ** (p - 1) * z + 3 * x * y ** p - z ** p
    lap = (p * (p - 1) * x ** (p - 2) * y ** (p - 1) * z
           + (p - 1) * (p - 2) * x ** p * y ** max(p - 3, 0) * z * (1 if p >= 3 else 0)
           + 3 * p * (p - 1) * x * y ** (p - 2)
           - p * (p - 1) * z ** (p - 2))
    f = -mu * lap
    interior = ~orc.constrained_mask(mesh, p)
    Ku = K @ u
    Mf = M @ f
    scale = np.abs(Ku).max()
    assert np.abs(Ku - Mf)[interior].max() < 1e-11 * scale
    # a dropped/shifted term would break it on boundary rows only if the test were weak:
    # check boundary rows really differ (the identity needs phi_I to vanish on the boundary)
    assert np.abs(Ku - Mf)[~interior].max() > 1e-6 * scale


# --------------------------------------------------------------------------
# P4  patch test on a distorted (trilinear) mesh: K (a.x + c) = 0 at interior rows
# --------------------------------------------------------------------------

@pytest.mark.parametrize("p,nq", [(2, 4), (3, 5)])
def test_patch_test_distorted(p, nq):
    nx, ny, nz = 3, 3, 2
    verts = inputs.perturbed_vertices(nx, ny, nz, seed=7, amp=0.25)
    mesh = orc.Mesh(nx, ny, nz, periodic=False, vertices=verts)
    K = orc.assemble(mesh, p, nq, mu=0.5, constrain=False)
    # nodal coordinates: interpolate the trilinear map at GLL nodes through the
    # quadrature-point routine of a GLL rule with n_p points (nodes == points)
    pts = orc.quad_points(mesh, p, p + 1, kind=orc.GLL)
    n = orc.num_dofs(mesh, p)
    xyz = np.zeros((n, 3))
    for e in range(mesh.num_cells):
        xyz[orc.cell_dofs(mesh, p, e)] = pts[e]
    u = 0.7 * xyz[:, 0] - 1.3 * xyz[:, 1] + 0.4 * xyz[:, 2] + 2.0
    r = K @ u
    interior = ~orc.constrained_mask(mesh, p)
    assert np.abs(r[interior]).max() < 1e-12
    assert np.abs(r[~interior]).max() > 1e-4


# --------------------------------------------------------------------------
# P5  null space (periodic), P6 volume, P7 symmetry, P10 constant potential
# --------------------------------------------------------------------------

def test_periodic_null_space_and_volume():
    p, nq = 3, 5
    mesh = orc.Mesh(3, 2, 4, periodic=True)
    K = orc.assemble(mesh, p, nq, mu=0.5, constrain=False)
    assert K.shape[0] == (3 * p) * (2 * p) * (4 * p)
    assert np.abs(K @ np.ones(K.shape[0])).max() < 1e-13
    ones = np.ones((mesh.num_cells, nq ** 3))
    M = orc.assemble(mesh, p, nq, mu=0.0, Vq=ones, constrain=False)
    assert abs(np.ones(K.shape[0]) @ (M @ np.ones(K.shape[0])) - 1.0) < 1e-13


def test_volume_distorted_and_box():
    p, nq = 2, 4
    verts = inputs.perturbed_vertices(3, 2, 2, seed=3)
    mesh = orc.Mesh(3, 2, 2, vertices=verts)
    E = mesh.num_cells
    M = orc.assemble(mesh, p, nq, mu=0.0, Vq=np.ones((E, nq ** 3)), constrain=False)
    one = np.ones(M.shape[0])
    assert abs(one @ (M @ one) - 1.0) < 1e-13
    mesh = orc.Mesh(2, 2, 3, lo=(0, 0, 0), hi=(2.0, 0.5, 3.0))
    c = 2 * math.pi
    M = orc.assemble(mesh, p, nq, mu=0.0, Vq=c * np.ones((mesh.num_cells, nq ** 3)), constrain=False)
    one = np.ones(M.shape[0])
    assert abs(one @ (M @ one) - c * 3.0) < 1e-12


def test_symmetry_and_constant_potential():
    p, nq = 3, 5
    verts = inputs.perturbed_vertices(2, 3, 2, seed=11)
    mesh = orc.Mesh(2, 3, 2, vertices=verts)
    E = mesh.num_cells
    rng = np.random.default_rng(0)
    V = rng.uniform(-1, 1, (E, nq ** 3))
    A = orc.assemble(mesh, p, nq, mu=0.5, Vq=V, constrain=True)
    assert abs(A - A.T).max() < 1e-14 * abs(A).max()
    x, y = rng.standard_normal((2, A.shape[0]))
    assert abs(x @ (A @ y) - y @ (A @ x)) < 1e-12 * np.abs(A @ y).sum()
    # linearity in V: A(mu=1, V=2 pi) = K(mu=1) + 2 pi M   (the paper's Helmholtz setting, Sec. 4)
    K = orc.assemble(mesh, p, nq, mu=1.0, constrain=False)
    M = orc.assemble(mesh, p, nq, mu=0.0, Vq=np.ones((E, nq ** 3)), constrain=False)
    H = orc.assemble(mesh, p, nq, mu=1.0, Vq=2 * math.pi * np.ones((E, nq ** 3)), constrain=False)
    assert abs(H - (K + 2 * math.pi * M)).max() < 1e-13 * abs(H).max()


def test_dirichlet_constraint_is_PAP():
    p, nq = 2, 4
    mesh = orc.Mesh(2, 2, 3)
    E = mesh.num_cells
    V = np.random.default_rng(1).uniform(0, 1, (E, nq ** 3))
    A = orc.assemble(mesh, p, nq, mu=0.5, Vq=V, constrain=False).toarray()
    Ac = orc.assemble(mesh, p, nq, mu=0.5, Vq=V, constrain=True).toarray()
    P = np.diag((~orc.constrained_mask(mesh, p)).astype(float))
    np.testing.assert_allclose(Ac, P @ A @ P, atol=1e-15)
    # exactly 2 (p) layers: boundary nodes are those on the box faces
    assert (~orc.constrained_mask(mesh, p)).sum() == (2 * p - 1) * (2 * p - 1) * (3 * p - 1)


# --------------------------------------------------------------------------
# P8  eigenvalues of -1/2 lap on the unit cube: lambda_min = 3 pi^2 / 2, error ~ h^(2p)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("p", [2, 3])
def test_eigenvalue_convergence(p):
    nq = p + 2
    exact = 1.5 * math.pi ** 2
    errs = []
    for n in (2, 4):
        mesh = orc.Mesh(n, n, n)
        K = orc.assemble(mesh, p, nq, mu=0.5, constrain=True).toarray()
        M = orc.assemble(mesh, p, nq, mu=0.0, Vq=np.ones((mesh.num_cells, nq ** 3)), constrain=True).toarray()
        keep = ~orc.constrained_mask(mesh, p)
        lam = scipy.linalg.eigh(K[np.ix_(keep, keep)], M[np.ix_(keep, keep)], eigvals_only=True)
        assert lam[0] > exact  # conforming Galerkin: upper bound
        errs.append(lam[0] - exact)
    rate = math.log2(errs[0] / errs[1])
    assert 2 * p - 0.6 < rate < 2 * p + 1.0, (errs, rate)


def test_periodic_spectrum():
    # periodic unit box, mu = 1/2: eigenvalues 2 pi^2 |k|^2, zero simple
    p, nq = 3, 5
    mesh = orc.Mesh(3, 3, 3, periodic=True)
    K = orc.assemble(mesh, p, nq, mu=0.5, constrain=False).toarray()
    M = orc.assemble(mesh, p, nq, mu=0.0, Vq=np.ones((27, nq ** 3)), constrain=False).toarray()
    lam = scipy.linalg.eigh(K, M, eigvals_only=True)
    assert abs(lam[0]) < 1e-9
    assert lam[1] > 1.0
    np.testing.assert_allclose(lam[1:7], 2 * math.pi ** 2, rtol=2e-3)


# --------------------------------------------------------------------------
# P9  brute force on 1-2 cells: monomial basis, numpy's Gauss rule, own geometry
# --------------------------------------------------------------------------

def _brute_cell_matrix(corners, p, nq, mu, Vq):
    """A^(e) in the Lagrange/GLL basis through a monomial basis: A_L = C^T A_mono C."""
    xq, wq = np.polynomial.legendre.leggauss(nq)
    r = np.polynomial.legendre.Legendre.basis(p).deriv().roots() if p > 1 else np.array([])
    gll = np.concatenate([[-1.0], np.sort(np.real(r)), [1.0]])
    Vd = np.vander(gll, p + 1, increasing=True)       # Vd[i, a] = x_i^a
    C1 = np.linalg.inv(Vd)                            # phi_i = sum_a C1[a, i] x^a
    C = np.kron(np.kron(C1, C1), C1)                  # ordering: (a3, a2, a1) x (i3, i2, i1)
    n = p + 1
    nm = n ** 3
    Am = np.zeros((nm, nm))
    for q3 in range(nq):
        for q2 in range(nq):
            for q1 in range(nq):
                xi = np.array([xq[q1], xq[q2], xq[q3]])
                # trilinear geometry
                J = np.zeros((3, 3))
                for c in range(2):
                    for b in range(2):
                        for a in range(2):
                            P = corners[a + 2 * b + 4 * c]
                            la = [(1 - xi[0]) / 2, (1 + xi[0]) / 2][a]
                            lb = [(1 - xi[1]) / 2, (1 + xi[1]) / 2][b]
                            lc = [(1 - xi[2]) / 2, (1 + xi[2]) / 2][c]
                            da, db, dc = [-0.5, 0.5][a], [-0.5, 0.5][b], [-0.5, 0.5][c]
                            J[:, 0] += P * da * lb * lc
                            J[:, 1] += P * la * db * lc
                            J[:, 2] += P * la * lb * dc
                detJ = np.linalg.det(J)
                Jit = np.linalg.inv(J).T
                m1 = [xi[0] ** a for a in range(n)]
                m2 = [xi[1] ** a for a in range(n)]
                m3 = [xi[2] ** a for a in range(n)]
                d1 = [a * xi[0] ** (a - 1) if a else 0.0 for a in range(n)]
                d2 = [a * xi[1] ** (a - 1) if a else 0.0 for a in range(n)]
                d3 = [a * xi[2] ** (a - 1) if a else 0.0 for a in range(n)]
                val = np.zeros(nm)
                grad = np.zeros((nm, 3))
                for a3 in range(n):
                    for a2 in range(n):
                        for a1 in range(n):
                            k = a1 + n * (a2 + n * a3)
                            val[k] = m1[a1] * m2[a2] * m3[a3]
                            grad[k] = [d1[a1] * m2[a2] * m3[a3], m1[a1] * d2[a2] * m3[a3], m1[a1] * m2[a2] * d3[a3]]
                gph = grad @ Jit.T
                Q = q1 + nq * (q2 + nq * q3)
                w = wq[q1] * wq[q2] * wq[q3] * detJ
                Am += w * (mu * gph @ gph.T + Vq[Q] * np.outer(val, val))
    # index k = a1 + n a2 + n^2 a3 corresponds to kron ordering (a3, a2, a1)
    return C.T @ Am @ C


@pytest.mark.parametrize("distorted", [False, True])
@pytest.mark.parametrize("p", [1, 2, 3])
def test_brute_force_two_cells(p, distorted):
    nq = p + 2
    nx, ny, nz = 2, 1, 1
    verts = None
    if distorted:
        verts = inputs.perturbed_vertices(nx, ny, nz, seed=5, amp=0.0)
        verts = verts + np.random.default_rng(9).uniform(-0.08, 0.08, verts.shape)
    mesh = orc.Mesh(nx, ny, nz, lo=(0, 0, 0), hi=(1.0, 0.6, 0.8), vertices=verts)
    rng = np.random.default_rng(p)
    V = rng.uniform(-1, 1, (2, nq ** 3))
    A = orc.assemble(mesh, p, nq, mu=0.5, Vq=V, constrain=False).toarray()
    B = np.zeros_like(A)
    for e in range(2):
        if verts is None:
            h = np.array([0.5, 0.6, 0.8])
            lo = np.array([0.5 * e, 0, 0])
            corners = [lo + h * np.array([a, b, c]) for c in range(2) for b in range(2) for a in range(2)]
        else:
            corners = []
            for c in range(2):
                for b in range(2):
                    for a in range(2):
                        vi = (e + a) + (nx + 1) * (b + (ny + 1) * c)
                        corners.append(verts[vi])
        Ae = _brute_cell_matrix(corners, p, nq, 0.5, V[e])
        np.testing.assert_allclose(orc.cell_matrix(mesh, p, nq, orc.GAUSS, 0.5, V, e), Ae,
                                   atol=1e-12 * np.abs(Ae).max())
        d = orc.cell_dofs(mesh, p, e)
        B[np.ix_(d, d)] += Ae
    np.testing.assert_allclose(A, B, atol=1e-12 * np.abs(B).max())


# --------------------------------------------------------------------------
# P11  the paper's DoF counts (golden fixture), periodic count, row sampling
# --------------------------------------------------------------------------

def test_paper_dof_counts():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_dof_counts.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) >= 9
    for r in rows:
        dofs, order, n = int(r[0]), int(r[1]), int(r[2])
        assert orc.num_dofs(orc.Mesh(n, n, n), order) == dofs
    assert orc.num_dofs(orc.Mesh(32, 32, 32, periodic=True), 6) == 7077888
    assert orc.num_dofs(orc.Mesh(4, 4, 4), 4) == 4913


def test_apply_rows_matches_csr():
    p, nq = 3, 5
    verts = inputs.perturbed_vertices(3, 2, 2, seed=2)
    for periodic, v in ((False, verts), (True, None)):
        mesh = orc.Mesh(3, 2, 2, periodic=periodic, vertices=v)
        E = mesh.num_cells
        V = np.random.default_rng(4).uniform(-1, 1, (E, nq ** 3))
        X = np.random.default_rng(5).standard_normal((orc.num_dofs(mesh, p), 3))
        Y = orc.apply(mesh, p, nq, X, Vq=V)
        rows = np.arange(0, X.shape[0], 7)
        Yr = orc.apply_rows(mesh, p, nq, X, rows, Vq=V)
        np.testing.assert_allclose(Yr, Y[rows], atol=1e-13 * np.abs(Y).max())


@pytest.mark.parametrize("periodic,distorted", [(False, False), (True, False), (False, True)])
def test_row_block_assembly_equals_full_assembly(periodic, distorted):
    """Rows assembled on their own are the rows of the full CSR matrix (same
    sums, same merge), and their CSR x block product equals the oracle's
    row-by-row product."""
    from paper_2208_07129_gb300 import inputs
    verts = inputs.perturbed_vertices(3, 2, 2, seed=5) if distorted else None
    mesh = orc.Mesh(3, 2, 2, periodic=periodic, vertices=verts)
    p, nq = 3, 5
    V = np.random.default_rng(1).uniform(-1, 1, mesh.num_cells * nq ** 3)
    A = orc.assemble(mesh, p, nq, Vq=V)
    rows = np.array([0, 5, 17, 40, 41, 42, orc.num_dofs(mesh, p) - 1])
    B = orc.assemble_rows(mesh, p, nq, rows, Vq=V)
    np.testing.assert_array_equal(B.toarray(), A[rows].toarray())
    X = np.random.default_rng(2).normal(size=(orc.num_dofs(mesh, p), 5))
    np.testing.assert_allclose(orc.spmm(B, X), orc.apply_rows(mesh, p, nq, X, rows, Vq=V), rtol=1e-13, atol=1e-13)


def _gll_nodes_numpy(p):
    """GLL nodes from numpy alone: the end points and the roots of P_p'."""
    inner = np.polynomial.legendre.Legendre.basis(p).deriv().roots().real
    return np.concatenate([[-1.0], np.sort(inner), [1.0]])


def _lagrange_by_vandermonde(nodes, t):
    """Values and first derivatives at the points t of the Lagrange basis on
    `nodes`, from the monomial coefficients (inverse Vandermonde matrix);
    rows are points, columns basis functions."""
    n = len(nodes)
    C = np.linalg.inv(np.vander(nodes, n, increasing=True))
    T = np.vander(t, n, increasing=True)
    dT = np.zeros_like(T)
    dT[:, 1:] = T[:, :-1] * np.arange(1, n)
    return T @ C, dT @ C


@pytest.mark.parametrize("p,nq", [(2, 4), (3, 5), (4, 6)])
def test_box_cell_matrix_is_a_kronecker_sum(p, nq):
    """On an axis-aligned box cell J = diag(h/2) is diagonal, and so is the
    metric mu det J J^-1 J^-T: the cell matrix (Sec. 2.2, the cell stiffness
    and mass by the tensor quadrature) separates into
        mu det J sum_d (2/h_d)^2 K^ (x) M^ (x) M^ (K^ along direction d)
        + c det J M^ (x) M^ (x) M^              (V = c constant)
    with the 1D matrices K^ = D^T W D and M^ = N^T W N of the reference
    interval, built here from numpy's Gauss rule and a Vandermonde Lagrange
    basis on numpy's GLL nodes.  No mixed d/dx d/dy term appears: this is the
    reading the CUDA-core kernels use for box cells (three scalings of the
    gradient at every quadrature point)."""
    mu, c = 0.5, 1.7
    lo, hi = (0.1, -0.2, 0.3), (0.6, 0.5, 0.55)
    h = [hi[d] - lo[d] for d in range(3)]
    mesh = orc.Mesh(1, 1, 1, lo=lo, hi=hi)
    Vq = np.full(nq ** 3, c)
    A = orc.cell_matrix(mesh, p, nq, orc.GAUSS, mu, Vq, 0)

    xq, wq = np.polynomial.legendre.leggauss(nq)
    N, D = _lagrange_by_vandermonde(_gll_nodes_numpy(p), xq)
    M1 = N.T @ (wq[:, None] * N)
    K1 = D.T @ (wq[:, None] * D)
    det = h[0] * h[1] * h[2] / 8.0
    kron3 = lambda a3, a2, a1: np.kron(a3, np.kron(a2, a1))   # local index i1 + n_p (i2 + n_p i3)
    ref = mu * det * ((2 / h[0]) ** 2 * kron3(M1, M1, K1) + (2 / h[1]) ** 2 * kron3(M1, K1, M1)
                      + (2 / h[2]) ** 2 * kron3(K1, M1, M1)) + c * det * kron3(M1, M1, M1)
    assert np.abs(A - ref).max() <= 1e-12 * np.abs(ref).max()
