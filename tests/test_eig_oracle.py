"""Pins of the eigenvalue-layer oracle (oracle/eig_oracle.py) against facts
that do not come from the oracle itself: textbook GLL weights, the domain
volume, the collocation property, a library generalised eigensolver, the
Laplacian's closed-form spectrum and numpy's Chebyshev evaluation."""
import numpy as np
import pytest

from oracle import eig_oracle as eo
from oracle import oracle as orc
from paper_2208_07129_gb300 import inputs


def test_gll_mass_single_cell_textbook():
    # unit cube, p = 2: GLL weights on [-1, 1] are (1/3, 4/3, 1/3), det J = 1/8
    mesh = orc.Mesh(1, 1, 1)
    m = eo.gll_mass(mesh, 2, constrain=False)
    w = np.array([1 / 3, 4 / 3, 1 / 3])
    want = np.einsum("k,j,i->kji", w, w, w).ravel() / 8.0     # index gx + 3 (gy + 3 gz)
    np.testing.assert_allclose(m, want, rtol=1e-14)


@pytest.mark.parametrize("p", [2, 3, 4])
@pytest.mark.parametrize("periodic,distorted", [(False, False), (True, False), (False, True)])
def test_gll_mass_sums_to_volume(p, periodic, distorted):
    # the p+1-point GLL rule integrates det J (degree <= 2 per direction) exactly for p >= 2
    lo, hi = (-0.5, 0.0, 1.0), (1.0, 0.25, 3.0)
    verts = inputs.perturbed_vertices(3, 2, 2, seed=5) if distorted else None
    mesh = orc.Mesh(3, 2, 2, periodic=periodic, lo=lo, hi=hi, vertices=verts)
    vol = 1.0 if distorted else np.prod(np.subtract(hi, lo))
    m = eo.gll_mass(mesh, p, constrain=False)
    assert abs(m.sum() - vol) <= 1e-13 * vol
    assert np.all(m > 0)


def test_gll_mass_is_diagonal():
    mesh = orc.Mesh(2, 2, 2, vertices=inputs.perturbed_vertices(2, 2, 2, seed=9))
    m = eo.gll_mass(mesh, 3, constrain=False)
    assert eo.mass_offdiag_max(mesh, 3) <= 1e-15 * m.max()


def test_scaled_operator_matches_generalised_eigenproblem():
    """eig(M^-1/2 A M^-1/2) = eig(A, M): the standard form of Sec. 4.3,
    checked against LAPACK's generalised solver on the free rows."""
    import scipy.linalg as sla
    mesh = orc.Mesh(2, 2, 2)
    p, nq = 3, 5
    V = inputs.gaussian_potential(orc.quad_points(mesh, p, nq), 4, False)
    A = orc.assemble(mesh, p, nq, Vq=V)
    mask = orc.constrained_mask(mesh, p)
    m = eo.gll_mass(mesh, p)
    Ht = eo.scaled_operator(A, m, mask)
    lam, _ = eo.dense_eigs(Ht, mask)
    free = ~mask
    lam_g = sla.eigh(A[free][:, free].toarray(), np.diag(m[free]), eigvals_only=True)
    np.testing.assert_allclose(lam, lam_g, rtol=1e-10, atol=1e-10 * np.abs(lam_g).max())


def test_laplacian_spectrum_converges():
    """-1/2 lap on the unit cube, Dirichlet: eigenvalues (pi^2/2)(l^2+m^2+n^2);
    the smallest is simple (3 pi^2 / 2), the next is triple (3 pi^2).  The
    discrete values approach them under refinement."""
    errs = []
    for nx in (2, 3):
        mesh = orc.Mesh(nx, nx, nx)
        p = 3
        A = orc.assemble(mesh, p, p + 2, Vq=None)
        mask = orc.constrained_mask(mesh, p)
        Ht = eo.scaled_operator(A, eo.gll_mass(mesh, p), mask)
        lam, _ = eo.dense_eigs(Ht, mask, k=5)
        exact = np.pi ** 2 / 2 * np.array([3, 6, 6, 6, 9])
        errs.append(np.abs(lam - exact) / exact)
        assert np.all(np.abs(lam[1:4] - lam[1:4].mean()) <= 1e-9 * lam[1])   # the triple
    assert errs[1].max() < errs[0].max()
    assert errs[1].max() < 2e-3


def test_chebyshev_filter_closed_form():
    """The recurrence multiplies each eigenvector of H~ by
    T_m((lam - c)/e) / T_m((lam_min - c)/e)."""
    mesh = orc.Mesh(2, 2, 2, periodic=True)
    p, nq = 2, 4
    V = inputs.gaussian_potential(orc.quad_points(mesh, p, nq), 7, True)
    A = orc.assemble(mesh, p, nq, Vq=V)
    Ht = eo.scaled_operator(A, eo.gll_mass(mesh, p))
    lam, Q = eo.dense_eigs(Ht)
    X = inputs.random_block(Ht.shape[0], 3, "normal", 11)
    lam_min, lam_u, lam_max = lam[0], lam[6], lam[-1] * 1.01
    for m in (1, 2, 9):
        got = eo.chebyshev_filter(Ht, X, m, lam_min, lam_u, lam_max)
        g = eo.chebyshev_gain(lam, m, lam_min, lam_u, lam_max)
        want = Q @ (g[:, None] * (Q.T @ X))
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-10 * np.abs(want).max())
    # the damped interval stays bounded by 1 / |T_m(t0)|, the wanted end is amplified relative to it
    g = eo.chebyshev_gain(lam, 9, lam_min, lam_u, lam_max)
    assert np.all(np.abs(g[lam >= lam_u]) <= np.abs(g[0]) * 1e-3)
