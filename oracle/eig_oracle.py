"""FP64 oracle of the eigenvalue layer (Sec. 4.3 and Algorithm 6 of the paper).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference legs of ``bench.py`` may use this module; the
product path never does.  It imports nothing from the CUDA package; it builds
on the operator oracle (``oracle.py``) and numpy / scipy.

The paper turns the generalised problem H U = M U Lambda (H the discrete
operator, M the overlap matrix) into a standard one with
H~ = M^-1/2 H M^-1/2, integrating M with the GLL rule of the element's own
nodes so that M is diagonal (Sec. 4.3).  The Chebyshev-filtered subspace
iteration (Algorithm 6) repeatedly applies the fused product
Y = a M^-1/2 H M^-1/2 X + b X + c Y (the cell kernel of its ChFSI appendix).

Functions, each with the passage it follows:
  gll_mass          -- the diagonal overlap matrix by the n_p-point GLL rule (Sec. 4.3)
  scaled_apply      -- Y' = a H~ X + b X + c Y, constrained rows 0 (ChFSI appendix)
  chebyshev_filter  -- the scaled three-term recurrence of Algorithm 6
  chebyshev_gain    -- the polynomial that recurrence applies, in closed form
  dense_eigs        -- eigenpairs of H~ by a dense symmetric eigensolver

Readings (the paper is silent or garbled here):
  * Algorithm 6 as printed never updates sigma inside the filter loop; the
    scaled Chebyshev recurrence it restates (Zhou and Saad's) sets
    sigma <- sigma_2 after every step, which is what makes the filtered block
    equal T_m((H~ - c)/e) / T_m((lambda_min - c)/e) applied to X.  The oracle
    takes that reading, and chebyshev_gain pins it.
  * Dirichlet boxes: H~ acts on the interior nodes only (P H~ P); constrained
    rows of every product are 0 and the mass of a constrained row is reported
    as 1 (it never enters a product).
"""
from __future__ import annotations

from typing import Optional

import numpy as np

from . import oracle as orc


def gll_mass(mesh: "orc.Mesh", p: int, constrain: bool = True) -> np.ndarray:
    """Diagonal of the overlap matrix M_IJ = int phi_I phi_J integrated with the
    tensor GLL rule on the element's n_p = p + 1 nodes (Sec. 4.3).  The basis
    is collocated at those nodes, so the assembled matrix is diagonal; it is
    assembled in full by the operator oracle (mu = 0, V = 1, GLL quadrature
    with n_p points) and its diagonal returned.  Constrained rows get 1 when
    `constrain` is set."""
    n3 = (p + 1) ** 3
    ones = np.ones((mesh.num_cells, n3))
    A = orc.assemble(mesh, p, p + 1, kind=orc.GLL, mu=0.0, Vq=ones, constrain=False)
    d = A.diagonal().copy()
    if constrain:
        d[orc.constrained_mask(mesh, p)] = 1.0
    return d


def mass_offdiag_max(mesh: "orc.Mesh", p: int) -> float:
    """Largest |off-diagonal| entry of the GLL-integrated overlap matrix
    (zero up to rounding: the collocation property)."""
    n3 = (p + 1) ** 3
    A = orc.assemble(mesh, p, p + 1, kind=orc.GLL, mu=0.0, Vq=np.ones((mesh.num_cells, n3)), constrain=False).tocoo()
    off = A.row != A.col
    return float(np.abs(A.data[off]).max()) if off.any() else 0.0


def scaled_operator(A, mass: np.ndarray, mask: Optional[np.ndarray] = None):
    """H~ = M^-1/2 A M^-1/2 as a sparse matrix (rows and columns of constrained
    nodes are zero: A from the operator oracle is already P A P)."""
    import scipy.sparse as sp
    s = 1.0 / np.sqrt(mass)
    if mask is not None:
        s = np.where(mask, 0.0, s)
    D = sp.diags(s)
    return (D @ A @ D).tocsr()


def scaled_apply(Ht, X: np.ndarray, Y: Optional[np.ndarray], a: float, b: float, c: float,
                 mask: Optional[np.ndarray] = None) -> np.ndarray:
    """a H~ X + b X + c Y (the fused product of the ChFSI kernel), with the
    rows of constrained nodes set to 0.  Y may be None when c = 0."""
    out = a * orc.spmm(Ht, X)
    if b != 0.0:
        out = out + b * X
    if c != 0.0:
        out = out + c * Y
    if mask is not None:
        out[mask] = 0.0
    return out


def chebyshev_filter(Ht, X: np.ndarray, m: int, lam_min: float, lam_u: float, lam_max: float,
                     mask: Optional[np.ndarray] = None) -> np.ndarray:
    """The filter loop of Algorithm 6: a degree-m Chebyshev polynomial in H~
    that damps [lam_u, lam_max] and is scaled to 1 at lam_min, evaluated by
    the scaled three-term recurrence, each step one fused product."""
    e = (lam_max - lam_u) / 2.0
    c = (lam_max + lam_u) / 2.0
    sigma = e / (lam_min - c)
    sigma1 = sigma
    gamma = 2.0 / sigma1
    alpha1 = sigma1 / e
    alpha2 = -c
    Xk = X.copy()
    Yk = scaled_apply(Ht, Xk, None, alpha1, alpha1 * alpha2, 0.0, mask)
    for _ in range(2, m + 1):
        sigma2 = 1.0 / (gamma - sigma)
        alpha1 = 2.0 * sigma2 / e
        alpha2 = -sigma * sigma2
        Xn = scaled_apply(Ht, Yk, Xk, alpha1, -c * alpha1, alpha2, mask)
        Xk, Yk = Yk, Xn
        sigma = sigma2
    return Yk


def chebyshev_gain(lam: np.ndarray, m: int, lam_min: float, lam_u: float, lam_max: float) -> np.ndarray:
    """T_m((lam - c)/e) / T_m((lam_min - c)/e): what the filter multiplies an
    eigenvector of eigenvalue lam by (numpy's Chebyshev series evaluation)."""
    from numpy.polynomial import chebyshev as C
    e = (lam_max - lam_u) / 2.0
    c = (lam_max + lam_u) / 2.0
    coef = np.zeros(m + 1)
    coef[m] = 1.0
    return C.chebval((np.asarray(lam) - c) / e, coef) / C.chebval((lam_min - c) / e, coef)


def dense_eigs(Ht, mask: Optional[np.ndarray] = None, k: Optional[int] = None):
    """Eigenvalues (ascending) and orthonormal eigenvectors of H~ on the free
    rows (all rows when mask is None), by LAPACK's dense symmetric solver;
    eigenvectors are returned at full length with constrained rows 0."""
    import scipy.linalg as sla
    free = np.ones(Ht.shape[0], dtype=bool) if mask is None else ~mask
    H = Ht[free][:, free].toarray()
    H = 0.5 * (H + H.T)
    sel = None if k is None else (0, k - 1)
    lam, V = sla.eigh(H, subset_by_index=sel)
    full = np.zeros((Ht.shape[0], V.shape[1]))
    full[free] = V
    return lam, full
