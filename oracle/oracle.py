"""Python binding of the FP64 CPU oracle (``fe_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference legs of ``bench.py`` may use this module; the
product path never does.  It imports nothing from the CUDA package.

The oracle defines the discrete operator of Sec. 2.1-2.2 of the paper,

    A_IJ = sum_e sum_Q w_Q det J [ mu (J^-T grad N_I).(J^-T grad N_J) + V(x_Q) N_I N_J ],

with degree-p Lagrange shape functions on GLL nodes and the tensor n_q-point
quadrature rule, assembles it row by row into a CSR matrix and multiplies it
with a DoF-major block of vectors.  Dirichlet boxes are constrained as P A P
(P zeroes boundary nodes); periodic boxes wrap the node numbering.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fe_oracle.c")
_LIB = os.path.join(_HERE, "libfe_oracle.so")

GAUSS = 0
GLL = 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -fopenmp) into oracle/libfe_oracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _CMesh(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("periodic", ctypes.c_int),
        ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
        ("vertex_xyz", ctypes.POINTER(ctypes.c_double)),
    ]


_lib = None


def _L():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        lp = ctypes.POINTER(ctypes.c_long)
        mp = ctypes.POINTER(_CMesh)
        _lib.oracle_gauss.argtypes = [ctypes.c_int, dp, dp]
        _lib.oracle_gll.argtypes = [ctypes.c_int, dp, dp]
        _lib.oracle_lagrange.argtypes = [ctypes.c_int, dp, ctypes.c_double, dp, dp]
        _lib.oracle_lagrange.restype = None
        _lib.oracle_num_dofs.argtypes = [mp, ctypes.c_int]
        _lib.oracle_num_dofs.restype = ctypes.c_long
        _lib.oracle_num_cells.argtypes = [mp]
        _lib.oracle_num_cells.restype = ctypes.c_long
        _lib.oracle_cell_dofs.argtypes = [mp, ctypes.c_int, ctypes.c_long, lp]
        _lib.oracle_is_constrained.argtypes = [mp, ctypes.c_int, ctypes.c_long]
        _lib.oracle_quad_points.argtypes = [mp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
        _lib.oracle_cell_matrix.argtypes = [mp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                            dp, ctypes.c_long, dp]
        _lib.oracle_assemble_csr.argtypes = [mp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                             dp, ctypes.c_int, lp, lp, dp]
        _lib.oracle_csr_spmm.argtypes = [ctypes.c_long, lp, lp, dp, dp, ctypes.c_int, dp]
        _lib.oracle_assemble_rows_csr.argtypes = [mp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                                  dp, ctypes.c_int, lp, ctypes.c_long, lp, lp, dp]
        _lib.oracle_apply_rows.argtypes = [mp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                           dp, ctypes.c_int, dp, ctypes.c_int, lp, ctypes.c_long, dp]
        _lib.oracle_num_threads.restype = ctypes.c_int
    return _lib


def _dp(a: Optional[np.ndarray]):
    if a is None:
        return ctypes.POINTER(ctypes.c_double)()
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _lp(a: np.ndarray):
    assert a.dtype == np.int64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_long))


def _check(status: int, what: str):
    if status != 0:
        raise RuntimeError(f"oracle {what} failed with status {status}")


@dataclass
class Mesh:
    """Structured hexahedral mesh of nx*ny*nz cells on the box [lo, hi].

    ``vertices`` (optional) holds the (nx+1)(ny+1)(nz+1) x 3 vertex coordinates,
    x fastest; each cell is the trilinear image of the reference cube.
    """
    nx: int
    ny: int
    nz: int
    periodic: bool = False
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (1.0, 1.0, 1.0)
    vertices: Optional[np.ndarray] = None
    _c: _CMesh = field(default=None, repr=False)

    def c(self) -> _CMesh:
        m = _CMesh()
        m.nx, m.ny, m.nz = self.nx, self.ny, self.nz
        m.periodic = int(self.periodic)
        for d in range(3):
            m.lo[d] = float(self.lo[d])
            m.hi[d] = float(self.hi[d])
        if self.vertices is not None:
            v = np.ascontiguousarray(self.vertices, dtype=np.float64)
            assert v.size == (self.nx + 1) * (self.ny + 1) * (self.nz + 1) * 3
            self._vkeep = v
            m.vertex_xyz = _dp(v)
        self._c = m
        return m

    @property
    def num_cells(self) -> int:
        return self.nx * self.ny * self.nz


def gauss(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    _check(_L().oracle_gauss(n, _dp(x), _dp(w)), "gauss")
    return x, w


def gll(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    _check(_L().oracle_gll(n, _dp(x), _dp(w)), "gll")
    return x, w


def lagrange(nodes: np.ndarray, t: float):
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    phi = np.zeros(len(nodes))
    dphi = np.zeros(len(nodes))
    _L().oracle_lagrange(len(nodes), _dp(nodes), float(t), _dp(phi), _dp(dphi))
    return phi, dphi


def num_dofs(mesh: Mesh, p: int) -> int:
    return int(_L().oracle_num_dofs(ctypes.byref(mesh.c()), p))


def cell_dofs(mesh: Mesh, p: int, e: int) -> np.ndarray:
    out = np.zeros((p + 1) ** 3, dtype=np.int64)
    _check(_L().oracle_cell_dofs(ctypes.byref(mesh.c()), p, e, _lp(out)), "cell_dofs")
    return out


def constrained_mask(mesh: Mesh, p: int) -> np.ndarray:
    """Boolean mask of Dirichlet-constrained DoFs (all False when periodic)."""
    n = num_dofs(mesh, p)
    m = mesh.c()
    lib = _L()
    return np.array([bool(lib.oracle_is_constrained(ctypes.byref(m), p, i)) for i in range(n)])


def quad_points(mesh: Mesh, p: int, nq: int, kind: int = GAUSS) -> np.ndarray:
    """Physical quadrature points, shape (E, nq^3, 3), Q = q1 + nq (q2 + nq q3)."""
    out = np.zeros((mesh.num_cells, nq ** 3, 3))
    _check(_L().oracle_quad_points(ctypes.byref(mesh.c()), p, nq, kind, _dp(out)), "quad_points")
    return out


def cell_matrix(mesh: Mesh, p: int, nq: int, kind: int, mu: float, Vq: Optional[np.ndarray], e: int) -> np.ndarray:
    n3 = (p + 1) ** 3
    out = np.zeros((n3, n3))
    Vq = None if Vq is None else np.ascontiguousarray(Vq, dtype=np.float64)
    _check(_L().oracle_cell_matrix(ctypes.byref(mesh.c()), p, nq, kind, mu, _dp(Vq), e, _dp(out)), "cell_matrix")
    return out


def assemble(mesh: Mesh, p: int, nq: int, kind: int = GAUSS, mu: float = 0.5,
             Vq: Optional[np.ndarray] = None, constrain: bool = True):
    """Global matrix A as (rowptr, col, val) CSR arrays (int64, int64, float64)."""
    import scipy.sparse as sp
    n = num_dofs(mesh, p)
    Vq = None if Vq is None else np.ascontiguousarray(Vq, dtype=np.float64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    m = mesh.c()
    lib = _L()
    null_l = ctypes.POINTER(ctypes.c_long)()
    _check(lib.oracle_assemble_csr(ctypes.byref(m), p, nq, kind, mu, _dp(Vq), int(constrain),
                                   _lp(rowptr), null_l, _dp(None)), "assemble(count)")
    nnz = int(rowptr[-1])
    col = np.zeros(nnz, dtype=np.int64)
    val = np.zeros(nnz)
    _check(lib.oracle_assemble_csr(ctypes.byref(m), p, nq, kind, mu, _dp(Vq), int(constrain),
                                   _lp(rowptr), _lp(col), _dp(val)), "assemble(fill)")
    return sp.csr_matrix((val, col, rowptr), shape=(n, n))


def assemble_rows(mesh: Mesh, p: int, nq: int, rows: np.ndarray, kind: int = GAUSS, mu: float = 0.5,
                  Vq: Optional[np.ndarray] = None, constrain: bool = True):
    """Rows ``rows`` of the global matrix as a CSR block (len(rows) x num_dofs),
    each row assembled from the matching rows of its cells' matrices."""
    import scipy.sparse as sp
    n = num_dofs(mesh, p)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    Vq = None if Vq is None else np.ascontiguousarray(Vq, dtype=np.float64)
    rowptr = np.zeros(len(rows) + 1, dtype=np.int64)
    m = mesh.c()
    lib = _L()
    null_l = ctypes.POINTER(ctypes.c_long)()
    _check(lib.oracle_assemble_rows_csr(ctypes.byref(m), p, nq, kind, mu, _dp(Vq), int(constrain), _lp(rows),
                                        len(rows), _lp(rowptr), null_l, _dp(None)), "assemble_rows(count)")
    nnz = int(rowptr[-1])
    col = np.zeros(nnz, dtype=np.int64)
    val = np.zeros(nnz)
    _check(lib.oracle_assemble_rows_csr(ctypes.byref(m), p, nq, kind, mu, _dp(Vq), int(constrain), _lp(rows),
                                        len(rows), _lp(rowptr), _lp(col), _dp(val)), "assemble_rows(fill)")
    return sp.csr_matrix((val, col, rowptr), shape=(len(rows), n))


def spmm(A, X: np.ndarray) -> np.ndarray:
    """Y = A X with the oracle's own OpenMP CSR x dense-block product."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    if X.ndim == 1:
        X = X[:, None]
    nv = X.shape[1]
    Y = np.zeros((A.shape[0], nv))
    rowptr = np.ascontiguousarray(A.indptr, dtype=np.int64)
    col = np.ascontiguousarray(A.indices, dtype=np.int64)
    val = np.ascontiguousarray(A.data, dtype=np.float64)
    _check(_L().oracle_csr_spmm(A.shape[0], _lp(rowptr), _lp(col), _dp(val), _dp(X), nv, _dp(Y)), "spmm")
    return Y


def apply(mesh: Mesh, p: int, nq: int, X: np.ndarray, kind: int = GAUSS, mu: float = 0.5,
          Vq: Optional[np.ndarray] = None, constrain: bool = True) -> np.ndarray:
    """Y = A X through the assembled CSR matrix."""
    return spmm(assemble(mesh, p, nq, kind, mu, Vq, constrain), X)


def apply_rows(mesh: Mesh, p: int, nq: int, X: np.ndarray, rows: np.ndarray, kind: int = GAUSS,
               mu: float = 0.5, Vq: Optional[np.ndarray] = None, constrain: bool = True) -> np.ndarray:
    """Rows ``rows`` of Y = A X, each assembled on the fly (for meshes too big for CSR)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    n, nv = X.shape
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.zeros((len(rows), nv))
    Vq = None if Vq is None else np.ascontiguousarray(Vq, dtype=np.float64)
    _check(_L().oracle_apply_rows(ctypes.byref(mesh.c()), p, nq, kind, mu, _dp(Vq), int(constrain),
                                  _dp(X), nv, _lp(rows), len(rows), _dp(out)), "apply_rows")
    return out


def num_threads() -> int:
    return int(_L().oracle_num_threads())
