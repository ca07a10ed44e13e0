"""FP64 oracle of the operator on a one-level adaptively refined mesh with
hanging-node constraints (Sec. 3.2.2 and the adaptive-mesh benchmarks of
Sec. 4 of the paper).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference legs of ``bench.py`` may use this module; the
product path never does.  It imports nothing from the CUDA package; the cell
matrices come from the operator oracle (``oracle.py``) evaluated on one-cell
meshes.

Mesh.  A box [lo, hi] of nx x ny x nz coarse cells of size H (per
direction), homogeneous Dirichlet on its boundary; the coarse cells with
index in [r_lo, r_hi) (per direction) are split once into 2 x 2 x 2 children
of size H/2.  Cells are listed coarse cell by coarse cell (x fastest), a
refined cell replaced by its 8 children (x fastest).

Nodes.  Every cell carries the (p+1)^3 tensor GLL nodes.  Along one
direction a node position is one of: a vertex of the half-size grid, m H/2
(key ('v', m)); an interior GLL node i of coarse cell c, c H + (1 + g_i) H/2
(key ('c', c, i)), except the middle node of an even degree, which is the
vertex 2c + 1; an interior GLL node j of fine cell f, f H/2 + (1 + g_j) H/4
(key ('f', f, j)).  Two nodes are the same DoF when their three keys agree.

Numbering (a definition both sides implement): DoFs sorted by position,
z slowest and x fastest, positions compared in units of H/4 per direction:
('v', m) -> 2m, ('c', c, i) -> 4c + 2(1 + g_i), ('f', f, j) -> 2f + (1 + g_j).

Constraints (Sec. 3.2.2: u_S = W u_M).  A node of a fine cell that lies on
the closure of an unrefined coarse cell C without being one of C's nodes is
a hanging (slave) node: its value is the interpolant of C's nodal values at
that point, u_s = sum_m phi_m^C(x_s) u_m, with phi^C the degree-p Lagrange
basis of C on its GLL nodes.  Masters on the Dirichlet boundary carry the
value 0 and are dropped; a slave on the boundary is a Dirichlet node.

Operator.  With C the matrix that maps the free values (the nodes that are
neither slaves nor on the boundary) to all nodes, the constrained operator is
C^T A_full C, where A_full is assembled over all cells from the cell
matrices of the operator oracle.  On full-length vectors: the rows of slaves
and boundary nodes of Y are 0, and their entries in X are ignored.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from . import oracle as orc


@dataclass
class RefinedMesh:
    nx: int
    ny: int
    nz: int
    r_lo: tuple
    r_hi: tuple
    p: int
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (1.0, 1.0, 1.0)
    cells: list = field(default_factory=list)      # (level 0 coarse / 1 fine, (i, j, k) cell index on its level)
    keys: list = field(default_factory=list)       # 3D node key per DoF
    values: np.ndarray = None                      # (n, 3) positions in units of H/4
    cell_dofs: np.ndarray = None                   # (E, (p+1)^3)
    boundary: np.ndarray = None                    # (n,) bool
    slaves: dict = field(default_factory=dict)     # dof -> [(master dof, weight)]


def _refined(m: RefinedMesh, cx, cy, cz) -> bool:
    return all(m.r_lo[d] <= c < m.r_hi[d] for d, c in enumerate((cx, cy, cz)))


def _comp(level: int, c: int, i: int, p: int, g: np.ndarray):
    """1D key and position (units of H/4) of node i of cell c on a level."""
    if level == 0:
        if i == 0:
            return ("v", 2 * c), 4.0 * c
        if i == p:
            return ("v", 2 * c + 2), 4.0 * c + 4.0
        if p % 2 == 0 and i == p // 2:
            return ("v", 2 * c + 1), 4.0 * c + 2.0
        return ("c", c, i), 4.0 * c + 2.0 * (1.0 + g[i])
    if i == 0:
        return ("v", c), 2.0 * c
    if i == p:
        return ("v", c + 1), 2.0 * c + 2.0
    return ("f", c, i), 2.0 * c + (1.0 + g[i])


def build(nx, ny, nz, r_lo, r_hi, p, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)) -> RefinedMesh:
    """Cells, the numbering and the hanging-node constraints."""
    m = RefinedMesh(nx, ny, nz, tuple(r_lo), tuple(r_hi), p, tuple(lo), tuple(hi))
    g, _ = orc.gll(p + 1)
    for cz in range(nz):
        for cy in range(ny):
            for cx in range(nx):
                if _refined(m, cx, cy, cz):
                    for k in range(8):
                        m.cells.append((1, (2 * cx + (k & 1), 2 * cy + ((k >> 1) & 1), 2 * cz + ((k >> 2) & 1))))
                else:
                    m.cells.append((0, (cx, cy, cz)))
    where = {}
    node_keys = []
    for level, idx in m.cells:
        comps = [[_comp(level, idx[d], i, p, g) for i in range(p + 1)] for d in range(3)]
        lst = []
        for i3 in range(p + 1):
            for i2 in range(p + 1):
                for i1 in range(p + 1):
                    key = (comps[0][i1][0], comps[1][i2][0], comps[2][i3][0])
                    where[key] = (comps[0][i1][1], comps[1][i2][1], comps[2][i3][1])
                    lst.append(key)
        node_keys.append(lst)
    m.keys = sorted(where, key=lambda k: (where[k][2], where[k][1], where[k][0]))
    index = {k: i for i, k in enumerate(m.keys)}
    m.values = np.array([where[k] for k in m.keys])
    m.cell_dofs = np.array([[index[k] for k in lst] for lst in node_keys], dtype=np.int64)
    n_c = (nx, ny, nz)
    m.boundary = np.array([any(k[d][0] == "v" and k[d][1] in (0, 2 * n_c[d]) for d in range(3)) for k in m.keys])
    on_fine = np.zeros(len(m.keys), dtype=bool)
    for e, (level, _) in enumerate(m.cells):
        if level == 1:
            on_fine[m.cell_dofs[e]] = True

    # hanging nodes: nodes of fine cells on the closure of an unrefined coarse cell C
    # that are not nodes of C; u_s = sum over C's nodes of phi_m^C(x_s) u_m
    for s_, key in enumerate(m.keys):
        if m.boundary[s_] or not on_fine[s_]:
            continue
        v = m.values[s_]
        cand = [sorted({int(np.floor(v[d] / 4.0)), int(np.ceil(v[d] / 4.0)) - 1} & set(range(n_c[d])))
                for d in range(3)]
        owners = [(cx, cy, cz) for cz in cand[2] for cy in cand[1] for cx in cand[0]
                  if not _refined(m, cx, cy, cz)]
        own_node = any(all(key[d] in [_comp(0, c3[d], i, p, g)[0] for i in range(p + 1)] for d in range(3))
                       for c3 in owners)
        if not owners or own_node:
            continue                                # interior to the refined region, or shared with C
        found = owners[0]
        c3 = found
        xi = [(v[d] - 4.0 * c3[d]) / 2.0 - 1.0 for d in range(3)]
        ph = [orc.lagrange(g, float(x))[0] for x in xi]
        masters = []
        for i3 in range(p + 1):
            for i2 in range(p + 1):
                for i1 in range(p + 1):
                    w = ph[0][i1] * ph[1][i2] * ph[2][i3]
                    if abs(w) <= 1e-14:
                        continue
                    mk = tuple(_comp(0, c3[d], i, p, g)[0] for d, i in enumerate((i1, i2, i3)))
                    md = index[mk]
                    if not m.boundary[md]:
                        masters.append((md, w))
        m.slaves[s_] = masters
    return m


def cell_box(m: RefinedMesh, k: int):
    level, idx = m.cells[k]
    H = np.array([(m.hi[d] - m.lo[d]) / n for d, n in enumerate((m.nx, m.ny, m.nz))])
    w = H if level == 0 else H / 2.0
    clo = np.array(m.lo) + np.array(idx) * w
    return clo, clo + w


def quad_points(m: RefinedMesh, nq: int) -> np.ndarray:
    """Physical quadrature points (E, nq^3, 3) of every cell, in cell order."""
    out = []
    for k in range(len(m.cells)):
        clo, chi = cell_box(m, k)
        out.append(orc.quad_points(orc.Mesh(1, 1, 1, lo=tuple(clo), hi=tuple(chi)), m.p, nq)[0])
    return np.array(out)


def assemble_full(m: RefinedMesh, nq: int, mu: float = 0.5, Vq: Optional[np.ndarray] = None):
    """A_full: the sum over all cells of the cell matrices (no constraints)."""
    import scipy.sparse as sp
    n = len(m.keys)
    rows, cols, vals = [], [], []
    for k in range(len(m.cells)):
        clo, chi = cell_box(m, k)
        one = orc.Mesh(1, 1, 1, lo=tuple(clo), hi=tuple(chi))
        Ae = orc.cell_matrix(one, m.p, nq, orc.GAUSS, mu, None if Vq is None else Vq[k:k + 1], 0)
        d = m.cell_dofs[k]
        rows.append(np.repeat(d, len(d)))
        cols.append(np.tile(d, len(d)))
        vals.append(Ae.ravel())
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))


def constraint_matrix(m: RefinedMesh):
    """C: full-length vectors from free values (columns = all DoFs, only free
    columns used): identity on free nodes, the weights on slaves, zero rows
    on boundary nodes."""
    import scipy.sparse as sp
    n = len(m.keys)
    rows, cols, vals = [], [], []
    for i in range(n):
        if m.boundary[i]:
            continue
        if i in m.slaves:
            for md, w in m.slaves[i]:
                rows.append(i)
                cols.append(md)
                vals.append(w)
        else:
            rows.append(i)
            cols.append(i)
            vals.append(1.0)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def free_mask(m: RefinedMesh) -> np.ndarray:
    f = ~m.boundary.copy()
    for s in m.slaves:
        f[s] = False
    return f


def operator(m: RefinedMesh, nq: int, mu: float = 0.5, Vq: Optional[np.ndarray] = None):
    """The constrained operator on full-length vectors, C^T A_full C with the
    rows of non-free nodes zeroed."""
    import scipy.sparse as sp
    C = constraint_matrix(m)
    A = (C.T @ assemble_full(m, nq, mu, Vq) @ C).tocsr()
    D = sp.diags(free_mask(m).astype(float))
    return (D @ A @ D).tocsr()


def apply(m: RefinedMesh, nq: int, X: np.ndarray, mu: float = 0.5, Vq: Optional[np.ndarray] = None) -> np.ndarray:
    return orc.spmm(operator(m, nq, mu, Vq), X)
