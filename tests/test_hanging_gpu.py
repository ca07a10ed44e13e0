"""GPU parity of the refined-mesh product with hanging nodes (fe_setup_refined)
against the hanging-node oracle (oracle/hanging_oracle.py), through the C ABI.

Element-wise against the oracle's C^T A C on small meshes (FP64 and the
double-float mode within 1e-12, FP32 within 2e-6 on FP32-rounded inputs); the
numbering, the node coordinates and the slave count must agree exactly.  At
the size the benchmark times, the Galerkin identity K u = M f for a
polynomial u in the constrained space is checked instead (it holds at any
size)."""
import numpy as np
import pytest

from oracle import hanging_oracle as ho
from paper_2208_07129_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "df64": 1e-12, "fp32": 2e-6}

MESHES = [
    # (nx, ny, nz, p, nq, refine_lo, refine_hi)
    (3, 3, 3, 2, 4, (1, 1, 1), (2, 2, 2)),
    (3, 3, 3, 3, 5, (1, 1, 1), (2, 2, 2)),
    (4, 3, 3, 4, 6, (1, 1, 0), (3, 2, 2)),      # refined block on the z = 0 boundary
    (3, 2, 2, 6, 8, (0, 0, 0), (2, 1, 1)),      # corner block, p = 6
    (2, 2, 2, 5, 7, (0, 0, 0), (2, 2, 2)),      # everything refined: no hanging nodes
    (3, 3, 2, 8, 10, (1, 0, 0), (2, 2, 1)),     # p = 8
]


@pytest.fixture(scope="module")
def fe():
    from paper_2208_07129_gb300 import build, fe as fe_mod
    build.build()
    fe_mod.lib()
    return fe_mod


def _oracle_xyz(m):
    H = np.array([(m.hi[d] - m.lo[d]) / n for d, n in enumerate((m.nx, m.ny, m.nz))])
    return np.array(m.lo)[None, :] + m.values * (H / 4.0)[None, :]


@pytest.mark.parametrize("mode", ["fp64", "df64", "fp32"])
@pytest.mark.parametrize("case", MESHES, ids=lambda c: f"{c[0]}x{c[1]}x{c[2]}_p{c[3]}_r{c[5]}-{c[6]}")
def test_refined_matches_oracle(fe, case, mode):
    nx, ny, nz, p, nq, rlo, rhi = case
    ctx = fe.fe_setup_refined(nx, ny, nz, p, nq, rlo, rhi)
    try:
        m = ho.build(nx, ny, nz, rlo, rhi, p)
        n = fe.fe_num_dofs(ctx)
        assert n == len(m.keys)
        assert fe.fe_num_slaves(ctx) == len(m.slaves)
        np.testing.assert_allclose(fe.fe_node_coords(ctx), _oracle_xyz(m), rtol=0, atol=1e-14)
        Vg = inputs.gaussian_potential(fe.fe_quadrature_points(ctx), 70 + p, False)
        fe.fe_set_potential(ctx, Vg)
        Vo = inputs.gaussian_potential(ho.quad_points(m, nq), 70 + p, False)
        fe.fe_set_mode(ctx, mode)
        dt = torch.float32 if mode == "fp32" else torch.float64
        X = torch.from_numpy(inputs.random_block(n, 9, "uniform", 5 + p)).to(device="cuda", dtype=dt)
        Y = torch.full_like(X, float("nan"))
        fe.fe_apply(ctx, X, Y)
        torch.cuda.synchronize()
        got = Y.double().cpu().numpy()
        want = ho.apply(m, nq, X.double().cpu().numpy(), Vq=Vo)
        assert np.all(np.isfinite(got))
        rel = np.linalg.norm(got - want) / np.linalg.norm(want)
        err = np.abs(got - want).max() / np.abs(want).max()
        assert rel <= TOL[mode] and err <= TOL[mode], (rel, err)
        assert np.all(got[~ho.free_mask(m)] == 0.0)
    finally:
        fe.fe_destroy(ctx)


def test_unrefined_equals_structured(fe):
    """With nothing refined the map kernel computes the structured product
    (same numbering, colours and arithmetic; the box metric is formed by a
    different FP64 expression, so agreement is to rounding)."""
    a = fe.fe_setup_refined(3, 2, 2, 4, 6, (0, 0, 0), (0, 0, 0))
    b = fe.fe_setup(3, 2, 2, 4, 6)
    try:
        assert fe.fe_num_dofs(a) == fe.fe_num_dofs(b) and fe.fe_num_slaves(a) == 0
        np.testing.assert_allclose(fe.fe_node_coords(a), fe.fe_node_coords(b), rtol=0, atol=1e-15)
        V = inputs.gaussian_potential(fe.fe_quadrature_points(b), 9, False)
        fe.fe_set_potential(a, V)
        fe.fe_set_potential(b, V)
        X = torch.from_numpy(inputs.random_block(fe.fe_num_dofs(a), 5, "normal", 3)).cuda()
        Ya, Yb = torch.empty_like(X), torch.empty_like(X)
        fe.fe_apply(a, X, Ya)
        fe.fe_apply(b, X, Yb)
        torch.cuda.synchronize()
        d = ((Ya - Yb).abs().max() / Yb.abs().max()).item()
        assert d <= 1e-14, d
    finally:
        fe.fe_destroy(a)
        fe.fe_destroy(b)


def test_refined_galerkin_identity_full_size(fe):
    """The refined 14^3 box with its central 8^3 cells split (p = 6), the
    size the benchmark times: u = (x(1-x) y(1-y) z(1-z))^3 is in Q_6 and in
    the constrained space, and f = -1/2 lap u vanishes on the boundary, so
    the stiffness operator (mu = 1/2, V = 0) applied to u equals the mass
    operator (mu = 0, V = 1) applied to f at every free row."""
    w = inputs.WORKLOADS["h1"]
    rlo, rhi = w.extra["refine_lo"], w.extra["refine_hi"]
    K = fe.fe_setup_refined(w.nx, w.ny, w.nz, w.p, w.nq, rlo, rhi, mu=0.5)
    M = fe.fe_setup_refined(w.nx, w.ny, w.nz, w.p, w.nq, rlo, rhi, mu=0.0)
    try:
        fe.fe_set_potential(M, np.ones(fe.fe_num_cells(M) * w.nq ** 3))
        xyz = fe.fe_node_coords(K)
        x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
        a, b, c = x * (1 - x), y * (1 - y), z * (1 - z)
        # lap(a^3) = 6 a (a')^2 + 3 a^2 a'' with a' = 1 - 2x, a'' = -2
        la = 6 * a * (1 - 2 * x) ** 2 - 6 * a * a
        lb = 6 * b * (1 - 2 * y) ** 2 - 6 * b * b
        lc = 6 * c * (1 - 2 * z) ** 2 - 6 * c * c
        u = (a * b * c) ** 3
        f = -0.5 * (la * b ** 3 * c ** 3 + a ** 3 * lb * c ** 3 + a ** 3 * b ** 3 * lc)
        # K u cancels heavily (|K| |u| / |K u| ~ 1e3 here), which amplifies the
        # unit roundoff: 2^-53 for FP64, about 2^-48 for double-float
        for mode, tol in (("fp64", 1e-11), ("df64", 1e-10)):
            fe.fe_set_mode(K, mode)
            fe.fe_set_mode(M, mode)
            U = torch.from_numpy(np.stack([u, -2.0 * u], axis=1)).cuda()
            F = torch.from_numpy(np.stack([f, -2.0 * f], axis=1)).cuda()
            KU, MF = torch.empty_like(U), torch.empty_like(F)
            fe.fe_apply(K, U, KU)
            fe.fe_apply(M, F, MF)
            torch.cuda.synchronize()
            d = (KU - MF).abs().max().item() / MF.abs().max().item()
            print(mode, d)
            assert d <= tol, (mode, d)
    finally:
        fe.fe_destroy(K)
        fe.fe_destroy(M)
