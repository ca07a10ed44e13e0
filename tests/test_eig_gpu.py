"""GPU parity of the eigenvalue layer (include/fe_eig.h) against the FP64
oracle (oracle/eig_oracle.py), through the C ABI: the GLL mass, the fused
scaled product a M^-1/2 A M^-1/2 X + b X + c Y, the Chebyshev filter of
Algorithm 6 and the subspace iteration's eigenpairs.

Tolerances: FP64 products 1e-12 relative (as fe_apply); FP32 products 2e-6
(inputs rounded to FP32 on both sides); eigenvalues 1e-9 relative to the
dense solver once the residuals are below 1e-7 (the error of a Ritz value is
about residual^2 / gap)."""
import numpy as np
import pytest

from oracle import eig_oracle as eo
from oracle import oracle as orc
from paper_2208_07129_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fe():
    from paper_2208_07129_gb300 import build, fe as fe_mod
    build.build()
    fe_mod.lib()
    return fe_mod


def _pair(fe, nx, ny, nz, p, nq, periodic=False, distorted=False, seed=0, potential=True):
    verts = inputs.perturbed_vertices(nx, ny, nz, seed=40 + seed) if distorted else None
    ctx = fe.fe_setup(nx, ny, nz, p, nq, periodic=periodic, vertices=verts)
    mesh = orc.Mesh(nx, ny, nz, periodic=periodic, vertices=verts)
    Vo = None
    if potential:
        fe.fe_set_potential(ctx, inputs.gaussian_potential(fe.fe_quadrature_points(ctx), 60 + seed, periodic))
        Vo = inputs.gaussian_potential(orc.quad_points(mesh, p, nq), 60 + seed, periodic)
    A = orc.assemble(mesh, p, nq, Vq=Vo)
    mask = orc.constrained_mask(mesh, p)
    m = eo.gll_mass(mesh, p)
    return ctx, mesh, mask, eo.scaled_operator(A, m, mask), m


MESHES = [
    # (nx, ny, nz, p, nq, periodic, distorted)
    (3, 2, 2, 4, 6, False, False),
    (3, 2, 3, 6, 8, True, False),     # odd periodic count: three colours along x and z
    (2, 2, 2, 3, 5, False, True),     # trilinear cells
    (2, 3, 2, 2, 3, True, True),
]


@pytest.mark.parametrize("case", MESHES, ids=lambda c: f"{c[0]}x{c[1]}x{c[2]}_p{c[3]}_{'per' if c[5] else 'dir'}"
                         f"{'_dist' if c[6] else ''}")
def test_mass_matches_oracle(fe, case):
    nx, ny, nz, p, nq, periodic, distorted = case
    ctx, mesh, mask, Ht, m = _pair(fe, nx, ny, nz, p, nq, periodic, distorted)
    try:
        got = fe.fe_mass_gll(ctx)
        np.testing.assert_allclose(got, m, rtol=1e-13, atol=0)
    finally:
        fe.fe_destroy(ctx)


@pytest.mark.parametrize("mode,tol", [("fp64", 1e-12), ("df64", 1e-12), ("fp32", 2e-6)])
@pytest.mark.parametrize("case", MESHES, ids=lambda c: f"{c[0]}x{c[1]}x{c[2]}_p{c[3]}_{'per' if c[5] else 'dir'}"
                         f"{'_dist' if c[6] else ''}")
def test_scaled_apply_matches_oracle(fe, case, mode, tol):
    nx, ny, nz, p, nq, periodic, distorted = case
    ctx, mesh, mask, Ht, m = _pair(fe, nx, ny, nz, p, nq, periodic, distorted, seed=p)
    try:
        fe.fe_set_mode(ctx, mode)
        dt = torch.float64 if mode in ("fp64", "df64") else torch.float32
        n = fe.fe_num_dofs(ctx)
        for (a, b, c, nv) in ((0.7, -0.3, 0.45, 11), (1.0, 0.0, 0.0, 3), (-2.5, 1.25, 0.0, 17)):
            Xd = torch.from_numpy(inputs.random_block(n, nv, "uniform", 3 + nv)).to(device="cuda", dtype=dt)
            if c != 0.0:
                Yd = torch.from_numpy(inputs.random_block(n, nv, "normal", 5 + nv)).to(device="cuda", dtype=dt)
            else:
                Yd = torch.full((n, nv), float("nan"), dtype=dt, device="cuda")   # must not be read
            Y0 = Yd.double().cpu().numpy()
            Xr = Xd.double().cpu().numpy()
            fe.fe_apply_scaled(ctx, Xd, Yd, a, b, c)
            torch.cuda.synchronize()
            got = Yd.double().cpu().numpy()
            want = eo.scaled_apply(Ht, Xr, None if c == 0 else Y0, a, b, c, mask)
            assert np.all(np.isfinite(got))
            rel = np.linalg.norm(got - want) / np.linalg.norm(want)
            err = np.abs(got - want).max() / np.abs(want).max()
            assert rel <= tol and err <= tol, (a, b, c, rel, err)
    finally:
        fe.fe_destroy(ctx)


@pytest.mark.parametrize("mode", ["fp64", "df64"])
def test_chebyshev_filter_matches_oracle(fe, mode):
    ctx, mesh, mask, Ht, m = _pair(fe, 3, 2, 2, 4, 6)
    try:
        fe.fe_set_mode(ctx, mode)
        lam, _ = eo.dense_eigs(Ht, mask)
        lmin, lu, lmax = lam[0], lam[12], lam[-1] * 1.02
        n = fe.fe_num_dofs(ctx)
        X0 = inputs.random_block(n, 9, "normal", 21)
        X0[mask] = 0.0
        for deg in (1, 2, 11):
            X = torch.from_numpy(X0).cuda()
            Y = torch.empty_like(X)
            fe.fe_chebyshev_filter(ctx, X, Y, deg, lmin, lu, lmax)
            torch.cuda.synchronize()
            got = X.cpu().numpy()
            want = eo.chebyshev_filter(Ht, X0, deg, lmin, lu, lmax, mask)
            rel = np.linalg.norm(got - want) / np.linalg.norm(want)
            assert rel <= 1e-11, (deg, rel)
    finally:
        fe.fe_destroy(ctx)


def _check_eigs(fe, ctx, Ht, mask, U, res, n_wanted, tol):
    lam_ref, _ = eo.dense_eigs(Ht, mask, k=n_wanted)
    lam = res["eigenvalues"][:n_wanted]
    np.testing.assert_allclose(lam, lam_ref, rtol=1e-9, atol=0)
    Uh = U.cpu().numpy()
    assert np.all(Uh[mask] == 0.0)
    k = Uh.shape[1]
    assert np.abs(Uh.T @ Uh - np.eye(k)).max() <= 1e-10
    # residuals recomputed by the oracle from the returned vectors
    R = orc.spmm(Ht, Uh[:, :n_wanted]) - Uh[:, :n_wanted] * lam[None, :]
    r = np.linalg.norm(R, axis=0)
    assert np.all(r <= 1.01 * tol + 1e-12), r
    # below ~1e-9 both are rounding noise of applying H~ (|H~| ~ 1e4 here)
    np.testing.assert_allclose(r, res["residuals"][:n_wanted], rtol=1e-3, atol=1e-9)


# The wanted set ends at a gap of the spectrum: on the periodic cube the
# Laplacian's eigenvalues come in clusters of 1, 6, 12, ... (split only
# slightly by the potential), and a subspace edge inside a cluster converges
# at the rate of the cluster's width.
@pytest.mark.parametrize("periodic,n_wanted,k,mode", [(False, 10, 16, "fp64"), (True, 7, 20, "fp64"),
                                                       (False, 10, 16, "df64")])
def test_chfsi_eigenpairs(fe, periodic, n_wanted, k, mode):
    ctx, mesh, mask, Ht, m = _pair(fe, 3, 3, 3, 4, 6, periodic=periodic, seed=2)
    try:
        n = fe.fe_num_dofs(ctx)
        U = torch.from_numpy(inputs.random_block(n, k, "normal", 8)).cuda()
        tol = 1e-7
        res = fe.fe_chfsi(ctx, U, n_wanted=n_wanted, degree=12, tol=tol, max_iter=60, filter_mode=mode)
        assert res["status"] == fe.FE_OK, res
        assert res["converged"] == n_wanted and res["max_residual"] <= tol
        assert res["filter_applies"] == 12 * res["iterations"]
        _check_eigs(fe, ctx, Ht, mask, U, res, n_wanted, tol)
    finally:
        fe.fe_destroy(ctx)


def test_chfsi_fp32_filter_then_fp64(fe):
    """Mixed precision: FP32 filter passes while the residual is above 1e-3,
    FP64 after; the result meets the FP64 tolerance."""
    ctx, mesh, mask, Ht, m = _pair(fe, 3, 3, 3, 4, 6, distorted=True, seed=3)
    try:
        n = fe.fe_num_dofs(ctx)
        U = torch.from_numpy(inputs.random_block(n, 16, "normal", 9)).cuda()
        tol = 1e-7
        res = fe.fe_chfsi(ctx, U, n_wanted=10, degree=12, tol=tol, max_iter=60, filter_mode="fp32",
                          fp32_switch=1e-3)
        assert res["status"] == fe.FE_OK, res
        assert res["fp32_passes"] >= 1
        _check_eigs(fe, ctx, Ht, mask, U, res, 10, tol)
    finally:
        fe.fe_destroy(ctx)


def test_chfsi_reports_nonconvergence(fe):
    ctx, mesh, mask, Ht, m = _pair(fe, 2, 2, 2, 3, 5, seed=4)
    try:
        n = fe.fe_num_dofs(ctx)
        U = torch.from_numpy(inputs.random_block(n, 6, "normal", 10)).cuda()
        res = fe.fe_chfsi(ctx, U, n_wanted=4, degree=2, tol=1e-14, max_iter=1)
        assert res["status"] == fe.FE_ENOTCONV
        assert res["iterations"] == 1 and res["max_residual"] > 1e-14
        assert np.all(np.isfinite(res["eigenvalues"]))
    finally:
        fe.fe_destroy(ctx)


def test_scaled_product_full_size(fe):
    """The paper-size eigen case in the filter's launch configuration (17^3,
    p = 6, k = 1280): sampled rows of the GLL mass equal the oracle's (a row
    of the GLL-assembled overlap matrix times a vector of ones), and the
    fused product equals its composition a M^-1/2 A (M^-1/2 X) + b X + c Y
    from fe_apply, a property that holds at any size."""
    w = inputs.WORKLOADS["e1"]
    ctx = fe.setup_workload(w)
    try:
        n, k, p = w.num_dofs, w.n_vec, w.p
        m = fe.fe_mass_gll(ctx)
        mesh = orc.Mesh(w.nx, w.ny, w.nz, periodic=w.periodic)
        mask = w.boundary_mask()
        rng = np.random.default_rng(5)
        rows = np.unique(np.concatenate([rng.integers(0, n, 64), [0, n - 1, n // 2]]))
        mref = orc.apply_rows(mesh, p, p + 1, np.ones((n, 1)), rows, kind=orc.GLL, mu=0.0,
                              Vq=np.ones((w.num_cells, (p + 1) ** 3)), constrain=False)[:, 0]
        mref[mask[rows]] = 1.0
        np.testing.assert_allclose(m[rows], mref, rtol=1e-13, atol=0)

        g = torch.Generator(device="cuda")
        g.manual_seed(3)
        X = torch.randn(n, k, device="cuda", dtype=torch.float64, generator=g)
        Y = torch.randn(n, k, device="cuda", dtype=torch.float64, generator=g)
        Y0 = Y.clone()
        a, b, c = 0.3, -0.7, 0.2
        fe.fe_apply_scaled(ctx, X, Y, a, b, c)
        msq = torch.from_numpy(1.0 / np.sqrt(m)).cuda()[:, None]
        Xs = X * msq
        AXs = torch.empty_like(X)
        fe.fe_apply(ctx, Xs, AXs)
        ref = a * msq * AXs + b * X + c * Y0
        ref[torch.from_numpy(mask).cuda()] = 0.0
        rel = (torch.linalg.norm(Y - ref) / torch.linalg.norm(ref)).item()
        assert rel <= 1e-12, rel
    finally:
        fe.fe_destroy(ctx)
