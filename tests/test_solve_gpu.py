"""Block-PCG through the C ABI: the solution is checked against a sparse
direct solve of the oracle's assembled matrix, and every final residual
against the FP64 operator."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

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


def _problem(fe, nx=3, p=4, nq=6, n_vec=6, distorted=False, seed=0):
    verts = inputs.perturbed_vertices(nx, nx, nx, seed=5) if distorted else None
    ctx = fe.fe_setup(nx, nx, nx, p, nq, vertices=verts)
    mesh = orc.Mesh(nx, nx, nx, vertices=verts)
    V = lambda xyz: inputs.gaussian_potential(xyz, 15, False, 0.125) + 1.0   # V + sigma, sigma = 1
    fe.fe_set_potential(ctx, V(fe.fe_quadrature_points(ctx)))
    A = orc.assemble(mesh, p, nq, Vq=V(orc.quad_points(mesh, p, nq)))
    mask = orc.constrained_mask(mesh, p)
    B = inputs.random_block(fe.fe_num_dofs(ctx), n_vec, "normal", seed)
    B[mask] = 0.0
    keep = ~mask
    Xref = np.zeros_like(B)
    Aint = A[keep][:, keep].tocsc()
    lu = spla.splu(Aint)
    Xref[keep] = lu.solve(B[keep])
    return ctx, B, Xref


@pytest.mark.parametrize("precond,inner", [("jacobi", "fp64"), ("none", "fp64"), ("jacobi", "fp32"),
                                           ("jacobi", "tf32"), ("jacobi", "bf16"), ("jacobi", "tf32x3"),
                                           ("jacobi", "df64")])
@pytest.mark.parametrize("n_vec", [6, 8], ids=["nv6", "nv8"])
def test_pcg_solution(fe, precond, inner, n_vec):
    """n_vec = 8 runs the 16-byte vector kernels in FP64 and FP32; n_vec = 6
    runs them in FP64 only (FP32 needs a multiple of 4 columns)."""
    ctx, B, Xref = _problem(fe, n_vec=n_vec, distorted=(inner != "fp64"))
    try:
        Bd = torch.from_numpy(B).cuda()
        Xd = torch.zeros_like(Bd)
        res = fe.fe_solve(ctx, Bd, Xd, rtol=1e-9, max_it=5000, precond=precond, inner_mode=inner)
        assert res["status"] == fe.FE_OK, res
        assert res["converged_columns"] == B.shape[1]
        assert res["max_rel_residual"] <= 1e-9
        assert np.all(res["rel_res"] <= 1e-9)
        X = Xd.cpu().numpy()
        err = np.linalg.norm(X - Xref) / np.linalg.norm(Xref)
        assert err < 1e-6, err
        if inner == "df64":
            # FP64 PCG on the double-float operator: only the final check is an FP64 apply
            assert res["outer_iterations"] == 0 and res["fp64_applies"] == 1
        elif inner != "fp64":
            # FP64 refinement around the reduced-precision inner solve: one FP64
            # residual per outer step, plus the initial and the judging one
            assert res["outer_iterations"] >= 1 and res["fp64_applies"] == res["outer_iterations"] + 2
    finally:
        fe.fe_destroy(ctx)


def test_pcg_reports_nonconvergence(fe):
    ctx, B, Xref = _problem(fe, n_vec=3)
    try:
        Bd = torch.from_numpy(B).cuda()
        Xd = torch.zeros_like(Bd)
        res = fe.fe_solve(ctx, Bd, Xd, rtol=1e-12, max_it=3, precond="jacobi", inner_mode="fp64")
        assert res["status"] == fe.FE_ENOTCONV
        assert res["iterations"] == 3
        assert res["max_rel_residual"] > 1e-12
    finally:
        fe.fe_destroy(ctx)


def test_jacobi_beats_none(fe):
    ctx, B, Xref = _problem(fe, nx=4, p=3, nq=5, n_vec=4)
    try:
        Bd = torch.from_numpy(B).cuda()
        its = {}
        for pc in ("none", "jacobi"):
            Xd = torch.zeros_like(Bd)
            its[pc] = fe.fe_solve(ctx, Bd, Xd, rtol=1e-8, max_it=5000, precond=pc)["iterations"]
        assert its["jacobi"] < its["none"], its
    finally:
        fe.fe_destroy(ctx)
