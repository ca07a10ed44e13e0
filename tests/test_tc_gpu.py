"""The tcgen05 tensor-core cell kernel (FE_TF32, FE_BF16 and FE_BF16S with
BF16 storage) against the FP64 oracle, through the C ABI.

Every degree and quadrature size the kernel covers (n_p, n_q <= 8), Dirichlet
and periodic boxes (odd cell counts: three colours along a direction),
distorted trilinear cells (per-point metric), ragged vector tails, one cell,
one vector.  The same cases run through the warp-level MMA kernel
(fe_set_tile variant 1) as a cross-check, and through the tcgen05 kernel with
per-thread loads and stores (variant 2); variant 0 moves cell tiles with TMA
boxes and bulk reduce-adds wherever n_vec fills whole 16-byte units (the
n_vec = 8, 16, 24, 40 cases), else falls back to the thread path.  Inputs are rounded to the storage
type first and the oracle is applied to the rounded inputs, so the comparison
measures the arithmetic only.

Tolerances (relative Frobenius error and max element error / max |Y_ref|):
TF32 5e-3 and BF16 5e-2, the bounds of the warp-MMA kernel, whose measured
errors were 6.8e-4 - 1.5e-3 (TF32) and 2.5e-3 - 9.9e-3 (BF16).  BF16 storage
adds one rounding of every output to bfloat16 (2^-9 relative) and of every
colour-ordered partial sum (at most 8 per node); it is held to the BF16 bound.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2208_07129_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"tf32": 5e-3, "bf16": 5e-2, "bf16s": 5e-2}


@pytest.fixture(scope="module")
def fe():
    from paper_2208_07129_gb300 import build, fe as fe_mod
    build.build()
    fe_mod.lib()
    return fe_mod


def _pair(fe, nx, ny, nz, p, nq, periodic=False, distorted=False, quad=0, seed=0):
    verts = inputs.perturbed_vertices(nx, ny, nz, seed=31 + seed) if distorted else None
    ctx = fe.fe_setup(nx, ny, nz, p, nq, periodic=periodic, vertices=verts, quad=quad)
    mesh = orc.Mesh(nx, ny, nz, periodic=periodic, vertices=verts)
    fe.fe_set_potential(ctx, inputs.gaussian_potential(fe.fe_quadrature_points(ctx), 200 + seed, periodic))
    Vo = inputs.gaussian_potential(orc.quad_points(mesh, p, nq, quad), 200 + seed, periodic)
    return ctx, mesh, Vo


def _apply(fe, ctx, X, mode):
    fe.fe_set_mode(ctx, mode)
    dt = fe.block_dtype(ctx)
    Xd = torch.from_numpy(X).to(device="cuda", dtype=dt).contiguous()
    Yd = torch.full_like(Xd, float("nan"))
    fe.fe_apply(ctx, Xd, Yd)
    torch.cuda.synchronize()
    return Yd.double().cpu().numpy(), Xd.double().cpu().numpy()


def _compare(Y, Yref, tol):
    assert np.all(np.isfinite(Y))
    rel = np.linalg.norm(Y - Yref) / np.linalg.norm(Yref)
    err = np.abs(Y - Yref).max() / np.abs(Yref).max()
    assert rel <= tol and err <= tol, (rel, err)
    return rel, err


CASES = [
    # (nx, ny, nz, p, nq, periodic, distorted, quad, n_vec)
    (4, 4, 4, 4, 6, False, False, 0, 8),      # the 4^3 p=4 workload
    (3, 2, 3, 6, 8, True, False, 0, 13),      # periodic p=6 (the 32^3 workload's shape), 3 colours, ragged tail
    (2, 3, 2, 6, 8, False, True, 0, 21),      # distorted p=6: per-point metric
    (3, 3, 2, 1, 2, False, False, 0, 1),      # p=1, one vector
    (2, 2, 3, 3, 4, True, False, 1, 7),       # GLL rule, n_q = n_p
    (2, 3, 2, 5, 8, False, True, 0, 33),      # n_q = n_p + 2, distorted, several vector blocks + tail
    (2, 2, 2, 7, 8, True, False, 0, 16),      # p=7: n_p = n_q = 8, nothing padded
    (3, 2, 2, 2, 5, False, False, 0, 9),      # n_q = n_p + 2 at p=2
    (1, 1, 1, 2, 4, False, False, 0, 3),      # one cell
    (4, 3, 5, 3, 5, True, True, 0, 8),        # periodic and distorted together, odd counts
    (3, 3, 3, 6, 8, False, False, 0, 24),     # Dirichlet p=6, n_q = 8 (the n_q = E kernel), 3 vector blocks
    (3, 2, 3, 6, 8, True, True, 0, 40),       # periodic seams along x/y/z, distorted, 5 vector blocks
    (2, 3, 3, 4, 5, True, False, 0, 12),      # FP32 storage: box with a half-empty last vector block
    (3, 2, 2, 1, 2, True, False, 0, 16),      # p=1 periodic: most of the box is guard and padding
]


def _case_id(c):
    return f"{c[0]}x{c[1]}x{c[2]}_p{c[3]}_q{c[4]}_{'per' if c[5] else 'dir'}{'_dist' if c[6] else ''}_nv{c[8]}"


@pytest.mark.parametrize("variant", [0, 1, 2], ids=["tcgen05", "warp_mma", "tcgen05_threads"])
@pytest.mark.parametrize("mode", ["tf32", "bf16", "bf16s"])
@pytest.mark.parametrize("case", CASES, ids=_case_id)
def test_tc_matches_oracle(fe, case, mode, variant):
    nx, ny, nz, p, nq, periodic, distorted, quad, n_vec = case
    if mode == "bf16s" and variant == 1:
        pytest.skip("BF16 storage runs on the tcgen05 kernel only")
    ctx, mesh, Vo = _pair(fe, nx, ny, nz, p, nq, periodic, distorted, quad, seed=p)
    try:
        fe.fe_set_tile(ctx, mode, 8, 8, variant)
        X = inputs.random_block(fe.fe_num_dofs(ctx), n_vec, "uniform", seed=11 + p)
        Y, Xr = _apply(fe, ctx, X, mode)
        Yref = orc.apply(mesh, p, nq, Xr, kind=quad, Vq=Vo)
        rel, err = _compare(Y, Yref, TOL[mode])
        print(f"{mode} v{variant} rel {rel:.3e} max {err:.3e}")
    finally:
        fe.fe_destroy(ctx)


def test_tc_dirichlet_rows_deterministic_and_inputs_ignored(fe):
    """Boundary rows of Y are written 0 and boundary entries of X are ignored;
    two applies agree bit for bit (colour-ordered assembly, fixed order of
    every sum on the tensor cores)."""
    ctx, mesh, Vo = _pair(fe, 3, 2, 2, 6, 8)
    try:
        n = fe.fe_num_dofs(ctx)
        mask = orc.constrained_mask(mesh, 6)
        for mode in ("tf32", "bf16", "bf16s"):
            fe.fe_set_mode(ctx, mode)
            X = torch.from_numpy(inputs.random_block(n, 24, "normal", 4)).to(device="cuda", dtype=fe.block_dtype(ctx))
            X2 = X.clone()
            X2[torch.from_numpy(mask).cuda()] = 1e3
            Y1, Y2, Y3 = (torch.full_like(X, float("nan")) for _ in range(3))
            fe.fe_apply(ctx, X, Y1)
            fe.fe_apply(ctx, X, Y2)
            fe.fe_apply(ctx, X2, Y3)
            torch.cuda.synchronize()
            assert torch.equal(Y1, Y2), mode
            assert torch.equal(Y1, Y3), mode
            assert torch.all(Y1[torch.from_numpy(mask).cuda()] == 0), mode
    finally:
        fe.fe_destroy(ctx)


def test_tc_many_tasks_per_cta(fe):
    """More tasks than resident CTAs: every persistent CTA loops over several
    (cell, vector block) tasks and carries its barrier phase across them."""
    ctx, mesh, Vo = _pair(fe, 10, 10, 10, 3, 5, periodic=True, seed=5)
    try:
        n = fe.fe_num_dofs(ctx)
        X = inputs.random_block(n, 40, "uniform", 8)
        rows = np.random.default_rng(0).choice(n, 400, replace=False)
        ref = orc.apply_rows(mesh, 3, 5, X.astype(np.float32).astype(np.float64), rows, Vq=Vo)
        for mode in ("tf32", "bf16"):
            Y, _ = _apply(fe, ctx, X, mode)
            _compare(Y[rows], ref, TOL[mode])
    finally:
        fe.fe_destroy(ctx)


def test_tc_unsupported_shapes(fe):
    """BF16 storage needs the tcgen05 kernel (n_p, n_q <= 8); FE_TF32 and
    FE_BF16 fall back to the warp-MMA kernel there; variant 3 is invalid, and
    so is the warp-MMA kernel for BF16 storage."""
    ctx = fe.fe_setup(2, 2, 2, 8, 10)
    try:
        fe.fe_set_mode(ctx, "bf16s")
        X = torch.zeros(fe.fe_num_dofs(ctx), 8, dtype=torch.bfloat16, device="cuda")
        with pytest.raises(fe.FeError) as ei:
            fe.fe_apply(ctx, X, torch.empty_like(X))
        assert ei.value.status == fe.FE_EUNSUPPORTED
        with pytest.raises(fe.FeError):
            fe.fe_set_tile(ctx, "tf32", 8, 8, 3)
        with pytest.raises(fe.FeError):
            fe.fe_set_tile(ctx, "bf16s", 8, 8, 1)
    finally:
        fe.fe_destroy(ctx)


@pytest.mark.parametrize("mode", ["tf32", "bf16", "bf16s"])
def test_tc_tma_path_equals_thread_path(fe, mode):
    """The TMA boxes with bulk reduce-adds and the per-thread loads and stores
    form every node's sum in the same order (Y starts at zero, colours run in
    order, and the first colour's store equals 0 + its value), so FP32
    storage gives bitwise the same Y.  BF16 storage rounds each colour's
    contribution to bfloat16 before the reduce adds it, the thread path adds
    it in FP32 and rounds the sum once: the two differ by a few bfloat16
    roundings of the partial sums (at most 8 per node).  Dirichlet and periodic boxes, several vector blocks,
    unaligned blocks (which take the thread path under variant 0 too)."""
    for periodic in (False, True):
        ctx, mesh, Vo = _pair(fe, 3, 4, 3, 6, 8, periodic=periodic, seed=9)
        try:
            fe.fe_set_mode(ctx, mode)
            n = fe.fe_num_dofs(ctx)
            X = torch.from_numpy(inputs.random_block(n, 32, "normal", 5)).to(device="cuda", dtype=fe.block_dtype(ctx))
            Ys = []
            for variant in (0, 2, 0):
                fe.fe_set_tile(ctx, mode, 8, 8, variant)
                Y = torch.full_like(X, float("nan"))
                fe.fe_apply(ctx, X, Y)
                Ys.append(Y)
            torch.cuda.synchronize()
            assert torch.equal(Ys[0], Ys[2])      # deterministic
            if mode == "bf16s":
                d = (Ys[0].double() - Ys[1].double()).abs().max().item()
                assert d <= 2.0 ** -5 * Ys[1].double().abs().max().item(), d
            else:
                assert torch.equal(Ys[0], Ys[1])
            # an unaligned block (offset by one element) takes the thread path
            base = torch.empty(n * 32 + 8, dtype=X.dtype, device="cuda")
            Xu = base[1:1 + n * 32].view(n, 32)
            Xu.copy_(X)
            Yu_base = torch.full_like(base, float("nan"))
            Yu = Yu_base[1:1 + n * 32].view(n, 32)
            fe.fe_set_tile(ctx, mode, 8, 8, 0)
            fe.fe_apply(ctx, Xu, Yu)
            torch.cuda.synchronize()
            assert torch.equal(Yu, Ys[1])
        finally:
            fe.fe_destroy(ctx)
