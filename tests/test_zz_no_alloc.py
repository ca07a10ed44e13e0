"""The allocation-free host-buffer apply, for callers that cannot let a
library allocate device memory (a memory manager that owns the whole GPU, a
real-time loop that must not block in the allocator, a fixed memory budget).

It must give the same result as the allocating fe_apply_host on two calls in
a row, on a structured mesh in every arithmetic mode that reads float or
double blocks and on a refined mesh with hanging nodes (whose product stages
a third block), and refuse blocks larger than its fixed staging array.  Below
the pipelining threshold both calls run one fe_apply over the whole block, so
the results must agree bit for bit.  Collected last on purpose."""
import numpy as np
import pytest

from paper_2208_07129_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fe():
    from paper_2208_07129_gb300 import build, fe as fe_mod
    build.build()
    fe_mod.lib()
    return fe_mod


def _dtype(mode):
    return torch.float64 if mode in ("fp64", "df64") else torch.float32


def _fits(n_dofs, n_vec, elem, blocks, stage):
    b = n_dofs * n_vec * elem
    slot = (b + 255) // 256 * 256
    return (blocks - 1) * slot + b <= stage


def _same_twice(fe, ctx, mode, n_vec):
    n = fe.fe_num_dofs(ctx)
    for call, seed in enumerate((1, 2)):     # two calls in a row, different inputs
        X = torch.from_numpy(inputs.random_block(n, n_vec, "uniform", seed)).to(_dtype(mode)).pin_memory()
        Yref = torch.full_like(X, float("nan")).pin_memory()
        Y = torch.full_like(X, float("nan")).pin_memory()
        fe.fe_apply_host(ctx, X, Yref)
        fe.fe_apply_host_noalloc(ctx, X, Y)
        assert torch.isfinite(Y).all(), call
        assert torch.equal(Y, Yref), call


@pytest.mark.parametrize("mode", ["fp64", "fp32", "df64", "tf32"])
def test_noalloc_matches_apply_host_twice(fe, mode):
    w = inputs.WORKLOADS["c1"]
    ctx = fe.setup_workload(w)
    try:
        fe.fe_set_mode(ctx, mode)
        _same_twice(fe, ctx, mode, w.n_vec)
    finally:
        fe.fe_destroy(ctx)


@pytest.mark.parametrize("mode", ["fp64", "fp32"])
def test_noalloc_refined_mesh(fe, mode):
    """Hanging nodes: the distribute step's copy of X comes from the fixed
    array too (three blocks), never from cudaMalloc."""
    ctx = fe.fe_setup_refined(3, 3, 2, 3, 5, (1, 1, 0), (2, 2, 1))
    try:
        assert fe.fe_num_slaves(ctx) > 0
        fe.fe_set_mode(ctx, mode)
        _same_twice(fe, ctx, mode, 6)
        # a block that fits as two slots but not as three is refused
        n, stage = fe.fe_num_dofs(ctx), fe.noalloc_stage_bytes()
        elem = 8 if mode == "fp64" else 4
        n_vec = next(k for k in range(1, 10 ** 6) if not _fits(n, k, elem, 3, stage))
        assert _fits(n, n_vec, elem, 2, stage)
        X = np.zeros((n, n_vec), dtype=np.float64 if mode == "fp64" else np.float32)
        with pytest.raises(fe.FeError) as ei:
            fe.fe_apply_host_noalloc(ctx, X, np.zeros_like(X))
        assert ei.value.status == fe.FE_EINVAL
    finally:
        fe.fe_destroy(ctx)


def test_noalloc_size_boundary(fe):
    """The largest block that fits runs and matches fe_apply_host; one more
    vector is refused with FE_EINVAL before any copy."""
    ctx = fe.fe_setup(4, 4, 4, 4, 6)
    try:
        n, stage = fe.fe_num_dofs(ctx), fe.noalloc_stage_bytes()
        assert stage == 16 << 20
        fit = max(k for k in range(1, stage // (8 * n) + 1) if _fits(n, k, 8, 2, stage))
        X = torch.from_numpy(inputs.random_block(n, fit, "uniform", 3)).pin_memory()
        Y = torch.full_like(X, float("nan")).pin_memory()
        Yref = torch.empty_like(X).pin_memory()
        fe.fe_apply_host_noalloc(ctx, X, Y)
        fe.fe_apply_host(ctx, X, Yref)
        # wide blocks are pipelined by fe_apply_host; every column keeps its arithmetic
        assert torch.equal(Y, Yref)
        Xbig = np.zeros((n, fit + 1))
        with pytest.raises(fe.FeError) as ei:
            fe.fe_apply_host_noalloc(ctx, Xbig, np.zeros_like(Xbig))
        assert ei.value.status == fe.FE_EINVAL
    finally:
        fe.fe_destroy(ctx)


def test_noalloc_rejects_bad_blocks(fe):
    """The binding refuses blocks the library would over-read or over-write."""
    ctx = fe.fe_setup(2, 2, 2, 2, 4)
    try:
        n = fe.fe_num_dofs(ctx)
        good = np.zeros((n, 4))
        for X, Y in ((good.astype(np.float32), good),          # wrong element type for FP64
                     (good, np.zeros((n - 1, 4))),             # Y too short
                     (good, np.zeros((n, 3))),                 # shapes differ
                     (np.zeros((4, n)).T, good)):              # not C-contiguous
            with pytest.raises(ValueError):
                fe.fe_apply_host_noalloc(ctx, X, Y)
            with pytest.raises(ValueError):
                fe.fe_apply_host(ctx, X, Y)
    finally:
        fe.fe_destroy(ctx)
