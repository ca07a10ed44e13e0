"""The allocation-free host-buffer apply, for callers that cannot let a
library allocate device memory (a memory manager that owns the whole GPU, a
real-time loop, a fixed memory budget).  It must give the same result as the
allocating fe_apply_host on two calls in a row, and refuse blocks larger than
its fixed staging array.  Collected last on purpose."""
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


@pytest.mark.parametrize("mode,tol", [("fp64", 1e-12), ("fp32", 2e-6)])
def test_noalloc_matches_apply_host_twice(fe, mode, tol):
    w = inputs.WORKLOADS["c1"]
    ctx = fe.setup_workload(w)
    try:
        fe.fe_set_mode(ctx, mode)
        dt = torch.float64 if mode == "fp64" else torch.float32
        for call, seed in enumerate((1, 2)):     # two calls in a row, different inputs
            X = torch.from_numpy(w.make_x(seed=seed)).to(dt).pin_memory()
            Yref = torch.empty_like(X).pin_memory()
            Y = torch.full_like(X, float("nan")).pin_memory()
            fe.fe_apply_host(ctx, X, Yref)
            fe.fe_apply_host_noalloc(ctx, X, Y)
            a, b = Y.double().numpy(), Yref.double().numpy()
            assert np.all(np.isfinite(a))
            assert np.linalg.norm(a - b) <= tol * np.linalg.norm(b), call
            assert np.abs(a - b).max() <= tol * np.abs(b).max(), call
    finally:
        fe.fe_destroy(ctx)


def test_noalloc_rejects_oversize(fe):
    ctx = fe.fe_setup(4, 4, 4, 4, 6)
    try:
        n = fe.fe_num_dofs(ctx)
        n_vec = fe.NOALLOC_STAGE_BYTES // (2 * 8 * n) + 1    # X and Y no longer fit
        X = np.zeros((n, n_vec))
        Y = np.zeros_like(X)
        with pytest.raises(fe.FeError) as ei:
            fe.fe_apply_host_noalloc(ctx, X, Y)
        assert ei.value.status == fe.FE_EINVAL
    finally:
        fe.fe_destroy(ctx)
