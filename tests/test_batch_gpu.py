"""Batched persistent launch (CUDA graph) over uneven problems: every output
equals the per-problem fe_apply bit for bit, and a sample matches the FP64
oracle."""
import numpy as np
import pytest

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


PROBLEMS = [  # (n, p, n_vec, periodic)
    (3, 3, 5, True), (2, 8, 17, False), (4, 4, 40, True), (3, 6, 8, True), (5, 5, 3, False), (2, 7, 64, True),
    (3, 3, 1, False),
]


@pytest.mark.parametrize("mode", ["fp64", "df64", "fp32"])
@pytest.mark.parametrize("autotune", [False, True])
def test_batch_matches_per_problem(fe, mode, autotune):
    ctxs, Xs, Ys, Yref = [], [], [], []
    dt = torch.float64 if mode in ("fp64", "df64") else torch.float32
    try:
        for k, (n, p, nv, per) in enumerate(PROBLEMS):
            w = inputs.Workload(f"b{k}", n, n, n, per, p, p + 2, nv, "normal", 40 + k, "gauss", v_seed=140 + k)
            ctx = fe.setup_workload(w)
            ctxs.append(ctx)
            X = torch.from_numpy(w.make_x()).to(device="cuda", dtype=dt)
            Xs.append(X)
            Ys.append(torch.full_like(X, float("nan")))
            fe.fe_set_mode(ctx, mode)   # default kernel: the even-odd line kernel, whose cell body the batch runs
            Y = torch.empty_like(X)
            fe.fe_apply(ctx, X, Y)
            Yref.append(Y)
        b = fe.fe_batch_create(ctxs, [P[2] for P in PROBLEMS], mode=mode, autotune=autotune)
        try:
            for rep in range(2):                      # graph replay twice
                for Y in Ys:
                    Y.fill_(float("nan"))
                fe.fe_batch_apply(b, Xs, Ys)
                torch.cuda.synchronize()
                for Y, R in zip(Ys, Yref):
                    assert torch.equal(Y, R)
            st = fe.fe_batch_stats(b, len(PROBLEMS))
            assert st["device_status"] == 0 and st["work_items"] > 0 and st["phases"] >= 8
        finally:
            fe.fe_batch_destroy(b)
        # one problem against the oracle
        n, p, nv, per = PROBLEMS[1]
        w = inputs.Workload("b1", n, n, n, per, p, p + 2, nv, "normal", 41, "gauss", v_seed=141)
        mesh = orc.Mesh(n, n, n, periodic=per)
        Vo = w.potential_at(orc.quad_points(mesh, p, p + 2))
        ref = orc.apply(mesh, p, p + 2, Xs[1].double().cpu().numpy(), Vq=Vo)
        got = Ys[1].double().cpu().numpy()
        tol = 2e-6 if mode == "fp32" else 1e-12
        assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)
    finally:
        for c in ctxs:
            fe.fe_destroy(c)


def test_batch_rejects_unsupported(fe):
    ctx = fe.fe_setup(2, 2, 2, 2, 4)
    try:
        with pytest.raises(fe.FeError):
            fe.fe_batch_create([ctx], [4])            # p = 2 is outside the batch kinds
    finally:
        fe.fe_destroy(ctx)


def test_bounded_wait_runs_out_and_recovers(fe):
    """A colour whose completion count can never be reached (injected on the
    host) makes the next colour's waits run out after the wait limit: the
    launch ends, the status word reports FE_ETIMEOUT, and after the count is
    restored the same batch gives the per-problem results again."""
    ctxs, Xs, Ys, Yref = [], [], [], []
    try:
        for k, (n, p, nv, per) in enumerate([(3, 3, 5, True), (2, 4, 8, False)]):
            w = inputs.Workload(f"t{k}", n, n, n, per, p, p + 2, nv, "normal", 60 + k, "gauss", v_seed=160 + k)
            ctx = fe.setup_workload(w)
            ctxs.append(ctx)
            X = torch.from_numpy(w.make_x()).cuda()
            Xs.append(X)
            Ys.append(torch.empty_like(X))
            Y = torch.empty_like(X)
            fe.fe_apply(ctx, X, Y)
            Yref.append(Y)
        b = fe.fe_batch_create(ctxs, [5, 8], mode="fp64", autotune=False)
        try:
            fe.fe_batch_set_wait_limit(b, 0.02)
            fe.fe_batch_hold_color(b, 0, 0, True)
            fe.fe_batch_apply(b, Xs, Ys)
            torch.cuda.synchronize()
            assert fe.fe_batch_stats(b, 2)["device_status"] == fe.FE_ETIMEOUT
            fe.fe_batch_hold_color(b, 0, 0, False)
            fe.fe_batch_apply(b, Xs, Ys)
            torch.cuda.synchronize()
            assert fe.fe_batch_stats(b, 2)["device_status"] == 0
            for Y, R in zip(Ys, Yref):
                assert torch.equal(Y, R)
            with pytest.raises(fe.FeError):
                fe.fe_batch_hold_color(b, 5, 0, True)     # no such problem
        finally:
            fe.fe_batch_destroy(b)
    finally:
        for c in ctxs:
            fe.fe_destroy(c)
