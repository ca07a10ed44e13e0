"""Learned cell-patch preconditioner through the C ABI: training gradients
against the FP64 numpy oracle, the tensor-core inference kernel against the
oracle (with the same bfloat16 roundings), save/load, and what the trained
network gains over Jacobi inside the mixed-precision block-PCG solve."""
import os

import numpy as np
import pytest

from oracle import mlp_oracle as mo
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


def _weights(n3, seed, scale=0.2):
    rng = np.random.default_rng(seed)
    return (rng.normal(0, scale, (128, n3)).astype(np.float32), rng.normal(0, 0.1, 128).astype(np.float32),
            rng.normal(0, scale, (n3, 128)).astype(np.float32), rng.normal(0, 0.1, n3).astype(np.float32))


def test_gradients_match_oracle(fe):
    ctx = fe.fe_setup(2, 2, 2, 3, 5)
    try:
        n3 = fe.fe_precond_input_size(ctx)
        W = _weights(n3, 0)
        fe.fe_precond_set_weights(ctx, *W)
        rng = np.random.default_rng(1)
        U = rng.normal(size=(300, n3)).astype(np.float32)
        T = rng.normal(size=(300, n3)).astype(np.float32)
        loss, g = fe.fe_mlp_gradients(ctx, torch.from_numpy(U).cuda(), torch.from_numpy(T).cuda())
        ref = mo.loss_and_grads(*[w.astype(np.float64) for w in W], U.astype(np.float64), T.astype(np.float64))
        assert abs(loss.item() - ref[0]) <= 1e-5 * ref[0]
        for got, want in zip(g, ref[1:]):
            got = got.cpu().numpy()
            assert np.linalg.norm(got - want) <= 1e-4 * np.linalg.norm(want)
    finally:
        fe.fe_destroy(ctx)


@pytest.mark.parametrize("p,nx,periodic", [(3, 2, False), (2, 3, True)])
def test_energy_gradients_match_oracle(fe, p, nx, periodic):
    """The objective training actually uses (energy norm of what the
    preconditioner misses, operator in the loop, patch scale s_e, partition
    weights) against the FP64 oracle, through the C ABI."""
    nq = p + 2
    ctx = fe.fe_setup(nx, nx, nx, p, nq, periodic=periodic)
    mesh = orc.Mesh(nx, nx, nx, periodic=periodic)
    try:
        n, n3, nv = fe.fe_num_dofs(ctx), (p + 1) ** 3, 12
        V = np.full(mesh.num_cells * nq ** 3, 0.7)
        fe.fe_set_potential(ctx, V)
        A = orc.assemble(mesh, p, nq, Vq=V)
        W = _weights(n3, 10 + p)
        fe.fe_precond_set_weights(ctx, *W)
        rng = np.random.default_rng(p)
        con = orc.constrained_mask(mesh, p)
        xs, xk = rng.normal(size=(n, nv)), rng.normal(size=(n, nv))
        xs[con] = 0.0
        xk[con] = 0.0
        xs, xk = xs.astype(np.float32), xk.astype(np.float32)
        r = (A @ (xs.astype(np.float64) - xk)).astype(np.float32)
        d = torch.empty(n, dtype=torch.float64, device="cuda")
        fe.fe_diagonal(ctx, d)
        dinv = (1.0 / d.cpu().numpy()).astype(np.float32).astype(np.float64)
        loss, g = fe.fe_energy_gradients(ctx, *[torch.from_numpy(a).cuda() for a in (r, xk, xs)])
        ref = mo.energy_loss_and_grads(mesh, p, A, dinv, *[w.astype(np.float64) for w in W],
                                       r.astype(np.float64), xk.astype(np.float64), xs.astype(np.float64))
        assert abs(loss.item() - ref[0]) <= 1e-4 * ref[0], (loss.item(), ref[0])
        for got, want in zip(g, ref[1:]):
            got = got.cpu().numpy()
            assert np.linalg.norm(got - want) <= 1e-4 * np.linalg.norm(want)
    finally:
        fe.fe_destroy(ctx)


@pytest.mark.parametrize("p,nv,periodic", [(3, 128, False), (6, 130, False), (4, 40, True)])
def test_inference_matches_oracle(fe, p, nv, periodic):
    nx = 3 if p < 6 else 2
    ctx = fe.fe_setup(nx, nx, nx, p, p + 2, periodic=periodic)
    mesh = orc.Mesh(nx, nx, nx, periodic=periodic)
    try:
        n = fe.fe_num_dofs(ctx)
        n3 = (p + 1) ** 3
        W = _weights(n3, p)
        fe.fe_precond_set_weights(ctx, *W)
        r = inputs.random_block(n, nv, "normal", 3).astype(np.float32)
        r[orc.constrained_mask(mesh, p)] = 0
        Z = torch.empty(n, nv, dtype=torch.float32, device="cuda")
        fe.fe_precond_apply(ctx, torch.from_numpy(r).cuda(), Z)
        torch.cuda.synchronize()
        d = torch.empty(n, dtype=torch.float64, device="cuda")
        fe.fe_diagonal(ctx, d)
        dinv = (1.0 / d.cpu().numpy()).astype(np.float32).astype(np.float64)
        ref = mo.precond(mesh, p, r.astype(np.float64), dinv, *[w.astype(np.float64) for w in W], bf16=True)
        got = Z.cpu().numpy().astype(np.float64)
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert rel < 2e-3, rel
        assert np.abs(got - ref).max() < 2e-2 * np.abs(ref).max()
    finally:
        fe.fe_destroy(ctx)


def test_save_load_roundtrip(fe, tmp_path):
    ctx = fe.fe_setup(2, 2, 2, 3, 5)
    ctx2 = fe.fe_setup(2, 2, 2, 3, 5)
    try:
        fe.fe_precond_init(ctx, seed=5)
        path = str(tmp_path / "w.bin")
        fe.fe_precond_save(ctx, path)
        fe.fe_precond_load(ctx2, path)
        for a, b in zip(fe.fe_precond_get_weights(ctx), fe.fe_precond_get_weights(ctx2)):
            assert np.array_equal(a, b)
        ctx3 = fe.fe_setup(2, 2, 2, 4, 6)
        with pytest.raises(fe.FeError):
            fe.fe_precond_load(ctx3, path)   # n3 mismatch
        fe.fe_destroy(ctx3)
    finally:
        fe.fe_destroy(ctx)
        fe.fe_destroy(ctx2)


def test_training_gain_over_jacobi(fe):
    """Train on a 12^3, p=6 problem (V + sigma as in the block-PCG workload;
    energy-norm objective, checkpoint picked on held-out right-hand sides),
    then solve 16 fresh right-hand sides with the mixed-precision block PCG:
    Jacobi vs the learned preconditioner, both checked with the FP64 operator."""
    w = inputs.Workload("12^3 p=6", 12, 12, 12, False, 6, 8, 16, "normal", 77, "gauss", v_seed=15, v_amp=0.125,
                        v_shift=1.0)
    ctx = fe.setup_workload(w)
    try:
        info = fe.fe_precond_train(ctx, n_rhs=16, snapshots=16, snapshot_every=16, epochs=12, batch=2048, lr=3e-3,
                                   traj_rtol=1e-6, seed=3, objective="energy", n_val=4)
        assert info["samples"] > 0 and info["steps"] > 0
        assert info["loss_last_epoch"] < info["loss_first_epoch"]
        assert info["val_learned_iterations"] <= info["val_jacobi_iterations"]
        B = torch.from_numpy(w.make_rhs(16)).cuda()
        its = {}
        for pc in ("jacobi", "learned"):
            X = torch.zeros_like(B)
            r = fe.fe_solve(ctx, B, X, rtol=1e-8, max_it=20000, precond=pc, inner_mode="fp32")
            assert r["status"] == fe.FE_OK and r["max_rel_residual"] <= 1e-8
            assert np.all(r["rel_res"] <= 1e-8)
            its[pc] = r["iterations"]
        print("iterations", its, "train", info)
        # what the trained network gains over the same solver without it
        assert its["learned"] < its["jacobi"], its
    finally:
        fe.fe_destroy(ctx)


def test_checkpoint_never_worse_than_jacobi(fe):
    """The kept checkpoint is never worse than Jacobi on the held-out
    right-hand sides.  With no training epoch the only candidate is epoch 0,
    the network with a zero output layer, which is exactly Jacobi: the kept
    weights must have W2 = b2 = 0 and the learned solve must converge like
    Jacobi (the same preconditioner; the flexible-CG coefficient only changes
    the rounding).  After one real epoch the validation count may not exceed
    Jacobi's either."""
    w = inputs.Workload("4^3 p=4", 4, 4, 4, False, 4, 6, 8, "normal", 78, "gauss", v_seed=15, v_amp=0.125,
                        v_shift=1.0)
    ctx = fe.setup_workload(w)
    try:
        fe.fe_precond_init(ctx, seed=9)
        info = fe.fe_precond_train(ctx, n_rhs=8, snapshots=2, snapshot_every=5, epochs=0, batch=256, lr=1e-3,
                                   traj_rtol=1e-6, seed=5, objective="energy", n_val=4)
        assert info["best_epoch"] == 0
        assert info["val_learned_iterations"] == info["val_jacobi_iterations"]
        W1, b1, W2, b2 = fe.fe_precond_get_weights(ctx)
        assert not np.any(W2) and not np.any(b2)
        B = torch.from_numpy(w.make_rhs(8)).cuda()
        its = {}
        for pc in ("jacobi", "learned"):
            X = torch.zeros_like(B)
            r = fe.fe_solve(ctx, B, X, rtol=1e-8, max_it=20000, precond=pc, inner_mode="fp32")
            assert r["status"] == fe.FE_OK and r["max_rel_residual"] <= 1e-8
            its[pc] = r["iterations"]
        assert abs(its["learned"] - its["jacobi"]) <= max(2, its["jacobi"] // 50), its
        info = fe.fe_precond_train(ctx, n_rhs=8, snapshots=2, snapshot_every=5, epochs=1, batch=256, lr=1e-9,
                                   traj_rtol=1e-6, seed=5, objective="energy", n_val=4)
        assert info["val_learned_iterations"] <= info["val_jacobi_iterations"]
    finally:
        fe.fe_destroy(ctx)
