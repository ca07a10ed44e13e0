"""Python binding of libfe (include/fe.h).

The functions carry the C names and do argument marshalling only: every step
of the operator runs inside libfe's CUDA kernels.  Device buffers are torch
CUDA tensors (PyTorch provides memory and streams); host arrays are numpy.
The library must have been built (``paper_2208_07129_gb300.build``): there is
no fallback, and a missing or unloadable libfe.so raises immediately.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfe.so")

FE_OK, FE_EINVAL, FE_ENOMEM, FE_ECUDA, FE_ENOTCONV, FE_EBREAKDOWN, FE_ENONFINITE, FE_ETIMEOUT, FE_EUNSUPPORTED = range(9)
FE_BC_DIRICHLET0, FE_BC_PERIODIC = 0, 1
FE_QUAD_GAUSS, FE_QUAD_GLL = 0, 1
FE_FP64, FE_FP32, FE_TF32, FE_BF16, FE_TF32X3, FE_DF64, FE_BF16S = 0, 1, 2, 3, 4, 5, 6
MODES = {"fp64": FE_FP64, "fp32": FE_FP32, "tf32": FE_TF32, "bf16": FE_BF16, "tf32x3": FE_TF32X3, "df64": FE_DF64,
         "bf16s": FE_BF16S}


class FeError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        detail = ""
        if status in (2, 3):   # FE_ENOMEM, FE_ECUDA: name the CUDA runtime error behind it
            try:
                detail = f" [{lib().fe_last_cuda_error().decode()}]"
            except Exception:
                pass
        super().__init__(f"{what}: {status_str(status)} ({status}){detail}")


class fe_mesh_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("bc", ctypes.c_int), ("vertex_xyz", ctypes.POINTER(ctypes.c_double))]


class fe_solve_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("outer_iterations", ctypes.c_int), ("fp64_applies", ctypes.c_int),
                ("converged_columns", ctypes.c_int), ("max_rel_residual", ctypes.c_double),
                ("seconds", ctypes.c_double)]


FE_PRECOND_NONE, FE_PRECOND_JACOBI, FE_PRECOND_LEARNED = 0, 1, 2
PRECONDS = {"none": FE_PRECOND_NONE, "jacobi": FE_PRECOND_JACOBI, "learned": FE_PRECOND_LEARNED}


class fe_train_desc(ctypes.Structure):
    _fields_ = [("n_rhs", ctypes.c_int), ("snapshots", ctypes.c_int), ("snapshot_every", ctypes.c_int),
                ("epochs", ctypes.c_int), ("batch", ctypes.c_int), ("lr", ctypes.c_float),
                ("traj_rtol", ctypes.c_double), ("seed", ctypes.c_ulonglong), ("objective", ctypes.c_int),
                ("n_val", ctypes.c_int)]


FE_TRAIN_OPERATOR_RESIDUAL, FE_TRAIN_PATCH_ERROR, FE_TRAIN_ENERGY = 0, 1, 2
OBJECTIVES = {"operator": FE_TRAIN_OPERATOR_RESIDUAL, "patch_error": FE_TRAIN_PATCH_ERROR, "energy": FE_TRAIN_ENERGY}


class fe_train_info(ctypes.Structure):
    _fields_ = [("samples", ctypes.c_longlong), ("steps", ctypes.c_int), ("trajectory_iterations", ctypes.c_int),
                ("loss_first_step", ctypes.c_float), ("loss_first_epoch", ctypes.c_float),
                ("loss_last_epoch", ctypes.c_float), ("seconds", ctypes.c_double),
                ("val_jacobi_iterations", ctypes.c_int), ("val_learned_iterations", ctypes.c_int),
                ("best_epoch", ctypes.c_int), ("val_loss_jacobi", ctypes.c_float), ("val_loss_kept", ctypes.c_float)]


class fe_batch_info(ctypes.Structure):
    _fields_ = [("problems", ctypes.c_int), ("work_items", ctypes.c_int), ("phases", ctypes.c_int),
                ("grid", ctypes.c_int), ("smem_bytes", ctypes.c_longlong), ("autotune_ms", ctypes.c_float),
                ("device_status", ctypes.c_int)]


class fe_chfsi_desc(ctypes.Structure):
    _fields_ = [("n_wanted", ctypes.c_int), ("degree", ctypes.c_int), ("tol", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("lanczos_steps", ctypes.c_int), ("filter_mode", ctypes.c_int),
                ("fp32_switch", ctypes.c_double), ("seed", ctypes.c_ulonglong)]


class fe_chfsi_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("filter_applies", ctypes.c_int), ("fp32_passes", ctypes.c_int),
                ("converged", ctypes.c_int), ("max_residual", ctypes.c_double), ("lambda_min", ctypes.c_double),
                ("lambda_u", ctypes.c_double), ("lambda_max", ctypes.c_double), ("seconds", ctypes.c_double),
                ("seconds_filter", ctypes.c_double), ("seconds_orth", ctypes.c_double),
                ("seconds_rr", ctypes.c_double)]


class fe_refined_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("refine_lo", ctypes.c_int * 3), ("refine_hi", ctypes.c_int * 3)]


class fe_quad_desc(ctypes.Structure):
    _fields_ = [("n_q", ctypes.c_int), ("kind", ctypes.c_int)]


_lib = None
_VP = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)


def lib() -> ctypes.CDLL:
    """Load libfe.so (raises if it is missing: the product path has no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libfe.so not built at {LIB_PATH}; run paper_2208_07129_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "fe_setup": (ctypes.c_int, [ctypes.POINTER(fe_mesh_desc), ctypes.c_int, ctypes.POINTER(fe_quad_desc),
                                    ctypes.c_double, ctypes.POINTER(_VP)]),
        "fe_destroy": (None, [_VP]),
        "fe_num_dofs": (ctypes.c_size_t, [_VP]),
        "fe_num_cells": (ctypes.c_size_t, [_VP]),
        "fe_num_quad_points_1d": (ctypes.c_int, [_VP]),
        "fe_quadrature_points": (ctypes.c_int, [_VP, _DP]),
        "fe_set_potential": (ctypes.c_int, [_VP, _DP]),
        "fe_set_mode": (ctypes.c_int, [_VP, ctypes.c_int]),
        "fe_get_mode": (ctypes.c_int, [_VP]),
        "fe_apply": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, _VP]),
        "fe_apply_host": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, _VP]),
        "fe_apply_host_noalloc": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, _VP]),
        "fe_noalloc_stage_bytes": (ctypes.c_size_t, []),
        "fe_diagonal": (ctypes.c_int, [_VP, _VP, _VP]),
        "fe_last_device_status": (ctypes.c_int, [_VP]),
        "fe_solve": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, ctypes.POINTER(fe_solve_info), _DP, _VP]),
        "fe_status_str": (ctypes.c_char_p, [ctypes.c_int]),
        "fe_last_cuda_error": (ctypes.c_char_p, []),
        "fe_set_tile": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
        "fe_precond_init": (ctypes.c_int, [_VP, ctypes.c_ulonglong]),
        "fe_batch_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                           ctypes.c_int, ctypes.c_int, ctypes.POINTER(_VP)]),
        "fe_batch_apply": (ctypes.c_int, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), _VP]),
        "fe_batch_stats": (ctypes.c_int, [_VP, ctypes.POINTER(fe_batch_info), ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int)]),
        "fe_batch_destroy": (None, [_VP]),
        "fe_batch_set_wait_limit": (ctypes.c_int, [_VP, ctypes.c_double]),
        "fe_batch_hold_color": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
        "fe_precond_train": (ctypes.c_int, [_VP, ctypes.POINTER(fe_train_desc), ctypes.POINTER(fe_train_info), _VP]),
        "fe_precond_apply": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, _VP]),
        "fe_precond_set_weights": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
        "fe_precond_get_weights": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
        "fe_precond_input_size": (ctypes.c_int, [_VP]),
        "fe_precond_save": (ctypes.c_int, [_VP, ctypes.c_char_p]),
        "fe_precond_load": (ctypes.c_int, [_VP, ctypes.c_char_p]),
        "fe_mlp_gradients": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, _VP, _VP, _VP, _VP, _VP, _VP]),
        "fe_energy_gradients": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int, _VP, _VP, _VP, _VP, _VP, _VP]),
        "fe_mass_gll": (ctypes.c_int, [_VP, _DP]),
        "fe_setup_refined": (ctypes.c_int, [ctypes.POINTER(fe_refined_desc), ctypes.c_int,
                                            ctypes.POINTER(fe_quad_desc), ctypes.c_double, ctypes.POINTER(_VP)]),
        "fe_num_slaves": (ctypes.c_int, [_VP]),
        "fe_node_coords": (ctypes.c_int, [_VP, _DP]),
        "fe_apply_scaled": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, _VP]),
        "fe_chebyshev_filter": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_double, _VP]),
        "fe_chfsi": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.POINTER(fe_chfsi_desc), _DP, _DP,
                                    ctypes.POINTER(fe_chfsi_info), _VP]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def status_str(s: int) -> str:
    try:
        return lib().fe_status_str(int(s)).decode()
    except Exception:
        return "unknown"


def _check(status: int, what: str):
    if status != FE_OK:
        raise FeError(status, what)


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def fe_setup(nx: int, ny: int, nz: int, p: int, n_q: int, *, periodic: bool = False,
             lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), vertices: Optional[np.ndarray] = None,
             quad: int = FE_QUAD_GAUSS, mu: float = 0.5) -> int:
    md = fe_mesh_desc()
    md.nx, md.ny, md.nz = nx, ny, nz
    for d in range(3):
        md.lo[d] = float(lo[d])
        md.hi[d] = float(hi[d])
    md.bc = FE_BC_PERIODIC if periodic else FE_BC_DIRICHLET0
    keep = None
    if vertices is not None:
        keep = np.ascontiguousarray(vertices, dtype=np.float64)
        if keep.size != (nx + 1) * (ny + 1) * (nz + 1) * 3:
            raise ValueError("vertices must hold (nx+1)(ny+1)(nz+1) x 3 coordinates")
        md.vertex_xyz = keep.ctypes.data_as(_DP)
    qd = fe_quad_desc(n_q, quad)
    out = _VP()
    _check(lib().fe_setup(ctypes.byref(md), p, ctypes.byref(qd), mu, ctypes.byref(out)), "fe_setup")
    return out.value


def fe_setup_refined(nx: int, ny: int, nz: int, p: int, n_q: int, refine_lo, refine_hi, *,
                     lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), quad: int = FE_QUAD_GAUSS, mu: float = 0.5) -> int:
    """One-level refined Dirichlet box with hanging nodes (include/fe.h)."""
    d = fe_refined_desc()
    d.nx, d.ny, d.nz = nx, ny, nz
    for k in range(3):
        d.lo[k], d.hi[k] = float(lo[k]), float(hi[k])
        d.refine_lo[k], d.refine_hi[k] = int(refine_lo[k]), int(refine_hi[k])
    q = fe_quad_desc(n_q, quad)
    out = _VP()
    _check(lib().fe_setup_refined(ctypes.byref(d), p, ctypes.byref(q), mu, ctypes.byref(out)), "fe_setup_refined")
    return out.value


def fe_num_slaves(ctx: int) -> int:
    return int(lib().fe_num_slaves(ctx))


def fe_node_coords(ctx: int) -> np.ndarray:
    xyz = np.zeros((fe_num_dofs(ctx), 3))
    _check(lib().fe_node_coords(ctx, xyz.ctypes.data_as(_DP)), "fe_node_coords")
    return xyz


def fe_destroy(ctx: int) -> None:
    lib().fe_destroy(ctx)


def fe_num_dofs(ctx: int) -> int:
    return int(lib().fe_num_dofs(ctx))


def fe_num_cells(ctx: int) -> int:
    return int(lib().fe_num_cells(ctx))


def fe_num_quad_points_1d(ctx: int) -> int:
    return int(lib().fe_num_quad_points_1d(ctx))


def fe_quadrature_points(ctx: int) -> np.ndarray:
    E, nq = fe_num_cells(ctx), fe_num_quad_points_1d(ctx)
    out = np.zeros((E, nq ** 3, 3))
    _check(lib().fe_quadrature_points(ctx, out.ctypes.data_as(_DP)), "fe_quadrature_points")
    return out


def fe_set_potential(ctx: int, Vq: Optional[np.ndarray]) -> None:
    if Vq is None:
        _check(lib().fe_set_potential(ctx, None), "fe_set_potential")
        return
    E, nq = fe_num_cells(ctx), fe_num_quad_points_1d(ctx)
    v = np.ascontiguousarray(Vq, dtype=np.float64).reshape(-1)
    if v.size != E * nq ** 3:
        raise ValueError("Vq must hold E * n_q^3 values")
    _check(lib().fe_set_potential(ctx, v.ctypes.data_as(_DP)), "fe_set_potential")


def fe_set_mode(ctx: int, mode) -> None:
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    _check(lib().fe_set_mode(ctx, m), "fe_set_mode")


def fe_set_tile(ctx: int, mode, vectors_per_cta: int, lines: int, variant: int = 0) -> None:
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    _check(lib().fe_set_tile(ctx, m, vectors_per_cta, lines, variant), "fe_set_tile")


def fe_get_mode(ctx: int) -> int:
    return int(lib().fe_get_mode(ctx))


def block_dtype(ctx: int):
    """torch dtype of the blocks of the context's current mode."""
    import torch
    mode = fe_get_mode(ctx)
    return torch.float64 if mode in (FE_FP64, FE_DF64) else torch.bfloat16 if mode == FE_BF16S else torch.float32


def _check_block(ctx: int, t, what: str):
    want = block_dtype(ctx)
    if not t.is_cuda or t.dtype != want or not t.is_contiguous() or t.dim() != 2 or t.shape[0] != fe_num_dofs(ctx):
        raise ValueError(f"{what}: need a contiguous CUDA {want} tensor of shape (num_dofs, n_vec)")


def fe_apply(ctx: int, X, Y, stream=None) -> None:
    """Y = A X on the device (torch tensors, DoF-major (num_dofs, n_vec))."""
    _check_block(ctx, X, "X")
    _check_block(ctx, Y, "Y")
    if X.shape != Y.shape:
        raise ValueError("X and Y must have the same shape")
    _check(lib().fe_apply(ctx, X.data_ptr(), Y.data_ptr(), X.shape[1], _stream_ptr(stream)), "fe_apply")


def _host_blocks(ctx: int, X, Y) -> int:
    """Check a pair of host blocks for the host-buffer applies and return
    n_vec: torch CPU tensors or numpy arrays of the context's element type
    (float64 in FE_FP64 / FE_DF64 mode, float32 otherwise), C-contiguous,
    2-D (num_dofs, n_vec), X and Y of the same shape.  The library reads and
    writes exactly num_dofs * n_vec elements through the raw pointers, so a
    mismatch here would be an out-of-bounds host access there."""
    import torch
    tdt = block_dtype(ctx)
    want = {torch.float64: np.float64, torch.float32: np.float32}.get(tdt)   # numpy has no bfloat16
    n = fe_num_dofs(ctx)
    shapes = []
    for a, nm in ((X, "X"), (Y, "Y")):
        if isinstance(a, torch.Tensor):
            ok = not a.is_cuda and a.dtype == tdt and a.is_contiguous()
        elif isinstance(a, np.ndarray):
            ok = want is not None and a.dtype == want and a.flags["C_CONTIGUOUS"]
        else:
            ok = False
        if not ok or a.ndim != 2 or a.shape[0] != n:
            raise ValueError(f"{nm}: need a C-contiguous host block of {tdt} of shape (num_dofs={n}, n_vec)")
        shapes.append(tuple(a.shape))
    if shapes[0] != shapes[1]:
        raise ValueError(f"X and Y must have the same shape, got {shapes[0]} and {shapes[1]}")
    return shapes[0][1]


def _host_ptr(a) -> int:
    import torch
    return a.data_ptr() if isinstance(a, torch.Tensor) else a.ctypes.data


def fe_apply_host(ctx: int, X, Y, stream=None) -> None:
    """Y = A X with host buffers (pinned torch CPU tensors or numpy arrays)."""
    n_vec = _host_blocks(ctx, X, Y)
    _check(lib().fe_apply_host(ctx, _host_ptr(X), _host_ptr(Y), n_vec, _stream_ptr(stream)), "fe_apply_host")


def noalloc_stage_bytes() -> int:
    """Size of the fixed device staging array of fe_apply_host_noalloc, as
    compiled into the library."""
    return int(lib().fe_noalloc_stage_bytes())


def fe_apply_host_noalloc(ctx: int, X, Y, stream=None) -> None:
    """fe_apply_host without any device allocation by the library: the
    staging lives in a fixed device array of noalloc_stage_bytes() (for
    callers that cannot let a library allocate device memory).  Overlapping
    calls race."""
    n_vec = _host_blocks(ctx, X, Y)
    _check(lib().fe_apply_host_noalloc(ctx, _host_ptr(X), _host_ptr(Y), n_vec, _stream_ptr(stream)),
           "fe_apply_host_noalloc")


def fe_diagonal(ctx: int, diag, stream=None) -> None:
    import torch
    if not diag.is_cuda or diag.dtype != torch.float64 or diag.numel() != fe_num_dofs(ctx):
        raise ValueError("diag must be a CUDA float64 tensor with num_dofs entries")
    _check(lib().fe_diagonal(ctx, diag.data_ptr(), _stream_ptr(stream)), "fe_diagonal")


def fe_solve(ctx: int, B, X, rtol: float = 1e-8, max_it: int = 10000, precond="jacobi", inner_mode="fp64",
             stream=None) -> dict:
    """Block PCG for A X = B (FP64 torch tensors on the device; X = initial
    guess in, solution out).  Returns the solve info with the per-column FP64
    relative residuals; raises FeError unless the status is FE_OK or
    FE_ENOTCONV (reported in the result)."""
    import torch
    for t, nm in ((B, "B"), (X, "X")):
        if not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous() or t.shape[0] != fe_num_dofs(ctx):
            raise ValueError(f"{nm}: need a contiguous CUDA float64 tensor of shape (num_dofs, n_vec)")
    n_vec = B.shape[1]
    info = fe_solve_info()
    rel = np.zeros(n_vec)
    pc = PRECONDS[precond] if isinstance(precond, str) else int(precond)
    im = MODES[inner_mode] if isinstance(inner_mode, str) else int(inner_mode)
    st = lib().fe_solve(ctx, B.data_ptr(), X.data_ptr(), n_vec, rtol, max_it, pc, im, ctypes.byref(info),
                        rel.ctypes.data_as(_DP), _stream_ptr(stream))
    if st not in (FE_OK, FE_ENOTCONV):
        raise FeError(st, "fe_solve")
    return {"status": st, "iterations": info.iterations, "outer_iterations": info.outer_iterations,
            "fp64_applies": info.fp64_applies, "converged_columns": info.converged_columns,
            "max_rel_residual": info.max_rel_residual, "seconds": info.seconds, "rel_res": rel}


HIDDEN = 128


def fe_precond_input_size(ctx: int) -> int:
    return int(lib().fe_precond_input_size(ctx))


def fe_precond_init(ctx: int, seed: int = 0) -> None:
    _check(lib().fe_precond_init(ctx, seed), "fe_precond_init")


def fe_precond_set_weights(ctx: int, W1, b1, W2, b2) -> None:
    arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in (W1, b1, W2, b2)]
    n3 = fe_precond_input_size(ctx)
    if arrs[0].shape != (HIDDEN, n3) or arrs[1].shape != (HIDDEN,) or arrs[2].shape != (n3, HIDDEN) \
            or arrs[3].shape != (n3,):
        raise ValueError("weights must be W1 (128, n3), b1 (128,), W2 (n3, 128), b2 (n3,)")
    _check(lib().fe_precond_set_weights(ctx, *[a.ctypes.data for a in arrs]), "fe_precond_set_weights")


def fe_precond_get_weights(ctx: int):
    n3 = fe_precond_input_size(ctx)
    out = [np.zeros((HIDDEN, n3), np.float32), np.zeros(HIDDEN, np.float32), np.zeros((n3, HIDDEN), np.float32),
           np.zeros(n3, np.float32)]
    _check(lib().fe_precond_get_weights(ctx, *[a.ctypes.data for a in out]), "fe_precond_get_weights")
    return out


def fe_precond_train(ctx: int, n_rhs=8, snapshots=8, snapshot_every=25, epochs=4, batch=4096, lr=1e-3,
                     traj_rtol=1e-6, seed=0, objective="energy", n_val=4, stream=None) -> dict:
    d = fe_train_desc(n_rhs, snapshots, snapshot_every, epochs, batch, lr, traj_rtol, seed, OBJECTIVES[objective],
                      n_val)
    info = fe_train_info()
    _check(lib().fe_precond_train(ctx, ctypes.byref(d), ctypes.byref(info), _stream_ptr(stream)), "fe_precond_train")
    return {f: getattr(info, f) for f, _ in fe_train_info._fields_}


def fe_precond_apply(ctx: int, R, Z, stream=None) -> None:
    import torch
    for t, nm in ((R, "R"), (Z, "Z")):
        if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous() or t.shape[0] != fe_num_dofs(ctx):
            raise ValueError(f"{nm}: need a contiguous CUDA float32 tensor of shape (num_dofs, n_vec)")
    _check(lib().fe_precond_apply(ctx, R.data_ptr(), Z.data_ptr(), R.shape[1], _stream_ptr(stream)),
           "fe_precond_apply")


def fe_precond_save(ctx: int, path: str) -> None:
    _check(lib().fe_precond_save(ctx, path.encode()), "fe_precond_save")


def fe_precond_load(ctx: int, path: str) -> None:
    _check(lib().fe_precond_load(ctx, path.encode()), "fe_precond_load")


def fe_mlp_gradients(ctx: int, U, T, stream=None):
    """Loss and gradients of the training objective (device tensors in, torch tensors out)."""
    import torch
    n3 = fe_precond_input_size(ctx)
    dev = U.device
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    g = [torch.zeros(HIDDEN, n3, device=dev), torch.zeros(HIDDEN, device=dev), torch.zeros(n3, HIDDEN, device=dev),
         torch.zeros(n3, device=dev)]
    _check(lib().fe_mlp_gradients(ctx, U.data_ptr(), T.data_ptr(), U.shape[0], loss.data_ptr(),
                                  *[x.data_ptr() for x in g], _stream_ptr(stream)), "fe_mlp_gradients")
    return loss, g


def fe_energy_gradients(ctx: int, R, Xk, Xstar, stream=None):
    """Loss and gradients of the energy training objective on one snapshot
    (r_k, x_k, x*: CUDA float32 blocks (num_dofs, n_vec)); torch tensors out."""
    import torch
    for t, nm in ((R, "R"), (Xk, "Xk"), (Xstar, "Xstar")):
        if (not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous() or t.dim() != 2
                or t.shape != R.shape or t.shape[0] != fe_num_dofs(ctx)):
            raise ValueError(f"{nm}: need a contiguous CUDA float32 tensor of shape (num_dofs, n_vec)")
    n3 = fe_precond_input_size(ctx)
    dev = R.device
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    g = [torch.zeros(HIDDEN, n3, device=dev), torch.zeros(HIDDEN, device=dev), torch.zeros(n3, HIDDEN, device=dev),
         torch.zeros(n3, device=dev)]
    _check(lib().fe_energy_gradients(ctx, R.data_ptr(), Xk.data_ptr(), Xstar.data_ptr(), R.shape[1],
                                     loss.data_ptr(), *[x.data_ptr() for x in g], _stream_ptr(stream)),
           "fe_energy_gradients")
    return loss, g


def fe_batch_create(ctxs, n_vec, mode="fp64", autotune=True) -> int:
    n = len(ctxs)
    arr = (_VP * n)(*ctxs)
    nv = (ctypes.c_int * n)(*n_vec)
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    out = _VP()
    _check(lib().fe_batch_create(arr, n, nv, m, int(bool(autotune)), ctypes.byref(out)), "fe_batch_create")
    return out.value


def fe_batch_apply(batch: int, X, Y, stream=None) -> None:
    n = len(X)
    xs = (_VP * n)(*[t.data_ptr() for t in X])
    ys = (_VP * n)(*[t.data_ptr() for t in Y])
    _check(lib().fe_batch_apply(batch, xs, ys, _stream_ptr(stream)), "fe_batch_apply")


def fe_batch_stats(batch: int, n: int) -> dict:
    info = fe_batch_info()
    vb = (ctypes.c_int * n)()
    cb = (ctypes.c_int * n)()
    _check(lib().fe_batch_stats(batch, ctypes.byref(info), vb, cb), "fe_batch_stats")
    d = {f: getattr(info, f) for f, _ in fe_batch_info._fields_}
    d["vectors_per_cta"] = list(vb)
    d["cells_per_item"] = list(cb)
    return d


def fe_batch_set_wait_limit(batch: int, seconds: float) -> None:
    _check(lib().fe_batch_set_wait_limit(batch, float(seconds)), "fe_batch_set_wait_limit")


def fe_batch_hold_color(batch: int, problem: int, color: int, hold: bool) -> None:
    """Host-side fault injection for the bounded waits (see fe_batch.h)."""
    _check(lib().fe_batch_hold_color(batch, problem, color, int(bool(hold))), "fe_batch_hold_color")


def fe_batch_destroy(batch: int) -> None:
    lib().fe_batch_destroy(batch)


def fe_mass_gll(ctx: int) -> np.ndarray:
    """Diagonal of the GLL-integrated overlap matrix (host FP64; constrained rows 1)."""
    m = np.zeros(fe_num_dofs(ctx))
    _check(lib().fe_mass_gll(ctx, m.ctypes.data_as(_DP)), "fe_mass_gll")
    return m


def fe_apply_scaled(ctx: int, X, Y, a: float, b: float = 0.0, c: float = 0.0, stream=None) -> None:
    """Y = a M^-1/2 A M^-1/2 X + b X + c Y on the device (mode FP64 or FP32)."""
    _check_block(ctx, X, "X")
    _check_block(ctx, Y, "Y")
    if X.shape != Y.shape:
        raise ValueError("X and Y must have the same shape")
    _check(lib().fe_apply_scaled(ctx, X.data_ptr(), Y.data_ptr(), X.shape[1], float(a), float(b), float(c),
                                 _stream_ptr(stream)), "fe_apply_scaled")


def fe_chebyshev_filter(ctx: int, X, Y, degree: int, lambda_min: float, lambda_u: float, lambda_max: float,
                        stream=None) -> None:
    """X <- p_m(M^-1/2 A M^-1/2) X (Algorithm 6's filter); Y is scratch."""
    _check_block(ctx, X, "X")
    _check_block(ctx, Y, "Y")
    if X.shape != Y.shape:
        raise ValueError("X and Y must have the same shape")
    _check(lib().fe_chebyshev_filter(ctx, X.data_ptr(), Y.data_ptr(), X.shape[1], degree, lambda_min, lambda_u,
                                     lambda_max, _stream_ptr(stream)), "fe_chebyshev_filter")


def fe_chfsi(ctx: int, U, n_wanted: int, degree: int, tol: float, max_iter: int = 50, lanczos_steps: int = 20,
             filter_mode="fp64", fp32_switch: float = 0.0, seed: int = 1, stream=None) -> dict:
    """Chebyshev-filtered subspace iteration (Algorithm 6) on U (CUDA float64,
    (num_dofs, k)); returns the Ritz values, residuals and the run info.
    Raises unless the status is FE_OK or FE_ENOTCONV (reported)."""
    import torch
    if not U.is_cuda or U.dtype != torch.float64 or not U.is_contiguous() or U.dim() != 2 \
            or U.shape[0] != fe_num_dofs(ctx):
        raise ValueError("U: need a contiguous CUDA float64 tensor of shape (num_dofs, k)")
    k = U.shape[1]
    d = fe_chfsi_desc(n_wanted, degree, tol, max_iter, lanczos_steps, MODES[filter_mode], fp32_switch, seed)
    info = fe_chfsi_info()
    lam = np.zeros(k)
    res = np.zeros(k)
    st = lib().fe_chfsi(ctx, U.data_ptr(), k, ctypes.byref(d), lam.ctypes.data_as(_DP), res.ctypes.data_as(_DP),
                        ctypes.byref(info), _stream_ptr(stream))
    if st not in (FE_OK, FE_ENOTCONV):
        raise FeError(st, "fe_chfsi")
    out = {f: getattr(info, f) for f, _ in fe_chfsi_info._fields_}
    out.update(status=st, eigenvalues=lam, residuals=res)
    return out


def fe_last_device_status(ctx: int) -> int:
    return int(lib().fe_last_device_status(ctx))


def setup_workload(w, mu: Optional[float] = None) -> int:
    """fe_setup + fe_set_potential for an ``inputs.Workload`` (V evaluated at
    the library's own quadrature points)."""
    ctx = fe_setup(w.nx, w.ny, w.nz, w.p, w.nq, periodic=w.periodic, vertices=w.vertices(),
                   mu=w.mu if mu is None else mu)
    V = w.potential_at(fe_quadrature_points(ctx))
    if V is not None:
        fe_set_potential(ctx, V)
    return ctx
