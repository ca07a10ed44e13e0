"""Seeded synthetic inputs for the matrix-free operator workloads.

This module holds no operator arithmetic: it only draws random multivectors,
perturbs mesh vertices and defines the potential V(x) as a plain function of
physical coordinates.  Both the CUDA path (through the library's own
quadrature points) and the FP64 oracle (through its own) evaluate V with the
functions here, so the two sides share nothing but their inputs.

Workloads (the paper measures on random multivectors over uniform meshes,
Sec. 4.1; the shapes below follow its FEOrder 4-8 cases):

* ``c1``  4^3 unit cube, p=4, 6-point Gauss, Dirichlet-0, n_vec=8,
          X ~ U[-1,1] (seed 1), V = -1/(|x-c|+0.5), c = (1/2,1/2,1/2).
* ``c2``  32^3 periodic unit box, p=6, n_q=8, n_vec=64, X ~ N(0,1) (seed 2),
          V = -sum of 8 Gaussians, centres U[0,1]^3, widths U[0.05,0.2]
          (seed 12), minimum-image distance.
* ``c3``  16^3 unit cube with interior vertices moved by U[-0.2h,0.2h]
          (seed 13), trilinear cells, p=8, n_q=10, n_vec=256, Dirichlet-0,
          X ~ U[-1,1] (seed 3), Gaussian V (seed 23, non-periodic distance).
* ``c4``  24 periodic problems, n ~ U{4..24}, p ~ U{3..8}, n_q = p+2,
          n_vec = round(exp(U[ln 8, ln 512])), Gaussian V; seeds 400+i.
* ``c5``  24^3 unit cube, p=6, n_q=8, Dirichlet-0, n_vec=128 right-hand
          sides B ~ N(0,1) (seed 5), V = Gaussians with amplitude 1/8
          (seed 15) shifted by sigma = 1 (so V + sigma >= 0).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    periodic: bool
    p: int
    nq: int
    n_vec: int
    x_dist: str = "uniform"
    x_seed: int = 0
    potential: str = "none"          # none | coulomb | gauss
    v_seed: int = 0
    v_amp: float = 1.0
    v_shift: float = 0.0
    perturb_seed: Optional[int] = None
    perturb_amp: float = 0.2
    mu: float = 0.5
    extra: dict = field(default_factory=dict)

    @property
    def num_cells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def num_dofs(self) -> int:
        add = 0 if self.periodic else 1
        return (self.nx * self.p + add) * (self.ny * self.p + add) * (self.nz * self.p + add)

    def vertices(self) -> Optional[np.ndarray]:
        if self.perturb_seed is None:
            return None
        return perturbed_vertices(self.nx, self.ny, self.nz, self.perturb_seed, self.perturb_amp)

    def potential_at(self, xyz: np.ndarray) -> Optional[np.ndarray]:
        """V at an (..., 3) array of physical points (None when V = 0)."""
        if self.potential == "none":
            v = None
        elif self.potential == "coulomb":
            v = coulomb_potential(xyz)
        elif self.potential == "gauss":
            v = gaussian_potential(xyz, self.v_seed, self.periodic, self.v_amp)
        else:
            raise ValueError(self.potential)
        if self.v_shift != 0.0:
            v = (np.zeros(xyz.shape[:-1]) if v is None else v) + self.v_shift
        return v

    def boundary_mask(self) -> np.ndarray:
        """True on the Dirichlet boundary nodes (all False for a periodic box)."""
        if self.periodic:
            return np.zeros(self.num_dofs, dtype=bool)
        N = [self.nx * self.p + 1, self.ny * self.p + 1, self.nz * self.p + 1]
        g = np.arange(self.num_dofs)
        gx, gy, gz = g % N[0], (g // N[0]) % N[1], g // (N[0] * N[1])
        return (gx == 0) | (gy == 0) | (gz == 0) | (gx == N[0] - 1) | (gy == N[1] - 1) | (gz == N[2] - 1)

    def make_rhs(self, n_vec: Optional[int] = None) -> np.ndarray:
        """Right-hand sides: the seeded block with its Dirichlet rows set to 0."""
        B = self.make_x(n_vec)
        B[self.boundary_mask()] = 0.0
        return B

    def make_x(self, n_vec: Optional[int] = None, seed: Optional[int] = None) -> np.ndarray:
        return random_block(self.num_dofs, self.n_vec if n_vec is None else n_vec,
                            self.x_dist, self.x_seed if seed is None else seed)


def random_block(n_dofs: int, n_vec: int, dist: str, seed: int) -> np.ndarray:
    """DoF-major, vector-contiguous block X[dof, v] (float64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if dist == "uniform":
        return rng.uniform(-1.0, 1.0, size=(n_dofs, n_vec))
    if dist == "normal":
        return rng.standard_normal(size=(n_dofs, n_vec))
    raise ValueError(dist)


def perturbed_vertices(nx: int, ny: int, nz: int, seed: int, amp: float = 0.2) -> np.ndarray:
    """Vertices of the unit cube's nx*ny*nz grid, interior ones moved by
    U[-amp h, amp h] per coordinate; shape ((nx+1)(ny+1)(nz+1), 3), x fastest."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gz, gy, gx = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    h = np.array([1.0 / nx, 1.0 / ny, 1.0 / nz])
    v = np.stack([gx * h[0], gy * h[1], gz * h[2]], axis=-1).reshape(-1, 3)
    interior = ((gx > 0) & (gx < nx) & (gy > 0) & (gy < ny) & (gz > 0) & (gz < nz)).reshape(-1)
    delta = rng.uniform(-amp, amp, size=v.shape) * h[None, :]
    v[interior] += delta[interior]
    return np.ascontiguousarray(v)


def coulomb_potential(xyz: np.ndarray, centre=(0.5, 0.5, 0.5)) -> np.ndarray:
    r = np.linalg.norm(xyz - np.asarray(centre), axis=-1)
    return -1.0 / (r + 0.5)


def gaussian_params(seed: int, count: int = 8):
    rng = np.random.Generator(np.random.PCG64(seed))
    centres = rng.uniform(0.0, 1.0, size=(count, 3))
    widths = rng.uniform(0.05, 0.2, size=count)
    return centres, widths


def gaussian_potential(xyz: np.ndarray, seed: int, periodic: bool, amp: float = 1.0) -> np.ndarray:
    centres, widths = gaussian_params(seed)
    out = np.zeros(xyz.shape[:-1])
    for c, s in zip(centres, widths):
        d = xyz - c
        if periodic:
            d = d - np.round(d)
        out -= amp * np.exp(-np.sum(d * d, axis=-1) / (2.0 * s * s))
    return out


WORKLOADS = {
    "c1": Workload("unit cube 4^3, p=4, 6-pt Gauss, Dirichlet-0, n_vec=8", 4, 4, 4, False, 4, 6, 8,
                   "uniform", 1, "coulomb"),
    "c2": Workload("periodic box 32^3, p=6, n_q=8, n_vec=64", 32, 32, 32, True, 6, 8, 64,
                   "normal", 2, "gauss", v_seed=12),
    "c3": Workload("perturbed 16^3 trilinear, p=8, n_q=10, Dirichlet-0, n_vec=256", 16, 16, 16, False, 8, 10, 256,
                   "uniform", 3, "gauss", v_seed=23, perturb_seed=13),
    # a smaller case of the same kernel for hardware-counter captures (inputs still above L2)
    "c2s": Workload("periodic box 12^3, p=6, n_q=8, n_vec=64", 12, 12, 12, True, 6, 8, 64,
                    "normal", 2, "gauss", v_seed=12),
    "c5": Workload("24^3 unit cube, p=6, n_q=8, Dirichlet-0, 128 right-hand sides", 24, 24, 24, False, 6, 8, 128,
                   "normal", 5, "gauss", v_seed=15, v_amp=0.125, v_shift=1.0),
    # eigenproblems (Sec. 4.3): n_vec is the subspace size k of the filtered subspace iteration
    "e0": Workload("unit cube 8^3, p=6, n_q=8, Dirichlet-0: 100 smallest eigenpairs, 128-vector subspace, "
                   "Chebyshev degree 40, residual 5e-5", 8, 8, 8, False, 6, 8, 128, "normal", 7, "gauss", v_seed=17,
                   extra={"n_wanted": 100, "degree": 40, "tol": 5e-5}),
    # the size of the paper's GPU eigen case for FEOrder 6 (1,092,727 DoFs, 1024 wanted + 25 % buffer,
    # Chebyshev degree 67)
    "e1": Workload("unit cube 17^3, p=6, n_q=8, Dirichlet-0 (1,092,727 DoFs): 1024 wanted eigenpairs, "
                   "1280-vector subspace, Chebyshev degree 67", 17, 17, 17, False, 6, 8, 1280, "normal", 8, "gauss",
                   v_seed=18, extra={"n_wanted": 1024, "degree": 67, "tol": 5e-5}),
    # one-level adaptive refinement with hanging nodes (the paper's adaptive-mesh cases have
    # 1.2-2.1M DoFs): coarse 14^3 unit cube, the central 8^3 coarse cells split into 2x2x2;
    # nx/ny/nz are the coarse counts (num_dofs does not apply: ask the context)
    "h1": Workload("unit cube 14^3 coarse cells, central 8^3 refined once (hanging nodes), p=6, n_q=8, "
                   "Dirichlet-0, n_vec=64", 14, 14, 14, False, 6, 8, 64, "normal", 9, "gauss", v_seed=19,
                   extra={"refine_lo": (3, 3, 3), "refine_hi": (11, 11, 11)}),
}


def batch_workloads(count: int = 24, seed: int = 400, max_footprint_bytes: float = 0.7 * 280e9):
    """The uneven batch: `count` periodic problems with random size, degree and
    block width.  A problem whose X+Y (FP64) would push the running total over
    `max_footprint_bytes` is redrawn with the next seed."""
    out = []
    total = 0.0
    s = seed
    while len(out) < count:
        rng = np.random.Generator(np.random.PCG64(s))
        n = int(rng.integers(4, 25))
        p = int(rng.integers(3, 9))
        n_vec = int(round(math.exp(rng.uniform(math.log(8), math.log(512)))))
        w = Workload(f"batch[{len(out)}] {n}^3 p={p} n_vec={n_vec}", n, n, n, True, p, p + 2, n_vec,
                     "normal", s, "gauss", v_seed=s + 1000)
        foot = 2.0 * 8.0 * w.num_dofs * n_vec
        s += 1
        if total + foot > max_footprint_bytes:
            continue
        total += foot
        out.append(w)
    return out
