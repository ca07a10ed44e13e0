// FP32 cell kernel with register-resident planes (CUDA cores).
//
// Same operation as cell_apply_kernel (Algorithm 2 per cell, extraction and
// assembly fused as in Algorithm 4, colour-ordered conflict-free assembly),
// re-tiled for single precision, where shared-memory bandwidth -- not the FMA
// pipe -- limits a line-per-thread design.  Lanes are 32 vectors; warp w owns
// xy-plane w of the cell for all 32 vectors, so every x and y contraction runs
// on a plane held in registers and only the z direction goes through shared
// memory:
//   A  (plane i3)   gather, N along x and y in registers      -> SA[i3][q2][q1]
//   B  (z-line)     N along z, D~ along z                      -> ST (T), S2 (T2)
//   C  (plane q3)   D~ along x and y in registers, quadrature-point operation,
//                   transposed x and y passes into the plane   -> ST (out), S2 (h2)
//   D  (z-line)     transposed D~ along z, transposed N along z -> SA
//   E  (plane i3)   transposed N along y and x in registers, assembly
// Four barriers per cell instead of nine, and about half the shared-memory
// words per cell and vector.
#pragma once

#include "fe_cell_kernel.cuh"

namespace fe {

template <int NP, int NQ, bool GEN>
__global__ void __launch_bounds__(32 * NQ, 1) plane_apply_kernel(const Tables<float, NP, NQ> tab, const MeshDev m,
                                                                 const Geom<float> geo, const int* __restrict__ cells,
                                                                 int n_vec, int n_vb, const float* __restrict__ X,
                                                                 float* __restrict__ Y) {
  constexpr int P = NP - 1;
  constexpr int NQ2 = NQ * NQ, NQ3 = NQ * NQ * NQ;
  constexpr int NW = NQ;  // warps
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* SA = reinterpret_cast<float*>(smem_raw);   // NP x NQ^2 x 32
  float* ST = SA + NP * NQ2 * 32;                    // NQ^3 x 32
  float* S2 = ST + NQ3 * 32;                         // NQ^3 x 32

  const int v = threadIdx.x, w = threadIdx.y;
  const int vb = blockIdx.x % n_vb;
  const int e = cells[blockIdx.x / n_vb];
  const int vg = vb * 32 + v;
  const bool active = vg < n_vec;
  const int cx = e % m.nx, cy = (e / m.nx) % m.ny, cz = e / (m.nx * m.ny);

  // ---- A: gather plane i3, N along x then y (registers) ----
  if (w < NP) {
    const int i3 = w;
    const int gz = node_coord(cz, i3, P, m.Nz, m.periodic);
    const bool con_z = on_boundary(gz, m.Nz, m.periodic);
    float a[NP][NQ];
#pragma unroll
    for (int i2 = 0; i2 < NP; ++i2) {
      const int gy = node_coord(cy, i2, P, m.Ny, m.periodic);
      const bool con_yz = con_z || on_boundary(gy, m.Ny, m.periodic);
      const size_t row = (size_t)(gy + (size_t)m.Ny * gz) * m.Nx;
      float u[NP];
#pragma unroll
      for (int i1 = 0; i1 < NP; ++i1) {
        const int gx = node_coord(cx, i1, P, m.Nx, m.periodic);
        const bool con = con_yz || on_boundary(gx, m.Nx, m.periodic);
        u[i1] = (active && !con) ? __ldg(X + (row + gx) * n_vec + vg) : 0.f;
      }
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < NP; ++i) s = fmaf(tab.N[q][i], u[i], s);
        a[i2][q] = s;
      }
    }
#pragma unroll
    for (int q1 = 0; q1 < NQ; ++q1)
#pragma unroll
      for (int q2 = 0; q2 < NQ; ++q2) {
        float s = 0.f;
#pragma unroll
        for (int i2 = 0; i2 < NP; ++i2) s = fmaf(tab.N[q2][i2], a[i2][q1], s);
        SA[((i3 * NQ + q2) * NQ + q1) * 32 + v] = s;
      }
  }
  __syncthreads();
  // ---- B: z-lines, N along z and D~ along z ----
  for (int l = w; l < NQ2; l += NW) {
    float s[NP], t[NQ];
#pragma unroll
    for (int i = 0; i < NP; ++i) s[i] = SA[(i * NQ2 + l) * 32 + v];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      float acc = 0.f;
#pragma unroll
      for (int i = 0; i < NP; ++i) acc = fmaf(tab.N[q][i], s[i], acc);
      t[q] = acc;
      ST[(q * NQ2 + l) * 32 + v] = acc;
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < NQ; ++k) acc = fmaf(tab.D[q][k], t[k], acc);
      S2[(q * NQ2 + l) * 32 + v] = acc;
    }
  }
  __syncthreads();
  // ---- C: plane q3: gradients along x, y, quadrature-point operation, transposed x, y ----
  {
    const int q3 = w;
    float T[NQ][NQ], out[NQ][NQ];
#pragma unroll
    for (int q2 = 0; q2 < NQ; ++q2)
#pragma unroll
      for (int q1 = 0; q1 < NQ; ++q1) {
        T[q2][q1] = ST[((q3 * NQ + q2) * NQ + q1) * 32 + v];
        out[q2][q1] = 0.f;
      }
    float g00, g01, g02, g11, g12, g22;
    if (!GEN) {
      g00 = geo.cellG[e * 6 + 0]; g01 = geo.cellG[e * 6 + 1]; g02 = geo.cellG[e * 6 + 2];
      g11 = geo.cellG[e * 6 + 3]; g12 = geo.cellG[e * 6 + 4]; g22 = geo.cellG[e * 6 + 5];
    }
    const float* ptC = geo.ptC + (size_t)e * NQ3;
#pragma unroll
    for (int q2 = 0; q2 < NQ; ++q2) {
      float h0[NQ], h1[NQ];
#pragma unroll
      for (int q1 = 0; q1 < NQ; ++q1) {
        float d0 = 0.f, d1 = 0.f;
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
          d0 = fmaf(tab.D[q1][k], T[q2][k], d0);
          d1 = fmaf(tab.D[q2][k], T[k][q1], d1);
        }
        const int Q = (q3 * NQ + q2) * NQ + q1;
        const float d2 = S2[Q * 32 + v];
        if (GEN) {
          const float* pg = geo.ptG + (size_t)e * 6 * NQ3 + Q;
          g00 = pg[0]; g01 = pg[NQ3]; g02 = pg[2 * NQ3]; g11 = pg[3 * NQ3]; g12 = pg[4 * NQ3]; g22 = pg[5 * NQ3];
        }
        h0[q1] = g00 * d0 + g01 * d1 + g02 * d2;
        h1[q1] = g01 * d0 + g11 * d1 + g12 * d2;
        S2[Q * 32 + v] = g02 * d0 + g12 * d1 + g22 * d2;
        out[q2][q1] = fmaf(ptC[Q], T[q2][q1], out[q2][q1]);
      }
#pragma unroll
      for (int k = 0; k < NQ; ++k) {
        float acc = out[q2][k];
#pragma unroll
        for (int q1 = 0; q1 < NQ; ++q1) acc = fmaf(tab.D[q1][k], h0[q1], acc);
        out[q2][k] = acc;
      }
#pragma unroll
      for (int k = 0; k < NQ; ++k)
#pragma unroll
        for (int q1 = 0; q1 < NQ; ++q1) out[k][q1] = fmaf(tab.D[q2][k], h1[q1], out[k][q1]);
    }
#pragma unroll
    for (int q2 = 0; q2 < NQ; ++q2)
#pragma unroll
      for (int q1 = 0; q1 < NQ; ++q1) ST[((q3 * NQ + q2) * NQ + q1) * 32 + v] = out[q2][q1];
  }
  __syncthreads();
  // ---- D: z-lines, transposed D~ along z, transposed N along z ----
  for (int l = w; l < NQ2; l += NW) {
    float o[NQ], h[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      o[q] = ST[(q * NQ2 + l) * 32 + v];
      h[q] = S2[(q * NQ2 + l) * 32 + v];
    }
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
      float acc = o[k];
#pragma unroll
      for (int q = 0; q < NQ; ++q) acc = fmaf(tab.D[q][k], h[q], acc);
      o[k] = acc;
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      float acc = 0.f;
#pragma unroll
      for (int q = 0; q < NQ; ++q) acc = fmaf(tab.N[q][i], o[q], acc);
      SA[(i * NQ2 + l) * 32 + v] = acc;
    }
  }
  __syncthreads();
  // ---- E: plane i3, transposed N along y then x, assembly ----
  if (w < NP && active) {
    const int i3 = w;
    float c[NP][NQ];
    {
      float b[NQ][NQ];
#pragma unroll
      for (int q2 = 0; q2 < NQ; ++q2)
#pragma unroll
        for (int q1 = 0; q1 < NQ; ++q1) b[q2][q1] = SA[((i3 * NQ + q2) * NQ + q1) * 32 + v];
#pragma unroll
      for (int q1 = 0; q1 < NQ; ++q1)
#pragma unroll
        for (int i2 = 0; i2 < NP; ++i2) {
          float acc = 0.f;
#pragma unroll
          for (int q2 = 0; q2 < NQ; ++q2) acc = fmaf(tab.N[q2][i2], b[q2][q1], acc);
          c[i2][q1] = acc;
        }
    }
    const int gz = node_coord(cz, i3, P, m.Nz, m.periodic);
    const bool con_z = on_boundary(gz, m.Nz, m.periodic);
    const bool first_z = first_along(cz, m.nz, i3, P, m.periodic, m.last_odd_z);
#pragma unroll
    for (int i2 = 0; i2 < NP; ++i2) {
      const int gy = node_coord(cy, i2, P, m.Ny, m.periodic);
      const bool con_yz = con_z || on_boundary(gy, m.Ny, m.periodic);
      const bool first_yz = first_z && first_along(cy, m.ny, i2, P, m.periodic, m.last_odd_y);
      const size_t row = (size_t)(gy + (size_t)m.Ny * gz) * m.Nx;
#pragma unroll
      for (int i1 = 0; i1 < NP; ++i1) {
        float acc = 0.f;
#pragma unroll
        for (int q1 = 0; q1 < NQ; ++q1) acc = fmaf(tab.N[q1][i1], c[i2][q1], acc);
        const int gx = node_coord(cx, i1, P, m.Nx, m.periodic);
        const bool con = con_yz || on_boundary(gx, m.Nx, m.periodic);
        const bool first = first_yz && first_along(cx, m.nx, i1, P, m.periodic, m.last_odd_x);
        float* dst = Y + (row + gx) * n_vec + vg;
        if (first) *dst = con ? 0.f : acc;
        else if (!con) *dst += acc;
      }
    }
  }
}

template <int NP, int NQ, bool GEN>
cudaError_t launch_plane(const fe_ctx* c, const float* X, float* Y, int n_vec, cudaStream_t s) {
  auto kern = plane_apply_kernel<NP, NQ, GEN>;
  const size_t smem = (size_t)(NP * NQ * NQ + 2 * NQ * NQ * NQ) * 32 * sizeof(float);
  {
    cudaError_t e = ensure_dyn_smem(reinterpret_cast<const void*>(kern), smem);
    if (e != cudaSuccess) return e;
  }
  const Tables<float, NP, NQ> tab = make_tables<float, NP, NQ>(c);
  const Geom<float> geo = make_geom<float>(c);
  const int n_vb = (n_vec + 31) / 32;
  for (int k = 0; k < c->colors.n_colors; ++k) {
    const int n = c->colors.offset[k + 1] - c->colors.offset[k];
    if (n == 0) continue;
    const long long blocks = (long long)n * n_vb;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    kern<<<(unsigned)blocks, dim3(32, NQ), smem, s>>>(tab, c->mdev, geo, c->d_cells + c->colors.offset[k], n_vec,
                                                      n_vb, X, Y);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace fe
