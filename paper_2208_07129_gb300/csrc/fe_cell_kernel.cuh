// Fused matrix-free cell kernel on CUDA cores (FP64 or FP32).
//
// One CTA evaluates V^(e) = (K^(e) + M^{V,(e)}) U^(e) for one cell e and one
// block of B vectors, in the order of Algorithm 2 of the paper:
//   T = N U (three 1D passes, Algorithm 1), gradients by the collocation
//   derivative D~ along each direction (the factorisation D = D~ N of Sec. 2.2),
//   the quadrature-point operation [T0 T1 T2] <- G [T0 T1 T2] and T <- c T,
//   the transposed derivative passes accumulated into T, and N^T.
// Extraction (Q C X) is fused into the first pass and assembly (C^T Q^T) into
// the last, as in Algorithm 4, but assembly is conflict-free: CTAs of one
// launch belong to one cell colour, so no two of them share a node, and the
// first colour to reach a node stores while later colours add (no atomics,
// no pre-zeroing of Y, bitwise reproducible).
//
// Thread layout: threadIdx.x = vector within the block (B lanes, so global
// loads and stores of one node are contiguous), threadIdx.y = 1D line.  Each
// thread holds one line in registers and forms every output of the line as a
// linear combination of the line's inputs with coefficients taken from the
// kernel-parameter tables (constant bank).  Shared memory holds three
// n_q^3 x B tiles: T, and T0 / T1 (also reused for the n_p-sized
// intermediates of the N passes).  T2 never leaves registers: the z-lines
// compute it, apply the quadrature-point operation and its transpose at once.
#pragma once

#include "fe_internal.h"

namespace fe {

__host__ __device__ __forceinline__ int dir_color(int c, int n, int last_odd) {
  return (last_odd && c == n - 1) ? 2 : (c & 1);
}

// True if cell coordinate c owns the lowest colour among the cells that share
// the node at local index i (0..P) along one direction.
__host__ __device__ __forceinline__ bool first_along(int c, int n, int i, int P, int periodic, int last_odd) {
  const int k = dir_color(c, n, last_odd);
  if (i == 0 && (c > 0 || periodic)) {
    const int cn = c > 0 ? c - 1 : n - 1;
    if (dir_color(cn, n, last_odd) < k) return false;
  }
  if (i == P && (c < n - 1 || periodic)) {
    const int cn = c < n - 1 ? c + 1 : 0;
    if (dir_color(cn, n, last_odd) < k) return false;
  }
  return true;
}

// Global node coordinate along one direction (wrap-around when periodic).
__host__ __device__ __forceinline__ int node_coord(int c, int i, int P, int N, int periodic) {
  int g = c * P + i;
  if (periodic && g >= N) g -= N;
  return g;
}

__host__ __device__ __forceinline__ bool on_boundary(int g, int N, int periodic) {
  return !periodic && (g == 0 || g == N - 1);
}

// Scatter of the scaled product for one node: the first writer of the node
// (colour order) stores a M^-1/2 (cell sum) + b X + c Y_old (0 on constrained
// rows), later writers add their a M^-1/2 (cell sum).  b X and c Y are only
// read when the coefficient is nonzero, so Y may start uninitialised when c = 0.
template <typename T>
__device__ __forceinline__ void scaled_store(T* dst, const T* x, T val, bool first, bool con, const Scale<T>& sc) {
  if (first) {
    if (con) {
      *dst = T(0);
    } else {
      if (sc.b != T(0)) val += sc.b * __ldg(x);
      if (sc.c != T(0)) val += sc.c * *dst;
      *dst = val;
    }
  } else if (!con) {
    *dst += val;
  }
}

// The work of one CTA: cell e, vector block vb of B vectors; thread (v, ty) of
// a B x nty thread block; smem holds 3 n_q^3 x B values.  Shared by the
// per-colour launches below and by the persistent batch kernel.  With SC the
// gather scales X by M^-1/2 and the scatter writes the scaled product
// a M^-1/2 (.) + b X + c Y (see Scale).
template <typename T, int NP, int NQ, bool GEN, bool SC = false>
__device__ __forceinline__ void cell_body(const Tables<T, NP, NQ>& tab, const MeshDev& m, const Geom<T>& geo, int e,
                                          int vb, int B, int v, int ty, int nty, int n_vec, const T* __restrict__ X,
                                          T* __restrict__ Y, T* smem, const Scale<T>& sc = Scale<T>{}) {
  constexpr int P = NP - 1;
  constexpr int NQ3 = NQ * NQ * NQ;
  T* ST = smem;
  T* S0 = ST + NQ3 * B;
  T* S1 = S0 + NQ3 * B;
  const int vg = vb * B + v;
  const bool active = vg < n_vec;
  const int cx = e % m.nx, cy = (e / m.nx) % m.ny, cz = e / (m.nx * m.ny);

  // ---- extraction fused with the x pass of N:  S0[i3][i2][q1] ----
  for (int l = ty; l < NP * NP; l += nty) {
    const int i2 = l % NP, i3 = l / NP;
    const int gy = node_coord(cy, i2, P, m.Ny, m.periodic), gz = node_coord(cz, i3, P, m.Nz, m.periodic);
    const bool con_yz = on_boundary(gy, m.Ny, m.periodic) || on_boundary(gz, m.Nz, m.periodic);
    const size_t row = (size_t)(gy + (size_t)m.Ny * gz) * m.Nx;
    T u[NP];
#pragma unroll
    for (int i1 = 0; i1 < NP; ++i1) {
      const int gx = node_coord(cx, i1, P, m.Nx, m.periodic);
      const bool con = con_yz || on_boundary(gx, m.Nx, m.periodic);
      u[i1] = (active && !con) ? __ldg(X + (row + gx) * n_vec + vg) : T(0);
      if constexpr (SC) u[i1] *= __ldg(sc.msq + row + gx);
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      T s = T(0);
#pragma unroll
      for (int i = 0; i < NP; ++i) s += tab.N[q][i] * u[i];
      S0[((i3 * NP + i2) * NQ + q) * B + v] = s;
    }
  }
  __syncthreads();
  // ---- y pass of N:  S1[i3][q2][q1] ----
  for (int l = ty; l < NQ * NP; l += nty) {
    const int q1 = l % NQ, i3 = l / NQ;
    T a[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) a[i] = S0[((i3 * NP + i) * NQ + q1) * B + v];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      T s = T(0);
#pragma unroll
      for (int i = 0; i < NP; ++i) s += tab.N[q][i] * a[i];
      S1[((i3 * NQ + q) * NQ + q1) * B + v] = s;
    }
  }
  __syncthreads();
  // ---- z pass of N:  ST[q3][q2][q1] ----
  for (int l = ty; l < NQ * NQ; l += nty) {
    T a[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) a[i] = S1[(i * NQ * NQ + l) * B + v];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      T s = T(0);
#pragma unroll
      for (int i = 0; i < NP; ++i) s += tab.N[q][i] * a[i];
      ST[(q * NQ * NQ + l) * B + v] = s;
    }
  }
  __syncthreads();
  // ---- reference gradients along x (-> S0) and y (-> S1) ----
  for (int l = ty; l < 2 * NQ * NQ; l += nty) {
    const bool ydir = l >= NQ * NQ;
    const int ll = ydir ? l - NQ * NQ : l;
    // x-lines: ll = q2 + NQ q3, stride 1;  y-lines: ll = q1 + NQ q3, stride NQ
    const int base = ydir ? (ll % NQ) + (ll / NQ) * NQ * NQ : ll * NQ;
    const int stride = ydir ? NQ : 1;
    T t[NQ];
#pragma unroll
    for (int k = 0; k < NQ; ++k) t[k] = ST[(base + k * stride) * B + v];
    T* dst = ydir ? S1 : S0;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      T s = T(0);
#pragma unroll
      for (int k = 0; k < NQ; ++k) s += tab.D[q][k] * t[k];
      dst[(base + q * stride) * B + v] = s;
    }
  }
  __syncthreads();
  // ---- z-lines: gradient along z, quadrature-point operation, transposed z pass ----
  T g00, g01, g02, g11, g12, g22;
  if (!GEN) {
    g00 = geo.cellG[e * 6 + 0]; g01 = geo.cellG[e * 6 + 1]; g02 = geo.cellG[e * 6 + 2];
    g11 = geo.cellG[e * 6 + 3]; g12 = geo.cellG[e * 6 + 4]; g22 = geo.cellG[e * 6 + 5];
  }
  const T* ptC = geo.ptC + (size_t)e * NQ3;
  for (int l = ty; l < NQ * NQ; l += nty) {
    T t[NQ], h2[NQ];
#pragma unroll
    for (int k = 0; k < NQ; ++k) t[k] = ST[(k * NQ * NQ + l) * B + v];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      T s = T(0);
#pragma unroll
      for (int k = 0; k < NQ; ++k) s += tab.D[q][k] * t[k];
      h2[q] = s;
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const T d2 = h2[q];
      const int Q = q * NQ * NQ + l;
      const T d0 = S0[Q * B + v], d1 = S1[Q * B + v];
      if (GEN) {
        const T* pg = geo.ptG + (size_t)e * 6 * NQ3 + Q;
        g00 = pg[0]; g01 = pg[NQ3]; g02 = pg[2 * NQ3]; g11 = pg[3 * NQ3]; g12 = pg[4 * NQ3]; g22 = pg[5 * NQ3];
      }
      S0[Q * B + v] = g00 * d0 + g01 * d1 + g02 * d2;
      S1[Q * B + v] = g01 * d0 + g11 * d1 + g12 * d2;
      h2[q] = g02 * d0 + g12 * d1 + g22 * d2;
      t[q] = ptC[Q] * t[q];
    }
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
      T s = t[k];
#pragma unroll
      for (int q = 0; q < NQ; ++q) s += tab.D[q][k] * h2[q];
      ST[(k * NQ * NQ + l) * B + v] = s;
    }
  }
  __syncthreads();
  // ---- transposed x pass of D~ accumulated into T ----
  for (int l = ty; l < NQ * NQ; l += nty) {
    const int base = l * NQ;
    T h[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) h[q] = S0[(base + q) * B + v];
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
      T s = ST[(base + k) * B + v];
#pragma unroll
      for (int q = 0; q < NQ; ++q) s += tab.D[q][k] * h[q];
      ST[(base + k) * B + v] = s;
    }
  }
  __syncthreads();
  // ---- transposed y pass of D~ accumulated into T ----
  for (int l = ty; l < NQ * NQ; l += nty) {
    const int base = (l % NQ) + (l / NQ) * NQ * NQ;
    T h[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) h[q] = S1[(base + q * NQ) * B + v];
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
      T s = ST[(base + k * NQ) * B + v];
#pragma unroll
      for (int q = 0; q < NQ; ++q) s += tab.D[q][k] * h[q];
      ST[(base + k * NQ) * B + v] = s;
    }
  }
  __syncthreads();
  // ---- transposed z pass of N:  S1[i3][q2][q1] ----
  for (int l = ty; l < NQ * NQ; l += nty) {
    T t[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) t[q] = ST[(q * NQ * NQ + l) * B + v];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      T s = T(0);
#pragma unroll
      for (int q = 0; q < NQ; ++q) s += tab.N[q][i] * t[q];
      S1[(i * NQ * NQ + l) * B + v] = s;
    }
  }
  __syncthreads();
  // ---- transposed y pass of N:  S0[i3][i2][q1] ----
  for (int l = ty; l < NQ * NP; l += nty) {
    const int q1 = l % NQ, i3 = l / NQ;
    T t[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) t[q] = S1[((i3 * NQ + q) * NQ + q1) * B + v];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      T s = T(0);
#pragma unroll
      for (int q = 0; q < NQ; ++q) s += tab.N[q][i] * t[q];
      S0[((i3 * NP + i) * NQ + q1) * B + v] = s;
    }
  }
  __syncthreads();
  // ---- transposed x pass of N fused with assembly ----
  for (int l = ty; l < NP * NP; l += nty) {
    const int i2 = l % NP, i3 = l / NP;
    T t[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) t[q] = S0[((i3 * NP + i2) * NQ + q) * B + v];
    if (!active) continue;
    const int gy = node_coord(cy, i2, P, m.Ny, m.periodic), gz = node_coord(cz, i3, P, m.Nz, m.periodic);
    const bool con_yz = on_boundary(gy, m.Ny, m.periodic) || on_boundary(gz, m.Nz, m.periodic);
    const bool first_yz = first_along(cy, m.ny, i2, P, m.periodic, m.last_odd_y) &&
                          first_along(cz, m.nz, i3, P, m.periodic, m.last_odd_z);
    const size_t row = (size_t)(gy + (size_t)m.Ny * gz) * m.Nx;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      T s = T(0);
#pragma unroll
      for (int q = 0; q < NQ; ++q) s += tab.N[q][i] * t[q];
      const int gx = node_coord(cx, i, P, m.Nx, m.periodic);
      const bool con = con_yz || on_boundary(gx, m.Nx, m.periodic);
      const bool first = first_yz && first_along(cx, m.nx, i, P, m.periodic, m.last_odd_x);
      T* dst = Y + (row + gx) * n_vec + vg;
      if constexpr (SC) {
        scaled_store(dst, X + (row + gx) * n_vec + vg, sc.a * __ldg(sc.msq + row + gx) * s, first, con, sc);
      } else {
        if (first) *dst = con ? T(0) : s;
        else if (!con) *dst += s;
      }
    }
  }
}

template <typename T, int NP, int NQ, bool GEN>
__global__ void __launch_bounds__(256) cell_apply_kernel(const Tables<T, NP, NQ> tab, const MeshDev m,
                                                         const Geom<T> geo, const int* __restrict__ cells,
                                                         int n_vec, int n_vb, const T* __restrict__ X,
                                                         T* __restrict__ Y) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cell_body<T, NP, NQ, GEN>(tab, m, geo, cells[blockIdx.x / n_vb], blockIdx.x % n_vb, blockDim.x, threadIdx.x,
                            threadIdx.y, blockDim.y, n_vec, X, Y, reinterpret_cast<T*>(smem_raw));
}

// The scaled product of the Chebyshev filter, Y = a M^-1/2 A M^-1/2 X + b X + c Y.
template <typename T, int NP, int NQ, bool GEN>
__global__ void __launch_bounds__(256) cell_apply_scaled_kernel(const Tables<T, NP, NQ> tab, const MeshDev m,
                                                                const Geom<T> geo, const int* __restrict__ cells,
                                                                int n_vec, int n_vb, const T* __restrict__ X,
                                                                T* __restrict__ Y, const Scale<T> sc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cell_body<T, NP, NQ, GEN, true>(tab, m, geo, cells[blockIdx.x / n_vb], blockIdx.x % n_vb, blockDim.x, threadIdx.x,
                                  threadIdx.y, blockDim.y, n_vec, X, Y, reinterpret_cast<T*>(smem_raw), sc);
}

// diag(A): one thread per (cell, local node), sum over the quadrature points of
//   (grad phi_i)^T G (grad phi_i) + c phi_i^2  with the folded tables, where
//   grad phi_i at Q = ((D~N)[q1][i1] N[q2][i2] N[q3][i3], ...), assembled by
// colours with the same first-writer rule as the apply kernel; constrained
// rows get 1.
template <int NP, int NQ, bool GEN>
__global__ void cell_diag_kernel(const Tables<double, NP, NQ> tab, const MeshDev m, const Geom<double> geo,
                                 const int* __restrict__ cells, int n_cells, double* __restrict__ diag) {
  constexpr int P = NP - 1;
  constexpr int NP3 = NP * NP * NP, NQ3 = NQ * NQ * NQ;
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= n_cells * NP3) return;
  const int e = cells[gid / NP3];
  const int I = gid % NP3;
  const int i1 = I % NP, i2 = (I / NP) % NP, i3 = I / (NP * NP);
  double DN[NQ][NP];
#pragma unroll
  for (int q = 0; q < NQ; ++q)
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      double s = 0;
#pragma unroll
      for (int k = 0; k < NQ; ++k) s += tab.D[q][k] * tab.N[k][i];
      DN[q][i] = s;
    }
  double acc = 0.0;
  for (int q3 = 0; q3 < NQ; ++q3)
    for (int q2 = 0; q2 < NQ; ++q2)
      for (int q1 = 0; q1 < NQ; ++q1) {
        const int Q = q1 + NQ * (q2 + NQ * q3);
        const double n1 = tab.N[q1][i1], n2 = tab.N[q2][i2], n3 = tab.N[q3][i3];
        const double a0 = DN[q1][i1] * n2 * n3, a1 = n1 * DN[q2][i2] * n3, a2 = n1 * n2 * DN[q3][i3];
        const double* G = GEN ? geo.ptG + (size_t)e * 6 * NQ3 + Q : geo.cellG + e * 6;
        const int st = GEN ? NQ3 : 1;
        const double g00 = G[0], g01 = G[st], g02 = G[2 * st], g11 = G[3 * st], g12 = G[4 * st], g22 = G[5 * st];
        acc += a0 * (g00 * a0 + g01 * a1 + g02 * a2) + a1 * (g01 * a0 + g11 * a1 + g12 * a2) +
               a2 * (g02 * a0 + g12 * a1 + g22 * a2) + geo.ptC[(size_t)e * NQ3 + Q] * (n1 * n2 * n3) * (n1 * n2 * n3);
      }
  const int cx = e % m.nx, cy = (e / m.nx) % m.ny, cz = e / (m.nx * m.ny);
  const int gx = node_coord(cx, i1, P, m.Nx, m.periodic), gy = node_coord(cy, i2, P, m.Ny, m.periodic),
            gz = node_coord(cz, i3, P, m.Nz, m.periodic);
  const bool con = on_boundary(gx, m.Nx, m.periodic) || on_boundary(gy, m.Ny, m.periodic) ||
                   on_boundary(gz, m.Nz, m.periodic);
  const bool first = first_along(cx, m.nx, i1, P, m.periodic, m.last_odd_x) &&
                     first_along(cy, m.ny, i2, P, m.periodic, m.last_odd_y) &&
                     first_along(cz, m.nz, i3, P, m.periodic, m.last_odd_z);
  double* dst = diag + gx + (size_t)m.Nx * (gy + (size_t)m.Ny * gz);
  if (first) *dst = con ? 1.0 : acc;
  else if (!con) *dst += acc;
}

}  // namespace fe
