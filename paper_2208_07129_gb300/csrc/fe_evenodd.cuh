// Even-odd decomposition of the 1D contractions (FP64 cell kernel).
//
// The 1D matrices are (skew-)centrosymmetric: GLL nodes and the quadrature
// points are symmetric about 0, so N(n_q-1-q, n_p-1-i) = N(q, i) and
// D~(n_q-1-q, n_q-1-k) = -D~(q, k); folding sqrt(w) keeps both symmetries.
// For such an M (sign s), out = M in splits into an even and an odd half:
//   e_i = in_i + in_{n-1-i},  o_i = in_i - in_{n-1-i},
//   E_q = sum_i (M_qi + M_q,n-1-i)/2 e_i (+ M_q,mid in_mid),
//   O_q = sum_i (M_qi - M_q,n-1-i)/2 o_i,
//   out_q = E_q + O_q,   out_{m-1-q} = s (E_q - O_q),
// about half the multiply-adds of the plain product (the paper's even-odd
// scheme for its CPU kernels, Sec. 3.2.4; it kept the plain form on V100
// because of warp stalls -- on GB300 the FP64 pipe is the bound, so the
// saved FP64 operations are the saved time).  Transposed products use the
// tables of M^T, which has the same symmetry.
#pragma once

#include <algorithm>

#include "fe_cell_kernel.cuh"

namespace fe {

// Tables of out = M in for an NO x NI matrix M with M(NO-1-o, NI-1-i) = S M(o, i).
template <typename T, int NO, int NI>
struct EOTab {
  static constexpr int HO = (NO + 1) / 2;   // outputs computed directly
  static constexpr int HE = (NI + 1) / 2;   // even inputs (with the middle one)
  static constexpr int HOD = NI / 2 > 0 ? NI / 2 : 1;
  T E[HO][HE];
  T O[HO][HOD];
};

template <typename T, int NP, int NQ>
struct EOTables {
  EOTab<T, NQ, NP> N;     // values at points from nodes
  EOTab<T, NP, NQ> Nt;    // transposed
  EOTab<T, NQ, NQ> D;     // collocation derivative
  EOTab<T, NQ, NQ> Dt;    // transposed
};

template <typename T, int NO, int NI, int S>
__device__ __forceinline__ void eo_apply(const EOTab<T, NO, NI>& t, const T* in, T* out) {
  constexpr int HI = NI / 2, HO = (NO + 1) / 2, HE = (NI + 1) / 2;
  T ie[HE], io[HI > 0 ? HI : 1];
#pragma unroll
  for (int i = 0; i < HI; ++i) {
    ie[i] = in[i] + in[NI - 1 - i];
    io[i] = in[i] - in[NI - 1 - i];
  }
  if (NI & 1) ie[HI] = in[HI];
#pragma unroll
  for (int o = 0; o < HO; ++o) {
    T e = T(0), d = T(0);
#pragma unroll
    for (int i = 0; i < HE; ++i) e += t.E[o][i] * ie[i];
#pragma unroll
    for (int i = 0; i < HI; ++i) d += t.O[o][i] * io[i];
    out[o] = e + d;
    if (o != NO - 1 - o) out[NO - 1 - o] = S > 0 ? e - d : d - e;
  }
}

// Same as cell_body (identical data flow, tiles and assembly, the same SC
// epilogue), with every 1D contraction in even-odd form.  With MAP the cell's
// nodes come from an explicit map (see map_node) instead of the structured
// numbering: the refined meshes with hanging nodes.
// LOCAL: the cell's result is written to Y[(e n_p^3 + local node) n_vec + v]
// (a per-cell scratch block, every local node, constrained ones included)
// instead of being assembled into the global vector.
template <typename T, int NP, int NQ, bool GEN, bool SC = false, bool MAP = false, bool LOCAL = false>
__device__ __forceinline__ void cell_body_eo(const EOTables<T, NP, NQ>& tab, const MeshDev& m, const Geom<T>& geo,
                                             int e, int vb, int B, int v, int ty, int nty, int n_vec,
                                             const T* __restrict__ X, T* __restrict__ Y, T* smem,
                                             const Scale<T>& sc = Scale<T>{}, const int* __restrict__ map = nullptr) {
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
    T u[NP], a[NQ];
#pragma unroll
    for (int i1 = 0; i1 < NP; ++i1) {
      size_t node;
      bool con;
      if constexpr (MAP) {
        const int code = __ldg(map + (size_t)e * NP * NP * NP + l * NP + i1);
        node = (size_t)(code & kMapIndex);
        con = (code & kMapConstrained) != 0;
      } else {
        const int gx = node_coord(cx, i1, P, m.Nx, m.periodic);
        node = row + gx;
        con = con_yz || on_boundary(gx, m.Nx, m.periodic);
      }
      u[i1] = (active && !con) ? __ldg(X + node * n_vec + vg) : T(0);
      if constexpr (SC) u[i1] *= __ldg(sc.msq + node);
    }
    eo_apply<T, NQ, NP, 1>(tab.N, u, a);
#pragma unroll
    for (int q = 0; q < NQ; ++q) S0[((i3 * NP + i2) * NQ + q) * B + v] = a[q];
  }
  __syncthreads();
  // ---- y pass of N:  S1[i3][q2][q1] ----
  for (int l = ty; l < NQ * NP; l += nty) {
    const int q1 = l % NQ, i3 = l / NQ;
    T a[NP], b[NQ];
#pragma unroll
    for (int i = 0; i < NP; ++i) a[i] = S0[((i3 * NP + i) * NQ + q1) * B + v];
    eo_apply<T, NQ, NP, 1>(tab.N, a, b);
#pragma unroll
    for (int q = 0; q < NQ; ++q) S1[((i3 * NQ + q) * NQ + q1) * B + v] = b[q];
  }
  __syncthreads();
  // ---- z pass of N:  ST[q3][q2][q1] ----
  for (int l = ty; l < NQ * NQ; l += nty) {
    T a[NP], b[NQ];
#pragma unroll
    for (int i = 0; i < NP; ++i) a[i] = S1[(i * NQ * NQ + l) * B + v];
    eo_apply<T, NQ, NP, 1>(tab.N, a, b);
#pragma unroll
    for (int q = 0; q < NQ; ++q) ST[(q * NQ * NQ + l) * B + v] = b[q];
  }
  __syncthreads();
  // ---- reference gradients along x (-> S0) and y (-> S1) ----
  for (int l = ty; l < 2 * NQ * NQ; l += nty) {
    const bool ydir = l >= NQ * NQ;
    const int ll = ydir ? l - NQ * NQ : l;
    const int base = ydir ? (ll % NQ) + (ll / NQ) * NQ * NQ : ll * NQ;
    const int stride = ydir ? NQ : 1;
    T t[NQ], g[NQ];
#pragma unroll
    for (int k = 0; k < NQ; ++k) t[k] = ST[(base + k * stride) * B + v];
    eo_apply<T, NQ, NQ, -1>(tab.D, t, g);
    T* dst = ydir ? S1 : S0;
#pragma unroll
    for (int q = 0; q < NQ; ++q) dst[(base + q * stride) * B + v] = g[q];
  }
  __syncthreads();
  // ---- z-lines: gradient along z, quadrature-point operation, transposed z pass ----
  // Cells without per-point geometry are axis-aligned boxes (checked at
  // setup): their metric is diagonal, and the point operation scales each
  // gradient component by one coefficient.
  T g00, g01, g02, g11, g12, g22;
  if (!GEN) {
    g00 = geo.cellG[e * 6 + 0]; g11 = geo.cellG[e * 6 + 3]; g22 = geo.cellG[e * 6 + 5];
  }
  const T* ptC = geo.ptC + (size_t)e * NQ3;
  for (int l = ty; l < NQ * NQ; l += nty) {
    T t[NQ], h2[NQ], o[NQ];
#pragma unroll
    for (int k = 0; k < NQ; ++k) t[k] = ST[(k * NQ * NQ + l) * B + v];
    eo_apply<T, NQ, NQ, -1>(tab.D, t, h2);
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const T d2 = h2[q];
      const int Q = q * NQ * NQ + l;
      const T d0 = S0[Q * B + v], d1 = S1[Q * B + v];
      if (GEN) {
        const T* pg = geo.ptG + (size_t)e * 6 * NQ3 + Q;
        g00 = pg[0]; g01 = pg[NQ3]; g02 = pg[2 * NQ3]; g11 = pg[3 * NQ3]; g12 = pg[4 * NQ3]; g22 = pg[5 * NQ3];
        S0[Q * B + v] = g00 * d0 + g01 * d1 + g02 * d2;
        S1[Q * B + v] = g01 * d0 + g11 * d1 + g12 * d2;
        h2[q] = g02 * d0 + g12 * d1 + g22 * d2;
      } else {
        S0[Q * B + v] = g00 * d0;
        S1[Q * B + v] = g11 * d1;
        h2[q] = g22 * d2;
      }
      t[q] = ptC[Q] * t[q];
    }
    eo_apply<T, NQ, NQ, -1>(tab.Dt, h2, o);
#pragma unroll
    for (int k = 0; k < NQ; ++k) ST[(k * NQ * NQ + l) * B + v] = t[k] + o[k];
  }
  __syncthreads();
  // ---- transposed x pass of D~ accumulated into T ----
  for (int l = ty; l < NQ * NQ; l += nty) {
    const int base = l * NQ;
    T h[NQ], o[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) h[q] = S0[(base + q) * B + v];
    eo_apply<T, NQ, NQ, -1>(tab.Dt, h, o);
#pragma unroll
    for (int k = 0; k < NQ; ++k) ST[(base + k) * B + v] += o[k];
  }
  __syncthreads();
  // ---- transposed y pass of D~ accumulated into T ----
  for (int l = ty; l < NQ * NQ; l += nty) {
    const int base = (l % NQ) + (l / NQ) * NQ * NQ;
    T h[NQ], o[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) h[q] = S1[(base + q * NQ) * B + v];
    eo_apply<T, NQ, NQ, -1>(tab.Dt, h, o);
#pragma unroll
    for (int k = 0; k < NQ; ++k) ST[(base + k * NQ) * B + v] += o[k];
  }
  __syncthreads();
  // ---- transposed z pass of N:  S1[i3][q2][q1] ----
  for (int l = ty; l < NQ * NQ; l += nty) {
    T t[NQ], o[NP];
#pragma unroll
    for (int q = 0; q < NQ; ++q) t[q] = ST[(q * NQ * NQ + l) * B + v];
    eo_apply<T, NP, NQ, 1>(tab.Nt, t, o);
#pragma unroll
    for (int i = 0; i < NP; ++i) S1[(i * NQ * NQ + l) * B + v] = o[i];
  }
  __syncthreads();
  // ---- transposed y pass of N:  S0[i3][i2][q1] ----
  for (int l = ty; l < NQ * NP; l += nty) {
    const int q1 = l % NQ, i3 = l / NQ;
    T t[NQ], o[NP];
#pragma unroll
    for (int q = 0; q < NQ; ++q) t[q] = S1[((i3 * NQ + q) * NQ + q1) * B + v];
    eo_apply<T, NP, NQ, 1>(tab.Nt, t, o);
#pragma unroll
    for (int i = 0; i < NP; ++i) S0[((i3 * NP + i) * NQ + q1) * B + v] = o[i];
  }
  __syncthreads();
  // ---- transposed x pass of N fused with assembly ----
  for (int l = ty; l < NP * NP; l += nty) {
    const int i2 = l % NP, i3 = l / NP;
    T t[NQ], o[NP];
#pragma unroll
    for (int q = 0; q < NQ; ++q) t[q] = S0[((i3 * NP + i2) * NQ + q) * B + v];
    if (!active) continue;
    eo_apply<T, NP, NQ, 1>(tab.Nt, t, o);
    if constexpr (LOCAL) {
      T* w = Y + ((size_t)e * NP * NP * NP + (size_t)l * NP) * n_vec + vg;
#pragma unroll
      for (int i = 0; i < NP; ++i) w[(size_t)i * n_vec] = o[i];
      continue;
    }
    const int gy = node_coord(cy, i2, P, m.Ny, m.periodic), gz = node_coord(cz, i3, P, m.Nz, m.periodic);
    const bool con_yz = on_boundary(gy, m.Ny, m.periodic) || on_boundary(gz, m.Nz, m.periodic);
    const bool first_yz = first_along(cy, m.ny, i2, P, m.periodic, m.last_odd_y) &&
                          first_along(cz, m.nz, i3, P, m.periodic, m.last_odd_z);
    const size_t row = (size_t)(gy + (size_t)m.Ny * gz) * m.Nx;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      size_t node;
      bool con, first;
      if constexpr (MAP) {
        const int code = __ldg(map + (size_t)e * NP * NP * NP + l * NP + i);
        node = (size_t)(code & kMapIndex);
        con = (code & kMapConstrained) != 0;
        first = (code & kMapFirst) != 0;
      } else {
        const int gx = node_coord(cx, i, P, m.Nx, m.periodic);
        node = row + gx;
        con = con_yz || on_boundary(gx, m.Nx, m.periodic);
        first = first_yz && first_along(cx, m.nx, i, P, m.periodic, m.last_odd_x);
      }
      T* dst = Y + node * n_vec + vg;
      if constexpr (SC) {
        scaled_store(dst, X + node * n_vec + vg, sc.a * __ldg(sc.msq + node) * o[i], first, con, sc);
      } else {
        if (first) *dst = con ? T(0) : o[i];
        else if (!con) *dst += o[i];
      }
    }
  }
}

template <typename T, int NP, int NQ, bool GEN>
__global__ void __launch_bounds__(256) cell_apply_eo_kernel(const EOTables<T, NP, NQ> tab, const MeshDev m,
                                                            const Geom<T> geo, const int* __restrict__ cells,
                                                            int n_vec, int n_vb, const T* __restrict__ X,
                                                            T* __restrict__ Y) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cell_body_eo<T, NP, NQ, GEN>(tab, m, geo, cells[blockIdx.x / n_vb], blockIdx.x % n_vb, blockDim.x, threadIdx.x,
                               threadIdx.y, blockDim.y, n_vec, X, Y, reinterpret_cast<T*>(smem_raw));
}

// The scaled product of the Chebyshev filter with even-odd contractions.
template <typename T, int NP, int NQ, bool GEN>
__global__ void __launch_bounds__(256) cell_apply_eo_scaled_kernel(const EOTables<T, NP, NQ> tab, const MeshDev m,
                                                                   const Geom<T> geo, const int* __restrict__ cells,
                                                                   int n_vec, int n_vb, const T* __restrict__ X,
                                                                   T* __restrict__ Y, const Scale<T> sc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cell_body_eo<T, NP, NQ, GEN, true>(tab, m, geo, cells[blockIdx.x / n_vb], blockIdx.x % n_vb, blockDim.x,
                                     threadIdx.x, threadIdx.y, blockDim.y, n_vec, X, Y,
                                     reinterpret_cast<T*>(smem_raw), sc);
}

// Small meshes: every cell in one launch, results to the per-cell scratch W.
template <typename T, int NP, int NQ, bool GEN>
__global__ void __launch_bounds__(256) cell_apply_eo_local_kernel(const EOTables<T, NP, NQ> tab, const MeshDev m,
                                                                  const Geom<T> geo, int n_vec, int n_vb,
                                                                  const T* __restrict__ X, T* __restrict__ W) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cell_body_eo<T, NP, NQ, GEN, false, false, true>(tab, m, geo, blockIdx.x / n_vb, blockIdx.x % n_vb, blockDim.x,
                                                   threadIdx.x, threadIdx.y, blockDim.y, n_vec, X, W,
                                                   reinterpret_cast<T*>(smem_raw));
}

// The cells sharing a node along one direction (one, or two at a cell
// boundary), as (cell coordinate, local index), ordered by the direction's
// cell colour.
__device__ __forceinline__ int node_cells(int g, int n, int P, int periodic, int last_odd, int* c, int* l) {
  int k;
  if (periodic) {
    c[0] = g / P;
    l[0] = g - c[0] * P;
    k = 1;
    if (l[0] == 0) { c[1] = c[0] > 0 ? c[0] - 1 : n - 1; l[1] = P; k = 2; }
  } else {
    c[0] = g / P < n - 1 ? g / P : n - 1;
    l[0] = g - c[0] * P;
    k = 1;
    if (l[0] == 0 && c[0] > 0) { c[1] = c[0] - 1; l[1] = P; k = 2; }
  }
  if (k == 2 && dir_color(c[1], n, last_odd) < dir_color(c[0], n, last_odd)) {
    int t = c[0]; c[0] = c[1]; c[1] = t;
    t = l[0]; l[0] = l[1]; l[1] = t;
  }
  return k;
}

// Y[dof][v] = sum over the cells sharing dof of W[cell][local][v], added in
// ascending cell colour (z colour slowest, x fastest), which is the order of
// the colour-ordered launches: the result equals theirs bit for bit.
// Dirichlet rows are 0.
template <typename T, int NP>
__global__ void assemble_local_kernel(const MeshDev m, const T* __restrict__ W, T* __restrict__ Y, size_t n_dofs,
                                      int n_vec) {
  constexpr int P = NP - 1, NP3 = NP * NP * NP;
  const size_t total = n_dofs * n_vec;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const size_t dof = idx / n_vec;
    const int v = (int)(idx - dof * n_vec);
    const int gx = (int)(dof % m.Nx), gy = (int)((dof / m.Nx) % m.Ny), gz = (int)(dof / ((size_t)m.Nx * m.Ny));
    if (on_boundary(gx, m.Nx, m.periodic) || on_boundary(gy, m.Ny, m.periodic) ||
        on_boundary(gz, m.Nz, m.periodic)) {
      Y[idx] = T(0);
      continue;
    }
    int cx[2], lx[2], cy[2], ly[2], cz[2], lz[2];
    const int kx = node_cells(gx, m.nx, P, m.periodic, m.last_odd_x, cx, lx);
    const int ky = node_cells(gy, m.ny, P, m.periodic, m.last_odd_y, cy, ly);
    const int kz = node_cells(gz, m.nz, P, m.periodic, m.last_odd_z, cz, lz);
    T acc = T(0);
    bool first = true;
    for (int a = 0; a < kz; ++a)
      for (int b = 0; b < ky; ++b)
        for (int d = 0; d < kx; ++d) {
          const size_t e = cx[d] + (size_t)m.nx * (cy[b] + (size_t)m.ny * cz[a]);
          const T val = W[(e * NP3 + (lz[a] * NP + ly[b]) * NP + lx[d]) * n_vec + v];
          acc = first ? val : acc + val;
          first = false;
        }
    Y[idx] = acc;
  }
}

// Host: even-odd tables of an NO x NI row-major matrix M with symmetry S.
template <typename T, int NO, int NI>
void make_eotab(EOTab<T, NO, NI>& t, const double* M) {
  constexpr int HI = NI / 2, HO = (NO + 1) / 2, HE = (NI + 1) / 2;
  for (int o = 0; o < HO; ++o) {
    for (int i = 0; i < HI; ++i) {
      t.E[o][i] = (T)(0.5 * (M[o * NI + i] + M[o * NI + NI - 1 - i]));
      t.O[o][i] = (T)(0.5 * (M[o * NI + i] - M[o * NI + NI - 1 - i]));
    }
    if (HE > HI) t.E[o][HI] = (T)M[o * NI + HI];
  }
}

template <typename T, int NP, int NQ>
EOTables<T, NP, NQ> make_eotables(const fe_ctx* c) {
  EOTables<T, NP, NQ> t;
  double Nt[NP * NQ], Dt[NQ * NQ];
  for (int q = 0; q < NQ; ++q) {
    for (int i = 0; i < NP; ++i) Nt[i * NQ + q] = c->Nf[q * NP + i];
    for (int k = 0; k < NQ; ++k) Dt[k * NQ + q] = c->Df[q * NQ + k];
  }
  make_eotab<T, NQ, NP>(t.N, c->Nf.data());
  make_eotab<T, NP, NQ>(t.Nt, Nt);
  make_eotab<T, NQ, NQ>(t.D, c->Df.data());
  make_eotab<T, NQ, NQ>(t.Dt, Dt);
  return t;
}

template <typename T, int NP, int NQ, bool GEN, bool SC = false>
cudaError_t launch_apply_eo(const fe_ctx* c, const T* X, T* Y, int n_vec, cudaStream_t s, int want_vb,
                            int want_lines, const Scale<T>& sc = Scale<T>{}) {
  const void* kern;
  if constexpr (SC) kern = reinterpret_cast<const void*>(cell_apply_eo_scaled_kernel<T, NP, NQ, GEN>);
  else kern = reinterpret_cast<const void*>(cell_apply_eo_kernel<T, NP, NQ, GEN>);
  const int vb = pick_vb<T, NQ>(want_vb, n_vec);
  int nty = want_lines;
  if (vb * nty > 256) nty = 256 / vb;
  while ((vb * nty) % 32 != 0 && vb * nty < 256) ++nty;
  const size_t smem = (size_t)3 * NQ * NQ * NQ * vb * sizeof(T);
  {
    cudaError_t e = ensure_dyn_smem(reinterpret_cast<const void*>(kern), smem);
    if (e != cudaSuccess) return e;
  }
  const EOTables<T, NP, NQ> tab = make_eotables<T, NP, NQ>(c);
  const Geom<T> geo = make_geom<T>(c);
  if constexpr (!SC) {
    // Small meshes (scratch allocated at setup): one launch over all cells
    // (one vector per CTA, so even a few cells fill the GPU) writing each
    // cell's result to the scratch, then one gather in colour order.
    if (c->d_small && (size_t)n_vec * NP * NP * NP * c->n_cells * sizeof(T) <= c->small_bytes) {
      auto lk = cell_apply_eo_local_kernel<T, NP, NQ, GEN>;
      constexpr int lines = NQ * NQ < 64 ? 32 : 64;
      const size_t lsm = (size_t)3 * NQ * NQ * NQ * sizeof(T);
      cudaError_t e = ensure_dyn_smem(reinterpret_cast<const void*>(lk), lsm);
      if (e != cudaSuccess) return e;
      T* W = static_cast<T*>(c->d_small);
      lk<<<(unsigned)(c->n_cells * (size_t)n_vec), dim3(1, lines), lsm, s>>>(tab, c->mdev, geo, n_vec, n_vec, X, W);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      const size_t tot = c->n_dofs * (size_t)n_vec;
      assemble_local_kernel<T, NP><<<(unsigned)std::min<size_t>((tot + 255) / 256, 152 * 8), 256, 0, s>>>(
          c->mdev, W, Y, c->n_dofs, n_vec);
      return cudaGetLastError();
    }
  }
  const int n_vb = (n_vec + vb - 1) / vb;
  for (int k = 0; k < c->colors.n_colors; ++k) {
    const int n = c->colors.offset[k + 1] - c->colors.offset[k];
    if (n == 0) continue;
    const long long blocks = (long long)n * n_vb;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    if constexpr (SC)
      cell_apply_eo_scaled_kernel<T, NP, NQ, GEN><<<(unsigned)blocks, dim3(vb, nty), smem, s>>>(
          tab, c->mdev, geo, c->d_cells + c->colors.offset[k], n_vec, n_vb, X, Y, sc);
    else
      cell_apply_eo_kernel<T, NP, NQ, GEN><<<(unsigned)blocks, dim3(vb, nty), smem, s>>>(
          tab, c->mdev, geo, c->d_cells + c->colors.offset[k], n_vec, n_vb, X, Y);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace fe
