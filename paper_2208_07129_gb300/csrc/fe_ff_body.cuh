// FE_DF64: FP64 data, the cell body in double-float arithmetic (fe_ff.cuh).
//
// Same data flow, tiles, tables and colour-ordered assembly as the FP64
// even-odd line kernel (fe_evenodd.cuh); only the arithmetic differs.  Every
// 1D contraction output is one compensated dot product (acc_first /
// acc_fma / acc_value), the even/odd pre- and post-combinations are
// double-float sums, and the quadrature-point operation is a compensated
// 3-term dot product.  X is split into hi + lo on the gather, results are
// added back to FP64 on the scatter, and the colour-ordered accumulation of
// Y stays in FP64.  Error: about 2^-44 relative per contraction, ~1e-14 on
// the product (against 1e-12 allowed for FP64).  Instantiated in
// fe_df64.cu (structured meshes) and fe_apply_refined.cu (explicit maps).
#pragma once

#include "fe_dispatch.cuh"
#include "fe_evenodd.cuh"

namespace fe {

template <int NO, int NI, int S>
__device__ __forceinline__ void eo_apply_ff(const EOTab<ff, NO, NI>& t, const ff* in, ff* out) {
  constexpr int HI = NI / 2, HO = (NO + 1) / 2, HE = (NI + 1) / 2;
  ff ie[HE], io[HI > 0 ? HI : 1];
#pragma unroll
  for (int i = 0; i < HI; ++i) {
    ie[i] = ff_add(in[i], in[NI - 1 - i]);
    io[i] = ff_sub(in[i], in[NI - 1 - i]);
  }
  if (NI & 1) ie[HI] = in[HI];
#pragma unroll
  for (int o = 0; o < HO; ++o) {
    ffacc e = acc_first(t.E[o][0], ie[0]);
#pragma unroll
    for (int i = 1; i < HE; ++i) acc_fma(e, t.E[o][i], ie[i]);
    const ff E = acc_value(e);
    if (HI > 0) {
      ffacc d = acc_first(t.O[o][0], io[0]);
#pragma unroll
      for (int i = 1; i < HI; ++i) acc_fma(d, t.O[o][i], io[i]);
      const ff D = acc_value(d);
      out[o] = ff_add(E, D);
      if (o != NO - 1 - o) out[NO - 1 - o] = S > 0 ? ff_sub(E, D) : ff_sub(D, E);
    } else {
      out[o] = E;
      if (o != NO - 1 - o) out[NO - 1 - o] = S > 0 ? E : ff(-E.hi, -E.lo);
    }
  }
}

// SC: the scaled product of the Chebyshev filter (see Scale); the M^-1/2
// scalings and the b X + c Y terms are applied in FP64 at the gather and the
// scatter.
template <int NP, int NQ, bool GEN, bool SC, bool MAP = false>
__device__ __forceinline__ void cell_body_ff(const EOTables<ff, NP, NQ>& tab, const MeshDev& m, const Geom<ff>& geo,
                                             int e, int vb, int B, int v, int ty, int nty, int n_vec,
                                             const double* __restrict__ X, double* __restrict__ Y, ff* smem,
                                             const Scale<double>& sc, const int* __restrict__ map = nullptr) {
  constexpr int P = NP - 1;
  constexpr int NQ3 = NQ * NQ * NQ;
  ff* ST = smem;
  ff* S0 = ST + NQ3 * B;
  ff* S1 = S0 + NQ3 * B;
  const int vg = vb * B + v;
  const bool active = vg < n_vec;
  const int cx = e % m.nx, cy = (e / m.nx) % m.ny, cz = e / (m.nx * m.ny);

  // ---- extraction fused with the x pass of N:  S0[i3][i2][q1] ----
  for (int l = ty; l < NP * NP; l += nty) {
    const int i2 = l % NP, i3 = l / NP;
    const int gy = node_coord(cy, i2, P, m.Ny, m.periodic), gz = node_coord(cz, i3, P, m.Nz, m.periodic);
    const bool con_yz = on_boundary(gy, m.Ny, m.periodic) || on_boundary(gz, m.Nz, m.periodic);
    const size_t row = (size_t)(gy + (size_t)m.Ny * gz) * m.Nx;
    ff u[NP], a[NQ];
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
      double x = (active && !con) ? __ldg(X + node * n_vec + vg) : 0.0;
      if constexpr (SC) x *= __ldg(sc.msq + node);
      u[i1] = ff(x);
    }
    eo_apply_ff<NQ, NP, 1>(tab.N, u, a);
#pragma unroll
    for (int q = 0; q < NQ; ++q) S0[((i3 * NP + i2) * NQ + q) * B + v] = a[q];
  }
  __syncthreads();
  // ---- y pass of N:  S1[i3][q2][q1] ----
  for (int l = ty; l < NQ * NP; l += nty) {
    const int q1 = l % NQ, i3 = l / NQ;
    ff a[NP], b[NQ];
#pragma unroll
    for (int i = 0; i < NP; ++i) a[i] = S0[((i3 * NP + i) * NQ + q1) * B + v];
    eo_apply_ff<NQ, NP, 1>(tab.N, a, b);
#pragma unroll
    for (int q = 0; q < NQ; ++q) S1[((i3 * NQ + q) * NQ + q1) * B + v] = b[q];
  }
  __syncthreads();
  // ---- z pass of N:  ST[q3][q2][q1] ----
  for (int l = ty; l < NQ * NQ; l += nty) {
    ff a[NP], b[NQ];
#pragma unroll
    for (int i = 0; i < NP; ++i) a[i] = S1[(i * NQ * NQ + l) * B + v];
    eo_apply_ff<NQ, NP, 1>(tab.N, a, b);
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
    ff t[NQ], g[NQ];
#pragma unroll
    for (int k = 0; k < NQ; ++k) t[k] = ST[(base + k * stride) * B + v];
    eo_apply_ff<NQ, NQ, -1>(tab.D, t, g);
    ff* dst = ydir ? S1 : S0;
#pragma unroll
    for (int q = 0; q < NQ; ++q) dst[(base + q * stride) * B + v] = g[q];
  }
  __syncthreads();
  // ---- z-lines: gradient along z, quadrature-point operation, transposed z pass ----
  // cells without per-point geometry are axis-aligned boxes: diagonal metric
  ff g00, g01, g02, g11, g12, g22;
  if (!GEN) {
    g00 = geo.cellG[e * 6 + 0]; g11 = geo.cellG[e * 6 + 3]; g22 = geo.cellG[e * 6 + 5];
  }
  const ff* ptC = geo.ptC + (size_t)e * NQ3;
  for (int l = ty; l < NQ * NQ; l += nty) {
    ff t[NQ], h2[NQ], o[NQ];
#pragma unroll
    for (int k = 0; k < NQ; ++k) t[k] = ST[(k * NQ * NQ + l) * B + v];
    eo_apply_ff<NQ, NQ, -1>(tab.D, t, h2);
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const ff d2 = h2[q];
      const int Q = q * NQ * NQ + l;
      const ff d0 = S0[Q * B + v], d1 = S1[Q * B + v];
      if (GEN) {
        const ff* pg = geo.ptG + (size_t)e * 6 * NQ3 + Q;
        g00 = pg[0]; g01 = pg[NQ3]; g02 = pg[2 * NQ3]; g11 = pg[3 * NQ3]; g12 = pg[4 * NQ3]; g22 = pg[5 * NQ3];
        ffacc r0 = acc_first(g00, d0), r1 = acc_first(g01, d0), r2 = acc_first(g02, d0);
        acc_fma(r0, g01, d1); acc_fma(r0, g02, d2);
        acc_fma(r1, g11, d1); acc_fma(r1, g12, d2);
        acc_fma(r2, g12, d1); acc_fma(r2, g22, d2);
        S0[Q * B + v] = acc_value(r0);
        S1[Q * B + v] = acc_value(r1);
        h2[q] = acc_value(r2);
      } else {
        S0[Q * B + v] = ff_mul(g00, d0);
        S1[Q * B + v] = ff_mul(g11, d1);
        h2[q] = ff_mul(g22, d2);
      }
      t[q] = ff_mul(ptC[Q], t[q]);
    }
    eo_apply_ff<NQ, NQ, -1>(tab.Dt, h2, o);
#pragma unroll
    for (int k = 0; k < NQ; ++k) ST[(k * NQ * NQ + l) * B + v] = ff_add(t[k], o[k]);
  }
  __syncthreads();
  // ---- transposed x pass of D~ accumulated into T ----
  for (int l = ty; l < NQ * NQ; l += nty) {
    const int base = l * NQ;
    ff h[NQ], o[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) h[q] = S0[(base + q) * B + v];
    eo_apply_ff<NQ, NQ, -1>(tab.Dt, h, o);
#pragma unroll
    for (int k = 0; k < NQ; ++k) ST[(base + k) * B + v] = ff_add(ST[(base + k) * B + v], o[k]);
  }
  __syncthreads();
  // ---- transposed y pass of D~ accumulated into T ----
  for (int l = ty; l < NQ * NQ; l += nty) {
    const int base = (l % NQ) + (l / NQ) * NQ * NQ;
    ff h[NQ], o[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) h[q] = S1[(base + q * NQ) * B + v];
    eo_apply_ff<NQ, NQ, -1>(tab.Dt, h, o);
#pragma unroll
    for (int k = 0; k < NQ; ++k) ST[(base + k * NQ) * B + v] = ff_add(ST[(base + k * NQ) * B + v], o[k]);
  }
  __syncthreads();
  // ---- transposed z pass of N:  S1[i3][q2][q1] ----
  for (int l = ty; l < NQ * NQ; l += nty) {
    ff t[NQ], o[NP];
#pragma unroll
    for (int q = 0; q < NQ; ++q) t[q] = ST[(q * NQ * NQ + l) * B + v];
    eo_apply_ff<NP, NQ, 1>(tab.Nt, t, o);
#pragma unroll
    for (int i = 0; i < NP; ++i) S1[(i * NQ * NQ + l) * B + v] = o[i];
  }
  __syncthreads();
  // ---- transposed y pass of N:  S0[i3][i2][q1] ----
  for (int l = ty; l < NQ * NP; l += nty) {
    const int q1 = l % NQ, i3 = l / NQ;
    ff t[NQ], o[NP];
#pragma unroll
    for (int q = 0; q < NQ; ++q) t[q] = S1[((i3 * NQ + q) * NQ + q1) * B + v];
    eo_apply_ff<NP, NQ, 1>(tab.Nt, t, o);
#pragma unroll
    for (int i = 0; i < NP; ++i) S0[((i3 * NP + i) * NQ + q1) * B + v] = o[i];
  }
  __syncthreads();
  // ---- transposed x pass of N fused with assembly (FP64) ----
  for (int l = ty; l < NP * NP; l += nty) {
    const int i2 = l % NP, i3 = l / NP;
    ff t[NQ], o[NP];
#pragma unroll
    for (int q = 0; q < NQ; ++q) t[q] = S0[((i3 * NP + i2) * NQ + q) * B + v];
    if (!active) continue;
    eo_apply_ff<NP, NQ, 1>(tab.Nt, t, o);
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
      double* dst = Y + node * n_vec + vg;
      if constexpr (SC) {
        scaled_store(dst, X + node * n_vec + vg, sc.a * __ldg(sc.msq + node) * ff_to_double(o[i]), first, con, sc);
      } else {
        if (first) *dst = con ? 0.0 : ff_to_double(o[i]);
        else if (!con) *dst += ff_to_double(o[i]);
      }
    }
  }
}

template <int NP, int NQ, bool GEN, bool SC, bool MAP>
__global__ void __launch_bounds__(256) cell_apply_df64_kernel(const EOTables<ff, NP, NQ> tab, const MeshDev m,
                                                              const Geom<ff> geo, const int* __restrict__ cells,
                                                              int n_vec, int n_vb, const double* __restrict__ X,
                                                              double* __restrict__ Y, const Scale<double> sc,
                                                              const int* __restrict__ map) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cell_body_ff<NP, NQ, GEN, SC, MAP>(tab, m, geo, cells[blockIdx.x / n_vb], blockIdx.x % n_vb, blockDim.x,
                                     threadIdx.x, threadIdx.y, blockDim.y, n_vec, X, Y,
                                     reinterpret_cast<ff*>(smem_raw), sc, map);
}

template <int NP, int NQ, bool GEN, bool SC, bool MAP = false>
cudaError_t launch_df64(const fe_ctx* c, const double* X, double* Y, int n_vec, cudaStream_t s,
                        const Scale<double>& sc) {
  auto kern = cell_apply_df64_kernel<NP, NQ, GEN, SC, MAP>;
  const int vb = pick_vb<double, NQ>(c->vbdf, n_vec);   // ff tiles take the bytes of FP64 tiles
  int nty = c->ntydf;
  if (vb * nty > 256) nty = 256 / vb;
  while ((vb * nty) % 32 != 0 && vb * nty < 256) ++nty;
  const size_t smem = (size_t)3 * NQ * NQ * NQ * vb * sizeof(ff);
  {
    cudaError_t e = ensure_dyn_smem(reinterpret_cast<const void*>(kern), smem);
    if (e != cudaSuccess) return e;
  }
  const EOTables<ff, NP, NQ> tab = make_eotables<ff, NP, NQ>(c);
  const Geom<ff> geo{c->d_cellGff, c->d_ptGff, c->d_ptCff};
  const int n_vb = (n_vec + vb - 1) / vb;
  for (int k = 0; k < c->colors.n_colors; ++k) {
    const int n = c->colors.offset[k + 1] - c->colors.offset[k];
    if (n == 0) continue;
    const long long blocks = (long long)n * n_vb;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    kern<<<(unsigned)blocks, dim3(vb, nty), smem, s>>>(tab, c->mdev, geo, c->d_cells + c->colors.offset[k], n_vec,
                                                       n_vb, X, Y, sc, c->d_map);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}


}  // namespace fe
