// Launch glue for the CUDA-core cell kernels: one instantiation per
// (p, n_q, geometry kind), selected at run time.
#pragma once

#include <cstdio>

#include "fe_cell_kernel.cuh"

namespace fe {

template <typename T, int NP, int NQ>
Tables<T, NP, NQ> make_tables(const fe_ctx* c) {
  Tables<T, NP, NQ> t;
  for (int q = 0; q < NQ; ++q) {
    for (int i = 0; i < NP; ++i) t.N[q][i] = (T)c->Nf[q * NP + i];
    for (int k = 0; k < NQ; ++k) t.D[q][k] = (T)c->Df[q * NQ + k];
  }
  return t;
}

template <typename T>
Geom<T> make_geom(const fe_ctx* c);
template <>
inline Geom<double> make_geom<double>(const fe_ctx* c) {
  return Geom<double>{c->d_cellG64, c->d_ptG64, c->d_ptC64};
}
template <>
inline Geom<float> make_geom<float>(const fe_ctx* c) {
  return Geom<float>{c->d_cellG32, c->d_ptG32, c->d_ptC32};
}

// Vectors per CTA: the largest power of two not above `want`, the padded
// n_vec, and what three n_q^3 x B tiles allow in 200 KB of shared memory.
template <typename T, int NQ>
inline int pick_vb(int want, int n_vec) {
  int vb = 1;
  while (vb * 2 <= want) vb *= 2;
  while (vb > 1 && (size_t)3 * NQ * NQ * NQ * vb * sizeof(T) > 200 * 1024) vb /= 2;
  while (vb > 1 && vb / 2 >= n_vec) vb /= 2;
  return vb;
}

template <typename T, int NP, int NQ, bool GEN, bool SC = false>
cudaError_t launch_apply(const fe_ctx* c, const T* X, T* Y, int n_vec, cudaStream_t s, int want_vb, int want_lines,
                         const Scale<T>& sc = Scale<T>{}) {
  const void* kern;
  if constexpr (SC) kern = reinterpret_cast<const void*>(cell_apply_scaled_kernel<T, NP, NQ, GEN>);
  else kern = reinterpret_cast<const void*>(cell_apply_kernel<T, NP, NQ, GEN>);
  const int vb = pick_vb<T, NQ>(want_vb, n_vec);
  int nty = want_lines;
  if (vb * nty > 256) nty = 256 / vb;
  while ((vb * nty) % 32 != 0 && vb * nty < 256) ++nty;
  const size_t smem = (size_t)3 * NQ * NQ * NQ * vb * sizeof(T);
  {
    cudaError_t e = ensure_dyn_smem(reinterpret_cast<const void*>(kern), smem);
    if (e != cudaSuccess) return e;
  }
  const Tables<T, NP, NQ> tab = make_tables<T, NP, NQ>(c);
  const Geom<T> geo = make_geom<T>(c);
  const int n_vb = (n_vec + vb - 1) / vb;
  for (int k = 0; k < c->colors.n_colors; ++k) {
    const int n = c->colors.offset[k + 1] - c->colors.offset[k];
    if (n == 0) continue;
    const long long blocks = (long long)n * n_vb;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    if constexpr (SC)
      cell_apply_scaled_kernel<T, NP, NQ, GEN><<<(unsigned)blocks, dim3(vb, nty), smem, s>>>(
          tab, c->mdev, geo, c->d_cells + c->colors.offset[k], n_vec, n_vb, X, Y, sc);
    else
      cell_apply_kernel<T, NP, NQ, GEN><<<(unsigned)blocks, dim3(vb, nty), smem, s>>>(
          tab, c->mdev, geo, c->d_cells + c->colors.offset[k], n_vec, n_vb, X, Y);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <int NP, int NQ, bool GEN>
cudaError_t launch_diag(const fe_ctx* c, double* diag, cudaStream_t s) {
  const Tables<double, NP, NQ> tab = make_tables<double, NP, NQ>(c);
  const Geom<double> geo = make_geom<double>(c);
  constexpr int NP3 = NP * NP * NP;
  for (int k = 0; k < c->colors.n_colors; ++k) {
    const int n = c->colors.offset[k + 1] - c->colors.offset[k];
    if (n == 0) continue;
    const long long threads = (long long)n * NP3;
    cell_diag_kernel<NP, NQ, GEN><<<(unsigned)((threads + 127) / 128), 128, 0, s>>>(
        tab, c->mdev, geo, c->d_cells + c->colors.offset[k], n, diag);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace fe

// Expands F(P, NQ) for every supported degree and quadrature size.
#define FE_FOR_EACH_P_NQ(F) \
  F(1, 2) F(1, 3) F(1, 4)   \
  F(2, 3) F(2, 4) F(2, 5)   \
  F(3, 4) F(3, 5) F(3, 6)   \
  F(4, 5) F(4, 6) F(4, 7)   \
  F(5, 6) F(5, 7) F(5, 8)   \
  F(6, 7) F(6, 8) F(6, 9)   \
  F(7, 8) F(7, 9) F(7, 10)  \
  F(8, 9) F(8, 10) F(8, 11)
