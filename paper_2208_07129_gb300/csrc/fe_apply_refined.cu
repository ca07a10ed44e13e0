// The product on refined meshes with hanging nodes (Sec. 3.2.2):
//   1. distribute: Xc = X with every slave row replaced by sum_m w_sm X_m
//      (u_S = W u_M; Dirichlet masters are already dropped from W);
//   2. the cell kernels with the explicit cell -> DoF map, colour by colour,
//      on Xc (first writers store, later colours add, Dirichlet rows 0);
//   3. condense: Y_m += sum_s w_sm Y_s for every master m (master rows, no
//      write conflicts);
//   4. slave rows of Y set to 0.
// Together Y = C^T A C X on the free rows, 0 on slave and Dirichlet rows.
#include "fe_dispatch.cuh"
#include "fe_evenodd.cuh"
#include "fe_ff_body.cuh"

namespace fe {

namespace {

template <typename T, typename W>
__global__ void distribute_kernel(const T* __restrict__ X, T* __restrict__ Xc, const int* __restrict__ row_slave,
                                  const int* __restrict__ ptr, const int* __restrict__ idx, const W* __restrict__ w,
                                  size_t n, int nv) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n * nv; i += (size_t)gridDim.x * blockDim.x) {
    const size_t r = i / nv;
    const int v = (int)(i - r * nv);
    const int s = __ldg(row_slave + r);
    if (s < 0) {
      Xc[i] = X[i];
      continue;
    }
    T acc = T(0);
    for (int k = __ldg(ptr + s); k < __ldg(ptr + s + 1); ++k) acc += (T)__ldg(w + k) * X[(size_t)__ldg(idx + k) * nv + v];
    Xc[i] = acc;
  }
}

template <typename T, typename W>
__global__ void condense_kernel(T* __restrict__ Y, const int* __restrict__ rows, const int* __restrict__ ptr,
                                const int* __restrict__ idx, const W* __restrict__ w, int n_rows, int nv) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)n_rows * nv;
       i += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(i / nv), v = (int)(i - (size_t)j * nv);
    T acc = T(0);
    for (int k = __ldg(ptr + j); k < __ldg(ptr + j + 1); ++k) acc += (T)__ldg(w + k) * Y[(size_t)__ldg(idx + k) * nv + v];
    Y[(size_t)__ldg(rows + j) * nv + v] += acc;
  }
}

template <typename T>
__global__ void zero_rows_kernel(T* __restrict__ Y, const int* __restrict__ rows, int n_rows, int nv) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)n_rows * nv;
       i += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(i / nv), v = (int)(i - (size_t)j * nv);
    Y[(size_t)__ldg(rows + j) * nv + v] = T(0);
  }
}

template <typename T, int NP, int NQ>
__global__ void __launch_bounds__(256) cell_apply_eo_map_kernel(const EOTables<T, NP, NQ> tab, const MeshDev m,
                                                                const Geom<T> geo, const int* __restrict__ cells,
                                                                int n_vec, int n_vb, const T* __restrict__ X,
                                                                T* __restrict__ Y, const int* __restrict__ map) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cell_body_eo<T, NP, NQ, false, false, true>(tab, m, geo, cells[blockIdx.x / n_vb], blockIdx.x % n_vb, blockDim.x,
                                              threadIdx.x, threadIdx.y, blockDim.y, n_vec, X, Y,
                                              reinterpret_cast<T*>(smem_raw), Scale<T>{}, map);
}

template <typename T, int NP, int NQ>
cudaError_t launch_eo_map(const fe_ctx* c, const T* X, T* Y, int n_vec, cudaStream_t s, int want_vb,
                          int want_lines) {
  auto kern = cell_apply_eo_map_kernel<T, NP, NQ>;
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
  const int n_vb = (n_vec + vb - 1) / vb;
  for (int k = 0; k < c->colors.n_colors; ++k) {
    const int n = c->colors.offset[k + 1] - c->colors.offset[k];
    if (n == 0) continue;
    const long long blocks = (long long)n * n_vb;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    kern<<<(unsigned)blocks, dim3(vb, nty), smem, s>>>(tab, c->mdev, geo, c->d_cells + c->colors.offset[k], n_vec,
                                                       n_vb, X, Y, c->d_map);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t cells_refined(const fe_ctx* c, const void* X, void* Y, int n_vec, cudaStream_t s) {
  const Scale<double> none{};
#define FE_CASE(P, NQ)                                                                                       \
  if (c->p == P && c->nq == NQ) {                                                                            \
    if (c->mode == FE_FP64)                                                                                  \
      return launch_eo_map<double, P + 1, NQ>(c, static_cast<const double*>(X), static_cast<double*>(Y),    \
                                              n_vec, s, c->vb64, c->nty64);                                  \
    if (c->mode == FE_FP32)                                                                                  \
      return launch_eo_map<float, P + 1, NQ>(c, static_cast<const float*>(X), static_cast<float*>(Y), n_vec, \
                                             s, c->vb32, c->nty32);                                          \
    return launch_df64<P + 1, NQ, false, false, true>(c, static_cast<const double*>(X),                      \
                                                      static_cast<double*>(Y), n_vec, s, none);              \
  }
  FE_FOR_EACH_P_NQ(FE_CASE)
#undef FE_CASE
  return cudaErrorInvalidValue;
}

template <typename T, typename W>
cudaError_t constrained(fe_ctx* c, const void* X, void* Y, int n_vec, cudaStream_t s, const W* sl_w, const W* ma_w,
                        void* xc) {
  const size_t n = c->n_dofs, tot = n * (size_t)n_vec;
  const void* Xin = X;
  if (c->n_slaves > 0) {
    const size_t bytes = tot * sizeof(T);
    if (!xc && c->xc_bytes < bytes) {
      cudaFree(c->d_xc);
      c->d_xc = nullptr;
      c->xc_bytes = 0;
      cudaError_t e = cudaMalloc(&c->d_xc, bytes);
      if (e != cudaSuccess) return e;
      c->xc_bytes = bytes;
    }
    if (!xc) xc = c->d_xc;
    const unsigned grid = (unsigned)std::min<size_t>((tot + 255) / 256, 152 * 16);
    distribute_kernel<T, W><<<grid, 256, 0, s>>>(static_cast<const T*>(X), static_cast<T*>(xc), c->d_row_slave,
                                                 c->d_sl_ptr, c->d_sl_idx, sl_w, n, n_vec);
    Xin = xc;
  }
  cudaError_t e = cells_refined(c, Xin, Y, n_vec, s);
  if (e != cudaSuccess) return e;
  if (c->n_masters > 0) {
    const size_t t = (size_t)c->n_masters * n_vec;
    condense_kernel<T, W><<<(unsigned)std::min<size_t>((t + 255) / 256, 152 * 16), 256, 0, s>>>(
        static_cast<T*>(Y), c->d_ma_rows, c->d_ma_ptr, c->d_ma_idx, ma_w, c->n_masters, n_vec);
  }
  if (c->n_slaves > 0) {
    const size_t t = (size_t)c->n_slaves * n_vec;
    zero_rows_kernel<T><<<(unsigned)std::min<size_t>((t + 255) / 256, 152 * 16), 256, 0, s>>>(
        static_cast<T*>(Y), c->d_slaves, c->n_slaves, n_vec);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t apply_refined(fe_ctx* c, const void* X, void* Y, int n_vec, cudaStream_t s, void* xc_scratch) {
  if (c->mode == FE_FP32) return constrained<float, float>(c, X, Y, n_vec, s, c->d_sl_w32, c->d_ma_w32, xc_scratch);
  return constrained<double, double>(c, X, Y, n_vec, s, c->d_sl_w, c->d_ma_w, xc_scratch);
}

}  // namespace fe
