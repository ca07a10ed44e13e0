// Block preconditioned conjugate gradients for A X = B (one CG recurrence per
// column, all columns advanced together), with a Jacobi or learned
// preconditioner, in FP64 or as FP64 iterative refinement around an FP32
// inner solve.  The paper points to block Krylov methods for many right-hand
// sides (Sec. 5); the operator is the matrix-free fe_apply.
//
// Every vector kernel streams DoF-major (n x nv) blocks with the column index
// contiguous.  Column reductions are deterministic: each CTA writes one
// partial sum per column to a scratch array, a second kernel sums the partials
// of each column in a fixed order.
#include <cmath>
#include <cstring>
#include <vector>

#include "fe_internal.h"

namespace fe {

constexpr int kRedBlocks = 304;   // 2 x 152 SMs
constexpr int kColTile = 32;

// ---------------------------------------------------------------------------
// column reductions
// ---------------------------------------------------------------------------

// partial[b * nv + c] = sum over rows of CTA b of f(row, c), f = a*b or a*a.
template <typename T>
__global__ void col_dot_partial(const T* __restrict__ a, const T* __restrict__ b, size_t n, int nv,
                                double* __restrict__ partial) {
  __shared__ double red[8][kColTile];
  const int c = blockIdx.y * kColTile + threadIdx.x;
  double s = 0.0;
  if (c < nv) {
    const size_t rows_per = (n + gridDim.x - 1) / gridDim.x;
    const size_t r0 = (size_t)blockIdx.x * rows_per;
    const size_t r1 = r0 + rows_per < n ? r0 + rows_per : n;
    const size_t st = blockDim.y;
    size_t r = r0 + threadIdx.y;
    double s2 = 0.0;
    for (; r + st < r1; r += 2 * st) {   // two rows in flight per thread
      const size_t i = r * nv + c, j = (r + st) * nv + c;
      s += (double)a[i] * (double)b[i];
      s2 += (double)a[j] * (double)b[j];
    }
    if (r < r1) s += (double)a[r * nv + c] * (double)b[r * nv + c];
    s += s2;
  }
  red[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && c < nv) {
    for (int k = 1; k < (int)blockDim.y; ++k) s += red[k][threadIdx.x];
    partial[(size_t)blockIdx.x * nv + c] = s;
  }
}

// out[c] = sum_b partial[b * nv + c] (fixed order).
__global__ void col_sum_partials(const double* __restrict__ partial, int nblocks, int nv, double* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nv) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += partial[(size_t)b * nv + c];
  out[c] = s;
}

template <typename T>
cudaError_t col_dot(const T* a, const T* b, size_t n, int nv, double* partial, double* out, cudaStream_t s);

// ---------------------------------------------------------------------------
// wide variants: 16-byte accesses (4 floats or 2 doubles of consecutive
// columns per thread) and enough CTAs to fill every SM, for blocks whose
// column count is a multiple of the vector width.  Same deterministic
// per-CTA partials, summed in a fixed order.
// ---------------------------------------------------------------------------

constexpr int kWideBlocks = 152 * 8;

template <typename T>
struct Wide;
template <>
struct Wide<float> {
  using V = float4;
  static constexpr int N = 4;
  __device__ static float get(const V& v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }
  __device__ static void set(V& v, int k, float x) {
    if (k == 0) v.x = x; else if (k == 1) v.y = x; else if (k == 2) v.z = x; else v.w = x;
  }
};
template <>
struct Wide<double> {
  using V = double2;
  static constexpr int N = 2;
  __device__ static double get(const V& v, int k) { return k == 0 ? v.x : v.y; }
  __device__ static void set(V& v, int k, double x) {
    if (k == 0) v.x = x; else v.y = x;
  }
};

template <typename T>
inline bool wide_ok(int nv, const void* const* ptrs, int n_ptrs) {
  if (nv % Wide<T>::N != 0) return false;
  for (int k = 0; k < n_ptrs; ++k)
    if (ptrs[k] && (reinterpret_cast<uintptr_t>(ptrs[k]) & 15) != 0) return false;
  return true;
}

// Rows of CTA b: [b * rows_per, ...); thread (x, y): column group x of the
// CTA's column tile (32 groups of Wide<T>::N columns), rows y, y + 8, ...
#define FE_WIDE_PROLOGUE(T)                                                            \
  using W = Wide<T>;                                                                   \
  using V = typename W::V;                                                             \
  const int ncg = nv / W::N;                                                           \
  const int cg = blockIdx.y * 32 + threadIdx.x;                                        \
  const bool col_ok = cg < ncg;                                                        \
  const size_t rows_per = (n + gridDim.x - 1) / gridDim.x;                             \
  const size_t r0 = (size_t)blockIdx.x * rows_per;                                     \
  const size_t r1 = r0 + rows_per < n ? r0 + rows_per : n;

// Per-thread column sums of products.  FP64 blocks accumulate in FP64.  FP32
// blocks accumulate in FP32 with Kahan's compensation (the running error is
// fed back into the next term, so the sum is accurate to a few FP32 ulps
// whatever its length) and are converted to FP64 once, for the cross-thread
// reduction: GB300 runs FP64 at 1/64 of the FP32 rate, and two conversions
// plus an FP64 multiply-add per element would bound these streaming kernels.
template <typename T>
struct ColAcc;
template <>
struct ColAcc<double> {
  double s = 0.0;
  __device__ void add(double a, double b) { s = fma(a, b, s); }
  __device__ double value() const { return s; }
};
template <>
struct ColAcc<float> {
  float s = 0.f, c = 0.f;
  __device__ void add(float a, float b) {
    const float y = __fsub_rn(__fmul_rn(a, b), c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
  __device__ double value() const { return (double)s - (double)c; }
};

// partial[b][c] over columns c of the thread's group
template <typename T>
__device__ __forceinline__ void wide_store_partials(double (&s)[Wide<T>::N], bool col_ok, int cg, int nv,
                                                    double* __restrict__ partial) {
  __shared__ double red[8][32][Wide<T>::N];
#pragma unroll
  for (int k = 0; k < Wide<T>::N; ++k) red[threadIdx.y][threadIdx.x][k] = s[k];
  __syncthreads();
  if (threadIdx.y == 0 && col_ok) {
#pragma unroll
    for (int k = 0; k < Wide<T>::N; ++k) {
      double t = s[k];
      for (int y = 1; y < 8; ++y) t += red[y][threadIdx.x][k];
      partial[(size_t)blockIdx.x * nv + cg * Wide<T>::N + k] = t;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) col_dot_partial_wide(const T* __restrict__ a, const T* __restrict__ b,
                                                            size_t n, int nv, double* __restrict__ partial) {
  FE_WIDE_PROLOGUE(T)
  ColAcc<T> acc[W::N];
  if (col_ok) {
    for (size_t r = r0 + threadIdx.y; r < r1; r += 8) {
      const V va = reinterpret_cast<const V*>(a + r * nv)[cg];
      const V vb = reinterpret_cast<const V*>(b + r * nv)[cg];
#pragma unroll
      for (int k = 0; k < W::N; ++k) acc[k].add(W::get(va, k), W::get(vb, k));
    }
  }
  double s[W::N];
#pragma unroll
  for (int k = 0; k < W::N; ++k) s[k] = acc[k].value();
  wide_store_partials<T>(s, col_ok, cg, nv, partial);
}

// x += alpha_c p, r -= alpha_c q, z = dinv .* r, partial r.z (one pass)
template <typename T>
__global__ void __launch_bounds__(256) cg_step_kernel_wide(T* __restrict__ x, T* __restrict__ r, T* __restrict__ z,
                                                           const T* __restrict__ p, const T* __restrict__ q,
                                                           const T* __restrict__ dinv,
                                                           const double* __restrict__ alpha, size_t n, int nv,
                                                           double* __restrict__ partial) {
  FE_WIDE_PROLOGUE(T)
  ColAcc<T> acc[W::N];
  if (col_ok) {
    T a[W::N];
#pragma unroll
    for (int k = 0; k < W::N; ++k) a[k] = (T)alpha[cg * W::N + k];
    for (size_t row = r0 + threadIdx.y; row < r1; row += 8) {
      const size_t o = row * nv;
      V vx = reinterpret_cast<const V*>(x + o)[cg];
      V vr = reinterpret_cast<const V*>(r + o)[cg];
      const V vp = reinterpret_cast<const V*>(p + o)[cg];
      const V vq = reinterpret_cast<const V*>(q + o)[cg];
      const T d = dinv ? dinv[row] : T(1);
      V vz;
#pragma unroll
      for (int k = 0; k < W::N; ++k) {
        W::set(vx, k, W::get(vx, k) + a[k] * W::get(vp, k));
        const T rn = W::get(vr, k) - a[k] * W::get(vq, k);
        W::set(vr, k, rn);
        const T zn = rn * d;
        W::set(vz, k, zn);
        acc[k].add(rn, zn);
      }
      reinterpret_cast<V*>(x + o)[cg] = vx;
      reinterpret_cast<V*>(r + o)[cg] = vr;
      reinterpret_cast<V*>(z + o)[cg] = vz;
    }
  }
  double s[W::N];
#pragma unroll
  for (int k = 0; k < W::N; ++k) s[k] = acc[k].value();
  wide_store_partials<T>(s, col_ok, cg, nv, partial);
}

// p = z + beta_c p
template <typename T>
__global__ void __launch_bounds__(256) cg_direction_kernel_wide(T* __restrict__ p, const T* __restrict__ z,
                                                                const double* __restrict__ beta, size_t n, int nv) {
  FE_WIDE_PROLOGUE(T)
  if (!col_ok) return;
  T bc[W::N];
#pragma unroll
  for (int k = 0; k < W::N; ++k) bc[k] = (T)beta[cg * W::N + k];
  for (size_t row = r0 + threadIdx.y; row < r1; row += 8) {
    const size_t o = row * nv;
    V vp = reinterpret_cast<const V*>(p + o)[cg];
    const V vz = reinterpret_cast<const V*>(z + o)[cg];
#pragma unroll
    for (int k = 0; k < W::N; ++k) W::set(vp, k, W::get(vz, k) + bc[k] * W::get(vp, k));
    reinterpret_cast<V*>(p + o)[cg] = vp;
  }
}
// x += alpha_c p, r -= alpha_c q  (learned preconditioner: z comes from the network)
template <typename T>
__global__ void __launch_bounds__(256) cg_update_kernel_wide(T* __restrict__ x, T* __restrict__ r,
                                                             const T* __restrict__ p, const T* __restrict__ q,
                                                             const double* __restrict__ alpha, size_t n, int nv) {
  FE_WIDE_PROLOGUE(T)
  if (!col_ok) return;
  T a[W::N];
#pragma unroll
  for (int k = 0; k < W::N; ++k) a[k] = (T)alpha[cg * W::N + k];
  for (size_t row = r0 + threadIdx.y; row < r1; row += 8) {
    const size_t o = row * nv;
    V vx = reinterpret_cast<const V*>(x + o)[cg];
    V vr = reinterpret_cast<const V*>(r + o)[cg];
    const V vp = reinterpret_cast<const V*>(p + o)[cg];
    const V vq = reinterpret_cast<const V*>(q + o)[cg];
#pragma unroll
    for (int k = 0; k < W::N; ++k) {
      W::set(vx, k, W::get(vx, k) + a[k] * W::get(vp, k));
      W::set(vr, k, W::get(vr, k) - a[k] * W::get(vq, k));
    }
    reinterpret_cast<V*>(x + o)[cg] = vx;
    reinterpret_cast<V*>(r + o)[cg] = vr;
  }
}

// z = dinv .* r on the columns whose r.z is not positive (descent safeguard of
// flexible CG); other columns are left as they are and not even read.
template <typename T>
__global__ void __launch_bounds__(256) fcg_safeguard_kernel_wide(const T* __restrict__ r, const T* __restrict__ dinv,
                                                                 T* __restrict__ z, const double* __restrict__ rz,
                                                                 size_t n, int nv) {
  FE_WIDE_PROLOGUE(T)
  if (!col_ok) return;
  bool bad[W::N], any = false;
#pragma unroll
  for (int k = 0; k < W::N; ++k) {
    bad[k] = !(rz[cg * W::N + k] > 0.0);
    any = any || bad[k];
  }
  if (!any) return;
  for (size_t row = r0 + threadIdx.y; row < r1; row += 8) {
    const size_t o = row * nv;
    const V vr = reinterpret_cast<const V*>(r + o)[cg];
    V vz = reinterpret_cast<const V*>(z + o)[cg];
    const T d = dinv[row];
#pragma unroll
    for (int k = 0; k < W::N; ++k)
      if (bad[k]) W::set(vz, k, W::get(vr, k) * d);
    reinterpret_cast<V*>(z + o)[cg] = vz;
  }
}
#undef FE_WIDE_PROLOGUE

// out[c] = sum_b partial[b * nv + c]: one warp per column, lane l adds the
// partials l, l + 32, ... in order, then a fixed butterfly (deterministic).
__global__ void col_sum_partials_warp(const double* __restrict__ partial, int nblocks, int nv,
                                      double* __restrict__ out) {
  const int c = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
  if (c >= nv) return;
  double s = 0.0;
  for (int b = lane; b < nblocks; b += 32) s += partial[(size_t)b * nv + c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[c] = s;
}

inline dim3 wide_grid(int nv, int vec) { return dim3(kWideBlocks, (unsigned)((nv / vec + 31) / 32)); }

template <typename T>
cudaError_t col_dot(const T* a, const T* b, size_t n, int nv, double* partial, double* out, cudaStream_t s) {
  const void* ptrs[2] = {a, b};
  if (wide_ok<T>(nv, ptrs, 2)) {
    col_dot_partial_wide<T><<<wide_grid(nv, Wide<T>::N), dim3(32, 8), 0, s>>>(a, b, n, nv, partial);
    col_sum_partials_warp<<<(nv + 7) / 8, 256, 0, s>>>(partial, kWideBlocks, nv, out);
    return cudaGetLastError();
  }
  dim3 grid(kRedBlocks, (nv + kColTile - 1) / kColTile);
  col_dot_partial<T><<<grid, dim3(kColTile, 8), 0, s>>>(a, b, n, nv, partial);
  col_sum_partials<<<(nv + 127) / 128, 128, 0, s>>>(partial, kRedBlocks, nv, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// element-wise kernels
// ---------------------------------------------------------------------------

// r = b - r   (r holds A x on entry)
template <typename T>
__global__ void residual_kernel(const T* __restrict__ b, T* __restrict__ r, size_t total) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
    r[i] = b[i] - r[i];
}

// z = dinv .* r (row scaling, dinv per DoF) or z = r
template <typename T>
__global__ void precond_jacobi_kernel(const T* __restrict__ r, const T* __restrict__ dinv, T* __restrict__ z,
                                      size_t n, int nv) {
  const size_t total = n * nv;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
    z[i] = dinv ? r[i] * dinv[i / nv] : r[i];
}

// x += alpha_c p ; r -= alpha_c q
template <typename T>
__global__ void cg_update_kernel(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p,
                                 const T* __restrict__ q, const double* __restrict__ alpha, size_t total, int nv) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const T a = (T)alpha[i % nv];
    x[i] += a * p[i];
    r[i] -= a * q[i];
  }
}

// p = z + beta_c p   (column-structured like the reductions: no index division)
template <typename T>
__global__ void cg_direction_kernel(T* __restrict__ p, const T* __restrict__ z, const double* __restrict__ beta,
                                    size_t n, int nv) {
  const int c = blockIdx.y * kColTile + threadIdx.x;
  if (c >= nv) return;
  const T bc = (T)beta[c];
  const size_t rows_per = (n + gridDim.x - 1) / gridDim.x;
  const size_t r0 = (size_t)blockIdx.x * rows_per;
  const size_t r1 = r0 + rows_per < n ? r0 + rows_per : n;
  for (size_t r = r0 + threadIdx.y; r < r1; r += blockDim.y) {
    const size_t i = r * nv + c;
    p[i] = z[i] + bc * p[i];
  }
}

// One pass of the PCG step after alpha is known (Jacobi or no preconditioner):
//   x += alpha_c p,  r -= alpha_c q,  z = dinv .* r,  partial[b][c] = sum r.z
// (the separate update, preconditioner and dot-product kernels read r and z
// again; fused they stream every vector once).
template <typename T>
__global__ void cg_step_kernel(T* __restrict__ x, T* __restrict__ r, T* __restrict__ z, const T* __restrict__ p,
                               const T* __restrict__ q, const T* __restrict__ dinv, const double* __restrict__ alpha,
                               size_t n, int nv, double* __restrict__ partial) {
  __shared__ double red[8][kColTile];
  const int c = blockIdx.y * kColTile + threadIdx.x;
  double s = 0.0;
  if (c < nv) {
    const T a = (T)alpha[c];
    const size_t rows_per = (n + gridDim.x - 1) / gridDim.x;
    const size_t r0 = (size_t)blockIdx.x * rows_per;
    const size_t r1 = r0 + rows_per < n ? r0 + rows_per : n;
    for (size_t row = r0 + threadIdx.y; row < r1; row += blockDim.y) {
      const size_t i = row * nv + c;
      x[i] += a * p[i];
      const T rn = r[i] - a * q[i];
      r[i] = rn;
      const T zn = dinv ? rn * dinv[row] : rn;
      z[i] = zn;
      s += (double)rn * (double)zn;
    }
  }
  red[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && c < nv) {
    for (int k = 1; k < (int)blockDim.y; ++k) s += red[k][threadIdx.x];
    partial[(size_t)blockIdx.x * nv + c] = s;
  }
}

// alpha = active ? rz / pq : 0 ; flags a breakdown when pq <= 0 on an active column
__global__ void cg_alpha_kernel(const double* rz, const double* pq, const int* active, double* alpha, int nv,
                                int* status) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nv) return;
  double a = 0.0;
  if (active[c]) {
    if (!(pq[c] > 0.0) || !isfinite(pq[c])) {
      atomicMax(status, (int)FE_EBREAKDOWN);
    } else {
      a = rz[c] / pq[c];
    }
  }
  alpha[c] = a;
}

// beta = rz_new / rz_old (standard PCG) or, for a variable preconditioner,
// beta = -(z_new . A p) / (p . A p) (flexible CG, Notay 2000); then rz_old = rz_new.
__global__ void cg_beta_kernel(const double* rz_new, const double* zq, const double* pq, double* rz_old,
                               const int* active, double* beta, int nv, int flexible) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nv) return;
  double b = 0.0;
  if (active[c]) {
    if (flexible) b = pq[c] > 0.0 ? -zq[c] / pq[c] : 0.0;
    else if (rz_old[c] != 0.0) b = rz_new[c] / rz_old[c];
  }
  beta[c] = b;
  rz_old[c] = rz_new[c];
}

// dst = (T) (src * scale_c)  between precisions, per-column scale
template <typename TD, typename TS>
__global__ void scale_convert_kernel(TD* __restrict__ dst, const TS* __restrict__ src, const double* __restrict__ scale,
                                     size_t total, int nv, int add) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const double v = (double)src[i] * (scale ? scale[i % nv] : 1.0);
    if (add) dst[i] = (TD)((double)dst[i] + v);
    else dst[i] = (TD)v;
  }
}

__global__ void inv_kernel(const double* d, double* dinv64, float* dinv32, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double v = 1.0 / d[i];
    dinv64[i] = v;
    dinv32[i] = (float)v;
  }
}

inline unsigned ew_grid(size_t total) {
  size_t g = (total + 255) / 256;
  return (unsigned)(g < 152 * 16 ? (g ? g : 1) : 152 * 16);
}

}  // namespace fe

using namespace fe;

namespace {

fe_status from_cuda(cudaError_t e) {
  return fe::cuda_status(e);
}

template <typename T>
cudaError_t grow(T** p, size_t* cap, size_t n) {
  if (*cap >= n) return cudaSuccess;
  cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  cudaError_t e = cudaMalloc(p, n * sizeof(T));
  if (e == cudaSuccess) *cap = n;
  return e;
}

}  // namespace

namespace fe {

cudaError_t solver_workspace(fe_ctx* c, int nv) {
  SolveWs& w = c->ws;
  const size_t n = c->n_dofs, tot = n * (size_t)nv;
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = grow(&w.v64[k], &w.cap64[k], tot);
  for (int k = 0; k < 6 && e == cudaSuccess; ++k) e = grow(&w.v32[k], &w.cap32[k], tot);
  if (e == cudaSuccess) e = grow(&w.colbuf, &w.cap_col, (size_t)nv * 12);
  if (e == cudaSuccess) e = grow(&w.partial, &w.cap_partial, (size_t)kWideBlocks * nv);
  if (e == cudaSuccess) e = grow(&w.active, &w.cap_active, (size_t)nv);
  if (e == cudaSuccess && !w.dinv64) {
    e = cudaMalloc(&w.dinv64, n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&w.dinv32, n * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&w.diag, n * sizeof(double));
    if (e == cudaSuccess) e = diagonal_f64(c, w.diag, 0);
    if (e == cudaSuccess) inv_kernel<<<ew_grid(n), 256>>>(w.diag, w.dinv64, w.dinv32, n);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  }
  return e;
}

// Mode-typed apply through the public entry (keeps the kernel dispatch in one place).
template <typename T>
static fe_status apply_mode(fe_ctx* c, const T* X, T* Y, int nv, cudaStream_t s) {
  const fe_mode saved = c->mode;
  c->mode = sizeof(T) == 8 ? c->op64 : c->inner_mode;
  fe_status st = fe_apply(c, X, Y, nv, s);
  c->mode = saved;
  return st;
}

// One preconditioned CG solve in precision T for A x = b with x0 = x (in/out).
// Stops when every column has ||r_j|| <= tol_j (recurrence residual) or after
// max_it iterations.  Returns the iterations performed.
using PcgHook = void (*)(void* user, int it, const void* x, const void* r, cudaStream_t s);

// With the learned (nonlinear) preconditioner, columns whose r.z is not
// positive fall back to the Jacobi direction (descent safeguard).
template <typename T>
__global__ void fcg_safeguard_kernel(const T* __restrict__ r, const T* __restrict__ dinv, T* __restrict__ z,
                                     const double* __restrict__ rz, size_t total, int nv) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
    if (!(rz[i % nv] > 0.0)) z[i] = r[i] * dinv[i / nv];
}

template <typename T>
fe_status pcg(fe_ctx* c, const T* b, T* x, int nv, const double* tol_host, int max_it, int precond, cudaStream_t s,
              T* r, T* z, T* p, T* q, int* iters_out, int check_every, PcgHook hook = nullptr,
              void* hook_user = nullptr) {
  SolveWs& w = c->ws;
  const size_t n = c->n_dofs, tot = n * (size_t)nv;
  double* rz = w.colbuf;
  double* pq = w.colbuf + nv;
  double* alpha = w.colbuf + 2 * nv;
  double* beta = w.colbuf + 3 * nv;
  double* rznew = w.colbuf + 4 * nv;
  double* rr = w.colbuf + 5 * nv;
  double* rzmid = w.colbuf + 6 * nv;
  const T* dinv = nullptr;
  const T* dinv_all = (const T*)(sizeof(T) == 8 ? (const void*)w.dinv64 : (const void*)w.dinv32);
  if (precond == FE_PRECOND_JACOBI) dinv = dinv_all;
  const bool learned = precond == FE_PRECOND_LEARNED;
  const void* vecs[6] = {x, r, z, p, q, b};
  const bool wide = wide_ok<T>(nv, vecs, 6);
  cudaError_t e;
  std::vector<double> rr_h(nv);
  std::vector<int> act_h(nv, 1);

  // r = b - A x
  fe_status st = apply_mode<T>(c, x, r, nv, s);
  if (st != FE_OK) return st;
  residual_kernel<T><<<ew_grid(tot), 256, 0, s>>>(b, r, tot);
  if (hook) hook(hook_user, 0, x, r, s);
  if (learned) st = learned_precond_apply(c, r, z, nv, sizeof(T) == 8, s);
  else precond_jacobi_kernel<T><<<ew_grid(tot), 256, 0, s>>>(r, dinv, z, n, nv);
  if (st != FE_OK) return st;
  if ((e = col_dot<T>(r, z, n, nv, w.partial, rz, s)) != cudaSuccess) return from_cuda(e);
  if (learned) {
    fcg_safeguard_kernel<T><<<ew_grid(tot), 256, 0, s>>>(r, dinv_all, z, rz, tot, nv);
    if ((e = col_dot<T>(r, z, n, nv, w.partial, rz, s)) != cudaSuccess) return from_cuda(e);
  }
  if ((e = cudaMemcpyAsync(p, z, tot * sizeof(T), cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return from_cuda(e);
  if ((e = col_dot<T>(r, r, n, nv, w.partial, rr, s)) != cudaSuccess) return from_cuda(e);
  cudaMemcpyAsync(rr_h.data(), rr, nv * sizeof(double), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  for (int j = 0; j < nv; ++j) act_h[j] = std::sqrt(rr_h[j]) > tol_host[j];
  cudaMemcpyAsync(w.active, act_h.data(), nv * sizeof(int), cudaMemcpyHostToDevice, s);
  int it = 0;
  bool done = true;
  for (int j = 0; j < nv; ++j) done = done && !act_h[j];
  while (!done && it < max_it) {
    st = apply_mode<T>(c, p, q, nv, s);
    if (st != FE_OK) return st;
    if ((e = col_dot<T>(p, q, n, nv, w.partial, pq, s)) != cudaSuccess) return from_cuda(e);
    cg_alpha_kernel<<<(nv + 127) / 128, 128, 0, s>>>(rz, pq, w.active, alpha, nv, c->d_status);
    if (learned) {
      if (wide)
        cg_update_kernel_wide<T><<<wide_grid(nv, Wide<T>::N), dim3(32, 8), 0, s>>>(x, r, p, q, alpha, n, nv);
      else
        cg_update_kernel<T><<<ew_grid(tot), 256, 0, s>>>(x, r, p, q, alpha, tot, nv);
      st = learned_precond_apply(c, r, z, nv, sizeof(T) == 8, s);
      if (st != FE_OK) return st;
      if ((e = col_dot<T>(r, z, n, nv, w.partial, rznew, s)) != cudaSuccess) return from_cuda(e);
    } else {
      if (wide) {
        cg_step_kernel_wide<T><<<wide_grid(nv, Wide<T>::N), dim3(32, 8), 0, s>>>(x, r, z, p, q, dinv, alpha, n, nv,
                                                                                 w.partial);
        col_sum_partials_warp<<<(nv + 7) / 8, 256, 0, s>>>(w.partial, kWideBlocks, nv, rznew);
      } else {
        const dim3 grid(kRedBlocks, (nv + kColTile - 1) / kColTile);
        cg_step_kernel<T><<<grid, dim3(kColTile, 8), 0, s>>>(x, r, z, p, q, dinv, alpha, n, nv, w.partial);
        col_sum_partials<<<(nv + 127) / 128, 128, 0, s>>>(w.partial, kRedBlocks, nv, rznew);
      }
    }
    if (learned) {
      if (wide)
        fcg_safeguard_kernel_wide<T><<<wide_grid(nv, Wide<T>::N), dim3(32, 8), 0, s>>>(r, dinv_all, z, rznew, n, nv);
      else
        fcg_safeguard_kernel<T><<<ew_grid(tot), 256, 0, s>>>(r, dinv_all, z, rznew, tot, nv);
      if ((e = col_dot<T>(r, z, n, nv, w.partial, rznew, s)) != cudaSuccess) return from_cuda(e);
      // flexible CG (Notay): beta = -(z_new . A p) / (p . A p)
      if ((e = col_dot<T>(z, q, n, nv, w.partial, rzmid, s)) != cudaSuccess) return from_cuda(e);
    }
    cg_beta_kernel<<<(nv + 127) / 128, 128, 0, s>>>(rznew, rzmid, pq, rz, w.active, beta, nv, learned ? 1 : 0);
    if (wide)
      cg_direction_kernel_wide<T><<<wide_grid(nv, Wide<T>::N), dim3(32, 8), 0, s>>>(p, z, beta, n, nv);
    else
      cg_direction_kernel<T><<<dim3(kRedBlocks, (nv + kColTile - 1) / kColTile), dim3(kColTile, 8), 0, s>>>(
          p, z, beta, n, nv);
    ++it;
    if (hook) hook(hook_user, it, x, r, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return from_cuda(e);
    if (it % check_every == 0 || it == max_it) {
      if ((e = col_dot<T>(r, r, n, nv, w.partial, rr, s)) != cudaSuccess) return from_cuda(e);
      cudaMemcpyAsync(rr_h.data(), rr, nv * sizeof(double), cudaMemcpyDeviceToHost, s);
      if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return from_cuda(e);
      int hs = 0;
      cudaMemcpy(&hs, c->d_status, sizeof(int), cudaMemcpyDeviceToHost);
      if (hs == FE_EBREAKDOWN) {
        cudaMemset(c->d_status, 0, sizeof(int));
        *iters_out = it;
        return FE_EBREAKDOWN;
      }
      done = true;
      for (int j = 0; j < nv; ++j) {
        if (!std::isfinite(rr_h[j])) { *iters_out = it; return FE_ENONFINITE; }
        act_h[j] = std::sqrt(rr_h[j]) > tol_host[j];
        done = done && !act_h[j];
      }
      cudaMemcpyAsync(w.active, act_h.data(), nv * sizeof(int), cudaMemcpyHostToDevice, s);
    }
  }
  *iters_out = it;
  return FE_OK;
}

// ||b_j - A64 x_j|| / ||b_j|| for every column (FP64 operator), into rel (host).
fe_status true_residual(fe_ctx* c, const double* B, const double* X, int nv, double* r64, double* rel, double* bnorm,
                        cudaStream_t s) {
  SolveWs& w = c->ws;
  const size_t n = c->n_dofs, tot = n * (size_t)nv;
  double* rr = w.colbuf + 7 * nv;
  fe_status st = apply_mode<double>(c, X, r64, nv, s);
  if (st != FE_OK) return st;
  residual_kernel<double><<<ew_grid(tot), 256, 0, s>>>(B, r64, tot);
  cudaError_t e = col_dot<double>(r64, r64, n, nv, w.partial, rr, s);
  if (e != cudaSuccess) return from_cuda(e);
  std::vector<double> h(nv);
  cudaMemcpyAsync(h.data(), rr, nv * sizeof(double), cudaMemcpyDeviceToHost, s);
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return from_cuda(e);
  for (int j = 0; j < nv; ++j) rel[j] = bnorm[j] > 0 ? std::sqrt(h[j]) / bnorm[j] : std::sqrt(h[j]);
  return FE_OK;
}

fe_status pcg_f32_hooked(fe_ctx* c, const float* b, float* x, int nv, const double* tol, int max_it, PcgHook hook,
                         void* user, int* its, cudaStream_t s, int check_every) {
  SolveWs& w = c->ws;
  const fe_mode saved = c->inner_mode;
  c->inner_mode = FE_FP32;
  fe_status st = pcg<float>(c, b, x, nv, tol, max_it, FE_PRECOND_JACOBI, s, w.v32[0], w.v32[1], w.v32[2], w.v32[5],
                            its, check_every, hook, user);
  c->inner_mode = saved;
  return st;
}

fe_status pcg_f32(fe_ctx* c, const float* b, float* x, int nv, const double* tol, int max_it, int precond, int* its,
                  cudaStream_t s) {
  SolveWs& w = c->ws;
  const fe_mode saved = c->inner_mode;
  c->inner_mode = FE_FP32;
  fe_status st = pcg<float>(c, b, x, nv, tol, max_it, precond, s, w.v32[0], w.v32[1], w.v32[2], w.v32[5], its, 4);
  c->inner_mode = saved;
  return st;
}

void free_solver_workspace(fe_ctx* c) {
  SolveWs& w = c->ws;
  for (int k = 0; k < 4; ++k) cudaFree(w.v64[k]);
  for (int k = 0; k < 6; ++k) cudaFree(w.v32[k]);
  cudaFree(w.colbuf); cudaFree(w.partial); cudaFree(w.active);
  cudaFree(w.diag); cudaFree(w.dinv64); cudaFree(w.dinv32);
  w = SolveWs();
}

}  // namespace fe

extern "C" fe_status fe_solve(fe_ctx* c, const double* B, double* X, int nv, double rtol, int max_it, int precond,
                              int inner_mode, fe_solve_info* info, double* rel_res, void* stream) {
  if (!c || !B || !X || nv <= 0 || !(rtol > 0.0) || max_it < 0) return FE_EINVAL;
  if (c->refined) return FE_EUNSUPPORTED;
  if (precond != FE_PRECOND_NONE && precond != FE_PRECOND_JACOBI && precond != FE_PRECOND_LEARNED) return FE_EINVAL;
  if (inner_mode != FE_FP64 && inner_mode != FE_FP32 && inner_mode != FE_TF32 && inner_mode != FE_BF16 &&
      inner_mode != FE_TF32X3 && inner_mode != FE_DF64)
    return FE_EINVAL;
  if (precond == FE_PRECOND_LEARNED && !learned_ready(c, nv)) return FE_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = solver_workspace(c, nv);
  if (e != cudaSuccess) return from_cuda(e);
  SolveWs& w = c->ws;
  const size_t n = c->n_dofs, tot = n * (size_t)nv;
  c->inner_mode = (fe_mode)inner_mode;
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  cudaEventRecord(t0, s);

  // ||b_j||
  std::vector<double> bnorm(nv), rel(nv), tol(nv);
  double* bb = w.colbuf + 8 * nv;
  if ((e = col_dot<double>(B, B, n, nv, w.partial, bb, s)) != cudaSuccess) return from_cuda(e);
  cudaMemcpyAsync(bnorm.data(), bb, nv * sizeof(double), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  for (int j = 0; j < nv; ++j) bnorm[j] = std::sqrt(bnorm[j]);

  fe_solve_info inf{};
  fe_status st = FE_OK;
  int fp64_applies = 0;
  if (inner_mode == FE_FP64 || inner_mode == FE_DF64) {
    // FP64 PCG (operator in FP64, or in double-float arithmetic for
    // FE_DF64); the recurrence residual is trusted to rtol/2, then the FP64
    // operator checks the result.
    for (int j = 0; j < nv; ++j) tol[j] = 0.5 * rtol * bnorm[j];
    int its = 0;
    c->op64 = (fe_mode)inner_mode;
    st = pcg<double>(c, B, X, nv, tol.data(), max_it, precond, s, w.v64[0], w.v64[1], w.v64[2], w.v64[3], &its, 1);
    c->op64 = FE_FP64;
    inf.iterations = its;
    fp64_applies = inner_mode == FE_FP64 ? its + 1 : 0;   // the final check below adds one
  } else {
    // FP64 iterative refinement: r = b - A64 x; solve A32 d = r / ||r|| in the
    // inner precision to the reduction still needed (rtol ||b|| / ||r||), but
    // no further than FP32 can resolve (kInnerFloor); x += ||r|| d.
    const double kInnerFloor = 2e-6;
    int total = 0, outer = 0;
    double* scale = w.colbuf + 9 * nv;
    double* unscale = w.colbuf + 10 * nv;
    while (outer < 30 && total < max_it) {
      st = true_residual(c, B, X, nv, w.v64[0], rel.data(), bnorm.data(), s);
      ++fp64_applies;
      if (st != FE_OK) break;
      double worst = 0;
      for (int j = 0; j < nv; ++j) worst = std::fmax(worst, rel[j]);
      if (worst <= rtol) break;
      std::vector<double> sc(nv), us(nv);
      for (int j = 0; j < nv; ++j) {
        const double rn = rel[j] * bnorm[j];
        const bool act = rel[j] > rtol && rn > 0;
        sc[j] = act ? 1.0 / rn : 0.0;   // converged columns get a zero right-hand side
        us[j] = act ? rn : 0.0;
        tol[j] = act ? std::fmax(0.5 * rtol / rel[j], kInnerFloor) : 0.0;
      }
      cudaMemcpyAsync(scale, sc.data(), nv * sizeof(double), cudaMemcpyHostToDevice, s);
      cudaMemcpyAsync(unscale, us.data(), nv * sizeof(double), cudaMemcpyHostToDevice, s);
      float* b32 = w.v32[4];
      float* d32 = w.v32[3];
      scale_convert_kernel<float, double><<<ew_grid(tot), 256, 0, s>>>(b32, w.v64[0], scale, tot, nv, 0);
      cudaMemsetAsync(d32, 0, tot * sizeof(float), s);
      int its = 0;
      // tolerance relative to the scaled right-hand side (norm 1 per active column)
      st = pcg<float>(c, b32, d32, nv, tol.data(), max_it - total, precond, s, w.v32[0], w.v32[1], w.v32[2],
                      w.v32[5], &its, 4);
      total += its;
      if (st != FE_OK) break;
      scale_convert_kernel<double, float><<<ew_grid(tot), 256, 0, s>>>(X, d32, unscale, tot, nv, 1);
      ++outer;
    }
    inf.iterations = total;
    inf.outer_iterations = outer;
  }
  fe_status st2 = true_residual(c, B, X, nv, w.v64[0], rel.data(), bnorm.data(), s);
  ++fp64_applies;
  if (st == FE_OK) st = st2;
  cudaEventRecord(t1, s);
  cudaEventSynchronize(t1);
  float ms = 0;
  cudaEventElapsedTime(&ms, t0, t1);
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  double worst = 0;
  int conv = 0;
  for (int j = 0; j < nv; ++j) {
    worst = std::fmax(worst, rel[j]);
    conv += rel[j] <= rtol;
  }
  inf.fp64_applies = fp64_applies;
  inf.max_rel_residual = worst;
  inf.converged_columns = conv;
  inf.seconds = ms * 1e-3;
  if (info) *info = inf;
  if (rel_res) std::memcpy(rel_res, rel.data(), nv * sizeof(double));
  if (st == FE_OK && conv < nv) st = FE_ENOTCONV;
  return st;
}
