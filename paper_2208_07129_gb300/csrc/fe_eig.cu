// Eigenvalue layer (include/fe_eig.h): GLL diagonal mass, the scaled product
// Y = a M^-1/2 A M^-1/2 X + b X + c Y, the Chebyshev filter and the
// Chebyshev-filtered subspace iteration of Algorithm 6 (Sec. 4.3).
//
// The filter is a sequence of fused scaled products (the cell kernels with
// the Scale epilogue); the dense steps of each round -- Gram matrices,
// Cholesky QR, the k x k Rayleigh-Ritz eigenproblem and the rotations --
// are plain GEMM / LAPACK work and go to cuBLAS and cuSOLVER.  In the
// DoF-major layout a num_dofs x k block is, to a column-major BLAS, the
// k x num_dofs matrix B^T with leading dimension k; every call below is
// written in that view.
#include <cublas_v2.h>
#include <cusolverDn.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "fe_cell_kernel.cuh"
#include "fe_eig.h"
#include "fe_internal.h"

using namespace fe;

namespace {

fe_status from_cuda(cudaError_t e) {
  return fe::cuda_status(e);
}

bool overlaps(const void* a, const void* b, size_t bytes) {
  const char* x = static_cast<const char*>(a);
  const char* y = static_cast<const char*>(b);
  return x < y + bytes && y < x + bytes;
}

cudaError_t ensure_msq(fe_ctx* c) {
  if (c->d_msq64) return cudaSuccess;
  build_gll_mass(c);
  std::vector<double> s64(c->n_dofs);
  std::vector<float> s32(c->n_dofs);
  for (size_t i = 0; i < c->n_dofs; ++i) {
    s64[i] = 1.0 / std::sqrt(c->mass[i]);
    s32[i] = (float)s64[i];
  }
  cudaError_t e = cudaMalloc(&c->d_msq64, c->n_dofs * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_msq32, c->n_dofs * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(c->d_msq64, s64.data(), c->n_dofs * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_msq32, s32.data(), c->n_dofs * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(c->d_msq64);
    cudaFree(c->d_msq32);
    c->d_msq64 = nullptr;
    c->d_msq32 = nullptr;
  }
  return e;
}

// Arithmetic of a scaled product: FP32 data and arithmetic, FP64, or FP64
// data with double-float arithmetic.
enum Prec { kF32 = 0, kF64 = 1, kDF64 = 2 };

// Y = a H~ X + b X + c Y (no argument checks).
cudaError_t scaled(fe_ctx* c, int prec, const void* X, void* Y, int n_vec, double a, double b, double cc,
                   cudaStream_t s) {
  if (prec != kF32) {
    const Scale<double> sc{c->d_msq64, a, b, cc};
    if (prec == kDF64)
      return apply_scaled_df64(c, static_cast<const double*>(X), static_cast<double*>(Y), n_vec, sc, s);
    return apply_scaled_f64(c, static_cast<const double*>(X), static_cast<double*>(Y), n_vec, sc, s);
  }
  const Scale<float> sc{c->d_msq32, (float)a, (float)b, (float)cc};
  return apply_scaled_f32(c, static_cast<const float*>(X), static_cast<float*>(Y), n_vec, sc, s);
}

// The filter loop of Algorithm 6 (sigma updated after every step).  The
// result is left in *X (the two buffer pointers are swapped as needed).
cudaError_t filter(fe_ctx* c, int prec, void** X, void** Y, int n_vec, int m, double lmin, double lu, double lmax,
                   cudaStream_t s) {
  const double e = (lmax - lu) / 2.0, cen = (lmax + lu) / 2.0;
  double sigma = e / (lmin - cen);
  const double sigma1 = sigma, gamma = 2.0 / sigma1;
  double alpha1 = sigma1 / e, alpha2 = -cen;
  cudaError_t err = scaled(c, prec, *X, *Y, n_vec, alpha1, alpha1 * alpha2, 0.0, s);
  for (int d = 2; d <= m && err == cudaSuccess; ++d) {
    const double sigma2 = 1.0 / (gamma - sigma);
    alpha1 = 2.0 * sigma2 / e;
    alpha2 = -sigma * sigma2;
    // X <- alpha1 H~ Y - c alpha1 Y + alpha2 X, then swap(X, Y)
    err = scaled(c, prec, *Y, *X, n_vec, alpha1, -cen * alpha1, alpha2, s);
    std::swap(*X, *Y);
    sigma = sigma2;
  }
  std::swap(*X, *Y);
  return err;
}

__global__ void zero_constrained_kernel(double* __restrict__ U, int k, MeshDev m, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n * k; i += (size_t)gridDim.x * blockDim.x) {
    const size_t dof = i / k;
    const int gx = (int)(dof % m.Nx), gy = (int)((dof / m.Nx) % m.Ny), gz = (int)(dof / ((size_t)m.Nx * m.Ny));
    if (on_boundary(gx, m.Nx, m.periodic) || on_boundary(gy, m.Ny, m.periodic) || on_boundary(gz, m.Nz, m.periodic))
      U[i] = 0.0;
  }
}

// Uniform [-1, 1) from a 64-bit counter (splitmix64 finaliser).
__device__ __forceinline__ double hash_uniform(unsigned long long x) {
  x += 0x9e3779b97f4a7c15ull;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
  x ^= x >> 31;
  return (double)(x >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

__global__ void random_vector_kernel(double* __restrict__ v, size_t n, unsigned long long seed) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    v[i] = hash_uniform(seed * 0x100000001b3ull + i);
}

template <typename A, typename B>
__global__ void convert_kernel(const A* __restrict__ x, B* __restrict__ y, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = (B)x[i];
}

// Column residuals ||W_j - lambda_j U_j||_2: per-block partial sums of
// squares over a slice of rows, then a fixed-order sum (deterministic).
constexpr int kResRows = 128;
template <typename T>
__global__ void residual_partial_kernel(const T* __restrict__ U, const T* __restrict__ W, const T* __restrict__ lam,
                                        size_t n, int k, double* __restrict__ part) {
  __shared__ double red[8][33];
  const int col = blockIdx.x * 32 + threadIdx.x;
  double acc = 0.0;
  if (col < k) {
    const T l = lam[col];
    for (size_t r = blockIdx.y * 8 + threadIdx.y; r < n; r += (size_t)gridDim.y * 8) {
      const double d = (double)(W[r * k + col] - l * U[r * k + col]);
      acc += d * d;
    }
  }
  red[threadIdx.y][threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.y == 0 && col < k) {
    double s = 0.0;
    for (int t = 0; t < 8; ++t) s += red[t][threadIdx.x];
    part[(size_t)blockIdx.y * k + col] = s;
  }
}

__global__ void residual_final_kernel(const double* __restrict__ part, int k, int rows, double* __restrict__ res) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= k) return;
  double s = 0.0;
  for (int r = 0; r < rows; ++r) s += part[(size_t)r * k + col];
  res[col] = std::sqrt(s);
}

template <typename T>
__global__ void add_diagonal_kernel(T* __restrict__ S, int k, T shift) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < k) S[(size_t)i * k + i] += shift;
}

// The dense kernels in either precision (cuBLAS / cuSOLVER, column-major).
template <typename T>
struct Dense;
template <>
struct Dense<double> {
  static cublasStatus_t gemm(cublasHandle_t h, cublasOperation_t ta, cublasOperation_t tb, int m, int n, int k,
                             const double* A, int lda, const double* B, int ldb, double* C, int ldc) {
    const double one = 1.0, zero = 0.0;
    return cublasDgemm(h, ta, tb, m, n, k, &one, A, lda, B, ldb, &zero, C, ldc);
  }
  static cublasStatus_t trsm_lt(cublasHandle_t h, int m, int n, const double* R, double* B) {
    const double one = 1.0;
    return cublasDtrsm(h, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_T, CUBLAS_DIAG_NON_UNIT, m, n, &one,
                       R, m, B, m);
  }
  static cublasStatus_t asum(cublasHandle_t h, int n, const double* x, int inc, double* r) {
    return cublasDasum(h, n, x, inc, r);
  }
  static cusolverStatus_t potrf_buf(cusolverDnHandle_t h, int k, double* S, int* lw) {
    return cusolverDnDpotrf_bufferSize(h, CUBLAS_FILL_MODE_UPPER, k, S, k, lw);
  }
  static cusolverStatus_t potrf(cusolverDnHandle_t h, int k, double* S, double* w, int lw, int* info) {
    return cusolverDnDpotrf(h, CUBLAS_FILL_MODE_UPPER, k, S, k, w, lw, info);
  }
  static cusolverStatus_t syevd_buf(cusolverDnHandle_t h, int k, double* S, double* lam, int* lw) {
    return cusolverDnDsyevd_bufferSize(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, k, S, k, lam, lw);
  }
  static cusolverStatus_t syevd(cusolverDnHandle_t h, int k, double* S, double* lam, double* w, int lw, int* info) {
    return cusolverDnDsyevd(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, k, S, k, lam, w, lw, info);
  }
  static constexpr double shift = 1e-13;   // relative diagonal shift of the fallback Cholesky QR
};
template <>
struct Dense<float> {
  static cublasStatus_t gemm(cublasHandle_t h, cublasOperation_t ta, cublasOperation_t tb, int m, int n, int k,
                             const float* A, int lda, const float* B, int ldb, float* C, int ldc) {
    const float one = 1.f, zero = 0.f;
    return cublasSgemm(h, ta, tb, m, n, k, &one, A, lda, B, ldb, &zero, C, ldc);
  }
  static cublasStatus_t trsm_lt(cublasHandle_t h, int m, int n, const float* R, float* B) {
    const float one = 1.f;
    return cublasStrsm(h, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_T, CUBLAS_DIAG_NON_UNIT, m, n, &one,
                       R, m, B, m);
  }
  static cublasStatus_t asum(cublasHandle_t h, int n, const float* x, int inc, float* r) {
    return cublasSasum(h, n, x, inc, r);
  }
  static cusolverStatus_t potrf_buf(cusolverDnHandle_t h, int k, float* S, int* lw) {
    return cusolverDnSpotrf_bufferSize(h, CUBLAS_FILL_MODE_UPPER, k, S, k, lw);
  }
  static cusolverStatus_t potrf(cusolverDnHandle_t h, int k, float* S, float* w, int lw, int* info) {
    return cusolverDnSpotrf(h, CUBLAS_FILL_MODE_UPPER, k, S, k, w, lw, info);
  }
  static cusolverStatus_t syevd_buf(cusolverDnHandle_t h, int k, float* S, float* lam, int* lw) {
    return cusolverDnSsyevd_bufferSize(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, k, S, k, lam, lw);
  }
  static cusolverStatus_t syevd(cusolverDnHandle_t h, int k, float* S, float* lam, float* w, int lw, int* info) {
    return cusolverDnSsyevd(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, k, S, k, lam, w, lw, info);
  }
  static constexpr float shift = 1e-5f;
};

cudaError_t handles(fe_ctx* c, cudaStream_t s, cublasHandle_t* hb, cusolverDnHandle_t* hs) {
  if (!c->blas) {
    cublasHandle_t h;
    if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
    c->blas = h;
  }
  if (!c->solver) {
    cusolverDnHandle_t h;
    if (cusolverDnCreate(&h) != CUSOLVER_STATUS_SUCCESS) return cudaErrorUnknown;
    c->solver = h;
  }
  *hb = static_cast<cublasHandle_t>(c->blas);
  *hs = static_cast<cusolverDnHandle_t>(c->solver);
  if (cublasSetStream(*hb, s) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
  if (cusolverDnSetStream(*hs, s) != CUSOLVER_STATUS_SUCCESS) return cudaErrorUnknown;
  return cudaSuccess;
}

// Smallest and largest eigenvalue of the symmetric tridiagonal matrix
// (alpha on the diagonal, beta[i] coupling i-1 and i) by bisection on the
// Sturm sequence count.
int sturm_below(const std::vector<double>& a, const std::vector<double>& b, double x) {
  int cnt = 0;
  double q = a[0] - x;
  if (q < 0) ++cnt;
  for (size_t i = 1; i < a.size(); ++i) {
    if (q == 0.0) q = 1e-300;
    q = a[i] - x - b[i] * b[i] / q;
    if (q < 0) ++cnt;
  }
  return cnt;
}

void tridiag_extremes(const std::vector<double>& a, const std::vector<double>& b, double* mn, double* mx) {
  double lo = a[0], hi = a[0];
  for (size_t i = 0; i < a.size(); ++i) {
    const double r = (i > 0 ? std::fabs(b[i]) : 0.0) + (i + 1 < a.size() ? std::fabs(b[i + 1]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  const int n = (int)a.size();
  auto bisect = [&](int idx) {  // the idx-th smallest eigenvalue
    double l = lo, h = hi;
    for (int it = 0; it < 200 && h - l > 1e-14 * std::max(1.0, std::fabs(h)); ++it) {
      const double mid = 0.5 * (l + h);
      if (sturm_below(a, b, mid) > idx) h = mid;
      else l = mid;
    }
    return 0.5 * (l + h);
  };
  *mn = bisect(0);
  *mx = bisect(n - 1);
}

// One precision's share of the subspace iteration: the current block U, the
// work blocks W and T (n x k each), and the k x k dense state.
template <typename T>
struct Chfsi {
  fe_ctx* c;
  cudaStream_t s;
  cublasHandle_t hb;
  cusolverDnHandle_t hs;
  size_t n;
  int k;
  T *U = nullptr, *W = nullptr, *Tb = nullptr, *S = nullptr, *lam = nullptr, *work = nullptr;
  double *res = nullptr, *part = nullptr;
  int* info = nullptr;
  int lwork = 0;
  bool owns_u = false;
  int prec = sizeof(T) == 8 ? kF64 : kF32;   // arithmetic of the scaled products

  // U: the caller's block (FP64) or nullptr to allocate one (FP32).
  cudaError_t alloc(T* user) {
    const size_t blk = n * (size_t)k * sizeof(T);
    cudaError_t e = cudaSuccess;
    if (user) U = user;
    else { e = cudaMalloc(&U, blk); owns_u = true; }
    if (e == cudaSuccess) e = cudaMalloc(&W, blk);
    if (e == cudaSuccess) e = cudaMalloc(&Tb, blk);
    if (e == cudaSuccess) e = cudaMalloc(&S, (size_t)k * k * sizeof(T));
    if (e == cudaSuccess) e = cudaMalloc(&lam, k * sizeof(T));
    if (e == cudaSuccess) e = cudaMalloc(&res, k * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&part, (size_t)kResRows * k * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&info, sizeof(int));
    if (e != cudaSuccess) return e;
    int l1 = 0, l2 = 0;
    if (Dense<T>::potrf_buf(hs, k, S, &l1) != CUSOLVER_STATUS_SUCCESS ||
        Dense<T>::syevd_buf(hs, k, S, lam, &l2) != CUSOLVER_STATUS_SUCCESS)
      return cudaErrorUnknown;
    lwork = std::max(l1, l2);
    return cudaMalloc(&work, std::max(1, lwork) * sizeof(T));
  }
  // Frees the work blocks; the caller's block (wherever it sits among U, W
  // and Tb after the pointer swaps) is left alone.
  void release(const T* user) {
    for (T* p : {U, W, Tb})
      if (p != user) cudaFree(p);
    for (T* p : {S, lam, work}) cudaFree(p);
    cudaFree(res);
    cudaFree(part);
    cudaFree(info);
  }
  int read_info() {
    int h = -1;
    if (cudaMemcpyAsync(&h, info, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return -1;
    if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
    return h;
  }
  fe_status gram(const T* A, const T* B) {   // S = A^T B
    return Dense<T>::gemm(hb, CUBLAS_OP_N, CUBLAS_OP_T, k, k, (int)n, A, k, B, k, S, k) == CUBLAS_STATUS_SUCCESS
               ? FE_OK : FE_ECUDA;
  }

  // Cholesky QR of U in place (U <- U R^-1 with U^T U = R^T R), twice; a Gram
  // matrix that is not numerically positive definite gets a relative
  // diagonal shift (Dense<T>::shift x trace) and a third pass.
  fe_status cholqr() {
    int passes = 2;
    for (int pass = 0; pass < passes; ++pass) {
      fe_status st = gram(U, U);
      if (st != FE_OK) return st;
      if (Dense<T>::potrf(hs, k, S, work, lwork, info) != CUSOLVER_STATUS_SUCCESS) return FE_ECUDA;
      int inf = read_info();
      if (inf < 0) return FE_ECUDA;
      if (inf > 0) {
        if ((st = gram(U, U)) != FE_OK) return st;
        T tr = 0;
        if (Dense<T>::asum(hb, k, S, k + 1, &tr) != CUBLAS_STATUS_SUCCESS) return FE_ECUDA;
        if (!(tr > 0) || !std::isfinite((double)tr)) return FE_ENONFINITE;
        add_diagonal_kernel<T><<<(k + 255) / 256, 256, 0, s>>>(S, k, Dense<T>::shift * tr);
        if (Dense<T>::potrf(hs, k, S, work, lwork, info) != CUSOLVER_STATUS_SUCCESS) return FE_ECUDA;
        if (read_info() != 0) return FE_EBREAKDOWN;
        passes = 3;
      }
      // U^T <- R^-T U^T  (U <- U R^-1)
      if (Dense<T>::trsm_lt(hb, k, (int)n, S, U) != CUBLAS_STATUS_SUCCESS) return FE_ECUDA;
    }
    return FE_OK;
  }

  // Rayleigh-Ritz on the orthonormal U: W = H~ U, P = U^T W = Q Lambda Q^T,
  // U <- U Q; then W = H~ U again for the residuals (one scaled product costs
  // 2 k / 441 of the k x k rotation of W it replaces at p = 6).  lam (device)
  // ascending, res (device, FP64) the residual norms.
  fe_status rayleigh_ritz() {
    cudaError_t e = scaled(c, prec, U, W, k, 1.0, 0.0, 0.0, s);
    if (e != cudaSuccess) return from_cuda(e);
    fe_status st = gram(U, W);
    if (st != FE_OK) return st;
    if (Dense<T>::syevd(hs, k, S, lam, work, lwork, info) != CUSOLVER_STATUS_SUCCESS) return FE_ECUDA;
    const int inf = read_info();
    if (inf != 0) return inf < 0 ? FE_ECUDA : FE_ENONFINITE;
    // (U Q)^T = Q^T U^T
    if (Dense<T>::gemm(hb, CUBLAS_OP_T, CUBLAS_OP_N, k, (int)n, k, S, k, U, k, Tb, k) != CUBLAS_STATUS_SUCCESS)
      return FE_ECUDA;
    std::swap(U, Tb);
    e = scaled(c, prec, U, W, k, 1.0, 0.0, 0.0, s);
    if (e != cudaSuccess) return from_cuda(e);
    residual_partial_kernel<T><<<dim3((k + 31) / 32, kResRows), dim3(32, 8), 0, s>>>(U, W, lam, n, k, part);
    residual_final_kernel<<<(k + 127) / 128, 128, 0, s>>>(part, k, kResRows, res);
    return from_cuda(cudaGetLastError());
  }

  // The filter pass of Algorithm 6 on U, with Tb as scratch.
  fe_status filter_pass(int m, double lmin, double lu, double lmax) {
    void* x = U;
    void* y = Tb;
    cudaError_t e = filter(c, prec, &x, &y, k, m, lmin, lu, lmax, s);
    if (e != cudaSuccess) return from_cuda(e);
    if (x != U) std::swap(U, Tb);
    return from_cuda(cudaGetLastError());
  }

  fe_status pull(std::vector<double>& hlam, std::vector<double>& hres) {
    std::vector<T> l(k);
    cudaError_t e = cudaMemcpyAsync(l.data(), lam, k * sizeof(T), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hres.data(), res, k * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return FE_ECUDA;
    for (int j = 0; j < k; ++j) {
      hlam[j] = (double)l[j];
      if (!std::isfinite(hlam[j]) || !std::isfinite(hres[j])) return FE_ENONFINITE;
    }
    return FE_OK;
  }
};

// Lanczos on H~ from a random free vector (FP64): the extreme Ritz values of
// the tridiagonal matrix and the last off-diagonal (theta_max + |beta|
// bounds the spectrum from above).  v, the previous v and w live in the two
// work blocks (each n x k, k >= 2).
fe_status lanczos(Chfsi<double>& ch, int steps, unsigned long long seed, double* theta_min, double* theta_max,
                  double* beta_last) {
  const size_t n = ch.n;
  const int ni = (int)n;
  cublasHandle_t hb = ch.hb;
  double* v = ch.Tb;
  double* vp = ch.Tb + n;
  double* w = ch.W;
  random_vector_kernel<<<1024, 256, 0, ch.s>>>(v, n, seed);
  zero_constrained_kernel<<<1024, 256, 0, ch.s>>>(v, 1, ch.c->mdev, n);
  cudaError_t e = cudaMemsetAsync(vp, 0, n * sizeof(double), ch.s);
  if (e != cudaSuccess) return from_cuda(e);
  double nv = 0.0;
  if (cublasDnrm2(hb, ni, v, 1, &nv) != CUBLAS_STATUS_SUCCESS || !(nv > 0)) return FE_ECUDA;
  double inv = 1.0 / nv;
  cublasDscal(hb, ni, &inv, v, 1);
  std::vector<double> al, be(1, 0.0);
  double beta = 0.0;
  for (int j = 0; j < steps; ++j) {
    e = scaled(ch.c, ch.prec, v, w, 1, 1.0, 0.0, 0.0, ch.s);
    if (e != cudaSuccess) return from_cuda(e);
    double alpha = 0.0;
    if (cublasDdot(hb, ni, w, 1, v, 1, &alpha) != CUBLAS_STATUS_SUCCESS) return FE_ECUDA;
    const double ma = -alpha, mb = -beta;
    cublasDaxpy(hb, ni, &ma, v, 1, w, 1);
    cublasDaxpy(hb, ni, &mb, vp, 1, w, 1);
    if (cublasDnrm2(hb, ni, w, 1, &beta) != CUBLAS_STATUS_SUCCESS) return FE_ECUDA;
    if (!std::isfinite(alpha) || !std::isfinite(beta)) return FE_ENONFINITE;
    al.push_back(alpha);
    if (j + 1 < steps) be.push_back(beta);
    if (beta <= 1e-300) break;
    cublasDcopy(hb, ni, v, 1, vp, 1);
    const double ib = 1.0 / beta;
    cublasDcopy(hb, ni, w, 1, v, 1);
    cublasDscal(hb, ni, &ib, v, 1);
  }
  be.resize(al.size());
  tridiag_extremes(al, be, theta_min, theta_max);
  *beta_last = beta;
  return FE_OK;
}

}  // namespace

namespace fe {
void free_eig(fe_ctx* c) {
  cudaFree(c->d_msq64);
  cudaFree(c->d_msq32);
  c->d_msq64 = nullptr;
  c->d_msq32 = nullptr;
  if (c->blas) cublasDestroy(static_cast<cublasHandle_t>(c->blas));
  if (c->solver) cusolverDnDestroy(static_cast<cusolverDnHandle_t>(c->solver));
  c->blas = nullptr;
  c->solver = nullptr;
}
}  // namespace fe

extern "C" fe_status fe_mass_gll(fe_ctx* c, double* m_host) {
  if (!c || !m_host) return FE_EINVAL;
  if (c->refined) return FE_EUNSUPPORTED;
  build_gll_mass(c);
  std::copy(c->mass.begin(), c->mass.end(), m_host);
  return FE_OK;
}

extern "C" fe_status fe_apply_scaled(fe_ctx* c, const void* X, void* Y, int n_vec, double a, double b, double cc,
                                     void* stream) {
  if (!c || n_vec < 0) return FE_EINVAL;
  if (n_vec == 0) return FE_OK;
  if (!X || !Y || !std::isfinite(a) || !std::isfinite(b) || !std::isfinite(cc)) return FE_EINVAL;
  if (c->refined || (c->mode != FE_FP64 && c->mode != FE_FP32 && c->mode != FE_DF64)) return FE_EUNSUPPORTED;
  const int prec = c->mode == FE_FP64 ? kF64 : (c->mode == FE_DF64 ? kDF64 : kF32);
  if (overlaps(X, Y, c->n_dofs * (size_t)n_vec * (prec != kF32 ? 8 : 4))) return FE_EINVAL;
  cudaError_t e = ensure_msq(c);
  if (e != cudaSuccess) return from_cuda(e);
  return from_cuda(scaled(c, prec, X, Y, n_vec, a, b, cc, static_cast<cudaStream_t>(stream)));
}

extern "C" fe_status fe_chebyshev_filter(fe_ctx* c, void* X, void* Y, int n_vec, int degree, double lmin, double lu,
                                         double lmax, void* stream) {
  if (!c || n_vec < 0 || degree < 1) return FE_EINVAL;
  if (n_vec == 0) return FE_OK;
  if (!X || !Y || !(lmin < lu && lu < lmax) || !std::isfinite(lmin) || !std::isfinite(lmax)) return FE_EINVAL;
  if (c->refined || (c->mode != FE_FP64 && c->mode != FE_FP32 && c->mode != FE_DF64)) return FE_EUNSUPPORTED;
  const int prec = c->mode == FE_FP64 ? kF64 : (c->mode == FE_DF64 ? kDF64 : kF32);
  const size_t bytes = c->n_dofs * (size_t)n_vec * (prec != kF32 ? 8 : 4);
  if (overlaps(X, Y, bytes)) return FE_EINVAL;
  cudaError_t e = ensure_msq(c);
  if (e != cudaSuccess) return from_cuda(e);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void* x = X;
  void* y = Y;
  e = filter(c, prec, &x, &y, n_vec, degree, lmin, lu, lmax, s);
  if (e == cudaSuccess && x != X) e = cudaMemcpyAsync(X, x, bytes, cudaMemcpyDeviceToDevice, s);
  return from_cuda(e);
}

extern "C" fe_status fe_chfsi(fe_ctx* c, double* U, int k, const fe_chfsi_desc* d, double* lambda, double* residual,
                              fe_chfsi_info* info, void* stream) {
  if (!c || !U || !d) return FE_EINVAL;
  if (k < 2 || d->n_wanted < 1 || d->n_wanted > k || d->degree < 1 || d->max_iter < 1 || d->lanczos_steps < 2 ||
      !(d->tol > 0) || (d->filter_mode != FE_FP64 && d->filter_mode != FE_FP32 && d->filter_mode != FE_DF64))
    return FE_EINVAL;
  if (c->refined) return FE_EUNSUPPORTED;
  size_t free_dofs = c->n_dofs;
  if (!c->periodic) free_dofs = (size_t)(c->mdev.Nx - 2) * (c->mdev.Ny - 2) * (c->mdev.Nz - 2);
  if ((size_t)k > free_dofs) return FE_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = ensure_msq(c);
  if (e != cudaSuccess) return from_cuda(e);
  cublasHandle_t hb;
  cusolverDnHandle_t hs;
  e = handles(c, s, &hb, &hs);
  if (e != cudaSuccess) return from_cuda(e);
  cublasSetPointerMode(hb, CUBLAS_POINTER_MODE_HOST);
  const bool mixed = d->filter_mode == FE_FP32;
  Chfsi<double> d64{c, s, hb, hs, c->n_dofs, k};
  Chfsi<float> d32{c, s, hb, hs, c->n_dofs, k};
  // FP64-data products in double-float arithmetic unless plain FP64 is asked for
  d64.prec = d->filter_mode == FE_FP64 ? kF64 : kDF64;
  e = d64.alloc(U);
  if (e == cudaSuccess && mixed) e = d32.alloc(nullptr);
  if (e != cudaSuccess) {
    d64.release(U);
    if (mixed) d32.release(nullptr);
    return from_cuda(e);
  }
  cudaEvent_t ev[2];
  cudaEventCreate(&ev[0]);
  cudaEventCreate(&ev[1]);
  fe_chfsi_info inf{};
  double t_total = 0.0, t_lz = 0.0;
  auto timed = [&](double* acc, auto&& fn) -> fe_status {
    cudaEventRecord(ev[0], s);
    const fe_status st = fn();
    cudaEventRecord(ev[1], s);
    cudaEventSynchronize(ev[1]);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev[0], ev[1]);
    *acc += ms * 1e-3;
    t_total += ms * 1e-3;
    return st;
  };
  std::vector<double> hlam(k), hres(k);
  auto max_res = [&]() { return *std::max_element(hres.begin(), hres.begin() + d->n_wanted); };
  double th_min = 0, th_max = 0, beta = 0;
  fe_status st = timed(&t_lz, [&] { return lanczos(d64, d->lanczos_steps, d->seed, &th_min, &th_max, &beta); });
  const double lmax0 = th_max + std::fabs(beta);
  const size_t nk = c->n_dofs * (size_t)k;
  // Rounds run in FP32 (filter, Cholesky QR, Rayleigh-Ritz) while the mixed
  // mode's residual is above fp32_switch; the FP64 rounds decide convergence.
  bool fp32 = mixed;
  auto round_start = [&]() -> fe_status {   // orthonormalise + project the current block
    fe_status r = fp32 ? timed(&inf.seconds_orth, [&] { return d32.cholqr(); })
                       : timed(&inf.seconds_orth, [&] { return d64.cholqr(); });
    if (r == FE_OK)
      r = fp32 ? timed(&inf.seconds_rr, [&] { return d32.rayleigh_ritz(); })
               : timed(&inf.seconds_rr, [&] { return d64.rayleigh_ritz(); });
    if (r == FE_OK) r = fp32 ? d32.pull(hlam, hres) : d64.pull(hlam, hres);
    return r;
  };
  if (st == FE_OK) {
    zero_constrained_kernel<<<1024, 256, 0, s>>>(d64.U, k, c->mdev, c->n_dofs);
    if (fp32) convert_kernel<double, float><<<2048, 256, 0, s>>>(d64.U, d32.U, nk);
    st = round_start();
  }
  double lmax = lmax0, lu = 0, lmin = 0;
  while (st == FE_OK) {
    if (fp32 && max_res() <= std::max(d->fp32_switch, d->tol)) {
      // switch to FP64: take the FP32 block over and re-project it
      convert_kernel<float, double><<<2048, 256, 0, s>>>(d32.U, d64.U, nk);
      fp32 = false;
      st = round_start();
      continue;
    }
    if (!fp32 && max_res() <= d->tol) break;
    if (inf.iterations >= d->max_iter) break;
    lu = hlam[k - 1];
    lmin = hlam[0];
    lmax = std::max(lmax0, lu + 1e-3 * std::fabs(lu));
    if (!(lmin < lu)) lmin = lu - 1e-3 * (lmax - lu);
    st = fp32 ? timed(&inf.seconds_filter, [&] { return d32.filter_pass(d->degree, lmin, lu, lmax); })
              : timed(&inf.seconds_filter, [&] { return d64.filter_pass(d->degree, lmin, lu, lmax); });
    inf.filter_applies += d->degree;
    if (fp32) inf.fp32_passes++;
    inf.iterations++;
    if (st == FE_OK) st = round_start();
  }
  if (st == FE_OK && fp32) {
    // max_iter ended an FP32 run: finish with an FP64 projection so that the
    // reported pairs and residuals are FP64
    convert_kernel<float, double><<<2048, 256, 0, s>>>(d32.U, d64.U, nk);
    fp32 = false;
    st = round_start();
  }
  if (d64.U != U) {
    cudaError_t e2 = cudaMemcpyAsync(U, d64.U, nk * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e2 != cudaSuccess && st == FE_OK) st = FE_ECUDA;
  }
  cudaStreamSynchronize(s);
  d64.release(U);
  if (mixed) d32.release(nullptr);
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  if (st == FE_OK) {
    inf.max_residual = max_res();
    for (int j = 0; j < d->n_wanted; ++j) inf.converged += hres[j] <= d->tol;
    if (lambda) std::copy(hlam.begin(), hlam.end(), lambda);
    if (residual) std::copy(hres.begin(), hres.end(), residual);
    if (inf.max_residual > d->tol) st = FE_ENOTCONV;
  }
  inf.lambda_min = lmin;
  inf.lambda_u = lu;
  inf.lambda_max = lmax;
  inf.seconds = t_total;
  if (info) *info = inf;
  return st;
}
