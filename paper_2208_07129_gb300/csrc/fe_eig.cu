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
  return e == cudaSuccess ? FE_OK : (e == cudaErrorMemoryAllocation ? FE_ENOMEM : FE_ECUDA);
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

// Y = a H~ X + b X + c Y in FP64 or FP32 (no argument checks).
cudaError_t scaled(fe_ctx* c, bool fp64, const void* X, void* Y, int n_vec, double a, double b, double cc,
                   cudaStream_t s) {
  if (fp64) {
    const Scale<double> sc{c->d_msq64, a, b, cc};
    return apply_scaled_f64(c, static_cast<const double*>(X), static_cast<double*>(Y), n_vec, sc, s);
  }
  const Scale<float> sc{c->d_msq32, (float)a, (float)b, (float)cc};
  return apply_scaled_f32(c, static_cast<const float*>(X), static_cast<float*>(Y), n_vec, sc, s);
}

// The filter loop of Algorithm 6 (sigma updated after every step).  The
// result is left in *X (the two buffer pointers are swapped as needed).
cudaError_t filter(fe_ctx* c, bool fp64, void** X, void** Y, int n_vec, int m, double lmin, double lu, double lmax,
                   cudaStream_t s) {
  const double e = (lmax - lu) / 2.0, cen = (lmax + lu) / 2.0;
  double sigma = e / (lmin - cen);
  const double sigma1 = sigma, gamma = 2.0 / sigma1;
  double alpha1 = sigma1 / e, alpha2 = -cen;
  cudaError_t err = scaled(c, fp64, *X, *Y, n_vec, alpha1, alpha1 * alpha2, 0.0, s);
  for (int d = 2; d <= m && err == cudaSuccess; ++d) {
    const double sigma2 = 1.0 / (gamma - sigma);
    alpha1 = 2.0 * sigma2 / e;
    alpha2 = -sigma * sigma2;
    // X <- alpha1 H~ Y - c alpha1 Y + alpha2 X, then swap(X, Y)
    err = scaled(c, fp64, *Y, *X, n_vec, alpha1, -cen * alpha1, alpha2, s);
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
__global__ void residual_partial_kernel(const double* __restrict__ U, const double* __restrict__ W,
                                        const double* __restrict__ lam, size_t n, int k, double* __restrict__ part) {
  __shared__ double red[8][33];
  const int col = blockIdx.x * 32 + threadIdx.x;
  double acc = 0.0;
  if (col < k) {
    const double l = lam[col];
    for (size_t r = blockIdx.y * 8 + threadIdx.y; r < n; r += (size_t)gridDim.y * 8) {
      const double d = W[r * k + col] - l * U[r * k + col];
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

__global__ void add_diagonal_kernel(double* __restrict__ S, int k, double shift) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < k) S[(size_t)i * k + i] += shift;
}

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

struct Chfsi {
  fe_ctx* c;
  cudaStream_t s;
  cublasHandle_t hb;
  cusolverDnHandle_t hs;
  size_t n;
  int k;
  double *W = nullptr, *T = nullptr, *S = nullptr, *lam = nullptr, *res = nullptr, *part = nullptr, *work = nullptr;
  int* info = nullptr;
  int lwork = 0;

  cudaError_t alloc() {
    const size_t blk = n * (size_t)k * sizeof(double);
    cudaError_t e = cudaMalloc(&W, blk);
    if (e == cudaSuccess) e = cudaMalloc(&T, blk);
    if (e == cudaSuccess) e = cudaMalloc(&S, (size_t)k * k * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&lam, k * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&res, k * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&part, (size_t)kResRows * k * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&info, sizeof(int));
    if (e != cudaSuccess) return e;
    int l1 = 0, l2 = 0;
    if (cusolverDnDpotrf_bufferSize(hs, CUBLAS_FILL_MODE_UPPER, k, S, k, &l1) != CUSOLVER_STATUS_SUCCESS ||
        cusolverDnDsyevd_bufferSize(hs, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, k, S, k, lam, &l2) !=
            CUSOLVER_STATUS_SUCCESS)
      return cudaErrorUnknown;
    lwork = std::max(l1, l2);
    return cudaMalloc(&work, std::max(1, lwork) * sizeof(double));
  }
  void release() {
    for (double* p : {W, T, S, lam, res, part, work}) cudaFree(p);
    cudaFree(info);
  }
  int read_info() {
    int h = -1;
    if (cudaMemcpyAsync(&h, info, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return -1;
    if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
    return h;
  }

  // Cholesky QR of U in place (U <- U R^-1 with U^T U = R^T R), twice; a
  // Gram matrix that is not numerically positive definite gets a diagonal
  // shift of 1e-13 trace(S) and a third pass.
  fe_status cholqr(double* U) {
    const double one = 1.0, zero = 0.0;
    int passes = 2;
    for (int pass = 0; pass < passes; ++pass) {
      if (cublasDsyrk(hb, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N, k, (int)n, &one, U, k, &zero, S, k) !=
          CUBLAS_STATUS_SUCCESS)
        return FE_ECUDA;
      if (cusolverDnDpotrf(hs, CUBLAS_FILL_MODE_UPPER, k, S, k, work, lwork, info) != CUSOLVER_STATUS_SUCCESS)
        return FE_ECUDA;
      int st = read_info();
      if (st < 0) return FE_ECUDA;
      if (st > 0) {
        if (cublasDsyrk(hb, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N, k, (int)n, &one, U, k, &zero, S, k) !=
            CUBLAS_STATUS_SUCCESS)
          return FE_ECUDA;
        double tr = 0.0;
        if (cublasDasum(hb, k, S, k + 1, &tr) != CUBLAS_STATUS_SUCCESS) return FE_ECUDA;
        if (!(tr > 0.0) || !std::isfinite(tr)) return FE_ENONFINITE;
        add_diagonal_kernel<<<(k + 255) / 256, 256, 0, s>>>(S, k, 1e-13 * tr);
        if (cusolverDnDpotrf(hs, CUBLAS_FILL_MODE_UPPER, k, S, k, work, lwork, info) != CUSOLVER_STATUS_SUCCESS)
          return FE_ECUDA;
        st = read_info();
        if (st != 0) return FE_EBREAKDOWN;
        passes = std::min(3, pass + 3);
      }
      // U^T <- R^-T U^T  (U <- U R^-1)
      if (cublasDtrsm(hb, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_T, CUBLAS_DIAG_NON_UNIT, k, (int)n,
                      &one, S, k, U, k) != CUBLAS_STATUS_SUCCESS)
        return FE_ECUDA;
    }
    return FE_OK;
  }

  // Rayleigh-Ritz on orthonormal *U: W = H~ U, P = U^T W = Q Lambda Q^T,
  // U <- U Q, W <- W Q; lam (device) ascending, res (device) residual norms.
  fe_status rayleigh_ritz(double** U) {
    const double one = 1.0, zero = 0.0;
    cudaError_t e = scaled(c, true, *U, W, k, 1.0, 0.0, 0.0, s);
    if (e != cudaSuccess) return from_cuda(e);
    if (cublasDgemm(hb, CUBLAS_OP_N, CUBLAS_OP_T, k, k, (int)n, &one, *U, k, W, k, &zero, S, k) !=
        CUBLAS_STATUS_SUCCESS)
      return FE_ECUDA;
    if (cusolverDnDsyevd(hs, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, k, S, k, lam, work, lwork, info) !=
        CUSOLVER_STATUS_SUCCESS)
      return FE_ECUDA;
    const int st = read_info();
    if (st != 0) return st < 0 ? FE_ECUDA : FE_ENONFINITE;
    // (U Q)^T = Q^T U^T
    if (cublasDgemm(hb, CUBLAS_OP_T, CUBLAS_OP_N, k, (int)n, k, &one, S, k, *U, k, &zero, T, k) !=
        CUBLAS_STATUS_SUCCESS)
      return FE_ECUDA;
    std::swap(*U, T);
    if (cublasDgemm(hb, CUBLAS_OP_T, CUBLAS_OP_N, k, (int)n, k, &one, S, k, W, k, &zero, T, k) !=
        CUBLAS_STATUS_SUCCESS)
      return FE_ECUDA;
    std::swap(W, T);
    residual_partial_kernel<<<dim3((k + 31) / 32, kResRows), dim3(32, 8), 0, s>>>(*U, W, lam, n, k, part);
    residual_final_kernel<<<(k + 127) / 128, 128, 0, s>>>(part, k, kResRows, res);
    return from_cuda(cudaGetLastError());
  }

  // Lanczos on H~ from a random free vector: returns the extreme Ritz values
  // and the last off-diagonal (|beta_s| + theta_max bounds the spectrum).
  fe_status lanczos(int steps, unsigned long long seed, double* theta_min, double* theta_max, double* beta_last) {
    double* v = T;            // v and the previous v in T (n x k holds both for k >= 2), w in W
    double* w = W;
    double* vp = T + n;
    if (k < 2) return FE_EINVAL;
    random_vector_kernel<<<1024, 256, 0, s>>>(v, n, seed);
    zero_constrained_kernel<<<1024, 256, 0, s>>>(v, 1, c->mdev, n);
    cudaError_t e = cudaMemsetAsync(vp, 0, n * sizeof(double), s);
    if (e != cudaSuccess) return from_cuda(e);
    double nv = 0.0;
    if (cublasDnrm2(hb, (int)n, v, 1, &nv) != CUBLAS_STATUS_SUCCESS || !(nv > 0)) return FE_ECUDA;
    double inv = 1.0 / nv;
    cublasDscal(hb, (int)n, &inv, v, 1);
    std::vector<double> al, be(1, 0.0);
    double beta = 0.0;
    for (int j = 0; j < steps; ++j) {
      e = scaled(c, true, v, w, 1, 1.0, 0.0, 0.0, s);
      if (e != cudaSuccess) return from_cuda(e);
      double alpha = 0.0;
      if (cublasDdot(hb, (int)n, w, 1, v, 1, &alpha) != CUBLAS_STATUS_SUCCESS) return FE_ECUDA;
      const double ma = -alpha, mb = -beta;
      cublasDaxpy(hb, (int)n, &ma, v, 1, w, 1);
      cublasDaxpy(hb, (int)n, &mb, vp, 1, w, 1);
      if (cublasDnrm2(hb, (int)n, w, 1, &beta) != CUBLAS_STATUS_SUCCESS) return FE_ECUDA;
      if (!std::isfinite(alpha) || !std::isfinite(beta)) return FE_ENONFINITE;
      al.push_back(alpha);
      if (j + 1 < steps) be.push_back(beta);
      if (beta <= 1e-300) break;
      // vp <- v, v <- w / beta
      cublasDcopy(hb, (int)n, v, 1, vp, 1);
      const double ib = 1.0 / beta;
      cublasDcopy(hb, (int)n, w, 1, v, 1);
      cublasDscal(hb, (int)n, &ib, v, 1);
    }
    be.resize(al.size());
    tridiag_extremes(al, be, theta_min, theta_max);
    *beta_last = beta;
    return FE_OK;
  }
};

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
  build_gll_mass(c);
  std::copy(c->mass.begin(), c->mass.end(), m_host);
  return FE_OK;
}

extern "C" fe_status fe_apply_scaled(fe_ctx* c, const void* X, void* Y, int n_vec, double a, double b, double cc,
                                     void* stream) {
  if (!c || n_vec < 0) return FE_EINVAL;
  if (n_vec == 0) return FE_OK;
  if (!X || !Y || !std::isfinite(a) || !std::isfinite(b) || !std::isfinite(cc)) return FE_EINVAL;
  if (c->mode != FE_FP64 && c->mode != FE_FP32) return FE_EUNSUPPORTED;
  const bool fp64 = c->mode == FE_FP64;
  if (overlaps(X, Y, c->n_dofs * (size_t)n_vec * (fp64 ? 8 : 4))) return FE_EINVAL;
  cudaError_t e = ensure_msq(c);
  if (e != cudaSuccess) return from_cuda(e);
  return from_cuda(scaled(c, fp64, X, Y, n_vec, a, b, cc, static_cast<cudaStream_t>(stream)));
}

extern "C" fe_status fe_chebyshev_filter(fe_ctx* c, void* X, void* Y, int n_vec, int degree, double lmin, double lu,
                                         double lmax, void* stream) {
  if (!c || n_vec < 0 || degree < 1) return FE_EINVAL;
  if (n_vec == 0) return FE_OK;
  if (!X || !Y || !(lmin < lu && lu < lmax) || !std::isfinite(lmin) || !std::isfinite(lmax)) return FE_EINVAL;
  if (c->mode != FE_FP64 && c->mode != FE_FP32) return FE_EUNSUPPORTED;
  const bool fp64 = c->mode == FE_FP64;
  const size_t bytes = c->n_dofs * (size_t)n_vec * (fp64 ? 8 : 4);
  if (overlaps(X, Y, bytes)) return FE_EINVAL;
  cudaError_t e = ensure_msq(c);
  if (e != cudaSuccess) return from_cuda(e);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void* x = X;
  void* y = Y;
  e = filter(c, fp64, &x, &y, n_vec, degree, lmin, lu, lmax, s);
  if (e == cudaSuccess && x != X) e = cudaMemcpyAsync(X, x, bytes, cudaMemcpyDeviceToDevice, s);
  return from_cuda(e);
}

extern "C" fe_status fe_chfsi(fe_ctx* c, double* U, int k, const fe_chfsi_desc* d, double* lambda, double* residual,
                              fe_chfsi_info* info, void* stream) {
  if (!c || !U || !d) return FE_EINVAL;
  if (k < 2 || d->n_wanted < 1 || d->n_wanted > k || d->degree < 1 || d->max_iter < 1 || d->lanczos_steps < 2 ||
      !(d->tol > 0) || (d->filter_mode != FE_FP64 && d->filter_mode != FE_FP32))
    return FE_EINVAL;
  size_t free_dofs = c->n_dofs;
  if (!c->periodic)
    free_dofs = (size_t)(c->mdev.Nx - 2) * (c->mdev.Ny - 2) * (c->mdev.Nz - 2);
  if ((size_t)k > free_dofs) return FE_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = ensure_msq(c);
  if (e != cudaSuccess) return from_cuda(e);
  Chfsi ch;
  ch.c = c;
  ch.s = s;
  ch.n = c->n_dofs;
  ch.k = k;
  e = handles(c, s, &ch.hb, &ch.hs);
  if (e != cudaSuccess) return from_cuda(e);
  cublasSetPointerMode(ch.hb, CUBLAS_POINTER_MODE_HOST);
  e = ch.alloc();
  if (e != cudaSuccess) {
    ch.release();
    return from_cuda(e);
  }
  cudaEvent_t ev[2];
  cudaEventCreate(&ev[0]);
  cudaEventCreate(&ev[1]);
  fe_chfsi_info inf{};
  double t_total = 0.0;
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

  double* Ucur = U;
  std::vector<double> hlam(k), hres(k);
  fe_status st = FE_OK;
  double th_min = 0, th_max = 0, beta = 0;
  double t_lz = 0.0;
  st = timed(&t_lz, [&] { return ch.lanczos(d->lanczos_steps, d->seed, &th_min, &th_max, &beta); });
  const double lmax0 = th_max + std::fabs(beta);
  auto pull = [&]() -> fe_status {
    cudaError_t e2 = cudaMemcpyAsync(hlam.data(), ch.lam, k * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e2 == cudaSuccess) e2 = cudaMemcpyAsync(hres.data(), ch.res, k * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(s);
    if (e2 != cudaSuccess) return FE_ECUDA;
    for (int j = 0; j < k; ++j)
      if (!std::isfinite(hlam[j]) || !std::isfinite(hres[j])) return FE_ENONFINITE;
    return FE_OK;
  };
  auto max_res = [&]() { return *std::max_element(hres.begin(), hres.begin() + d->n_wanted); };
  if (st == FE_OK) {
    zero_constrained_kernel<<<1024, 256, 0, s>>>(Ucur, k, c->mdev, ch.n);
    st = timed(&inf.seconds_orth, [&] { return ch.cholqr(Ucur); });
  }
  if (st == FE_OK) st = timed(&inf.seconds_rr, [&] { return ch.rayleigh_ritz(&Ucur); });
  if (st == FE_OK) st = pull();
  double lmax = lmax0, lu = 0, lmin = 0;
  while (st == FE_OK && inf.iterations < d->max_iter && max_res() > d->tol) {
    lu = hlam[k - 1];
    lmin = hlam[0];
    lmax = std::max(lmax0, lu + 1e-3 * std::fabs(lu));
    if (!(lmin < lu)) lmin = lu - 1e-3 * (lmax - lu);
    const bool fp32 = d->filter_mode == FE_FP32 && max_res() > d->fp32_switch;
    st = timed(&inf.seconds_filter, [&]() -> fe_status {
      cudaError_t e2;
      if (fp32) {
        // the FP32 pair lives in W (free during the filter): two n x k float blocks
        float* x32 = reinterpret_cast<float*>(ch.W);
        float* y32 = x32 + ch.n * (size_t)k;
        convert_kernel<double, float><<<2048, 256, 0, s>>>(Ucur, x32, ch.n * (size_t)k);
        void* x = x32;
        void* y = y32;
        e2 = filter(c, false, &x, &y, k, d->degree, lmin, lu, lmax, s);
        if (e2 == cudaSuccess)
          convert_kernel<float, double><<<2048, 256, 0, s>>>(static_cast<float*>(x), Ucur, ch.n * (size_t)k);
      } else {
        void* x = Ucur;
        void* y = ch.T;
        e2 = filter(c, true, &x, &y, k, d->degree, lmin, lu, lmax, s);
        if (e2 == cudaSuccess && x != Ucur) {
          // the filtered block is in T: take T as the current block
          ch.T = Ucur;
          Ucur = static_cast<double*>(x);
        }
      }
      if (e2 == cudaSuccess) e2 = cudaGetLastError();
      return from_cuda(e2);
    });
    inf.filter_applies += d->degree;
    if (fp32) inf.fp32_passes++;
    if (st == FE_OK) st = timed(&inf.seconds_orth, [&] { return ch.cholqr(Ucur); });
    if (st == FE_OK) st = timed(&inf.seconds_rr, [&] { return ch.rayleigh_ritz(&Ucur); });
    if (st == FE_OK) st = pull();
    inf.iterations++;
  }
  if (Ucur != U) {
    // the result sits in one of the work blocks: copy it home, and hand the
    // user's block back to the work set so that release() frees the right ones
    cudaError_t e2 = cudaMemcpyAsync(U, Ucur, ch.n * (size_t)k * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(s);
    if (ch.W == U) ch.W = Ucur;
    else if (ch.T == U) ch.T = Ucur;
    if (e2 != cudaSuccess && st == FE_OK) st = FE_ECUDA;
  }
  cudaStreamSynchronize(s);
  ch.release();
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  if (st == FE_OK || st == FE_ENOTCONV) {
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
