// Learned cell-patch preconditioner for the block-PCG solve.
//
//   z = D^-1 r + sum_e R_e^T ( w_e .* s_e MLP(R_e r / s_e) ),
//   MLP(u) = W2 relu(W1 u + b1) + b2,   W1: 128 x n_p^3,  W2: n_p^3 x 128,
//
// s_e = ||R_e r|| per cell and column (the network sees unit-norm patches and
// its output is scaled back, so z is positively homogeneous in r), w_e the
// partition-of-unity weights 1 / (number of cells sharing the node), D the
// diagonal of A.  With W2 = 0 and b2 = 0 the preconditioner is Jacobi.  The
// network is trained on the residual / error trajectory (r_k, e_k = x* - x_k)
// of a Jacobi-PCG solve of the same operator.  Default objective: the energy
// norm of what the preconditioner misses, mean ||e_k - z(r_k)||_A^2 -- the
// norm CG minimises -- with the operator itself in the loss and its gradient;
// alternatives: the operator residual ||A z(r_k) - r_k||^2, or patch
// regression onto the oscillatory part of e_k - D^-1 r_k.  The paper
// has no learned component; this layer sits on top of its operator.
//
// Kernels:
//  * inference: one fused kernel per cell colour.  A CTA takes one cell and
//    128 columns (patches): it gathers the 128 x n_p^3 patch tile into shared
//    memory as BF16, runs GEMM1 (128 x 128 x K1) and GEMM2 (128 x K1 x 128) on
//    the 5th-generation tensor cores (tcgen05.mma kind::f16, BF16 operands,
//    FP32 accumulators in tensor memory), applies 1/s, b1 and ReLU between
//    them, and scales and assembles the output into z.  Colours make the
//    assembly conflict-free, as in the operator.
//  * training: FP32 CUDA-core GEMMs (strided, tiled) for forward and backward,
//    column-sum bias gradients, and Adam, all on the device.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include <cuda_bf16.h>

#include "fe_internal.h"
#include "fe_cell_kernel.cuh"
#include "fe_umma.cuh"
#include "../../include/fe_learn.h"

namespace fe {

constexpr int kHidden = 128;
constexpr int kTile = 128;          // patches (columns) per CTA
constexpr uint32_t kTmemCols = 512;

struct LearnedPrecond {
  int n3 = 0, K1 = 0;
  float *W1 = nullptr, *b1 = nullptr, *W2 = nullptr, *b2 = nullptr;        // FP32 master
  float *mW1 = nullptr, *vW1 = nullptr, *mb1 = nullptr, *vb1 = nullptr;   // Adam moments
  float *mW2 = nullptr, *vW2 = nullptr, *mb2 = nullptr, *vb2 = nullptr;
  __nv_bfloat16 *W1img = nullptr, *W2img = nullptr;                       // tensor-core operand images
  int adam_t = 0;
  bool images_valid = false;
};

// Byte offset of element (row, k) in a K-major no-swizzle tile with `kdim` K.
__host__ __device__ __forceinline__ size_t core_offset(int row, int k, int kdim) {
  return (size_t)(row >> 3) * (kdim / 8) * 128 + (size_t)(k >> 3) * 128 + ((row & 7) * 8 + (k & 7)) * 2;
}

// Local node i of cell (cx,cy,cz): global index, constrained flag, and the
// partition-of-unity weight 1 / (cells sharing the node).
__device__ __forceinline__ void node_info(const MeshDev& m, int P, int np, int cx, int cy, int cz, int i,
                                          size_t* dof, bool* con, float* w) {
  const int i1 = i % np, i2 = (i / np) % np, i3 = i / (np * np);
  const int gx = node_coord(cx, i1, P, m.Nx, m.periodic), gy = node_coord(cy, i2, P, m.Ny, m.periodic),
            gz = node_coord(cz, i3, P, m.Nz, m.periodic);
  *dof = gx + (size_t)m.Nx * (gy + (size_t)m.Ny * gz);
  *con = on_boundary(gx, m.Nx, m.periodic) || on_boundary(gy, m.Ny, m.periodic) || on_boundary(gz, m.Nz, m.periodic);
  auto shared_along = [&](int c, int n, int li) {
    return ((li == 0 && (c > 0 || m.periodic)) || (li == P && (c < n - 1 || m.periodic))) ? 2 : 1;
  };
  *w = 1.0f / (float)(shared_along(cx, m.nx, i1) * shared_along(cy, m.ny, i2) * shared_along(cz, m.nz, i3));
}

struct MlpArgs {
  const __nv_bfloat16* W1img;  // N = 128 hidden x K = K1 inputs, K-major core layout
  const __nv_bfloat16* W2img;  // N = K1 outputs x K = 128 hidden, K-major core layout
  const float* b1;             // 128
  const float* b2;             // n3
  int n3, K1, np;
};

// z += sum over this colour's cells of R_e^T (w .* s MLP(R_e r / s)) for 128
// columns per CTA.  256 threads: thread t serves column (row of the tile)
// t % 128 and half t / 128 of the work of that row (alternate node chunks in
// the gather, alternate 32-column groups in the epilogues), so twice as many
// loads and stores are in flight; warp w reads the TMEM lanes of its quarter
// w % 4.
constexpr int kMlpThreads = 256;
__global__ void __launch_bounds__(kMlpThreads, 1) mlp_precond_kernel(const MlpArgs a, const MeshDev m,
                                                                     const int* __restrict__ cells,
                                                                     const float* __restrict__ R,
                                                                     float* __restrict__ Z, int n_vec, int n_cb,
                                                                     int* status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const size_t img = (size_t)kTile * a.K1 * 2;
  unsigned char* reg0 = smem;             // patch tile, then W2 image
  unsigned char* reg1 = smem + img;       // W1 image
  unsigned char* reg2 = reg1 + img;       // hidden tile (128 x 128 BF16)
  uint64_t* mbar = reinterpret_cast<uint64_t*>(reg2 + kTile * kHidden * 2);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  float* ssq = reinterpret_cast<float*>(tslot + 4);   // [2][128] partial squared norms
  long long* noff = reinterpret_cast<long long*>(ssq + 2 * kTile);   // per node: global DoF, -1 if constrained
  float* nw = reinterpret_cast<float*>(noff + a.K1);                // per node: partition-of-unity weight

  const int t = threadIdx.x, warp = t >> 5;
  const int row = t & (kTile - 1), half = t >> 7;
  const int cb = blockIdx.x % n_cb;
  const int e = cells[blockIdx.x / n_cb];
  const int col = cb * kTile + row;
  const bool active = col < n_vec;
  const int P = a.np - 1;
  const int cx = e % m.nx, cy = (e / m.nx) % m.ny, cz = e / (m.nx * m.ny);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (t == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));

  // the cell's node offsets and weights, once per CTA
  for (int i = t; i < a.K1; i += kMlpThreads) {
    long long off = -1;
    float wgt = 0.f;
    if (i < a.n3) {
      size_t dof;
      bool con;
      node_info(m, P, a.np, cx, cy, cz, i, &dof, &con, &wgt);
      off = con ? -1 : (long long)dof;
    }
    noff[i] = off;
    nw[i] = wgt;
  }
  // W1 image -> shared (straight 16-byte copy)
  {
    const uint4* src = reinterpret_cast<const uint4*>(a.W1img);
    uint4* dst = reinterpret_cast<uint4*>(reg1);
#pragma unroll 4
    for (size_t k = t; k < img / 16; k += kMlpThreads) dst[k] = __ldg(src + k);
  }
  __syncthreads();
  // gather the patch of column `col` (row `row` of the tile), 8 nodes per 16-byte chunk
  float ss = 0.f;
#pragma unroll 4
  for (int kg = half; kg < a.K1 / 8; kg += 2) {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const long long off = noff[kg * 8 + u];
      v[u] = (active && off >= 0) ? __ldg(R + off * n_vec + col) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) ss += v[u] * v[u];
    uint4 chunk;
    chunk.x = pack_bf16(v[0], v[1]);
    chunk.y = pack_bf16(v[2], v[3]);
    chunk.z = pack_bf16(v[4], v[5]);
    chunk.w = pack_bf16(v[6], v[7]);
    *reinterpret_cast<uint4*>(reg0 + core_offset(row, kg * 8, a.K1)) = chunk;
  }
  ssq[half * kTile + row] = ss;

  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("fence.mbarrier_init.release.cluster;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;
  const float s2 = ssq[row] + ssq[kTile + row];
  const float s = sqrtf(s2);
  const float inv_s = s2 > 0.f ? 1.0f / s : 0.f;
  const uint32_t sbo1 = (uint32_t)(a.K1 / 8) * 128;

  // GEMM1: D1[128 patches x 128 hidden] = tile[128 x K1] . W1^T
  if (t == 0) {
    const uint32_t idesc = umma_idesc_bf16(kTile, kHidden);
    for (int k = 0; k < a.K1 / 16; ++k)
      umma_bf16(tmem, umma_desc(smem_u32(reg0) + k * 256, 128, sbo1), umma_desc(smem_u32(reg1) + k * 256, 128, sbo1),
                idesc, k > 0);
    umma_commit(mbar);
  }
  bool ok = mbar_wait_timed(mbar, 0);
  asm volatile("tcgen05.fence::after_thread_sync;");
  // every thread must see GEMM1 complete before the patch tile is overwritten
  __syncthreads();
  const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
  if (ok) {
    // the patch tile is consumed: bring the W2 image into its place
    const uint4* src = reinterpret_cast<const uint4*>(a.W2img);
    uint4* dst = reinterpret_cast<uint4*>(reg0);
#pragma unroll 4
    for (size_t k = t; k < img / 16; k += kMlpThreads) dst[k] = __ldg(src + k);
    // h = relu(D1 / s + b1) -> BF16 hidden tile, row `row`, columns of this half
    for (int c0 = half * 32; c0 < kHidden; c0 += 64) {
      float d[32];
      tmem_ld32(lane_base + c0, d);
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        float h[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) h[u] = fmaxf(fmaf(d[g * 8 + u], inv_s, __ldg(a.b1 + c0 + g * 8 + u)), 0.f);
        uint4 chunk;
        chunk.x = pack_bf16(h[0], h[1]);
        chunk.y = pack_bf16(h[2], h[3]);
        chunk.z = pack_bf16(h[4], h[5]);
        chunk.w = pack_bf16(h[6], h[7]);
        *reinterpret_cast<uint4*>(reg2 + core_offset(row, c0 + g * 8, kHidden)) = chunk;
      }
    }
  } else if (t == 0) {
    atomicMax(status, (int)FE_ETIMEOUT);
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");

  // GEMM2: D2[128 x K1] = hidden[128 x 128] . W2^T, in N chunks of <= 256
  if (ok && t == 0) {
    const uint32_t sbo2 = (uint32_t)(kHidden / 8) * 128;
    for (int n0 = 0; n0 < a.K1; n0 += 256) {
      const int nn = a.K1 - n0 < 256 ? a.K1 - n0 : 256;
      const uint32_t idesc = umma_idesc_bf16(kTile, nn);
      for (int k = 0; k < kHidden / 16; ++k)
        umma_bf16(tmem + kHidden + n0, umma_desc(smem_u32(reg2) + k * 256, 128, sbo2),
                  umma_desc(smem_u32(reg0) + (uint32_t)(n0 / 8) * sbo2 + k * 256, 128, sbo2), idesc, k > 0);
    }
    umma_commit(mbar);
  }
  if (ok) ok = mbar_wait_timed(mbar, 1);
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok) {
    for (int c0 = half * 32; c0 < a.K1; c0 += 64) {
      float d[32];
      tmem_ld32(lane_base + kHidden + c0, d);
      if (!active) continue;
      // all 32 reads of z are issued before the first store (a store may
      // alias a later read as far as the compiler knows), so they overlap
      float zold[32];
#pragma unroll
      for (int u = 0; u < 32; ++u) {
        const int i = c0 + u;
        const long long off = i < a.n3 ? noff[i] : -1;
        zold[u] = off >= 0 ? Z[off * n_vec + col] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 32; ++u) {
        const int i = c0 + u;
        const long long off = i < a.n3 ? noff[i] : -1;
        if (off >= 0) Z[off * n_vec + col] = zold[u] + (d[u] + __ldg(a.b2 + i)) * s * nw[i];
      }
    }
  } else if (t == 0) {
    atomicMax(status, (int)FE_ETIMEOUT);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// z = dinv .* r
__global__ void jacobi_init_kernel(const float* __restrict__ r, const float* __restrict__ dinv, float* __restrict__ z,
                                   size_t n, int nv) {
  const size_t total = n * nv;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
    z[i] = r[i] * dinv[i / nv];
}

// Operand images: W1 (128 x n3, row-major) -> N=128 x K=K1 core layout;
// W2 (n3 x 128) -> N=K1 x K=128 core layout; padding zero.
__global__ void build_images_kernel(const float* W1, const float* W2, __nv_bfloat16* W1img, __nv_bfloat16* W2img,
                                    int n3, int K1) {
  const int total = kHidden * K1;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const int h = idx / K1, k = idx % K1;   // W1 element (h, k)
    const float v1 = k < n3 ? W1[(size_t)h * n3 + k] : 0.f;
    *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<char*>(W1img) + core_offset(h, k, K1)) = __float2bfloat16(v1);
    const int o = idx / kHidden, j = idx % kHidden;   // W2 element (o, j)
    const float v2 = o < n3 ? W2[(size_t)o * kHidden + j] : 0.f;
    *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<char*>(W2img) + core_offset(o, j, kHidden)) =
        __float2bfloat16(v2);
  }
}

// ---------------------------------------------------------------------------
// training kernels (FP32, CUDA cores)
// ---------------------------------------------------------------------------

// C[m][n] = sum_k A(m,k) B(k,n), A(m,k) = A[m sam + k sak], B(k,n) = B[k sbk + n sbn], C row-major ldc.
// blockIdx.z takes the slice [z kchunk, (z + 1) kchunk) of k and writes its
// partial product to C + z c_slice (one slice: the whole product).
__global__ void __launch_bounds__(256) sgemm_strided(int M, int N, int K, const float* __restrict__ A, long sam,
                                                     long sak, const float* __restrict__ B, long sbk, long sbn,
                                                     float* __restrict__ C, int ldc, int kchunk, size_t c_slice) {
  __shared__ float As[16][64 + 1];
  __shared__ float Bs[16][64 + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
  C += blockIdx.z * c_slice;
  float acc[4][4] = {};
  for (int k0 = kb; k0 < ke; k0 += 16) {
    for (int l = threadIdx.x; l < 16 * 64; l += 256) {
      const int kk = l / 64, mm = l % 64;
      const int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < M && gk < ke) ? A[gm * sam + gk * sak] : 0.f;
      const int gn = n0 + mm;
      Bs[kk][mm] = (gn < N && gk < ke) ? B[gk * sbk + gn * sbn] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gm = m0 + ty * 4 + i, gn = n0 + tx * 4 + j;
      if (gm < M && gn < N) C[(size_t)gm * ldc + gn] = acc[i][j];
    }
}

// C[i] = sum over the S slices of part[z][i], in slice order (deterministic).
__global__ void sum_slices_kernel(const float* __restrict__ part, int S, size_t n, float* __restrict__ C) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int z = 0; z < S; ++z) acc += part[z * n + i];
    C[i] = acc;
  }
}

constexpr int kMaxSlices = 32;   // slices of k of a split product (part holds kMaxSlices x M x N)

// C = A B (M x N, row-major).  A product with few 64 x 64 output tiles and a
// long k (the weight gradients: k runs over every patch of a snapshot) is
// split into slices of k, so that about two CTAs per SM work on it, when a
// slice buffer `part` is given; the slices are then summed in order.
static cudaError_t gemm(int M, int N, int K, const float* A, long sam, long sak, const float* B, long sbk, long sbn,
                        float* C, cudaStream_t s, float* part = nullptr) {
  dim3 grid((N + 63) / 64, (M + 63) / 64);
  const int tiles = (int)(grid.x * grid.y);
  int S = 1;
  if (part && tiles < 152) S = std::min(std::min(kMaxSlices, (2 * 152 + tiles - 1) / tiles), std::max(1, K / 1024));
  if (S <= 1) {
    sgemm_strided<<<grid, 256, 0, s>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, N, K, 0);
    return cudaGetLastError();
  }
  const int kc = ((K + S - 1) / S + 15) / 16 * 16;
  grid.z = (K + kc - 1) / kc;
  const size_t mn = (size_t)M * N;
  sgemm_strided<<<grid, 256, 0, s>>>(M, N, K, A, sam, sak, B, sbk, sbn, part, N, kc, mn);
  sum_slices_kernel<<<(unsigned)std::min<size_t>((mn + 255) / 256, 1024), 256, 0, s>>>(part, (int)grid.z, mn, C);
  return cudaGetLastError();
}

// X[r][c] = act(X[r][c] + b[c]); act = relu when relu != 0
__global__ void bias_act_kernel(float* X, const float* b, int rows, int cols, int relu) {
  const size_t total = (size_t)rows * cols;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const float v = X[i] + b[i % cols];
    X[i] = relu ? fmaxf(v, 0.f) : v;
  }
}

// dY = (2 / (rows cols)) (Y - T), partial squared errors per CTA
__global__ void mse_grad_kernel(const float* Y, const float* T, float* dY, size_t total, float scale, float* partial) {
  __shared__ float red[256];
  float acc = 0.f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const float d = Y[i] - T[i];
    dY[i] = 2.f * scale * d;
    acc += d * d;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// out = sum of partial[0..n) (one CTA, fixed order)
__global__ void sum_kernel(const float* partial, int n, float scale, float* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    float s = 0.f;
    for (int i = 0; i < n; ++i) s += partial[i];
    *out = s * scale;
  }
}

// g[c] = sum_r X[r][c]
__global__ void colsum_kernel(const float* X, int rows, int cols, float* g) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += X[(size_t)r * cols + c];
  g[c] = s;
}

// dH .*= (H > 0)
__global__ void relu_grad_kernel(float* dH, const float* H, size_t total) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
    if (!(H[i] > 0.f)) dH[i] = 0.f;
}

__global__ void adam_kernel(float* w, const float* g, float* mo, float* ve, size_t n, float lr, float b1, float b2,
                            float bc1, float bc2, float eps) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float m = b1 * mo[i] + (1.f - b1) * gi;
    const float v = b2 * ve[i] + (1.f - b2) * gi * gi;
    mo[i] = m;
    ve[i] = v;
    w[i] -= lr * (m / bc1) / (sqrtf(v / bc2) + eps);
  }
}

struct Gll {
  float x[16];
};

// Training patches of one snapshot: for cell cells[k / ncol] and column k % ncol,
// U = R_e r / s and T = HF(R_e (e - dinv r)) / s with s = ||R_e r||, where HF
// removes the trilinear interpolant of the patch's eight corner values (the
// part of the correction a cell-local map cannot see; vertices keep Jacobi).
__global__ void gather_samples_kernel(const MeshDev m, int np, int n3, const int* cells, int ncol,
                                      const float* __restrict__ r, const float* __restrict__ err,
                                      const float* __restrict__ dinv, int nv, float* U, float* T, size_t row0,
                                      const Gll gll) {
  __shared__ float red[128];
  const int k = blockIdx.x;
  const int e = cells[k / ncol], j = k % ncol;
  const int cx = e % m.nx, cy = (e / m.nx) % m.ny, cz = e / (m.nx * m.ny);
  const int P = np - 1;
  float ss = 0.f;
  for (int i = threadIdx.x; i < n3; i += blockDim.x) {
    size_t dof;
    bool con;
    float w;
    node_info(m, P, np, cx, cy, cz, i, &dof, &con, &w);
    const float v = con ? 0.f : r[dof * nv + j];
    ss += v * v;
  }
  red[threadIdx.x] = ss;
  __syncthreads();
  for (int s = 64; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  const float inv = red[0] > 0.f ? rsqrtf(red[0]) : 0.f;
  float* u = U + (row0 + k) * n3;
  float* t = T + (row0 + k) * n3;
  __shared__ float corner[8];
  auto corr = [&](int i, float* rvo) {
    size_t dof;
    bool con;
    float w;
    node_info(m, P, np, cx, cy, cz, i, &dof, &con, &w);
    const float rv = con ? 0.f : r[dof * nv + j];
    if (rvo) *rvo = rv;
    return con ? 0.f : err[dof * nv + j] - dinv[dof] * rv;
  };
  if (threadIdx.x < 8) {
    const int a = threadIdx.x & 1, b = (threadIdx.x >> 1) & 1, c = threadIdx.x >> 2;
    corner[threadIdx.x] = corr(a * P + np * (b * P + np * c * P), nullptr);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n3; i += blockDim.x) {
    float rv;
    const float ev = corr(i, &rv);
    const int i1 = i % np, i2 = (i / np) % np, i3 = i / (np * np);
    const float l1[2] = {0.5f * (1.f - gll.x[i1]), 0.5f * (1.f + gll.x[i1])};
    const float l2[2] = {0.5f * (1.f - gll.x[i2]), 0.5f * (1.f + gll.x[i2])};
    const float l3[2] = {0.5f * (1.f - gll.x[i3]), 0.5f * (1.f + gll.x[i3])};
    float smooth = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) smooth += corner[q] * l1[q & 1] * l2[(q >> 1) & 1] * l3[q >> 2];
    u[i] = rv * inv;
    t[i] = (ev - smooth) * inv;
  }
}

// dst[b] = src[idx[b]] rows of length n3 (mini-batch gather)
__global__ void gather_rows_kernel(const float* src, const int* idx, int rows, int n3, float* dst) {
  const size_t total = (size_t)rows * n3;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t r = i / n3, c = i % n3;
    dst[i] = src[(size_t)idx[r] * n3 + c];
  }
}

// Operator-in-the-loop objective: inputs of every (cell, column) patch,
// U[row] = R_e r / s and S[row] = s = ||R_e r||, row = k * ncol + j for cells[k].
__global__ void gather_inputs_kernel(const MeshDev m, int np, int n3, const int* cells, int ncol,
                                     const float* __restrict__ r, int nv, float* U, float* S) {
  __shared__ float red[128];
  const int k = blockIdx.x;
  const int e = cells[k / ncol], j = k % ncol;
  const int cx = e % m.nx, cy = (e / m.nx) % m.ny, cz = e / (m.nx * m.ny);
  const int P = np - 1;
  float ss = 0.f;
  for (int i = threadIdx.x; i < n3; i += blockDim.x) {
    size_t dof;
    bool con;
    float w;
    node_info(m, P, np, cx, cy, cz, i, &dof, &con, &w);
    const float v = con ? 0.f : r[dof * nv + j];
    ss += v * v;
  }
  red[threadIdx.x] = ss;
  __syncthreads();
  for (int s = 64; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  const float sn = sqrtf(red[0]);
  const float inv = sn > 0.f ? 1.0f / sn : 0.f;
  if (threadIdx.x == 0) S[k] = sn;
  for (int i = threadIdx.x; i < n3; i += blockDim.x) {
    size_t dof;
    bool con;
    float w;
    node_info(m, P, np, cx, cy, cz, i, &dof, &con, &w);
    U[(size_t)k * n3 + i] = con ? 0.f : r[dof * nv + j] * inv;
  }
}

// z += R_e^T (w .* s Y[row])  (training assembly, FP32 atomics)
__global__ void scatter_outputs_kernel(const MeshDev m, int np, int n3, const int* cells, int ncol, const float* Y,
                                       const float* S, float* z, int nv) {
  const int k = blockIdx.x;
  const int e = cells[k / ncol], j = k % ncol;
  const int cx = e % m.nx, cy = (e / m.nx) % m.ny, cz = e / (m.nx * m.ny);
  const float sn = S[k];
  for (int i = threadIdx.x; i < n3; i += blockDim.x) {
    size_t dof;
    bool con;
    float w;
    node_info(m, np - 1, np, cx, cy, cz, i, &dof, &con, &w);
    if (!con) atomicAdd(z + dof * nv + j, w * sn * Y[(size_t)k * n3 + i]);
  }
}

// dY[row][i] = s w_i g[dof(e, i)][j]  (adjoint of the assembly)
__global__ void gather_grad_kernel(const MeshDev m, int np, int n3, const int* cells, int ncol, const float* g,
                                   const float* S, float* dY, int nv) {
  const int k = blockIdx.x;
  const int e = cells[k / ncol], j = k % ncol;
  const int cx = e % m.nx, cy = (e / m.nx) % m.ny, cz = e / (m.nx * m.ny);
  const float sn = S[k];
  for (int i = threadIdx.x; i < n3; i += blockDim.x) {
    size_t dof;
    bool con;
    float w;
    node_info(m, np - 1, np, cx, cy, cz, i, &dof, &con, &w);
    dY[(size_t)k * n3 + i] = con ? 0.f : sn * w * g[dof * nv + j];
  }
}

// g = (2 / N) (q - r) and partial sums of (q - r)^2
__global__ void residual_loss_kernel(const float* q, const float* r, float* g, size_t total, float two_over_n,
                                     float* partial) {
  __shared__ float red[256];
  float acc = 0.f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const float d = q[i] - r[i];
    g[i] = two_over_n * d;
    acc += d * d;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// dst[:, j] = src[:, j] / ||src[:, j]||  (one CTA per column)
__global__ void col_normalize_kernel(const float* src, float* dst, size_t n, int nv) {
  __shared__ float red[256];
  const int j = blockIdx.x;
  float acc = 0.f;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) {
    const float v = src[i * nv + j];
    acc += v * v;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  const float inv = red[0] > 0.f ? rsqrtf(red[0]) : 0.f;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) dst[i * nv + j] = src[i * nv + j] * inv;
}

// scale[j] = 1 / ||src[:, j]||  (one CTA per column)
__global__ void col_invnorm_kernel(const float* src, float* scale, size_t n, int nv) {
  __shared__ float red[256];
  const int j = blockIdx.x;
  float acc = 0.f;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) {
    const float v = src[i * nv + j];
    acc += v * v;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) scale[j] = red[0] > 0.f ? rsqrtf(red[0]) : 0.f;
}

// scale[j] = 1 / sqrt((xs - x)_j . r_j): one over the energy norm of the error
// of column j, since r = A (x* - x); falls back to 1 / ||r_j|| if not positive.
__global__ void col_inv_energy_kernel(const float* xs, const float* x, const float* r, float* scale, size_t n,
                                      int nv) {
  __shared__ float red[2][256];
  const int j = blockIdx.x;
  float er = 0.f, rr = 0.f;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) {
    const float rv = r[i * nv + j];
    er += (xs[i * nv + j] - x[i * nv + j]) * rv;
    rr += rv * rv;
  }
  red[0][threadIdx.x] = er;
  red[1][threadIdx.x] = rr;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      red[0][threadIdx.x] += red[0][threadIdx.x + s];
      red[1][threadIdx.x] += red[1][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    scale[j] = red[0][0] > 0.f ? rsqrtf(red[0][0]) : (red[1][0] > 0.f ? rsqrtf(red[1][0]) : 0.f);
}

// dst = scale_col .* src ; if sub != nullptr: dst = scale_col .* (sub - src)
__global__ void col_scale_kernel(const float* src, const float* sub, const float* scale, float* dst, size_t total,
                                 int nv) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const float v = sub ? sub[i] - src[i] : src[i];
    dst[i] = scale[i % nv] * v;
  }
}

// energy objective: g = (2 / N) q with q = A d, partial sums of d . q
__global__ void energy_loss_kernel(const float* d, const float* q, float* g, size_t total, float two_over_n,
                                   float* partial) {
  __shared__ float red[256];
  float acc = 0.f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    g[i] = two_over_n * q[i];
    acc += d[i] * q[i];
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// err = xs - x  (xs the converged solution)
__global__ void sub_kernel(const float* xs, const float* x, float* err, size_t total) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
    err[i] = xs[i] - x[i];
}

static unsigned grid_for(size_t total) {
  size_t g = (total + 255) / 256;
  return (unsigned)(g == 0 ? 1 : (g > 152 * 16 ? 152 * 16 : g));
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

static fe_status from_cuda(cudaError_t e) {
  return fe::cuda_status(e);
}

static size_t smem_bytes(int K1) {
  return (size_t)2 * kTile * K1 * 2 + kTile * kHidden * 2 + 32 + 2 * kTile * 4 + (size_t)K1 * 12;
}

static cudaError_t alloc_learned(fe_ctx* c) {
  if (c->learned) return cudaSuccess;
  LearnedPrecond* L = new LearnedPrecond();
  L->n3 = c->np * c->np * c->np;
  L->K1 = (L->n3 + 15) / 16 * 16;
  const size_t w1 = (size_t)kHidden * L->n3, w2 = (size_t)L->n3 * kHidden;
  float** bufs[] = {&L->W1, &L->mW1, &L->vW1, &L->W2, &L->mW2, &L->vW2};
  const size_t sz[] = {w1, w1, w1, w2, w2, w2};
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 6 && e == cudaSuccess; ++k) {
    e = cudaMalloc(bufs[k], sz[k] * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(*bufs[k], 0, sz[k] * sizeof(float));
  }
  float** vb[] = {&L->b1, &L->mb1, &L->vb1};
  for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
    e = cudaMalloc(vb[k], kHidden * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(*vb[k], 0, kHidden * sizeof(float));
  }
  float** vb2[] = {&L->b2, &L->mb2, &L->vb2};
  for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
    e = cudaMalloc(vb2[k], L->n3 * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(*vb2[k], 0, L->n3 * sizeof(float));
  }
  if (e == cudaSuccess) e = cudaMalloc(&L->W1img, (size_t)kTile * L->K1 * 2);
  if (e == cudaSuccess) e = cudaMalloc(&L->W2img, (size_t)kTile * L->K1 * 2);
  c->learned = L;
  return e;
}

static cudaError_t refresh_images(fe_ctx* c, cudaStream_t s) {
  LearnedPrecond* L = c->learned;
  build_images_kernel<<<grid_for((size_t)kHidden * L->K1), 256, 0, s>>>(L->W1, L->W2, L->W1img, L->W2img, L->n3,
                                                                       L->K1);
  L->images_valid = true;
  return cudaGetLastError();
}

void free_learned(fe_ctx* c) {
  LearnedPrecond* L = c->learned;
  if (!L) return;
  for (float* p : {L->W1, L->b1, L->W2, L->b2, L->mW1, L->vW1, L->mb1, L->vb1, L->mW2, L->vW2, L->mb2, L->vb2})
    cudaFree(p);
  cudaFree(L->W1img);
  cudaFree(L->W2img);
  delete L;
  c->learned = nullptr;
}

bool learned_ready(const fe_ctx* c, int) {
  return c && c->learned && c->learned->images_valid && c->learned->K1 <= 352;
}

fe_status precond_apply_f32(fe_ctx* c, const float* r, float* z, int nv, cudaStream_t s) {
  LearnedPrecond* L = c->learned;
  if (!L || !L->images_valid) return FE_EINVAL;
  if (L->K1 > 352) return FE_EUNSUPPORTED;
  cudaError_t e = solver_workspace(c, 1);
  if (e != cudaSuccess) return from_cuda(e);
  const size_t n = c->n_dofs;
  jacobi_init_kernel<<<grid_for(n * nv), 256, 0, s>>>(r, c->ws.dinv32, z, n, nv);
  const size_t smem = smem_bytes(L->K1);
  e = ensure_dyn_smem(reinterpret_cast<const void*>(mlp_precond_kernel), smem);
  if (e != cudaSuccess) return from_cuda(e);
  MlpArgs a{L->W1img, L->W2img, L->b1, L->b2, L->n3, L->K1, c->np};
  const int n_cb = (nv + kTile - 1) / kTile;
  for (int k = 0; k < c->colors.n_colors; ++k) {
    const int nc = c->colors.offset[k + 1] - c->colors.offset[k];
    if (nc == 0) continue;
    mlp_precond_kernel<<<(unsigned)((long long)nc * n_cb), kMlpThreads, smem, s>>>(
        a, c->mdev, c->d_cells + c->colors.offset[k], r, z, nv, n_cb, c->d_status);
    if ((e = cudaGetLastError()) != cudaSuccess) return from_cuda(e);
  }
  return FE_OK;
}

fe_status learned_precond_apply(fe_ctx* c, const void* r, void* z, int nv, bool fp64, cudaStream_t s) {
  if (fp64) return FE_EUNSUPPORTED;
  return precond_apply_f32(c, static_cast<const float*>(r), static_cast<float*>(z), nv, s);
}

// One Adam step on a mini-batch (U, T: rows x n3).  Returns the batch loss in *loss_dev.
struct TrainBufs {
  float *Hpre = nullptr, *Y = nullptr, *dY = nullptr, *dH = nullptr;
  float *gW1 = nullptr, *gb1 = nullptr, *gW2 = nullptr, *gb2 = nullptr, *partial = nullptr, *loss = nullptr;
  float* slices = nullptr;   // k slices of the weight-gradient products
};

static cudaError_t alloc_train(TrainBufs& b, int rows, int n3) {
  cudaError_t e = cudaSuccess;
  const size_t sizes[] = {(size_t)rows * kHidden, (size_t)rows * n3, (size_t)rows * n3, (size_t)rows * kHidden,
                          (size_t)kHidden * n3, (size_t)kHidden, (size_t)n3 * kHidden, (size_t)n3, 2048, 1,
                          (size_t)kMaxSlices * kHidden * n3};
  float** ptrs[] = {&b.Hpre, &b.Y, &b.dY, &b.dH, &b.gW1, &b.gb1, &b.gW2, &b.gb2, &b.partial, &b.loss, &b.slices};
  for (int k = 0; k < 11 && e == cudaSuccess; ++k) e = cudaMalloc(ptrs[k], sizes[k] * sizeof(float));
  return e;
}

static void free_train(TrainBufs& b) {
  for (float* p : {b.Hpre, b.Y, b.dY, b.dH, b.gW1, b.gb1, b.gW2, b.gb2, b.partial, b.loss, b.slices}) cudaFree(p);
}

// Forward and backward of the MSE loss for a batch; gradients into b.g*.
static cudaError_t forward_backward(LearnedPrecond* L, TrainBufs& b, const float* U, const float* T, int rows,
                                    cudaStream_t s) {
  const int n3 = L->n3, H = kHidden;
  cudaError_t e;
  // Hpre = U W1^T ; H = relu(Hpre + b1)   (stored in b.Hpre)
  if ((e = gemm(rows, H, n3, U, n3, 1, L->W1, 1, n3, b.Hpre, s)) != cudaSuccess) return e;
  bias_act_kernel<<<grid_for((size_t)rows * H), 256, 0, s>>>(b.Hpre, L->b1, rows, H, 1);
  // Y = H W2^T + b2
  if ((e = gemm(rows, n3, H, b.Hpre, H, 1, L->W2, 1, H, b.Y, s)) != cudaSuccess) return e;
  bias_act_kernel<<<grid_for((size_t)rows * n3), 256, 0, s>>>(b.Y, L->b2, rows, n3, 0);
  const size_t tot = (size_t)rows * n3;
  const int nb = 512;
  mse_grad_kernel<<<nb, 256, 0, s>>>(b.Y, T, b.dY, tot, 1.0f / (float)tot, b.partial);
  sum_kernel<<<1, 32, 0, s>>>(b.partial, nb, 1.0f / (float)tot, b.loss);
  // dW2 = dY^T H ; db2 = colsum dY
  if ((e = gemm(n3, H, rows, b.dY, 1, n3, b.Hpre, H, 1, b.gW2, s, b.slices)) != cudaSuccess) return e;
  colsum_kernel<<<(n3 + 127) / 128, 128, 0, s>>>(b.dY, rows, n3, b.gb2);
  // dH = dY W2 ; relu'
  if ((e = gemm(rows, H, n3, b.dY, n3, 1, L->W2, H, 1, b.dH, s)) != cudaSuccess) return e;
  relu_grad_kernel<<<grid_for((size_t)rows * H), 256, 0, s>>>(b.dH, b.Hpre, (size_t)rows * H);
  // dW1 = dH^T U ; db1 = colsum dH
  if ((e = gemm(H, n3, rows, b.dH, 1, H, U, n3, 1, b.gW1, s, b.slices)) != cudaSuccess) return e;
  colsum_kernel<<<1, 128, 0, s>>>(b.dH, rows, H, b.gb1);
  return cudaGetLastError();
}

static void adam_step(LearnedPrecond* L, TrainBufs& b, float lr, cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  L->adam_t++;
  const float bc1 = 1.f - std::pow(b1, (float)L->adam_t), bc2 = 1.f - std::pow(b2, (float)L->adam_t);
  const size_t w = (size_t)kHidden * L->n3;
  adam_kernel<<<grid_for(w), 256, 0, s>>>(L->W1, b.gW1, L->mW1, L->vW1, w, lr, b1, b2, bc1, bc2, eps);
  adam_kernel<<<1, 128, 0, s>>>(L->b1, b.gb1, L->mb1, L->vb1, kHidden, lr, b1, b2, bc1, bc2, eps);
  adam_kernel<<<grid_for(w), 256, 0, s>>>(L->W2, b.gW2, L->mW2, L->vW2, w, lr, b1, b2, bc1, bc2, eps);
  adam_kernel<<<grid_for(L->n3), 256, 0, s>>>(L->b2, b.gb2, L->mb2, L->vb2, L->n3, lr, b1, b2, bc1, bc2, eps);
}

// Snapshot recorder used as the hook of the trajectory solve.
struct Recorder {
  int every, max_snap, count = 0;
  size_t tot;
  std::vector<float*> r, x;
};

static void record_hook(void* user, int it, const void* x, const void* r, cudaStream_t s) {
  Recorder* rec = static_cast<Recorder*>(user);
  if (rec->count >= rec->max_snap || it % rec->every != 0) return;
  cudaMemcpyAsync(rec->r[rec->count], r, rec->tot * sizeof(float), cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(rec->x[rec->count], x, rec->tot * sizeof(float), cudaMemcpyDeviceToDevice, s);
  rec->count++;
}

}  // namespace fe

using namespace fe;

extern "C" fe_status fe_precond_init(fe_ctx* c, unsigned long long seed) {
  if (!c) return FE_EINVAL;
  if (c->refined) return FE_EUNSUPPORTED;
  cudaError_t e = alloc_learned(c);
  if (e != cudaSuccess) return from_cuda(e);
  LearnedPrecond* L = c->learned;
  std::mt19937_64 rng(seed);
  const float a1 = 1.0f / std::sqrt((float)L->n3), a2 = 1e-3f / std::sqrt((float)kHidden);
  std::uniform_real_distribution<float> u(-1.f, 1.f);
  std::vector<float> W1((size_t)kHidden * L->n3), W2((size_t)L->n3 * kHidden);
  for (auto& v : W1) v = a1 * u(rng);
  for (auto& v : W2) v = a2 * u(rng);
  std::vector<float> zb1(kHidden, 0.f), zb2(L->n3, 0.f);
  return fe_precond_set_weights(c, W1.data(), zb1.data(), W2.data(), zb2.data());
}

extern "C" fe_status fe_precond_set_weights(fe_ctx* c, const float* W1, const float* b1, const float* W2,
                                            const float* b2) {
  if (!c || !W1 || !b1 || !W2 || !b2) return FE_EINVAL;
  cudaError_t e = alloc_learned(c);
  if (e != cudaSuccess) return from_cuda(e);
  LearnedPrecond* L = c->learned;
  const size_t w = (size_t)kHidden * L->n3;
  e = cudaMemcpy(L->W1, W1, w * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(L->b1, b1, kHidden * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(L->W2, W2, w * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(L->b2, b2, L->n3 * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = refresh_images(c, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return from_cuda(e);
}

extern "C" fe_status fe_precond_get_weights(const fe_ctx* c, float* W1, float* b1, float* W2, float* b2) {
  if (!c || !c->learned || !W1 || !b1 || !W2 || !b2) return FE_EINVAL;
  const LearnedPrecond* L = c->learned;
  const size_t w = (size_t)kHidden * L->n3;
  cudaError_t e = cudaMemcpy(W1, L->W1, w * sizeof(float), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(b1, L->b1, kHidden * sizeof(float), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(W2, L->W2, w * sizeof(float), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(b2, L->b2, L->n3 * sizeof(float), cudaMemcpyDeviceToHost);
  return from_cuda(e);
}

extern "C" int fe_precond_input_size(const fe_ctx* c) { return c ? c->np * c->np * c->np : 0; }

extern "C" fe_status fe_precond_apply(fe_ctx* c, const float* R, float* Z, int n_vec, void* stream) {
  if (!c || !R || !Z || n_vec <= 0) return FE_EINVAL;
  if (!c->learned || !c->learned->images_valid) return FE_EINVAL;
  return precond_apply_f32(c, R, Z, n_vec, static_cast<cudaStream_t>(stream));
}

extern "C" fe_status fe_mlp_gradients(fe_ctx* c, const float* U, const float* T, int rows, float* loss, float* gW1,
                                      float* gb1, float* gW2, float* gb2, void* stream) {
  if (!c || !c->learned || !U || !T || rows <= 0 || !loss || !gW1 || !gb1 || !gW2 || !gb2) return FE_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  LearnedPrecond* L = c->learned;
  TrainBufs b;
  cudaError_t e = alloc_train(b, rows, L->n3);
  if (e == cudaSuccess) e = forward_backward(L, b, U, T, rows, s);
  const size_t w = (size_t)kHidden * L->n3;
  if (e == cudaSuccess) e = cudaMemcpyAsync(loss, b.loss, sizeof(float), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(gW1, b.gW1, w * sizeof(float), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(gb1, b.gb1, kHidden * sizeof(float), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(gW2, b.gW2, w * sizeof(float), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(gb2, b.gb2, L->n3 * sizeof(float), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  free_train(b);
  return from_cuda(e);
}

namespace fe {
fe_status pcg_f32(fe_ctx* c, const float* b, float* x, int nv, const double* tol, int max_it, int precond, int* its,
                  cudaStream_t s);
fe_status pcg_f32_hooked(fe_ctx* c, const float* b, float* x, int nv, const double* tol, int max_it,
                         void (*hook)(void*, int, const void*, const void*, cudaStream_t), void* user, int* its,
                         cudaStream_t s, int check_every);
}

namespace fe {
// Held-out data for the checkpoint choice: n_val random right-hand sides of
// their own, solved once by FP32 Jacobi-PCG to relative tolerance 1e-7 (the
// iteration count Jacobi needs, and x* for the held-out snapshots), with
// snapshots (r_k, x_k) of that solve recorded every snapshot_every iterations.
struct Validation {
  float *b = nullptr, *x = nullptr;
  int nv = 0;
  std::vector<double> tol;
  Recorder rec;
};

// Iterations of an FP32 block PCG with the given preconditioner on the
// held-out right-hand sides (capped at max_it; max_it + 1 when it fails),
// recording snapshots into rec when rec is given.
static int validate(fe_ctx* c, Validation& v, int precond, int max_it, Recorder* rec, cudaStream_t s) {
  cudaMemsetAsync(v.x, 0, c->n_dofs * (size_t)v.nv * sizeof(float), s);
  int its = 0;
  fe_status st = rec ? pcg_f32_hooked(c, v.b, v.x, v.nv, v.tol.data(), max_it, record_hook, rec, &its, s, 4)
                     : pcg_f32(c, v.b, v.x, v.nv, v.tol.data(), max_it, precond, &its, s);
  return st == FE_OK ? its : max_it + 1;
}

struct Checkpoint {
  float *W1 = nullptr, *b1 = nullptr, *W2 = nullptr, *b2 = nullptr;
};

static void copy_weights(LearnedPrecond* L, float* W1, float* b1, float* W2, float* b2, bool to_ckpt, cudaStream_t s) {
  const size_t w = (size_t)kHidden * L->n3;
  auto cp = [&](float* ck, float* live, size_t n) {
    if (to_ckpt) cudaMemcpyAsync(ck, live, n * sizeof(float), cudaMemcpyDeviceToDevice, s);
    else cudaMemcpyAsync(live, ck, n * sizeof(float), cudaMemcpyDeviceToDevice, s);
  };
  cp(W1, L->W1, w);
  cp(b1, L->b1, kHidden);
  cp(W2, L->W2, w);
  cp(b2, L->b2, L->n3);
}

// Buffers of the operator-in-the-loop objectives for one snapshot of nv columns.
struct OpBufs {
  float *U = nullptr, *S = nullptr, *rn = nullptr, *z = nullptr, *q = nullptr, *g = nullptr, *en = nullptr,
        *cs = nullptr;
};

static cudaError_t alloc_op(OpBufs& o, size_t rows, int n3, size_t tot, int nv) {
  cudaError_t e = cudaMalloc(&o.U, rows * n3 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&o.S, rows * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&o.cs, nv * sizeof(float));
  for (float** p : {&o.rn, &o.z, &o.q, &o.g, &o.en})
    if (e == cudaSuccess) e = cudaMalloc(p, tot * sizeof(float));
  return e;
}

static void free_op(OpBufs& o) {
  for (float* p : {o.U, o.S, o.rn, o.z, o.q, o.g, o.en, o.cs}) cudaFree(p);
  o = OpBufs{};
}

// Loss and gradients of an operator-in-the-loop objective on one snapshot
// (r = r_k, xk = x_k, xstar = x*; device FP32, num_dofs x nv), for the network
// in L and all cells' patches at once (cells: device list of every cell):
//  energy:   columns scaled by 1 / ||x* - x_k||_A = 1 / sqrt((x* - x_k) . r_k),
//            loss = (1/nv) sum_j (z - e)_j^T A (z - e)_j, dL/dz = (2/nv) A (z - e)
//            (one FP32 operator application);
//  residual: columns scaled by 1 / ||r_k||, loss = (1/nv) ||A z - r||_F^2,
//            dL/dz = (2/nv) A (A z - r) (two applications; A symmetric).
// dL/dz is pulled back through the assembly (s_e w_i per patch entry; s_e is a
// function of the input alone) and then through the network.  Leaves the loss
// in tb.loss and the gradients in tb.gW1, tb.gb1, tb.gW2, tb.gb2.
// what = kLossOnly stops after the loss; kJacobiLoss also takes the network's
// output as zero (z = D^-1 r, the loss of plain Jacobi).
enum { kLossAndGrads = 0, kLossOnly = 1, kJacobiLoss = 2 };
static fe_status operator_step(fe_ctx* c, bool energy, TrainBufs& tb, OpBufs& o, const int* cells, int nv,
                               const float* r, const float* xk, const float* xstar, cudaStream_t s,
                               int what = kLossAndGrads) {
  LearnedPrecond* L = c->learned;
  const int n3 = L->n3;
  const size_t n = c->n_dofs, tot = n * nv;
  const size_t rows = c->n_cells * (size_t)nv;
  cudaError_t e;
  if (energy) col_inv_energy_kernel<<<nv, 256, 0, s>>>(xstar, xk, r, o.cs, n, nv);
  else col_invnorm_kernel<<<nv, 256, 0, s>>>(r, o.cs, n, nv);
  col_scale_kernel<<<grid_for(tot), 256, 0, s>>>(r, nullptr, o.cs, o.rn, tot, nv);
  if (energy) col_scale_kernel<<<grid_for(tot), 256, 0, s>>>(xk, xstar, o.cs, o.en, tot, nv);
  if (what != kJacobiLoss) {
    gather_inputs_kernel<<<(unsigned)rows, 128, 0, s>>>(c->mdev, c->np, n3, cells, nv, o.rn, nv, o.U, o.S);
    if ((e = gemm((int)rows, kHidden, n3, o.U, n3, 1, L->W1, 1, n3, tb.Hpre, s)) != cudaSuccess) return from_cuda(e);
    bias_act_kernel<<<grid_for(rows * kHidden), 256, 0, s>>>(tb.Hpre, L->b1, (int)rows, kHidden, 1);
    if ((e = gemm((int)rows, n3, kHidden, tb.Hpre, kHidden, 1, L->W2, 1, kHidden, tb.Y, s)) != cudaSuccess)
      return from_cuda(e);
    bias_act_kernel<<<grid_for(rows * n3), 256, 0, s>>>(tb.Y, L->b2, (int)rows, n3, 0);
  }
  jacobi_init_kernel<<<grid_for(tot), 256, 0, s>>>(o.rn, c->ws.dinv32, o.z, n, nv);
  if (what != kJacobiLoss)
    scatter_outputs_kernel<<<(unsigned)rows, 128, 0, s>>>(c->mdev, c->np, n3, cells, nv, tb.Y, o.S, o.z, nv);
  const fe_mode saved = c->mode;
  c->mode = FE_FP32;
  fe_status st;
  if (energy) {
    // loss = sum over columns of (z - e)^T A (z - e), divided by the number of
    // columns (an O(1) value per column at any mesh size, which keeps the
    // gradients well above Adam's epsilon); dL/dz = 2 A (z - e) / n_col
    sub_kernel<<<grid_for(tot), 256, 0, s>>>(o.z, o.en, o.g, tot);
    st = fe_apply(c, o.g, o.q, nv, s);
    if (st == FE_OK) {
      energy_loss_kernel<<<512, 256, 0, s>>>(o.g, o.q, o.rn, tot, 2.0f / (float)nv, tb.partial);
      sum_kernel<<<1, 32, 0, s>>>(tb.partial, 512, 1.0f / (float)nv, tb.loss);
      std::swap(o.q, o.rn);   // the gradient dL/dz now sits in q (rn is rebuilt next step)
    }
  } else {
    st = fe_apply(c, o.z, o.q, nv, s);
    if (st == FE_OK) {
      residual_loss_kernel<<<512, 256, 0, s>>>(o.q, o.rn, o.g, tot, 2.0f / (float)nv, tb.partial);
      sum_kernel<<<1, 32, 0, s>>>(tb.partial, 512, 1.0f / (float)nv, tb.loss);
      st = fe_apply(c, o.g, o.q, nv, s);   // q <- A g = dL/dz
    }
  }
  c->mode = saved;
  if (st != FE_OK) return st;
  if (what != kLossAndGrads) return from_cuda(cudaGetLastError());
  gather_grad_kernel<<<(unsigned)rows, 128, 0, s>>>(c->mdev, c->np, n3, cells, nv, o.q, o.S, tb.dY, nv);
  if ((e = gemm(n3, kHidden, (int)rows, tb.dY, 1, n3, tb.Hpre, kHidden, 1, tb.gW2, s, tb.slices)) != cudaSuccess)
    return from_cuda(e);
  colsum_kernel<<<(n3 + 127) / 128, 128, 0, s>>>(tb.dY, (int)rows, n3, tb.gb2);
  if ((e = gemm((int)rows, kHidden, n3, tb.dY, n3, 1, L->W2, kHidden, 1, tb.dH, s)) != cudaSuccess)
    return from_cuda(e);
  relu_grad_kernel<<<grid_for(rows * kHidden), 256, 0, s>>>(tb.dH, tb.Hpre, rows * kHidden);
  if ((e = gemm(kHidden, n3, (int)rows, tb.dH, 1, kHidden, o.U, n3, 1, tb.gW1, s, tb.slices)) != cudaSuccess)
    return from_cuda(e);
  colsum_kernel<<<1, 128, 0, s>>>(tb.dH, (int)rows, kHidden, tb.gb1);
  return from_cuda(cudaGetLastError());
}

// Train by an operator-in-the-loop objective (operator_step) over the
// recorded snapshots, one snapshot per Adam step, with the validation-based
// checkpoint choice described in fe_learn.h.
static fe_status train_operator_loss(fe_ctx* c, const fe_train_desc* d, Recorder& rec, const int* cells, int nv,
                                     fe_train_info* inf, cudaStream_t s, const float* xstar, Validation& val) {
  const bool energy = d->objective == FE_TRAIN_ENERGY;
  LearnedPrecond* L = c->learned;
  const int n3 = L->n3;
  const size_t n = c->n_dofs, tot = n * nv;
  const size_t rows = c->n_cells * (size_t)nv;
  TrainBufs tb;
  OpBufs ob;
  cudaError_t e = alloc_train(tb, (int)rows, n3);
  if (e == cudaSuccess) e = alloc_op(ob, rows, n3, tot, nv);
  fe_status st = from_cuda(e);
  std::mt19937_64 rng(d->seed + 29);
  // checkpoints: epoch 0 is the network with a zero output layer (exactly Jacobi)
  Checkpoint best;
  const size_t wsz = (size_t)kHidden * n3;
  if (st == FE_OK) {
    e = cudaMalloc(&best.W1, wsz * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&best.b1, kHidden * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&best.W2, wsz * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&best.b2, n3 * sizeof(float));
    st = from_cuda(e);
  }
  int val_jac = 0, best_its = 0, best_epoch = 0;
  float val_loss_jac = 0.f, best_loss = 0.f, last_loss = 0.f;
  // mean loss of the live network (or of Jacobi) over the held-out snapshots
  auto held_out_loss = [&](int what, float& out) -> fe_status {
    double sum = 0.0;
    for (int k = 0; k < val.rec.count; ++k) {
      fe_status q = operator_step(c, energy, tb, ob, cells, val.nv, val.rec.r[k], val.rec.x[k], val.x, s, what);
      if (q != FE_OK) return q;
      float h = 0.f;
      cudaMemcpyAsync(&h, tb.loss, sizeof(float), cudaMemcpyDeviceToHost, s);
      cudaError_t ce = cudaStreamSynchronize(s);
      if (ce != cudaSuccess) return from_cuda(ce);
      sum += h;
    }
    out = val.rec.count ? (float)(sum / val.rec.count) : 0.f;
    return FE_OK;
  };
  const bool use_val = st == FE_OK && val.nv > 0;
  if (use_val) {
    // the Jacobi solve of the held-out right-hand sides: iterations to beat,
    // x* and the held-out snapshots
    val_jac = validate(c, val, FE_PRECOND_JACOBI, 100000, &val.rec, s);
    best_its = val_jac;
    copy_weights(L, best.W1, best.b1, best.W2, best.b2, true, s);
    cudaMemsetAsync(best.W2, 0, wsz * sizeof(float), s);
    cudaMemsetAsync(best.b2, 0, n3 * sizeof(float), s);
    st = held_out_loss(kJacobiLoss, val_loss_jac);
    best_loss = val_loss_jac;
  }
  float first = 0.f, last = 0.f, ep_first = 0.f;
  int step = 0;
  const int per_epoch = rec.count;
  for (int ep = 0; ep < d->epochs && st == FE_OK; ++ep) {
    std::vector<int> order(per_epoch);
    for (int k = 0; k < per_epoch; ++k) order[k] = k;
    std::shuffle(order.begin(), order.end(), rng);
    float ep_loss = 0.f;
    for (int oi = 0; oi < per_epoch && st == FE_OK; ++oi) {
      const int k = order[oi];
      st = operator_step(c, energy, tb, ob, cells, nv, rec.r[k], rec.x[k], xstar, s);
      if (st != FE_OK) break;
      adam_step(L, tb, d->lr, s);
      float h = 0.f;
      cudaMemcpyAsync(&h, tb.loss, sizeof(float), cudaMemcpyDeviceToHost, s);
      if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
      if (step == 0) first = h;
      ep_loss += h;
      ++step;
    }
    if (e != cudaSuccess && st == FE_OK) st = from_cuda(e);
    last = per_epoch ? ep_loss / per_epoch : 0.f;
    if (ep == 0) ep_first = last;
    if (st == FE_OK && use_val) {
      float lv = 0.f;
      st = held_out_loss(kLossOnly, lv);
      last_loss = lv;
      if (st == FE_OK && lv < best_loss) {
        best_loss = lv;
        best_epoch = ep + 1;
        copy_weights(L, best.W1, best.b1, best.W2, best.b2, true, s);
      }
    }
  }
  if (st == FE_OK && use_val) {
    // Candidates, in this order: the epoch of the lowest held-out loss and the
    // last epoch.  The first that needs fewer iterations than Jacobi in one
    // held-out solve is kept; if none does, the zero output layer (Jacobi).
    Checkpoint lastw;
    e = cudaMalloc(&lastw.W1, wsz * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&lastw.b1, kHidden * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&lastw.W2, wsz * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&lastw.b2, n3 * sizeof(float));
    if (e != cudaSuccess) st = from_cuda(e);
    if (st == FE_OK) copy_weights(L, lastw.W1, lastw.b1, lastw.W2, lastw.b2, true, s);
    const int last_epoch = d->epochs;
    int cand[2] = {best_epoch, last_epoch != best_epoch ? last_epoch : 0};
    bool kept = false;
    for (int ci = 0; ci < 2 && st == FE_OK && !kept; ++ci) {
      if (cand[ci] <= 0) continue;
      const Checkpoint& w = cand[ci] == best_epoch ? best : lastw;
      copy_weights(L, w.W1, w.b1, w.W2, w.b2, false, s);
      if ((e = refresh_images(c, s)) != cudaSuccess) { st = from_cuda(e); break; }
      const int its = validate(c, val, FE_PRECOND_LEARNED, 2 * val_jac + 10, nullptr, s);
      if (its < val_jac) {
        kept = true;
        best_its = its;
        if (cand[ci] != best_epoch) best_loss = last_loss;
        best_epoch = cand[ci];
      }
    }
    if (st == FE_OK && !kept) {
      copy_weights(L, best.W1, best.b1, best.W2, best.b2, false, s);
      cudaMemsetAsync(L->W2, 0, wsz * sizeof(float), s);
      cudaMemsetAsync(L->b2, 0, n3 * sizeof(float), s);
      best_epoch = 0;
      best_its = val_jac;
      best_loss = val_loss_jac;
    }
    cudaStreamSynchronize(s);
    for (float* p : {lastw.W1, lastw.b1, lastw.W2, lastw.b2}) cudaFree(p);
  }
  inf->val_loss_jacobi = val_loss_jac;
  inf->val_loss_kept = best_loss;
  inf->val_jacobi_iterations = val_jac;
  inf->val_learned_iterations = best_its;
  inf->best_epoch = best_epoch;
  for (float* p : {best.W1, best.b1, best.W2, best.b2}) cudaFree(p);
  inf->loss_first_step = first;
  inf->loss_first_epoch = ep_first;
  inf->loss_last_epoch = last;
  inf->steps = step;
  inf->samples = (long long)rows * rec.count;
  free_train(tb);
  free_op(ob);
  return st;
}
}  // namespace fe

extern "C" fe_status fe_energy_gradients(fe_ctx* c, const float* R, const float* Xk, const float* Xstar, int n_vec,
                                         float* loss, float* gW1, float* gb1, float* gW2, float* gb2, void* stream) {
  if (!c || !c->learned || !R || !Xk || !Xstar || n_vec <= 0 || !loss || !gW1 || !gb1 || !gW2 || !gb2)
    return FE_EINVAL;
  if (c->refined) return FE_EUNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  LearnedPrecond* L = c->learned;
  const int n3 = L->n3;
  const size_t tot = c->n_dofs * (size_t)n_vec, rows = c->n_cells * (size_t)n_vec;
  cudaError_t e = solver_workspace(c, n_vec);   // the Jacobi diagonal of z = D^-1 r + ...
  if (e != cudaSuccess) return from_cuda(e);
  std::vector<int> hcells(c->n_cells);
  for (size_t k = 0; k < c->n_cells; ++k) hcells[k] = (int)k;
  int* cells = nullptr;
  TrainBufs tb;
  OpBufs ob;
  e = cudaMalloc(&cells, c->n_cells * sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(cells, hcells.data(), c->n_cells * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = alloc_train(tb, (int)rows, n3);
  if (e == cudaSuccess) e = alloc_op(ob, rows, n3, tot, n_vec);
  fe_status st = from_cuda(e);
  if (st == FE_OK) st = operator_step(c, true, tb, ob, cells, n_vec, R, Xk, Xstar, s);
  const size_t w = (size_t)kHidden * n3;
  if (st == FE_OK) {
    e = cudaMemcpyAsync(loss, tb.loss, sizeof(float), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(gW1, tb.gW1, w * sizeof(float), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(gb1, tb.gb1, kHidden * sizeof(float), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(gW2, tb.gW2, w * sizeof(float), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(gb2, tb.gb2, n3 * sizeof(float), cudaMemcpyDeviceToDevice, s);
    st = from_cuda(e);
  }
  cudaError_t e2 = cudaStreamSynchronize(s);
  if (st == FE_OK) st = from_cuda(e2);
  free_train(tb);
  free_op(ob);
  cudaFree(cells);
  return st;
}

extern "C" fe_status fe_precond_train(fe_ctx* c, const fe_train_desc* d, fe_train_info* info, void* stream) {
  if (!c || !d || d->n_rhs <= 0 || d->snapshots <= 0 || d->snapshot_every <= 0 || d->epochs < 0 || d->batch <= 0 ||
      !(d->lr > 0.f) || !(d->traj_rtol > 0.0) ||
      (d->objective != FE_TRAIN_OPERATOR_RESIDUAL && d->objective != FE_TRAIN_PATCH_ERROR &&
       d->objective != FE_TRAIN_ENERGY))
    return FE_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  cudaEventRecord(t0, s);
  fe_status st = FE_OK;
  if (!c->learned) st = fe_precond_init(c, d->seed);
  if (st != FE_OK) return st;
  LearnedPrecond* L = c->learned;
  const int nv = d->n_rhs, n3 = L->n3;
  const size_t n = c->n_dofs, tot = n * nv;
  cudaError_t e = solver_workspace(c, nv);
  if (e != cudaSuccess) return from_cuda(e);

  // right-hand sides ~ N(0,1), Dirichlet rows zero (host PRNG, seeded)
  std::vector<float> hb(tot);
  {
    std::mt19937_64 rng(d->seed ^ 0x9E3779B97F4A7C15ULL);
    std::normal_distribution<float> nd(0.f, 1.f);
    const int Nx = c->mdev.Nx, Ny = c->mdev.Ny, Nz = c->mdev.Nz;
    for (size_t i = 0; i < n; ++i) {
      const int gx = (int)(i % Nx), gy = (int)((i / Nx) % Ny), gz = (int)(i / ((size_t)Nx * Ny));
      const bool con = !c->periodic && (gx == 0 || gy == 0 || gz == 0 || gx == Nx - 1 || gy == Ny - 1 || gz == Nz - 1);
      for (int j = 0; j < nv; ++j) hb[i * nv + j] = con ? 0.f : nd(rng);
    }
  }
  float *b = nullptr, *x = nullptr, *err = nullptr, *U = nullptr, *T = nullptr, *Ub = nullptr, *Tb = nullptr;
  int *cells = nullptr, *bidx = nullptr;
  Recorder rec;
  rec.every = d->snapshot_every;
  rec.max_snap = d->snapshots;
  rec.tot = tot;
  TrainBufs tb;
  fe_train_info inf{};
  std::vector<int> hcells(c->n_cells);
  for (size_t k = 0; k < c->n_cells; ++k) hcells[k] = (int)k;
  const size_t per_snap = c->n_cells * (size_t)nv;
  const size_t samples = d->objective == FE_TRAIN_PATCH_ERROR ? per_snap * d->snapshots : 1;
  e = cudaMalloc(&b, tot * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&x, tot * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&err, tot * sizeof(float));
  for (int k = 0; k < d->snapshots && e == cudaSuccess; ++k) {
    float *pr = nullptr, *px = nullptr;
    e = cudaMalloc(&pr, tot * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&px, tot * sizeof(float));
    rec.r.push_back(pr);
    rec.x.push_back(px);
  }
  if (e == cudaSuccess) e = cudaMemcpy(b, hb.data(), tot * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(x, 0, tot * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&cells, c->n_cells * sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(cells, hcells.data(), c->n_cells * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&U, samples * n3 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&T, samples * n3 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&Ub, (size_t)d->batch * n3 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&Tb, (size_t)d->batch * n3 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&bidx, (size_t)d->batch * sizeof(int));
  if (e == cudaSuccess) e = alloc_train(tb, d->batch, n3);
  if (e != cudaSuccess) st = from_cuda(e);

  // Jacobi-PCG trajectory in FP32 with snapshots (r_k, x_k), solved on to traj_rtol for x*
  if (st == FE_OK) {
    std::vector<double> tol(nv, d->traj_rtol);
    // tolerance is absolute on ||r_j||: scale by ||b_j||
    std::vector<double> bn(nv, 0.0);
    for (size_t i = 0; i < n; ++i)
      for (int j = 0; j < nv; ++j) bn[j] += (double)hb[i * nv + j] * hb[i * nv + j];
    for (int j = 0; j < nv; ++j) tol[j] = d->traj_rtol * std::sqrt(bn[j]);
    int its = 0;
    st = pcg_f32_hooked(c, b, x, nv, tol.data(), 200000, record_hook, &rec, &its, s, 8);
    inf.trajectory_iterations = its;
  }
  const bool patch_mode = d->objective == FE_TRAIN_PATCH_ERROR;
  Validation val;
  if (st == FE_OK && !patch_mode && d->n_val > 0) {
    // held-out right-hand sides (their own seed), relative tolerance 1e-7
    val.nv = std::min(d->n_val, nv);
    std::vector<float> hv(n * (size_t)val.nv);
    std::mt19937_64 vr(d->seed ^ 0xD1B54A32D192ED03ULL);
    std::normal_distribution<float> nd(0.f, 1.f);
    std::vector<double> bn(val.nv, 0.0);
    const int Nx = c->mdev.Nx, Ny = c->mdev.Ny, Nz = c->mdev.Nz;
    for (size_t i = 0; i < n; ++i) {
      const int gx = (int)(i % Nx), gy = (int)((i / Nx) % Ny), gz = (int)(i / ((size_t)Nx * Ny));
      const bool con = !c->periodic && (gx == 0 || gy == 0 || gz == 0 || gx == Nx - 1 || gy == Ny - 1 || gz == Nz - 1);
      for (int j = 0; j < val.nv; ++j) {
        const float v = con ? 0.f : nd(vr);
        hv[i * val.nv + j] = v;
        bn[j] += (double)v * v;
      }
    }
    val.tol.resize(val.nv);
    for (int j = 0; j < val.nv; ++j) val.tol[j] = 1e-7 * std::sqrt(bn[j]);
    e = cudaMalloc(&val.b, hv.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&val.x, hv.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(val.b, hv.data(), hv.size() * sizeof(float), cudaMemcpyHostToDevice);
    // held-out snapshots: up to four, spread over the iterations the training
    // snapshots span
    val.rec.max_snap = std::min(d->snapshots, 4);
    val.rec.every = d->snapshot_every * std::max(1, d->snapshots / 4);
    val.rec.tot = hv.size();
    for (int k = 0; k < val.rec.max_snap && e == cudaSuccess; ++k) {
      float *pr = nullptr, *px = nullptr;
      e = cudaMalloc(&pr, hv.size() * sizeof(float));
      if (e == cudaSuccess) e = cudaMalloc(&px, hv.size() * sizeof(float));
      val.rec.r.push_back(pr);
      val.rec.x.push_back(px);
    }
    if (e != cudaSuccess) st = from_cuda(e);
  }
  if (st == FE_OK && !patch_mode) st = train_operator_loss(c, d, rec, cells, nv, &inf, s, x, val);
  cudaFree(val.b);
  cudaFree(val.x);
  for (float* p : val.rec.r) cudaFree(p);
  for (float* p : val.rec.x) cudaFree(p);
  // patch regression: U = R_e r_k / s, T = HF(R_e (x* - x_k - D^-1 r_k)) / s
  Gll gll{};
  for (int i = 0; i < c->np && i < 16; ++i) gll.x[i] = (float)c->gll[i];
  if (st == FE_OK && patch_mode) {
    for (int k = 0; k < rec.count; ++k) {
      sub_kernel<<<grid_for(tot), 256, 0, s>>>(x, rec.x[k], err, tot);
      gather_samples_kernel<<<(unsigned)per_snap, 128, 0, s>>>(c->mdev, c->np, n3, cells, nv, rec.r[k], err,
                                                               c->ws.dinv32, nv, U, T, (size_t)k * per_snap, gll);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) st = from_cuda(e);
  }
  const size_t nsamp = patch_mode ? per_snap * rec.count : 0;
  if (patch_mode) inf.samples = (long long)nsamp;
  // Adam epochs over shuffled mini-batches
  if (st == FE_OK && patch_mode && nsamp > 0) {
    std::mt19937_64 rng(d->seed + 17);
    std::vector<int> perm(nsamp);
    for (size_t i = 0; i < nsamp; ++i) perm[i] = (int)i;
    const int steps_per_epoch = (int)(nsamp / d->batch);
    float first = 0.f, last = 0.f;
    int step = 0;
    for (int ep = 0; ep < d->epochs && st == FE_OK; ++ep) {
      std::shuffle(perm.begin(), perm.end(), rng);
      float ep_loss = 0.f;
      for (int bi = 0; bi < steps_per_epoch; ++bi) {
        cudaMemcpyAsync(bidx, perm.data() + (size_t)bi * d->batch, d->batch * sizeof(int), cudaMemcpyHostToDevice, s);
        gather_rows_kernel<<<grid_for((size_t)d->batch * n3), 256, 0, s>>>(U, bidx, d->batch, n3, Ub);
        gather_rows_kernel<<<grid_for((size_t)d->batch * n3), 256, 0, s>>>(T, bidx, d->batch, n3, Tb);
        if ((e = forward_backward(L, tb, Ub, Tb, d->batch, s)) != cudaSuccess) { st = from_cuda(e); break; }
        adam_step(L, tb, d->lr, s);
        float h = 0.f;
        cudaMemcpyAsync(&h, tb.loss, sizeof(float), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        ep_loss += h;
        if (step == 0) first = h;
        ++step;
      }
      last = steps_per_epoch ? ep_loss / steps_per_epoch : 0.f;
      if (ep == 0) inf.loss_first_epoch = last;
    }
    inf.loss_first_step = first;
    inf.loss_last_epoch = last;
    inf.steps = step;
  }
  if (st == FE_OK) {
    e = refresh_images(c, s);
    if (e != cudaSuccess) st = from_cuda(e);
  }
  cudaEventRecord(t1, s);
  cudaEventSynchronize(t1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, t0, t1);
  inf.seconds = ms * 1e-3;
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  cudaFree(b); cudaFree(x); cudaFree(err); cudaFree(U); cudaFree(T); cudaFree(Ub); cudaFree(Tb);
  cudaFree(cells); cudaFree(bidx);
  for (float* p : rec.r) cudaFree(p);
  for (float* p : rec.x) cudaFree(p);
  free_train(tb);
  if (info) *info = inf;
  return st;
}

extern "C" fe_status fe_precond_save(const fe_ctx* c, const char* path) {
  if (!c || !c->learned || !path) return FE_EINVAL;
  const LearnedPrecond* L = c->learned;
  const size_t w = (size_t)kHidden * L->n3;
  std::vector<float> W1(w), b1(kHidden), W2(w), b2(L->n3);
  fe_status st = fe_precond_get_weights(c, W1.data(), b1.data(), W2.data(), b2.data());
  if (st != FE_OK) return st;
  FILE* f = std::fopen(path, "wb");
  if (!f) return FE_EINVAL;
  const int hdr[4] = {0x4645504c /* "FEPL" */, 1, L->n3, kHidden};
  bool ok = std::fwrite(hdr, sizeof(int), 4, f) == 4;
  ok = ok && std::fwrite(W1.data(), sizeof(float), w, f) == w;
  ok = ok && std::fwrite(b1.data(), sizeof(float), kHidden, f) == (size_t)kHidden;
  ok = ok && std::fwrite(W2.data(), sizeof(float), w, f) == w;
  ok = ok && std::fwrite(b2.data(), sizeof(float), L->n3, f) == (size_t)L->n3;
  ok = (std::fclose(f) == 0) && ok;
  return ok ? FE_OK : FE_EINVAL;
}

extern "C" fe_status fe_precond_load(fe_ctx* c, const char* path) {
  if (!c || !path) return FE_EINVAL;
  FILE* f = std::fopen(path, "rb");
  if (!f) return FE_EINVAL;
  int hdr[4] = {0, 0, 0, 0};
  const int n3 = c->np * c->np * c->np;
  bool ok = std::fread(hdr, sizeof(int), 4, f) == 4 && hdr[0] == 0x4645504c && hdr[1] == 1 && hdr[2] == n3 &&
            hdr[3] == kHidden;
  const size_t w = (size_t)kHidden * n3;
  std::vector<float> W1(w), b1(kHidden), W2(w), b2(n3);
  ok = ok && std::fread(W1.data(), sizeof(float), w, f) == w;
  ok = ok && std::fread(b1.data(), sizeof(float), kHidden, f) == (size_t)kHidden;
  ok = ok && std::fread(W2.data(), sizeof(float), w, f) == w;
  ok = ok && std::fread(b2.data(), sizeof(float), n3, f) == (size_t)n3;
  std::fclose(f);
  if (!ok) return FE_EINVAL;
  return fe_precond_set_weights(c, W1.data(), b1.data(), W2.data(), b2.data());
}
