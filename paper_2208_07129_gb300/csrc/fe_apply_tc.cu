// Host side of the tcgen05 cell kernel (fe_tc_kernel.cuh): the B operands of
// the six passes, built once per context from the FP64 1D tables, the tensor
// maps of X and Y for the TMA boxes, and the per-colour persistent launches.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include <cudaTypedefs.h>

#include "fe_dispatch.cuh"
#include "fe_tc_kernel.cuh"

namespace fe {

namespace {

constexpr int kTcQueues = 32;   // at least the largest colour count (27)
static_assert(kTcCvBytes == kTcCvWords * 4 && tc_cv_index(7, 7, 7) < kTcCvWords,
              "the staged c block built at setup is the one the kernel copies");

using Shape8TF32 = TcShape<8, 2, kTcTF32>;
using Shape8BF16 = TcShape<8, 2, kTcBF16>;

// Entry (n', k') of the per-line B matrix of pass s: rows n' are outputs,
// columns k' inputs, both in blocks of E (quantity, 1D index).  Forward
// passes map nodes i to points q, backward passes points to nodes; N(q, i)
// and D(q, i) are the value and derivative tables with sqrt(w_q) folded in.
// With a metric g (box meshes: one G for every cell, entries 00 01 02 11 12
// 22), B-z takes [c val | dz | dy | dx] and applies G itself:
//   r_aa = N^T (c val) + D^T (g02 dx + g12 dy + g22 dz),
//   r_ab = N^T (g01 dx + g11 dy + g12 dz),  r_ba = N^T (g00 dx + g01 dy + g02 dz).
double tc_bline(int s, int E, int np, int nq, const std::vector<double>& Nf, const std::vector<double>& Df1, int nn,
                int kk, const double* g) {
  const int nb = nn / E, kb = kk / E;
  const bool fwd = s <= 2;
  const int q = fwd ? nn % E : kk % E, i = fwd ? kk % E : nn % E;
  if (q >= nq || i >= np) return 0.0;
  const double Nv = Nf[q * np + i], Dv = Df1[q * np + i];
  switch (s) {
    case 0: return kb == 0 ? (nb == 0 ? Nv : nb == 1 ? Dv : 0.0) : 0.0;                 // [a | b] <- u
    case 1: return (nb == 0 && kb == 0) ? Nv : (nb == 1 && kb == 0) ? Dv : (nb == 2 && kb == 1) ? Nv : 0.0;
    case 2:                                                                              // [val dz dy dx]
      return (nb == 0 && kb == 0) ? Nv : (nb == 1 && kb == 0) ? Dv : (nb == 2 && kb == 1) ? Nv
             : (nb == 3 && kb == 2) ? Nv : 0.0;
    case 3:                                                                              // <- [hv hz hy hx]
      if (g != nullptr) {                                                                // <- [c val dz dy dx]
        static const int row[3][3] = {{5, 4, 2}, {4, 3, 1}, {2, 1, 0}};   // G entry of (output, dz/dy/dx)
        if (kb == 0) return nb == 0 ? Nv : 0.0;
        return g[row[nb][kb - 1]] * (nb == 0 ? Dv : Nv);
      }
      return (nb == 0 && kb == 0) ? Nv : (nb == 0 && kb == 1) ? Dv : (nb == 1 && kb == 2) ? Nv
             : (nb == 2 && kb == 3) ? Nv : 0.0;
    case 4: return (nb == 0 && kb == 0) ? Nv : (nb == 0 && kb == 1) ? Dv : (nb == 1 && kb == 2) ? Nv : 0.0;
    default: return (nb == 0 && kb == 0) ? Nv : (nb == 0 && kb == 1) ? Dv : 0.0;       // out <- [r_a | r_b]
  }
}

uint32_t f32_bits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
}

// Round to TF32 (nearest, ties away from zero: the rounding of cvt.rna) and
// to BF16 (nearest, ties to even).
uint32_t tf32_bits(double x) { return (f32_bits((float)x) + 0x1000u) & 0xffffe000u; }
uint16_t bf16_bits(double x) {
  const uint32_t u = f32_bits((float)x);
  return (uint16_t)((u + 0x7fffu + ((u >> 16) & 1u)) >> 16);
}

template <class SH>
std::vector<unsigned char> tc_image(const fe_ctx* c, const double* g) {
  constexpr int E = SH::E, G = SH::G;
  const int np = c->np, nq = c->nq;
  // derivative of the shape functions at the points, sqrt(w_q) folded in:
  // D(q, i) = sum_k D~(q, k) N(k, i) sqrt(w_q)  (D~ N is exact for n_q >= n_p)
  std::vector<double> Df1((size_t)nq * np, 0.0);
  for (int q = 0; q < nq; ++q)
    for (int i = 0; i < np; ++i) {
      double s = 0.0;
      for (int k = 0; k < nq; ++k) s += c->D1[q * nq + k] * c->N1[k * np + i];
      Df1[q * np + i] = s * std::sqrt(c->qw[q]);
    }
  std::vector<unsigned char> img(SH::B_BYTES, 0);
  for (int s = 0; s < 6; ++s) {
    const int KL = tc_kline(s) * E, NL = tc_nline(s) * E;
    for (int nn = 0; nn < NL; ++nn)
      for (int kk = 0; kk < KL; ++kk) {
        const double v = tc_bline(s, E, np, nq, c->Nf, Df1, nn, kk, g);
        for (int g = 0; g < G; ++g) {
          unsigned char* p = img.data() + SH::b_off(s) + tc_off<SH::ES>(g * NL + nn, g * KL + kk, SH::Kr(s));
          if (SH::KIND == kTcTF32) {
            const uint32_t b = tf32_bits(v);
            std::memcpy(p, &b, 4);
          } else {
            const uint16_t b = bf16_bits(v);
            std::memcpy(p, &b, 2);
          }
        }
      }
  }
  return img;
}

// cuTensorMapEncodeTiled from the driver, looked up once.
PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// Tensor map of a block (node-major, n_vec values per node) as the 4-D
// tensor (vector, x, y, z) of the stored node grid, with the box of one task:
// 8 vectors x n_p^3 nodes.  False where TMA cannot address the block: a base
// not 16-byte aligned, or a node row (n_vec values) not a multiple of 16
// bytes, or fewer vectors than one box row.
bool tc_tensor_map(CUtensorMap* map, const fe_ctx* c, const void* base, int n_vec, bool bf16) {
  const size_t es = bf16 ? 2 : 4;
  if (reinterpret_cast<uintptr_t>(base) % 16 != 0 || (n_vec * es) % 16 != 0 || n_vec < kTcVectors) return false;
  const PFN_cuTensorMapEncodeTiled_v12000 fn = encode_tiled();
  if (fn == nullptr) return false;
  const MeshDev& m = c->mdev;
  const cuuint64_t dims[4] = {(cuuint64_t)n_vec, (cuuint64_t)m.Nx, (cuuint64_t)m.Ny, (cuuint64_t)m.Nz};
  const cuuint64_t strides[3] = {(cuuint64_t)n_vec * es, (cuuint64_t)n_vec * es * m.Nx,
                                 (cuuint64_t)n_vec * es * m.Nx * m.Ny};
  const cuuint32_t box[4] = {(cuuint32_t)kTcVectors, (cuuint32_t)c->np, (cuuint32_t)c->np, (cuuint32_t)c->np};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void*>(base),
            dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int E, int G, int KIND, typename TIO, bool GEN, bool TMA, bool QF>
cudaError_t launch_tc(const fe_ctx* c, const unsigned char* img, const TIO* X, TIO* Y, int n_vec, cudaStream_t s,
                      const CUtensorMap& xm, const CUtensorMap& ym) {
  using SH = TcShape<E, G, KIND>;
  auto kern = tc_apply_kernel<E, G, KIND, TIO, GEN, TMA, QF>;
  // One CTA per SM: its shared-memory request (more than half of an SM's)
  // keeps a second CTA, which would need tensor-memory columns the first
  // holds, off the SM.
  constexpr size_t smem = SH::SMEM_BYTES;
  static_assert(2 * (SH::SMEM_BYTES + 1024) > 228 * 1024, "two CTAs must not fit on one SM");
  cudaError_t e = ensure_dyn_smem(reinterpret_cast<const void*>(kern), smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  // the bulk reduces add every colour's result to Y; every colour's task
  // counter starts at zero
  if (TMA && (e = cudaMemsetAsync(Y, 0, c->n_dofs * (size_t)n_vec * sizeof(TIO), s)) != cudaSuccess) return e;
  if (TMA && (e = cudaMemsetAsync(c->d_tcq, 0, kTcQueues * sizeof(int), s)) != cudaSuccess) return e;
  const Geom<float> geo = make_geom<float>(c);
  TcArgs a{img, nullptr, c->np, c->nq, c->d_status, nullptr, c->d_ptCtc};
  if (QF && TMA && c->d_ptCtc == nullptr) return cudaErrorInvalidValue;
  const int n_vb = (n_vec + kTcVectors - 1) / kTcVectors;
  if (TMA && c->colors.n_colors > kTcQueues) return cudaErrorInvalidValue;
  for (int k = 0; k < c->colors.n_colors; ++k) {
    const int n = c->colors.offset[k + 1] - c->colors.offset[k];
    if (n == 0) continue;
    const long long tasks = (long long)n * n_vb;
    if (tasks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const int grid = (int)std::min<long long>((tasks + SH::SLOTS - 1) / SH::SLOTS, (long long)sms);
    a.cmask = c->d_tcmask + c->colors.offset[k];
    a.queue = c->d_tcq + k;
    kern<<<grid, 128 * SH::SLOTS, smem, s>>>(a, c->mdev, geo, c->d_cells + c->colors.offset[k], (int)tasks, n_vec,
                                              n_vb, X, Y, xm, ym);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// TMA boxes where the blocks allow them (and fe_set_tile has not chosen the
// thread path), the n_q = 8 specialisation where it applies.
template <int KIND, typename TIO>
cudaError_t run_tc(const fe_ctx* c, const unsigned char* img, const void* Xv, void* Yv, int n_vec, cudaStream_t s) {
  const TIO* X = static_cast<const TIO*>(Xv);
  TIO* Y = static_cast<TIO*>(Yv);
  constexpr bool bf16 = sizeof(TIO) == 2;
  const bool gen = c->general != 0;
  CUtensorMap xm, ym;
  std::memset(&xm, 0, sizeof(xm));
  std::memset(&ym, 0, sizeof(ym));
  const bool tma = c->tc_variant != 2 && tc_tensor_map(&xm, c, X, n_vec, bf16) && tc_tensor_map(&ym, c, Y, n_vec, bf16);
  if (tma) {
    if (c->nq == 8)
      return gen ? launch_tc<8, 2, KIND, TIO, true, true, true>(c, img, X, Y, n_vec, s, xm, ym)
                 : launch_tc<8, 2, KIND, TIO, false, true, true>(c, img, X, Y, n_vec, s, xm, ym);
    return gen ? launch_tc<8, 2, KIND, TIO, true, true, false>(c, img, X, Y, n_vec, s, xm, ym)
               : launch_tc<8, 2, KIND, TIO, false, true, false>(c, img, X, Y, n_vec, s, xm, ym);
  }
  return gen ? launch_tc<8, 2, KIND, TIO, true, false, false>(c, img, X, Y, n_vec, s, xm, ym)
             : launch_tc<8, 2, KIND, TIO, false, false, false>(c, img, X, Y, n_vec, s, xm, ym);
}

}  // namespace

// Per cell, in colour order: bits 0-7 / 16-23 / 32-39 mark the nodes along
// x / y / z that exist (index < n_p) and are not Dirichlet nodes, bits 8-15 /
// 24-31 / 40-47 those whose first writer (in colour order) the cell is, by
// the same rules as the cell kernels' assembly.
static std::vector<unsigned long long> tc_cell_masks(const fe_ctx* c) {
  const MeshDev& m = c->mdev;
  const int P = c->p, np = c->np;
  std::vector<unsigned long long> out(c->n_cells);
  for (size_t k = 0; k < c->n_cells; ++k) {
    const int e = c->cells_by_color[k];
    const int cc[3] = {e % m.nx, (e / m.nx) % m.ny, e / (m.nx * m.ny)};
    const int n[3] = {m.nx, m.ny, m.nz}, N[3] = {m.Nx, m.Ny, m.Nz};
    const int odd[3] = {m.last_odd_x, m.last_odd_y, m.last_odd_z};
    unsigned long long w = 0;
    for (int d = 0; d < 3; ++d)
      for (int i = 0; i < np; ++i) {
        const int g = node_coord(cc[d], i, P, N[d], m.periodic);
        if (!on_boundary(g, N[d], m.periodic)) w |= 1ull << (16 * d + i);
        if (first_along(cc[d], n[d], i, P, m.periodic, odd[d])) w |= 1ull << (16 * d + 8 + i);
      }
    out[k] = w;
  }
  return out;
}

cudaError_t build_tc_images(fe_ctx* c) {
  if (c->refined || c->np > 8 || c->nq > 8) return cudaSuccess;   // no tcgen05 kernel for this shape
  // Box meshes: every cell has the same metric (the same diagonal Jacobian;
  // the FP64 values of different cells agree to rounding), folded into B-z.
  const double* g = nullptr;
  if (!c->general) {
    g = c->cellG.data();
    for (size_t e = 1; e < c->n_cells; ++e)
      for (int k = 0; k < 6; ++k)
        if (std::fabs(c->cellG[e * 6 + k] - g[k]) > 1e-12 * (std::fabs(g[k]) + std::fabs(g[0])))
          return cudaSuccess;   // not one metric: no tcgen05 kernel
  }
  const std::vector<unsigned char> t = tc_image<Shape8TF32>(c, g), b = tc_image<Shape8BF16>(c, g);
  const std::vector<unsigned long long> masks = tc_cell_masks(c);
  cudaError_t e = cudaMalloc(&c->d_tcmask, masks.size() * sizeof(unsigned long long));
  if (e == cudaSuccess)
    e = cudaMemcpy(c->d_tcmask, masks.data(), masks.size() * sizeof(unsigned long long), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_tcq, kTcQueues * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_tcimg[0], t.size());
  if (e == cudaSuccess) e = cudaMemcpy(c->d_tcimg[0], t.data(), t.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_tcimg[1], b.size());
  if (e == cudaSuccess) e = cudaMemcpy(c->d_tcimg[1], b.data(), b.size(), cudaMemcpyHostToDevice);
  return e;
}

bool tc_supported(const fe_ctx* c) {
  return c->d_tcimg[0] != nullptr && c->d_tcimg[1] != nullptr && c->d_tcmask != nullptr && c->d_tcq != nullptr;
}

cudaError_t apply_tc(const fe_ctx* c, const void* X, void* Y, int n_vec, cudaStream_t s, fe_mode mode) {
  if (!tc_supported(c)) return cudaErrorInvalidValue;
  if (mode == FE_TF32) return run_tc<kTcTF32, float>(c, c->d_tcimg[0], X, Y, n_vec, s);
  if (mode == FE_BF16) return run_tc<kTcBF16, float>(c, c->d_tcimg[1], X, Y, n_vec, s);
  if (mode == FE_BF16S) return run_tc<kTcBF16, __nv_bfloat16>(c, c->d_tcimg[1], X, Y, n_vec, s);
  return cudaErrorInvalidValue;
}

}  // namespace fe
