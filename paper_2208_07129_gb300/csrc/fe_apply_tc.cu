// Host side of the tcgen05 cell kernel (fe_tc_kernel.cuh): the B operands of
// the six passes, built once per context from the FP64 1D tables, and the
// per-colour persistent launches.
#include <cmath>
#include <cstring>
#include <vector>

#include "fe_dispatch.cuh"
#include "fe_tc_kernel.cuh"

namespace fe {

namespace {

using Shape8TF32 = TcShape<8, 2, kTcTF32>;
using Shape8BF16 = TcShape<8, 2, kTcBF16>;

// Entry (n', k') of the per-line B matrix of pass s: rows n' are outputs,
// columns k' inputs, both in blocks of E (quantity, 1D index).  Forward
// passes map nodes i to points q, backward passes points to nodes; N(q, i)
// and D(q, i) are the value and derivative tables with sqrt(w_q) folded in.
double tc_bline(int s, int E, int np, int nq, const std::vector<double>& Nf, const std::vector<double>& Df1, int nn,
                int kk) {
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
std::vector<unsigned char> tc_image(const fe_ctx* c) {
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
        const double v = tc_bline(s, E, np, nq, c->Nf, Df1, nn, kk);
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

template <int E, int G, int KIND, typename TIO, bool GEN>
cudaError_t launch_tc(const fe_ctx* c, const unsigned char* img, const TIO* X, TIO* Y, int n_vec, cudaStream_t s) {
  using SH = TcShape<E, G, KIND>;
  auto kern = tc_apply_kernel<E, G, KIND, TIO, GEN>;
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
  const Geom<float> geo = make_geom<float>(c);
  TcArgs a{img, nullptr, c->np, c->nq, c->d_status};
  const int n_vb = (n_vec + kTcVectors - 1) / kTcVectors;
  for (int k = 0; k < c->colors.n_colors; ++k) {
    const int n = c->colors.offset[k + 1] - c->colors.offset[k];
    if (n == 0) continue;
    const long long tasks = (long long)n * n_vb;
    if (tasks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const int grid = (int)std::min<long long>((tasks + SH::SLOTS - 1) / SH::SLOTS, (long long)sms);
    a.cmask = c->d_tcmask + c->colors.offset[k];
    kern<<<grid, 128 * SH::SLOTS, smem, s>>>(a, c->mdev, geo, c->d_cells + c->colors.offset[k], (int)tasks, n_vec,
                                              n_vb, X, Y);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
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
  const std::vector<unsigned char> t = tc_image<Shape8TF32>(c), b = tc_image<Shape8BF16>(c);
  const std::vector<unsigned long long> masks = tc_cell_masks(c);
  cudaError_t e = cudaMalloc(&c->d_tcmask, masks.size() * sizeof(unsigned long long));
  if (e == cudaSuccess)
    e = cudaMemcpy(c->d_tcmask, masks.data(), masks.size() * sizeof(unsigned long long), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_tcimg[0], t.size());
  if (e == cudaSuccess) e = cudaMemcpy(c->d_tcimg[0], t.data(), t.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_tcimg[1], b.size());
  if (e == cudaSuccess) e = cudaMemcpy(c->d_tcimg[1], b.data(), b.size(), cudaMemcpyHostToDevice);
  return e;
}

bool tc_supported(const fe_ctx* c) {
  return c->d_tcimg[0] != nullptr && c->d_tcimg[1] != nullptr && c->d_tcmask != nullptr;
}

cudaError_t apply_tc(const fe_ctx* c, const void* X, void* Y, int n_vec, cudaStream_t s, fe_mode mode) {
  if (!tc_supported(c)) return cudaErrorInvalidValue;
  const bool gen = c->general != 0;
  if (mode == FE_TF32) {
    const float* x = static_cast<const float*>(X);
    float* y = static_cast<float*>(Y);
    return gen ? launch_tc<8, 2, kTcTF32, float, true>(c, c->d_tcimg[0], x, y, n_vec, s)
               : launch_tc<8, 2, kTcTF32, float, false>(c, c->d_tcimg[0], x, y, n_vec, s);
  }
  if (mode == FE_BF16) {
    const float* x = static_cast<const float*>(X);
    float* y = static_cast<float*>(Y);
    return gen ? launch_tc<8, 2, kTcBF16, float, true>(c, c->d_tcimg[1], x, y, n_vec, s)
               : launch_tc<8, 2, kTcBF16, float, false>(c, c->d_tcimg[1], x, y, n_vec, s);
  }
  if (mode == FE_BF16S) {
    const __nv_bfloat16* x = static_cast<const __nv_bfloat16*>(X);
    __nv_bfloat16* y = static_cast<__nv_bfloat16*>(Y);
    return gen ? launch_tc<8, 2, kTcBF16, __nv_bfloat16, true>(c, c->d_tcimg[1], x, y, n_vec, s)
               : launch_tc<8, 2, kTcBF16, __nv_bfloat16, false>(c, c->d_tcimg[1], x, y, n_vec, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace fe
