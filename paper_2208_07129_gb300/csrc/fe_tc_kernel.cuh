// Tensor-core cell kernel on the 5th-generation tensor cores (tcgen05):
// the sum-factorised contractions of Algorithm 2 as batched GEMMs
// (Sec. 3.2.4, eqs. tc1-tc3: each 1D pass is a matrix product over all lines
// of a cell and a block of vectors), FP32 accumulation in tensor memory.
//
// Work unit (task): one cell and 8 vectors.  The cell's data for the 8
// vectors is a set of 1D lines; a "row" of an operand is one (line group,
// vector) pair, where a line group holds G lines that differ in the
// coordinate the NEXT pass contracts.  Every pass is one GEMM per 128 rows,
//   D[row][n] = sum_k A[row][k] B[n][k],
// with A in shared memory (K-major core matrices), B a small constant matrix
// built from the 1D tables, D in tensor memory.  Six passes per task:
//   F-x: a = N_x u, b = D_x u                (K = u along x)
//   F-y: aa = N_y a, ab = D_y a, ba = N_y b  (K = [a | b] along y)
//   F-z: val = N_z aa, dz = D_z aa, dy = N_z ab, dx = N_z ba
//        then the quadrature-point operation in registers:
//        [hx hy hz] = G [dx dy dz] (G = mu det J J^-1 J^-T), hv = c val
//        (c = det J V); weights are folded into N and D as sqrt(w)
//   B-z: r_aa = N_z^T hv + D_z^T hz, r_ab = N_z^T hy, r_ba = N_z^T hx
//   B-y: r_a = N_y^T r_aa + D_y^T r_ab, r_b = N_y^T r_ba
//   B-x: out = N_x^T r_a + D_x^T r_b, then the colour-ordered scatter.
// N and D here are the 1D value and derivative matrices at the quadrature
// points (n_q x n_p); sums of several products land in one GEMM by
// concatenating the operands along K, and a line group's G lines by a
// block-diagonal B.  All 1D extents are padded to E.
//
// Between passes each thread reads its row of D from tensor memory and writes
// the values, transposed, into the next pass's A layout: a warp holds 4 line
// groups x 8 vectors, which land in one 128-byte core matrix per store, so the
// stores are free of bank conflicts.  After F-z the thread owns all four
// quadrature-point quantities of its lines and applies the point operation
// without any exchange.
//
// Operands: TF32 (kind::tf32, G = 1) or BF16 (kind::f16, G = 2), both rounded
// to nearest from FP32; the quadrature-point operation is FP32.  Storage of X
// and Y: FP32 or BF16.  Assembly: colour-ordered, the first writer of a node
// stores and later colours add, as in the CUDA-core kernels.
#pragma once

#include <cuda_bf16.h>

#include "fe_cell_kernel.cuh"
#include "fe_umma.cuh"

namespace fe {

constexpr int kTcTF32 = 0, kTcBF16 = 1;
constexpr int kTcVectors = 8;   // vectors per task (the rows of a core matrix)

__host__ __device__ constexpr int tc_round_up(int x, int m) { return (x + m - 1) / m * m; }
// K and N per line of pass s (0 F-x, 1 F-y, 2 F-z, 3 B-z, 4 B-y, 5 B-x) in units of E.
__host__ __device__ constexpr int tc_kline(int s) { return s == 0 ? 1 : s == 1 ? 2 : s == 2 ? 3 : s == 3 ? 4 : s == 4 ? 3 : 2; }
__host__ __device__ constexpr int tc_nline(int s) { return s == 0 ? 2 : s == 1 ? 3 : s == 2 ? 4 : s == 3 ? 3 : s == 4 ? 2 : 1; }

template <int E_, int G_, int KIND_>
struct TcShape {
  static constexpr int E = E_, G = G_, KIND = KIND_;
  static constexpr int ES = KIND == kTcTF32 ? 4 : 2;          // bytes per operand element
  static constexpr int KC = 16 / ES;                          // K per core matrix
  static constexpr int KI = KIND == kTcTF32 ? 8 : 16;         // K per MMA instruction
  static constexpr int H = E / G;                             // line groups per line coordinate
  static constexpr int LINES = E * H;                         // line groups per pass
  static constexpr int ROWS = LINES * kTcVectors;
  static constexpr int T = (ROWS + 127) / 128;                // M = 128 tiles per pass
  static_assert(E % G == 0 && G * ES == 4, "a packed store holds G operands in 4 bytes");
  __host__ __device__ static constexpr int Kr(int s) { return tc_round_up(G * tc_kline(s) * E, KI); }
  __host__ __device__ static constexpr int Nr(int s) { return tc_round_up(G * tc_nline(s) * E, 16); }
  __host__ __device__ static constexpr int b_off(int s) {
    return s == 0 ? 0 : b_off(s - 1) + Nr(s - 1) * Kr(s - 1) * ES;
  }
  static constexpr int B_BYTES = b_off(6);
  static constexpr int S_BYTES = T * 128 * Kr(0) * ES;        // A of F-x (the gathered cell tile)
  __host__ __device__ static constexpr int kr_max() {
    int m = 0;
    for (int s = 1; s < 6; ++s) m = Kr(s) > m ? Kr(s) : m;
    return m;
  }
  static constexpr int M_BYTES = T * 128 * kr_max() * ES;     // A of the other passes (one buffer, reused)
  __host__ __device__ static constexpr int d_cols_max() {
    int m = 0;
    for (int s = 0; s < 6; ++s) m = T * Nr(s) > m ? T * Nr(s) : m;
    return m;
  }
  static constexpr int TMEM_COLS = d_cols_max() <= 32 ? 32 : d_cols_max() <= 64 ? 64 : d_cols_max() <= 128 ? 128
                                   : d_cols_max() <= 256 ? 256 : 512;
  static constexpr int SMEM_BYTES = B_BYTES + S_BYTES + M_BYTES + 64;
};

// Byte offset of element (row, k) of a K-major operand whose rows hold kr values.
template <int ES>
__host__ __device__ __forceinline__ int tc_off(int row, int k, int kr) {
  constexpr int KC = 16 / ES;
  return (row >> 3) * (kr / KC) * 128 + (k / KC) * 128 + (row & 7) * 16 + (k % KC) * ES;
}

// G operands packed into one 32-bit word (element k in the low bits).
template <int KIND>
__device__ __forceinline__ uint32_t tc_pack1(float x) { return tf32_rna(x); }
template <int KIND>
__device__ __forceinline__ uint32_t tc_pack2(float x0, float x1) { return pack_bf16(x0, x1); }

template <typename TIO>
__device__ __forceinline__ float tc_load(const TIO* p) {
  if constexpr (sizeof(TIO) == 4) return __ldg(reinterpret_cast<const float*>(p));
  else return __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(p));
}
template <typename TIO>
__device__ __forceinline__ void tc_store(TIO* p, float v, bool add) {
  if constexpr (sizeof(TIO) == 4) {
    float* q = reinterpret_cast<float*>(p);
    *q = add ? *q + v : v;
  } else {
    __nv_bfloat16* q = reinterpret_cast<__nv_bfloat16*>(p);
    *q = __float2bfloat16_rn(add ? __bfloat162float(*q) + v : v);
  }
}

struct TcArgs {
  const unsigned char* bimg;   // B operands of the six passes (device, core layout)
  int np, nq;
  int* status;                 // FE_ETIMEOUT is raised here when a bounded wait gives up
};

// Transposed write of one row of D (pass S) into the A layout of pass S + 1.
// The row's line group has slow coordinate `a` and lines f = G b + g; D
// column (g, qty, n) is quantity qty at output index n of line g.  SLOWN:
// the next pass's slow coordinate is n (F-x, B-z), else it stays a (F-y, B-y).
template <class SH, int NQT, bool SLOWN, int KRN>
__device__ __forceinline__ void tc_write_transposed(const float* d, int a, int b, int v, unsigned char* Mb) {
  constexpr int E = SH::E, G = SH::G, H = SH::H;
  constexpr int NL = NQT * E;   // D columns per line = K per line of the next pass
#pragma unroll
  for (int n = 0; n < E; ++n) {
    const int ap = SLOWN ? n : a, fp = SLOWN ? a : n;
    const int rowp = (ap * H + fp / G) * kTcVectors + v;
    const int gp = fp % G;
#pragma unroll
    for (int q = 0; q < NQT; ++q) {
      const int k = gp * NL + q * E + G * b;
      uint32_t w;
      if constexpr (G == 1) w = tc_pack1<SH::KIND>(d[q * E + n]);
      else w = tc_pack2<SH::KIND>(d[q * E + n], d[NL + q * E + n]);
      *reinterpret_cast<uint32_t*>(Mb + tc_off<SH::ES>(rowp, k, KRN)) = w;
    }
  }
}

// Row `row` of an operand with kr values per row, written whole from vals[0..kr).
template <class SH, int KR>
__device__ __forceinline__ void tc_write_row(const float* vals, int row, unsigned char* base) {
#pragma unroll
  for (int c = 0; c < KR; c += SH::KC) {
    uint4 w;
    if constexpr (SH::KIND == kTcTF32) {
      w.x = tf32_rna(vals[c]); w.y = tf32_rna(vals[c + 1]); w.z = tf32_rna(vals[c + 2]); w.w = tf32_rna(vals[c + 3]);
    } else {
      w.x = pack_bf16(vals[c], vals[c + 1]); w.y = pack_bf16(vals[c + 2], vals[c + 3]);
      w.z = pack_bf16(vals[c + 4], vals[c + 5]); w.w = pack_bf16(vals[c + 6], vals[c + 7]);
    }
    *reinterpret_cast<uint4*>(base + tc_off<SH::ES>(row, c, KR)) = w;
  }
}

// Issue pass S: all tiles, all K steps, one commit (thread 0 only).
template <class SH, int S>
__device__ __forceinline__ void tc_issue(uint32_t tmem, const unsigned char* A, const unsigned char* Bs,
                                         uint64_t* mbar) {
  constexpr int KR = SH::Kr(S), NR = SH::Nr(S);
  constexpr uint32_t sbo = (uint32_t)(KR / SH::KC) * 128;
  constexpr uint32_t idesc = SH::KIND == kTcTF32 ? umma_idesc_tf32(128, NR) : umma_idesc_bf16(128, NR);
  const uint32_t a0 = smem_u32(A), b0 = smem_u32(Bs + SH::b_off(S));
  tc_fence_after();
#pragma unroll
  for (int j = 0; j < SH::T; ++j)
#pragma unroll
    for (int ks = 0; ks < KR / SH::KI; ++ks) {
      const uint64_t ad = umma_desc(a0 + (uint32_t)j * 16 * sbo + ks * 256, 128, sbo);
      const uint64_t bd = umma_desc(b0 + ks * 256, 128, sbo);
      if constexpr (SH::KIND == kTcTF32) umma_tf32(tmem + j * NR, ad, bd, idesc, ks > 0);
      else umma_bf16(tmem + j * NR, ad, bd, idesc, ks > 0);
    }
  umma_commit(mbar);
}

// One persistent CTA per slot: loops over the (cell, 8-vector block) tasks of
// one colour.  128 threads: thread t owns TMEM lane t, i.e. row t of every
// 128-row tile of a pass.
template <int E, int G, int KIND, typename TIO, bool GEN>
__global__ void __launch_bounds__(128) tc_apply_kernel(const TcArgs args, const MeshDev m, const Geom<float> geo,
                                                       const int* __restrict__ cells, int n_tasks, int n_vec,
                                                       int n_vb, const TIO* __restrict__ X, TIO* __restrict__ Y) {
  using SH = TcShape<E, G, KIND>;
  constexpr int H = SH::H, T = SH::T;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* Bs = smem;
  unsigned char* Sb = smem + SH::B_BYTES;
  unsigned char* Mb = Sb + SH::S_BYTES;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(Mb + SH::M_BYTES);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int t = threadIdx.x, warp = t >> 5;
  const int np = args.np, nq = args.nq, P = np - 1;
  const int nq3 = nq * nq * nq;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(SH::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (t == 0) mbar_init(mbar, 1);
  {  // B operands -> shared; the A buffers start at zero (padding stays finite)
    const uint4* src = reinterpret_cast<const uint4*>(args.bimg);
    uint4* dst = reinterpret_cast<uint4*>(Bs);
    for (int k = t; k < SH::B_BYTES / 16; k += 128) dst[k] = __ldg(src + k);
    uint4* z = reinterpret_cast<uint4*>(Sb);
    for (int k = t; k < (SH::S_BYTES + SH::M_BYTES) / 16; k += 128) z[k] = make_uint4(0, 0, 0, 0);
  }
  fence_async_smem();
  asm volatile("fence.mbarrier_init.release.cluster;");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t tlane = tmem + ((uint32_t)(warp * 32) << 16);
  bool fail = false;

  for (int task = blockIdx.x; task < n_tasks && !fail; task += gridDim.x) {
    const int e = cells[task / n_vb];
    const int v0 = (task % n_vb) * kTcVectors;
    const int cx = e % m.nx, cy = (e / m.nx) % m.ny, cz = e / (m.nx * m.ny);

    // ---- gather: row (i3, b) x v, lines i2 = G b + g, K = [g][i1] ----
#pragma unroll
    for (int j = 0; j < T; ++j) {
      const int r = j * 128 + t, L = r >> 3, v = r & 7;
      if (L >= SH::LINES) continue;
      const int i3 = L / H, b = L % H;
      const bool vok = v0 + v < n_vec;
      float vals[SH::Kr(0)];
#pragma unroll
      for (int k = 0; k < SH::Kr(0); ++k) vals[k] = 0.f;
      const int gz = node_coord(cz, i3, P, m.Nz, m.periodic);
      const bool con_z = i3 >= np || on_boundary(gz, m.Nz, m.periodic);
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int i2 = G * b + g;
        const int gy = node_coord(cy, i2, P, m.Ny, m.periodic);
        if (!vok || con_z || i2 >= np || on_boundary(gy, m.Ny, m.periodic)) continue;
        const size_t rowoff = (size_t)(gy + (size_t)m.Ny * gz) * m.Nx;
#pragma unroll
        for (int i1 = 0; i1 < E; ++i1) {
          if (i1 >= np) continue;
          const int gx = node_coord(cx, i1, P, m.Nx, m.periodic);
          if (on_boundary(gx, m.Nx, m.periodic)) continue;
          vals[g * E + i1] = tc_load(X + (rowoff + gx) * n_vec + v0 + v);
        }
      }
      tc_write_row<SH, SH::Kr(0)>(vals, r, Sb);
    }

    // ---- the six passes ----
    // pass index s = 0..5, mbarrier phase = s & 1 (six completions per task)
    // Every thread's writes of the A operand become visible to the tensor
    // cores, thread 0 issues the pass, everyone waits for its completion
    // (bounded; a timeout anywhere ends the loop for the whole CTA).  The
    // pass reads A from shared memory and writes D to tensor memory only, so
    // the next A may overwrite this one as soon as the pass is complete.
#define FE_TC_ISSUE(S, ABUF)                                                   \
  fence_async_smem();                                                          \
  tc_fence_before();                                                           \
  __syncthreads();                                                             \
  if (t == 0) tc_issue<SH, S>(tmem, ABUF, Bs, mbar);                           \
  if (__syncthreads_or(!mbar_wait(mbar, (S) & 1))) { fail = true; break; }      \
  tc_fence_after();

    FE_TC_ISSUE(0, Sb)
#pragma unroll
    for (int j = 0; j < T; ++j) {   // F-x: row (i3, b), lines i2 -> A of F-y: (q1, i3 / G)
      float d[SH::Nr(0)];
      tmem_load<SH::Nr(0)>(tlane + j * SH::Nr(0), d);
      const int r = j * 128 + t, L = r >> 3;
      if (L < SH::LINES) tc_write_transposed<SH, 2, true, SH::Kr(1)>(d, L / H, L % H, r & 7, Mb);
    }
    FE_TC_ISSUE(1, Mb)
#pragma unroll
    for (int j = 0; j < T; ++j) {   // F-y: row (q1, b), lines i3 -> A of F-z: (q1, q2 / G)
      float d[SH::Nr(1)];
      tmem_load<SH::Nr(1)>(tlane + j * SH::Nr(1), d);
      const int r = j * 128 + t, L = r >> 3;
      if (L < SH::LINES) tc_write_transposed<SH, 3, false, SH::Kr(2)>(d, L / H, L % H, r & 7, Mb);
    }
    FE_TC_ISSUE(2, Mb)
#pragma unroll
    for (int j = 0; j < T; ++j) {   // F-z and the quadrature-point operation: row (q1, b), lines q2 = G b + g
      float d[SH::Nr(2)];
      tmem_load<SH::Nr(2)>(tlane + j * SH::Nr(2), d);
      const int r = j * 128 + t, L = r >> 3;
      if (L >= SH::LINES) continue;
      const int q1 = L / H, b = L % H;
      float g00 = 0.f, g01 = 0.f, g02 = 0.f, g11 = 0.f, g12 = 0.f, g22 = 0.f;
      if (!GEN) {
        const float* cg = geo.cellG + (size_t)e * 6;
        g00 = __ldg(cg); g01 = __ldg(cg + 1); g02 = __ldg(cg + 2);
        g11 = __ldg(cg + 3); g12 = __ldg(cg + 4); g22 = __ldg(cg + 5);
      }
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int q2 = G * b + g;
        float* dl = d + g * 4 * E;   // [val | dz | dy | dx] along q3, becomes [hv | hz | hy | hx]
#pragma unroll
        for (int q3 = 0; q3 < E; ++q3) {
          float hv = 0.f, hx = 0.f, hy = 0.f, hz = 0.f;
          if (q1 < nq && q2 < nq && q3 < nq) {
            const int Q = q1 + nq * (q2 + nq * q3);
            if (GEN) {
              const float* pg = geo.ptG + (size_t)e * 6 * nq3 + Q;
              g00 = __ldg(pg); g01 = __ldg(pg + nq3); g02 = __ldg(pg + 2 * nq3);
              g11 = __ldg(pg + 3 * nq3); g12 = __ldg(pg + 4 * nq3); g22 = __ldg(pg + 5 * nq3);
            }
            const float dz = dl[E + q3], dy = dl[2 * E + q3], dx = dl[3 * E + q3];
            hx = g00 * dx + g01 * dy + g02 * dz;
            hy = g01 * dx + g11 * dy + g12 * dz;
            hz = g02 * dx + g12 * dy + g22 * dz;
            hv = __ldg(geo.ptC + (size_t)e * nq3 + Q) * dl[q3];
          }
          dl[q3] = hv;
          dl[E + q3] = hz;
          dl[2 * E + q3] = hy;
          dl[3 * E + q3] = hx;
        }
      }
      tc_write_row<SH, SH::Kr(3)>(d, r, Mb);
    }
    FE_TC_ISSUE(3, Mb)
#pragma unroll
    for (int j = 0; j < T; ++j) {   // B-z: row (q1, b), lines q2 -> A of B-y: (i3, q1 / G)
      float d[SH::Nr(3)];
      tmem_load<SH::Nr(3)>(tlane + j * SH::Nr(3), d);
      const int r = j * 128 + t, L = r >> 3;
      if (L < SH::LINES) tc_write_transposed<SH, 3, true, SH::Kr(4)>(d, L / H, L % H, r & 7, Mb);
    }
    FE_TC_ISSUE(4, Mb)
#pragma unroll
    for (int j = 0; j < T; ++j) {   // B-y: row (i3, b), lines q1 -> A of B-x: (i3, i2 / G)
      float d[SH::Nr(4)];
      tmem_load<SH::Nr(4)>(tlane + j * SH::Nr(4), d);
      const int r = j * 128 + t, L = r >> 3;
      if (L < SH::LINES) tc_write_transposed<SH, 2, false, SH::Kr(5)>(d, L / H, L % H, r & 7, Mb);
    }
    FE_TC_ISSUE(5, Mb)
#pragma unroll
    for (int j = 0; j < T; ++j) {   // B-x and assembly: row (i3, b), lines i2 = G b + g, D = [g][i1]
      float d[SH::Nr(5)];
      tmem_load<SH::Nr(5)>(tlane + j * SH::Nr(5), d);
      const int r = j * 128 + t, L = r >> 3, v = r & 7;
      if (L >= SH::LINES || v0 + v >= n_vec) continue;
      const int i3 = L / H, b = L % H;
      if (i3 >= np) continue;
      const int gz = node_coord(cz, i3, P, m.Nz, m.periodic);
      const bool con_z = on_boundary(gz, m.Nz, m.periodic);
      const bool first_z = first_along(cz, m.nz, i3, P, m.periodic, m.last_odd_z);
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int i2 = G * b + g;
        if (i2 >= np) continue;
        const int gy = node_coord(cy, i2, P, m.Ny, m.periodic);
        const bool con_yz = con_z || on_boundary(gy, m.Ny, m.periodic);
        const bool first_yz = first_z && first_along(cy, m.ny, i2, P, m.periodic, m.last_odd_y);
        const size_t rowoff = (size_t)(gy + (size_t)m.Ny * gz) * m.Nx;
#pragma unroll
        for (int i1 = 0; i1 < E; ++i1) {
          if (i1 >= np) continue;
          const int gx = node_coord(cx, i1, P, m.Nx, m.periodic);
          const bool con = con_yz || on_boundary(gx, m.Nx, m.periodic);
          const bool first = first_yz && first_along(cx, m.nx, i1, P, m.periodic, m.last_odd_x);
          TIO* dst = Y + (rowoff + gx) * n_vec + v0 + v;
          if (first) tc_store(dst, con ? 0.f : d[g * E + i1], false);
          else if (!con) tc_store(dst, d[g * E + i1], true);
        }
      }
    }
#undef FE_TC_ISSUE
  }

  if (fail && t == 0) {
    atomicMax(args.status, (int)FE_ETIMEOUT);
    // let any MMA still in flight finish before the tensor memory is released
    mbar_wait(mbar, 0, 1 << 20);
    mbar_wait(mbar, 1, 1 << 20);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(SH::TMEM_COLS));
}

}  // namespace fe
