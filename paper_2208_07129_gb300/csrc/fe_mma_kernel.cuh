// Tensor-core cell kernel: the 1D contractions of Algorithm 2 as warp-level
// MMAs (TF32 m16n8k8 or BF16 m16n8k16, FP32 accumulation), FP32 data.
//
// One CTA = one cell x 16 vectors.  Every 1D contraction of a line is a small
// dense GEMM  out[v][n] = sum_k in[v][k] M(k, n)  with the 16 vectors as the
// MMA's M dimension, the line's n_p or n_q entries as K and the outputs as N
// (Sec. 3.2.4: the contractions recast as batched matrix products over the
// vector block).  The 1D matrix fragments (N, D~, and their transposes) stay
// in registers for a whole pass; line operands go through shared memory
// tiles [element][16 vectors].  Order of the passes as in Algorithm 2; the
// quadrature-point operation is applied to the accumulator fragments of the
// z-gradient pass, whose transposed z pass takes c T as its accumulator input.
// Operands are rounded to TF32 (cvt.rna) or BF16 (round to nearest even);
// every sum is accumulated in FP32.  The split-TF32 kind (3xTF32) writes
// every operand as hi + lo, both TF32, and accumulates lo*hi + hi*lo + hi*hi:
// three MMAs per product, with only the lo*lo term (relative size 2^-22)
// dropped, which gives FP32-level accuracy on the tensor cores (the
// error-free splitting of Ootomo and Yokota, 2022).  Assembly: colour-ordered,
// first writer stores, as in the CUDA-core kernels.
#pragma once

#include <cuda_bf16.h>

#include "fe_cell_kernel.cuh"

namespace fe {

constexpr int kMmaVB = 16;   // vectors per CTA (the MMA's M)
constexpr int kMmaWarps = 8;

// Operand kinds of the tensor-core kernel.
constexpr int kTF32 = 0, kBF16 = 1, kTF32x3 = 2;

// x rounded to the nearest TF32 value (10 explicit mantissa bits; ties away
// from zero), as an FP32 bit pattern with the 13 low bits clear.  Used for the
// hi/lo split, where both parts must be exact TF32 values.
__device__ __forceinline__ uint32_t tf32_round_bits(float x) {
  return (__float_as_uint(x) + 0x1000u) & 0xffffe000u;
}

// x = hi + lo + O(2^-22 |x|), hi and lo both TF32.
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_round_bits(x);
  lo = tf32_round_bits(x - __uint_as_float(hi));
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// A 3D tile [e2][e1][e0] x 16 vectors in shared memory.  With an even e0 <= 8
// (measured: at e0 = 10 the extra index arithmetic costs more than the
// conflicts it removes) the tile is swizzled so that the four entries k of an MMA operand fragment,
// which lie on one line along x, y or z, fall into four different bank groups:
// element slot = elem ^ ((y + z) & 1) (this swaps x and x ^ 1 inside a row, so
// the slot's parity is (x + y + z) & 1 and selects the 16-word half of a
// 32-bank row) and the vector index is XORed with 8 ((x/2 + y/2 + z/2) & 1)
// (the 8-word half inside it).  Four consecutive positions along any axis have
// distinct (c & 1, (c >> 1) & 1), hence distinct bank groups.
struct Tile {
  float* p;
  int e0, e1, e2;
  __device__ __forceinline__ float& at(int x, int y, int z, int v) const {
    int elem = (z * e1 + y) * e0 + x;
    if (!(e0 & 1) && e0 <= 8) {
      elem ^= (y + z) & 1;
      v ^= (((x >> 1) + (y >> 1) + (z >> 1)) & 1) << 3;
    }
    return p[elem * 16 + v];
  }
};

// Coordinates of entry k of line `line` along axis `ax` of a tile with extents (e0, e1, e2).
__device__ __forceinline__ void line_coord(int ax, int line, int k, int e0, int e1, int* x, int* y, int* z) {
  if (ax == 0) { *x = k; *y = line % e1; *z = line / e1; }
  else if (ax == 1) { *x = line % e0; *y = k; *z = line / e0; }
  else { *x = line % e0; *y = line / e0; *z = k; }
}

// Matrix fragments of one pass: M(k, n) for k < KIN, n < NOUT, as B operands
// of the MMA (col layout), for every (k-step, n-tile).
template <int KIND, int KIN, int NOUT>
struct BFrags {
  static constexpr bool BF16 = KIND == kBF16;
  static constexpr int KS = BF16 ? (KIN + 15) / 16 : (KIN + 7) / 8;   // k-steps
  static constexpr int NT = (NOUT + 7) / 8;                           // n-tiles
  static constexpr int KSL = KIND == kTF32x3 ? KS : 1;                // lo parts (split kind only)
  static constexpr int NTL = KIND == kTF32x3 ? NT : 1;
  uint32_t b[KS][NT][2];
  uint32_t bl[KSL][NTL][2];
};

// M(k, n) = tab[n][k] (forward: rows of N or D~ are outputs) or tab[k][n] (transposed).
template <int KIND, int KIN, int NOUT, int R, int C>
__device__ __forceinline__ void load_bfrags(BFrags<KIND, KIN, NOUT>& f, const float (&tab)[R][C], bool trans) {
  constexpr bool BF16 = KIND == kBF16;
  const int lane = threadIdx.x & 31, g = lane >> 2, t4 = lane & 3;
  auto M = [&](int k, int n) -> float {
    if (k >= KIN || n >= NOUT) return 0.f;
    return trans ? tab[k][n] : tab[n][k];
  };
#pragma unroll
  for (int ks = 0; ks < BFrags<KIND, KIN, NOUT>::KS; ++ks)
#pragma unroll
    for (int nt = 0; nt < BFrags<KIND, KIN, NOUT>::NT; ++nt) {
      const int n = nt * 8 + g;
      if (BF16) {
        const int k0 = ks * 16 + 2 * t4;
        f.b[ks][nt][0] = pack_bf16x2(M(k0, n), M(k0 + 1, n));
        f.b[ks][nt][1] = pack_bf16x2(M(k0 + 8, n), M(k0 + 9, n));
      } else if (KIND == kTF32x3) {
        const int k0 = ks * 8 + t4;
        split_tf32(M(k0, n), f.b[ks][nt][0], f.bl[ks % f.KSL][nt % f.NTL][0]);
        split_tf32(M(k0 + 4, n), f.b[ks][nt][1], f.bl[ks % f.KSL][nt % f.NTL][1]);
      } else {
        const int k0 = ks * 8 + t4;
        f.b[ks][nt][0] = to_tf32(M(k0, n));
        f.b[ks][nt][1] = to_tf32(M(k0 + 4, n));
      }
    }
}

// Accumulator fragment of one line: d[nt][r], element (v, n) with
// v = g + 8 (r >> 1), n = nt * 8 + 2 t4 + (r & 1).
template <int NT>
struct DFrag {
  float d[NT][4];
};

// A-operand loader: a(v, k) for the 16 vectors.  `get(v, k)` returns the FP32 value.
template <int KIND, int KIN, int NOUT, typename Get>
__device__ __forceinline__ void line_mma(const BFrags<KIND, KIN, NOUT>& f, DFrag<BFrags<KIND, KIN, NOUT>::NT>& acc,
                                         Get get) {
  constexpr bool BF16 = KIND == kBF16;
  const int lane = threadIdx.x & 31, g = lane >> 2, t4 = lane & 3;
  constexpr int KS = BFrags<KIND, KIN, NOUT>::KS, NT = BFrags<KIND, KIN, NOUT>::NT;
#pragma unroll
  for (int ks = 0; ks < KS; ++ks) {
    uint32_t a[4];
    if (KIND == kTF32x3) {
      const int k0 = ks * 8 + t4;
      auto v = [&](int vv, int k) { return k < KIN ? get(vv, k) : 0.f; };
      uint32_t al[4];
      split_tf32(v(g, k0), a[0], al[0]);
      split_tf32(v(g + 8, k0), a[1], al[1]);
      split_tf32(v(g, k0 + 4), a[2], al[2]);
      split_tf32(v(g + 8, k0 + 4), a[3], al[3]);
      // small terms first
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        mma_tf32(acc.d[nt], al, f.b[ks][nt]);
        mma_tf32(acc.d[nt], a, f.bl[ks % f.KSL][nt % f.NTL]);
        mma_tf32(acc.d[nt], a, f.b[ks][nt]);
      }
      continue;
    }
    if (BF16) {
      const int k0 = ks * 16 + 2 * t4;
      auto v = [&](int vv, int k) { return k < KIN ? get(vv, k) : 0.f; };
      a[0] = pack_bf16x2(v(g, k0), v(g, k0 + 1));
      a[1] = pack_bf16x2(v(g + 8, k0), v(g + 8, k0 + 1));
      a[2] = pack_bf16x2(v(g, k0 + 8), v(g, k0 + 9));
      a[3] = pack_bf16x2(v(g + 8, k0 + 8), v(g + 8, k0 + 9));
    } else {
      const int k0 = ks * 8 + t4;
      auto v = [&](int vv, int k) { return k < KIN ? get(vv, k) : 0.f; };
      a[0] = to_tf32(v(g, k0));
      a[1] = to_tf32(v(g + 8, k0));
      a[2] = to_tf32(v(g, k0 + 4));
      a[3] = to_tf32(v(g + 8, k0 + 4));
    }
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      if (BF16) mma_bf16(acc.d[nt], a, f.b[ks][nt]);
      else mma_tf32(acc.d[nt], a, f.b[ks][nt]);
    }
  }
}

// Visit every accumulator element (v, n < NOUT) of a line fragment.
template <int NT, int NOUT, typename F>
__device__ __forceinline__ void for_frag(DFrag<NT>& acc, F fn) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t4 = lane & 3;
#pragma unroll
  for (int nt = 0; nt < NT; ++nt)
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int n = nt * 8 + 2 * t4 + (r & 1);
      if (n < NOUT) fn(g + 8 * (r >> 1), n, acc.d[nt][r]);
    }
}

// One pass over all lines along axis `ax`: dst(line, n) (+)= sum_k src(line, k) M(k, n).
template <int KIND, int KIN, int NOUT, bool ACC>
__device__ __forceinline__ void pass(const BFrags<KIND, KIN, NOUT>& f, const Tile& src, const Tile& dst, int ax,
                                     int n_lines) {
  constexpr int NT = BFrags<KIND, KIN, NOUT>::NT;
  const int warp = threadIdx.x >> 5;
  for (int line = warp; line < n_lines; line += kMmaWarps) {
    DFrag<NT> acc;
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) acc.d[nt][0] = acc.d[nt][1] = acc.d[nt][2] = acc.d[nt][3] = 0.f;
    if (ACC) {
      for_frag<NT, NOUT>(acc, [&](int v, int n, float& x) {
        int a, b, c;
        line_coord(ax, line, n, dst.e0, dst.e1, &a, &b, &c);
        x = dst.at(a, b, c, v);
      });
    }
    line_mma<KIND, KIN, NOUT>(f, acc, [&](int v, int k) {
      int a, b, c;
      line_coord(ax, line, k, src.e0, src.e1, &a, &b, &c);
      return src.at(a, b, c, v);
    });
    for_frag<NT, NOUT>(acc, [&](int v, int n, float& x) {
      int a, b, c;
      line_coord(ax, line, n, dst.e0, dst.e1, &a, &b, &c);
      dst.at(a, b, c, v) = x;
    });
  }
}

template <int NP, int NQ, bool GEN, int KIND>
__global__ void __launch_bounds__(32 * kMmaWarps) mma_apply_kernel(const Tables<float, NP, NQ> tab, const MeshDev m,
                                                                   const Geom<float> geo,
                                                                   const int* __restrict__ cells, int n_vec, int n_vb,
                                                                   const float* __restrict__ X,
                                                                   float* __restrict__ Y) {
  constexpr int P = NP - 1;
  constexpr int NQ3 = NQ * NQ * NQ;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* base = reinterpret_cast<float*>(smem_raw);
  const int warp = threadIdx.x >> 5;
  const int vb = blockIdx.x % n_vb;
  const int e = cells[blockIdx.x / n_vb];
  const int v0 = vb * kMmaVB;
  const int cx = e % m.nx, cy = (e / m.nx) % m.ny, cz = e / (m.nx * m.ny);
  const Tile ST{base, NQ, NQ, NQ}, S0q{base + NQ3 * 16, NQ, NQ, NQ}, S1q{base + 2 * NQ3 * 16, NQ, NQ, NQ};

  // ---- extraction fused with the x pass of N: S0[i3][i2][q1] ----
  {
    BFrags<KIND, NP, NQ> f;
    load_bfrags(f, tab.N, false);
    const Tile dst{S0q.p, NQ, NP, NP};
    constexpr int NT = BFrags<KIND, NP, NQ>::NT;
    for (int line = warp; line < NP * NP; line += kMmaWarps) {
      const int i2 = line % NP, i3 = line / NP;
      const int gy = node_coord(cy, i2, P, m.Ny, m.periodic), gz = node_coord(cz, i3, P, m.Nz, m.periodic);
      const bool con_yz = on_boundary(gy, m.Ny, m.periodic) || on_boundary(gz, m.Nz, m.periodic);
      const size_t row = (size_t)(gy + (size_t)m.Ny * gz) * m.Nx;
      DFrag<NT> acc;
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) acc.d[nt][0] = acc.d[nt][1] = acc.d[nt][2] = acc.d[nt][3] = 0.f;
      line_mma<KIND, NP, NQ>(f, acc, [&](int v, int k) {
        const int gx = node_coord(cx, k, P, m.Nx, m.periodic);
        const bool con = con_yz || on_boundary(gx, m.Nx, m.periodic);
        return (v0 + v < n_vec && !con) ? __ldg(X + (row + gx) * n_vec + v0 + v) : 0.f;
      });
      for_frag<NT, NQ>(acc, [&](int v, int n, float& x) { dst.at(n, i2, i3, v) = x; });
    }
  }
  __syncthreads();
  {  // y pass of N: S1[i3][q2][q1]
    BFrags<KIND, NP, NQ> f;
    load_bfrags(f, tab.N, false);
    pass<KIND, NP, NQ, false>(f, Tile{S0q.p, NQ, NP, NP}, Tile{S1q.p, NQ, NQ, NP}, 1, NQ * NP);
  }
  __syncthreads();
  {  // z pass of N: T[q3][q2][q1]
    BFrags<KIND, NP, NQ> f;
    load_bfrags(f, tab.N, false);
    pass<KIND, NP, NQ, false>(f, Tile{S1q.p, NQ, NQ, NP}, ST, 2, NQ * NQ);
  }
  __syncthreads();
  {  // gradients along x (-> S0) and y (-> S1)
    BFrags<KIND, NQ, NQ> f;
    load_bfrags(f, tab.D, false);
    pass<KIND, NQ, NQ, false>(f, ST, S0q, 0, NQ * NQ);
    pass<KIND, NQ, NQ, false>(f, ST, S1q, 1, NQ * NQ);
  }
  __syncthreads();
  {  // z-lines: gradient along z, quadrature-point operation, transposed z pass with c T as accumulator
    BFrags<KIND, NQ, NQ> fd, fdt;
    load_bfrags(fd, tab.D, false);
    load_bfrags(fdt, tab.D, true);
    constexpr int NT = BFrags<KIND, NQ, NQ>::NT;
    float g00, g01, g02, g11, g12, g22;
    if (!GEN) {
      g00 = geo.cellG[e * 6 + 0]; g01 = geo.cellG[e * 6 + 1]; g02 = geo.cellG[e * 6 + 2];
      g11 = geo.cellG[e * 6 + 3]; g12 = geo.cellG[e * 6 + 4]; g22 = geo.cellG[e * 6 + 5];
    }
    const float* ptC = geo.ptC + (size_t)e * NQ3;
    for (int line = warp; line < NQ * NQ; line += kMmaWarps) {
      const int q1 = line % NQ, q2 = line / NQ;
      DFrag<NT> t2, ct;
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) t2.d[nt][0] = t2.d[nt][1] = t2.d[nt][2] = t2.d[nt][3] = 0.f;
      line_mma<KIND, NQ, NQ>(fd, t2, [&](int v, int k) { return ST.at(q1, q2, k, v); });
      // point operation on the fragment elements (each (v, q3) owned by one thread)
#pragma unroll
      for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int lane = threadIdx.x & 31;
          const int v = (lane >> 2) + 8 * (r >> 1), q3 = nt * 8 + 2 * (lane & 3) + (r & 1);
          ct.d[nt][r] = 0.f;
          if (q3 < NQ) {
            const int Q = (q3 * NQ + q2) * NQ + q1;
            if (GEN) {
              const float* pg = geo.ptG + (size_t)e * 6 * NQ3 + Q;
              g00 = pg[0]; g01 = pg[NQ3]; g02 = pg[2 * NQ3]; g11 = pg[3 * NQ3]; g12 = pg[4 * NQ3]; g22 = pg[5 * NQ3];
            }
            const float d0 = S0q.at(q1, q2, q3, v), d1 = S1q.at(q1, q2, q3, v), d2 = t2.d[nt][r];
            S0q.at(q1, q2, q3, v) = g00 * d0 + g01 * d1 + g02 * d2;
            S1q.at(q1, q2, q3, v) = g01 * d0 + g11 * d1 + g12 * d2;
            t2.d[nt][r] = g02 * d0 + g12 * d1 + g22 * d2;
            ct.d[nt][r] = ptC[Q] * ST.at(q1, q2, q3, v);
          }
        }
      __syncwarp();
      // the z-line of T is no longer needed: park h2 there, reload it as the A operand
      for_frag<NT, NQ>(t2, [&](int v, int n, float& x) { ST.at(q1, q2, n, v) = x; });
      __syncwarp();
      line_mma<KIND, NQ, NQ>(fdt, ct, [&](int v, int k) { return ST.at(q1, q2, k, v); });
      __syncwarp();
      for_frag<NT, NQ>(ct, [&](int v, int n, float& x) { ST.at(q1, q2, n, v) = x; });
    }
  }
  __syncthreads();
  {  // transposed x pass of D~, then transposed y pass, accumulated into T
    BFrags<KIND, NQ, NQ> f;
    load_bfrags(f, tab.D, true);
    pass<KIND, NQ, NQ, true>(f, S0q, ST, 0, NQ * NQ);
    __syncthreads();
    pass<KIND, NQ, NQ, true>(f, S1q, ST, 1, NQ * NQ);
  }
  __syncthreads();
  {  // transposed z pass of N: S1[i3][q2][q1]
    BFrags<KIND, NQ, NP> f;
    load_bfrags(f, tab.N, true);
    pass<KIND, NQ, NP, false>(f, ST, Tile{S1q.p, NQ, NQ, NP}, 2, NQ * NQ);
  }
  __syncthreads();
  {  // transposed y pass of N: S0[i3][i2][q1]
    BFrags<KIND, NQ, NP> f;
    load_bfrags(f, tab.N, true);
    pass<KIND, NQ, NP, false>(f, Tile{S1q.p, NQ, NQ, NP}, Tile{S0q.p, NQ, NP, NP}, 1, NQ * NP);
  }
  __syncthreads();
  {  // transposed x pass of N fused with assembly
    BFrags<KIND, NQ, NP> f;
    load_bfrags(f, tab.N, true);
    const Tile src{S0q.p, NQ, NP, NP};
    constexpr int NT = BFrags<KIND, NQ, NP>::NT;
    for (int line = warp; line < NP * NP; line += kMmaWarps) {
      const int i2 = line % NP, i3 = line / NP;
      DFrag<NT> acc;
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) acc.d[nt][0] = acc.d[nt][1] = acc.d[nt][2] = acc.d[nt][3] = 0.f;
      line_mma<KIND, NQ, NP>(f, acc, [&](int v, int k) { return src.at(k, i2, i3, v); });
      const int gy = node_coord(cy, i2, P, m.Ny, m.periodic), gz = node_coord(cz, i3, P, m.Nz, m.periodic);
      const bool con_yz = on_boundary(gy, m.Ny, m.periodic) || on_boundary(gz, m.Nz, m.periodic);
      const bool first_yz = first_along(cy, m.ny, i2, P, m.periodic, m.last_odd_y) &&
                            first_along(cz, m.nz, i3, P, m.periodic, m.last_odd_z);
      const size_t row = (size_t)(gy + (size_t)m.Ny * gz) * m.Nx;
      for_frag<NT, NP>(acc, [&](int v, int i1, float& x) {
        if (v0 + v >= n_vec) return;
        const int gx = node_coord(cx, i1, P, m.Nx, m.periodic);
        const bool con = con_yz || on_boundary(gx, m.Nx, m.periodic);
        const bool first = first_yz && first_along(cx, m.nx, i1, P, m.periodic, m.last_odd_x);
        float* dst = Y + (row + gx) * n_vec + v0 + v;
        if (first) *dst = con ? 0.f : x;
        else if (!con) *dst += x;
      });
    }
  }
}

template <int NP, int NQ, bool GEN, int KIND>
cudaError_t launch_mma(const fe_ctx* c, const float* X, float* Y, int n_vec, cudaStream_t s) {
  auto kern = mma_apply_kernel<NP, NQ, GEN, KIND>;
  const size_t smem = (size_t)3 * NQ * NQ * NQ * kMmaVB * sizeof(float);
  if (smem > 220 * 1024) return cudaErrorInvalidValue;
  {
    cudaError_t e = ensure_dyn_smem(reinterpret_cast<const void*>(kern), smem);
    if (e != cudaSuccess) return e;
  }
  const Tables<float, NP, NQ> tab = make_tables<float, NP, NQ>(c);
  const Geom<float> geo = make_geom<float>(c);
  const int n_vb = (n_vec + kMmaVB - 1) / kMmaVB;
  for (int k = 0; k < c->colors.n_colors; ++k) {
    const int n = c->colors.offset[k + 1] - c->colors.offset[k];
    if (n == 0) continue;
    const long long blocks = (long long)n * n_vb;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    kern<<<(unsigned)blocks, 32 * kMmaWarps, smem, s>>>(tab, c->mdev, geo, c->d_cells + c->colors.offset[k], n_vec,
                                                         n_vb, X, Y);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace fe
