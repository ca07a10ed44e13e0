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
//        (box meshes: every cell has the same G, which is folded into the
//        B operand of B-z, so only hv = c val is formed per point)
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
// Operands: TF32 (kind::tf32) or BF16 (kind::f16), G = 2, both rounded
// to nearest from FP32; the quadrature-point operation is FP32.  Storage of X
// and Y: FP32 or BF16.  Data movement: TMA boxes of 8 vectors x n_p^3 nodes
// in and bulk reduce-adds out where the block layout allows, else per-thread
// loads and stores.  Assembly: colour-ordered either way (see the kernel).
#pragma once

#include <cuda_bf16.h>

#include "fe_cell_kernel.cuh"
#include "fe_tma.cuh"
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
  static_assert(E % G == 0 && (G * ES == 4 || G * ES == 8), "a packed store holds the G operands of a word");
  static_assert(16 % H == 0, "a thread's line-group index b is the same in every tile");
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
  static constexpr int SLOT_COLS = d_cols_max() <= 32 ? 32 : d_cols_max() <= 64 ? 64 : d_cols_max() <= 128 ? 128
                                   : d_cols_max() <= 256 ? 256 : 512;
  // Task slots per CTA (one warpgroup each, own tensor-memory columns and A
  // buffers, one shared copy of the B operands): as many as 227 KB of shared
  // memory and the 512 tensor-memory columns allow, at most 4.
  static constexpr int SLOT_BYTES = S_BYTES + M_BYTES;
  static constexpr int SLOTS_SMEM = (227 * 1024 - B_BYTES - 256) / SLOT_BYTES;
  static constexpr int SLOTS = SLOTS_SMEM < 512 / SLOT_COLS ? (SLOTS_SMEM < 4 ? SLOTS_SMEM : 4)
                                                            : (512 / SLOT_COLS < 4 ? 512 / SLOT_COLS : 4);
  static constexpr int TMEM_COLS = SLOTS * SLOT_COLS <= 128 ? 128 : SLOTS * SLOT_COLS <= 256 ? 256 : 512;
  static constexpr int SMEM_BYTES = B_BYTES + SLOTS * SLOT_BYTES + 128;
  static_assert(SLOTS >= 1, "one task slot must fit");
};

// Byte offset of element (row, k) of a K-major operand whose rows hold kr values.
template <int ES>
__host__ __device__ __forceinline__ int tc_off(int row, int k, int kr) {
  constexpr int KC = 16 / ES;
  return (row >> 3) * (kr / KC) * 128 + (k / KC) * 128 + (row & 7) * 16 + (k % KC) * ES;
}

// Line group held by row group R of the F-x and B-x operands.  With four
// line groups per slow index (H = 4) the groups b = 2, 3 of slow indices
// 2k and 2k + 1 trade places: the 32 rows of a warp then hold (a, 0), (a, 1),
// (a ^ 1, 2), (a ^ 1, 3), whose node rows in a cell box start in four
// different bank groups (a box read or write of one element per row meets
// no bank conflict), while the packed operand stores of those rows still
// fill distinct words of one 128-byte core matrix.  The map is its own
// inverse.
template <class SH>
__host__ __device__ __forceinline__ constexpr int tc_lg(int R) {
  return SH::H == 4 ? (R ^ ((R & 2) ? 4 : 0)) : R;
}

// G operands packed into one 32-bit word (element k in the low bits).
template <int KIND>
__device__ __forceinline__ uint32_t tc_pack1(float x) { return tf32_rna(x); }
template <int KIND>
__device__ __forceinline__ uint32_t tc_pack2(float x0, float x1) { return pack_bf16(x0, x1); }

template <typename TIO>
__device__ __forceinline__ float tc_load(const TIO* p) {
  if constexpr (sizeof(TIO) == 4) return *reinterpret_cast<const float*>(p);
  else return __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(p));
}
template <typename TIO>
__device__ __forceinline__ void tc_store(TIO* p, float v) {
  if constexpr (sizeof(TIO) == 4) *reinterpret_cast<float*>(p) = v;
  else *reinterpret_cast<__nv_bfloat16*>(p) = __float2bfloat16_rn(v);
}

struct TcArgs {
  const unsigned char* bimg;   // B operands of the six passes (device, core layout)
  const unsigned long long* cmask;   // per cell of the launch: node masks (see tc_cell_masks)
  int np, nq;
  int* status;                 // FE_ETIMEOUT is raised here when a bounded wait gives up
  int* queue;                  // TMA kernels: task counter of the launch (zero at launch)
  const float* cvs;            // n_q = 8: c values per cell in the staged layout (tc_cv_index)
};

// Word of c at point (q1, q2, q3) in a cell's staged block (n_q = 8): plane
// q3 at a pitch of 72 floats, rows q2 >= 4 shifted by 4, so that the four
// line groups of a warp (q2 = 2b + g) read four different banks.
__host__ __device__ __forceinline__ constexpr int tc_cv_index(int q1, int q2, int q3) {
  return 72 * q3 + 8 * q2 + (q2 >= 4 ? 4 : 0) + q1;
}
constexpr int kTcCvBytes = 8 * 72 * 4;

// Transposed write of one row of D (pass S) into the A layout of pass S + 1.
// The row's line group has slow coordinate `a` and lines f = G b + g; D
// column (g, qty, n) is quantity qty at output index n of line g.  SLOWN:
// the next pass's slow coordinate is n (F-x, B-z), else it stays a (F-y, B-y).
// Every quantity block starts on a core-matrix boundary (E a multiple of
// KC), so the address of word (n, qty) is a per-thread base plus a
// compile-time offset: one packed store per word.
template <class SH, int NQT, bool SLOWN, int KRN, bool PERM = false>
__device__ __forceinline__ void tc_write_transposed(const float* d, int a, int b, int v, unsigned char* Mb) {
  constexpr int E = SH::E, G = SH::G, H = SH::H, KC = SH::KC, ES = SH::ES;
  constexpr int NL = NQT * E;              // D columns per line = K per line of the next pass
  constexpr int RB = (KRN / KC) * 128;     // bytes per group of 8 rows of the next pass's A
  static_assert(E % KC == 0 && NL % KC == 0, "quantity blocks must start on core-matrix boundaries");
  const int kb = G * b;                    // k of the first line of the group inside its quantity block
  int base = (kb / KC) * 128 + v * 16 + (kb % KC) * ES;
  if (SLOWN) base += (a / G) * RB + ((a % G) * NL / KC) * 128;
  else base += a * H * RB;
  unsigned char* p = Mb + base;
  // PERM (rows of the next pass placed by tc_lg): row group a H + n / G goes
  // to the row group of slow index a ^ 1 when (n / G) & 2
  const int alt = (a & 1) ? -H * RB : H * RB;
#pragma unroll
  for (int n = 0; n < E; ++n) {
#pragma unroll
    for (int q = 0; q < NQT; ++q) {
      const int off = SLOWN ? n * H * RB + q * (E / KC) * 128
                            : (n / G) * RB + ((n % G) * NL / KC) * 128 + q * (E / KC) * 128 +
                                  ((PERM && SH::H == 4 && ((n / G) & 2)) ? alt : 0);
      if constexpr (G * ES == 8) {   // two TF32 operands: one 8-byte store
        *reinterpret_cast<uint2*>(p + off) = make_uint2(tf32_rna(d[q * E + n]), tf32_rna(d[NL + q * E + n]));
      } else {
        uint32_t w;
        if constexpr (G == 1) w = tc_pack1<SH::KIND>(d[q * E + n]);
        else w = tc_pack2<SH::KIND>(d[q * E + n], d[NL + q * E + n]);
        *reinterpret_cast<uint32_t*>(p + off) = w;
      }
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

// Named barrier of the 128 threads of one task slot (ids 1..4; 0 is the CTA
// barrier), plain and with an OR reduction of a predicate.
__device__ __forceinline__ void slot_sync(int id) { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }
__device__ __forceinline__ bool slot_sync_or(int id, bool v) {
  uint32_t r;
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.u32 q, %2, 0;\nbar.red.or.pred p, %1, 128, q;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(r)
      : "r"(id), "r"((uint32_t)v)
      : "memory");
  return r != 0;
}

// Node rows past the n_p^3 rows of a TMA-loaded cell tile that the F-x
// operand build reads: line groups and x indices padded to E alias later rows
// of the tile (their B entries are zero), and the rows past its end must read
// as zero.
template <int E>
__host__ __device__ constexpr int tc_guard_rows(int np) {
  return (E - 1) * (np + 1) - np * np + 1 > 0 ? (E - 1) * (np + 1) - np * np + 1 : 0;
}

// Largest loaded box with its guard rows, in node rows, over n_p = 2 .. E.
template <int E>
__host__ __device__ constexpr int tc_box_rows_max() {
  int m = 0;
  for (int n = 2; n <= E; ++n) m = n * n * n + tc_guard_rows<E>(n) > m ? n * n * n + tc_guard_rows<E>(n) : m;
  return m;
}

// Task nt exists and its box lies inside the node grid (not on a periodic seam).
__device__ __forceinline__ bool tc_box_task(int nt, int n_tasks, int n_vb, const int* cells, const MeshDev& m) {
  if (nt >= n_tasks) return false;
  const int e = cells[nt / n_vb];
  const int cx = e % m.nx, cy = (e / m.nx) % m.ny, cz = e / (m.nx * m.ny);
  return !(m.periodic && (cx == m.nx - 1 || cy == m.ny - 1 || cz == m.nz - 1));
}

template <typename TIO>
__device__ __forceinline__ TIO tc_zero() {
  if constexpr (sizeof(TIO) == 4) return 0.f;
  else return __ushort_as_bfloat16((unsigned short)0);
}
__device__ __forceinline__ void tc_atomic_add(float* p, float v) { atomicAdd(p, v); }
__device__ __forceinline__ void tc_atomic_add(__nv_bfloat16* p, float v) { atomicAdd(p, __float2bfloat16_rn(v)); }

// One persistent CTA per SM with SH::SLOTS task slots.  Slot s is warpgroup s
// (threads 128 s ... 128 s + 127): it loops over the (cell, 8-vector block)
// tasks s, s + SLOTS, ... of this CTA's share of one colour, with its own
// tensor-memory columns, A buffers and mbarriers, so the slots' passes overlap
// one another's latencies.  Thread lt of a slot owns TMEM lane lt, i.e. row
// lt of every 128-row tile of a pass.
//
// TMA: the cell's values for the task's 8 vectors arrive as one tensor-map
// box (8 vectors x n_p^3 nodes, dense) in the slot's A buffer (loaded while
// the slot's previous task runs its last passes); Dirichlet nodes are zeroed,
// then every thread builds its rows of the F-x operand from the box.  The
// result is written into the same buffer as a box of the same shape
// (Dirichlet nodes 0) and added to Y by one bulk reduce; Y starts at zero,
// cells of one colour share no node, and colours run in order, so every sum
// is formed in the same order as by the colour-ordered stores and adds of
// the thread path.  Cells on a periodic seam, whose boxes would reach past
// the end of the node grid, take the thread path.  Without TMA (n_vec not a
// multiple of 16 bytes, unaligned blocks, or fe_set_tile variant 2) every
// thread loads and stores its own values, first writers storing and later
// colours adding.
// QF: n_q = E, so every quadrature point of the padded lines exists; with
// TMA, the cell's c values are then staged by one bulk copy into the F-x
// operand buffer once F-x has read it.
// GEN: per-point metric (trilinear cells); otherwise the one metric of the
// box mesh is part of the B operand of B-z and the point operation is c val.
template <int E, int G, int KIND, typename TIO, bool GEN, bool TMA, bool QF>
__global__ void __launch_bounds__(128 * TcShape<E, G, KIND>::SLOTS, 1)
    tc_apply_kernel(const TcArgs args, const MeshDev m, const Geom<float> geo, const int* __restrict__ cells,
                    int n_tasks, int n_vec, int n_vb, const TIO* __restrict__ X, TIO* __restrict__ Y,
                    const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap ymap) {
  using SH = TcShape<E, G, KIND>;
  constexpr int H = SH::H, T = SH::T, SLOTS = SH::SLOTS, V = kTcVectors;
  // A buffer (Mb) during a task with TMA: the result box at offset 0 (after
  // B-x), the next task's loaded box from BOX_IN on (issued once B-y is
  // complete; until then the operands of F-y ... B-y use the whole buffer,
  // and from then on the operand of B-x lies below BOX_IN)
  constexpr int BOX_OUT_MAX = E * E * E * V * (int)sizeof(TIO);
  constexpr int BX_A = 128 * SH::T * SH::Kr(5) * SH::ES;
  constexpr int BOX_IN = (BX_A > BOX_OUT_MAX ? BX_A : BOX_OUT_MAX + 127) / 128 * 128;
  static_assert(!TMA || BOX_IN + tc_box_rows_max<E>() * V * (int)sizeof(TIO) <= SH::M_BYTES,
                "result box, B-x operand and the next loaded box fit the A buffer");
  static_assert(SH::B_BYTES % 128 == 0 && SH::SLOT_BYTES % 128 == 0 && SH::S_BYTES % 128 == 0,
                "A buffers start 128 bytes apart");
  extern __shared__ __align__(128) unsigned char smem[];
  const int t = threadIdx.x, warp = t >> 5, slot = t >> 7, lt = t & 127;
  unsigned char* Bs = smem;
  unsigned char* Sb = smem + SH::B_BYTES + slot * SH::SLOT_BYTES;
  unsigned char* Mb = Sb + SH::S_BYTES;
  uint64_t* mbars = reinterpret_cast<uint64_t*>(smem + SH::B_BYTES + SLOTS * SH::SLOT_BYTES);
  uint64_t* mbar = mbars + slot;            // MMA completions (six per task)
  uint64_t* lbar = mbars + SLOTS + slot;    // box loads (one per task)
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbars + 2 * SLOTS);
  // per slot: 2 x (the task taken from the queue) + (its box is being loaded)
  int* tnext = reinterpret_cast<int*>(tslot + 1);
  TIO* box = reinterpret_cast<TIO*>(Mb);              // result box
  TIO* box_in = reinterpret_cast<TIO*>(Mb + BOX_IN);   // loaded box
  const int bar = 1 + slot;
  const int np = args.np, nq = QF ? E : args.nq, P = np - 1;
  const int nq2 = nq * nq, nq3 = nq2 * nq;
  const int np2 = np * np, np3 = np2 * np;
  // the cell's c values (n_q^3 floats, contiguous) are staged in shared memory
  constexpr bool CVS = TMA && QF;
  if constexpr (TMA) {
    // box destinations must be 128-byte aligned; the layout keeps every A
    // buffer at a multiple of 128 bytes from the base of shared memory
    if (smem_u32(smem) & 127u) {
      if (t == 0) atomicMax(args.status, (int)FE_EUNSUPPORTED);
      return;
    }
  }

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(SH::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (lt == 0) {
    mbar_init(mbar, 1);
    mbar_init(lbar, 1);
    if constexpr (TMA) {
      tma_prefetch_map(&xmap);
      tma_prefetch_map(&ymap);
    }
  }
  {  // B operands -> shared (once per CTA); the A buffers start at zero
    const uint4* src = reinterpret_cast<const uint4*>(args.bimg);
    uint4* dst = reinterpret_cast<uint4*>(Bs);
    for (int k = t; k < SH::B_BYTES / 16; k += blockDim.x) dst[k] = __ldg(src + k);
    uint4* z = reinterpret_cast<uint4*>(smem + SH::B_BYTES);
    for (int k = t; k < SLOTS * SH::SLOT_BYTES / 16; k += blockDim.x) z[k] = make_uint4(0, 0, 0, 0);
  }
  fence_async_smem();
  asm volatile("fence.mbarrier_init.release.cluster;");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot + (uint32_t)(slot * SH::SLOT_COLS);
  const uint32_t tlane = tmem + ((uint32_t)((warp & 3) * 32) << 16);
  bool fail = false, load_pending = false;
  uint32_t lphase = 0;

  // TMA kernels take their tasks from the launch's counter, one at a time
  // (the next one while the current task's last passes run), so that slots
  // whose tasks take the thread path do not hold up the launch; otherwise
  // slot s of CTA b takes tasks 4 b + s, 4 b + s + 4 grid, ...
  int next_task = (int)blockIdx.x * SLOTS + slot;
  if constexpr (TMA) {
    if (lt == 0) tnext[slot] = atomicAdd(args.queue, 1);
    slot_sync(bar);
    next_task = tnext[slot];
  }
  for (int task = next_task; task < n_tasks && !fail; task = next_task) {
    if constexpr (!TMA) next_task = task + (int)gridDim.x * SLOTS;
    // TMA: thread 0 takes the next task now; the counter's answer is used
    // once B-y is complete, long after it has arrived
    int taken = 0;
    if (TMA && lt == 0) taken = atomicAdd(args.queue, 1);
    const int e = cells[task / n_vb];
    const int v0 = (task % n_vb) * kTcVectors;
    const int cx = e % m.nx, cy = (e / m.nx) % m.ny, cz = e / (m.nx * m.ny);
    // This thread's rows: tile j, line group L = 16 j + lt / 8 = (slow, b)
    // with b = (lt / 8) % H fixed and slow = (16 j + lt / 8) / H; vector v.
    const int v = lt & 7, bq = (lt >> 3) % H;
    const bool vok = v0 + v < n_vec;
    // Per-task node tables: validity and first-writer bit masks precomputed
    // per cell on the host (bit i: node i along the direction).
    const unsigned long long cm = __ldg(args.cmask + task / n_vb);
    const unsigned xv = (unsigned)(cm & 0xffu), xf = (unsigned)((cm >> 8) & 0xffu);
    const unsigned yv_all = (unsigned)((cm >> 16) & 0xffu), yf_all = (unsigned)((cm >> 24) & 0xffu);
    const unsigned zv_all = (unsigned)((cm >> 32) & 0xffu), zf_all = (unsigned)((cm >> 40) & 0xffu);
    const size_t plane = (size_t)m.Nx * m.Ny * n_vec;
    // The cell lies across a periodic seam (its box would reach past the end
    // of the node grid along x / y / z).  With TMA, such a cell takes the
    // thread path: a box that reaches outside the tensor is moved at a much
    // lower rate than one inside it.
    const bool seam = m.periodic && (cx == m.nx - 1 || cy == m.ny - 1 || cz == m.nz - 1);
    const bool thr = !TMA || seam;
    // thread path: element offsets along x (all E entries) and along the
    // thread's G lines in y
    int xo[E];
    int yo[G];
    unsigned yv = 0, yf = 0;
    // TMA path: a "clean" cell has no Dirichlet node
    bool clean = true;
    if (thr) {
#pragma unroll
      for (int i = 0; i < E; ++i) xo[i] = node_coord(cx, i, P, m.Nx, m.periodic) * n_vec;
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int i2 = G * bq + g;
        yo[g] = node_coord(cy, i2, P, m.Ny, m.periodic) * m.Nx * n_vec;
        yv |= ((yv_all >> i2) & 1u) << g;
        yf |= ((yf_all >> i2) & 1u) << g;
      }
    }

    if (TMA && !thr) {
      // ---- gather: one box load (prefetched by the previous task unless
      // this is the slot's first box), Dirichlet nodes zeroed, operand rows ----
      const unsigned full = (1u << np) - 1u;
      clean = xv == full && yv_all == full && zv_all == full;
      // the previous task's reduce has read its result box before F-y's
      // operand overwrites it (the barrier below orders every later write)
      if (lt == 0) bulk_wait_read_all();
      if (!load_pending) {   // nothing prefetched for this task
        if (lt == 0) {
          mbar_arrive_expect_tx(lbar, (uint32_t)(np3 * V * (int)sizeof(TIO)));
          tma_load_4d(box_in, &xmap, v0, cx * P, cy * P, cz * P, lbar);
        }
        const int words = tc_guard_rows<E>(np) * V * (int)sizeof(TIO) / 16;
        uint4* gz = reinterpret_cast<uint4*>(box_in + np3 * V);
        for (int k = lt; k < words; k += 128) gz[k] = make_uint4(0, 0, 0, 0);
        load_pending = true;
      }
      if (slot_sync_or(bar, !mbar_wait_timed(lbar, lphase))) {
        fail = true;
        break;
      }
      load_pending = false;
      lphase ^= 1u;
      if (!clean) {   // the same for every thread of the slot
        for (int n = lt; n < np3; n += 128) {
          const int i1 = n % np, i2 = (n / np) % np, i3 = n / np2;
          if (!((xv >> i1) & (yv_all >> i2) & (zv_all >> i3) & 1u)) {
            TIO* row = box_in + n * V;
#pragma unroll
            for (int k = 0; k < V; ++k) row[k] = tc_zero<TIO>();
          }
        }
        slot_sync(bar);
      }
#pragma unroll
      for (int j = 0; j < T; ++j) {
        const int r = j * 128 + lt, L = tc_lg<SH>(r >> 3);
        if (L >= SH::LINES) continue;
        const int i3 = L / H;
        float vals[SH::Kr(0)];
#pragma unroll
        for (int k = 0; k < SH::Kr(0); ++k) vals[k] = 0.f;
        if (i3 < np) {
          const TIO* s0 = box_in + (i3 * np + G * (L % H)) * np * V + v;
#pragma unroll
          for (int g = 0; g < G; ++g) {
            const TIO* sg = s0 + g * np * V;
#pragma unroll
            for (int i1 = 0; i1 < E; ++i1) vals[g * E + i1] = tc_load(sg + i1 * V);
          }
        }
        tc_write_row<SH, SH::Kr(0)>(vals, r, Sb);
      }
    } else {
      // ---- gather: row (i3, b) x v, lines i2 = G b + g, K = [g][i1]; every
      // load of the thread is issued before the first use ----
#pragma unroll
      for (int j = 0; j < T; ++j) {
        const int r = j * 128 + lt, L = tc_lg<SH>(r >> 3);
        if (L >= SH::LINES) continue;
        const int i3 = L / H;
        const int gz = node_coord(cz, i3, P, m.Nz, m.periodic);
        const bool zok = vok && ((zv_all >> i3) & 1u);
        const TIO* xz = X + (size_t)gz * plane + v0 + v;
        float vals[SH::Kr(0)];
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const bool ok = zok && ((yv >> g) & 1u);
#pragma unroll
          for (int i1 = 0; i1 < E; ++i1)
            vals[g * E + i1] = (ok && ((xv >> i1) & 1u)) ? tc_load(xz + yo[g] + xo[i1]) : 0.f;
        }
#pragma unroll
        for (int k = G * E; k < SH::Kr(0); ++k) vals[k] = 0.f;
        tc_write_row<SH, SH::Kr(0)>(vals, r, Sb);
      }
    }
    // ---- the six passes ----
    // pass index s = 0..5, mbarrier phase = s & 1 (six completions per task).
    // Every thread's writes of the A operand become visible to the tensor
    // cores, the slot's thread 0 issues the pass, the slot waits for its
    // completion (bounded by time; a timeout ends the slot's loop).  The pass
    // reads A from shared memory and writes D to tensor memory only, so the
    // next A may overwrite this one as soon as the pass is complete.
    // Only the slot's first warp polls the mbarrier; the other three sleep
    // in the named barrier that follows.
#define FE_TC_ISSUE_X(S, ABUF, EXTRA_FAIL)                                     \
  fence_async_smem();                                                          \
  tc_fence_before();                                                           \
  slot_sync(bar);                                                              \
  if (lt == 0) tc_issue<SH, S>(tmem, ABUF, Bs, mbar);                          \
  if (slot_sync_or(bar, (lt < 32 && !mbar_wait_timed(mbar, (S) & 1)) || (EXTRA_FAIL))) { \
    fail = true;                                                               \
    break;                                                                     \
  }                                                                            \
  tc_fence_after();
#define FE_TC_ISSUE(S, ABUF) FE_TC_ISSUE_X(S, ABUF, false)

    FE_TC_ISSUE(0, Sb)
    if constexpr (CVS) {   // F-x has read its operand: the cell's c values take its place
      if (lt == 0) {
        mbar_arrive_expect_tx(lbar, (uint32_t)kTcCvBytes);
        bulk_load(Sb, args.cvs + (size_t)e * (kTcCvBytes / 4), (uint32_t)kTcCvBytes, lbar);
      }
      load_pending = true;
    }
#pragma unroll 1
    for (int j = 0; j < T; ++j) {   // F-x: row (i3, b), lines i2 -> A of F-y: (q1, i3 / G)
      float d[SH::Nr(0)];
      tmem_load<SH::Nr(0)>(tlane + j * SH::Nr(0), d);
      const int r = j * 128 + lt, L = tc_lg<SH>(r >> 3);
      if (L < SH::LINES) tc_write_transposed<SH, 2, true, SH::Kr(1)>(d, L / H, L % H, r & 7, Mb);
    }
    FE_TC_ISSUE(1, Mb)
#pragma unroll 1
    for (int j = 0; j < T; ++j) {   // F-y: row (q1, b), lines i3 -> A of F-z: (q1, q2 / G)
      float d[SH::Nr(1)];
      tmem_load<SH::Nr(1)>(tlane + j * SH::Nr(1), d);
      const int r = j * 128 + lt, L = r >> 3;
      if (L < SH::LINES) tc_write_transposed<SH, 3, false, SH::Kr(2)>(d, L / H, L % H, r & 7, Mb);
    }
    FE_TC_ISSUE_X(2, Mb, CVS && !mbar_wait_timed(lbar, lphase))
    if constexpr (CVS) {
      load_pending = false;
      lphase ^= 1u;
    }
#pragma unroll 1
    for (int j = 0; j < T; ++j) {   // F-z and the quadrature-point operation: row (q1, b), lines q2 = G b + g
      float d[SH::Nr(2)];
      tmem_load<SH::Nr(2)>(tlane + j * SH::Nr(2), d);
      const int r = j * 128 + lt, L = r >> 3;
      if (L >= SH::LINES) continue;
      const int q1 = L / H, b = L % H;
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int q2 = G * b + g;
        float* dl = d + g * 4 * E;   // [val | dz | dy | dx] along q3, becomes [hv | hz | hy | hx]
        // points (q1, q2, q3) of this line: q3 < nq exist when the line does
        // (values at padded points meet zero B entries in B-z)
        const bool line = QF || (q1 < nq && q2 < nq);
        const float* pc = CVS ? reinterpret_cast<const float*>(Sb) + tc_cv_index(q1, q2, 0)
                              : geo.ptC + (size_t)e * nq3 + q1 + nq * q2;
        const float* pg0 = GEN ? geo.ptG + (size_t)e * 6 * nq3 + q1 + nq * q2 : nullptr;
#pragma unroll
        for (int q3 = 0; q3 < E; ++q3) {
          float cv = 0.f;
          if (QF || (line && q3 < nq)) {
            cv = CVS ? pc[tc_cv_index(0, 0, q3)] : __ldg(pc + q3 * nq2);
            if (GEN) {
              const float* pg = pg0 + q3 * nq2;
              const float g00 = __ldg(pg), g01 = __ldg(pg + nq3), g02 = __ldg(pg + 2 * nq3);
              const float g11 = __ldg(pg + 3 * nq3), g12 = __ldg(pg + 4 * nq3), g22 = __ldg(pg + 5 * nq3);
              const float dz = dl[E + q3], dy = dl[2 * E + q3], dx = dl[3 * E + q3];
              dl[E + q3] = g02 * dx + g12 * dy + g22 * dz;
              dl[2 * E + q3] = g01 * dx + g11 * dy + g12 * dz;
              dl[3 * E + q3] = g00 * dx + g01 * dy + g02 * dz;
            }
          }
          dl[q3] = cv * dl[q3];
        }
      }
      tc_write_row<SH, SH::Kr(3)>(d, r, Mb);
    }
    FE_TC_ISSUE(3, Mb)
#pragma unroll 1
    for (int j = 0; j < T; ++j) {   // B-z: row (q1, b), lines q2 -> A of B-y: (i3, q1 / G)
      float d[SH::Nr(3)];
      tmem_load<SH::Nr(3)>(tlane + j * SH::Nr(3), d);
      const int r = j * 128 + lt, L = r >> 3;
      if (L < SH::LINES) tc_write_transposed<SH, 3, true, SH::Kr(4)>(d, L / H, L % H, r & 7, Mb);
    }
    FE_TC_ISSUE(4, Mb)
    if constexpr (TMA) {   // take the next task; prefetch its box unless it takes the thread path
      if (lt == 0) {
        const int nt = taken;
        const bool pf = tc_box_task(nt, n_tasks, n_vb, cells, m);
        tnext[slot] = 2 * nt + (pf ? 1 : 0);
        if (pf) {
          const int e2 = cells[nt / n_vb];
          const int cx2 = e2 % m.nx, cy2 = (e2 / m.nx) % m.ny, cz2 = e2 / (m.nx * m.ny);
          mbar_arrive_expect_tx(lbar, (uint32_t)(np3 * V * (int)sizeof(TIO)));
          tma_load_4d(box_in, &xmap, (nt % n_vb) * kTcVectors, cx2 * P, cy2 * P, cz2 * P, lbar);
          load_pending = true;
        }
      }
    }
#pragma unroll 1
    for (int j = 0; j < T; ++j) {   // B-y: row (i3, b), lines q1 -> A of B-x: (i3, i2 / G)
      float d[SH::Nr(4)];
      tmem_load<SH::Nr(4)>(tlane + j * SH::Nr(4), d);
      const int r = j * 128 + lt, L = r >> 3;
      if (L < SH::LINES) tc_write_transposed<SH, 2, false, SH::Kr(5), true>(d, L / H, L % H, r & 7, Mb);
    }
    FE_TC_ISSUE(5, Mb)
    if constexpr (TMA) {   // the task thread 0 took, and whether its box is loading
      const int tn = tnext[slot];   // written before the barrier above
      next_task = tn >> 1;
      if (tn & 1) {
        const int words = tc_guard_rows<E>(np) * V * (int)sizeof(TIO) / 16;
        uint4* gz = reinterpret_cast<uint4*>(box_in + np3 * V);
        for (int k = lt; k < words; k += 128) gz[k] = make_uint4(0, 0, 0, 0);
        load_pending = true;
      }
    }
    if (TMA && !thr) {
      // ---- result box (the A buffer is free once B-x is complete), then one
      // bulk reduce-add into Y ----
#pragma unroll 1
      for (int j = 0; j < T; ++j) {   // B-x: row (i3, b), lines i2 = G b + g, D = [g][i1]
        float d[SH::Nr(5)];
        tmem_load<SH::Nr(5)>(tlane + j * SH::Nr(5), d);
        const int r = j * 128 + lt, L = tc_lg<SH>(r >> 3);
        if (L >= SH::LINES) continue;
        const int i3 = L / H, b = L % H;
        if (i3 >= np) continue;
        const bool zok = (zv_all >> i3) & 1u;
        TIO* o = box + (i3 * np + G * b) * np * V + v;
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const int i2 = G * b + g;
          if (i2 >= np) continue;
          const unsigned ok = (zok && ((yv_all >> i2) & 1u)) ? xv : 0u;
#pragma unroll
          for (int i1 = 0; i1 < E; ++i1)
            if (i1 < np) tc_store(o + (g * np + i1) * V, ((ok >> i1) & 1u) ? d[g * E + i1] : 0.f);
        }
      }
      fence_async_smem();
      slot_sync(bar);
      if (lt == 0) {
        tma_reduce_add_4d(&ymap, box, v0, cx * P, cy * P, cz * P);
        bulk_commit();
      }
    } else {
#pragma unroll 1
      for (int j = 0; j < T; ++j) {   // B-x and assembly: row (i3, b), lines i2 = G b + g, D = [g][i1]
        float d[SH::Nr(5)];
        tmem_load<SH::Nr(5)>(tlane + j * SH::Nr(5), d);
        const int r = j * 128 + lt, L = tc_lg<SH>(r >> 3);
        if (L >= SH::LINES || !vok) continue;
        const int i3 = L / H;
        if (i3 >= np) continue;
        const int gz = node_coord(cz, i3, P, m.Nz, m.periodic);
        const bool zcon = !((zv_all >> i3) & 1u);
        const bool zfirst = (zf_all >> i3) & 1u;
        TIO* yz = Y + (size_t)gz * plane + v0 + v;
        // every read of Y (the partial sums of earlier colours) is issued
        // before the first store, so the loads overlap
        float old[G * E];
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const unsigned rd = (zcon || !((yv >> g) & 1u)) ? 0u
                              : xv & ~((zfirst && ((yf >> g) & 1u)) ? xf : 0u);
#pragma unroll
          for (int i1 = 0; i1 < E; ++i1) old[g * E + i1] = ((rd >> i1) & 1u) ? tc_load(yz + yo[g] + xo[i1]) : 0.f;
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
          if (G * bq + g >= np) continue;
          const bool ycon = zcon || !((yv >> g) & 1u);
          const unsigned first = (zfirst && ((yf >> g) & 1u)) ? xf : 0u;
          const unsigned valid = ycon ? 0u : xv;
#pragma unroll
          for (int i1 = 0; i1 < E; ++i1) {
            if (i1 >= np) continue;
            TIO* dst = yz + yo[g] + xo[i1];
            if ((first >> i1) & 1u) tc_store(dst, ((valid >> i1) & 1u) ? d[g * E + i1] : 0.f);
            else if ((valid >> i1) & 1u) tc_store(dst, old[g * E + i1] + d[g * E + i1]);
          }
        }
      }
    }
#undef FE_TC_ISSUE
#undef FE_TC_ISSUE_X
  }

  if (fail && lt == 0) {
    atomicMax(args.status, (int)FE_ETIMEOUT);
    // let any MMA or box load of this slot still in flight finish before the
    // shared and tensor memory are released
    mbar_wait_timed(mbar, 0, 100000000ull);
    mbar_wait_timed(mbar, 1, 100000000ull);
    if (load_pending) mbar_wait_timed(lbar, lphase, 100000000ull);
  }
  if constexpr (TMA) {
    if (lt == 0) bulk_wait_all();   // the reduces of this slot are complete
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*tslot), "r"(SH::TMEM_COLS));
}

}  // namespace fe
