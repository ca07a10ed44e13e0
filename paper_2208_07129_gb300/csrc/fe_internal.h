// Internal types of libfe shared by the host setup, the C ABI and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <vector>

#include "../../include/fe.h"
#include "fe_ff.cuh"

namespace fe {

constexpr int kMaxP = 8;
constexpr size_t kSmallSlots = 16384;   // cells x n_p^3 of a "small" mesh (see fe_ctx::d_small)
constexpr int kMaxNQ = kMaxP + 3;

// Entries of the explicit cell -> DoF map of refined meshes: the DoF index in
// the low 29 bits, bit 29 set for a Dirichlet node, bit 30 set when this
// (cell, node) is the node's first writer in colour order.
constexpr int kMapIndex = (1 << 29) - 1, kMapConstrained = 1 << 29, kMapFirst = 1 << 30;

// Structured-mesh description as the kernels see it.
struct MeshDev {
  int nx, ny, nz;     // cells
  int Nx, Ny, Nz;     // stored nodes per direction
  int periodic;       // 1: wrap-around numbering
  int cx_col, cy_col; // colours per direction in x and y (2 or 3); colour
                      // index = kx + cx_col (ky + cy_col kz)
  int last_odd_x, last_odd_y, last_odd_z;  // periodic with odd n: last cell takes colour 2
};

// 1D tables with the square roots of the quadrature weights folded in
// (Sec. 3.2.4: N(q,i) <- N(q,i) sqrt(w_q), D~(q1,q2) <- D~(q1,q2) sqrt(w_q1/w_q2)),
// so that the quadrature-point operation needs no weights.  Passed by value
// as a kernel parameter (constant bank) so every contraction reads its
// coefficients as uniform constant operands.
template <typename T, int NP, int NQ>
struct Tables {
  T N[NQ][NP];
  T D[NQ][NQ];
};

// Geometry of the quadrature-point operation.  With weights folded into the
// tables:  G_sd = mu det J (J^-1 J^-T)_sd   and   c = det J V.
// Affine cells (axis-aligned boxes): one G per cell (cellG[e*6 + k],
// k = 00,01,02,11,12,22), diagonal: the even-odd and double-float bodies
// read only k = 00, 11, 22.
// General (trilinear) cells: ptG[(e*6 + k) * nq3 + Q].  Always ptC[e*nq3 + Q].
template <typename T>
struct Geom {
  const T* cellG;
  const T* ptG;
  const T* ptC;
};

// Epilogue of the scaled product of the Chebyshev filter,
//   Y = a M^-1/2 A M^-1/2 X + b X + c Y   (msq = M^-1/2, one value per DoF),
// fused into the gather (X M^-1/2) and the first-writer scatter.
template <typename T>
struct Scale {
  const T* msq;
  T a, b, c;
};

struct ColorSet {
  int n_colors;
  std::vector<int> offset;  // n_colors + 1
};

// Workspace of the block-PCG solver, grown on demand and kept in the context.
struct SolveWs {
  double* v64[4] = {nullptr, nullptr, nullptr, nullptr};
  size_t cap64[4] = {0, 0, 0, 0};
  float* v32[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  size_t cap32[6] = {0, 0, 0, 0, 0, 0};
  double* colbuf = nullptr;  // per-column scalars
  size_t cap_col = 0;
  double* partial = nullptr; // per-CTA column partial sums
  size_t cap_partial = 0;
  int* active = nullptr;     // per-column "not yet converged" flags
  size_t cap_active = 0;
  double* diag = nullptr;
  double* dinv64 = nullptr;
  float* dinv32 = nullptr;
};

struct LearnedPrecond;

struct KernelLaunch {
  const int* cells;   // cell ids of this colour (device)
  int n_cells;
  int n_vec;
  int vb;             // vectors per CTA
  int nty;            // lines in flight per CTA (blockDim.y)
  cudaStream_t stream;
};

}  // namespace fe

// Floats per cell of fe_ctx::d_ptCtc: 8 planes of 72 (64 values, 8 of padding).
constexpr int kTcCvWords = 8 * 72;

struct fe_ctx {
  // mesh and discretisation
  int nx, ny, nz, periodic, p, np, nq, quad_kind;
  double mu;
  int general;                 // 1: per-point metric (trilinear cells)
  size_t n_dofs, n_cells;
  fe::MeshDev mdev;
  // host FP64 data
  std::vector<double> gll, wgll, qx, qw, N1, D1;   // N1[q*np+i], D1[q*nq+k] (unfolded)
  std::vector<double> Nf, Df;                // folded
  std::vector<double> vertices;              // copy of the vertex array (general)
  double box_lo[3] = {0, 0, 0}, box_h[3] = {1, 1, 1};  // uniform box: corner and cell size
  std::vector<double> detJ;                  // per point (E*nq3)
  std::vector<double> cellG, ptG;            // FP64 metric (affine / general)
  std::vector<int> cells_by_color;
  fe::ColorSet colors;
  // device data
  int* d_cells = nullptr;
  double *d_cellG64 = nullptr, *d_ptG64 = nullptr, *d_ptC64 = nullptr;
  float *d_cellG32 = nullptr, *d_ptG32 = nullptr, *d_ptC32 = nullptr;
  // n_q = 8 (tcgen05 kernel): the same FP32 c values per cell in the layout
  // the kernel stages them in (kTcCvWords floats per cell, see fe_setup.cu)
  float* d_ptCtc = nullptr;
  fe::ff *d_cellGff = nullptr, *d_ptGff = nullptr, *d_ptCff = nullptr;   // double-float copies
  double* d_detJ = nullptr;
  int* d_status = nullptr;
  // staging for fe_apply_host, and the copy streams and events of its
  // pipeline (created on first use)
  void* d_stage = nullptr;
  size_t stage_bytes = 0;
  cudaStream_t copy_in = nullptr, copy_out = nullptr;
  cudaEvent_t ev_start = nullptr, ev_in[2] = {}, ev_comp[2] = {}, ev_out[2] = {};
  fe_mode mode = FE_FP64;
  fe_mode inner_mode = FE_FP32;   // arithmetic of the inner solve (refinement)
  fe_mode op64 = FE_FP64;         // operator of FP64-data PCG: FE_FP64, or FE_DF64 (double-float)
  // one-level refined mesh with hanging nodes: explicit cell -> DoF map and
  // the constraints u_S = W u_M (slave rows for the distribute step, master
  // rows for the condense step)
  int refined = 0;
  int* d_map = nullptr;                 // E x n_p^3 entries (kMap* bits)
  std::vector<double> cell_lo, cell_h;  // per cell: box corner and size (3 each)
  std::vector<double> node_xyz;         // per DoF: physical coordinates
  int n_slaves = 0, n_masters = 0;
  int* d_row_slave = nullptr;           // per DoF: its slave number, or -1
  int *d_sl_ptr = nullptr, *d_sl_idx = nullptr;   // slave -> masters (CSR)
  double* d_sl_w = nullptr;
  float* d_sl_w32 = nullptr;
  int *d_slaves = nullptr;              // DoF of each slave
  int *d_ma_rows = nullptr, *d_ma_ptr = nullptr, *d_ma_idx = nullptr;   // master -> slaves (CSR)
  double* d_ma_w = nullptr;
  float* d_ma_w32 = nullptr;
  void* d_xc = nullptr;                 // X with the slave rows filled in
  size_t xc_bytes = 0;
  fe::SolveWs ws;
  fe::LearnedPrecond* learned = nullptr;
  // eigenvalue layer: GLL diagonal mass (host), M^-1/2 on the device, and the
  // dense linear-algebra handles of the subspace iteration (created on first use)
  std::vector<double> mass;
  double* d_msq64 = nullptr;
  float* d_msq32 = nullptr;
  void* blas = nullptr;
  void* solver = nullptr;
  // launch shape per mode (vectors per CTA, lines per CTA)
  int vb64 = 8, nty64 = 16, vb32 = 8, nty32 = 32, vbdf = 8, ntydf = 32;
  int fp32_variant = 0;   // 0 / 1: line kernel, 2: register-plane kernel, 3: even-odd line kernel
  int fp64_variant = 0;   // 0: even-odd line kernel, 1: plain line kernel
  int tc_variant = 0;     // FE_TF32 / FE_BF16 / FE_BF16S: 0 tcgen05 kernel (where built) with TMA boxes where
                          // the blocks allow, 1 warp-MMA kernel (not FE_BF16S), 2 tcgen05 with thread loads/stores
  // B operands of the tcgen05 kernel's six passes (TF32, BF16), built at setup
  // when n_p, n_q <= 8
  unsigned char* d_tcimg[2] = {nullptr, nullptr};
  // per cell (colour order): bit masks of its nodes along x, y, z that exist
  // and are free, and of those it writes first (tcgen05 kernel)
  unsigned long long* d_tcmask = nullptr;
  int* d_tcq = nullptr;     // tcgen05 TMA launches: one task counter per colour, zeroed by each product
  // small meshes (E n_p^3 <= kSmallSlots): per-cell result scratch for up to
  // 64 FP64 vectors, so that fe_apply runs as two launches instead of one per
  // colour; allocated at setup
  void* d_small = nullptr;
  size_t small_bytes = 0;
};

namespace fe {
// Raise a kernel's dynamic shared-memory limit to at least `smem` bytes on the
// current device.  The attribute belongs to the kernel as loaded on one
// device, so the highest value set is remembered per (kernel, device); the
// cache is guarded by a mutex, so host threads may launch concurrently.
cudaError_t ensure_dyn_smem(const void* kern, size_t smem);
// Status of a CUDA runtime result (FE_OK, FE_ENOMEM or FE_ECUDA); a failure
// is also recorded as the calling host thread's last CUDA error, with the
// step that met it when `where` (a static string) is given, which
// fe_last_cuda_error() reports.
fe_status cuda_status(cudaError_t e, const char* where = nullptr);
// Kernel dispatch (defined in the kernel translation units).
cudaError_t apply_cc_f64(const fe_ctx* c, const double* X, double* Y, int n_vec, cudaStream_t s);
cudaError_t apply_cc_f32(const fe_ctx* c, const float* X, float* Y, int n_vec, cudaStream_t s);
cudaError_t diagonal_f64(const fe_ctx* c, double* diag, cudaStream_t s);
cudaError_t apply_mma_f32(const fe_ctx* c, const float* X, float* Y, int n_vec, cudaStream_t s, fe_mode mode);
cudaError_t apply_df64(const fe_ctx* c, const double* X, double* Y, int n_vec, cudaStream_t s);
// tcgen05 cell kernel (fe_apply_tc.cu): FE_TF32, FE_BF16 (FP32 data) and FE_BF16S (BF16 data).
cudaError_t build_tc_images(fe_ctx* c);
bool tc_supported(const fe_ctx* c);
cudaError_t apply_tc(const fe_ctx* c, const void* X, void* Y, int n_vec, cudaStream_t s, fe_mode mode);
cudaError_t apply_scaled_df64(const fe_ctx* c, const double* X, double* Y, int n_vec, const Scale<double>& sc,
                              cudaStream_t s);
cudaError_t apply_scaled_f64(const fe_ctx* c, const double* X, double* Y, int n_vec, const Scale<double>& sc,
                             cudaStream_t s);
cudaError_t apply_scaled_f32(const fe_ctx* c, const float* X, float* Y, int n_vec, const Scale<float>& sc,
                             cudaStream_t s);
// Setup helpers shared by the structured and the refined-mesh setup (fe_setup.cu).
void build_tables(fe_ctx* c);
double lagrange_1d(const double* xs, int n, int k, double t);
cudaError_t upload_point_coeff(fe_ctx* c, const std::vector<double>& ptC);
cudaError_t upload_ints(int** dst, const std::vector<int>& src);
cudaError_t upload_doubles(double** dst, const std::vector<double>& src);
cudaError_t upload_floats(float** dst, const std::vector<double>& src);
cudaError_t upload_ffs(ff** dst, const std::vector<double>& src);
// Refined meshes with hanging nodes (fe_refined.cu / fe_apply_refined.cu).
// xc_scratch: device block of X's size for the distribute step (X with the
// slave rows filled in); NULL = the context's own, allocated on first use.
cudaError_t apply_refined(fe_ctx* c, const void* X, void* Y, int n_vec, cudaStream_t s, void* xc_scratch = nullptr);
void free_refined(fe_ctx* c);
// GLL diagonal mass of Sec. 4.3 into c->mass (host, FP64; constrained rows 1).
void build_gll_mass(fe_ctx* c);
void free_eig(fe_ctx* c);
// Solver workspace and the learned preconditioner (fe_solve.cu / fe_learn.cu).
cudaError_t solver_workspace(fe_ctx* c, int nv);
void free_solver_workspace(fe_ctx* c);
bool learned_ready(const fe_ctx* c, int nv);
fe_status learned_precond_apply(fe_ctx* c, const void* r, void* z, int nv, bool fp64, cudaStream_t s);
void free_learned(fe_ctx* c);
}  // namespace fe
