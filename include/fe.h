/*
 * fe.h -- C ABI of libfe: matrix-free multivector products Y = A X for the
 * finite-element operator A = -mu lap + V(x) on a structured hexahedral mesh,
 * degree-p Lagrange elements on Gauss-Lobatto-Legendre nodes, run by
 * hand-written CUDA kernels for sm_103a (GB300).
 *
 * Operation (paper: Sec. 2.1 stiffness / mass integrals; Sec. 2.2 the
 * decomposition V = A U = sum_e Q^T A^(e) Q U under the constraints C; the
 * cell products of Algorithm 2, executed batch-wise as in Algorithm 4):
 *
 *   A_IJ = sum_e sum_Q w_Q det J [ mu (J^-T grad N_I).(J^-T grad N_J) + V(x_Q) N_I N_J ]
 *
 * with the tensor n_q-point quadrature rule (Gauss or GLL).
 *
 * Conventions shared by every call:
 *  - Multivectors are DoF-major and vector-contiguous (the paper's batched
 *    contiguous layout, Sec. 3.2.1, with one batch holding all n_vec
 *    vectors): element (dof, v) lives at X[dof * n_vec + v].  The dtype is
 *    double in FE_FP64 and FE_DF64 modes, bfloat16 in FE_BF16S mode and float
 *    in every other mode.
 *  - Global node (gx, gy, gz) has index gx + Nx (gy + Ny gz), where Nx = nx p + 1
 *    for a Dirichlet box and Nx = nx p for a periodic box (wrap-around).
 *  - Cells are e = cx + nx (cy + ny cz); quadrature points Q = q1 + n_q (q2 + n_q q3).
 *  - Dirichlet (FE_BC_DIRICHLET0): the operator is P A P, P zeroing the boundary
 *    nodes (Sec. 3.2.2: Dirichlet constraints have no master nodes).  Boundary
 *    entries of X are ignored (read as 0) and boundary rows of Y are written 0.
 *  - Device pointers are caller-owned CUDA device memory unless the name says
 *    "host".  Calls are asynchronous on `stream` (a cudaStream_t, NULL = legacy
 *    default stream) unless stated otherwise.
 *  - No call aborts.  Invalid arguments return FE_EINVAL before any launch;
 *    CUDA errors return FE_ECUDA.  Errors raised by asynchronous device work
 *    surface at the next call or through fe_last_device_status().
 */
#ifndef FE_H_
#define FE_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fe_ctx fe_ctx;

typedef enum {
  FE_OK = 0,
  FE_EINVAL = 1,        /* invalid argument, detected before any launch */
  FE_ENOMEM = 2,        /* host or device allocation failed */
  FE_ECUDA = 3,         /* a CUDA runtime call or launch failed */
  FE_ENOTCONV = 4,      /* iterative solve stopped before reaching rtol */
  FE_EBREAKDOWN = 5,    /* Krylov breakdown (p^T A p <= 0 or r^T z <= 0) */
  FE_ENONFINITE = 6,    /* NaN or Inf met in a result */
  FE_ETIMEOUT = 7,      /* a bounded device wait gave up */
  FE_EUNSUPPORTED = 8   /* valid request outside the compiled kernel set */
} fe_status;

typedef enum { FE_BC_DIRICHLET0 = 0, FE_BC_PERIODIC = 1 } fe_bc;
typedef enum { FE_QUAD_GAUSS = 0, FE_QUAD_GLL = 1 } fe_quad_kind;

/* Arithmetic of the cell kernels.  FE_FP64: double data, double arithmetic.
 * FE_FP32: float data, float arithmetic on CUDA cores.  FE_TF32 / FE_BF16:
 * float data, the sum-factorised contractions on tensor cores with FP32
 * accumulation (operands rounded to TF32 / BF16); the quadrature-point
 * operation stays FP32.  FE_TF32X3: as FE_TF32, but every operand is split
 * into hi + lo TF32 parts and each product is accumulated as
 * lo*hi + hi*lo + hi*hi (three tensor-core products; the split-TF32 scheme of
 * Ootomo and Yokota, 2022), which restores FP32-level accuracy.  FE_DF64:
 * double data; the cell kernel computes in double-float arithmetic (each
 * value an unevaluated sum of two floats, ~48 significant bits; error-free
 * sums and products, compensated dot products) on the FP32 pipe, which
 * GB300 runs at 64 times its FP64 rate; errors stay within the FP64 bound
 * (1e-12 relative).  Both parts of a double-float value are floats, so the
 * mode has FP32's exponent range: X, the potential and the results must stay
 * below ~3.4e38 in magnitude (larger values overflow to infinity), and a
 * value below ~1e-31 in magnitude keeps fewer than 48 significant bits (its
 * low part falls into the subnormal range; below ~1e-38 the high part does
 * too), so blocks with entries that small relative to FP64's range lose the
 * FP64-level accuracy; FE_FP64 has no such limit.  FE_BF16S: as FE_BF16, but X and Y are bfloat16 in
 * device memory (half the bytes of FE_BF16); the colour-ordered accumulation
 * of Y rounds to bfloat16 after every add.  FE_TF32, FE_BF16 and FE_BF16S run
 * on the tcgen05 tensor cores (operands in shared memory, FP32 accumulators in
 * tensor memory) when n_p <= 8 and n_q <= 8; FE_TF32 and FE_BF16 fall back to
 * warp-level MMA kernels otherwise, FE_BF16S is then FE_EUNSUPPORTED.
 * Geometry is always computed in FP64. */
typedef enum { FE_FP64 = 0, FE_FP32 = 1, FE_TF32 = 2, FE_BF16 = 3, FE_TF32X3 = 4, FE_DF64 = 5, FE_BF16S = 6 } fe_mode;

typedef struct {
  int nx, ny, nz;          /* cells per direction, >= 1 (>= 2 when periodic) */
  double lo[3], hi[3];     /* box corners (used when vertex_xyz == NULL) */
  int bc;                  /* fe_bc */
  const double* vertex_xyz;/* host, optional: (nx+1)(ny+1)(nz+1) x 3 vertex
                              coordinates, x fastest; each cell is the trilinear
                              image of [-1,1]^3 and gets per-point Jacobians.
                              Copied during fe_setup. */
} fe_mesh_desc;

typedef struct {
  int n_q;                 /* points per direction; p+1 <= n_q <= p+3 */
  int kind;                /* fe_quad_kind */
} fe_quad_desc;

/* Build the operator for degree p (1..8) on `mesh` with quadrature `quad`
 * and diffusion coefficient mu (the paper's mu; 1/2 for -1/2 lap).  The
 * potential starts at V = 0 (see fe_set_potential).  Computes in FP64 on the
 * host: GLL nodes, quadrature, the 1D shape-value matrix N (n_q x n_p) and the
 * collocation derivative matrix D~ (n_q x n_q) of Sec. 2.2, the Jacobians at
 * every quadrature point (rejecting det J <= 0 with FE_EINVAL), the metric
 * terms mu det J J^-1 J^-T of the cell stiffness, and the cell colouring used
 * for conflict-free assembly; then uploads them.  *out receives an opaque
 * handle owned by the caller (free with fe_destroy).  Synchronous. */
fe_status fe_setup(const fe_mesh_desc* mesh, int p, const fe_quad_desc* quad, double mu, fe_ctx** out);

/* One-level adaptively refined mesh with hanging nodes (Sec. 3.2.2; the
 * adaptive meshes of the paper's Sec. 4 benchmarks).  A Dirichlet box
 * [lo, hi] of nx x ny x nz coarse cells of size H per direction; the coarse
 * cells with index in [refine_lo, refine_hi) per direction are split once
 * into 2 x 2 x 2 children of size H / 2.
 *  - Cells: coarse cell by coarse cell (x fastest), a refined cell replaced by
 *    its 8 children (x fastest); V at quadrature points follows this order
 *    (fe_quadrature_points, fe_set_potential).
 *  - Nodes: the (p+1)^3 GLL nodes of every cell.  Along one direction a node
 *    sits at a vertex m H/2 of the half-size grid, at an interior GLL node of
 *    a coarse cell c (c H + (1 + g_i) H/2; the middle node of an even degree
 *    is the vertex 2c + 1) or at an interior GLL node of a fine cell f
 *    (f H/2 + (1 + g_j) H/4); nodes of different cells at the same point are
 *    one DoF.  DoFs are numbered by position, z slowest and x fastest.
 *  - Hanging nodes: a node of a fine cell on the closure of an unrefined
 *    coarse cell C that is not one of C's nodes is a slave, u_s =
 *    sum_m phi_m^C(x_s) u_m over C's nodes (C's interpolant; masters on the
 *    boundary carry 0).  The product is Y = C^T A C X on the free rows (C:
 *    free values -> all nodes) with the slave and Dirichlet rows of Y written
 *    0 and those entries of X ignored.
 * Supported on such a context: fe_num_*, fe_quadrature_points,
 * fe_set_potential, fe_set_mode (FE_FP64, FE_DF64, FE_FP32), fe_set_tile,
 * fe_apply, fe_apply_host, fe_destroy; the other calls return
 * FE_EUNSUPPORTED.  Synchronous. */
typedef struct {
  int nx, ny, nz;
  double lo[3], hi[3];
  int refine_lo[3], refine_hi[3];
} fe_refined_desc;
fe_status fe_setup_refined(const fe_refined_desc* mesh, int p, const fe_quad_desc* quad, double mu, fe_ctx** out);

/* Number of hanging (slave) nodes of a refined-mesh context (0 otherwise). */
int fe_num_slaves(const fe_ctx* ctx);

/* Physical coordinates of every DoF: xyz_host[dof * 3 + d] (host, FP64,
 * num_dofs x 3), for evaluating data at the nodes.  Synchronous. */
fe_status fe_node_coords(const fe_ctx* ctx, double* xyz_host);

/* Release everything the context owns.  NULL is allowed. */
void fe_destroy(fe_ctx* ctx);

/* Stored DoFs (boundary nodes included) and cells. */
size_t fe_num_dofs(const fe_ctx* ctx);
size_t fe_num_cells(const fe_ctx* ctx);
int fe_num_quad_points_1d(const fe_ctx* ctx);

/* Physical coordinates of every quadrature point: xyz_host[(e n_q^3 + Q) 3 + d],
 * caller-owned host buffer of E n_q^3 3 doubles.  Synchronous. */
fe_status fe_quadrature_points(const fe_ctx* ctx, double* xyz_host);

/* Set V at the quadrature points: Vq_host[e n_q^3 + Q] (host, FP64, E n_q^3
 * values; NULL sets V = 0).  The product det J w_Q V(x_Q) of the weighted mass
 * (Sec. 2.2, the diagonal G of M^kappa = N^T G N) is formed in FP64 and
 * uploaded.  Synchronous. */
fe_status fe_set_potential(fe_ctx* ctx, const double* Vq_host);

/* Select the arithmetic mode of later fe_apply calls (default FE_FP64). */
fe_status fe_set_mode(fe_ctx* ctx, fe_mode mode);
fe_mode fe_get_mode(const fe_ctx* ctx);

/* Y = A X for n_vec >= 0 vectors (Algorithm 2 per cell, batched over cells and
 * vector blocks as in Algorithm 4, assembled by cell colours: no two cells of
 * a colour share a node and colours run in order, so every node's sum is
 * formed in a fixed order and results are deterministic; the tcgen05 kernel's
 * TMA path zeroes Y and adds each cell's result box with a bulk reduce).
 * X, Y: device, num_dofs x n_vec, dtype of the current mode, X != Y (no
 * overlap).  Y is overwritten, never accumulated.  Asynchronous on stream.
 * On a refined mesh with hanging nodes the product first distributes X into a
 * context-owned device block of X's size (X with the slave rows filled in);
 * the first call with a given or larger n_vec allocates that block
 * (cudaMalloc, which synchronises the device), later calls reuse it.
 * fe_apply_host_noalloc takes the block from its fixed array instead. */
fe_status fe_apply(fe_ctx* ctx, const void* X, void* Y, int n_vec, void* stream);

/* Launch shape of the CUDA-core cell kernels of one mode (the autotuner's
 * knob): vectors per CTA (power of two, 1..32; halved further when shared
 * memory does not hold it, and never above the padded n_vec), lines in flight
 * per CTA (1..256; CTAs are capped at 256 threads), and the variant
 * (FE_FP64: 0 = line kernel with even-odd contractions, 1 = plain line
 * kernel; FE_FP32: 0 or 1 = line kernel, 2 = register-plane kernel, n_q <= 8
 * only, 3 = line kernel with even-odd contractions; FE_DF64: 0, the
 * double-float even-odd line kernel).
 * FE_TF32 / FE_BF16 / FE_BF16S (one setting for the three): the tile is
 * fixed; variant 0 = tcgen05 kernel where built (n_p, n_q <= 8), moving each
 * cell's values with TMA boxes when X and Y are 16-byte aligned and a node's
 * n_vec values fill whole 16-byte units (n_vec >= 8, a multiple of 4 for
 * FP32 storage and of 8 for BF16 storage), else with per-thread loads and
 * stores; 1 = warp-level MMA kernel (FE_TF32 / FE_BF16 only); 2 = tcgen05
 * kernel with per-thread loads and stores always (the other arguments are
 * ignored).  FE_TF32X3: FE_EUNSUPPORTED.  Applies to later fe_apply calls. */
fe_status fe_set_tile(fe_ctx* ctx, fe_mode mode, int vectors_per_cta, int lines, int variant);

/* Same product with HOST buffers (num_dofs x n_vec, DoF-major, in the
 * context's element type); synchronises `stream` before returning.
 * FE_FP64 with both buffers page-locked and device-mapped (cudaHostAlloc,
 * cudaHostRegister, torch pin_memory): the cell kernels read X_host and write
 * Y_host in place over the host link (NVLink-C2C on GB300); the FP64
 * product's arithmetic hides the link traffic, so no staging copy is made.
 * Otherwise: copies X_host to library-owned device staging
 * memory, applies, copies the result to Y_host.  A block of at least two 128-byte column chunks (32 FP64
 * or 64 FP32 vectors) is pipelined: chunks of 16 (FP64) or 32 (FP32) columns
 * are copied in and out by strided copies on two library-owned streams while
 * the previous chunk is applied on `stream`, so the link transfers hide under
 * the product; each column's result is bitwise that of fe_apply on the whole
 * block.  Pinned host buffers give asynchronous DMA.  The staging memory (4
 * chunks, or X and Y for a narrow block), the streams and the events stay in
 * the context for reuse; concurrent calls on one context race. */
fe_status fe_apply_host(fe_ctx* ctx, const void* X_host, void* Y_host, int n_vec, void* stream);

/* Size of the fixed device staging array of fe_apply_host_noalloc (16 MiB). */
#define FE_NOALLOC_STAGE_BYTES ((size_t)16 << 20)

/* fe_apply_host for callers that cannot let a library allocate device memory
 * -- a process whose memory manager reserves the whole GPU up front, a
 * real-time loop that must never block in the allocator, or an application
 * held to a fixed, pre-measured memory budget.  (The paper has no
 * counterpart; it is a deployment variant of fe_apply_host.)  Same contract
 * as fe_apply_host, but the device staging of X and Y lives in one
 * file-scope device array of FE_NOALLOC_STAGE_BYTES that every GPU loading
 * the library holds until the process exits; the call itself performs no
 * cudaMalloc, cudaFree or other allocation.  Limits and caveats:
 *  - the staged blocks must fit in FE_NOALLOC_STAGE_BYTES, else FE_EINVAL
 *    before any copy: with b = num_dofs * n_vec * sizeof(element) and
 *    b' = b rounded up to 256 bytes, b' + b for X and Y, and 2 b' + b on a
 *    refined mesh with hanging nodes (fe_setup_refined), whose product also
 *    stages a copy of X with the slave rows filled in;
 *  - modes fe_apply rejects on the context are rejected with the same status;
 *    if the product fails after the copy of X_host was queued, the call
 *    synchronises `stream` before returning, so no copy is left in flight;
 *  - the first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress with that device current) and caches it; make
 *    that first call before any stream capture;
 *  - every call shares the one array: calls that overlap on the GPU (other
 *    streams, other threads, other contexts on the same device) race and
 *    must be serialised by the caller.  Nothing in the array needs to start
 *    at zero: X is copied in whole and Y written whole on every call. */
fe_status fe_apply_host_noalloc(fe_ctx* ctx, const void* X_host, void* Y_host, int n_vec, void* stream);

/* FE_NOALLOC_STAGE_BYTES as compiled into the library (the size of the fixed
 * staging array of fe_apply_host_noalloc). */
size_t fe_noalloc_stage_bytes(void);

/* diag(A) as a device FP64 vector of num_dofs entries (constrained rows get 1,
 * the convention of the Jacobi preconditioner), computed matrix-free from the
 * same tables: A_II = sum over cells containing I of A^(e)_ii. */
fe_status fe_diagonal(fe_ctx* ctx, double* diag, void* stream);

/* Preconditioners of fe_solve. */
typedef enum { FE_PRECOND_NONE = 0, FE_PRECOND_JACOBI = 1, FE_PRECOND_LEARNED = 2 } fe_precond;

typedef struct {
  int iterations;          /* CG iterations (all inner iterations under refinement) */
  int outer_iterations;    /* refinement steps (0 when inner_mode == FE_FP64) */
  int fp64_applies;        /* applications of the FP64 operator */
  int converged_columns;   /* columns with FP64 relative residual <= rtol */
  double max_rel_residual; /* max_j ||b_j - A x_j|| / ||b_j||, FP64 operator */
  double seconds;          /* device time of the whole solve (CUDA events) */
} fe_solve_info;

/* Solve A X = B for n_vec right-hand sides by block preconditioned conjugate
 * gradients: one CG recurrence per column, all columns advanced together
 * (the block Krylov setting the paper names for many right-hand sides; the
 * operator is the matrix-free product of fe_apply).  B, X: device FP64,
 * num_dofs x n_vec, DoF-major; X holds the initial guess on entry and the
 * solution on return.  For a Dirichlet box B's boundary rows should be 0 and
 * X's boundary rows stay 0.
 *   inner_mode == FE_FP64: PCG in FP64.
 *   inner_mode == FE_DF64: PCG in FP64 with the double-float operator
 *   (FE_DF64); the FP64 operator checks the result.
 *   otherwise (FE_FP32/TF32/BF16/TF32X3): FP64 iterative refinement -- r = B - A X with the FP64
 *   operator, an inner PCG in inner_mode (FP32 data; FE_FP32/TF32/BF16/TF32X3
 *   operator) on r / ||r|| to the relative reduction still needed
 *   (rtol ||b|| / (2 ||r||), at least 2e-6), X += ||r|| D -- until every
 *   column reaches rtol.
 * precond: FE_PRECOND_JACOBI (diag(A)^-1 from fe_diagonal), FE_PRECOND_NONE,
 * or FE_PRECOND_LEARNED (the trained cell-patch network, see fe_learn.h;
 * flexible CG, with FE_EINVAL when no network is loaded).
 * Stops after max_it iterations.  Every final residual is measured with the
 * FP64 operator; returns FE_ENOTCONV (with X and info filled) if a column
 * misses rtol, FE_EBREAKDOWN if p^T A p <= 0 on an active column.
 * info (host, optional) and rel_res (host, optional, n_vec doubles: the final
 * FP64 relative residual of each column) are written on return.  Workspace
 * (device) is allocated on first use and kept in the context.  Synchronous
 * with respect to the host. */
fe_status fe_solve(fe_ctx* ctx, const double* B, double* X, int n_vec, double rtol, int max_it, int precond,
                   int inner_mode, fe_solve_info* info, double* rel_res, void* stream);

/* Status word written by asynchronous device work (non-finite values met,
 * bounded waits that gave up); reading it synchronises the context's work and
 * clears it. */
fe_status fe_last_device_status(fe_ctx* ctx);

const char* fe_status_str(fe_status s);

/* Name of the CUDA runtime error (cudaGetErrorName, e.g.
 * "cudaErrorInvalidValue") behind the most recent FE_ECUDA or FE_ENOMEM that
 * any call of this library returned on the calling host thread, followed by
 * the step that met it where the library names one ("... in <step>"), or
 * "none".  Reading it does not clear it; the string belongs to the library
 * and stays valid until the thread's next failing call. */
const char* fe_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FE_H_ */
