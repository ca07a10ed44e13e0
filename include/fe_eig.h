/* libfe eigenvalue layer: the Helmholtz eigenproblem of Sec. 4.3 of
 * arXiv 2208.07129 solved by Chebyshev-filtered subspace iteration
 * (Algorithm 6), on top of the matrix-free operator of fe.h.
 *
 * The generalised problem H U = M U Lambda (H = the operator A of fe.h, M the
 * overlap matrix) becomes the standard problem H~ U~ = U~ Lambda with
 * H~ = M^-1/2 H M^-1/2 and U~ = M^1/2 U.  M is integrated with the GLL rule
 * on the element's own n_p nodes, which makes it diagonal (Sec. 4.3).
 * Dirichlet boxes: H~ acts on the free (interior) nodes; constrained rows of
 * every result are 0.
 *
 * Layouts as in fe.h: blocks are num_dofs x n_vec, DoF-major
 * (X[dof * n_vec + v]), in the element type of the context's mode.  Device
 * pointers are caller-owned; calls are asynchronous on `stream` unless stated
 * otherwise.  No call aborts; errors are fe_status codes.
 */
#ifndef FE_EIG_H_
#define FE_EIG_H_

#include "fe.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Diagonal of the GLL-integrated overlap matrix,
 *   m_I = sum over cells e containing node I of w_i w_j w_k det J_e(node),
 * with w the (p+1)-point GLL weights on [-1, 1] and det J the Jacobian of the
 * cell map at the node (Sec. 4.3).  Host FP64, num_dofs values; constrained
 * rows get 1.  Computed on the host once per context (also by the calls
 * below) and kept.  Synchronous. */
fe_status fe_mass_gll(fe_ctx* ctx, double* m_host);

/* The fused product of the paper's ChFSI kernel,
 *   Y = a M^-1/2 A M^-1/2 X + b X + c Y,
 * with the M^-1/2 scalings folded into the gather and the scatter and the
 * b X + c Y terms into the first write of each node (colour-ordered
 * assembly), so the product costs one pass over X and Y like fe_apply.
 * Mode FE_FP64 (even-odd cell kernel), FE_DF64 (FP64 data, double-float
 * arithmetic) or FE_FP32 (even-odd line kernel in FP32); the tensor-core
 * modes return FE_EUNSUPPORTED.  X and Y must not overlap.  Y is
 * read only when c != 0 (it may be uninitialised when c == 0).  Constrained
 * rows of Y are written 0. */
fe_status fe_apply_scaled(fe_ctx* ctx, const void* X, void* Y, int n_vec, double a, double b, double c,
                          void* stream);

/* The filter loop of Algorithm 6: X <- p_m(H~) X, where p_m is the degree-m
 * Chebyshev polynomial that damps [lambda_u, lambda_max] and equals 1 at
 * lambda_min (scaled three-term recurrence; sigma is updated after every
 * step).  m scaled products; the block ends in X, Y is scratch of the same
 * size.  Requires lambda_min < lambda_u < lambda_max (else FE_EINVAL) and
 * degree >= 1.  Element type per the context's mode (FE_FP64, FE_DF64 or
 * FE_FP32). */
fe_status fe_chebyshev_filter(fe_ctx* ctx, void* X, void* Y, int n_vec, int degree, double lambda_min,
                              double lambda_u, double lambda_max, void* stream);

typedef struct {
  int n_wanted;        /* pairs whose residual decides convergence, 1 <= n_wanted <= k */
  int degree;          /* Chebyshev degree m of each filter pass, >= 1 */
  double tol;          /* stop when max_{j < n_wanted} ||H~ u_j - lambda_j u_j||_2 <= tol */
  int max_iter;        /* filter + orthonormalise + Rayleigh-Ritz rounds, >= 1 */
  int lanczos_steps;   /* Lanczos steps bounding the spectrum (upper bound of H~), >= 2 */
  int filter_mode;     /* arithmetic of the scaled products (filter, projection, Lanczos):
                          FE_FP64: FP64 throughout;
                          FE_DF64: FP64 data, double-float products (FE_DF64 of fe.h);
                          FE_FP32: whole rounds (filter, Cholesky QR, Rayleigh-Ritz) in FP32 while the
                          wanted residual is above fp32_switch, then FP64 rounds with double-float
                          products.  FP64 rounds always decide convergence. */
  double fp32_switch;  /* residual below which an FE_FP32 run switches to FP64 rounds; keep it above
                          ~1e-6 x the largest wanted eigenvalue (the FP32 residual floor) */
  unsigned long long seed;  /* Lanczos start vector */
} fe_chfsi_desc;

typedef struct {
  int iterations;           /* rounds done */
  int filter_applies;       /* scaled products inside filter passes */
  int fp32_passes;          /* filter passes run in FP32 */
  int converged;            /* wanted pairs with residual <= tol */
  double max_residual;      /* max residual over the wanted pairs */
  double lambda_min, lambda_u, lambda_max;  /* bounds used by the last filter pass */
  double seconds;           /* device time of the whole call (CUDA events) */
  double seconds_filter, seconds_orth, seconds_rr;
} fe_chfsi_info;

/* Chebyshev-filtered subspace iteration (Algorithm 6) for the k smallest
 * eigenpairs of H~ (the context's FP64 operator).
 *   U: device FP64 num_dofs x k; in: a full-rank start block (random is
 *      fine); out: orthonormal Ritz vectors u_j of H~ (constrained rows 0).
 *      The eigenvectors of H U = M U Lambda are M^-1/2 u_j.
 *   lambda (host, k doubles, ascending) and residual (host, k doubles:
 *      ||H~ u_j - lambda_j u_j||_2): outputs, may be NULL.
 * Steps: a Lanczos run bounds the spectrum from above (largest Ritz value
 * plus the last off-diagonal); the start block is orthonormalised and
 * Rayleigh-Ritz projected; then each round filters U over
 * [lambda_u, lambda_max] normalised at lambda_min (lambda_u, lambda_min = the
 * largest and smallest current Ritz values), orthonormalises it (Cholesky QR,
 * twice, with a diagonal shift if the Gram matrix is not numerically
 * positive definite), and projects: W = H~ U, P = U^T W, P = Q Lambda Q^T,
 * U <- U Q, then W = H~ U again and the residuals from W - U Lambda.  The
 * dense steps use cuBLAS (Gram matrices, rotations, triangular solves) and
 * cuSOLVER (Cholesky, the k x k symmetric eigensolver).
 * Workspace: two more num_dofs x k FP64 blocks (and three FP32 blocks when
 * filter_mode is FE_FP32), allocated for the call.  Synchronous: returns
 * when the results are on the host.  FE_ENOTCONV if max_iter rounds end
 * above tol (U, lambda, residual still filled); FE_ENONFINITE on a
 * non-finite Ritz value.  k >= 2 and k <= the free DoFs. */
fe_status fe_chfsi(fe_ctx* ctx, double* U, int k, const fe_chfsi_desc* desc, double* lambda, double* residual,
                   fe_chfsi_info* info, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FE_EIG_H_ */
