/*
 * fe_learn.h -- learned cell-patch preconditioner of libfe (see fe.h).
 *
 * The paper has no learned component; this layer sits on top of its operator
 * (Sec. 2.2) and of the block Krylov solve (fe_solve).  The preconditioner is
 *
 *   z = D^-1 r + sum_e R_e^T ( w_e .* s_e MLP(R_e r / s_e) ),
 *   MLP(u) = W2 relu(W1 u + b1) + b2,
 *
 * with R_e the gather of the n3 = (p+1)^3 nodes of cell e (Dirichlet nodes read
 * as 0), s_e = ||R_e r|| per cell and column, w_e the partition-of-unity
 * weights 1 / (number of cells sharing the node), D = diag(A).  W1 is
 * 128 x n3 (row-major), b1 128, W2 n3 x 128 (row-major), b2 n3.  Inference
 * runs the two layers on tensor cores (BF16 weights and inputs, FP32
 * accumulation, hidden activations rounded to BF16); training runs in FP32.
 * Inference supports p <= 6 (n3 <= 343).
 */
#ifndef FE_LEARN_H_
#define FE_LEARN_H_

#include "fe.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Training objectives. */
typedef enum {
  /* mean over residual snapshots and columns (r scaled to norm 1) of
     ||A z(r) - r||^2:
     the network learns to make A z close to r; the gradient runs through the
     operator itself */
  FE_TRAIN_OPERATOR_RESIDUAL = 0,
  /* patch regression onto the oscillatory part of the error (see below) */
  FE_TRAIN_PATCH_ERROR = 1,
  /* mean over snapshots and columns of (e - z(r))^T A (e - z(r)), e = x* - x_k,
     both r and e scaled per column by 1 / ||e||_A = 1 / sqrt(e^T r): the
     relative energy norm of the error a preconditioned step leaves, the norm
     CG minimises */
  FE_TRAIN_ENERGY = 2
} fe_train_objective;

typedef struct {
  int n_rhs;               /* right-hand sides ~ N(0,1) of the training trajectories */
  int snapshots;           /* (r_k, x_k) snapshots recorded per trajectory, k = 0, every, 2 every, ... */
  int snapshot_every;      /* PCG iterations between snapshots */
  int epochs;              /* passes over the samples */
  int batch;               /* samples per Adam step */
  float lr;                /* Adam learning rate */
  double traj_rtol;        /* relative residual of the trajectory solve that gives x* */
  unsigned long long seed; /* seeds the right-hand sides, the initial weights and the shuffling */
  int objective;           /* fe_train_objective */
  int n_val;               /* held-out right-hand sides for checkpoint selection (0: keep the last epoch) */
} fe_train_desc;

typedef struct {
  long long samples;         /* (cell, column, snapshot) patches in the training set */
  int steps;                 /* Adam steps taken */
  int trajectory_iterations; /* Jacobi-PCG iterations of the trajectory solve */
  float loss_first_step;     /* MSE of the first mini-batch */
  float loss_first_epoch;    /* mean MSE over the first epoch */
  float loss_last_epoch;     /* mean MSE over the last epoch */
  double seconds;            /* device time, data generation included */
  int val_jacobi_iterations; /* FP32 PCG iterations to 1e-7 on the held-out columns, Jacobi */
  int val_learned_iterations;/* the same with the kept checkpoint (the Jacobi count when none beat it) */
  int best_epoch;            /* epoch of the kept checkpoint; 0 = zero output layer (Jacobi) */
  float val_loss_jacobi;     /* training objective on the held-out snapshots, Jacobi (zero output layer) */
  float val_loss_kept;       /* the same for the kept network */
} fe_train_info;

/* Random initial weights (W1 ~ U(+-1/sqrt(n3)), W2 ~ U(+-1e-3/sqrt(128)),
 * biases 0), seeded.  Synchronous. */
fe_status fe_precond_init(fe_ctx* ctx, unsigned long long seed);

/* Train on the residual / error trajectory of an FP32 Jacobi-PCG solve of this
 * operator (n_rhs random right-hand sides, snapshots (r_k, x_k) every
 * snapshot_every iterations, x* = the converged solution), with Adam:
 *  FE_TRAIN_ENERGY: one snapshot per step, loss mean over columns of
 *    (e_k - z)^T A (e_k - z)
 *    with z = z(r_k) over all cells' patches at once (one FP32 operator
 *    application per step, which also gives the gradient 2 A (z - e_k));
 *  FE_TRAIN_OPERATOR_RESIDUAL: one snapshot r_k per step, loss
 *    mean (A z(r_k) - r_k)^2 over all cells' patches at once (two FP32
 *    operator applications per step: A z and the gradient A (A z - r));
 *  With n_val > 0 (operator objectives), n_val held-out random right-hand
 *  sides are solved once by FP32 Jacobi-PCG to 1e-7 (its iteration count and
 *  solution x*), recording up to four held-out snapshots spread over the
 *  iterations the training snapshots span.  After every epoch the objective
 *  is evaluated on those snapshots; "epoch 0" is the network with its output
 *  layer set to zero, i.e. exactly Jacobi.  The epoch of the lowest held-out
 *  loss (when it is not epoch 0) and the last epoch are then tried, in that
 *  order, by one FP32 PCG solve of the held-out right-hand sides each: the
 *  first that needs fewer iterations than Jacobi is kept, otherwise the
 *  output layer is set to zero (Jacobi).  The kept network never needs more
 *  validation iterations than Jacobi.
 *  FE_TRAIN_PATCH_ERROR: inputs R_e r_k / s_e, targets
 *    HF(R_e(x* - x_k - D^-1 r_k)) / s_e, HF subtracting the trilinear
 *    interpolant of the patch's eight corner values, mini-batches of `batch`
 *    patches, mean squared error.  Initialises the weights first when none are set.
 * Device memory for the samples is allocated for the call and released.
 * info (host, optional) receives the statistics.  Synchronous. */
fe_status fe_precond_train(fe_ctx* ctx, const fe_train_desc* desc, fe_train_info* info, void* stream);

/* z = preconditioner(r) for n_vec columns: R, Z device FP32 num_dofs x n_vec,
 * DoF-major, distinct.  FE_EINVAL when no weights are set.  Asynchronous. */
fe_status fe_precond_apply(fe_ctx* ctx, const float* R, float* Z, int n_vec, void* stream);

/* Host FP32 weights in / out (layouts above).  Synchronous. */
fe_status fe_precond_set_weights(fe_ctx* ctx, const float* W1, const float* b1, const float* W2, const float* b2);
fe_status fe_precond_get_weights(const fe_ctx* ctx, float* W1, float* b1, float* W2, float* b2);
int fe_precond_input_size(const fe_ctx* ctx);   /* n3 = (p+1)^3 */

/* Weights to / from a file (little-endian header "FEPL", version, n3, 128,
 * then W1, b1, W2, b2 as FP32).  FE_EINVAL on I/O errors or a size mismatch. */
fe_status fe_precond_save(const fe_ctx* ctx, const char* path);
fe_status fe_precond_load(fe_ctx* ctx, const char* path);

/* Loss and gradients of the training objective for one batch (the training
 * kernels, exposed for checking): U, T device FP32 rows x n3 (inputs,
 * targets); writes the mean squared error to *loss and dL/dW1, dL/db1, dL/dW2,
 * dL/db2 to device buffers of the weight shapes.  Synchronous. */
fe_status fe_mlp_gradients(fe_ctx* ctx, const float* U, const float* T, int rows, float* loss, float* gW1,
                           float* gb1, float* gW2, float* gb2, void* stream);

/* Loss and gradients of the FE_TRAIN_ENERGY objective on one snapshot, as
 * one training step computes them (the training kernels, exposed for
 * checking).  R = r_k, Xk = x_k, Xstar = x* (device FP32, num_dofs x n_vec,
 * DoF-major; r_k = A (x* - x_k) for a snapshot of a solve, though any blocks
 * are accepted): every column is scaled by c_j = 1 / sqrt((x* - x_k)_j . r_j)
 * (1 / ||r_j|| when that product is not positive), r' = c r, e' = c (x* - x_k),
 * z = D^-1 r' + sum_e R_e^T (w_e .* s_e MLP(R_e r' / s_e)) with the current
 * network, and
 *   loss = (1 / n_vec) sum_j (z - e')_j^T A (z - e')_j
 * with the FP32 operator.  Writes the loss to *loss (device) and dL/dW1,
 * dL/db1, dL/dW2, dL/db2 to device buffers of the weight shapes (s_e depends
 * on r alone, so it carries no gradient).  FE_EINVAL when no weights are set.
 * Allocates its workspace for the call.  Synchronous. */
fe_status fe_energy_gradients(fe_ctx* ctx, const float* R, const float* Xk, const float* Xstar, int n_vec,
                              float* loss, float* gW1, float* gb1, float* gW2, float* gb2, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FE_LEARN_H_ */
