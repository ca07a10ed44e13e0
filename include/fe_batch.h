/*
 * fe_batch.h -- many operators applied in one persistent launch (see fe.h).
 *
 * The paper evaluates all cells and all vector batches of one operator
 * concurrently in a single kernel launch (Sec. 3.1.2, GPU batched strategy);
 * this call extends that to a batch of independent operators of different
 * size, degree and block width.  One persistent kernel takes work items
 * (problem, cell colour, range of cells, vector block) from a queue ordered
 * by colour phase; an item of colour k waits (bounded) until its problem's
 * colour k-1 items are done, so assembly stays conflict-free and every Y is
 * bitwise the one fe_apply produces.  The kernel and the reset of its queue
 * are captured once in a CUDA graph; each fe_batch_apply replays it.
 */
#ifndef FE_BATCH_H_
#define FE_BATCH_H_

#include "fe.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fe_batch fe_batch;

typedef struct {
  int problems;
  int work_items;
  int phases;           /* colour phases of the queue */
  int grid;             /* persistent CTAs */
  long long smem_bytes; /* dynamic shared memory per CTA */
  float autotune_ms;    /* device time spent timing candidate tiles */
  int device_status;    /* FE_ETIMEOUT if a bounded wait gave up during an apply since
                           the last fe_batch_stats, else 0 (cleared by the read) */
} fe_batch_info;

/* Plan a batch over n contexts (each a degree 3..8 operator with n_q = p + 2
 * on affine cells of a structured mesh; FE_EUNSUPPORTED otherwise) with
 * fixed block widths n_vec[i] > 0 (host array), in mode FE_FP64, FE_DF64
 * (FP64 data, double-float arithmetic) or FE_FP32.  Every work item runs the
 * cell body of the mode's default per-colour kernel, so results equal
 * fe_apply's bit for bit.  FE_FP64 runs one persistent kernel over all
 * problems; FE_DF64 and FE_FP32 run one persistent kernel per degree (its
 * tables as kernel parameters, its own queue) as parallel branches of the
 * graph.  All problems of one degree must use the same quadrature rule.  With autotune != 0 the vectors per work item of
 * every (degree, block-width bucket) are chosen by timing the candidates on
 * an 8^3 periodic proxy mesh (at most 64 vectors); otherwise a fixed rule is
 * used.  The contexts must outlive the batch.  Synchronous. */
fe_status fe_batch_create(fe_ctx* const* ctxs, int n, const int* n_vec, fe_mode mode, int autotune, fe_batch** out);

/* Y[i] = A_i X[i] for every problem: X, Y host arrays of n device pointers
 * (dtype of the batch's mode, num_dofs_i x n_vec[i], X[i] != Y[i]).  Waits
 * for earlier work on `stream`, uploads the pointer table and replays the
 * graph on `stream` (asynchronous from there). */
fe_status fe_batch_apply(fe_batch* b, const void* const* X, void* const* Y, void* stream);

/* Plan statistics; vectors_per_cta / cells_per_item (optional, n entries)
 * receive each problem's tile.  Synchronises the device, then reads and
 * clears the batch's device status word.  Synchronous. */
fe_status fe_batch_stats(const fe_batch* b, fe_batch_info* info, int* vectors_per_cta, int* cells_per_item);

/* Limit of every bounded wait of the batch kernels (an item of colour k
 * waiting for its problem's colour k-1 items), in seconds (default 10).  A
 * wait that runs out records FE_ETIMEOUT in the device status word
 * (fe_batch_stats) and lets its item proceed, so the launch always ends and
 * the context stays usable; the results of that apply are then not valid.
 * Takes effect from the next fe_batch_apply.  Synchronous. */
fe_status fe_batch_set_wait_limit(fe_batch* b, double seconds);

/* For exercising the bounded waits (fault injection on the host, no device
 * fault): hold != 0 makes the items of colour color + 1 of problem `problem`
 * wait for a completion count that colour `color` never reaches, so each of
 * those waits runs out; hold = 0 restores the true count.  FE_EINVAL when
 * the problem has no item of colour `color`.  Synchronous. */
fe_status fe_batch_hold_color(fe_batch* b, int problem, int color, int hold);

void fe_batch_destroy(fe_batch* b);

#ifdef __cplusplus
}
#endif

#endif /* FE_BATCH_H_ */
