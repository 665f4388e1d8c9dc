/*
 * lbm_axi_batch.h — batched stepping and autotuning on top of lbm_axi.h.
 *
 * Many independent solves (e.g. droplets of different sizes, temperatures and
 * relaxation times) advance together: each batch step is ONE launch of the
 * fused step kernel over a concatenation of all solves' (z-strip, row)
 * spaces, cut into equal shares for a one-wave grid; steps are replayed from
 * a CUDA graph.  The update of every solve is exactly the single-solve update
 * (Sec. II of arXiv:1512.01977); no arithmetic couples two solves, so a
 * solve's result is the same alone and in any batch.
 */
#ifndef LBM_AXI_BATCH_H
#define LBM_AXI_BATCH_H

#include "lbm_axi.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_axi_batch lbm_axi_batch;

/* strip: z-columns per CTA, 64 or 96; grid: CTAs per launch, 0 = one wave of
 * resident CTAs. */
typedef struct {
    int strip;
    int grid;
} lbm_axi_batch_tuning;

/* Group n >= 1 solves.  Every solve must be created on the current device,
 * initialised, on the fused path (nr >= 16), with the same precision and the
 * same multiphase / axis_terms switches; a solve may appear once.  The batch
 * borrows the solves: while it exists they must not be stepped, initialised or
 * destroyed through their own handles; their moments and mass may be read
 * after lbm_axi_batch_sync.  stream: a cudaStream_t for the batch's work, or
 * NULL for a stream the batch creates.  Allocates small device tables (about
 * 150 B per solve).  LBM_ERR_INVALID_ARG for a requirement not met. */
int lbm_axi_batch_create(lbm_axi* const* solves, int n, void* stream, lbm_axi_batch** out);

/* Advance every solve by nsteps >= 0 and wait.  Returns LBM_ERR_UNPHYSICAL if
 * any solve met rho <= 0, psi^2 < 0 or a non-finite value (per-solve detail in
 * lbm_axi_batch_status); the other solves are unaffected. */
int lbm_axi_batch_step(lbm_axi_batch* b, long long nsteps);

/* Enqueue nsteps without waiting; lbm_axi_batch_sync waits and returns the
 * status of the steps enqueued since the previous sync. */
int lbm_axi_batch_step_async(lbm_axi_batch* b, long long nsteps);
int lbm_axi_batch_sync(lbm_axi_batch* b);

/* status[i] = LBM_OK or LBM_ERR_UNPHYSICAL for solve i, accumulated since the
 * batch was created (sticky: a failed solve stays failed).  Waits for the stream. */
int lbm_axi_batch_status(lbm_axi_batch* b, int* status);

/* Steps taken by the batch so far. */
int lbm_axi_batch_steps(const lbm_axi_batch* b, long long* steps);

int lbm_axi_batch_get_tuning(const lbm_axi_batch* b, lbm_axi_batch_tuning* t);
int lbm_axi_batch_set_tuning(lbm_axi_batch* b, const lbm_axi_batch_tuning* t);

/* Autotuner: time `trials` launches of every candidate configuration (strip
 * 64 / 96 x grid of one or two resident waves) on this batch, keep the
 * fastest and return it in *chosen (may be NULL).  Non-destructive: trial
 * launches read the current populations and write only the buffer the next
 * step overwrites; error words raised by trials are cleared.  Synchronous. */
int lbm_axi_batch_autotune(lbm_axi_batch* b, int trials, lbm_axi_batch_tuning* chosen);

/* Autotuner for a single solve: times the fused path at rows_per_cta in
 * {0 (balanced wave), 32, 64, 144, 256} and the split path, keeps the fastest
 * (set as the solve's tuning) and returns it in *chosen (may be NULL).
 * Non-destructive like lbm_axi_batch_autotune.  Synchronous. */
int lbm_axi_autotune(lbm_axi* h, int trials, lbm_axi_tuning* chosen);

/* Release the batch (waits for its stream).  The solves remain valid and keep
 * the state the batch left them in. */
void lbm_axi_batch_destroy(lbm_axi_batch* b);

#ifdef __cplusplus
}
#endif

#endif /* LBM_AXI_BATCH_H */
