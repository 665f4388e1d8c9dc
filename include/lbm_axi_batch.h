/*
 * lbm_axi_batch.h — batched stepping and autotuning on top of lbm_axi.h.
 *
 * Many independent solves (e.g. droplets of different sizes, temperatures and
 * relaxation times) advance together: each batch step is ONE launch of the
 * fused step kernel over a work list of tiles -- row ranges of the solves'
 * z-strips -- dealt to the CTAs by lbm_axi_tile_plan; steps are replayed from
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

/* strip: z-columns per CTA, 64 or 112; grid: CTA slots the tiles are dealt to,
 * 0 = one wave of resident CTAs. */
typedef struct {
    int strip;
    int grid;
} lbm_axi_batch_tuning;

/* Group n >= 1 solves.  Every solve must be created on the current device,
 * initialised, with nr >= 16, EDM forcing and h_i at the node (the batched
 * kernel has neither the Guo nor the link-source form), the same precision and
 * the same multiphase / axis_terms switches; a solve may appear once.  The batch
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
 * 64 / 112 x tiles dealt to one or two resident waves) on this batch, keep the
 * fastest and return it in *chosen (may be NULL).  Non-destructive: trial
 * launches read the current populations and write only the buffer the next
 * step overwrites; error words raised by trials are cleared.  Synchronous. */
int lbm_axi_batch_autotune(lbm_axi_batch* b, int trials, lbm_axi_batch_tuning* chosen);

/* Autotuner for a single solve: times the fused path at rows_per_cta in
 * {0 (balanced wave), 32, 64, 144, 256} and the split path, keeps the fastest
 * (set as the solve's tuning) and returns it in *chosen (may be NULL).
 * Non-destructive like lbm_axi_batch_autotune.  Synchronous. */
int lbm_axi_autotune(lbm_axi* h, int trials, lbm_axi_tuning* chosen);

/* Work plan of a batched launch (performance only; no counterpart in the
 * paper).  Every solve's (z-strip, row) space -- strip columns per strip,
 * ceil(nz[i] / strip) strips -- is cut into tiles, rows [j0, jend) of one strip
 * of one solve, and the tiles are dealt to `slots` CTAs, largest first, each to
 * the CTA with the least work so far; a CTA marches its tiles one after
 * another.  A tile costs its rows plus 18 rows of pipeline fill (6 halo rows
 * above it and the 12-row lag between the kernel's first and last stage); of
 * the candidate cuts (whole strips, or the smallest chunk height of at least
 * 16 rows that fills 1..4 waves of slots) the one with the smallest largest
 * CTA cost is kept.  A single solve is planned the same way (wide strips, one
 * wave).  Host-only, no GPU.
 *   nz, nr: n >= 1 grid sizes (host arrays); strip >= 1; slots >= 1;
 *   tiles_out: 4 ints per tile (solve, strip, j0, jend), grouped by CTA,
 *   max_tiles of room; first_out: the tiles of CTA c are first_out[c] ..
 *   first_out[c + 1] - 1 (room for slots + 1 ints); *ntiles: tiles; *ncta: CTAs
 *   with work (first_out[*ncta] = *ntiles); *makespan (may be NULL): the
 *   largest CTA cost in rows.
 * Returns LBM_ERR_INVALID_ARG for bad sizes, NULL outputs, or max_tiles too
 * small (then *ntiles and *ncta still hold the counts needed). */
int lbm_axi_tile_plan(const int* nz, const int* nr, int n, int strip, int slots, int max_tiles, int* tiles_out,
                      int* first_out, int* ntiles, int* ncta, long long* makespan);

/* Release the batch (waits for its stream).  The solves remain valid and keep
 * the state the batch left them in. */
void lbm_axi_batch_destroy(lbm_axi_batch* b);

#ifdef __cplusplus
}
#endif

#endif /* LBM_AXI_BATCH_H */
