/*
 * dg_batch.h -- batched ensembles of independent DG shallow-water /
 * regularized-Bingham instances advanced together on one GPU.
 *
 * Each instance has its own mesh, order, regularization and parameters
 * (dg_swe.h types).  Instances are grouped by (dimension, order, wet/dry mode
 * dg_swe_params.positivity); every group
 * stores its instances' elements and faces contiguously ([field][element]
 * [node] over the group), so one launch per group and phase (E-step, face
 * flux, volume/lift/mass-solve/update) advances all of them.  Per-instance
 * physical parameters, boundary tables and scalar blocks (dt, t, steps,
 * mass) live in small device tables indexed through an element-to-instance
 * map; the stable step and the mass are FP64 reductions per instance (one
 * block per instance, deterministic order).  Steps are replayed from a CUDA
 * graph.  Thread-block sizes per group and kernel are chosen by
 * dg_batch_autotune (timed on the device) or set explicitly.
 *
 * The method per instance is exactly that of dg_swe.h (Sec. 5 of the paper,
 * Eq. WeakForm51/52, explicit SSP-RK3); a batched instance produces the same
 * state as the same instance run alone (tested bit for bit in FP64).
 * Conventions (status codes, workspace, streams) are those of dg_swe.h.
 */
#ifndef DG_BATCH_H
#define DG_BATCH_H

#include "dg_swe.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dg_batch dg_batch;

/* n instances: meshes[i], orders[i] (1..3), regs[i] (DG_REG_*), params[i].
 * All instances must use the same precision (params[i].precision).  Host
 * inputs are copied.  DG_ERR_ARG on any invalid instance (the message names it). */
dg_status dg_batch_init(int n, const dg_swe_mesh *meshes, const int *orders, const int *regs,
                        const dg_swe_params *params, dg_batch **out);

size_t dg_batch_workspace_size(const dg_batch *b);
/* 256-byte aligned device workspace owned by the caller; uploads geometry. */
dg_status dg_batch_set_workspace(dg_batch *b, void *dev_ptr, size_t bytes);
dg_status dg_batch_set_stream(dg_batch *b, void *cuda_stream);

/* Instance i's nodal state [nV][K_i][Np_i] (doubles, device or host) and its
 * time/step/mass reference reset. */
dg_status dg_batch_set_state(dg_batch *b, int i, const double *V, int on_device);
/* Copies instance i's state out; synchronizes; reports latched device errors. */
dg_status dg_batch_get_state(dg_batch *b, int i, double *V, int on_device);

/* Enqueue n_steps SSP-RK3 steps of every instance (each with its own
 * CFL-limited step), replayed from a CUDA graph captured on first use. */
dg_status dg_batch_advance(dg_batch *b, int64_t n_steps);
/* dg_batch_advance + per-instance mass reduction + synchronize; stats[n] may be NULL.
 * A latched device status of an instance is returned with its index in the
 * message: DG_ERR_NONFINITE (non-finite state) or DG_ERR_TIMEOUT (a bounded
 * wait of the staged volume kernel for its bulk copies ran out). */
dg_status dg_batch_run(dg_batch *b, int64_t n_steps, dg_swe_stats *stats);
/* Mass reduction + synchronize; fills stats[n]; reports latched statuses as
 * dg_batch_run does. */
dg_status dg_batch_stats(dg_batch *b, dg_swe_stats *stats);

/* Autotuner: for every group and each of the three stage kernels, times
 * thread-block sizes T in {32, 64, 128, 256} on the current state (n_iter
 * launches each, CUDA events) and keeps the fastest.  Kernel forms are
 * encoded in the block-size entry:
 *   E-step  T > 0: one thread per element; -T: a grid of resident blocks
 *           whose threads loop over elements, loading the next element's
 *           face neighbours while computing the current one;
 *   face    T > 0: one thread per edge point;
 *           -T: one thread per face evaluating every edge point, in a grid
 *           of resident blocks whose threads loop over faces and load the
 *           next face's connectivity while computing the current one;
 *   volume  T > 0: one thread per element, nodal values read from global
 *           memory; -T: staged: a persistent grid whose blocks bring the
 *           next tile of T elements into shared memory with bulk
 *           asynchronous copies while computing the current tile.
 * Every form gives bitwise the same results.  Forms whose shared memory does
 * not fit are skipped.  Synchronizes; the step graph is recaptured on the
 * next advance. */
dg_status dg_batch_autotune(dg_batch *b, int n_iter);
/* Current block sizes: out[3*g + k], k = 0 E-step, 1 face, 2 volume; returns
 * the number of groups in *n_groups. */
dg_status dg_batch_tiles(const dg_batch *b, int32_t *out, int cap, int32_t *n_groups);
/* Sets the block sizes (encoded as for dg_batch_autotune), n = 3 x groups.
 * DG_ERR_ARG for a size outside 32..256 or not a multiple of 32, or a
 * shared-memory form that does not fit on the device for that group. */
dg_status dg_batch_set_tiles(dg_batch *b, const int32_t *tiles, int n);

/* Profiling aid: average device milliseconds of one launch of each kernel
 * of every group, n_iter back-to-back launches timed with CUDA events on the
 * batch's stream: ms[4*g + k], k = 0 E-step, 1 face, 2 volume (writes a
 * scratch stage buffer), 3 per-instance stable step (time and step counters
 * are restored afterwards).  cap >= 4 * groups.  Synchronizes. */
dg_status dg_batch_time_kernels(dg_batch *b, int n_iter, double *ms, int cap);

/* Totals: elements, DOF (elements x nodes x V fields) and groups. */
dg_status dg_batch_info(const dg_batch *b, int64_t *elements, int64_t *dofs, int32_t *n_groups);
/* Kernel launches one step enqueues: 11 per group (14 per wet/dry group, whose
 * stages add a stage kernel after each volume pass), or 1 per group with
 * dg_batch_set_persistent. */
int32_t dg_batch_launches_per_step(const dg_batch *b);

/* Selects how a step is enqueued (the default, on = 0: for every (dimension,
 * order) group, the step-size reduction, then for each of the three SSP-RK3
 * stages the E-step, face-flux and volume kernels: 11 launches per group,
 * replayed from a CUDA graph).  on != 0: one persistent launch per group and
 * step, whose thread blocks claim the same work (128-element and
 * 128-face-point tiles, per-instance step sizes) in a fixed order from a
 * global counter and wait, per instance, only for the phase before theirs,
 * so the phases of different instances overlap; the arithmetic is the same
 * (FP64 results agree to rounding: the compiler may fuse some multiply-adds
 * differently in the two kernels).  Waits are bounded (one second); a wait that
 * gives up latches DG_ERR_TIMEOUT for its instance (reported by the next
 * synchronizing call).  Discards captured graphs.  Returns
 * DG_ERR_UNSUPPORTED for DG_PREC_FP32_TC batches (the persistent step runs
 * the CUDA-core volume pass) and for batches with a wet/dry group (it has no
 * wet/dry stage).  (A launch structure of
 * this library's explicit integrator; the paper's scheme is implicit.) */
dg_status dg_batch_set_persistent(dg_batch *b, int on);
const char *dg_batch_last_error(const dg_batch *b);
void dg_batch_destroy(dg_batch *b);

#ifdef __cplusplus
}
#endif
#endif /* DG_BATCH_H */
