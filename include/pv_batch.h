/*
 * pv_batch.h -- batched verification and re-trace of many scenes (C ABI).
 *
 * The per-frame path of pv.h (pose update, Sec. 3.1 origin update, Sec. 3.2
 * dynamic occlusions, Sec. 3.3 / Alg. 1 / Eq. 2 continuation, Sec. 5.2
 * compaction, Fig. 2 / Sec. 4 re-trace) run for up to PV_BATCH_MAX_SCENES
 * independent scenes at once: each step is one kernel launch over all
 * scenes (tiles of every scene in one grid; the continuation and the
 * re-trace are persistent kernels whose work lists span all scenes, so
 * small scenes fill the GPU together with large ones).  A frame is captured
 * once as a CUDA graph and replayed; the per-frame poses reach it through a
 * copy node that reads one of three pinned staging slots.  The paper
 * verifies one scene at a time; batching is a GB300 design choice.
 *
 * Every scene computes exactly what the single-scene calls compute
 * (pv_update_dynamic, pv_verify_paths, pv_retrace_invalid with the same
 * seed and frame): the same device code runs, only the mapping of work to
 * threads differs.  The statistics agree too, except the traversal counters
 * (node_visits, tri_tests) of the warp-per-path verify mapping, which counts
 * every (segment, object) pair it tests.
 *
 * The tuner (pv_batch_autotune) runs the next frames eagerly with candidate
 * configurations in two phases (re-trace parameters, then the verify
 * mapping), times each step with CUDA events, keeps per phase the candidate
 * whose whole frame is fastest and then captures the graph with it.
 */
#ifndef PV_BATCH_H
#define PV_BATCH_H

#include "pv.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pv_batch pv_batch;

#define PV_BATCH_MAX_SCENES 32

/* One scene of a batch.  The scene must be built without
 * PV_BUILD_DYN_REBUILD (the graph replays refits); paths are its path
 * buffers (pv_paths rules), d_list [paths.n] and d_count receive the frame's
 * re-trace list (device, caller-owned), d_stats (optional, device) is
 * accumulated like the single-scene calls' counters.  d_list and d_count
 * NULL for every scene of a batch: no lists are returned, and Alg. 1 runs
 * inside the persistent re-trace kernel as in pv_verify_retrace (records and
 * counters as pv_verify_retrace leaves them, which are those of the
 * separate calls). */
typedef struct {
  pv_scene* scene;
  pv_paths paths;
  uint32_t* d_list;
  uint32_t* d_count;
  pv_frame_stats* d_stats;
  uint64_t seed;
} pv_batch_scene;

/* Launch configuration of the batched kernels.
 *  verify_mapping   0: thread per path, 1: warp per path (lanes take the
 *                   (segment, moved object) pairs of one path at a time),
 *                   2: flat (each warp deals the segments of its 32 paths
 *                   out to its lanes; PV_MODE_ERROR only)
 *  verify_threads   64, 128 or 256 paths per verify block (tile size)
 *  trace_steps      16, 32 or 64: at most this many traversal steps between
 *                   work refills; a warp refills earlier once every lane's
 *                   ray has ended
 *  trace_blocks     persistent re-trace blocks per SM, 0 = occupancy limit
 *  stack            32 or 64 traversal stack entries for the continuation
 *                   and the re-trace; 32 only when every scene's wide tree
 *                   needs at most 32 (three per level of its deepest path) */
typedef struct {
  int32_t verify_mapping;
  int32_t verify_threads;
  int32_t trace_steps;
  int32_t trace_blocks;
  int32_t stack;
} pv_batch_config;

/* Create a batch over n (1..PV_BATCH_MAX_SCENES) scenes verified with the
 * same params; each scene must appear once; lists for every scene or for
 * none (PV_ERR_ARG otherwise).  The scenes stay owned by the
 * caller and must outlive the batch; while the batch exists they are driven
 * only through pv_batch_frame.  Allocates the batch's device tables and
 * pinned staging (synchronous).  Scenes with distribution maps (Sec. 3.1)
 * run compute DM_C (with the origin update), the two-pass prune of Eq. 1 and
 * the fill inside the frame, with the scene's seed and the frame number
 * keying the prune draws, as pv_verify_paths does with params seed and
 * frame; their batch must have lists, since prune and fill need every path's
 * Alg. 1 answer before the list is made.  PV_ERR_ARG for bad arguments,
 * PV_ERR_LIMIT for too many scenes, PV_ERR_STATE for a scene built with
 * PV_BUILD_DYN_REBUILD, or with distribution maps in a batch without lists. */
int pv_batch_create(const pv_batch_scene* scenes, uint32_t n, const pv_verify_params* params, void* stream,
                    pv_batch** out);

/* One frame for every scene: xforms[i] (host, [n_objects][12] like
 * pv_update_dynamic, or NULL) and lights[i] (host, or NULL) are scene i's new
 * poses; the frame number keys the re-trace's random numbers.  Enqueues the
 * whole frame on the stream (one graph launch once captured) and returns.  A
 * NULL stream means the batch's own blocking stream (graphs cannot be
 * captured on the legacy default stream, which it is ordered against);
 * blocks only when the staging slot it needs is still in use three frames
 * back.  Errors found on the device are recorded in each scene's status
 * (pv_read_device_status). */
int pv_batch_frame(pv_batch* b, const float* const* xforms, const pv_light* const* lights, uint32_t frame,
                   void* stream);

/* Start tuning: the next frames run eagerly, frames_per_candidate frames per
 * candidate configuration (at least 1), the candidates taken in turn (round
 * robin, so frame-to-frame drift of the workload weighs on all of them
 * alike); then the candidate with the fastest whole frame is kept and the
 * graph is captured again.  PV_ERR_ARG for a null batch. */
int pv_batch_autotune(pv_batch* b, uint32_t frames_per_candidate);

/* 1 while tuning, 0 otherwise; negative status for a null batch. */
int pv_batch_tuning(const pv_batch* b);

/* Set or read the launch configuration (set: PV_ERR_ARG for a value outside
 * the lists above or a stack the scenes cannot use; drops captured graphs). */
int pv_batch_set_config(pv_batch* b, const pv_batch_config* cfg);
int pv_batch_get_config(const pv_batch* b, pv_batch_config* cfg);

/* Per-frame CUDA-event times (milliseconds, mean over its tuning frames) of
 * the configuration the tuner kept: [0] pose update, [1] verify,
 * [2] continuation, [3] compaction, [4] re-trace (without lists: [2] is 0
 * and [4] holds Alg. 1 with the re-trace).  PV_ERR_STATE before a tuning run
 * has finished. */
int pv_batch_step_times(const pv_batch* b, float* ms5);

/* Synchronise the batch's last stream and free it (the scenes remain). */
void pv_batch_destroy(pv_batch* b);

#ifdef __cplusplus
}
#endif
#endif /* PV_BATCH_H */
