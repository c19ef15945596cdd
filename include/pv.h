/*
 * pv.h -- C ABI of the GB300 (sm_103a) path-verification library.
 *
 * The library implements the per-frame hot path of Moreau, Doggett, Sintorn,
 * "Path Verification for Dynamic Indirect Illumination" (arXiv 2111.06906):
 * photon paths traced in earlier frames are checked against the lights and
 * objects that moved (Sec. 3.1 "update path origins", Sec. 3.2 "dynamic
 * occlusions", Sec. 3.3 / Alg. 1 / Eq. 2 "error-based threshold"), the paths
 * that fail are compacted into a list (Sec. 5.2, pruned-paths array) and only
 * those are re-traced (Fig. 2 "generate rays" / "trace rays", Sec. 4).
 *
 * Conventions
 *  - Every call is asynchronous on the given CUDA stream (``stream`` is a
 *    cudaStream_t passed as void*; NULL = legacy default stream) and no call
 *    after pv_build_scene allocates device memory.
 *  - Host-detectable errors return a negative pv_status immediately and
 *    enqueue nothing.  Errors found on the device (traversal stack overflow,
 *    iteration caps) are recorded in a sticky status word read by
 *    pv_read_device_status; kernels never trap.
 *  - The scene (acceleration structures, poses, workspace) is owned by the
 *    library.  Path buffers, lists, counters, statistics and atlases are
 *    device memory owned by the caller.  One scene must not be used by two
 *    streams at once.
 *  - Coordinates are metres, y up; all path data are FP32.
 */
#ifndef PV_H
#define PV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pv_scene pv_scene;

typedef enum {
  PV_OK = 0,
  PV_ERR_ARG = -1,        /* bad argument (null pointer, size mismatch, unknown mode) */
  PV_ERR_CUDA = -2,       /* a CUDA runtime call failed */
  PV_ERR_OOM = -3,        /* device allocation failed (pv_build_scene only) */
  PV_ERR_STACK = -4,      /* device: BVH traversal stack overflow */
  PV_ERR_ITER_CAP = -5,   /* device: a bounded loop or wait hit its cap */
  PV_ERR_LIMIT = -6,      /* a format limit: bounces > 15, lights > 4, dynamic objects > 64 */
  PV_ERR_STATE = -7       /* call out of order (e.g. paths larger than the scene's workspace) */
} pv_status;

enum { PV_LIGHT_POINT = 0, PV_LIGHT_RECT = 1 };

/* Verification modes.  NAIVE_AABB: Sec. 3.2, each segment is tested in order
 * against the union of the old and new bounding boxes of every moved object;
 * the first hit schedules that segment and all later ones for re-tracing.
 * NAIVE_EXACT: same, with the moved objects' triangles at their new pose.
 * ERROR: Sec. 3.3 / Alg. 1 -- boxes flag segments, a ray re-finds the end of
 * each flagged segment and the path is kept while the reflected energy stays
 * within tau of the stored one (Eq. 2). */
enum { PV_MODE_NAIVE_AABB = 0, PV_MODE_NAIVE_EXACT = 1, PV_MODE_ERROR = 2 };
enum {
  PV_FLAG_TEST_OLD_TRIS = 1u,   /* exact tests also test the old pose's triangles */
  PV_FLAG_ERROR_EXACT = 2u      /* ERROR mode flags segments with triangles, not boxes */
};
enum {
  PV_BUILD_DYN_REBUILD = 1u,   /* rebuild dynamic BVHs every frame instead of refitting */
  PV_BUILD_STATIC_LBVH = 2u,   /* static tree from Morton codes (default: binned surface-area heuristic) */
  PV_BUILD_REFIT_CLIMB = 4u    /* refit the dynamic wide nodes level by level, the last child to arrive
                                  going on up (default: each node from the contiguous run of triangles
                                  under it, no dependent levels); both give the same boxes */
};

#define PV_MAX_LIGHTS 4
#define PV_MAX_DYN_OBJECTS 64
#define PV_MAX_BOUNCES 15

/* Info word (Sec. 4): DM cell (22 bits, here light index << 20), number of
 * segments (4), re-trace start vertex (4), replace (1), reuse the light's
 * position and direction (1). */
#define PV_INFO_CELL_MASK 0x003FFFFFu
#define PV_INFO_NSEG_SHIFT 22
#define PV_INFO_START_SHIFT 26
#define PV_INFO_REPLACE (1u << 30)
#define PV_INFO_REUSE_LIGHT (1u << 31)

/* A light pose (64 bytes).  POINT: isotropic, ``pos``.  RECT: a w x h
 * rectangle centred at ``pos`` emitting on the side of unit ``normal``;
 * ``size[0]`` runs along unit ``tangent``, ``size[1]`` along normal x tangent.
 * ``power`` is the RGB flux carried by the light's ``n_paths`` paths.  Paths
 * belong to lights in order: light 0 owns path ids [0, n0), light 1 the next
 * n1 ids, and so on. */
typedef struct {
  int32_t type;
  float pos[3], normal[3], tangent[3], size[2], power[3];
  uint32_t n_paths;
} pv_light;

/* Scene description; all arrays are HOST memory and are copied.
 *  verts          [n_tris][3][3]  triangle corners; object-local for dynamic objects
 *  tri_object     [n_tris]        object of each triangle (primitive id = index)
 *  object_dynamic [n_objects]     1 = rigid dynamic object (at most 64), 0 = static
 *  object_albedo  [n_objects][3]  Lambertian albedo (> 0 in some channel)
 *  object_xform   [n_objects][12] initial 3x4 row-major [R|t] pose, NULL = identity
 *  scene_diag     length unit of the tolerances: t_min = 1e-5 diag for rays
 *                 leaving a surface, AreClose = 1e-5 diag (Alg. 1)
 *  dm_rect        distribution map of every rectangle light (Sec. 3.1): cells
 *                 along its sample dimensions x, y, sin^2 theta, phi / 2 pi
 *                 (all zero: none), e.g. 8 x 8 x 64 x 64
 *  dm_point       distribution map of every point light over (1 - z) / 2 and
 *                 phi / 2 pi (all zero: none); a map holds at most 2^20 cells
 * With a map, pv_trace_all spreads each light's paths evenly over its cells
 * (DM_C = DM_T), fresh emissions sample inside the cell in the path's info
 * word, and pv_verify_paths computes DM_C, prunes (Eq. 1) and fills for every
 * light that moved (see pv_verify_paths). */
typedef struct {
  const float* verts;
  uint32_t n_tris;
  const uint32_t* tri_object;
  uint32_t n_objects;
  const uint8_t* object_dynamic;
  const float* object_albedo;
  const float* object_xform;
  uint32_t n_lights;
  const pv_light* lights;
  uint32_t max_bounces;
  float scene_diag;
  uint32_t flags;
  uint32_t dm_rect[4];
  uint32_t dm_point[2];
} pv_scene_desc;

/* Path buffers (device memory, caller-owned), the 2-D photon array of Sec. 4
 * with row k holding the k-th photon of every path, split in two coalesced
 * 16-byte planes:
 *  info   [n]         info word (above)
 *  origin [3][n]      emission point, x plane then y then z
 *  pa     [B][n][4]   photon hit position x,y,z and primitive id (int32 bits)
 *  pb     [B][n][4]   incident RGB energy and path length from the light     */
typedef struct {
  uint32_t n;
  uint32_t max_bounces;
  uint32_t* info;
  float* origin;
  float* pa;
  float* pb;
} pv_paths;

typedef struct {
  int32_t mode;     /* PV_MODE_* */
  float tau;        /* Eq. 2 threshold T (relative); INFINITY accepts every energy */
  uint32_t flags;   /* PV_FLAG_* */
  uint32_t frame;   /* frame number and seed of the prune draws (Philox counter */
  uint64_t seed;    /* (path, 16, frame), key seed); used only with distribution maps */
} pv_verify_params;

/* Top-down XZ atlas (device, caller-owned): data[height][width][3] unsigned
 * fixed point with 2^scale_log2 units per energy unit over [x0,x1] x [z0,z1];
 * a photon lands in texel floor((x-x0) * width/(x1-x0)), clamped, computed in
 * FP32 without fused operations. */
typedef struct {
  uint64_t* data;
  uint32_t width, height;
  float x0, z0, x1, z1;
  int32_t scale_log2;
} pv_atlas;

/* Per-frame counters (device, caller-owned, accumulated; zero them first). */
typedef struct {
  uint32_t n_paths;          /* paths verified */
  uint32_t n_listed;         /* paths in the re-trace list */
  uint32_t n_reemit;         /* re-traced from the light (start 0) */
  uint32_t n_tail;           /* re-traced from a vertex > 0 */
  uint32_t n_updated;        /* kept with moved vertices (Alg. 1) */
  uint32_t n_truncated;      /* shortened because a re-found segment escaped */
  uint32_t n_cont;           /* paths that entered Alg. 1 */
  uint32_t vis_rays;         /* point-light visibility rays (Sec. 3.1) */
  uint32_t cont_rays;        /* rays traced by Alg. 1 */
  uint32_t trace_rays;       /* rays traced by re-tracing / trace-all */
  uint32_t segments_tested;  /* segment-vs-moved-object tests */
  uint32_t photons_written;  /* photons stored by re-tracing / trace-all */
  uint32_t n_pruned;         /* paths pruned by Eq. 1 (distribution maps) */
  uint32_t n_filled;         /* free paths given a cell to fill (distribution maps) */
  uint64_t node_visits;      /* BVH nodes visited by every ray query of the call */
  uint64_t tri_tests;        /* ray-triangle tests of every ray query of the call */
} pv_frame_stats;

/* Build the static BVH and the dynamic objects' BVHs (Morton-code LBVH),
 * upload per-primitive data and size the per-frame workspace for the lights'
 * total path count.  Sets the initial pose as both old and new pose.
 * Returns PV_ERR_LIMIT for more than 4 lights, 64 dynamic objects or 15
 * bounces, PV_ERR_OOM if device memory runs out.  Synchronous. */
int pv_build_scene(const pv_scene_desc* desc, void* stream, pv_scene** out);

/* Advance one frame (no paper counterpart beyond the moving scene of Sec. 3):
 * the current pose becomes the old pose; ``xforms`` (host [n_objects][12],
 * only dynamic objects read; NULL = unchanged) and ``lights`` (host
 * [n_lights], NULL = unchanged) become the new pose.  Moved objects are
 * transformed and their BVHs refitted (or rebuilt) on the device.  An object
 * or light moved iff one of its float values changed bit for bit. */
int pv_update_dynamic(pv_scene* s, const float* xforms, const pv_light* lights, void* stream);

/* Verify every path against the change from the old to the new pose:
 * update origins (Sec. 3.1; point light: exact visibility ray replacing the
 * shadow map; area light: stored direction re-intersected with the new
 * light plane, with Eq. 2 on the primary energy for a tilted light), dynamic
 * occlusions (Sec. 3.2), and in PV_MODE_ERROR the threshold continuation
 * (Alg. 1, Eq. 2) which may move vertices in place.  Paths to re-trace get
 * the replace bit and a start vertex; their ids are written in ascending
 * order to d_list[0..*d_count) (d_list holds n entries).  d_stats may be
 * NULL.  Returns PV_ERR_ARG if paths->n differs from the lights' total.
 *
 * Distribution maps (Sec. 3.1), for a light with a map that moved: the
 * parametrisation (float32, correctly rounded basic operations; the angle
 * from half-angle steps and the Gregory series) decides each kept path's
 * cell and whether it still comes from the light (the rectangle's extent
 * test is replaced by it) -- "compute DM_C", fused with the origin update as
 * in Sec. 4; then paths of cells with DM_C > DM_T are pruned with
 * probability (DM_C - DM_T) / DM_C (Eq. 1), decided exactly on the 24-bit
 * draw of Philox counter (path, 16, frame), marking first and editing the
 * counts in a second pass (Sec. 4); then the free paths (pruned, or no
 * longer from the light) in ascending id order take the cells' deficits
 * DM_T - DM_C in cell order and spread any further ones evenly ("fill
 * DM_C").  DM_T(c) = floor(N (c + 1) / n) - floor(N c / n) for N paths and
 * n cells. */
int pv_verify_paths(pv_scene* s, const pv_paths* paths, const pv_verify_params* params,
                    uint32_t* d_list, uint32_t* d_count, pv_frame_stats* d_stats, void* stream);

/* Re-trace the listed paths at the new pose from their start vertex with a
 * persistent kernel: start 0 without reuse = fresh emission; start 0 with
 * reuse = same origin and primary direction; start k > 0 = Russian roulette
 * and a cosine-weighted bounce at photon k.  Random numbers are
 * Philox-4x32-10 keyed by (path, vertex, frame) with key ``seed``.  The
 * count is read on the device (no host synchronisation). */
int pv_retrace_invalid(pv_scene* s, const pv_paths* paths, const uint32_t* d_list,
                       const uint32_t* d_count, uint64_t seed, uint32_t frame,
                       pv_frame_stats* d_stats, void* stream);

/* One frame's verification and re-trace in one call (Fig. 2 from "verify
 * paths" to "trace rays"): the path records and every d_stats counter come
 * out bit for bit as after pv_verify_paths followed by pv_retrace_invalid on
 * its list with the seed and frame of ``params``.  No list is returned.  In
 * PV_MODE_ERROR, when something moved and no light has a distribution map,
 * Alg. 1 runs inside the persistent re-trace kernel: its closest-hit queries
 * interleave with the re-trace rays, and a path failing Eq. 2 goes on to its
 * re-trace from the failing vertex at once; the paths are processed in
 * another order, never with other arithmetic.  Otherwise the same kernels as
 * the two separate calls run.  The list is kept in the scene's workspace, so
 * calls on one scene must not overlap.  Errors as pv_verify_paths. */
int pv_verify_retrace(pv_scene* s, const pv_paths* paths, const pv_verify_params* params,
                      pv_frame_stats* d_stats, void* stream);

/* pv_verify_retrace followed by pv_deposit in one call (Fig. 2 from "verify
 * paths" to "splat/gather"), leaving the same records, counters and atlas bit
 * for bit.  Without distribution maps the deposit runs inside the persistent
 * re-trace kernel: each path is deposited by the lane that finishes it, and
 * the paths this frame does not touch (neither re-traced nor looked at by
 * Alg. 1) are deposited by lanes that have no rays left to trace.  The atlas
 * is cleared first and follows pv_deposit's rules.  Stage timing as
 * pv_verify_retrace (stage [3] then includes the deposit).  PV_ERR_ARG for a
 * null or invalid atlas, otherwise errors as pv_verify_paths. */
int pv_verify_retrace_deposit(pv_scene* s, const pv_paths* paths, const pv_verify_params* params,
                              const pv_atlas* atlas, pv_frame_stats* d_stats, void* stream);

/* pv_verify_retrace_deposit for an atlas that already holds pv_deposit of
 * ``paths`` as they are on entry (same atlas rectangle, resolution and
 * scale; e.g. pv_deposit after pv_trace_all, then this call every frame).
 * The atlas is not cleared: each path the frame re-traces or hands to
 * Alg. 1 has its entry photons taken out (the same fixed-point values,
 * subtracted modulo 2^64) and its final photons added; untouched paths are
 * not read.  Since the texel sums are integers, the atlas on return is the
 * one pv_verify_retrace_deposit leaves, bit for bit, and records and
 * counters are the same too.  With distribution maps the call clears the
 * atlas and deposits every path, as pv_verify_retrace_deposit.  An atlas
 * that does not hold the entry deposit gives an atlas that does not either
 * (the error is carried, not detected).  Errors as pv_verify_retrace_deposit. */
int pv_verify_retrace_deposit_delta(pv_scene* s, const pv_paths* paths, const pv_verify_params* params,
                                    const pv_atlas* atlas, pv_frame_stats* d_stats, void* stream);

/* Stage timing of pv_verify_retrace and the two deposit forms (no paper
 * counterpart).  With n > 0, each later call records five CUDA events on its
 * stream -- at its start, after its clears (atlas, counters), after k_verify,
 * before its re-trace kernel, at its end -- keeping the last n calls in a
 * ring; n = 0 turns it off.  The events between the kernels also keep the
 * re-trace kernel from starting before k_verify has ended, so a timed call
 * takes a little longer than an untimed one.  Creates (and destroys) events
 * and synchronises with the scene's last stream, so call it outside any
 * timed or captured region.  PV_ERR_ARG for n > 4096. */
int pv_stage_timing(pv_scene* s, uint32_t n);

/* Milliseconds of the recorded calls, oldest first, five per call (``ms``
 * holds 5 n floats): [0] the clears before verification (the atlas of the
 * deposit forms, the work counters), [1] verification (k_verify), [2] what
 * runs between it and the re-trace kernel (nothing with fusion, where
 * k_verify appends the re-trace list itself; otherwise the continuation, the
 * distribution-map steps and the compaction), [3] the re-trace kernel (with
 * fusion: Alg. 1, the re-trace and, with an atlas, the deposit), [4] the
 * whole call.  *count receives the number of calls recorded (at most n).
 * Waits for the events. */
int pv_stage_times(pv_scene* s, float* ms, uint32_t* count);

/* Baseline of Sec. 5: re-trace every path from the light (no reuse). */
int pv_trace_all(pv_scene* s, const pv_paths* paths, uint64_t seed, uint32_t frame,
                 pv_frame_stats* d_stats, void* stream);

/* pv_trace_all with the deposit of the stand-in for Fig. 2's splat/gather
 * step in the same kernel: ``atlas`` (caller-owned device memory, layout as
 * for pv_deposit) is cleared, then each photon is added as it is stored, from
 * the values written to pa/pb.  Records, counters and atlas are bit-identical
 * to pv_trace_all followed by pv_deposit (integer additions commute).  This
 * is the trace-all frame that the reuse frame of pv_verify_retrace_deposit is
 * measured against.  PV_ERR_ARG for a bad atlas (as pv_deposit). */
int pv_trace_all_deposit(pv_scene* s, const pv_paths* paths, uint64_t seed, uint32_t frame,
                         const pv_atlas* atlas, pv_frame_stats* d_stats, void* stream);

/* Ascending ids of the paths whose replace bit is set (Sec. 5.2 pattern:
 * the marked paths packed so that as few blocks as possible process them);
 * single-pass decoupled look-back scan using the scene's workspace. */
int pv_compact_replace(pv_scene* s, const pv_paths* paths, uint32_t* d_list, uint32_t* d_count,
                       void* stream);

/* Same result as pv_compact_replace over info[0..n), without a scene and
 * without allocating device memory (the paper has no counterpart; this serves
 * callers that must not allocate once running, e.g. a renderer that reserves
 * its memory budget at start-up or whose device memory belongs to another
 * allocator, and frame loops that cannot take the device-wide synchronisation
 * an allocation may cause).  d_info[n], d_list[n] and d_count are device
 * memory owned by the caller.  The scratch is one fixed array inside the
 * library, sized for at most PV_STATIC_COMPACT_MAX_PATHS paths (128 KiB,
 * kept on every GPU that loads the library until the process exits); larger
 * n returns PV_ERR_LIMIT.  The first call on a device looks up the array's
 * device address (make that first call before any stream capture).  All calls
 * share the array, so calls that overlap on the GPU race; serialise them (one
 * stream, or events).  Returns PV_ERR_ARG for null pointers.  No scene
 * holds a status word for this call: if a tile's look-back ever waits past
 * its spin cap (a predecessor tile never published its sum), the call writes
 * 0xFFFFFFFF to *d_count, and the list is then incomplete. */
#define PV_STATIC_COMPACT_MAX_PATHS (1u << 26)
int pv_compact_replace_static(const uint32_t* d_info, uint32_t n, uint32_t* d_list, uint32_t* d_count,
                              void* stream);

/* Clear the atlas and add every stored photon's incident energy to the
 * texel under it (stand-in for the renderer's splatting, Fig. 2). */
int pv_deposit(pv_scene* s, const pv_paths* paths, const pv_atlas* atlas, void* stream);

/* ---- differentiable deposit model (the paper has no counterpart) ----------
 * Serves to rank the paths invalidated by the Eq. 2 test when a ray budget
 * cannot re-trace them all.  Every stored path keeps its triangles and its
 * sampled directions; the light and the dynamic objects move by parameters
 * theta (float32, device memory, pv_theta_size floats):
 *   per light l:           theta[7l+0..2] position, theta[7l+3..5] normal
 *                          (rectangles; the tangent stays fixed),
 *                          theta[7l+6] intensity factor (1 = as traced);
 *   per dynamic object j   theta[7L+3j+0..2] translation (world space),
 *   (slot order = ascending object id among the dynamic objects).
 * Photon k is re-found on its triangle's plane (through the stored photon,
 * moved with its object's translation) along the stored incoming direction;
 * a point light re-aims from its position through the first stored photon, a
 * rectangle keeps the stored sample point and direction in its frame.  The
 * photon's energy times the intensity factor is splatted with the uniform
 * cubic B-spline (4 x 4 texels, twice continuously differentiable) into an
 * RGB float32 atlas of height x width texels over rect = {x0, z0, x1, z1}
 * (texel centres at half-integers, texels outside dropped).  At theta equal
 * to the current poses (positions, normals, factor 1, translations) the
 * model reproduces the stored photons.  Rotations are held at their current
 * value. */

/* Number of floats in theta, or PV_ERR_ARG for a null scene. */
int pv_theta_size(const pv_scene* s);

/* Write theta at the current poses into h_theta (host float[pv_theta_size]).
 * PV_ERR_ARG for null pointers. */
int pv_theta_current(const pv_scene* s, float* h_theta);

/* Add the model's splat of every path in paths to d_atlas (float32
 * [height][width][3], caller-owned device memory, NOT cleared here) with
 * float atomics.  rect: host float[4].  PV_ERR_ARG for null pointers, an
 * empty or inverted rect, or a side above 2^20 texels. */
int pv_model_deposit(pv_scene* s, const pv_paths* paths, const float* d_theta, float* d_atlas,
                     uint32_t width, uint32_t height, const float* rect, void* stream);

/* Reverse mode of pv_model_deposit for the loss gradient d_grad_atlas
 * (float32 [height][width][3], device): ADDS dL/dtheta into d_dtheta
 * (float32 [pv_theta_size], device, caller clears it) and writes, when
 * d_score is not null, each path's score |dL/d(intensity of that path)| =
 * |sum over its photons of G . E w| into d_score (float32 [n], device).
 * Same argument rules as pv_model_deposit. */
int pv_adjoint_deposit(pv_scene* s, const pv_paths* paths, const float* d_theta, const float* d_grad_atlas,
                       uint32_t width, uint32_t height, const float* rect, float* d_dtheta, float* d_score,
                       void* stream);

/* Ray budget: of the d_count listed paths (d_list, ascending ids, as
 * pv_verify_paths writes it), keep the min(budget, count) with the largest
 * d_score (ties and non-positive scores: smaller id first) and write them in
 * ascending id order to d_out, their number to d_out_count (device memory,
 * caller-owned, d_out sized for the scene's path count).  Uses the scene's
 * workspace (it overwrites the intersected-segment masks, which only live
 * inside pv_verify_paths).  PV_ERR_ARG for null pointers. */
int pv_budget_list(pv_scene* s, const uint32_t* d_list, const uint32_t* d_count, const float* d_score,
                   uint32_t budget, uint32_t* d_out, uint32_t* d_out_count, void* stream);

/* FP32 fused multiply-add probe (no paper counterpart): the measured
 * denominator of the traversal kernels' ALU roofline.  Enqueues one kernel of
 * ``blocks`` blocks of 256 threads; every thread runs 8 independent chains of
 * 16 * ``iters`` dependent fmaf, so the FMA pipe bounds it.  *fmas (host)
 * receives the number of fused multiply-adds the kernel executes; time it
 * with events on ``stream``.  d_sink: device memory of ``blocks`` floats,
 * written only in a case that the kernel's inputs never reach.  PV_ERR_ARG
 * for zero blocks or iterations or a null pointer. */
int pv_fma_probe(uint32_t blocks, uint32_t iters, float* d_sink, uint64_t* fmas, void* stream);

/* Cap the BVH node visits of every ray query (0 restores the default, which
 * no query on a valid tree reaches).  A query that reaches the cap stops,
 * counts as a miss and records PV_ERR_ITER_CAP in the device status: the way
 * to exercise device-side error reporting without faulting the GPU.
 * Returns PV_ERR_ARG for a null scene. */
int pv_set_traversal_limit(pv_scene* s, uint32_t max_visits);

/* Synchronise the scene's last stream and return the first device-side error
 * recorded since the last call (then clear it), or PV_OK. */
int pv_read_device_status(pv_scene* s);

/* Screen-space photon splat: the renderer's "splat/gather" step of Fig. 2,
 * whose method the paper only cites, as a plain radius kernel.  A pinhole
 * camera at ``pos`` looks at ``target`` (``up`` fixes the roll; vertical field
 * of view ``fov_y`` radians; width x height pixels, rays through pixel
 * centres).  Every pixel's primary ray finds its visible point p (normal
 * facing the camera, albedo rho of its object); every stored photon x with
 * energy E whose incoming segment arrives on the visible side adds
 *   rho / pi * E * 2 (1 - s^2) / (pi r^2),   s = |p - x| / radius < 1
 * to the pixel (the kernel integrates to 1 over a plane).  A photon whose
 * kernel cube reaches within 1e-3 scene diagonals of the camera plane is
 * skipped.  Evaluated as a gather over a hashed grid of the photons, so the
 * sum's order within a pixel is not fixed.  d_image: float32
 * [height][width][3] device memory, written.  d_work:
 * pv_splat_workspace_bytes(s, width, height) bytes of 256-byte-aligned
 * device memory (visible points, photon grid).  PV_ERR_ARG for a degenerate
 * camera (zero size, fov outside (0, 3.1), up parallel to the view
 * direction), radius <= 0, or a small or misaligned workspace; PV_ERR_LIMIT
 * for more than 2^27 paths. */
typedef struct {
  float pos[3], target[3], up[3];
  float fov_y;
  uint32_t width, height;
} pv_camera;

size_t pv_splat_workspace_bytes(const pv_scene* s, uint32_t width, uint32_t height);
int pv_splat(pv_scene* s, const pv_paths* paths, const pv_camera* cam, float radius, float* d_image, void* d_work,
             size_t work_bytes, void* stream);

/* Number of cells of light ``light``'s distribution map (0: none), or
 * PV_ERR_ARG.  pv_read_distribution_map synchronises the scene's last stream
 * and copies its current counts DM_C to h_counts (host, that many entries). */
int pv_distribution_map_cells(const pv_scene* s, uint32_t light);
int pv_read_distribution_map(pv_scene* s, uint32_t light, uint32_t* h_counts);

void pv_destroy_scene(pv_scene* s);
const char* pv_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* PV_H */
