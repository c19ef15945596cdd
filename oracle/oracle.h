/*
 * FP64 brute-force CPU oracle for per-frame photon-path verification
 * (Moreau, Doggett, Sintorn, "Path Verification for Dynamic Indirect
 * Illumination", arXiv 2111.06906).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA library; both sides receive the
 * same seeded scene arrays and each implements the Philox-4x32-10 counter
 * generator (Salmon et al., SC 2011) from its published definition.
 *
 * Every geometric query tests every triangle (no acceleration structure) in
 * double precision.  Path records are stored as FP32 (the method's storage
 * format, Sec. 4) and every step continues from the stored FP32 record.
 *
 * Alongside each result the oracle reports whether the result is ambiguous:
 * whether a perturbation of 1e-6 x scene diagonal (edge/plane proximity), a
 * near-tie in Eq. 2 or in the AreClose test of Alg. 1 could flip a decision.
 * For such a path the per-path entry points below take a decision script and
 * give, one run per script, every record the path admits when each ambiguous
 * decision takes each of its possible outcomes.
 */
#ifndef PV_ORACLE_H
#define PV_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A light pose (64 bytes): type 0 = isotropic point, 1 = rectangle emitting
 * on the side of ``normal``; ``size[0]`` runs along ``tangent`` and
 * ``size[1]`` along normal x tangent.  Paths are assigned to lights in order:
 * light 0 owns path ids [0, n0), light 1 the next n1 ids, ... */
typedef struct {
  int32_t type;
  float pos[3], normal[3], tangent[3], size[2], power[3];
  uint32_t n_paths;
} or_light;

/* One stored photon (32 bytes, Sec. 4): hit position (see the reading of the
 * record in the design notes), hit primitive id, incident RGB energy, and the
 * path length travelled from the light ("radius" slot). */
typedef struct {
  float pos[3];
  int32_t prim;
  float E[3];
  float radius;
} or_photon;

/* Info word bit fields (Sec. 4): DM cell (22 bits; light index << 20),
 * number of segments (4), retrace start vertex (4), replace (1), reuse light
 * position and direction (1). */
#define OR_INFO_CELL_MASK 0x003FFFFFu
#define OR_INFO_NSEG_SHIFT 22
#define OR_INFO_START_SHIFT 26
#define OR_INFO_REPLACE (1u << 30)
#define OR_INFO_REUSE_LIGHT (1u << 31)

/* verification modes */
#define OR_MODE_NAIVE_AABB 0
#define OR_MODE_NAIVE_EXACT 1
#define OR_MODE_ERROR 2
#define OR_FLAG_TEST_OLD_TRIS 1u
#define OR_FLAG_ERROR_EXACT 2u   /* error mode: exact triangle test instead of boxes */

/* ambiguity bits reported per path */
#define OR_AMB_TRACE 1u
#define OR_AMB_VERIFY 2u
#define OR_AMB_CONT 4u
#define OR_AMB_ENERGY 8u
#define OR_AMB_LIGHT 16u

typedef struct or_scene or_scene;

/* per-call counters (summed over the paths processed) */
typedef struct {
  uint64_t paths;            /* paths processed */
  uint64_t segments_tested;  /* segment-vs-object tests made */
  uint64_t segments_amb;     /* of which ambiguous */
  uint64_t vis_rays;         /* point-light visibility rays (Sec. 3.1) */
  uint64_t cont_rays;        /* closest-hit rays of Alg. 1 */
  uint64_t trace_rays;       /* closest-hit rays of tracing / re-tracing */
  uint64_t energy_tests;     /* Eq. 2 evaluations */
  uint64_t energy_amb;       /* Eq. 2 near-ties */
  uint64_t n_reemit;         /* paths to re-emit from the light (start 0) */
  uint64_t n_tail;           /* paths to re-trace from a vertex > 0 */
  uint64_t n_updated;        /* paths reused with moved vertices (Alg. 1) */
  uint64_t n_truncated;      /* paths shortened because a re-traced ray missed */
  uint64_t n_pruned;         /* paths pruned by Eq. 1 (distribution maps) */
  uint64_t n_filled;         /* free paths given a distribution-map cell to fill */
  uint64_t rays_amb;         /* ray queries (trace, Alg. 1, visibility) whose answer is ambiguous */
} or_stats;

/* Scene: verts [n_tris][3][3] (object-local for dynamic objects),
 * tri_object [n_tris], object_dynamic [n_objects], albedo [n_objects][3].
 * diag is the scene diagonal; eps = 1e-6 diag and t_min = 1e-5 diag. */
or_scene* or_scene_create(const float* verts, uint32_t n_tris, const uint32_t* tri_object,
                          uint32_t n_objects, const uint8_t* object_dynamic,
                          const float* albedo, double diag, uint32_t max_bounces);
void or_scene_destroy(or_scene* s);

/* Set the previous (old) and current (new) poses: xforms [n_objects][12]
 * row-major 3x4, lights [n_lights].  An object or light "moved" iff any of
 * its float32 pose values differ bit for bit. */
void or_scene_set_poses(or_scene* s, const float* xform_old, const float* xform_new,
                        const or_light* lights_old, const or_light* lights_new,
                        uint32_t n_lights);

/* Philox-4x32-10 block: out[4] = philox(ctr[4], key[2]). */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Paths are processed for a subset of ids; every per-path array below is
 * indexed by position in ``ids`` (n entries): info[n], origin[n][3],
 * photons[n][B], amb[n].  */

/* Trace every listed path from scratch at the current pose (emission +
 * bounces, Sec. 3 / Fig. 2 "generate rays" and "trace rays"). */
void or_trace(const or_scene* s, const uint32_t* ids, uint32_t n, uint64_t seed,
              uint32_t frame, uint32_t* info, float* origin, or_photon* photons,
              uint32_t* amb, or_stats* st);

/* Verify the listed paths against the pose change: update origins
 * (Sec. 3.1), dynamic occlusions (Sec. 3.2) and, in OR_MODE_ERROR, the
 * error-based threshold continuation (Sec. 3.3, Alg. 1, Eq. 2).  Sets the
 * replace / start / reuse-light bits, updates origins and moved vertices in
 * place, and returns the intersected-segment mask (bit i = segment i). */
void or_verify(const or_scene* s, const uint32_t* ids, uint32_t n, int32_t mode, double tau,
               uint32_t flags, uint64_t seed, uint32_t frame, uint32_t* info, float* origin,
               or_photon* photons, uint32_t* seg_mask, uint32_t* amb, or_stats* st);

/* Distribution maps (Sec. 3.1).  or_scene_set_dm (after the poses are set)
 * gives every rectangle light a map of rect[0] x rect[1] x rect[2] x rect[3]
 * cells over its sample space (x, y, sin^2 theta, phi / 2 pi) and every point
 * light one of point[0] x point[1] cells over ((1 - z) / 2, phi / 2 pi); a zero
 * resolution leaves that kind of light without a map; -1 if a map has more
 * than 2^20 cells.  With a map, a full trace puts path j of a light in cell
 * floor(((j + 1) n - 1) / N) (so DM_C = DM_T), fresh emissions sample inside
 * their cell, and or_verify, when the light moved, recomputes each kept
 * path's cell with the float32 parametrisation (a path it does not map is
 * invalid), counts DM_C, prunes with probability (DM_C - DM_T) / DM_C (Eq. 1;
 * Philox counter (path, 16, frame), exact on the 24-bit draw) marking first
 * and then editing the counts, and fills: the free paths in ascending order
 * take the cells' deficits in cell order and spread any rest evenly.  DM_T(c)
 * = floor(N (c + 1) / n) - floor(N c / n).  or_dm_reset sets DM_C = DM_T
 * (after a full trace). */
int32_t or_scene_set_dm(or_scene* s, const uint32_t rect[4], const uint32_t point[2]);
void or_dm_reset(or_scene* s);
uint32_t or_dm_cells(const or_scene* s, uint32_t light);
uint32_t or_dm_target(const or_scene* s, uint32_t light, uint32_t cell);
void or_dm_counts(const or_scene* s, uint32_t light, uint32_t* out);
void or_dm_set_counts(or_scene* s, uint32_t light, const uint32_t* in);
/* cell of a path (first photon x1, stored origin o) under the current pose, or -1 */
int32_t or_dm_cell_of(const or_scene* s, uint32_t light, const float x1[3], const float o[3]);
/* fraction of a turn of the angle of (x, y), as the parametrisation computes it */
float or_dm_turn(float x, float y);

/* Ascending list of the positions (into ids) whose replace bit is set;
 * returns the count (Sec. 5.2, pruned-paths array pattern). */
uint32_t or_compact(const uint32_t* info, uint32_t n, uint32_t* list);

/* Re-trace every listed path whose replace bit is set, from its start
 * vertex, at the current pose with the frame's random numbers. */
void or_retrace(const or_scene* s, const uint32_t* ids, uint32_t n, uint64_t seed,
                uint32_t frame, uint32_t* info, float* origin, or_photon* photons,
                uint32_t* amb, or_stats* st);

/* Deposit every stored photon's incident energy into a width x height
 * top-down XZ atlas over [x0,x1] x [z0,z1]; atlas is [height][width][3]
 * (accumulated, not cleared).  The texel index is computed in float32. */
void or_deposit(const uint32_t* info, uint32_t n, const or_photon* photons, uint32_t max_bounces,
                uint32_t width, uint32_t height, float x0, float z0, float x1, float z1,
                double* atlas);

/* The texel (tx, tz) or_deposit assigns to each stored photon: texels
 * [n][max_bounces][2], (-1, -1) past a path's photon count. */
void or_photon_texels(const uint32_t* info, uint32_t n, const or_photon* photons, uint32_t max_bounces,
                      uint32_t width, uint32_t height, float x0, float z0, float x1, float z1, int32_t* texels);

/* Screen-space photon splat (the renderer's "splat/gather" step of Fig. 2;
 * its splatting method is only cited, so a plain radius kernel): pinhole
 * camera at pos looking at target (up vector, vertical field of view fov_y in
 * radians, width x height pixels, pixel centres).  Every pixel's primary ray
 * finds its visible point p (normal facing the camera, albedo rho); every
 * photon x with energy E arriving on the visible side adds
 * rho/pi * E * 2 (1 - s^2) / (pi r^2), s = |p - x| / r < 1.  A photon whose
 * kernel cube reaches within 1e-3 diag of the camera plane is skipped.
 * image [height][width][3] (written), amb [height][width] (written). */
typedef struct {
  float pos[3], target[3], up[3];
  float fov_y;
  uint32_t width, height;
} or_camera;
void or_splat(const or_scene* s, const uint32_t* ids, uint32_t n, const uint32_t* info, const float* origin,
              const or_photon* photons, const or_camera* cam, double radius, double* image, uint8_t* amb);

/* Differentiable deposit model (no counterpart in the paper; used to rank the
 * paths to re-trace).  Every stored path keeps its triangles and sampled
 * directions; with parameters theta the emission point and direction follow
 * the light, each photon is re-found on its triangle's plane (translated with
 * its dynamic object) along its stored incoming direction, energies scale with
 * the light's intensity, and photons are splatted with the uniform cubic
 * B-spline over 4 x 4 texels (texel centres at half-integers, texels outside
 * the atlas dropped).  theta layout: for
 * every light pos[3], normal[3], intensity scale[1]; then for every dynamic
 * object (object order) its translation[3].  At theta = the current pose
 * (scale 1) the model reproduces the stored photons.
 * or_model_deposit adds the model atlas [h][w][3]; or_adjoint adds
 * dL/dtheta given G = dL/datlas and writes per-path scores
 * |sum_k,c dL/dE_kc E_kc| (may be NULL). */
uint32_t or_theta_size(const or_scene* s);
void or_theta_current(const or_scene* s, double* theta);
void or_model_deposit(const or_scene* s, const uint32_t* ids, uint32_t n, const uint32_t* info, const float* origin,
                      const or_photon* photons, const double* theta, uint32_t width, uint32_t height, float x0,
                      float z0, float x1, float z1, double* atlas);
void or_adjoint(const or_scene* s, const uint32_t* ids, uint32_t n, const uint32_t* info, const float* origin,
                const or_photon* photons, const double* theta, uint32_t width, uint32_t height, float x0, float z0,
                float x1, float z1, const double* G, double* dtheta, double* score);

/* Closest hit of one ray against the current pose (test helper): returns the
 * prim id or -1, writes the distance, ambiguity flag. */
int32_t or_closest_hit(const or_scene* s, const double o[3], const double d[3], double tlo,
                       int32_t exclude, double* t_out, int32_t* amb);

/* Decision script of one path.  Where a decision is ambiguous (see above),
 * alternative 0 is the FP64 decision and alternatives 1.. are the other
 * outcomes a perturbation within the band could give: the other side of a
 * box, plane, edge, light extent or Eq. 2 / AreClose threshold, the other
 * facing side or orthonormal-basis branch, and for a closest hit every
 * triangle that could be the nearest within the band (nearest first), or a
 * miss.  The j-th ambiguous decision met takes script[j] (alternative 0 past
 * the end of the script); ``pos`` counts the ambiguous decisions met so far
 * and ``n_alt_next`` receives the number of alternatives of the first one
 * past the script (left 0 if there is none).  With no script (NULL choice)
 * every decision is the FP64 one. */
typedef struct {
  const uint8_t* script;
  int32_t n_script;
  int32_t pos;
  int32_t n_alt_next;
  int32_t open;   /* set when a closest hit met a triangle whose crossing distance the band leaves
                     undetermined over more than 1e-4 diag (a ray running within eps of its plane):
                     a hit anywhere on that stretch is admissible, which no list of outcomes holds */
} or_choice;

/* One path through one step under a decision script (``ch`` carries the
 * script's position from call to call): the records of path ``pid`` --
 * info, origin[3], photons[B], amb -- are updated in place exactly as
 * or_trace / or_verify / or_retrace update them.  or_verify_path writes the
 * intersected-segment mask and returns -1 (doing nothing) for a scene with a
 * distribution map, whose prune and fill steps need every path at once. */
void or_trace_path(const or_scene* s, uint32_t pid, uint64_t seed, uint32_t frame, uint32_t* info, float* origin,
                   or_photon* photons, uint32_t* amb, or_choice* ch);
int32_t or_verify_path(const or_scene* s, uint32_t pid, int32_t mode, double tau, uint32_t flags, uint32_t* info,
                       float* origin, or_photon* photons, uint32_t* seg_mask, uint32_t* amb, or_choice* ch);
void or_retrace_path(const or_scene* s, uint32_t pid, uint64_t seed, uint32_t frame, uint32_t* info,
                     float* origin, or_photon* photons, uint32_t* amb, or_choice* ch);

/* Number of OpenMP threads the oracle uses. */
int32_t or_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
