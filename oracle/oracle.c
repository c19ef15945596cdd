/*
 * FP64 brute-force oracle for per-frame photon-path verification.
 * TEST INFRASTRUCTURE ONLY: see oracle.h for who may use it and why.
 *
 * Paper: Moreau, Doggett, Sintorn, "Path Verification for Dynamic Indirect
 * Illumination" (arXiv 2111.06906).  Each function names the passage it
 * follows.  Geometry is tested against every triangle, in double precision;
 * path records are FP32 and every step restarts from the stored record.
 *
 * Readings of the paper taken here (the paper is silent or ambiguous):
 *  - a photon record stores the hit position where Sec. 4 lists the incoming
 *    direction; directions are differences of consecutive positions;
 *  - "BRDF(Segment, NextSeg)" (Alg. 1) is the stored sample re-weighted for
 *    the new vertex:  E_N = E_i * rho' * max(0, n'_s . w') / (q_i * (n_s . w)),
 *    which equals E_O when nothing changed (Lambertian surfaces only, Sec. 6);
 *  - Eq. 2 is applied per RGB channel and all channels must pass;
 *  - AreClose (Alg. 1) = same primitive and |dx|_inf <= 1e-5 x diagonal; when
 *    it holds E_N := E_O;
 *  - after the skip branch of Alg. 1 the next segment is known valid and the
 *    check resumes with the segment after it;
 *  - a re-traced ray that misses everything truncates the path there;
 *  - area-light origins keep the stored direction and re-intersect the new
 *    light plane (Sec. 3.1); a path is invalid if the new origin leaves the
 *    rectangle, lies behind x1, or the direction leaves the emitting
 *    hemisphere; a tilted light re-weights the primary energy by
 *    (n'.d)/(n.d) and applies Eq. 2;
 *  - the point light's shadow-map check (Sec. 3.1) is an exact visibility ray.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define MAXL 4

struct or_scene {
  uint32_t n_tris, n_objects, B;
  double diag, eps, tmin, close_tol;
  float* verts;          /* [n_tris][9] as given */
  uint32_t* tri_object;  /* [n_tris] */
  uint8_t* dyn;          /* [n_objects] */
  float* albedo;         /* [n_objects][3] */
  double* world[2];      /* [n_tris][12] = v0,v1,v2,n (unnormalised) for pose 0=old, 1=new */
  uint32_t* obj_first;   /* CSR of triangles per object: [n_objects+1] */
  uint32_t* obj_tris;    /* [n_tris] */
  uint8_t* moved;        /* [n_objects] */
  uint32_t* moved_list;  /* [n_objects] */
  uint32_t n_moved;
  double* box;           /* [n_objects][2][6] lo/hi of old (0) and new (1) pose */
  float* xf_new;         /* [n_objects][12] current pose */
  int32_t* dyn_index;    /* [n_objects] position among the dynamic objects, -1 if static */
  uint32_t n_dynamic;
  or_light light[2][MAXL];
  uint32_t n_lights;
  uint32_t light_first[MAXL + 1];
  uint8_t light_moved[MAXL];
  uint8_t light_tilted[MAXL];
  /* distribution maps (Sec. 3.1): per light its resolution over the sample
   * dimensions (rectangle: x, y, theta, phi; point: theta, phi), cell count
   * and current counts DM_C (DM_T is computed as needed) */
  uint32_t dm_res[MAXL][4];
  uint32_t dm_dims[MAXL];
  uint32_t dm_cells[MAXL];
  uint32_t* dm_c[MAXL];
};

/* ------------------------------------------------------------------------ */
/* small vector helpers                                                       */
/* ------------------------------------------------------------------------ */
static inline double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static inline void sub3(const double* a, const double* b, double* r) {
  r[0] = a[0] - b[0]; r[1] = a[1] - b[1]; r[2] = a[2] - b[2];
}
static inline void cross3(const double* a, const double* b, double* r) {
  r[0] = a[1] * b[2] - a[2] * b[1];
  r[1] = a[2] * b[0] - a[0] * b[2];
  r[2] = a[0] * b[1] - a[1] * b[0];
}
static inline double norm3(const double* a) { return sqrt(dot3(a, a)); }
static inline void normalize3(double* a) {
  double l = norm3(a);
  a[0] /= l; a[1] /= l; a[2] /= l;
}
static inline void f2d(const float* f, double* d) { d[0] = f[0]; d[1] = f[1]; d[2] = f[2]; }
static inline double max3(const float* a) {
  double m = a[0];
  if (a[1] > m) m = a[1];
  if (a[2] > m) m = a[2];
  return m;
}

/* ------------------------------------------------------------------------ */
/* Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011): ten rounds of two     */
/* 32x32->64 multiplies; between rounds the key advances by the Weyl constants */
/* (golden ratio and sqrt(3)-1 in 32-bit fixed point).                         */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Four uniforms in [0,1) with 24 significant bits (exact in FP32 and FP64)
 * keyed by (path, vertex, frame).  Vertex 0: origin (u0,u1) and direction
 * (u2,u3) of an emission; vertex k>=1: direction (u0,u1) and Russian-roulette
 * draw (u2) of the bounce at photon k. */
static void rng4(uint64_t seed, uint32_t path, uint32_t vertex, uint32_t frame, double u[4]) {
  uint32_t ctr[4] = {path, vertex, frame, 0u};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t o[4];
  or_philox4x32_10(ctr, key, o);
  for (int j = 0; j < 4; ++j) u[j] = (double)(o[j] >> 8) * (1.0 / 16777216.0);
}

/* ------------------------------------------------------------------------ */
/* scene                                                                      */
/* ------------------------------------------------------------------------ */
or_scene* or_scene_create(const float* verts, uint32_t n_tris, const uint32_t* tri_object,
                          uint32_t n_objects, const uint8_t* object_dynamic, const float* albedo,
                          double diag, uint32_t max_bounces) {
  or_scene* s = (or_scene*)calloc(1, sizeof(or_scene));
  s->n_tris = n_tris;
  s->n_objects = n_objects;
  s->B = max_bounces;
  s->diag = diag;
  s->eps = 1e-6 * diag;
  s->tmin = 1e-5 * diag;
  s->close_tol = 1e-5 * diag;
  s->verts = (float*)malloc(sizeof(float) * 9 * (size_t)n_tris);
  memcpy(s->verts, verts, sizeof(float) * 9 * (size_t)n_tris);
  s->tri_object = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n_tris);
  memcpy(s->tri_object, tri_object, sizeof(uint32_t) * (size_t)n_tris);
  s->dyn = (uint8_t*)malloc(n_objects ? n_objects : 1);
  memcpy(s->dyn, object_dynamic, n_objects);
  s->albedo = (float*)malloc(sizeof(float) * 3 * (size_t)(n_objects ? n_objects : 1));
  memcpy(s->albedo, albedo, sizeof(float) * 3 * (size_t)n_objects);
  for (int p = 0; p < 2; ++p) s->world[p] = (double*)malloc(sizeof(double) * 12 * (size_t)(n_tris ? n_tris : 1));
  s->obj_first = (uint32_t*)calloc((size_t)n_objects + 1, sizeof(uint32_t));
  s->obj_tris = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n_tris ? n_tris : 1));
  for (uint32_t t = 0; t < n_tris; ++t) s->obj_first[tri_object[t] + 1]++;
  for (uint32_t o = 0; o < n_objects; ++o) s->obj_first[o + 1] += s->obj_first[o];
  uint32_t* fill = (uint32_t*)calloc((size_t)n_objects + 1, sizeof(uint32_t));
  for (uint32_t t = 0; t < n_tris; ++t) {
    uint32_t o = tri_object[t];
    s->obj_tris[s->obj_first[o] + fill[o]++] = t;
  }
  free(fill);
  s->moved = (uint8_t*)calloc(n_objects ? n_objects : 1, 1);
  s->moved_list = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n_objects ? n_objects : 1));
  s->box = (double*)malloc(sizeof(double) * 12 * (size_t)(n_objects ? n_objects : 1));
  s->xf_new = (float*)calloc(12 * (size_t)(n_objects ? n_objects : 1), sizeof(float));
  s->dyn_index = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_objects ? n_objects : 1));
  s->n_dynamic = 0;
  for (uint32_t o = 0; o < n_objects; ++o) s->dyn_index[o] = object_dynamic[o] ? (int32_t)s->n_dynamic++ : -1;
  return s;
}

void or_scene_destroy(or_scene* s) {
  if (!s) return;
  free(s->verts); free(s->tri_object); free(s->dyn); free(s->albedo);
  free(s->world[0]); free(s->world[1]);
  free(s->obj_first); free(s->obj_tris); free(s->moved); free(s->moved_list); free(s->box);
  free(s->xf_new); free(s->dyn_index);
  for (int l = 0; l < MAXL; ++l) free(s->dm_c[l]);
  free(s);
}

/* World triangles at a pose: static objects as given, dynamic ones through
 * their 3x4 transform [R|t] (row-major), in double precision. */
static void pose_world(or_scene* s, const float* xf, double* W) {
  for (uint32_t t = 0; t < s->n_tris; ++t) {
    uint32_t o = s->tri_object[t];
    const float* v = s->verts + 9 * (size_t)t;
    double* w = W + 12 * (size_t)t;
    for (int k = 0; k < 3; ++k) {
      if (s->dyn[o]) {
        const float* m = xf + 12 * (size_t)o;
        for (int r = 0; r < 3; ++r)
          w[3 * k + r] = (double)m[4 * r + 0] * v[3 * k + 0] + (double)m[4 * r + 1] * v[3 * k + 1] +
                         (double)m[4 * r + 2] * v[3 * k + 2] + (double)m[4 * r + 3];
      } else {
        w[3 * k + 0] = v[3 * k + 0];
        w[3 * k + 1] = v[3 * k + 1];
        w[3 * k + 2] = v[3 * k + 2];
      }
    }
    double e1[3], e2[3];
    sub3(w + 3, w, e1);
    sub3(w + 6, w, e2);
    cross3(e1, e2, w + 9);
  }
}

void or_scene_set_poses(or_scene* s, const float* xform_old, const float* xform_new,
                        const or_light* lights_old, const or_light* lights_new, uint32_t n_lights) {
  pose_world(s, xform_old, s->world[0]);
  pose_world(s, xform_new, s->world[1]);
  memcpy(s->xf_new, xform_new, sizeof(float) * 12 * (size_t)s->n_objects);
  s->n_moved = 0;
  for (uint32_t o = 0; o < s->n_objects; ++o) {
    s->moved[o] = s->dyn[o] && memcmp(xform_old + 12 * (size_t)o, xform_new + 12 * (size_t)o, 12 * sizeof(float)) != 0;
    if (s->moved[o]) s->moved_list[s->n_moved++] = o;
    for (int p = 0; p < 2; ++p) {
      double* b = s->box + 12 * (size_t)o + 6 * p;
      b[0] = b[1] = b[2] = INFINITY;
      b[3] = b[4] = b[5] = -INFINITY;
      for (uint32_t k = s->obj_first[o]; k < s->obj_first[o + 1]; ++k) {
        const double* w = s->world[p] + 12 * (size_t)s->obj_tris[k];
        for (int v = 0; v < 3; ++v)
          for (int a = 0; a < 3; ++a) {
            if (w[3 * v + a] < b[a]) b[a] = w[3 * v + a];
            if (w[3 * v + a] > b[3 + a]) b[3 + a] = w[3 * v + a];
          }
      }
    }
  }
  s->n_lights = n_lights > MAXL ? MAXL : n_lights;
  s->light_first[0] = 0;
  for (uint32_t l = 0; l < s->n_lights; ++l) {
    s->light[0][l] = lights_old[l];
    s->light[1][l] = lights_new[l];
    s->light_first[l + 1] = s->light_first[l] + lights_new[l].n_paths;
    const or_light *a = &lights_old[l], *b = &lights_new[l];
    s->light_moved[l] = memcmp(a->pos, b->pos, sizeof a->pos) != 0 || memcmp(a->normal, b->normal, sizeof a->normal) != 0 ||
                        memcmp(a->tangent, b->tangent, sizeof a->tangent) != 0 || memcmp(a->size, b->size, sizeof a->size) != 0;
    s->light_tilted[l] = memcmp(a->normal, b->normal, sizeof a->normal) != 0;
  }
}

static uint32_t light_of(const or_scene* s, uint32_t pid) {
  for (uint32_t l = 0; l + 1 < s->n_lights; ++l)
    if (pid < s->light_first[l + 1]) return l;
  return s->n_lights ? s->n_lights - 1 : 0;
}

/* ------------------------------------------------------------------------ */
/* decision scripts                                                          */
/* ------------------------------------------------------------------------ */
/* An ambiguous decision with n_alt possible outcomes: the outcome the script
 * gives it (0, the FP64 decision, without a script or past its end). */
static int choose(or_choice* ch, int n_alt) {
  if (!ch || n_alt < 2) return 0;
  const int j = ch->pos++;
  if (j < ch->n_script) return ch->script[j] < n_alt ? ch->script[j] : 0;
  if (j == ch->n_script && ch->n_alt_next == 0) ch->n_alt_next = n_alt;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* ray / triangle with ambiguity                                             */
/* ------------------------------------------------------------------------ */
typedef struct {
  double t, epst;
  int32_t prim;
  int hit, amb;
} cand_t;

/* A candidate whose crossing distance the band leaves undetermined over more
 * than 1e-4 diag (epst = eps / |cos| with eps = 1e-6 diag): the ray runs
 * within eps of the triangle's plane along that stretch. */
static int cand_open(const or_scene* s, const cand_t* c) { return c->amb && c->epst > 100.0 * s->eps; }

/* Classify triangle T (v0,v1,v2,n) against the ray o + t d (|d| = 1) for
 * t in (tlo, thi).  Hit: the ray meets the closed triangle inside the open
 * range.  Ambiguous: the ray line passes within eps of an edge line
 * (distance measured between the two lines), or the plane crossing lies
 * within eps/|cos| of a range end, or the ray runs parallel to the plane
 * within eps of it.  Returns 0 for a robust miss. */
static int tri_classify(const double* T, const double* o, const double* d, double tlo, double thi,
                        double eps, cand_t* c) {
  const double* n = T + 9;
  double nn = norm3(n);
  if (nn == 0.0) return 0;
  double nd = dot3(n, d);
  double cosang = nd / nn;
  double v0o[3];
  sub3(T, o, v0o);
  double pd = dot3(n, v0o) / nn;
  if (fabs(cosang) < 1e-12) {
    if (fabs(pd) < eps) {
      c->t = tlo; c->epst = INFINITY; c->hit = 0; c->amb = 1;
      return 1;
    }
    return 0;
  }
  double t = pd / cosang;
  double epst = eps / fabs(cosang);
  if (t <= tlo - epst || t >= thi + epst) return 0;
  double sgn = nd > 0.0 ? 1.0 : -1.0;
  double m = INFINITY;
  for (int e = 0; e < 3; ++e) {
    const double* a = T + 3 * e;
    const double* b = T + 3 * ((e + 1) % 3);
    double ab[3], cr[3], ao[3];
    sub3(b, a, ab);
    cross3(ab, d, cr);
    double cl = norm3(cr);
    sub3(a, o, ao);
    double dist = sgn * dot3(ao, cr) / cl;
    if (dist < m) m = dist;
  }
  if (m <= -eps) return 0;
  c->t = t;
  c->epst = epst;
  c->hit = (m >= 0.0) && t > tlo && t < thi;
  c->amb = (m < eps) || fabs(t - tlo) < epst || (isfinite(thi) && fabs(t - thi) < epst);
  return 1;
}

typedef struct {
  cand_t* c;
  size_t n, cap;
} candvec;

static void cv_push(candvec* v, const cand_t* c) {
  if (v->n == v->cap) {
    v->cap = v->cap ? 2 * v->cap : 64;
    v->c = (cand_t*)realloc(v->c, v->cap * sizeof(cand_t));
  }
  v->c[v->n++] = *c;
}

/* Closest hit over every triangle at pose p, t in (tlo, inf), skipping
 * primitive ``exclude``.  Ambiguous if the nearest result could change under
 * the eps perturbation: the nearest hit is itself ambiguous, an ambiguous
 * triangle lies in front of (or level with) it, or another hit lies within
 * the combined t tolerance. */
#define OR_MAX_HIT_ALTS 8

static int32_t closest_hit(const or_scene* s, int p, const double* o, const double* d, double tlo,
                           int32_t exclude, double* t_out, int* amb_out, or_choice* ch) {
  candvec cv = {0, 0, 0};
  int32_t best = -1;
  double best_t = INFINITY;
  const double* W = s->world[p];
  for (uint32_t t = 0; t < s->n_tris; ++t) {
    if ((int32_t)t == exclude) continue;
    cand_t c;
    if (!tri_classify(W + 12 * (size_t)t, o, d, tlo, INFINITY, s->eps, &c)) continue;
    c.prim = (int32_t)t;
    cv_push(&cv, &c);
    if (c.hit && c.t < best_t) {
      best_t = c.t;
      best = (int32_t)t;
    }
  }
  int amb = 0;
  double best_eps = 0.0;
  for (size_t i = 0; i < cv.n; ++i)
    if (cv.c[i].prim == best) {
      best_eps = cv.c[i].epst;
      if (cv.c[i].amb) amb = 1;
    }
  for (size_t i = 0; i < cv.n; ++i) {
    const cand_t* c = &cv.c[i];
    if (c->prim == best) continue;
    if (best < 0) {
      if (c->amb) amb = 1;
      continue;
    }
    if (c->amb && c->t - c->epst < best_t + best_eps) amb = 1;
    if (c->hit && fabs(c->t - best_t) < c->epst + best_eps) amb = 1;
  }
  if (amb && ch) {
    /* the outcomes the band admits: the FP64 nearest hit first; then, nearest
     * first, every triangle that could be hit in front of it or level with it;
     * and if the nearest hit could itself be missed, the next hit (or a miss) */
    int32_t alt_p[OR_MAX_HIT_ALTS];
    double alt_t[OR_MAX_HIT_ALTS];
    int na = 0;
    alt_p[na] = best; alt_t[na] = best_t; ++na;
    int best_amb = 0;
    for (size_t i = 0; i < cv.n; ++i)
      if (cv.c[i].prim == best && cv.c[i].amb) best_amb = 1;
    for (;;) {                                   /* insertion by distance, skipping what is listed */
      const cand_t* pick = NULL;
      for (size_t i = 0; i < cv.n; ++i) {
        const cand_t* c = &cv.c[i];
        int listed = 0;
        for (int k = 0; k < na; ++k) listed |= alt_p[k] == c->prim;
        if (listed) continue;
        const int admit = best < 0 ? c->amb
                                   : (c->amb && c->t - c->epst < best_t + best_eps) ||
                                         (c->hit && fabs(c->t - best_t) < c->epst + best_eps);
        if (admit && (!pick || c->t < pick->t)) pick = c;
      }
      if (!pick || na == OR_MAX_HIT_ALTS) break;
      alt_p[na] = pick->prim; alt_t[na] = pick->t; ++na;
    }
    if (best >= 0 && best_amb && na < OR_MAX_HIT_ALTS) {
      const cand_t* next = NULL;                 /* the nearest other hit, if the nearest is missed */
      for (size_t i = 0; i < cv.n; ++i) {
        const cand_t* c = &cv.c[i];
        if (c->prim == best || !c->hit) continue;
        if (!next || c->t < next->t) next = c;
      }
      int listed = 0;
      for (int k = 0; k < na; ++k) listed |= next ? alt_p[k] == next->prim : alt_p[k] < 0;
      if (!listed) {
        alt_p[na] = next ? next->prim : -1;
        alt_t[na] = next ? next->t : INFINITY;
        ++na;
      }
    }
    for (int k = 0; k < na; ++k)
      for (size_t i = 0; i < cv.n; ++i)
        if (cv.c[i].prim == alt_p[k] && cand_open(s, &cv.c[i])) ch->open = 1;
    const int k = choose(ch, na);
    best = alt_p[k];
    best_t = alt_t[k];
  }
  free(cv.c);
  *t_out = best_t;
  *amb_out = amb;
  return best;
}

int32_t or_closest_hit(const or_scene* s, const double o[3], const double d[3], double tlo,
                       int32_t exclude, double* t_out, int32_t* amb) {
  int a = 0;
  int32_t r = closest_hit(s, 1, o, d, tlo, exclude, t_out, &a, NULL);
  *amb = a;
  return r;
}

/* Any hit of the segment a->b, interior (tmin, len - tmin), against a set of
 * triangles (all triangles if list == NULL) at pose p.  *amb is set when no
 * robust hit exists but some triangle is ambiguous. */
static int any_hit(const or_scene* s, int p, const uint32_t* list, uint32_t count, const double* a,
                   const double* b, int32_t exclude, int* amb, or_choice* ch) {
  double d[3];
  sub3(b, a, d);
  double len = norm3(d);
  *amb = 0;
  if (!(len > 0.0)) return 0;
  d[0] /= len; d[1] /= len; d[2] /= len;
  double thi = len - s->tmin;
  int any_amb = 0, any = 0;
  const double* W = s->world[p];
  uint32_t n = list ? count : s->n_tris;
  for (uint32_t k = 0; k < n; ++k) {
    uint32_t t = list ? list[k] : k;
    if ((int32_t)t == exclude) continue;
    cand_t c;
    if (!tri_classify(W + 12 * (size_t)t, a, d, s->tmin, thi, s->eps, &c)) continue;
    if (c.hit) any = 1;
    if (c.hit && !c.amb) {
      *amb = 0;
      return 1;
    }
    if (c.amb) any_amb = 1;
  }
  *amb = any_amb;
  if (any_amb && choose(ch, 2)) any = !any;       /* only ambiguous triangles decide: either answer */
  return any;
}

/* Closed segment a->b against the closed box [lo,hi] (slab test); the result
 * is ambiguous when the box grown by eps and the box shrunk by eps (never
 * below zero thickness) disagree. */
static int seg_box_one(const double* a, const double* b, const double* lo, const double* hi) {
  double t0 = 0.0, t1 = 1.0;
  for (int k = 0; k < 3; ++k) {
    if (lo[k] > hi[k]) return 0;
    double dk = b[k] - a[k];
    if (dk == 0.0) {
      if (a[k] < lo[k] || a[k] > hi[k]) return 0;
      continue;
    }
    double u0 = (lo[k] - a[k]) / dk, u1 = (hi[k] - a[k]) / dk;
    if (u0 > u1) { double tt = u0; u0 = u1; u1 = tt; }
    if (u0 > t0) t0 = u0;
    if (u1 < t1) t1 = u1;
    if (t0 > t1) return 0;
  }
  return 1;
}

static int seg_box(const double* a, const double* b, const double* box /* lo[3],hi[3] */, double eps, int* amb) {
  double glo[3], ghi[3], slo[3], shi[3];
  for (int k = 0; k < 3; ++k) {
    /* shrinking stops at zero thickness: a flat box stays a flat box */
    double e = fmin(eps, 0.5 * (box[3 + k] - box[k]));
    glo[k] = box[k] - eps; ghi[k] = box[3 + k] + eps;
    slo[k] = box[k] + e; shi[k] = box[3 + k] - e;
  }
  int g = seg_box_one(a, b, glo, ghi);
  int sh = seg_box_one(a, b, slo, shi);
  int exact = seg_box_one(a, b, box, box + 3);
  *amb = g != sh;
  return exact;
}

/* ------------------------------------------------------------------------ */
/* sampling (Sec. 3, "generate rays")                                         */
/* ------------------------------------------------------------------------ */
static void unit_normal(const or_scene* s, int p, int32_t prim, double n[3]) {
  const double* w = s->world[p] + 12 * (size_t)prim;
  n[0] = w[9]; n[1] = w[10]; n[2] = w[11];
  normalize3(n);
}

/* Orthonormal basis around unit n (Duff, Burgess, Christensen, Hery, Kensler,
 * Liani, Villemin, JCGT 2017); the branch sg = +1 is the one taken for
 * n.z >= 0 and sg = -1 the one for n.z < 0. */
static void onb(const double* n, double sg, double* b1, double* b2) {
  double a = -1.0 / (sg + n[2]);
  double b = n[0] * n[1] * a;
  b1[0] = 1.0 + sg * n[0] * n[0] * a; b1[1] = sg * b; b1[2] = -sg * n[0];
  b2[0] = b; b2[1] = sg + n[1] * n[1] * a; b2[2] = -n[1];
}

/* Cosine-weighted direction about unit n (Malley's method: uniform disk point
 * lifted to the hemisphere). */
static void cosine_dir(const double* n, const double* b1, const double* b2, double u0, double u1, double* d) {
  double r = sqrt(u0);
  double ph = 2.0 * M_PI * u1;
  double x = r * cos(ph), y = r * sin(ph), z = sqrt(fmax(0.0, 1.0 - u0));
  for (int k = 0; k < 3; ++k) d[k] = x * b1[k] + y * b2[k] + z * n[k];
  normalize3(d);
}

/* Emission from light L with uniforms u: point = uniform sphere, rectangle =
 * uniform position and cosine-weighted direction about its normal. */
static void emit(const or_light* L, const double* u, double* o, double* d) {
  if (L->type == 0) {
    f2d(L->pos, o);
    double z = 1.0 - 2.0 * u[2];
    double r = sqrt(fmax(0.0, 1.0 - z * z));
    double ph = 2.0 * M_PI * u[3];
    d[0] = r * cos(ph); d[1] = r * sin(ph); d[2] = z;
    normalize3(d);
  } else {
    double c[3], n[3], t[3], b[3];
    f2d(L->pos, c); f2d(L->normal, n); f2d(L->tangent, t);
    cross3(n, t, b);
    double su = (u[0] - 0.5) * L->size[0], sv = (u[1] - 0.5) * L->size[1];
    for (int k = 0; k < 3; ++k) o[k] = c[k] + su * t[k] + sv * b[k];
    cosine_dir(n, t, b, u[2], u[3], d);
  }
}

/* Facing normal: the geometric normal flipped against the incoming ray.
 * With ``branch`` the orthonormal basis branch about it too (+1 for
 * n.z >= 0).  Either decision may be ambiguous: a script then picks it. */
static void facing(const or_scene* s, int p, int32_t prim, const double* d_in, double* ns, int* amb,
                   or_choice* ch, double* branch) {
  double n[3];
  unit_normal(s, p, prim, n);
  double c = dot3(n, d_in);
  double sg = c < 0.0 ? 1.0 : -1.0;
  if (fabs(c) < 1e-6) {
    *amb = 1;
    if (choose(ch, 2)) sg = -sg;
  }
  ns[0] = sg * n[0]; ns[1] = sg * n[1]; ns[2] = sg * n[2];
  double br = ns[2] >= 0.0 ? 1.0 : -1.0;
  if (ns[2] != 0.0 && fabs(ns[2]) < 1e-6) {   /* basis branch near n.z = 0 */
    *amb = 1;
    if (branch && choose(ch, 2)) br = -br;
  }
  if (branch) *branch = br;
}

static inline uint32_t info_nseg(uint32_t w) { return (w >> OR_INFO_NSEG_SHIFT) & 15u; }
static inline uint32_t info_start(uint32_t w) { return (w >> OR_INFO_START_SHIFT) & 15u; }
static inline uint32_t info_make(uint32_t cell, uint32_t nseg, uint32_t start, int replace, int reuse) {
  return (cell & OR_INFO_CELL_MASK) | (nseg << OR_INFO_NSEG_SHIFT) | (start << OR_INFO_START_SHIFT) |
         (replace ? OR_INFO_REPLACE : 0u) | (reuse ? OR_INFO_REUSE_LIGHT : 0u);
}

/* ------------------------------------------------------------------------ */
/* distribution maps (Sec. 3.1)                                              */
/* ------------------------------------------------------------------------ */
/* A cell is a box of the emission's sample space: a rectangle's uniforms
 * (u0, u1) pick the point and (u2, u3) = (sin^2 theta, phi / 2 pi) the
 * cosine-weighted direction; a point light's (u2, u3) = ((1 - z) / 2,
 * phi / 2 pi) pick the direction.  Every cell therefore has the same
 * emission probability, and sampling restricted to a cell is a uniform draw
 * inside its box.  The cell of a path is decided in float32 with correctly
 * rounded +, -, *, / and sqrt only (compiled without contraction), from the
 * stored float32 photon and origin and the float32 light pose. */
static const int dm_u_rect[4] = {0, 1, 2, 3};
static const int dm_u_point[2] = {2, 3};

/* Fraction of a full turn of the angle of (x, y), in [0, 1): the angle to the
 * nearer axis from two half-angle steps atan t = 2 atan(t / (1 + sqrt(1 + t^2)))
 * and the Gregory series to t^9 (|t| <= tan(pi/16), truncation < 2e-9). */
float or_dm_turn(float x, float y) {
  const float ax = fabsf(x), ay = fabsf(y);
  const float mx = ax > ay ? ax : ay, mn = ax > ay ? ay : ax;
  if (!(mx > 0.0f)) return 0.0f;
  float t = mn / mx;
  t = t / (1.0f + sqrtf(1.0f + t * t));
  t = t / (1.0f + sqrtf(1.0f + t * t));
  const float q = t * t;
  /* 1/9, 1/7, 1/5, 1/3, pi/2, pi, 2 pi rounded to float32 */
  float a = 0x1.c71c72p-4f;
  a = 0x1.24924ap-3f - q * a;
  a = 0x1.99999ap-3f - q * a;
  a = 0x1.555556p-2f - q * a;
  a = 1.0f - q * a;
  a = 4.0f * (t * a);
  if (ay > ax) a = 0x1.921fb6p+0f - a;
  if (x < 0.0f) a = 0x1.921fb6p+1f - a;
  if (y < 0.0f) a = 0x1.921fb6p+2f - a;
  const float f = a / 0x1.921fb6p+2f;
  return f < 1.0f ? f : 0.0f;
}

static inline float dotf(const float* a, const float* b) { return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2]; }

/* The light's bitangent n x t: products exact in double, one rounding each
 * way (as the pose is prepared for the GPU). */
static void bitangent_f(const or_light* L, float* b) {
  const double n0 = L->normal[0], n1 = L->normal[1], n2 = L->normal[2];
  const double t0 = L->tangent[0], t1 = L->tangent[1], t2 = L->tangent[2];
  b[0] = (float)(n1 * t2 - n2 * t1);
  b[1] = (float)(n2 * t0 - n0 * t2);
  b[2] = (float)(n0 * t1 - n1 * t0);
}

/* Sample-space coordinates of a path under pose L (the parametrisation
 * function of Sec. 3.1); 0 when the path does not come from the light. */
static int dm_param(const or_light* L, const float* x1, const float* o, float* u) {
  if (L->type == 0) {
    const float dx[3] = {x1[0] - L->pos[0], x1[1] - L->pos[1], x1[2] - L->pos[2]};
    const float len = sqrtf(dotf(dx, dx));
    if (!(len > 0.0f)) return 0;
    const float d[3] = {dx[0] / len, dx[1] / len, dx[2] / len};
    u[2] = (1.0f - d[2]) * 0.5f;
    u[3] = or_dm_turn(d[0], d[1]);
    return u[2] >= 0.0f && u[2] < 1.0f;
  }
  const float dv[3] = {x1[0] - o[0], x1[1] - o[1], x1[2] - o[2]};
  const float len = sqrtf(dotf(dv, dv));
  if (!(len > 0.0f)) return 0;
  const float d[3] = {dv[0] / len, dv[1] / len, dv[2] / len};
  float b[3];
  bitangent_f(L, b);
  const float nd = dotf(L->normal, d);
  if (!(nd > 0.0f)) return 0;
  const float x1c[3] = {x1[0] - L->pos[0], x1[1] - L->pos[1], x1[2] - L->pos[2]};
  const float tp = dotf(L->normal, x1c) / nd;
  if (!(tp > 0.0f)) return 0;
  const float rel[3] = {x1c[0] - tp * d[0], x1c[1] - tp * d[1], x1c[2] - tp * d[2]};
  u[0] = dotf(L->tangent, rel) / L->size[0] + 0.5f;
  u[1] = dotf(b, rel) / L->size[1] + 0.5f;
  const float dx = dotf(d, L->tangent), dy = dotf(d, b);
  u[2] = dx * dx + dy * dy;
  u[3] = or_dm_turn(dx, dy);
  for (int k = 0; k < 4; ++k)
    if (!(u[k] >= 0.0f && u[k] < 1.0f)) return 0;
  return 1;
}

/* Cell of sample-space coordinates u (row-major over the light's dimensions). */
static uint32_t dm_cell_of_u(const or_scene* s, uint32_t l, const float* u) {
  const int* ux = s->dm_dims[l] == 4 ? dm_u_rect : dm_u_point;
  uint32_t c = 0;
  for (uint32_t k = 0; k < s->dm_dims[l]; ++k) {
    const uint32_t n = s->dm_res[l][k];
    uint32_t i = (uint32_t)floorf(u[ux[k]] * (float)n);
    if (i >= n) i = n - 1;
    c = c * n + i;
  }
  return c;
}

int32_t or_dm_cell_of(const or_scene* s, uint32_t light, const float x1[3], const float o[3]) {
  if (light >= s->n_lights || !s->dm_c[light]) return -1;
  float u[4];
  if (!dm_param(&s->light[1][light], x1, o, u)) return -1;
  return (int32_t)dm_cell_of_u(s, light, u);
}

/* DM_T: N paths spread over the cells as evenly as integers allow. */
uint32_t or_dm_target(const or_scene* s, uint32_t l, uint32_t c) {
  const uint64_t N = s->light[1][l].n_paths, n = s->dm_cells[l];
  return (uint32_t)(((uint64_t)(c + 1) * N) / n - ((uint64_t)c * N) / n);
}

/* Cell of the j-th path of a light in a full trace: path j lies in cell c
 * when floor(N c / n) <= j < floor(N (c + 1) / n), so DM_C = DM_T exactly. */
static uint32_t dm_stratified(const or_scene* s, uint32_t l, uint32_t j) {
  const uint64_t N = s->light[1][l].n_paths, n = s->dm_cells[l];
  return (uint32_t)((((uint64_t)j + 1) * n - 1) / N);
}

/* Restrict the uniforms of an emission to cell c: u_k' = (i_k + u_k) / n_k,
 * rounded in float32 (each u_k has 24 bits and is exact in float32). */
static void dm_restrict(const or_scene* s, uint32_t l, uint32_t c, double* u) {
  const int* ux = s->dm_dims[l] == 4 ? dm_u_rect : dm_u_point;
  for (int k = (int)s->dm_dims[l] - 1; k >= 0; --k) {
    const uint32_t n = s->dm_res[l][k];
    const uint32_t i = c % n;
    c /= n;
    const float v = ((float)i + (float)u[ux[k]]) / (float)n;
    u[ux[k]] = (double)v;
  }
}

int32_t or_scene_set_dm(or_scene* s, const uint32_t rect[4], const uint32_t point[2]) {
  for (uint32_t l = 0; l < s->n_lights; ++l) {
    free(s->dm_c[l]);
    s->dm_c[l] = NULL;
    const int rectl = s->light[1][l].type != 0;
    const uint32_t dims = rectl ? 4u : 2u;
    uint64_t cells = 1;
    for (uint32_t k = 0; k < dims; ++k) {
      const uint32_t r = rectl ? rect[k] : point[k];
      if (r == 0) { cells = 0; break; }
      s->dm_res[l][k] = r;
      cells *= r;
    }
    if (cells == 0) continue;                 /* no map for this light */
    if (cells > (1u << 20)) return -1;        /* the info word holds light << 20 | cell */
    s->dm_dims[l] = dims;
    s->dm_cells[l] = (uint32_t)cells;
    s->dm_c[l] = (uint32_t*)calloc(cells, sizeof(uint32_t));
  }
  return 0;
}

void or_dm_reset(or_scene* s) {
  for (uint32_t l = 0; l < s->n_lights; ++l)
    if (s->dm_c[l])
      for (uint32_t c = 0; c < s->dm_cells[l]; ++c) s->dm_c[l][c] = or_dm_target(s, l, c);
}

uint32_t or_dm_cells(const or_scene* s, uint32_t light) { return light < s->n_lights && s->dm_c[light] ? s->dm_cells[light] : 0; }

void or_dm_counts(const or_scene* s, uint32_t light, uint32_t* out) {
  if (light < s->n_lights && s->dm_c[light]) memcpy(out, s->dm_c[light], sizeof(uint32_t) * s->dm_cells[light]);
}

void or_dm_set_counts(or_scene* s, uint32_t light, const uint32_t* in) {
  if (light < s->n_lights && s->dm_c[light]) memcpy(s->dm_c[light], in, sizeof(uint32_t) * s->dm_cells[light]);
}

/* Extend a path (Fig. 2 "generate rays" / "trace rays" loop): k photons are
 * stored already.  For k == 0 the first ray (o, d) carrying E is given;
 * for k >= 1 the path first scatters at photon k (Russian roulette with
 * q = max albedo, cosine-weighted direction about the facing normal,
 * E_{k+1} = E_k * albedo / q).  Returns the new photon count; rays[0]
 * counts the rays traced, rays[1] those whose answer is ambiguous. */
static uint32_t extend_path(const or_scene* s, uint32_t pid, uint64_t seed, uint32_t frame, uint32_t k,
                            double* o, double* d, double* E, double radius, const float* origin,
                            or_photon* ph, uint32_t* amb, uint64_t rays[2], or_choice* ch) {
  int32_t excl = -1;
  for (;;) {
    if (k >= 1) {
      if (k >= s->B) break;
      or_photon* v = &ph[k - 1];
      double u[4];
      rng4(seed, pid, k, frame, u);
      const float* alb = s->albedo + 3 * (size_t)s->tri_object[v->prim];
      double q = max3(alb);
      if (!(u[2] < q)) break;
      double xin[3], xk[3], din[3];
      if (k == 1) f2d(origin, xin); else f2d(ph[k - 2].pos, xin);
      f2d(v->pos, xk);
      sub3(xk, xin, din);
      normalize3(din);
      double ns[3], b1[3], b2[3], br;
      int a = 0;
      facing(s, 1, v->prim, din, ns, &a, ch, &br);
      if (a) *amb |= OR_AMB_TRACE;
      onb(ns, br, b1, b2);
      cosine_dir(ns, b1, b2, u[0], u[1], d);
      for (int c = 0; c < 3; ++c) E[c] = (double)v->E[c] * (double)alb[c] / q;
      f2d(v->pos, o);
      excl = v->prim;
      radius = v->radius;
    }
    double t;
    int a = 0;
    int32_t prim = closest_hit(s, 1, o, d, s->tmin, excl, &t, &a, ch);
    rays[0]++;
    if (a) {
      *amb |= OR_AMB_TRACE;
      rays[1]++;
    }
    if (prim < 0) break;
    or_photon* v = &ph[k];
    for (int c = 0; c < 3; ++c) {
      v->pos[c] = (float)(o[c] + t * d[c]);
      v->E[c] = (float)E[c];
    }
    v->prim = prim;
    v->radius = (float)(radius + t);
    ++k;
  }
  return k;
}

/* One path traced from the light; adds its rays and ambiguous rays to rays[2]. */
static void trace_path(const or_scene* s, uint32_t pid, uint64_t seed, uint32_t frame, uint32_t* info,
                       float* org, or_photon* ph, uint32_t* amb, uint64_t rays[2], or_choice* ch) {
  uint32_t l = light_of(s, pid);
  const or_light* L = &s->light[1][l];
  double u[4], o[3], d[3], E[3];
  rng4(seed, pid, 0, frame, u);
  uint32_t cell = 0;
  if (s->dm_c[l]) {                          /* stratified over the distribution map */
    cell = dm_stratified(s, l, pid - s->light_first[l]);
    dm_restrict(s, l, cell, u);
  }
  emit(L, u, o, d);
  for (int c = 0; c < 3; ++c) E[c] = (double)L->power[c] / (double)L->n_paths;
  for (int c = 0; c < 3; ++c) org[c] = (float)o[c];
  f2d(org, o);
  *amb = 0;
  uint32_t k = extend_path(s, pid, seed, frame, 0, o, d, E, 0.0, org, ph, amb, rays, ch);
  *info = info_make((l << 20) | cell, k, 0, 0, 0);
}

void or_trace(const or_scene* s, const uint32_t* ids, uint32_t n, uint64_t seed, uint32_t frame,
              uint32_t* info, float* origin, or_photon* photons, uint32_t* amb, or_stats* st) {
  uint64_t rays = 0, rays_a = 0;
#pragma omp parallel for schedule(dynamic, 8) reduction(+ : rays, rays_a)
  for (uint32_t i = 0; i < n; ++i) {
    uint64_t r[2] = {0, 0};
    trace_path(s, ids[i], seed, frame, &info[i], origin + 3 * (size_t)i, photons + (size_t)i * s->B, &amb[i], r,
               NULL);
    rays += r[0];
    rays_a += r[1];
  }
  if (st) {
    st->paths += n;
    st->trace_rays += rays;
    st->rays_amb += rays_a;
  }
}

void or_trace_path(const or_scene* s, uint32_t pid, uint64_t seed, uint32_t frame, uint32_t* info, float* origin,
                   or_photon* photons, uint32_t* amb, or_choice* ch) {
  uint64_t r[2] = {0, 0};
  trace_path(s, pid, seed, frame, info, origin, photons, amb, r, ch);
}

/* ------------------------------------------------------------------------ */
/* verification                                                              */
/* ------------------------------------------------------------------------ */

/* Eq. 2 per channel: -T*E_O <= E_N - E_O <= T*E_O.  *near is set on a
 * near-tie (| |E_N - E_O| - T*E_O | <= 1e-6 E_O). */
static int energy_close(const double* EN, const float* EOf, double tau, int* near) {
  int ok = 1;
  for (int c = 0; c < 3; ++c) {
    double EO = EOf[c];
    double diff = EN[c] - EO;
    if (EO == 0.0) {
      if (EN[c] != 0.0) ok = 0;
      continue;
    }
    double lim = tau * EO;
    if (!(-lim <= diff && diff <= lim)) ok = 0;
    if (fabs(fabs(diff) - lim) <= 1e-6 * EO) *near = 1;
  }
  return ok;
}

static int obj_moved(const or_scene* s, int32_t prim) { return prim >= 0 && s->moved[s->tri_object[prim]]; }

/* Segment a->b against the moved objects (Sec. 3.2): the bounding-box test
 * (naive mode, and the error-based mode of Sec. 3.3 whose skip case exists
 * because of it) uses the union of the old and new bounding boxes of each
 * moved object; the exact test (naive-exact mode, or error mode with
 * OR_FLAG_ERROR_EXACT) tests the open segment against the moved objects'
 * triangles at the new pose (and the old pose with OR_FLAG_TEST_OLD_TRIS). */
static int seg_vs_moved(const or_scene* s, int mode, uint32_t flags, const double* a, const double* b, int* amb,
                        or_choice* ch) {
  int any = 0, any_amb = 0;
  for (uint32_t m = 0; m < s->n_moved; ++m) {
    uint32_t o = s->moved_list[m];
    int am = 0, hit;
    if (mode == OR_MODE_NAIVE_AABB || (mode == OR_MODE_ERROR && !(flags & OR_FLAG_ERROR_EXACT))) {
      const double* bo = s->box + 12 * (size_t)o;
      double u[6];
      for (int k = 0; k < 3; ++k) {
        u[k] = fmin(bo[k], bo[6 + k]);
        u[3 + k] = fmax(bo[3 + k], bo[9 + k]);
      }
      hit = seg_box(a, b, u, s->eps, &am);
    } else {
      const uint32_t* lst = s->obj_tris + s->obj_first[o];
      uint32_t cnt = s->obj_first[o + 1] - s->obj_first[o];
      hit = any_hit(s, 1, lst, cnt, a, b, -1, &am, NULL);
      if (!(hit && !am) && (flags & OR_FLAG_TEST_OLD_TRIS)) {
        int am2 = 0;
        int h2 = any_hit(s, 0, lst, cnt, a, b, -1, &am2, NULL);
        if (h2 && !am2) {
          hit = 1;
          am = 0;
        } else {
          hit = hit || h2;
          am = am || am2;
        }
      }
    }
    if (hit && !am) {
      *amb = 0;
      return 1;
    }
    if (hit) any = 1;
    if (am) any_amb = 1;
  }
  *amb = any_amb;
  if (any_amb && choose(ch, 2)) any = !any;       /* no object decides robustly: either answer */
  return any;
}

/* per-path counters of a verification */
typedef struct {
  uint64_t seg_t, seg_a, vis, cont, et, ea, nre, ntail, nupd, ntr, rays_a;
} vcount;

/* One path of or_verify (everything before the distribution-map steps):
 * origins, dynamic occlusions and Alg. 1.  *counted: the path keeps its
 * origin on a moved light with a map (it counts in DM_C). */
static void verify_path(const or_scene* s, uint32_t pid, int32_t mode, double tau, uint32_t flags, uint32_t* info,
                        float* origin, or_photon* photons, uint32_t* seg_mask, uint32_t* ambv, uint8_t* counted,
                        vcount* vc, or_choice* ch) {
  uint32_t w = *info;
  uint32_t cell = w & OR_INFO_CELL_MASK;
  uint32_t L = info_nseg(w);
  uint32_t l = light_of(s, pid);
  or_photon* ph = photons;
  float* org = origin;
  uint32_t amb = 0;
  int seg1_blocked = 0;
  *seg_mask = 0;

  /* ---- Sec. 3.1 "update path origins" ---- */
  if (s->light_moved[l]) {
    const or_light* Ln = &s->light[1][l];
    const or_light* Lo = &s->light[0][l];
    int invalid = 0;
    int dm_cell = -1;
    if (L > 0 && s->dm_c[l]) {               /* Compute DM_C: the parametrisation decides */
      float u[4];
      if (dm_param(Ln, ph[0].pos, org, u)) dm_cell = (int)dm_cell_of_u(s, l, u);
    }
    if (L == 0 || (s->dm_c[l] && dm_cell < 0)) {
      invalid = 1;          /* an escaped path has no vertex to re-aim at; or off the map */
    } else if (Ln->type == 0) {
      for (int c = 0; c < 3; ++c) org[c] = Ln->pos[c];
      double a[3], b[3];
      f2d(org, a);
      f2d(ph[0].pos, b);
      int am = 0;
      seg1_blocked = any_hit(s, 1, NULL, 0, a, b, ph[0].prim, &am, ch);
      vc->vis++;
      if (am) {
        amb |= OR_AMB_VERIFY;
        vc->rays_a++;
      }
    } else {
      double x1[3], o0[3], d[3], c[3], nn[3], tt[3], bb[3], no[3];
      f2d(ph[0].pos, x1);
      f2d(org, o0);
      sub3(x1, o0, d);
      normalize3(d);
      f2d(Ln->pos, c); f2d(Ln->normal, nn); f2d(Ln->tangent, tt);
      cross3(nn, tt, bb);
      /* with a distribution map the float32 parametrisation has decided
       * validity; the double-precision tests below decide it otherwise */
      const int by_map = s->dm_c[l] != NULL;
      double ndv = dot3(nn, d);
      int facing_light = ndv > 0.0;
      if (!by_map && fabs(ndv) < 1e-6) {
        amb |= OR_AMB_LIGHT;
        if (choose(ch, 2)) facing_light = !facing_light;
      }
      if (!by_map && !facing_light) {
        invalid = 1;
      } else {
        double x1c[3];
        sub3(x1, c, x1c);
        double tp = dot3(nn, x1c) / ndv;
        int in_front = tp > 0.0;
        if (!by_map && fabs(tp) < s->eps) {
          amb |= OR_AMB_LIGHT;
          if (choose(ch, 2)) in_front = !in_front;
        }
        if (!by_map && !in_front) {
          invalid = 1;
        } else {
          double op[3], rel[3];
          for (int k = 0; k < 3; ++k) op[k] = x1[k] - tp * d[k];
          sub3(op, c, rel);
          double su = dot3(tt, rel), sv = dot3(bb, rel);
          double hw = 0.5 * Ln->size[0], hh = 0.5 * Ln->size[1];
          if (!by_map) {
            int outside = fabs(su) > hw || fabs(sv) > hh;
            if (fabs(fabs(su) - hw) < s->eps || fabs(fabs(sv) - hh) < s->eps) {
              amb |= OR_AMB_LIGHT;
              if (choose(ch, 2)) outside = !outside;
            }
            if (outside) invalid = 1;
          }
          if (!invalid && s->light_tilted[l]) {
            f2d(Lo->normal, no);
            double ratio = ndv / dot3(no, d);
            double EN[3];
            for (int k = 0; k < 3; ++k) EN[k] = (double)ph[0].E[k] * ratio;
            int near = 0;
            vc->et++;
            int pass = energy_close(EN, ph[0].E, tau, &near);
            if (near) {
              vc->ea++;
              amb |= OR_AMB_ENERGY;
              if (choose(ch, 2)) pass = !pass;
            }
            if (!pass) invalid = 1;
          }
          if (!invalid)
            for (int k = 0; k < 3; ++k) org[k] = (float)op[k];
        }
      }
    }
    if (invalid) {
      *info = info_make(cell, 0, 0, 1, 0);
      vc->nre++;
      *ambv = amb;
      return;
    }
    if (dm_cell >= 0) {
      cell = (l << 20) | (uint32_t)dm_cell;
      *info = (w & ~OR_INFO_CELL_MASK) | cell;
      *counted = 1;
    }
  }

  /* ---- Sec. 3.2 "dynamic occlusions": segments in order from the light ---- */
  uint32_t mask = 0;
  for (uint32_t k = 1; k <= L; ++k) {
    double a[3], b[3];
    if (k == 1) f2d(org, a); else f2d(ph[k - 2].pos, a);
    f2d(ph[k - 1].pos, b);
    int hit = obj_moved(s, ph[k - 1].prim) || (k >= 2 && obj_moved(s, ph[k - 2].prim)) || (k == 1 && seg1_blocked);
    if (!hit) {
      int am = 0;
      hit = seg_vs_moved(s, mode, flags, a, b, &am, ch);
      vc->seg_t++;
      if (am) { vc->seg_a++; amb |= OR_AMB_VERIFY; }
    }
    if (hit) {
      mask |= 1u << k;
      if (mode != OR_MODE_ERROR) break;
    }
  }
  *seg_mask = mask;
  if (!mask) {
    *ambv = amb;
    return;
  }
  uint32_t first = 0;
  while (!((mask >> first) & 1u)) ++first;

  if (mode != OR_MODE_ERROR) {
    if (first == 1) {
      *info = info_make(cell, 0, 0, 1, 1);   /* keep light position and direction */
      vc->nre++;
    } else {
      *info = info_make(cell, first - 1, first - 1, 1, 0);
      vc->ntail++;
    }
    *ambv = amb;
    return;
  }

  /* ---- Sec. 3.3, Alg. 1: error-based threshold continuation ---- */
  double xo[16][3];      /* original vertex positions, 0 = origin */
  int32_t po[16];
  f2d(org, xo[0]);
  po[0] = -1;
  for (uint32_t k = 1; k <= L; ++k) { f2d(ph[k - 1].pos, xo[k]); po[k] = ph[k - 1].prim; }
  uint32_t moved_origin = 0;
  int updated = 0, done = 0;
  uint32_t seg = first;
  while (seg <= L && !done) {
    if (!((mask >> seg) & 1u) && !((moved_origin >> seg) & 1u)) { ++seg; continue; }
    double a[3], b[3], d[3];
    if (seg == 1) f2d(org, a); else f2d(ph[seg - 2].pos, a);
    f2d(ph[seg - 1].pos, b);
    sub3(b, a, d);
    normalize3(d);
    int32_t excl = seg == 1 ? -1 : ph[seg - 2].prim;
    double t;
    int am = 0;
    int32_t pn = closest_hit(s, 1, a, d, s->tmin, excl, &t, &am, ch);
    vc->cont++;
    if (am) {
      amb |= OR_AMB_CONT;
      vc->rays_a++;
    }
    if (pn < 0) {                       /* nothing hit: the path ends here */
      L = seg - 1;
      vc->ntr++;
      done = 1;
      break;
    }
    float xn[3];
    double xnd[3];
    for (int c = 0; c < 3; ++c) { xn[c] = (float)(a[c] + t * d[c]); xnd[c] = xn[c]; }
    double dx = 0.0;
    for (int c = 0; c < 3; ++c) dx = fmax(dx, fabs(xnd[c] - b[c]));
    int close = pn == ph[seg - 1].prim && dx <= s->close_tol;
    if (pn == ph[seg - 1].prim && fabs(dx - s->close_tol) < s->eps) {
      amb |= OR_AMB_CONT;
      if (choose(ch, 2)) close = !close;
    }
    if (seg == L) {                     /* last photon: move it, nothing follows */
      for (int c = 0; c < 3; ++c) ph[seg - 1].pos[c] = xn[c];
      ph[seg - 1].prim = pn;
      updated = 1;
      done = 1;
      break;
    }
    double EN[3];
    const float* EO = ph[seg].E;
    if (close) {
      for (int c = 0; c < 3; ++c) EN[c] = EO[c];
    } else {
      /* new vertex: albedo, facing normal, direction to the stored next photon */
      const float* albn = s->albedo + 3 * (size_t)s->tri_object[pn];
      double nsn[3], w[3], xnext[3];
      int af = 0;
      facing(s, 1, pn, d, nsn, &af, ch, NULL);
      f2d(ph[seg].pos, xnext);
      sub3(xnext, xnd, w);
      double wl = norm3(w);
      double cosn = 0.0;
      if (wl > 0.0) {
        w[0] /= wl; w[1] /= wl; w[2] /= wl;
        cosn = fmax(0.0, dot3(nsn, w));
      }
      /* old vertex (old pose): RR probability, facing normal, sampled direction */
      const float* albo = s->albedo + 3 * (size_t)s->tri_object[po[seg]];
      double q = max3(albo);
      double dino[3], nso[3], wo[3];
      sub3(xo[seg], xo[seg - 1], dino);
      normalize3(dino);
      int af2 = 0;
      facing(s, 0, po[seg], dino, nso, &af2, ch, NULL);
      if (af || af2) amb |= OR_AMB_CONT;
      sub3(xo[seg + 1], xo[seg], wo);
      normalize3(wo);
      double coso = dot3(nso, wo);
      for (int c = 0; c < 3; ++c)
        EN[c] = coso > 0.0 ? (double)ph[seg - 1].E[c] * (double)albn[c] * cosn / (q * coso) : 0.0;
    }
    int near = 0;
    vc->et++;
    int pass = energy_close(EN, EO, tau, &near);
    if (near && !close) {
      vc->ea++;
      amb |= OR_AMB_ENERGY;
      if (choose(ch, 2)) pass = !pass;
    }
    if (!pass) {                        /* re-trace from the new vertex */
      for (int c = 0; c < 3; ++c) ph[seg - 1].pos[c] = xn[c];
      ph[seg - 1].prim = pn;
      *info = info_make(cell, seg, seg, 1, 0);
      vc->ntail++;
      done = 2;
      break;
    }
    if (close && !((mask >> (seg + 1)) & 1u) && !obj_moved(s, pn) && !obj_moved(s, ph[seg].prim)) {
      seg += 2;                         /* next segment known valid: skip its check */
      continue;
    }
    for (int c = 0; c < 3; ++c) ph[seg - 1].pos[c] = xn[c];
    ph[seg - 1].prim = pn;
    updated = 1;
    moved_origin |= 1u << (seg + 1);
    ++seg;
  }
  if (done != 2) {
    *info = info_make(cell, L, 0, 0, 0);
    if (updated) vc->nupd++;
  }
  *ambv = amb;
}

void or_verify(const or_scene* s, const uint32_t* ids, uint32_t n, int32_t mode, double tau,
               uint32_t flags, uint64_t seed, uint32_t frame, uint32_t* info, float* origin, or_photon* photons,
               uint32_t* seg_mask, uint32_t* ambv, or_stats* st) {
  uint64_t seg_t = 0, seg_a = 0, vis = 0, cont = 0, et = 0, ea = 0, nre = 0, ntail = 0, nupd = 0, ntr = 0, rays_a = 0;
  /* paths of a moved light with a distribution map that keep their origin (counted in DM_C) */
  uint8_t* counted = (uint8_t*)calloc(n ? n : 1, 1);
#pragma omp parallel for schedule(dynamic, 8) reduction(+ : seg_t, seg_a, vis, cont, et, ea, nre, ntail, nupd, ntr, rays_a)
  for (uint32_t i = 0; i < n; ++i) {
    vcount c = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    verify_path(s, ids[i], mode, tau, flags, &info[i], origin + 3 * (size_t)i, photons + (size_t)i * s->B,
                &seg_mask[i], &ambv[i], &counted[i], &c, NULL);
    seg_t += c.seg_t; seg_a += c.seg_a; vis += c.vis; cont += c.cont; et += c.et;
    ea += c.ea; nre += c.nre; ntail += c.ntail; nupd += c.nupd; ntr += c.ntr; rays_a += c.rays_a;
  }
  /* ---- Compute DM_C, prune paths (Eq. 1, mark then edit), fill DM_C (Sec. 3.1) ---- */
  uint64_t npr = 0, nfi = 0;
  for (uint32_t l = 0; l < s->n_lights; ++l) {
    if (!s->dm_c[l] || !s->light_moved[l]) continue;
    uint32_t* dmc = s->dm_c[l];
    const uint32_t ncell = s->dm_cells[l];
    memset(dmc, 0, sizeof(uint32_t) * ncell);
    for (uint32_t i = 0; i < n; ++i)
      if (counted[i] && light_of(s, ids[i]) == l) dmc[info[i] & 0xFFFFFu]++;
    /* pass 1: mark, with the counts before any pruning */
    uint8_t* pruned = (uint8_t*)calloc(n ? n : 1, 1);
    for (uint32_t i = 0; i < n; ++i) {
      if (!counted[i] || light_of(s, ids[i]) != l) continue;
      const uint32_t c = info[i] & 0xFFFFFu;
      const uint32_t dc = dmc[c], dt = or_dm_target(s, l, c);
      if (dc <= dt) continue;
      uint32_t ctr[4] = {ids[i], 16u, frame, 0u};
      uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
      uint32_t r[4];
      or_philox4x32_10(ctr, key, r);
      /* prune with probability (DM_C - DM_T) / DM_C, decided exactly on the 24-bit draw */
      if ((uint64_t)(r[0] >> 8) * dc < ((uint64_t)(dc - dt) << 24)) {
        pruned[i] = 1;
        info[i] = info_make((l << 20) | c, 0, 0, 1, 0);
        npr++;
      }
    }
    /* pass 2: edit the counts */
    for (uint32_t i = 0; i < n; ++i)
      if (pruned[i]) dmc[info[i] & 0xFFFFFu]--;
    free(pruned);
    /* fill: free paths (fresh emissions of this light) in ascending id order
     * take the cells' deficits in cell order; any further ones spread evenly */
    uint64_t D = 0;
    for (uint32_t c = 0; c < ncell; ++c) {
      const uint32_t dt = or_dm_target(s, l, c);
      if (dmc[c] < dt) D += dt - dmc[c];
    }
    uint64_t F = 0;
    for (uint32_t i = 0; i < n; ++i)
      if (light_of(s, ids[i]) == l && (info[i] & (OR_INFO_REPLACE | OR_INFO_REUSE_LIGHT | (15u << OR_INFO_START_SHIFT))) == OR_INFO_REPLACE) F++;
    uint64_t j = 0;
    uint32_t c = 0;
    uint64_t used = 0;                         /* deficit slots of cells before c already taken */
    for (uint32_t i = 0; i < n; ++i) {
      if (light_of(s, ids[i]) != l) continue;
      if ((info[i] & (OR_INFO_REPLACE | OR_INFO_REUSE_LIGHT | (15u << OR_INFO_START_SHIFT))) != OR_INFO_REPLACE) continue;
      uint32_t cell;
      if (j < D) {
        for (;;) {                              /* the cell whose deficit range holds j */
          const uint32_t dt = or_dm_target(s, l, c);
          const uint64_t def = dmc[c] < dt ? dt - dmc[c] : 0;
          if (j < used + def) break;
          used += def;
          ++c;
        }
        cell = c;
      } else {
        cell = (uint32_t)(((j - D) * ncell) / (F - D));
      }
      info[i] = info_make((l << 20) | cell, 0, 0, 1, 0);
      ++j;
      nfi++;
    }
    /* the filled cells now hold their new paths */
    for (uint32_t i = 0; i < n; ++i)
      if (light_of(s, ids[i]) == l &&
          (info[i] & (OR_INFO_REPLACE | OR_INFO_REUSE_LIGHT | (15u << OR_INFO_START_SHIFT))) == OR_INFO_REPLACE)
        dmc[info[i] & 0xFFFFFu]++;
  }
  free(counted);
  if (st) {
    st->n_pruned += npr;
    st->n_filled += nfi;
    st->paths += n;
    st->segments_tested += seg_t;
    st->segments_amb += seg_a;
    st->vis_rays += vis;
    st->cont_rays += cont;
    st->energy_tests += et;
    st->energy_amb += ea;
    st->n_reemit += nre;
    st->n_tail += ntail;
    st->n_updated += nupd;
    st->n_truncated += ntr;
    st->rays_amb += rays_a;
  }
}

uint32_t or_compact(const uint32_t* info, uint32_t n, uint32_t* list) {
  uint32_t c = 0;
  for (uint32_t i = 0; i < n; ++i)
    if (info[i] & OR_INFO_REPLACE) list[c++] = i;
  return c;
}

/* One path of or_retrace; adds its rays and ambiguous rays to rays[2]. */
static void retrace_path(const or_scene* s, uint32_t pid, uint64_t seed, uint32_t frame, uint32_t* info,
                         float* org, or_photon* ph, uint32_t* ambv, uint64_t rays[2], or_choice* ch) {
  uint32_t w = *info;
  if (!(w & OR_INFO_REPLACE)) return;
  uint32_t l = light_of(s, pid);
  const or_light* L = &s->light[1][l];
  uint32_t start = info_start(w);
  double o[3], d[3], E[3];
  uint32_t k;
  if (start == 0) {
    if (w & OR_INFO_REUSE_LIGHT) {
      double x1[3];
      f2d(org, o);
      f2d(ph[0].pos, x1);
      sub3(x1, o, d);
      normalize3(d);
      for (int c = 0; c < 3; ++c) E[c] = ph[0].E[c];
    } else {
      double u[4];
      rng4(seed, pid, 0, frame, u);
      if (s->dm_c[l]) dm_restrict(s, l, w & 0xFFFFFu, u);   /* within the path's cell */
      emit(L, u, o, d);
      for (int c = 0; c < 3; ++c) org[c] = (float)o[c];
      f2d(org, o);
      for (int c = 0; c < 3; ++c) E[c] = (double)L->power[c] / (double)L->n_paths;
    }
    k = extend_path(s, pid, seed, frame, 0, o, d, E, 0.0, org, ph, ambv, rays, ch);
  } else {
    k = extend_path(s, pid, seed, frame, start, o, d, E, 0.0, org, ph, ambv, rays, ch);
  }
  *info = info_make(w & OR_INFO_CELL_MASK, k, 0, 0, 0);
}

void or_retrace(const or_scene* s, const uint32_t* ids, uint32_t n, uint64_t seed, uint32_t frame,
                uint32_t* info, float* origin, or_photon* photons, uint32_t* ambv, or_stats* st) {
  uint64_t rays = 0, rays_a = 0;
#pragma omp parallel for schedule(dynamic, 8) reduction(+ : rays, rays_a)
  for (uint32_t i = 0; i < n; ++i) {
    uint64_t r[2] = {0, 0};
    retrace_path(s, ids[i], seed, frame, &info[i], origin + 3 * (size_t)i, photons + (size_t)i * s->B, &ambv[i], r,
                 NULL);
    rays += r[0];
    rays_a += r[1];
  }
  if (st) {
    st->trace_rays += rays;
    st->rays_amb += rays_a;
  }
}

void or_retrace_path(const or_scene* s, uint32_t pid, uint64_t seed, uint32_t frame, uint32_t* info,
                     float* origin, or_photon* photons, uint32_t* amb, or_choice* ch) {
  uint64_t r[2] = {0, 0};
  retrace_path(s, pid, seed, frame, info, origin, photons, amb, r, ch);
}

int32_t or_verify_path(const or_scene* s, uint32_t pid, int32_t mode, double tau, uint32_t flags, uint32_t* info,
                       float* origin, or_photon* photons, uint32_t* seg_mask, uint32_t* amb, or_choice* ch) {
  for (uint32_t l = 0; l < s->n_lights; ++l)
    if (s->dm_c[l]) return -1;
  vcount c = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  uint8_t counted = 0;
  verify_path(s, pid, mode, tau, flags, info, origin, photons, seg_mask, amb, &counted, &c, ch);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* deposit                                                                   */
/* ------------------------------------------------------------------------ */
/* Texel of a position in the top-down XZ atlas, decided in float32 with no
 * fused operations (the oracle is compiled with -ffp-contract=off). */
static inline int texel(float p, float lo, float hi, uint32_t res) {
  float scale = (float)res / (hi - lo);
  float u = (p - lo) * scale;
  float f = floorf(u);
  int i;
  if (!(f >= 0.0f)) i = 0;
  else if (f >= (float)res) i = (int)res - 1;
  else i = (int)f;
  return i;
}

void or_deposit(const uint32_t* info, uint32_t n, const or_photon* photons, uint32_t max_bounces,
                uint32_t width, uint32_t height, float x0, float z0, float x1, float z1, double* atlas) {
  for (uint32_t i = 0; i < n; ++i) {
    uint32_t L = info_nseg(info[i]);
    for (uint32_t k = 0; k < L; ++k) {
      const or_photon* v = &photons[(size_t)i * max_bounces + k];
      int tx = texel(v->pos[0], x0, x1, width);
      int tz = texel(v->pos[2], z0, z1, height);
      double* a = atlas + 3 * ((size_t)tz * width + tx);
      a[0] += v->E[0];
      a[1] += v->E[1];
      a[2] += v->E[2];
    }
  }
}

void or_photon_texels(const uint32_t* info, uint32_t n, const or_photon* photons, uint32_t max_bounces,
                      uint32_t width, uint32_t height, float x0, float z0, float x1, float z1, int32_t* texels) {
  for (uint32_t i = 0; i < n; ++i) {
    const uint32_t L = info_nseg(info[i]);
    for (uint32_t k = 0; k < max_bounces; ++k) {
      int32_t* t = texels + 2 * ((size_t)i * max_bounces + k);
      if (k < L) {
        const or_photon* v = &photons[(size_t)i * max_bounces + k];
        t[0] = texel(v->pos[0], x0, x1, width);
        t[1] = texel(v->pos[2], z0, z1, height);
      } else {
        t[0] = t[1] = -1;
      }
    }
  }
}

int32_t or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* screen-space photon splat (Fig. 2 "splat/gather")                         */
/* ------------------------------------------------------------------------ */
/* Pinhole camera basis: forward f, right r = f x up, true up u = r x f. */
static void cam_basis(const or_camera* c, double* pos, double* f, double* r, double* u, double* th) {
  double tg[3], up[3];
  f2d(c->pos, pos);
  f2d(c->target, tg);
  f2d(c->up, up);
  sub3(tg, pos, f);
  normalize3(f);
  cross3(f, up, r);
  normalize3(r);
  cross3(r, f, u);
  *th = tan(0.5 * (double)c->fov_y);
}

/* View depth of q. */
static double cam_depth(const double* pos, const double* f, const double* q) {
  double v[3];
  sub3(q, pos, v);
  return dot3(v, f);
}

/* G-buffer from primary rays through pixel centres, then for every pixel
 * with a visible surface point p (normal n facing the camera, albedo rho)
 * and every photon x with incident direction d_in (from the previous vertex,
 * the origin for the first) arriving on the visible side (n . d_in < 0):
 *   L += rho / pi * E * 2 (1 - s^2) / (pi r^2),   s = |p - x| / r < 1,
 * a radius kernel normalised over the disk (integral over the plane = 1).
 * A photon is skipped when any corner of its kernel cube lies less than
 * 1e-3 diag in front of the camera (no screen-space footprint).  amb[pixel]
 * is set when its hit, a side test or a near-plane decision is within the
 * tolerances. */
void or_splat(const or_scene* s, const uint32_t* ids, uint32_t n, const uint32_t* info, const float* origin,
              const or_photon* photons, const or_camera* cam, double radius, double* image, uint8_t* amb) {
  (void)ids;
  const uint32_t W = cam->width, H = cam->height;
  double pos[3], f[3], r[3], u[3], th;
  cam_basis(cam, pos, f, r, u, &th);
  const double aspect = (double)W / (double)H;
  const size_t npx = (size_t)W * H;
  double* gp = (double*)malloc(sizeof(double) * 3 * (npx ? npx : 1));
  double* gn = (double*)malloc(sizeof(double) * 3 * (npx ? npx : 1));
  int32_t* gprim = (int32_t*)malloc(sizeof(int32_t) * (npx ? npx : 1));
#pragma omp parallel for schedule(dynamic, 16)
  for (size_t px = 0; px < npx; ++px) {
    const uint32_t i = (uint32_t)(px % W), j = (uint32_t)(px / W);
    const double x = (2.0 * (i + 0.5) / W - 1.0) * th * aspect;
    const double y = (1.0 - 2.0 * (j + 0.5) / H) * th;
    double d[3];
    for (int k = 0; k < 3; ++k) d[k] = f[k] + x * r[k] + y * u[k];
    normalize3(d);
    double t;
    int a = 0;
    const int32_t prim = closest_hit(s, 1, pos, d, 0.0, -1, &t, &a, NULL);
    amb[px] = (uint8_t)(a != 0);
    gprim[px] = prim;
    if (prim >= 0) {
      for (int k = 0; k < 3; ++k) gp[3 * px + k] = pos[k] + t * d[k];
      double nn[3];
      unit_normal(s, 1, prim, nn);
      const double sg = dot3(nn, d) > 0.0 ? -1.0 : 1.0;
      for (int k = 0; k < 3; ++k) gn[3 * px + k] = sg * nn[k];
    }
  }
  /* photons: position, incident direction, energy, near-plane status */
  size_t np = 0;
  for (uint32_t i = 0; i < n; ++i) np += (info[i] >> OR_INFO_NSEG_SHIFT) & 15u;
  double* ph = (double*)malloc(sizeof(double) * 9 * (np ? np : 1));
  int8_t* ok = (int8_t*)malloc(np ? np : 1);   /* 1 splat, 0 skip, -1 skip but ambiguous */
  size_t q = 0;
  const double znear = 1e-3 * s->diag;
  for (uint32_t i = 0; i < n; ++i) {
    const uint32_t L = (info[i] >> OR_INFO_NSEG_SHIFT) & 15u;
    const or_photon* pp = photons + (size_t)i * s->B;
    for (uint32_t k = 0; k < L && k < s->B; ++k, ++q) {
      double x[3], prev[3];
      f2d(pp[k].pos, x);
      if (k == 0) f2d(origin + 3 * (size_t)i, prev); else f2d(pp[k - 1].pos, prev);
      double* e = ph + 9 * q;
      for (int c = 0; c < 3; ++c) { e[c] = x[c]; e[3 + c] = x[c] - prev[c]; e[6 + c] = pp[k].E[c]; }
      int8_t st = 1;
      for (int cx = -1; cx <= 1; cx += 2)
        for (int cy = -1; cy <= 1; cy += 2)
          for (int cz = -1; cz <= 1; cz += 2) {
            const double cor[3] = {x[0] + cx * radius, x[1] + cy * radius, x[2] + cz * radius};
            const double z = cam_depth(pos, f, cor);
            if (!(z > znear)) st = 0;
            else if (fabs(z - znear) < s->eps && st == 1) st = -1;
          }
      ok[q] = st;
    }
  }
  const double r2 = radius * radius;
  const double norm = 2.0 / (M_PI * r2);
#pragma omp parallel for schedule(dynamic, 16)
  for (size_t px = 0; px < npx; ++px) {
    double* L = image + 3 * px;
    L[0] = L[1] = L[2] = 0.0;
    if (gprim[px] < 0) continue;
    const double* p = gp + 3 * px;
    const double* nv = gn + 3 * px;
    const float* rho = s->albedo + 3 * (size_t)s->tri_object[gprim[px]];
    for (size_t k = 0; k < np; ++k) {
      const double* e = ph + 9 * k;
      double dx[3];
      sub3(p, e, dx);
      const double s2 = dot3(dx, dx) / r2;
      if (!(s2 < 1.0)) continue;
      if (ok[k] <= 0) {
        if (ok[k] < 0) amb[px] = 1;
        continue;
      }
      const double side = dot3(nv, e + 3);
      if (fabs(side) < 1e-6 * norm3(e + 3)) amb[px] = 1;
      if (!(side < 0.0)) continue;
      const double w = norm * (1.0 - s2) / M_PI;
      for (int c = 0; c < 3; ++c) L[c] += (double)rho[c] * e[6 + c] * w;
    }
  }
  free(gp); free(gn); free(gprim); free(ph); free(ok);
}

/* ------------------------------------------------------------------------ */
/* differentiable deposit model and its adjoint                               */
/* ------------------------------------------------------------------------ */
uint32_t or_theta_size(const or_scene* s) { return 7u * s->n_lights + 3u * s->n_dynamic; }

void or_theta_current(const or_scene* s, double* th) {
  for (uint32_t l = 0; l < s->n_lights; ++l) {
    const or_light* L = &s->light[1][l];
    for (int k = 0; k < 3; ++k) {
      th[7 * l + k] = L->pos[k];
      th[7 * l + 3 + k] = L->normal[k];
    }
    th[7 * l + 6] = 1.0;
  }
  for (uint32_t o = 0; o < s->n_objects; ++o)
    if (s->dyn_index[o] >= 0)
      for (int k = 0; k < 3; ++k) th[7 * s->n_lights + 3 * s->dyn_index[o] + k] = s->xf_new[12 * o + 4 * k + 3];
}

/* Forward chain of one path: emission point o, direction d0, and photon
 * positions x[1..L] under theta (plane of photon k: unit normal nu[k] through
 * the stored photon moved by its object's translation). */
typedef struct {
  uint32_t L, l;
  double o[3], d0[3], x[16][3], nu[16][3], d[16][3], tau1;
  double alpha, beta, ell[3], t[3];
  int32_t dyn[16];
} model_path;

static void model_forward(const or_scene* s, uint32_t w, const float* org, const or_photon* ph, const double* th,
                          model_path* m) {
  m->L = (w >> OR_INFO_NSEG_SHIFT) & 15u;
  if (m->L > s->B) m->L = s->B;
  m->l = (w >> 20) & 3u;
  const or_light* L0 = &s->light[1][m->l];
  const double* tl = th + 7 * m->l;
  double o0[3], p0[3], n0[3], x10[3], d00[3];
  f2d(org, o0);
  f2d(L0->pos, p0);
  f2d(L0->normal, n0);
  f2d(L0->tangent, m->t);
  if (m->L == 0) return;
  f2d(ph[0].pos, x10);
  sub3(x10, o0, d00);
  if (L0->type == 0) {
    for (int k = 0; k < 3; ++k) { m->o[k] = tl[k]; m->d0[k] = d00[k]; }
  } else {
    double b0[3], rel[3], nl[3], bl[3];
    cross3(n0, m->t, b0);
    sub3(o0, p0, rel);
    m->alpha = dot3(m->t, rel);
    m->beta = dot3(b0, rel);
    m->ell[0] = dot3(m->t, d00);
    m->ell[1] = dot3(b0, d00);
    m->ell[2] = dot3(n0, d00);
    for (int k = 0; k < 3; ++k) nl[k] = tl[3 + k];
    cross3(nl, m->t, bl);
    for (int k = 0; k < 3; ++k) {
      m->o[k] = tl[k] + m->alpha * m->t[k] + m->beta * bl[k];
      m->d0[k] = m->ell[0] * m->t[k] + m->ell[1] * bl[k] + m->ell[2] * nl[k];
    }
  }
  const double* prev = m->o;
  const double* dir = m->d0;
  for (uint32_t k = 1; k <= m->L; ++k) {
    const or_photon* v = &ph[k - 1];
    unit_normal(s, 1, v->prim, m->nu[k]);
    double q[3];
    f2d(v->pos, q);
    const int32_t di = s->dyn_index[s->tri_object[v->prim]];
    m->dyn[k] = di;
    if (di >= 0) {
      const uint32_t obj = s->tri_object[v->prim];
      for (int c = 0; c < 3; ++c) q[c] += th[7 * s->n_lights + 3 * di + c] - (double)s->xf_new[12 * obj + 4 * c + 3];
    }
    double qp[3];
    sub3(q, prev, qp);
    const double tau = dot3(m->nu[k], qp) / dot3(m->nu[k], dir);
    if (k == 1) m->tau1 = tau;
    for (int c = 0; c < 3; ++c) m->x[k][c] = prev[c] + tau * dir[c];
    if (k < m->L) {
      double xa[3], xb[3];
      f2d(ph[k - 1].pos, xa);
      f2d(ph[k].pos, xb);
      sub3(xb, xa, m->d[k]);           /* stored direction of segment k+1 (fixed) */
    }
    prev = m->x[k];
    dir = m->d[k];
  }
}

/* Uniform cubic B-spline splat of (x, z) (C2, so the model loss is twice
 * continuously differentiable in theta): with u = (x - x0) W/(x1 - x0) - 1/2
 * the texel-centre coordinate, i = floor(u) and f = u - i, the four texels
 * i-1 .. i+2 get the cardinal cubic B-spline weights
 *   b0 = (1-f)^3/6, b1 = (3f^3 - 6f^2 + 4)/6, b2 = (-3f^3 + 3f^2 + 3f + 1)/6,
 *   b3 = f^3/6      (sum 1), and the 2-D weight is the product over x and z.
 * Entry 4b+a is texel (i-1+a, j-1+b) with weight wx[a] wz[b] and gradient
 * (sx wx'[a] wz[b], sz wx[a] wz'[b]). */
static void bspline1(double f, double* w, double* dw) {
  const double g = 1.0 - f;
  w[0] = g * g * g / 6.0;
  w[1] = (3.0 * f * f * f - 6.0 * f * f + 4.0) / 6.0;
  w[2] = (-3.0 * f * f * f + 3.0 * f * f + 3.0 * f + 1.0) / 6.0;
  w[3] = f * f * f / 6.0;
  dw[0] = -g * g / 2.0;
  dw[1] = (3.0 * f * f - 4.0 * f) / 2.0;
  dw[2] = (-3.0 * f * f + 2.0 * f + 1.0) / 2.0;
  dw[3] = f * f / 2.0;
}

static void splat_weights(double x, double z, uint32_t W, uint32_t H, float x0, float z0, float x1, float z1,
                          int* ti, int* tj, double* wt, double* gx, double* gz) {
  const double sx = (double)W / ((double)x1 - (double)x0), sz = (double)H / ((double)z1 - (double)z0);
  const double u = (x - x0) * sx - 0.5, v = (z - z0) * sz - 0.5;
  const double fi = floor(u), fj = floor(v);
  double wx[4], dwx[4], wz[4], dwz[4];
  bspline1(u - fi, wx, dwx);
  bspline1(v - fj, wz, dwz);
  for (int b = 0; b < 4; ++b)
    for (int a = 0; a < 4; ++a) {
      const int k = 4 * b + a;
      ti[k] = (int)fi - 1 + a;
      tj[k] = (int)fj - 1 + b;
      wt[k] = wx[a] * wz[b];
      gx[k] = sx * dwx[a] * wz[b];
      gz[k] = sz * wx[a] * dwz[b];
    }
}

void or_model_deposit(const or_scene* s, const uint32_t* ids, uint32_t n, const uint32_t* info, const float* origin,
                      const or_photon* photons, const double* theta, uint32_t W, uint32_t H, float x0, float z0,
                      float x1, float z1, double* atlas) {
  (void)ids;
  for (uint32_t i = 0; i < n; ++i) {
    model_path m;
    model_forward(s, info[i], origin + 3 * (size_t)i, photons + (size_t)i * s->B, theta, &m);
    const double sc = theta[7 * m.l + 6];
    for (uint32_t k = 1; k <= m.L; ++k) {
      const or_photon* v = &photons[(size_t)i * s->B + k - 1];
      int ti[16], tj[16];
      double wt[16], gx[16], gz[16];
      splat_weights(m.x[k][0], m.x[k][2], W, H, x0, z0, x1, z1, ti, tj, wt, gx, gz);
      for (int q = 0; q < 16; ++q) {
        if (ti[q] < 0 || tj[q] < 0 || ti[q] >= (int)W || tj[q] >= (int)H) continue;
        double* a = atlas + 3 * ((size_t)tj[q] * W + ti[q]);
        for (int c = 0; c < 3; ++c) a[c] += sc * v->E[c] * wt[q];
      }
    }
  }
}

/* Reverse mode over one path: gradient of each photon's deposit with respect
 * to its position (g), carried back through the plane intersections
 * x_{k+1} = x_k + d_k nu.(q - x_k)/(nu.d_k):  dx_{k+1}/dx_k = I - d nu^T/(nu.d),
 * dx_{k+1}/dq = d nu^T/(nu.d); at the light x_1 = o + d0 tau with
 * dx_1/do = I - d0 nu^T/(nu.d0), dx_1/dd0 = tau (I - d0 nu^T/(nu.d0)). */
void or_adjoint(const or_scene* s, const uint32_t* ids, uint32_t n, const uint32_t* info, const float* origin,
                const or_photon* photons, const double* theta, uint32_t W, uint32_t H, float x0, float z0, float x1,
                float z1, const double* G, double* dtheta, double* score) {
  (void)ids;
  const uint32_t nt = or_theta_size(s);
  double* acc = (double*)calloc(nt, sizeof(double));
  for (uint32_t i = 0; i < n; ++i) {
    model_path m;
    model_forward(s, info[i], origin + 3 * (size_t)i, photons + (size_t)i * s->B, theta, &m);
    const double sc = theta[7 * m.l + 6];
    double gpos[16][3];
    double sgE = 0.0, gscale = 0.0;
    for (uint32_t k = 1; k <= m.L; ++k) {
      const or_photon* v = &photons[(size_t)i * s->B + k - 1];
      int ti[16], tj[16];
      double wt[16], gx[16], gz[16];
      splat_weights(m.x[k][0], m.x[k][2], W, H, x0, z0, x1, z1, ti, tj, wt, gx, gz);
      gpos[k][0] = gpos[k][1] = gpos[k][2] = 0.0;
      for (int q = 0; q < 16; ++q) {
        if (ti[q] < 0 || tj[q] < 0 || ti[q] >= (int)W || tj[q] >= (int)H) continue;
        const double* g = G + 3 * ((size_t)tj[q] * W + ti[q]);
        for (int c = 0; c < 3; ++c) {
          const double e = sc * v->E[c];
          gpos[k][0] += g[c] * e * gx[q];
          gpos[k][2] += g[c] * e * gz[q];
          sgE += g[c] * e * wt[q];
          gscale += g[c] * v->E[c] * wt[q];
        }
      }
    }
    if (score) score[i] = fabs(sgE);
    if (m.L == 0) continue;
    acc[7 * m.l + 6] += gscale;
    /* backward along the path */
    double g[3] = {0, 0, 0};
    for (uint32_t k = m.L; k >= 1; --k) {
      for (int c = 0; c < 3; ++c) g[c] += gpos[k][c];
      const double* dir = k == 1 ? m.d0 : m.d[k - 1];
      const double* nu = m.nu[k];
      const double dg = dot3(dir, g), nd = dot3(nu, dir);
      if (m.dyn[k] >= 0)   /* dx_k/dq_k = d nu^T / (nu.d): q moves with the translation */
        for (int c = 0; c < 3; ++c) acc[7 * s->n_lights + 3 * m.dyn[k] + c] += nu[c] * dg / nd;
      double gp[3];        /* g (I - d nu^T/(nu.d)) = g - nu (d.g)/(nu.d) */
      for (int c = 0; c < 3; ++c) gp[c] = g[c] - nu[c] * dg / nd;
      if (k == 1) {
        /* light: o and d0 */
        double go[3], gd[3];
        for (int c = 0; c < 3; ++c) { go[c] = gp[c]; gd[c] = m.tau1 * gp[c]; }
        const or_light* L0 = &s->light[1][m.l];
        for (int c = 0; c < 3; ++c) acc[7 * m.l + c] += go[c];
        if (L0->type != 0) {
          double tg[3], tgd[3];
          cross3(m.t, go, tg);      /* d/dn of beta (n x t) . go = beta (t x go) */
          cross3(m.t, gd, tgd);
          for (int c = 0; c < 3; ++c)
            acc[7 * m.l + 3 + c] += m.beta * tg[c] + m.ell[1] * tgd[c] + m.ell[2] * gd[c];
        }
      } else {
        for (int c = 0; c < 3; ++c) g[c] = gp[c];
      }
    }
  }
  for (uint32_t j = 0; j < nt; ++j) dtheta[j] += acc[j];
  free(acc);
}
