/*
 * Oracle -- TEST INFRASTRUCTURE ONLY.
 * FP64 Monte Carlo path tracer for the rendering step of Sec. 3.2 (every frame
 * I_k at time t_k = k / F_evt is path traced at a low sample count).  The paper
 * names the technique only; the estimator below is the project's specification:
 *
 *   camera ray: pinhole, vertical FOV from the camera record, jitter
 *     u = Philox(key=(seed lo, seed hi), ctr=(pixel, sample, frame, 0)),
 *     u32 -> [0,1) as (x >> 8) * 2^-24.
 *   for segment b = 1..max_depth:
 *     closest hit (watertight test of Woop, Benthin, Wald, JCGT 2013;
 *       minimum t, ties -> smaller triangle index);
 *     miss -> add beta * env, stop (the environment is not light-sampled);
 *     light triangle -> front face adds beta * Le, MIS-weighted (power
 *       heuristic) against light sampling when b > 1; stop;
 *     b == max_depth -> stop;
 *     next-event estimation with ctr word 3 = 4b+1: light picked by power
 *       (luminance * area), uniform point on the parallelogram, shadow ray from
 *       the offset origin to t < dist (1 - 1e-4);
 *     BSDF sample with ctr word 3 = 4b+2: Lambert cosine-weighted (Malley) or
 *       GGX visible-normal sampling (Heitz, JCGT 2018) with Schlick Fresnel
 *       (F0 = albedo) and separable Smith masking; beta *= f cos / pdf.
 *   origins are offset along the face-forward geometric normal by
 *   1e-4 (1 + max |x_i|).
 * The shading frame is the branchless orthonormal basis of Duff et al.,
 * JCGT 2017.  No Russian roulette.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <float.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include "oracle.h"

void orc_philox_block(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

#define LIGHT_BIT 0x80000000u
#define LEAF_MAX 4

typedef struct { double lo[3], hi[3]; int32_t left, right, first, count; } node_t;
typedef struct { double p0[3], e1[3], e2[3], n[3], L[3], area, prob; } light_t;

struct orc_scene {
  int64_t n;
  double* tri;      /* [n][9] */
  uint32_t* mat;    /* [n] */
  double* mats;     /* [n_mat][8] */
  int n_mat;
  light_t* lights;
  double* cdf;
  int n_l;
  double env;
  int use_bvh;
  node_t* nodes;
  int64_t n_nodes;
  int32_t* perm;
};

/* ----------------------------------------------------------------- vectors */
static void sub3(const double* a, const double* b, double* r) { r[0]=a[0]-b[0]; r[1]=a[1]-b[1]; r[2]=a[2]-b[2]; }
static double dot3(const double* a, const double* b) { return a[0]*b[0]+a[1]*b[1]+a[2]*b[2]; }
static void cross3(const double* a, const double* b, double* r) {
  r[0]=a[1]*b[2]-a[2]*b[1]; r[1]=a[2]*b[0]-a[0]*b[2]; r[2]=a[0]*b[1]-a[1]*b[0];
}
static void normalize3(double* a) { double l = sqrt(dot3(a,a)); a[0]/=l; a[1]/=l; a[2]/=l; }
static double u01(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }
static double lum(const double* c) { return 0.2126*c[0] + 0.7152*c[1] + 0.0722*c[2]; }

/* ------------------------------------------------------------------- scene */
static double surface_area(const double* lo, const double* hi) {
  double dx = hi[0]-lo[0], dy = hi[1]-lo[1], dz = hi[2]-lo[2];
  if (dx < 0 || dy < 0 || dz < 0) return 0.0;
  return 2.0*(dx*dy + dy*dz + dz*dx);
}

static const double* g_cent;   /* qsort context (single-threaded build) */
static int g_axis;
static int cmp_cent(const void* a, const void* b) {
  double ca = g_cent[3*(*(const int32_t*)a) + g_axis], cb = g_cent[3*(*(const int32_t*)b) + g_axis];
  if (ca < cb) return -1;
  if (ca > cb) return 1;
  return (*(const int32_t*)a) - (*(const int32_t*)b);
}

static void tri_bounds(const orc_scene* s, int32_t t, double* lo, double* hi) {
  const double* v = s->tri + 9*(int64_t)t;
  for (int k = 0; k < 3; ++k) {
    lo[k] = fmin(v[k], fmin(v[3+k], v[6+k]));
    hi[k] = fmax(v[k], fmax(v[3+k], v[6+k]));
  }
}

/* Full-sweep SAH: for each axis sort the centroids and evaluate every split. */
static int32_t build_node(orc_scene* s, const double* cent, int32_t first, int32_t count,
                          double* sweep, int32_t* tmp) {
  int32_t idx = (int32_t)s->n_nodes++;
  node_t* nd = &s->nodes[idx];
  double lo[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, hi[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
  for (int32_t i = 0; i < count; ++i) {
    double tl[3], th[3];
    tri_bounds(s, s->perm[first+i], tl, th);
    for (int k = 0; k < 3; ++k) { lo[k] = fmin(lo[k], tl[k]); hi[k] = fmax(hi[k], th[k]); }
  }
  memcpy(nd->lo, lo, sizeof lo); memcpy(nd->hi, hi, sizeof hi);
  nd->left = nd->right = -1; nd->first = first; nd->count = count;
  if (count <= 1) return idx;
  double sa = surface_area(lo, hi);
  double best = DBL_MAX; int best_axis = -1; int32_t best_split = -1;
  for (int ax = 0; ax < 3; ++ax) {
    g_cent = cent; g_axis = ax;
    qsort(s->perm + first, (size_t)count, sizeof(int32_t), cmp_cent);
    /* suffix areas */
    double rl[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, rh[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
    for (int32_t i = count - 1; i > 0; --i) {
      double tl[3], th[3];
      tri_bounds(s, s->perm[first+i], tl, th);
      for (int k = 0; k < 3; ++k) { rl[k] = fmin(rl[k], tl[k]); rh[k] = fmax(rh[k], th[k]); }
      sweep[i] = surface_area(rl, rh);
    }
    double ll[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, lh[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
    for (int32_t i = 1; i < count; ++i) {
      double tl[3], th[3];
      tri_bounds(s, s->perm[first+i-1], tl, th);
      for (int k = 0; k < 3; ++k) { ll[k] = fmin(ll[k], tl[k]); lh[k] = fmax(lh[k], th[k]); }
      double c = 1.0 + (surface_area(ll, lh) * i + sweep[i] * (count - i)) / (sa > 0 ? sa : 1.0);
      if (c < best) { best = c; best_axis = ax; best_split = i; }
    }
  }
  if (count <= LEAF_MAX && best >= (double)count) return idx;   /* leaf is cheaper */
  g_cent = cent; g_axis = best_axis;
  qsort(s->perm + first, (size_t)count, sizeof(int32_t), cmp_cent);
  int32_t l = build_node(s, cent, first, best_split, sweep, tmp);
  int32_t r = build_node(s, cent, first + best_split, count - best_split, sweep, tmp);
  nd = &s->nodes[idx];
  nd->left = l; nd->right = r; nd->count = 0;
  return idx;
}

orc_scene* orc_scene_new(const float* tri, const uint32_t* mat, int64_t n,
                         const double* mats, int n_mat, const float* lights, int n_l,
                         double env, int use_bvh) {
  orc_scene* s = (orc_scene*)calloc(1, sizeof(orc_scene));
  s->n = n + 2 * (int64_t)n_l;
  s->tri = (double*)malloc(sizeof(double) * 9 * (size_t)s->n);
  s->mat = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)s->n);
  for (int64_t i = 0; i < 9 * n; ++i) s->tri[i] = (double)tri[i];
  for (int64_t i = 0; i < n; ++i) s->mat[i] = mat[i];
  s->n_mat = n_mat;
  s->mats = (double*)malloc(sizeof(double) * 8 * (size_t)(n_mat > 0 ? n_mat : 1));
  memcpy(s->mats, mats, sizeof(double) * 8 * (size_t)n_mat);
  s->n_l = n_l;
  s->lights = (light_t*)calloc((size_t)(n_l > 0 ? n_l : 1), sizeof(light_t));
  s->cdf = (double*)calloc((size_t)(n_l > 0 ? n_l : 1), sizeof(double));
  double total = 0.0;
  for (int j = 0; j < n_l; ++j) {
    light_t* L = &s->lights[j];
    for (int k = 0; k < 3; ++k) {
      L->p0[k] = lights[12*j+k]; L->e1[k] = lights[12*j+3+k];
      L->e2[k] = lights[12*j+6+k]; L->L[k] = lights[12*j+9+k];
    }
    cross3(L->e1, L->e2, L->n);
    L->area = sqrt(dot3(L->n, L->n));
    normalize3(L->n);
    L->prob = lum(L->L) * L->area;
    total += L->prob;
    /* the two emitting triangles (p0, p0+e1, p0+e1+e2), (p0, p0+e1+e2, p0+e2);
       their vertices are rounded to float32 exactly as the CUDA library does */
    double a[3], b[3], c[3], d[3];
    for (int k = 0; k < 3; ++k) {
      a[k] = (double)(float)L->p0[k];
      b[k] = (double)(float)(lights[12*j+k] + lights[12*j+3+k]);
      c[k] = (double)(float)(lights[12*j+k] + lights[12*j+3+k] + lights[12*j+6+k]);
      d[k] = (double)(float)(lights[12*j+k] + lights[12*j+6+k]);
    }
    double* t0 = s->tri + 9 * (n + 2*j);
    double* t1 = t0 + 9;
    for (int k = 0; k < 3; ++k) { t0[k]=a[k]; t0[3+k]=b[k]; t0[6+k]=c[k]; t1[k]=a[k]; t1[3+k]=c[k]; t1[6+k]=d[k]; }
    s->mat[n + 2*j] = LIGHT_BIT | (uint32_t)j;
    s->mat[n + 2*j + 1] = LIGHT_BIT | (uint32_t)j;
  }
  double acc = 0.0;
  for (int j = 0; j < n_l; ++j) {
    s->lights[j].prob /= total;
    acc += s->lights[j].prob;
    s->cdf[j] = acc;
  }
  if (n_l > 0) s->cdf[n_l - 1] = 1.0;
  s->env = env;
  s->use_bvh = use_bvh;
  if (use_bvh && s->n > 0) {
    s->nodes = (node_t*)malloc(sizeof(node_t) * (size_t)(2 * s->n));
    s->perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)s->n);
    double* cent = (double*)malloc(sizeof(double) * 3 * (size_t)s->n);
    double* sweep = (double*)malloc(sizeof(double) * (size_t)(s->n + 1));
    for (int64_t i = 0; i < s->n; ++i) {
      s->perm[i] = (int32_t)i;
      for (int k = 0; k < 3; ++k)
        cent[3*i+k] = (s->tri[9*i+k] + s->tri[9*i+3+k] + s->tri[9*i+6+k]) / 3.0;
    }
    build_node(s, cent, 0, (int32_t)s->n, sweep, NULL);
    free(cent); free(sweep);
  }
  return s;
}

void orc_scene_free(orc_scene* s) {
  if (!s) return;
  free(s->tri); free(s->mat); free(s->mats); free(s->lights); free(s->cdf);
  free(s->nodes); free(s->perm); free(s);
}
int64_t orc_scene_ntris(const orc_scene* s) { return s->n; }
int64_t orc_bvh_nodes(const orc_scene* s) { return s->n_nodes; }

/* SAH cost with C_trav = 1, C_isect = 1, normalised by the root's area */
double orc_bvh_sah_cost(const orc_scene* s) {
  if (!s->use_bvh || s->n_nodes == 0) return 0.0;
  double root = surface_area(s->nodes[0].lo, s->nodes[0].hi), c = 0.0;
  for (int64_t i = 0; i < s->n_nodes; ++i) {
    double a = surface_area(s->nodes[i].lo, s->nodes[i].hi) / root;
    c += s->nodes[i].count > 0 ? a * s->nodes[i].count : a;
  }
  return c;
}

/* ------------------------------------------------------------ intersection */
typedef struct { double o[3], d[3], inv[3]; int kx, ky, kz; double Sx, Sy, Sz; } ray_t;

static void ray_setup(ray_t* r, const double* o, const double* d) {
  for (int k = 0; k < 3; ++k) { r->o[k] = o[k]; r->d[k] = d[k]; r->inv[k] = 1.0 / d[k]; }
  int kz = 0;
  if (fabs(d[1]) > fabs(d[kz])) kz = 1;
  if (fabs(d[2]) > fabs(d[kz])) kz = 2;
  int kx = (kz + 1) % 3, ky = (kx + 1) % 3;
  if (d[kz] < 0.0) { int t = kx; kx = ky; ky = t; }
  r->kx = kx; r->ky = ky; r->kz = kz;
  r->Sx = d[kx] / d[kz]; r->Sy = d[ky] / d[kz]; r->Sz = 1.0 / d[kz];
}

/* watertight ray/triangle test; returns t in (0, tmax) or -1 */
static double tri_hit(const ray_t* r, const double* v, double tmax) {
  double A[3], B[3], C[3];
  sub3(v, r->o, A); sub3(v + 3, r->o, B); sub3(v + 6, r->o, C);
  double Ax = A[r->kx] - r->Sx * A[r->kz], Ay = A[r->ky] - r->Sy * A[r->kz];
  double Bx = B[r->kx] - r->Sx * B[r->kz], By = B[r->ky] - r->Sy * B[r->kz];
  double Cx = C[r->kx] - r->Sx * C[r->kz], Cy = C[r->ky] - r->Sy * C[r->kz];
  double U = Cx * By - Cy * Bx, V = Ax * Cy - Ay * Cx, W = Bx * Ay - By * Ax;
  if ((U < 0 || V < 0 || W < 0) && (U > 0 || V > 0 || W > 0)) return -1.0;
  double det = U + V + W;
  if (det == 0.0) return -1.0;
  double T = U * (r->Sz * A[r->kz]) + V * (r->Sz * B[r->kz]) + W * (r->Sz * C[r->kz]);
  double t = T / det;
  if (!(t > 0.0) || !(t < tmax)) return -1.0;
  return t;
}

static const double GAMMA3 = 3.0 * DBL_EPSILON * 0.5 / (1.0 - 3.0 * DBL_EPSILON * 0.5);

/* conservative slab test (far distance widened by 1 + 2 gamma_3) */
static int box_hit(const ray_t* r, const node_t* n, double tmax, double* tnear) {
  double t0 = 0.0, t1 = tmax;
  for (int k = 0; k < 3; ++k) {
    double a = (n->lo[k] - r->o[k]) * r->inv[k], b = (n->hi[k] - r->o[k]) * r->inv[k];
    double lo = fmin(a, b), hi = fmax(a, b) * (1.0 + 2.0 * GAMMA3);
    t0 = fmax(t0, lo); t1 = fmin(t1, hi);
  }
  *tnear = t0;
  return t0 <= t1;
}

static void closest(const orc_scene* s, const double* o, const double* d, double tmax,
                    double* t_out, int32_t* p_out, int64_t* nv, int64_t* nt) {
  ray_t r; ray_setup(&r, o, d);
  double best = tmax; int32_t bp = -1; int found = 0;
  if (!s->use_bvh) {
    for (int64_t i = 0; i < s->n; ++i) {
      double t = tri_hit(&r, s->tri + 9*i, tmax);
      if (nt) ++*nt;
      if (t > 0 && (!found || t < best || (t == best && i < bp))) { best = t; bp = (int32_t)i; found = 1; }
    }
  } else if (s->n_nodes > 0) {
    int32_t stack[128]; int sp = 0; stack[sp++] = 0;
    while (sp) {
      const node_t* nd = &s->nodes[stack[--sp]];
      double tn;
      if (nv) ++*nv;
      if (!box_hit(&r, nd, found ? best * (1.0 + 2.0 * GAMMA3) : tmax, &tn)) continue;
      if (nd->count > 0) {
        for (int32_t i = 0; i < nd->count; ++i) {
          int32_t p = s->perm[nd->first + i];
          double t = tri_hit(&r, s->tri + 9*(int64_t)p, tmax);
          if (nt) ++*nt;
          if (t > 0 && (!found || t < best || (t == best && p < bp))) { best = t; bp = p; found = 1; }
        }
      } else {
        double tl, tr;
        int hl = box_hit(&r, &s->nodes[nd->left], found ? best * (1.0 + 2.0 * GAMMA3) : tmax, &tl);
        int hr = box_hit(&r, &s->nodes[nd->right], found ? best * (1.0 + 2.0 * GAMMA3) : tmax, &tr);
        if (hl && hr) {
          if (tl <= tr) { stack[sp++] = nd->right; stack[sp++] = nd->left; }
          else { stack[sp++] = nd->left; stack[sp++] = nd->right; }
        } else if (hl) stack[sp++] = nd->left;
        else if (hr) stack[sp++] = nd->right;
      }
    }
  }
  *t_out = found ? best : INFINITY;
  *p_out = found ? bp : -1;
}

static int occluded_n(const orc_scene* s, const double* o, const double* d, double tmax,
                      int64_t* nv, int64_t* nt) {
  ray_t r; ray_setup(&r, o, d);
  if (!s->use_bvh) {
    for (int64_t i = 0; i < s->n; ++i) {
      if (nt) ++*nt;
      if (tri_hit(&r, s->tri + 9*i, tmax) > 0) return 1;
    }
    return 0;
  }
  if (s->n_nodes == 0) return 0;
  int32_t stack[128]; int sp = 0; stack[sp++] = 0;
  while (sp) {
    const node_t* nd = &s->nodes[stack[--sp]];
    double tn;
    if (nv) ++*nv;
    if (!box_hit(&r, nd, tmax, &tn)) continue;
    if (nd->count > 0) {
      for (int32_t i = 0; i < nd->count; ++i) {
        if (nt) ++*nt;
        if (tri_hit(&r, s->tri + 9*(int64_t)s->perm[nd->first + i], tmax) > 0) return 1;
      }
    } else { stack[sp++] = nd->left; stack[sp++] = nd->right; }
  }
  return 0;
}

static int occluded(const orc_scene* s, const double* o, const double* d, double tmax) {
  return occluded_n(s, o, d, tmax, NULL, NULL);
}

void orc_intersect(const orc_scene* s, const double* o, const double* d, const double* tmax,
                   int64_t n, double* t_out, int32_t* prim_out, int64_t* node_visits,
                   int64_t* tri_tests) {
  int64_t nv = 0, nt = 0;
  for (int64_t i = 0; i < n; ++i)
    closest(s, o + 3*i, d + 3*i, tmax ? tmax[i] : INFINITY, t_out + i, prim_out + i, &nv, &nt);
  if (node_visits) *node_visits = nv;
  if (tri_tests) *tri_tests = nt;
}

void orc_occluded(const orc_scene* s, const double* o, const double* d, const double* tmax,
                  int64_t n, uint8_t* hit_out) {
  for (int64_t i = 0; i < n; ++i) hit_out[i] = (uint8_t)occluded(s, o + 3*i, d + 3*i, tmax[i]);
}

/* ------------------------------------------------------------------- BSDFs */
static void onb(const double* n, double* t, double* b) {
  double sgn = n[2] >= 0.0 ? 1.0 : -1.0;
  double a = -1.0 / (sgn + n[2]);
  double bb = n[0] * n[1] * a;
  t[0] = 1.0 + sgn * n[0] * n[0] * a; t[1] = sgn * bb; t[2] = -sgn * n[0];
  b[0] = bb; b[1] = sgn + n[1] * n[1] * a; b[2] = -n[1];
}

static double ggx_D(const double* m, double a2) {
  double c2 = m[2] * m[2];
  double den = c2 * (a2 - 1.0) + 1.0;
  return a2 / (M_PI * den * den);
}
static double ggx_G1(const double* v, double a2) {
  return 2.0 * v[2] / (v[2] + sqrt(a2 + (1.0 - a2) * v[2] * v[2]));
}

/* f * cos(theta_i) and the solid-angle pdf of sampling wi, local frame */
static void bsdf_eval(const double* mt, const double* wo, const double* wi, double* fcos, double* pdf) {
  int type = (int)mt[4];
  if (type == 0) {
    for (int k = 0; k < 3; ++k) fcos[k] = mt[k] * wi[2] / M_PI;
    *pdf = wi[2] / M_PI;
    return;
  }
  double a = mt[3], a2 = a * a;
  double h[3] = {wo[0]+wi[0], wo[1]+wi[1], wo[2]+wi[2]};
  normalize3(h);
  double D = ggx_D(h, a2), G1o = ggx_G1(wo, a2), G1i = ggx_G1(wi, a2);
  double c = 1.0 - dot3(wi, h);
  double c5 = c * c * c * c * c;
  for (int k = 0; k < 3; ++k) {
    double F = mt[k] + (1.0 - mt[k]) * c5;
    fcos[k] = D * G1o * G1i * F / (4.0 * wo[2]);
  }
  *pdf = G1o * D / (4.0 * wo[2]);
}

/* returns 0 if the path ends; weight = f cos / pdf */
static int bsdf_sample(const double* mt, const double* wo, double u0, double u1, double* wi,
                       double* weight, double* pdf) {
  int type = (int)mt[4];
  if (type == 0) {
    double r = sqrt(u0), phi = 2.0 * M_PI * u1;
    wi[0] = r * cos(phi); wi[1] = r * sin(phi); wi[2] = sqrt(fmax(0.0, 1.0 - u0));
    if (!(wi[2] > 0.0)) return 0;
    for (int k = 0; k < 3; ++k) weight[k] = mt[k];
    *pdf = wi[2] / M_PI;
    return 1;
  }
  double a = mt[3], a2 = a * a;
  /* visible-normal sampling in the hemisphere configuration */
  double vh[3] = {a * wo[0], a * wo[1], wo[2]};
  normalize3(vh);
  double lensq = vh[0] * vh[0] + vh[1] * vh[1];
  double T1[3], T2[3];
  if (lensq > 0.0) { double il = 1.0 / sqrt(lensq); T1[0] = -vh[1]*il; T1[1] = vh[0]*il; T1[2] = 0.0; }
  else { T1[0] = 1.0; T1[1] = 0.0; T1[2] = 0.0; }
  cross3(vh, T1, T2);
  double r = sqrt(u0), phi = 2.0 * M_PI * u1;
  double t1 = r * cos(phi), t2 = r * sin(phi);
  double sb = 0.5 * (1.0 + vh[2]);
  t2 = (1.0 - sb) * sqrt(1.0 - t1 * t1) + sb * t2;
  double tz = sqrt(fmax(0.0, 1.0 - t1 * t1 - t2 * t2));
  double nh[3];
  for (int k = 0; k < 3; ++k) nh[k] = t1 * T1[k] + t2 * T2[k] + tz * vh[k];
  double m[3] = {a * nh[0], a * nh[1], fmax(0.0, nh[2])};
  normalize3(m);
  double om = dot3(wo, m);
  for (int k = 0; k < 3; ++k) wi[k] = 2.0 * om * m[k] - wo[k];
  if (!(wi[2] > 0.0)) return 0;
  double c = 1.0 - dot3(wi, m);
  double c5 = c * c * c * c * c;
  double G1i = ggx_G1(wi, a2);
  for (int k = 0; k < 3; ++k) weight[k] = (mt[k] + (1.0 - mt[k]) * c5) * G1i;
  *pdf = ggx_G1(wo, a2) * ggx_D(m, a2) / (4.0 * wo[2]);
  return 1;
}

/* ------------------------------------------------------------------ render */
static void philox_u(uint32_t pix, uint32_t smp, uint32_t frame, uint32_t w3,
                     const uint32_t key[2], double u[4]) {
  uint32_t c[4] = {pix, smp, frame, w3}, o[4];
  orc_philox_block(c, key, o);
  for (int k = 0; k < 4; ++k) u[k] = u01(o[k]);
}

/* cond (optional, test infrastructure): the smallest light-side cosine of any
 * emitter hit or next-event sample, the smallest surface-side cosine of any
 * next-event sample, and the smallest roughness of any GGX shading point along
 * the path -- the quantities whose smallness amplifies the kernel's FP32
 * rounding (updated with min, so a pixel's samples share one record) */
static void cond_min(double* cond, int i, double v) {
  if (cond && v < cond[i]) cond[i] = v;
}

static void trace_sample(const orc_scene* s, const float* cam, int W, int H, int x, int y,
                         int smp, int frame, int max_depth, const uint32_t key[2], double* Lo,
                         int32_t* rec, int64_t* work, double* cond) {
  uint32_t pix = (uint32_t)(y * W + x);
  double u[4];
  philox_u(pix, (uint32_t)smp, (uint32_t)frame, 0u, key, u);
  double th = tan(0.5 * (double)cam[12] * M_PI / 180.0);
  double px = (2.0 * (x + u[0]) / W - 1.0) * th * ((double)W / (double)H);
  double py = (1.0 - 2.0 * (y + u[1]) / H) * th;
  double dc[3] = {px, py, -1.0};
  double o[3] = {cam[0], cam[1], cam[2]}, d[3];
  for (int i = 0; i < 3; ++i) d[i] = cam[3+3*i]*dc[0] + cam[3+3*i+1]*dc[1] + cam[3+3*i+2]*dc[2];
  normalize3(d);
  double beta[3] = {1, 1, 1}, L[3] = {0, 0, 0}, prev_pdf = 0.0;
  for (int b = 1; b <= max_depth; ++b) {
    double t; int32_t prim;
    closest(s, o, d, INFINITY, &t, &prim, &work[1], &work[2]);
    ++work[0];
    if (rec) rec[2*(b-1)] = prim;
    if (prim < 0) { for (int k = 0; k < 3; ++k) L[k] += beta[k] * s->env; break; }
    double x3[3] = {o[0] + t*d[0], o[1] + t*d[1], o[2] + t*d[2]};
    uint32_t m = s->mat[prim];
    if (m & LIGHT_BIT) {
      const light_t* lt = &s->lights[m & ~LIGHT_BIT];
      double cosl = -dot3(d, lt->n);
      if (cosl > 0.0) {
        if (b > 1) cond_min(cond, 0, cosl);
        double w = 1.0;
        if (b > 1) {
          double pl = lt->prob * t * t / (cosl * lt->area);
          w = prev_pdf * prev_pdf / (prev_pdf * prev_pdf + pl * pl);
        }
        for (int k = 0; k < 3; ++k) L[k] += beta[k] * lt->L[k] * w;
      }
      break;
    }
    if (b == max_depth) break;
    const double* v = s->tri + 9*(int64_t)prim;
    double e1[3], e2[3], ng[3];
    sub3(v + 3, v, e1); sub3(v + 6, v, e2); cross3(e1, e2, ng); normalize3(ng);
    double wo[3] = {-d[0], -d[1], -d[2]};
    if (dot3(ng, wo) < 0.0) { ng[0] = -ng[0]; ng[1] = -ng[1]; ng[2] = -ng[2]; }
    double eps = 1e-4 * (1.0 + fmax(fabs(x3[0]), fmax(fabs(x3[1]), fabs(x3[2]))));
    double on[3] = {x3[0] + ng[0]*eps, x3[1] + ng[1]*eps, x3[2] + ng[2]*eps};
    double tt[3], bt[3];
    onb(ng, tt, bt);
    double wol[3] = {dot3(wo, tt), dot3(wo, bt), dot3(wo, ng)};
    const double* mt = s->mats + 8 * (int64_t)m;
    if ((int)mt[4] == 1) cond_min(cond, 2, mt[3]);
    if (s->n_l > 0) {
      philox_u(pix, (uint32_t)smp, (uint32_t)frame, (uint32_t)(4*b + 1), key, u);
      int j = 0;
      while (j < s->n_l - 1 && !(u[0] < s->cdf[j])) ++j;
      const light_t* lt = &s->lights[j];
      double p[3], vv[3];
      for (int k = 0; k < 3; ++k) p[k] = lt->p0[k] + u[1] * lt->e1[k] + u[2] * lt->e2[k];
      sub3(p, on, vv);
      double dist2 = dot3(vv, vv), dist = sqrt(dist2);
      double wi[3] = {vv[0]/dist, vv[1]/dist, vv[2]/dist};
      double cosi = dot3(wi, ng), cosl = -dot3(wi, lt->n);
      int32_t nrec = -1;
      if (cosi > 0.0 && cosl > 0.0) {
        cond_min(cond, 0, cosl);
        cond_min(cond, 1, cosi);
        int vis = !occluded_n(s, on, wi, dist * (1.0 - 1e-4), &work[1], &work[2]);
        ++work[0];
        nrec = 2 * j + vis;
        if (vis) {
          double wil[3] = {dot3(wi, tt), dot3(wi, bt), cosi}, fc[3], pb;
          bsdf_eval(mt, wol, wil, fc, &pb);
          double pl = lt->prob * dist2 / (cosl * lt->area);
          double w = pl * pl / (pl * pl + pb * pb);
          for (int k = 0; k < 3; ++k) L[k] += beta[k] * fc[k] * lt->L[k] * w / pl;
        }
      }
      if (rec) rec[2*(b-1) + 1] = nrec;
    }
    philox_u(pix, (uint32_t)smp, (uint32_t)frame, (uint32_t)(4*b + 2), key, u);
    double wil[3], wgt[3], pdf;
    if (!bsdf_sample(mt, wol, u[0], u[1], wil, wgt, &pdf)) break;
    for (int k = 0; k < 3; ++k) {
      beta[k] *= wgt[k];
      d[k] = wil[0] * tt[k] + wil[1] * bt[k] + wil[2] * ng[k];
      o[k] = on[k];
    }
    prev_pdf = pdf;
  }
  for (int k = 0; k < 3; ++k) Lo[k] = L[k];
}

int orc_render(const orc_scene* s, const float* cams, int F, int first_frame, int W, int H,
               int y0, int y1, int spp, int max_depth, uint64_t seed, double* rgb,
               int32_t* records, double* cond, int nthreads, int64_t* work_out) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  int64_t tot_r = 0, tot_v = 0, tot_t = 0;
  int64_t rows = y1 - y0;
  int64_t npix = rows * W;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
  for (int f = 0; f < F; ++f) {
    const float* cam = cams + 13 * f;
    int64_t cr = 0, cv = 0, ct = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+:cr, cv, ct)
    for (int64_t q = 0; q < npix; ++q) {
      int y = y0 + (int)(q / W), x = (int)(q % W);
      double acc[3] = {0, 0, 0};
      for (int smp = 0; smp < spp; ++smp) {
        double Ls[3];
        int32_t* rec = NULL;
        if (records) {
          rec = records + ((((int64_t)f * H + y) * W + x) * spp + smp) * max_depth * 2;
          for (int i = 0; i < 2 * max_depth; ++i) rec[i] = (i % 2 == 0) ? -2 : -1;
        }
        int64_t work[3] = {0, 0, 0};
        double* cd = cond ? cond + (((int64_t)f * H + y) * W + x) * 3 : NULL;
        if (cd && smp == 0) cd[0] = cd[1] = cd[2] = INFINITY;
        trace_sample(s, cam, W, H, x, y, smp, first_frame + f, max_depth, key, Ls, rec, work, cd);
        cr += work[0]; cv += work[1]; ct += work[2];
        for (int k = 0; k < 3; ++k) acc[k] += Ls[k];
      }
      double* out = rgb + (((int64_t)f * H + y) * W + x) * 3;
      for (int k = 0; k < 3; ++k) out[k] = acc[k] / spp;
    }
    tot_r += cr; tot_v += cv; tot_t += ct;
  }
  if (work_out) { work_out[0] = tot_r; work_out[1] = tot_v; work_out[2] = tot_t; }
  return 0;
}

/* ------------------------------------------------------------- test hooks */
/* mat: {albedo r,g,b, roughness, type}; local-frame directions (normal = +z) */
void orc_bsdf_eval(const double* mat5, const double* wo, const double* wi, int64_t n,
                   double* fcos, double* pdf) {
  double mt[8] = {mat5[0], mat5[1], mat5[2], mat5[3], mat5[4], 0, 0, 0};
  for (int64_t i = 0; i < n; ++i) bsdf_eval(mt, wo + 3*i, wi + 3*i, fcos + 3*i, pdf + i);
}

void orc_bsdf_sample(const double* mat5, const double* wo, const double* u, int64_t n,
                     double* wi, double* weight, double* pdf, int32_t* ok) {
  double mt[8] = {mat5[0], mat5[1], mat5[2], mat5[3], mat5[4], 0, 0, 0};
  for (int64_t i = 0; i < n; ++i)
    ok[i] = bsdf_sample(mt, wo + 3*i, u[2*i], u[2*i+1], wi + 3*i, weight + 3*i, pdf + i);
}

/* nodes: [n_nodes][6] bounds (lo, hi); links: [n_nodes][4] (left, right, first, count) */
void orc_bvh_export(const orc_scene* s, double* bounds, int32_t* links, int32_t* perm) {
  for (int64_t i = 0; i < s->n_nodes; ++i) {
    const node_t* nd = &s->nodes[i];
    for (int k = 0; k < 3; ++k) { bounds[6*i+k] = nd->lo[k]; bounds[6*i+3+k] = nd->hi[k]; }
    links[4*i] = nd->left; links[4*i+1] = nd->right; links[4*i+2] = nd->first; links[4*i+3] = nd->count;
  }
  for (int64_t i = 0; i < s->n; ++i) perm[i] = s->perm[i];
}

/* ------------------------------------------------------------- annotations
 * Per pixel and frame, from the ray through the pixel centre (u = 1/2), the
 * free by-products of the primary hit (the paper's outputs carry extra
 * annotations such as depth and segmentation, Sec. 1):
 *   depth     distance of the hit along the viewing axis -c2 (t cos), +inf on a miss
 *   normal    unit geometric normal e1 x e2, turned to face the ray (0 on a miss)
 *   prim      triangle index, -1 on a miss; material: the triangle's material
 *             word (light triangles: LIGHT_BIT | light index), -1 on a miss
 *   flow      where the hit point lands in the next frame's image minus this
 *             pixel's centre, in pixels (x right, y down); NaN on a miss,
 *             without a next camera, or when the point is behind it
 * The next camera of frame f is cams[f + 1], and next_cam (may be NULL) for
 * the last frame. */
static void project(const float* cam, int W, int H, const double* p, double* xy) {
  double q[3] = {p[0] - cam[0], p[1] - cam[1], p[2] - cam[2]};
  double a = q[0]*cam[3] + q[1]*cam[6] + q[2]*cam[9];
  double b = q[0]*cam[4] + q[1]*cam[7] + q[2]*cam[10];
  double c = q[0]*cam[5] + q[1]*cam[8] + q[2]*cam[11];
  if (!(c < 0.0)) { xy[0] = xy[1] = NAN; return; }
  double th = tan(0.5 * (double)cam[12] * M_PI / 180.0);
  double px = a / -c, py = b / -c;
  xy[0] = (px / (th * ((double)W / (double)H)) + 1.0) * 0.5 * W;
  xy[1] = (1.0 - py / th) * 0.5 * H;
}

void orc_annotations(const orc_scene* s, const float* cams, int F, const float* next_cam, int W,
                     int H, double* depth, double* normal, int32_t* prim, int64_t* material,
                     double* flow) {
  for (int f = 0; f < F; ++f) {
    const float* cam = cams + 13 * f;
    const float* nxt = f + 1 < F ? cams + 13 * (f + 1) : next_cam;
    double th = tan(0.5 * (double)cam[12] * M_PI / 180.0);
#pragma omp parallel for schedule(dynamic, 16)
    for (int y = 0; y < H; ++y) {
      for (int x = 0; x < W; ++x) {
        int64_t o = ((int64_t)f * H + y) * W + x;
        double px = (2.0 * (x + 0.5) / W - 1.0) * th * ((double)W / (double)H);
        double py = (1.0 - 2.0 * (y + 0.5) / H) * th;
        double dc[3] = {px, py, -1.0}, org[3] = {cam[0], cam[1], cam[2]}, d[3];
        for (int i = 0; i < 3; ++i) d[i] = cam[3+3*i]*dc[0] + cam[3+3*i+1]*dc[1] + cam[3+3*i+2]*dc[2];
        normalize3(d);
        double t; int32_t p;
        closest(s, org, d, INFINITY, &t, &p, NULL, NULL);
        prim[o] = p;
        if (p < 0) {
          depth[o] = INFINITY;
          normal[3*o] = normal[3*o+1] = normal[3*o+2] = 0.0;
          material[o] = -1;
          flow[2*o] = flow[2*o+1] = NAN;
          continue;
        }
        double axis[3] = {-cam[5], -cam[8], -cam[11]};
        depth[o] = t * dot3(d, axis);
        const double* v = s->tri + 9 * (int64_t)p;
        double e1[3], e2[3], n[3];
        sub3(v + 3, v, e1); sub3(v + 6, v, e2); cross3(e1, e2, n); normalize3(n);
        if (dot3(n, d) > 0) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; }
        for (int k = 0; k < 3; ++k) normal[3*o+k] = n[k];
        material[o] = (int64_t)s->mat[p];
        if (!nxt) { flow[2*o] = flow[2*o+1] = NAN; continue; }
        double hp[3] = {org[0] + t*d[0], org[1] + t*d[1], org[2] + t*d[2]}, xy[2];
        project(nxt, W, H, hp, xy);
        flow[2*o] = xy[0] - (x + 0.5);
        flow[2*o+1] = xy[1] - (y + 0.5);
      }
    }
  }
}
