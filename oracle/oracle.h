/*
 * Oracle for the EventTracer hot path (arXiv 2508.18071) -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU restatement of what the method computes.  Only the
 * test-suite, the smoke check and the benchmark's CPU-baseline leg may load
 * it.  It shares no code with the CUDA library.
 *
 * Paper references are to sections / equations of the paper:
 *   Sec. 3.2, Eq. 1   luminance, log map, log differences X_k
 *   Sec. 3.3, Eq. 2-3 LIF / BiLIF charge, fire, reset
 *   Sec. 3.3, Eq. 5-6 EvSNet convolutions and projection
 *   Sec. 3.1          contrast-threshold event model (events fire when the
 *                     log change exceeds the contrast threshold)
 * The path tracer's estimator is not specified by the paper beyond
 * "Monte Carlo path tracing" (Sec. 3.2); the estimator below is the project's
 * specification, written once here in FP64.
 */
#ifndef ET_ORACLE_H
#define ET_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), n independent blocks. */
void orc_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n);
void orc_philox_block(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

typedef struct orc_scene orc_scene;

/* tri: [n][9] float32 (v0,v1,v2); mat: [n] material index.
 * mats: [n_mat][8] doubles {albedo r,g,b, roughness, type(0 Lambert,1 GGX), 0,0,0}
 * lights: [n_l][12] floats {p0[3], e1[3], e2[3], radiance[3]}; each light adds two
 * emitting triangles (p0,p0+e1,p0+e1+e2) and (p0,p0+e1+e2,p0+e2) after the user's.
 * use_bvh = 0 selects brute-force intersection (every triangle tested).   */
orc_scene* orc_scene_new(const float* tri, const uint32_t* mat, int64_t n,
                         const double* mats, int n_mat, const float* lights, int n_l,
                         double env, int use_bvh);
void orc_scene_free(orc_scene* s);
int64_t orc_scene_ntris(const orc_scene* s);
double orc_bvh_sah_cost(const orc_scene* s);
int64_t orc_bvh_nodes(const orc_scene* s);

/* closest hit for rays (o,d) with t in (0, tmax): t (inf on miss), prim (-1 on miss) */
void orc_intersect(const orc_scene* s, const double* o, const double* d, const double* tmax,
                   int64_t n, double* t_out, int32_t* prim_out, int64_t* node_visits,
                   int64_t* tri_tests);
/* any hit with t in (0, tmax) */
void orc_occluded(const orc_scene* s, const double* o, const double* d, const double* tmax,
                  int64_t n, uint8_t* hit_out);

/* cams: [F][13] floats {pos[3], rot[9] row-major camera-to-world, vfov_deg}
 * rgb: [F][H][W][3] double; rows [y0,y1) only.  records (optional):
 * [F][H][W][spp][max_depth][2] int32: (primID of segment b or -1 miss, -2 untraced),
 * (NEE record: 2*light + visible, -1 none).  cond (optional): [F][H][W][3]
 * double, over the pixel's samples the smallest light-side cosine (emitter hit
 * after the first segment, or next-event sample), surface-side cosine of a
 * next-event sample and GGX roughness at a shading point (+inf if none). */
int orc_render(const orc_scene* s, const float* cams, int F, int first_frame, int W, int H,
               int y0, int y1, int spp, int max_depth, uint64_t seed, double* rgb,
               int32_t* records, double* cond, int nthreads, int64_t* work);
/* work (optional): [3] = rays traced, BVH nodes visited, triangles tested */

/* Eq. 1: luminance and log map of linear RGB.  mode 0: ln(L + eps); mode 1: the
 * paper's lin-log with threshold rho. Output is rounded to float32. */
void orc_logl(const double* rgb, int64_t n, int mode, double eps_or_rho, float* logl);

/* contrast-threshold generator (Sec. 3.1).  logl [F][H][W] float32; ref [H*W] double
 * state; if *initialized == 0 the first frame only sets ref.  events out [cap][4]
 * int32 {x, y, t, p}; returns number of events (may exceed cap: only cap written). */
int64_t orc_threshold_events(const float* logl, int F, int H, int W, double C, int t0,
                             double* ref, int* initialized, int32_t* events, int64_t cap);

/* EvSNet forward (Eq. 5-6 with Eq. 2-3 BiLIF).  See events.c for the layer packing. */
int64_t orc_evsnet_forward(const float* logl, int F, int H, int W, int kind, int n_layers,
                           int C, int kt, int ks, int ks0, int delay, double beta, double vth,
                           double reset, const double* w, const double* b, int t0, double* V,
                           double* hist, double* last_l, int* initialized, int32_t* events,
                           int64_t cap, double* I_out, double* margin, int nthreads);

/* test hooks: BSDF in a local frame (normal +z); mat5 = {albedo rgb, roughness, type} */
void orc_bsdf_eval(const double* mat5, const double* wo, const double* wi, int64_t n,
                   double* fcos, double* pdf);
void orc_bsdf_sample(const double* mat5, const double* wo, const double* u, int64_t n,
                     double* wi, double* weight, double* pdf, int32_t* ok);
void orc_bvh_export(const orc_scene* s, double* bounds, int32_t* links, int32_t* perm);

/* event-sensor model (sensor.c): state [H*W][3] = (r, t_last, previous log
   intensity); events [n][4] int64 {x, y, t in microseconds, p} */
int64_t orc_sensor_events(const float* logl, int F, int H, int W, double C, double sigma,
                          double refractory_us, double leak_hz, double shot_hz, double frame_hz,
                          uint64_t seed, int t0, double* state, int* initialized,
                          int64_t* events, int64_t cap);
void orc_sensor_thresholds(int64_t npix, double C, double sigma, uint64_t seed, double* out);

/* primary-hit annotations through pixel centres (trace.c): depth [F][H][W],
   normal [F][H][W][3], prim [F][H][W], material [F][H][W] (-1: miss),
   flow [F][H][W][2]; next_cam: camera after the last frame or NULL */
void orc_annotations(const orc_scene* s, const float* cams, int F, const float* next_cam, int W,
                     int H, double* depth, double* normal, int32_t* prim, int64_t* material,
                     double* flow);

/* number of matched pairs between two event lists [n][4] {x,y,t,p} */
int64_t orc_event_matches(const int32_t* A, int64_t na, const int32_t* B, int64_t nb, int delta);

#ifdef __cplusplus
}
#endif
#endif
