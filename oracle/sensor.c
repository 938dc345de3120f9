/*
 * Oracle -- TEST INFRASTRUCTURE ONLY.
 * Event-sensor model with sub-frame timestamps and the non-idealities the paper
 * lists next to internal-state bias and saturation (Sec. 3.1: threshold
 * mismatch, leak events, shot noise; the reset period behind the saturation
 * effect).  The paper gives no formulas for them; this is the project's
 * reading, written as plainly as possible:
 *
 *   time            frames; frame k (absolute index) is at t = k; between two
 *                   frames the log intensity is linear in t
 *   thresholds      per pixel C_on = C max(0.01, 1 + sigma z_on), C_off likewise,
 *                   z = (u0 + u1 + u2 + u3 - 2) sqrt(3) (Irwin-Hall of four
 *                   uniforms, unit variance); u from Philox4x32-10, key = seed,
 *                   counter (pixel, 0xFFFFFFFF, 0 for ON / 1 for OFF, TAG)
 *   state           reference level r, time of the last event t_last and the
 *                   previous frame's log intensity (the call may start mid-clip)
 *   step (k-1 -> k) 1. leak: r <- r - C_on * leak_hz / frame_hz
 *                   2. repeat: lo = max(k - 1, t_last + T_ref); the pixel fires
 *                      at the earliest t in [lo, k] with l(t) - r >= C_on (ON) or
 *                      r - l(t) >= C_off (OFF); then r <- r +- C_on/off,
 *                      t_last <- t; stop when no such t exists
 *                   3. shot noise: with probability shot_hz / frame_hz an extra
 *                      event at t = k - 1 + v, polarity + if w < 1/2 else -,
 *                      (p, v, w) from Philox counter (pixel, k, 2, TAG); it does
 *                      not touch the state
 *   output          (x, y, floor(t * 1e6 / frame_hz) microseconds, polarity)
 * With sigma = 0, no refractory period, no leak and no shot noise every step
 * emits floor(|l_k - r| / C) events, as the contrast-threshold generator (up
 * to 1024 per pixel and step: a bound on the work, further crossings of that
 * step are dropped).
 */
#include <math.h>
#include <stdint.h>
#include "oracle.h"

#define SENSOR_TAG 0x53454E53u   /* "SENS" */
#define MAX_PER_STEP 1024         /* events of one pixel in one step; further crossings are dropped */

static double u01(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

static void draw4(uint32_t c0, uint32_t c1, uint32_t c2, uint64_t seed, double u[4]) {
  uint32_t ctr[4] = {c0, c1, c2, SENSOR_TAG};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t o[4];
  orc_philox_block(ctr, key, o);
  for (int i = 0; i < 4; ++i) u[i] = u01(o[i]);
}

static double mismatch(uint32_t pix, int which, uint64_t seed, double C, double sigma) {
  double u[4];
  draw4(pix, 0xFFFFFFFFu, (uint32_t)which, seed, u);
  double z = (u[0] + u[1] + u[2] + u[3] - 2.0) * sqrt(3.0);
  double f = 1.0 + sigma * z;
  if (f < 0.01) f = 0.01;
  return C * f;
}

void orc_sensor_thresholds(int64_t npix, double C, double sigma, uint64_t seed, double* out) {
  for (int64_t q = 0; q < npix; ++q) {
    out[2 * q] = mismatch((uint32_t)q, 0, seed, C, sigma);
    out[2 * q + 1] = mismatch((uint32_t)q, 1, seed, C, sigma);
  }
}

/* log intensity at time t of the step from a = k - 1 (value la) to a + 1 (lb) */
static double lerp_at(double la, double lb, double a, double t) { return la + (lb - la) * (t - a); }

int64_t orc_sensor_events(const float* logl, int F, int H, int W, double C, double sigma,
                          double refractory_us, double leak_hz, double shot_hz, double frame_hz,
                          uint64_t seed, int t0, double* state, int* initialized,
                          int64_t* events, int64_t cap) {
  const int64_t npix = (int64_t)H * W;
  const double t_ref = refractory_us * frame_hz * 1e-6;   /* frames */
  const double leak = leak_hz / frame_hz;                  /* thresholds per frame */
  const double p_shot = shot_hz / frame_hz;
  const double us_per_frame = 1e6 / frame_hz;
  int64_t n = 0;
  int f0 = 0;
  if (!*initialized) {
    if (F == 0) return 0;
    for (int64_t q = 0; q < npix; ++q) {
      state[3 * q] = (double)logl[q];
      state[3 * q + 1] = -1e300;
      state[3 * q + 2] = (double)logl[q];
    }
    *initialized = 1;
    f0 = 1;
  }
  for (int64_t q = 0; q < npix; ++q) {
    const double c_on = mismatch((uint32_t)q, 0, seed, C, sigma);
    const double c_off = mismatch((uint32_t)q, 1, seed, C, sigma);
    double r = state[3 * q], t_last = state[3 * q + 1], l_prev = state[3 * q + 2];
    for (int f = f0; f < F; ++f) {
      const int k = t0 + f;
      const double a = (double)(k - 1), b = (double)k;
      const double la = l_prev;
      const double lb = (double)logl[(int64_t)f * npix + q];
      r = r - c_on * leak;
      for (int n_step = 0;; ++n_step) {
        if (n_step >= MAX_PER_STEP) break;
        const double lo = t_last + t_ref > a ? t_last + t_ref : a;
        if (lo > b) break;
        const double l_lo = lerp_at(la, lb, a, lo);
        const double L_on = r + c_on, L_off = r - c_off;
        int has_on = 0, has_off = 0;
        double t_on = 0.0, t_off = 0.0;
        /* l is linear: if it is below the level at lo but reaches it by k, it
           crosses it once in between */
        if (l_lo >= L_on) { has_on = 1; t_on = lo; }
        else if (lb >= L_on) { has_on = 1; t_on = a + (L_on - la) / (lb - la); }
        if (l_lo <= L_off) { has_off = 1; t_off = lo; }
        else if (lb <= L_off) { has_off = 1; t_off = a + (L_off - la) / (lb - la); }
        if (has_on && t_on < lo) t_on = lo;     /* rounding of the crossing time */
        if (has_off && t_off < lo) t_off = lo;
        int p;
        double t;
        if (has_on && (!has_off || t_on <= t_off)) { p = 1; t = t_on; }
        else if (has_off) { p = -1; t = t_off; }
        else break;
        if (t > b) t = b;
        if (n < cap) {
          events[4 * n] = q % W; events[4 * n + 1] = q / W;
          events[4 * n + 2] = (int64_t)floor(t * us_per_frame); events[4 * n + 3] = p;
        }
        ++n;
        const double r_new = p > 0 ? r + c_on : r - c_off;
        t_last = t;
        if (r_new == r) break;                  /* threshold below the resolution of r */
        r = r_new;
      }
      if (p_shot > 0.0) {
        double u[4];
        draw4((uint32_t)q, (uint32_t)k, 2u, seed, u);
        if (u[0] < p_shot) {
          if (n < cap) {
            events[4 * n] = q % W; events[4 * n + 1] = q / W;
            events[4 * n + 2] = (int64_t)floor((a + u[1]) * us_per_frame);
            events[4 * n + 3] = u[2] < 0.5 ? 1 : -1;
          }
          ++n;
        }
      }
      l_prev = lb;
    }
    state[3 * q] = r;
    state[3 * q + 1] = t_last;
    state[3 * q + 2] = l_prev;
  }
  return n;
}
