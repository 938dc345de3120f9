/*
 * Oracle -- TEST INFRASTRUCTURE ONLY.
 * FP64 restatements of the event stage:
 *   Eq. 1      luminance L = 0.2126 R + 0.7152 G + 0.0722 B and its log map;
 *              X_k = L^log_k - L^log_{k-1}
 *   Sec. 3.1   contrast-threshold events: a pixel fires whenever its log change
 *              since the last event reaches the threshold C, one event per
 *              multiple of C, polarity the sign of the change
 *   Eq. 2-3    BiLIF: V' = beta V + I; S = sgn(V') 1(|V'| >= Vth); V = V' - r S
 *   Eq. 5-6    EvSNet: convolutional encoder, ReLU, residual blocks, point-wise
 *              projection to one input current per pixel and step, then BiLIF
 * Readings where the paper is silent: fire on the pre-reset potential V';
 * soft reset by r (r = Vth by default); causal temporal padding; zero spatial
 * padding at the image border; bias on every convolution.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include "oracle.h"

void orc_logl(const double* rgb, int64_t n, int mode, double p, float* out) {
  for (int64_t i = 0; i < n; ++i) {
    double L = 0.2126 * rgb[3*i] + 0.7152 * rgb[3*i+1] + 0.0722 * rgb[3*i+2];
    double l;
    if (mode == 0) l = log(L + p);
    else l = (L >= p) ? log(L) : (log(p) / p) * L;
    out[i] = (float)l;
  }
}

int64_t orc_threshold_events(const float* logl, int F, int H, int W, double C, int t0,
                             double* ref, int* initialized, int32_t* events, int64_t cap) {
  int64_t n = 0, npix = (int64_t)H * W;
  int f0 = 0;
  if (!*initialized) {
    if (F == 0) return 0;
    for (int64_t q = 0; q < npix; ++q) ref[q] = (double)logl[q];
    *initialized = 1;
    f0 = 1;
  }
  for (int f = f0; f < F; ++f) {
    for (int64_t q = 0; q < npix; ++q) {
      double d = (double)logl[(int64_t)f * npix + q] - ref[q];
      double k = floor(fabs(d) / C);
      if (k > 0.0) {
        int p = d > 0.0 ? 1 : -1;
        for (int64_t e = 0; e < (int64_t)k; ++e, ++n) {
          if (n < cap) {
            events[4*n] = (int32_t)(q % W); events[4*n+1] = (int32_t)(q / W);
            events[4*n+2] = t0 + f; events[4*n+3] = p;
          }
        }
        ref[q] += (double)p * k * C;
      }
    }
  }
  return n;
}

/* ---------------------------------------------------------------- EvSNet
 * Weight packing (an interface the library states on its own side too):
 * conv layers 0..n_layers-1 in order, each W[Cout][Cin][kt][ks][ks] with
 * Cin = 1 for layer 0 and C otherwise, Cout = C; then the projection W[1][C].
 * Biases: C per conv layer, then 1 for the projection.
 * kind 0 (plain stack): h = ReLU(conv_i(h)) for every layer.
 * kind 1 (residual, Eq. 5): n_layers = 1 + 2M; h0 = ReLU(conv_0(X));
 *   h_i = ReLU(h_{i-1} + conv_{2i}(ReLU(conv_{2i-1}(h_{i-1})))).
 * Temporal taps are causal: tap tau = kt-1 is the current step, tap 0 is
 * kt-1 steps back; steps before the start of the clip contribute zero.
 * hist: [n_layers][kt-1][C][H][W], the input of each layer at the last kt-1
 * steps (slot kt-2 = previous step); only channel 0 is used for layer 0.
 * Spatial stem (ks0 > 0): layer 0 is instead a one-step ks0 x ks0 spatial
 * convolution of the current X, W[C][1][1][ks0][ks0] (zero padding); its
 * history slots are unused.  ks0 = 0: layer 0 has the kt x ks x ks shape.
 * Delay: the events of step k carry t = t0 + k - delay (a centred window
 * labels its output with the window's centre); steps whose label would be
 * negative emit nothing.
 */
static void conv_layer(const double* in, const double* hist, int Cin, int Cout, int C,
                       int kt, int ks, int H, int W, const double* w, const double* b,
                       double* out) {
  int r = ks / 2;
  int64_t npix = (int64_t)H * W;
#pragma omp parallel for schedule(static)
  for (int64_t q = 0; q < npix; ++q) {
    int y = (int)(q / W), x = (int)(q % W);
    for (int co = 0; co < Cout; ++co) {
      double acc = b[co];
      for (int ci = 0; ci < Cin; ++ci)
        for (int tau = 0; tau < kt; ++tau) {
          const double* plane = (tau == kt - 1) ? in + (int64_t)ci * npix
                                                : hist + ((int64_t)tau * C + ci) * npix;
          for (int dy = 0; dy < ks; ++dy)
            for (int dx = 0; dx < ks; ++dx) {
              int yy = y + dy - r, xx = x + dx - r;
              if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
              acc += w[((((int64_t)co * Cin + ci) * kt + tau) * ks + dy) * ks + dx] *
                     plane[(int64_t)yy * W + xx];
            }
        }
      out[(int64_t)co * npix + q] = acc;
    }
  }
}

static void push_hist(double* hist, const double* in, int Cin, int C, int kt, int64_t npix) {
  if (kt <= 1) return;
  for (int tau = 0; tau < kt - 2; ++tau)
    memcpy(hist + (int64_t)tau * C * npix, hist + (int64_t)(tau + 1) * C * npix,
           sizeof(double) * (size_t)(C * npix));
  memcpy(hist + (int64_t)(kt - 2) * C * npix, in, sizeof(double) * (size_t)(Cin * npix));
}

int64_t orc_evsnet_forward(const float* logl, int F, int H, int W, int kind, int n_layers,
                           int C, int kt, int ks, int ks0, int delay, double beta, double vth,
                           double reset, const double* w, const double* b, int t0, double* V,
                           double* hist, double* last_l, int* initialized, int32_t* events,
                           int64_t cap, double* I_out, double* margin, int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
  int64_t npix = (int64_t)H * W, nev = 0;
  int64_t hist_layer = (int64_t)(kt > 1 ? kt - 1 : 0) * C * npix;
  /* per-layer weight / bias offsets */
  int64_t woff[64], boff[64];
  int64_t wo = 0, bo = 0;
  const int kt0 = ks0 > 0 ? 1 : kt, ks0e = ks0 > 0 ? ks0 : ks;   /* layer 0's shape */
  for (int i = 0; i < n_layers; ++i) {
    int cin = i == 0 ? 1 : C;
    woff[i] = wo; boff[i] = bo;
    wo += i == 0 ? (int64_t)C * kt0 * ks0e * ks0e : (int64_t)C * cin * kt * ks * ks;
    bo += C;
  }
  const double* wp = w + wo;
  const double* bp = b + bo;
  double* x = (double*)malloc(sizeof(double) * (size_t)npix);
  double* h = (double*)malloc(sizeof(double) * (size_t)(C * npix));
  double* a = (double*)malloc(sizeof(double) * (size_t)(C * npix));
  double* t = (double*)malloc(sizeof(double) * (size_t)(C * npix));
  int f0 = 0, step = 0;
  if (!*initialized) {
    if (F == 0) { free(x); free(h); free(a); free(t); return 0; }
    for (int64_t q = 0; q < npix; ++q) last_l[q] = (double)logl[q];
    *initialized = 1;
    f0 = 1;
  }
  for (int f = f0; f < F; ++f, ++step) {
    for (int64_t q = 0; q < npix; ++q) {   /* Eq. 1: X_k */
      double l = (double)logl[(int64_t)f * npix + q];
      x[q] = l - last_l[q];
      last_l[q] = l;
    }
    /* encoder */
    conv_layer(x, hist, 1, C, C, kt0, ks0e, H, W, w + woff[0], b + boff[0], h);
    if (kt0 > 1) push_hist(hist, x, 1, C, kt, npix);
    for (int64_t i = 0; i < C * npix; ++i) h[i] = h[i] > 0.0 ? h[i] : 0.0;
    if (kind == 0) {
      for (int l = 1; l < n_layers; ++l) {
        conv_layer(h, hist + l * hist_layer, C, C, C, kt, ks, H, W, w + woff[l], b + boff[l], t);
        push_hist(hist + l * hist_layer, h, C, C, kt, npix);
        for (int64_t i = 0; i < C * npix; ++i) h[i] = t[i] > 0.0 ? t[i] : 0.0;
      }
    } else {
      for (int l = 1; l + 1 < n_layers; l += 2) {
        conv_layer(h, hist + l * hist_layer, C, C, C, kt, ks, H, W, w + woff[l], b + boff[l], a);
        push_hist(hist + l * hist_layer, h, C, C, kt, npix);
        for (int64_t i = 0; i < C * npix; ++i) a[i] = a[i] > 0.0 ? a[i] : 0.0;
        conv_layer(a, hist + (l + 1) * hist_layer, C, C, C, kt, ks, H, W, w + woff[l + 1],
                   b + boff[l + 1], t);
        push_hist(hist + (l + 1) * hist_layer, a, C, C, kt, npix);
        for (int64_t i = 0; i < C * npix; ++i) { double v = h[i] + t[i]; h[i] = v > 0.0 ? v : 0.0; }
      }
    }
    /* Eq. 6: point-wise projection, then BiLIF (Eq. 2-3) */
    for (int64_t q = 0; q < npix; ++q) {
      double I = bp[0];
      for (int c = 0; c < C; ++c) I += wp[c] * h[(int64_t)c * npix + q];
      if (I_out) I_out[(int64_t)step * npix + q] = I;
      double vp = beta * V[q] + I;
      int S = vp >= vth ? 1 : (vp <= -vth ? -1 : 0);
      if (margin) {
        double m = fmin(fabs(vp - vth), fabs(vp + vth));
        if (m < margin[q]) margin[q] = m;
      }
      V[q] = vp - reset * S;
      if (S != 0 && (int64_t)t0 + f - delay >= 0) {
        if (nev < cap) {
          events[4*nev] = (int32_t)(q % W); events[4*nev+1] = (int32_t)(q / W);
          events[4*nev+2] = t0 + f - delay; events[4*nev+3] = S;
        }
        ++nev;
      }
    }
  }
  free(x); free(h); free(a); free(t);
  return nev;
}

/* ---------------------------------------------------------------- event F1
 * Events match when they share (x, y, p) and their frame indices differ by at
 * most delta; each event matches at most once.  Within one (x, y, p) the
 * candidates lie on a line and the admissible pairs form an interval graph, so
 * the greedy scan of both time-sorted lists gives a maximum matching.          */
static int cmp_ev(const void* pa, const void* pb) {
  const int32_t* a = (const int32_t*)pa; const int32_t* b = (const int32_t*)pb;
  static const int order[4] = {1, 0, 3, 2};   /* y, x, p, t */
  for (int i = 0; i < 4; ++i) {
    int k = order[i];
    if (a[k] != b[k]) return a[k] < b[k] ? -1 : 1;
  }
  return 0;
}

int64_t orc_event_matches(const int32_t* A, int64_t na, const int32_t* B, int64_t nb, int delta) {
  int32_t* a = (int32_t*)malloc(sizeof(int32_t) * 4 * (size_t)(na > 0 ? na : 1));
  int32_t* b = (int32_t*)malloc(sizeof(int32_t) * 4 * (size_t)(nb > 0 ? nb : 1));
  memcpy(a, A, sizeof(int32_t) * 4 * (size_t)na);
  memcpy(b, B, sizeof(int32_t) * 4 * (size_t)nb);
  qsort(a, (size_t)na, 4 * sizeof(int32_t), cmp_ev);
  qsort(b, (size_t)nb, 4 * sizeof(int32_t), cmp_ev);
  int64_t i = 0, j = 0, m = 0;
  while (i < na && j < nb) {
    const int32_t* ea = a + 4 * i; const int32_t* eb = b + 4 * j;
    int same = ea[0] == eb[0] && ea[1] == eb[1] && ea[3] == eb[3];
    if (!same) {
      if (cmp_ev(ea, eb) < 0) ++i; else ++j;
      continue;
    }
    int dt = ea[2] - eb[2];
    if (dt >= -delta && dt <= delta) { ++m; ++i; ++j; }
    else if (dt < 0) ++i;
    else ++j;
  }
  free(a); free(b);
  return m;
}
