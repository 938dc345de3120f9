// Per-path arithmetic of the path tracer (paper Sec. 3.2: every frame is path
// traced at low SPP), shared by the one-kernel and the wavefront renderers so
// that both compute identical values.
//
// Estimator (the paper names only "Monte Carlo path tracing"):
//   camera ray through (x + u0, y + u1), u = Philox(pixel, sample, frame, 0);
//   segment b = 1..max_depth: closest hit (watertight test, ties -> lower
//   triangle id); a miss adds beta * env; a light triangle's front face adds
//   beta * Le, MIS-weighted (power heuristic) against light sampling for b > 1;
//   the last segment ends there; otherwise next-event estimation (word 3 =
//   4b + 1: light by power, uniform point, shadow ray to dist (1 - 1e-4)) and a
//   BSDF sample (word 3 = 4b + 2: cosine-weighted Lambert, or GGX
//   visible-normal sampling with Schlick Fresnel and separable Smith masking).
#pragma once
#include <cfloat>
#include <climits>
#include "et_internal.cuh"

namespace pt {

constexpr int kStack = kMaxBvhDepth;
constexpr float kGamma3 = 3.0f * 5.9604645e-08f / (1.0f - 3.0f * 5.9604645e-08f);
constexpr float kPi = 3.14159265358979323846f;

struct Ray {
  f3 o, d, inv;
  int kx, ky, kz;
  float Sx, Sy, Sz;
};

__device__ __forceinline__ void ray_setup(Ray& r, f3 o, f3 d) {
  r.o = o; r.d = d;
  r.inv = mk(1.0f / d.x, 1.0f / d.y, 1.0f / d.z);
  int kz = 0;
  if (fabsf(d.y) > fabsf(d.x)) kz = 1;
  if (fabsf(d.z) > fabsf(comp(d, kz))) kz = 2;
  int kx = kz == 2 ? 0 : kz + 1, ky = kx == 2 ? 0 : kx + 1;
  if (comp(d, kz) < 0.0f) { int t = kx; kx = ky; ky = t; }
  r.kx = kx; r.ky = ky; r.kz = kz;
  float dz = comp(d, kz);
  r.Sx = comp(d, kx) / dz; r.Sy = comp(d, ky) / dz; r.Sz = 1.0f / dz;
}

// Watertight ray/triangle test (Woop, Benthin, Wald, JCGT 2013).  The edge
// functions use non-contracted products so that the two triangles sharing an
// edge evaluate it to exact negatives; a zero edge value is re-evaluated in FP64.
__device__ __forceinline__ float tri_hit(const Ray& r, float4 a, float4 b, float4 c, float tmax) {
  const f3 A = mk(a.x - r.o.x, a.y - r.o.y, a.z - r.o.z);
  const f3 B = mk(b.x - r.o.x, b.y - r.o.y, b.z - r.o.z);
  const f3 C = mk(c.x - r.o.x, c.y - r.o.y, c.z - r.o.z);
  const float Az = comp(A, r.kz), Bz = comp(B, r.kz), Cz = comp(C, r.kz);
  const float Ax = __fsub_rn(comp(A, r.kx), __fmul_rn(r.Sx, Az));
  const float Ay = __fsub_rn(comp(A, r.ky), __fmul_rn(r.Sy, Az));
  const float Bx = __fsub_rn(comp(B, r.kx), __fmul_rn(r.Sx, Bz));
  const float By = __fsub_rn(comp(B, r.ky), __fmul_rn(r.Sy, Bz));
  const float Cx = __fsub_rn(comp(C, r.kx), __fmul_rn(r.Sx, Cz));
  const float Cy = __fsub_rn(comp(C, r.ky), __fmul_rn(r.Sy, Cz));
  float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
  float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
  float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
  if (U == 0.0f || V == 0.0f || W == 0.0f) {
    U = (float)((double)Cx * (double)By - (double)Cy * (double)Bx);
    V = (float)((double)Ax * (double)Cy - (double)Ay * (double)Cx);
    W = (float)((double)Bx * (double)Ay - (double)By * (double)Ax);
  }
  if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return -1.0f;
  const float det = U + V + W;
  if (det == 0.0f) return -1.0f;
  const float T = U * (r.Sz * Az) + V * (r.Sz * Bz) + W * (r.Sz * Cz);
  const float t = T / det;
  if (!(t > 0.0f) || !(t < tmax)) return -1.0f;
  return t;
}

// conservative slab test of one box against [0, tmax]; returns entry distance
__device__ __forceinline__ bool slab(const Ray& r, float lx, float ly, float lz, float hx,
                                     float hy, float hz, float tmax, float& tnear) {
  const float ax = (lx - r.o.x) * r.inv.x, bx = (hx - r.o.x) * r.inv.x;
  const float ay = (ly - r.o.y) * r.inv.y, by = (hy - r.o.y) * r.inv.y;
  const float az = (lz - r.o.z) * r.inv.z, bz = (hz - r.o.z) * r.inv.z;
  const float t0 = fmaxf(fmaxf(fminf(ax, bx), fminf(ay, by)), fmaxf(fminf(az, bz), 0.0f));
  const float far = fminf(fminf(fmaxf(ax, bx), fmaxf(ay, by)), fmaxf(az, bz)) * (1.0f + 2.0f * kGamma3);
  const float t1 = fminf(far, tmax);
  tnear = t0;
  return t0 <= t1;
}

struct Hit { float t; int slot; uint32_t prim; };

// Resumable traversal of the two-wide hierarchy: `step` processes one node or
// one leaf and returns false once the ray is finished.  Pending subtrees sit on
// a per-thread stack of (reference, entry distance) pairs, one 8-byte access
// per push or pop.
template <bool kAnyHit>
struct Traversal {
  int2 st[kStack];
  int sp;
  int ref;
  float tmax;
  Hit h;

  __device__ __forceinline__ void start(const et_scene_dev& S, float tmax_) {
    sp = 0; ref = S.root_ref; tmax = tmax_;
    h.t = tmax_; h.slot = -1; h.prim = 0xFFFFFFFFu;
  }

  static constexpr int kDone = INT_MIN;   // no subtree left (leaf references are > INT_MIN)

  // Culling distance: a subtree is skipped only if it starts beyond the best hit
  // by more than the rounding of the slab entry distance, so that a triangle at
  // exactly the best distance with a lower index (the tie rule) is still tested.
  __device__ __forceinline__ float cull() const { return h.t * (1.0f + 2.0f * kGamma3); }

  // take the nearest pending subtree that can still hold a closer hit
  __device__ __forceinline__ void pop() {
    while (sp > 0) {
      --sp;
      const int2 e = st[sp];
      if (__int_as_float(e.y) <= cull()) { ref = e.x; return; }
    }
    ref = kDone;
  }

  __device__ __forceinline__ bool at_node() const { return ref >= 0; }
  __device__ __forceinline__ bool at_leaf() const { return ref < 0 && ref != kDone; }

  // one inner node: descend into the nearer hit child, push the farther
  __device__ __forceinline__ void visit_node(const et_scene_dev& S, const Ray& r) {
    const float4* np = reinterpret_cast<const float4*>(S.nodes + ref);
    const float4 a = __ldg(np), b = __ldg(np + 1), c = __ldg(np + 2);
    const int4 d = __ldg(reinterpret_cast<const int4*>(np + 3));
    float t0, t1;
    const bool h0 = slab(r, a.x, a.y, a.z, a.w, b.x, b.y, cull(), t0);
    const bool h1 = slab(r, b.z, b.w, c.x, c.y, c.z, c.w, cull(), t1);
    if (h0 && h1) {
      const bool first0 = t0 <= t1;
      st[sp] = make_int2(first0 ? d.y : d.x, __float_as_int(first0 ? t1 : t0));
      ++sp;
      ref = first0 ? d.x : d.y;
    } else if (h0) {
      ref = d.x;
    } else if (h1) {
      ref = d.y;
    } else {
      pop();
    }
  }

  // one leaf: test its triangles, then continue with the stack
  __device__ __forceinline__ void visit_leaf(const et_scene_dev& S, const Ray& r) {
    const int v = -ref - 1;
    const int first = v >> 3, cnt = v & 7;
    for (int i = 0; i < cnt; ++i) {
      const float4* tp = S.tris + 3 * (int64_t)(first + i);
      const float4 A = __ldg(tp), B = __ldg(tp + 1), C = __ldg(tp + 2);
      const float t = tri_hit(r, A, B, C, tmax);
      if (t > 0.0f) {
        const uint32_t prim = __float_as_uint(A.w);
        if (kAnyHit) { h.t = t; h.slot = first + i; h.prim = prim; ref = kDone; return; }
        if (t < h.t || (t == h.t && prim < h.prim)) { h.t = t; h.slot = first + i; h.prim = prim; }
      }
    }
    pop();
  }

  __device__ __forceinline__ bool step(const et_scene_dev& S, const Ray& r) {
    if (ref >= 0) {
      const float4* np = reinterpret_cast<const float4*>(S.nodes + ref);
      const float4 a = __ldg(np), b = __ldg(np + 1), c = __ldg(np + 2);
      const int4 d = __ldg(reinterpret_cast<const int4*>(np + 3));
      float t0, t1;
      const bool h0 = slab(r, a.x, a.y, a.z, a.w, b.x, b.y, cull(), t0);
      const bool h1 = slab(r, b.z, b.w, c.x, c.y, c.z, c.w, cull(), t1);
      if (h0 && h1) {
        const bool first0 = t0 <= t1;
        st[sp] = make_int2(first0 ? d.y : d.x, __float_as_int(first0 ? t1 : t0));
        ++sp;
        ref = first0 ? d.x : d.y;
        return true;
      }
      if (h0) { ref = d.x; return true; }
      if (h1) { ref = d.y; return true; }
    } else {
      const int v = -ref - 1;
      const int first = v >> 3, cnt = v & 7;
      for (int i = 0; i < cnt; ++i) {
        const float4* tp = S.tris + 3 * (int64_t)(first + i);
        const float4 A = __ldg(tp), B = __ldg(tp + 1), C = __ldg(tp + 2);
        const float t = tri_hit(r, A, B, C, tmax);
        if (t > 0.0f) {
          const uint32_t prim = __float_as_uint(A.w);
          if (kAnyHit) { h.t = t; h.slot = first + i; h.prim = prim; return false; }
          if (t < h.t || (t == h.t && prim < h.prim)) { h.t = t; h.slot = first + i; h.prim = prim; }
        }
      }
    }
    // pop the nearest pending subtree that can still hold a closer hit
    while (sp > 0) {
      --sp;
      const int2 e = st[sp];
      if (__int_as_float(e.y) <= cull()) { ref = e.x; return true; }
    }
    return false;
  }
};

template <bool kAnyHit>
__device__ __forceinline__ Hit traverse(const et_scene_dev& S, const Ray& r, float tmax) {
  Traversal<kAnyHit> tr;
  tr.start(S, tmax);
  while (tr.step(S, r)) {}
  return tr.h;
}

__device__ __forceinline__ void onb(f3 n, f3& t, f3& b) {
  const float sgn = n.z >= 0.0f ? 1.0f : -1.0f;
  const float a = -1.0f / (sgn + n.z);
  const float bb = n.x * n.y * a;
  t = mk(1.0f + sgn * n.x * n.x * a, sgn * bb, -sgn * n.x);
  b = mk(bb, sgn + n.y * n.y * a, -n.y);
}

__device__ __forceinline__ float ggx_D(f3 m, float a2) {
  const float c2 = m.z * m.z;
  const float den = c2 * (a2 - 1.0f) + 1.0f;
  return a2 / (kPi * den * den);
}
__device__ __forceinline__ float ggx_G1(f3 v, float a2) {
  return 2.0f * v.z / (v.z + sqrtf(a2 + (1.0f - a2) * v.z * v.z));
}

// f cos(theta_i) and pdf (solid angle) in the local frame
__device__ __forceinline__ f3 bsdf_eval(const DevMaterial& m, f3 wo, f3 wi, float& pdf) {
  const f3 alb = mk(m.albedo[0], m.albedo[1], m.albedo[2]);
  if (m.type == ET_LAMBERT) {
    pdf = wi.z * (1.0f / kPi);
    return alb * (wi.z * (1.0f / kPi));
  }
  const float a2 = m.roughness * m.roughness;
  const f3 h = normalize(wo + wi);
  const float D = ggx_D(h, a2), G1o = ggx_G1(wo, a2), G1i = ggx_G1(wi, a2);
  const float c = 1.0f - dot(wi, h);
  const float c5 = c * c * c * c * c;
  const float k = D * G1o * G1i / (4.0f * wo.z);
  pdf = G1o * D / (4.0f * wo.z);
  return mk((alb.x + (1.0f - alb.x) * c5) * k, (alb.y + (1.0f - alb.y) * c5) * k,
            (alb.z + (1.0f - alb.z) * c5) * k);
}

__device__ __forceinline__ bool bsdf_sample(const DevMaterial& m, f3 wo, float u0, float u1,
                                            f3& wi, f3& weight, float& pdf) {
  const f3 alb = mk(m.albedo[0], m.albedo[1], m.albedo[2]);
  float s, c;
  if (m.type == ET_LAMBERT) {
    const float r = sqrtf(u0);
    sincospif(2.0f * u1, &s, &c);
    wi = mk(r * c, r * s, sqrtf(fmaxf(0.0f, 1.0f - u0)));
    if (!(wi.z > 0.0f)) return false;
    weight = alb;
    pdf = wi.z * (1.0f / kPi);
    return true;
  }
  const float a = m.roughness, a2 = a * a;
  const f3 vh = normalize(mk(a * wo.x, a * wo.y, wo.z));
  const float lensq = vh.x * vh.x + vh.y * vh.y;
  f3 T1;
  if (lensq > 0.0f) { const float il = 1.0f / sqrtf(lensq); T1 = mk(-vh.y * il, vh.x * il, 0.0f); }
  else T1 = mk(1.0f, 0.0f, 0.0f);
  const f3 T2 = cross(vh, T1);
  const float r = sqrtf(u0);
  sincospif(2.0f * u1, &s, &c);
  const float t1 = r * c;
  float t2 = r * s;
  const float sb = 0.5f * (1.0f + vh.z);
  t2 = (1.0f - sb) * sqrtf(1.0f - t1 * t1) + sb * t2;
  const float tz = sqrtf(fmaxf(0.0f, 1.0f - t1 * t1 - t2 * t2));
  const f3 nh = T1 * t1 + T2 * t2 + vh * tz;
  const f3 mh = normalize(mk(a * nh.x, a * nh.y, fmaxf(0.0f, nh.z)));
  const float om = dot(wo, mh);
  wi = mh * (2.0f * om) - wo;
  if (!(wi.z > 0.0f)) return false;
  const float cc = 1.0f - dot(wi, mh);
  const float c5 = cc * cc * cc * cc * cc;
  const float G1i = ggx_G1(wi, a2);
  weight = mk((alb.x + (1.0f - alb.x) * c5) * G1i, (alb.y + (1.0f - alb.y) * c5) * G1i,
              (alb.z + (1.0f - alb.z) * c5) * G1i);
  pdf = ggx_G1(wo, a2) * ggx_D(mh, a2) / (4.0f * wo.z);
  return true;
}

struct Cam { f3 pos, c0, c1, c2; float th; };

__device__ __forceinline__ Cam load_cam(const et_camera& c) {
  Cam cam;
  cam.pos = mk(c.pos[0], c.pos[1], c.pos[2]);
  cam.c0 = mk(c.rot[0], c.rot[3], c.rot[6]);
  cam.c1 = mk(c.rot[1], c.rot[4], c.rot[7]);
  cam.c2 = mk(c.rot[2], c.rot[5], c.rot[8]);
  cam.th = tanf(0.5f * c.vfov_deg * (kPi / 180.0f));
  return cam;
}

__device__ __forceinline__ void camera_ray(const Cam& cam, int W, int H, int x, int y, uint32_t smp,
                                           uint32_t frame, uint32_t k0, uint32_t k1, f3& o, f3& d) {
  const uint32_t pix = (uint32_t)(y * W + x);
  const u4 u = philox10(pix, smp, frame, 0u, k0, k1);
  const float px = (2.0f * ((float)x + u24(u.x)) / (float)W - 1.0f) * cam.th * ((float)W / (float)H);
  const float py = (1.0f - 2.0f * ((float)y + u24(u.y)) / (float)H) * cam.th;
  d = normalize(cam.c0 * px + cam.c1 * py - cam.c2);
  o = cam.pos;
}

// Shading context at a surface vertex.
struct Vertex {
  f3 on, ng, tt, bt, wol;
  DevMaterial m;
};

// Segment b ended at hit h (or missed): adds the environment or the light's
// MIS-weighted emission to L.  Returns true when the path continues from a
// surface vertex (filled into v).
__device__ __forceinline__ bool arrive(const et_scene_dev& S, f3 o, f3 d, const Hit& h, int b,
                                       int max_depth, float prev_pdf, f3 beta, f3& L, Vertex& v) {
  if (h.slot < 0) { L = L + beta * S.env; return false; }
  const float4* tp = S.tris + 3 * (int64_t)h.slot;
  const float4 A = __ldg(tp), B = __ldg(tp + 1), C = __ldg(tp + 2);
  const uint32_t mat = __float_as_uint(B.w);
  if (mat & ET_LIGHT_BIT) {
    const DevLight& lt = S.lights[mat & ~ET_LIGHT_BIT];
    const f3 ln = mk(lt.n[0], lt.n[1], lt.n[2]);
    const float cosl = -dot(d, ln);
    if (cosl > 0.0f) {
      float w = 1.0f;
      if (b > 1) {
        const float pl = lt.prob * h.t * h.t / (cosl * lt.area);
        w = prev_pdf * prev_pdf / (prev_pdf * prev_pdf + pl * pl);
      }
      L = L + beta * mk(lt.L[0], lt.L[1], lt.L[2]) * w;
    }
    return false;
  }
  if (b == max_depth) return false;
  const f3 x3 = o + d * h.t;
  const f3 v0 = mk(A.x, A.y, A.z);
  f3 ng = normalize(cross(mk(B.x, B.y, B.z) - v0, mk(C.x, C.y, C.z) - v0));
  const f3 wo = -d;
  if (dot(ng, wo) < 0.0f) ng = -ng;
  const float eps = 1e-4f * (1.0f + fmaxf(fabsf(x3.x), fmaxf(fabsf(x3.y), fabsf(x3.z))));
  v.on = x3 + ng * eps;
  v.ng = ng;
  onb(ng, v.tt, v.bt);
  v.wol = mk(dot(wo, v.tt), dot(wo, v.bt), dot(wo, ng));
  v.m = S.mats[mat];
  return true;
}

// Next-event estimation at vertex v of segment b: picks a light and a point on
// it.  Returns true when a shadow ray (o = v.on, dir, tmax) must decide whether
// `contrib` is added; `light` is the chosen light.
__device__ __forceinline__ bool nee(const et_scene_dev& S, const Vertex& v, uint32_t pix,
                                    uint32_t smp, uint32_t frame, int b, uint32_t k0, uint32_t k1,
                                    f3 beta, f3& dir, float& tmax, f3& contrib, int& light) {
  const u4 u = philox10(pix, smp, frame, (uint32_t)(4 * b + 1), k0, k1);
  const float ul = u24(u.x);
  int j = 0;
  while (j < S.n_lights - 1 && !(ul < S.lights[j].cdf)) ++j;
  light = j;
  const DevLight& lt = S.lights[j];
  const float su = u24(u.y), sv = u24(u.z);
  const f3 p = mk(lt.p0[0] + su * lt.e1[0] + sv * lt.e2[0], lt.p0[1] + su * lt.e1[1] + sv * lt.e2[1],
                  lt.p0[2] + su * lt.e1[2] + sv * lt.e2[2]);
  const f3 vv = p - v.on;
  const float dist2 = dot(vv, vv), dist = sqrtf(dist2);
  const f3 wi = vv * (1.0f / dist);
  const float cosi = dot(wi, v.ng), cosl = -(wi.x * lt.n[0] + wi.y * lt.n[1] + wi.z * lt.n[2]);
  if (!(cosi > 0.0f && cosl > 0.0f)) return false;
  float pb;
  const f3 fc = bsdf_eval(v.m, v.wol, mk(dot(wi, v.tt), dot(wi, v.bt), cosi), pb);
  const float pl = lt.prob * dist2 / (cosl * lt.area);
  const float w = pl * pl / (pl * pl + pb * pb);
  contrib = beta * fc * mk(lt.L[0], lt.L[1], lt.L[2]) * (w / pl);
  dir = wi;
  tmax = dist * (1.0f - 1e-4f);
  return true;
}

// BSDF continuation from vertex v: new direction, beta *= f cos / pdf.
__device__ __forceinline__ bool continue_path(const Vertex& v, uint32_t pix, uint32_t smp, uint32_t frame,
                                              int b, uint32_t k0, uint32_t k1, f3& beta, f3& d,
                                              float& pdf) {
  const u4 u = philox10(pix, smp, frame, (uint32_t)(4 * b + 2), k0, k1);
  f3 wil, wgt;
  if (!bsdf_sample(v.m, v.wol, u24(u.x), u24(u.y), wil, wgt, pdf)) return false;
  beta = beta * wgt;
  d = v.tt * wil.x + v.bt * wil.y + v.ng * wil.z;
  return true;
}

// Eq. 1 log map of the pixel's mean radiance, luminance and log in FP32 (logf:
// at most 1 ulp from the correctly rounded logarithm); the oracle evaluates the
// log in FP64.
__device__ __forceinline__ float log_luminance(f3 m, int log_mode, float log_param) {
  const float Lum = 0.2126f * m.x + 0.7152f * m.y + 0.0722f * m.z;
  if (log_mode == ET_LOG_EPS) return logf(Lum + log_param);
  return Lum >= log_param ? logf(Lum) : (logf(log_param) / log_param) * Lum;
}

}  // namespace pt
