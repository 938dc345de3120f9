// Scene construction: geometry upload and an SAH BVH2.
//
// The paper renders with Falcor on hardware ray tracing (Sec. 3.2, Sec. 4.1);
// GB300 has no RT cores, so the library traverses its own two-wide BVH in
// software.  The hierarchy is built once per scene (all camera paths here move
// only the camera) with the surface-area heuristic, leaves of at most 4
// triangles, nodes storing both children's boxes so that one 64-byte fetch
// serves two box tests.  Builders: a full sweep over every split of the
// centroid order on the host (the default: on the 500k-triangle city block its
// hierarchy takes ~30 % fewer traversal cycles than the binned one, for ~0.5 s
// of build), 32-bin binning on the GPU, and the same binning on the host as the
// fallback for trees deeper than the traversal stack.
#include <atomic>
#include <vector>
#include <algorithm>
#include <cstring>
#include <cfloat>
#include <cmath>
#include "et_internal.cuh"
#include "scene_internal.h"
#include "bvh_build.h"

static thread_local cudaError_t g_last_cuda = cudaSuccess;
void et_set_last_cuda_error(cudaError_t e) { g_last_cuda = e; }

static std::atomic<uint64_t> g_launches{0};
void et_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
extern "C" uint64_t et_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

namespace {

constexpr int kBins = kSahBins;

struct Builder {
  const std::vector<Box>& tb;
  const std::vector<float>& cent;   // [n][3]
  std::vector<int> idx;
  std::vector<BuildNode> nodes;

  Builder(const std::vector<Box>& tb_, const std::vector<float>& c, int64_t n) : tb(tb_), cent(c) {
    idx.resize(n);
    for (int64_t i = 0; i < n; ++i) idx[i] = (int)i;
    nodes.reserve(2 * n + 1);
  }

  int max_depth = 0;

  void build_all(int64_t n) {
    struct Item { int node, first, count, depth; };
    std::vector<Item> stack;
    nodes.push_back(BuildNode());
    stack.push_back({0, 0, (int)n, 0});
    while (!stack.empty()) {
      Item it = stack.back(); stack.pop_back();
      max_depth = std::max(max_depth, it.depth);
      BuildNode nd;
      nd.box.reset();
      Box cb; cb.reset();
      for (int i = 0; i < it.count; ++i) {
        int t = idx[it.first + i];
        nd.box.grow(tb[t]);
        cb.grow(&cent[3 * (size_t)t]);
      }
      nd.left = nd.right = -1; nd.first = it.first; nd.count = it.count;
      int split = -1, axis = -1;
      double best = DBL_MAX;
      double sa = nd.box.area();
      if (it.count > 1) {
        for (int ax = 0; ax < 3; ++ax) {
          float ext = cb.hi[ax] - cb.lo[ax];
          if (!(ext > 0.0f)) continue;
          int cnt[kBins] = {0};
          Box bb[kBins];
          for (int b = 0; b < kBins; ++b) bb[b].reset();
          float scale = kBins / ext;
          for (int i = 0; i < it.count; ++i) {
            int t = idx[it.first + i];
            int b = std::min(kBins - 1, (int)((cent[3 * (size_t)t + ax] - cb.lo[ax]) * scale));
            cnt[b]++; bb[b].grow(tb[t]);
          }
          double rarea[kBins]; int rcnt[kBins];
          Box r; r.reset(); int rc = 0;
          for (int b = kBins - 1; b > 0; --b) { r.grow(bb[b]); rc += cnt[b]; rarea[b] = r.area(); rcnt[b] = rc; }
          Box l; l.reset(); int lc = 0;
          for (int b = 1; b < kBins; ++b) {
            l.grow(bb[b - 1]); lc += cnt[b - 1];
            if (lc == 0 || rcnt[b] == 0) continue;
            double c = 1.0 + (l.area() * lc + rarea[b] * rcnt[b]) / (sa > 0 ? sa : 1.0);
            if (c < best) { best = c; axis = ax; split = b; }
          }
        }
      }
      bool leaf = it.count == 1 || (it.count <= kLeafMax && (axis < 0 || best >= it.count));
      if (leaf) { nodes[it.node] = nd; continue; }
      int mid;
      if (axis >= 0) {
        float ext = cb.hi[axis] - cb.lo[axis], scale = kBins / ext, lo = cb.lo[axis];
        int* beg = idx.data() + it.first;
        int* p = std::partition(beg, beg + it.count, [&](int t) {
          int b = std::min(kBins - 1, (int)((cent[3 * (size_t)t + axis] - lo) * scale));
          return b < split;
        });
        mid = (int)(p - beg);
      } else {
        // all centroids coincide: split the index range in half
        mid = it.count / 2;
      }
      if (mid <= 0 || mid >= it.count) mid = it.count / 2;
      int L = (int)nodes.size(); nodes.push_back(BuildNode());
      int R = (int)nodes.size(); nodes.push_back(BuildNode());
      nd.left = L; nd.right = R; nd.count = 0;
      nodes[it.node] = nd;
      stack.push_back({R, it.first + mid, it.count - mid, it.depth + 1});
      stack.push_back({L, it.first, mid, it.depth + 1});
    }
  }
};

// Full-sweep SAH: at every node all n - 1 splits of the centroid order along
// each axis are evaluated (no binning).  The triangle indices are kept sorted
// by centroid along all three axes at once; a split stably partitions the two
// other orders by side, so each level costs O(n).
struct SweepBuilder {
  const std::vector<Box>& tb;
  const std::vector<float>& cent;
  std::vector<int> ord[3];
  std::vector<BuildNode> nodes;
  std::vector<int> idx;          // final permutation (leaf order)
  int max_depth = 0;

  SweepBuilder(const std::vector<Box>& tb_, const std::vector<float>& c, int64_t n) : tb(tb_), cent(c) {
    for (int a = 0; a < 3; ++a) {
      ord[a].resize(n);
      for (int64_t i = 0; i < n; ++i) ord[a][i] = (int)i;
      std::sort(ord[a].begin(), ord[a].end(), [&](int x, int y) {
        const float cx = cent[3 * (size_t)x + a], cy = cent[3 * (size_t)y + a];
        return cx < cy || (cx == cy && x < y);
      });
    }
    nodes.reserve(2 * n + 1);
  }

  void build_all(int64_t n) {
    struct Item { int node, first, count, depth; };
    std::vector<Item> stack;
    std::vector<double> rarea((size_t)n);
    std::vector<uint8_t> left((size_t)n, 0);
    std::vector<int> tmp((size_t)n);
    nodes.push_back(BuildNode());
    stack.push_back({0, 0, (int)n, 0});
    while (!stack.empty()) {
      Item it = stack.back(); stack.pop_back();
      max_depth = std::max(max_depth, it.depth);
      BuildNode nd;
      nd.box.reset();
      for (int i = 0; i < it.count; ++i) nd.box.grow(tb[ord[0][it.first + i]]);
      nd.left = nd.right = -1; nd.first = it.first; nd.count = it.count;
      const double sa = nd.box.area();
      double best = DBL_MAX;
      int axis = -1, split = -1;
      if (it.count > 1) {
        for (int a = 0; a < 3; ++a) {
          const int* o = ord[a].data() + it.first;
          Box r; r.reset();
          for (int i = it.count - 1; i > 0; --i) { r.grow(tb[o[i]]); rarea[i] = r.area(); }
          Box l; l.reset();
          for (int i = 1; i < it.count; ++i) {
            l.grow(tb[o[i - 1]]);
            const double c = 1.0 + (l.area() * i + rarea[i] * (it.count - i)) / (sa > 0 ? sa : 1.0);
            if (c < best) { best = c; axis = a; split = i; }
          }
        }
      }
      const bool leaf = it.count == 1 || (it.count <= kLeafMax && best >= it.count);
      if (leaf) {
        nodes[it.node] = nd;
        continue;
      }
      // side of every triangle, then stable partition of the other two orders
      for (int i = 0; i < it.count; ++i) left[ord[axis][it.first + i]] = i < split ? 1 : 0;
      for (int a = 0; a < 3; ++a) {
        if (a == axis) continue;
        int* o = ord[a].data() + it.first;
        int nl = 0, nr = split;
        for (int i = 0; i < it.count; ++i) {
          const int t = o[i];
          if (left[t]) tmp[nl++] = t; else tmp[nr++] = t;
        }
        std::memcpy(o, tmp.data(), sizeof(int) * it.count);
      }
      int L = (int)nodes.size(); nodes.push_back(BuildNode());
      int R = (int)nodes.size(); nodes.push_back(BuildNode());
      nd.left = L; nd.right = R; nd.count = 0;
      nodes[it.node] = nd;
      stack.push_back({R, it.first + split, it.count - split, it.depth + 1});
      stack.push_back({L, it.first, split, it.depth + 1});
    }
    idx = ord[0];
  }
};

int ref_of(const std::vector<BuildNode>& bn, const std::vector<int>& inner_index, int i) {
  const BuildNode& n = bn[i];
  if (n.count > 0) return -(((n.first) << 3) | n.count) - 1;
  return inner_index[i];
}

}  // namespace

extern "C" int et_build_scene(const float* tris, const uint32_t* tri_mat, int64_t n_tris,
                              const et_material* mats, int32_t n_mats,
                              const et_quad_light* lights, int32_t n_lights, float env,
                              et_scene** out, void* stream) {
  return et_build_scene_with(tris, tri_mat, n_tris, mats, n_mats, lights, n_lights, env,
                             ET_BVH_DEFAULT, out, stream);
}

extern "C" int et_build_scene_with(const float* tris, const uint32_t* tri_mat, int64_t n_tris,
                                   const et_material* mats, int32_t n_mats,
                                   const et_quad_light* lights, int32_t n_lights, float env,
                                   int32_t builder_req, et_scene** out, void* stream_) {
  if (!out || n_tris < 0 || n_mats < 0 || n_lights < 0) return ET_ERR_ARG;
  if (builder_req != ET_BVH_GPU && builder_req != ET_BVH_HOST && builder_req != ET_BVH_SWEEP &&
      builder_req != ET_BVH_GPU_SWEEP)
    return ET_ERR_ARG;
  if (n_tris > 0 && (!tris || !tri_mat)) return ET_ERR_ARG;
  if (n_mats > 0 && !mats) return ET_ERR_ARG;
  if (n_lights > 0 && !lights) return ET_ERR_ARG;
  for (int64_t i = 0; i < n_tris; ++i)
    if (tri_mat[i] >= (uint32_t)n_mats) return ET_ERR_ARG;
  const int64_t n = n_tris + 2 * (int64_t)n_lights;
  if (n >= (1LL << 27)) return ET_ERR_ARG;
  cudaStream_t stream = (cudaStream_t)stream_;
  *out = nullptr;

  // geometry in input order (user triangles, then two per light)
  std::vector<float> v((size_t)n * 9);
  std::vector<uint32_t> m((size_t)n);
  if (n_tris > 0) std::memcpy(v.data(), tris, sizeof(float) * 9 * (size_t)n_tris);
  for (int64_t i = 0; i < n_tris; ++i) m[i] = tri_mat[i];
  std::vector<DevLight> dl((size_t)std::max(n_lights, 1));
  double total = 0.0;
  for (int j = 0; j < n_lights; ++j) {
    const et_quad_light& q = lights[j];
    float a[3], b[3], c[3], d[3];
    for (int k = 0; k < 3; ++k) {
      a[k] = q.p0[k];
      b[k] = q.p0[k] + q.e1[k];
      c[k] = q.p0[k] + q.e1[k] + q.e2[k];
      d[k] = q.p0[k] + q.e2[k];
    }
    float* t0 = &v[(size_t)(n_tris + 2 * j) * 9];
    float* t1 = t0 + 9;
    for (int k = 0; k < 3; ++k) { t0[k] = a[k]; t0[3 + k] = b[k]; t0[6 + k] = c[k]; t1[k] = a[k]; t1[3 + k] = c[k]; t1[6 + k] = d[k]; }
    m[n_tris + 2 * j] = m[n_tris + 2 * j + 1] = ET_LIGHT_BIT | (uint32_t)j;
    DevLight& L = dl[j];
    double nx = (double)q.e1[1] * q.e2[2] - (double)q.e1[2] * q.e2[1];
    double ny = (double)q.e1[2] * q.e2[0] - (double)q.e1[0] * q.e2[2];
    double nz = (double)q.e1[0] * q.e2[1] - (double)q.e1[1] * q.e2[0];
    double area = std::sqrt(nx * nx + ny * ny + nz * nz);
    for (int k = 0; k < 3; ++k) { L.p0[k] = q.p0[k]; L.e1[k] = q.e1[k]; L.e2[k] = q.e2[k]; L.L[k] = q.radiance[k]; }
    L.n[0] = (float)(nx / area); L.n[1] = (float)(ny / area); L.n[2] = (float)(nz / area);
    L.area = (float)area;
    double lum = 0.2126 * q.radiance[0] + 0.7152 * q.radiance[1] + 0.0722 * q.radiance[2];
    L.prob = (float)(lum * area);
    total += lum * area;
  }
  double acc = 0.0;
  for (int j = 0; j < n_lights; ++j) {
    double p = (double)dl[j].prob / total;
    acc += p;
    dl[j].prob = (float)p;
    dl[j].cdf = (j == n_lights - 1) ? 1.0f : (float)acc;
  }

  // BVH
  std::vector<Box> tb((size_t)std::max<int64_t>(n, 1));
  std::vector<float> cent((size_t)std::max<int64_t>(n, 1) * 3);
  for (int64_t i = 0; i < n; ++i) {
    tb[i].reset();
    for (int j = 0; j < 3; ++j) tb[i].grow(&v[(size_t)i * 9 + 3 * j]);
    for (int k = 0; k < 3; ++k) cent[3 * i + k] = (v[i * 9 + k] + v[i * 9 + 3 + k] + v[i * 9 + 6 + k]) * (1.0f / 3.0f);
  }
  std::vector<BvhNode> hn;
  std::vector<float4> ht((size_t)std::max<int64_t>(n, 1) * 3);
  std::vector<int32_t> slot_tri((size_t)std::max<int64_t>(n, 1), 0);   // leaf slot -> input triangle
  std::vector<int> refit_order, refit_levels{0};                        // inner nodes, deepest level first
  int root_ref = -1;   // an empty leaf: first 0, count 0
  float box_lo[3] = {0, 0, 0}, box_hi[3] = {0, 0, 0};
  double sah = 0.0;
  int64_t n_nodes = 0;
  int builder = builder_req;
  if (n > 0) {
    // the traversal kernels keep at most one pending subtree per level on a
    // 64-entry stack: a requested build whose tree is deeper (or a GPU build
    // that fails) falls back to the host binned build; deeper hierarchies are
    // refused rather than overflowed
    std::vector<BuildNode> bn_store;
    std::vector<int> perm;
    int depth = 0;
    int grc = ET_ERR_UNIMPLEMENTED;
    if (builder == ET_BVH_SWEEP) {
      SweepBuilder B(tb, cent, n);
      B.build_all(n);
      bn_store.swap(B.nodes);
      perm.swap(B.idx);
      depth = B.max_depth;
      grc = ET_OK;
    } else if (builder == ET_BVH_GPU) {
      grc = gpu_binned_sah(v.data(), n, stream, bn_store, perm, depth);
    } else if (builder == ET_BVH_GPU_SWEEP) {
      grc = gpu_sweep_sah(v.data(), n, stream, bn_store, perm, depth);
    }
    if (grc != ET_OK || depth > kMaxBvhDepth) {
      if (grc == ET_ERR_CUDA || grc == ET_ERR_OOM) cudaGetLastError();
      builder = ET_BVH_HOST;
      Builder B(tb, cent, n);
      B.build_all(n);
      bn_store.swap(B.nodes);
      perm.swap(B.idx);
      depth = B.max_depth;
    }
    if (depth > kMaxBvhDepth) return ET_ERR_UNIMPLEMENTED;
    const auto& bn = bn_store;
    std::vector<int> inner_index(bn.size(), -1);
    int ni = 0;
    for (size_t i = 0; i < bn.size(); ++i) if (bn[i].count == 0) inner_index[i] = ni++;
    hn.resize((size_t)std::max(ni, 1));
    double root_area = bn[0].box.area();
    for (size_t i = 0; i < bn.size(); ++i) {
      double a = root_area > 0 ? bn[i].box.area() / root_area : 0.0;
      sah += bn[i].count > 0 ? a * bn[i].count : a;
      if (bn[i].count > 0) continue;
      const Box& l = bn[bn[i].left].box;
      const Box& r = bn[bn[i].right].box;
      BvhNode& o = hn[inner_index[i]];
      o.a = make_float4(l.lo[0], l.lo[1], l.lo[2], l.hi[0]);
      o.b = make_float4(l.hi[1], l.hi[2], r.lo[0], r.lo[1]);
      o.c = make_float4(r.lo[2], r.hi[0], r.hi[1], r.hi[2]);
      o.d = make_int4(ref_of(bn, inner_index, bn[i].left), ref_of(bn, inner_index, bn[i].right), 0, 0);
    }
    n_nodes = (int64_t)bn.size();
    root_ref = ref_of(bn, inner_index, 0);
    for (int k = 0; k < 3; ++k) { box_lo[k] = bn[0].box.lo[k]; box_hi[k] = bn[0].box.hi[k]; }
    {
      // refit schedule: inner nodes by depth, deepest first
      std::vector<std::vector<int>> by_depth;
      std::vector<std::pair<int, int>> stack{{0, 0}};
      while (!stack.empty()) {
        const auto [i, dep] = stack.back();
        stack.pop_back();
        if (bn[i].count > 0) continue;
        if ((int)by_depth.size() <= dep) by_depth.resize(dep + 1);
        by_depth[dep].push_back(inner_index[i]);
        stack.push_back({bn[i].left, dep + 1});
        stack.push_back({bn[i].right, dep + 1});
      }
      for (int dep = (int)by_depth.size() - 1; dep >= 0; --dep) {
        refit_order.insert(refit_order.end(), by_depth[dep].begin(), by_depth[dep].end());
        refit_levels.push_back((int)refit_order.size());
      }
    }
    for (int64_t s = 0; s < n; ++s) {
      int t = perm[s];
      slot_tri[s] = t;
      const float* p = &v[(size_t)t * 9];
      uint32_t prim = (uint32_t)t, mat = m[t];
      float pf, mf;
      std::memcpy(&pf, &prim, 4); std::memcpy(&mf, &mat, 4);
      ht[3 * s + 0] = make_float4(p[0], p[1], p[2], pf);
      ht[3 * s + 1] = make_float4(p[3], p[4], p[5], mf);
      ht[3 * s + 2] = make_float4(p[6], p[7], p[8], 0.0f);
    }
  } else {
    hn.resize(1);
    std::memset(hn.data(), 0, sizeof(BvhNode));
  }
  std::vector<DevMaterial> dm((size_t)std::max(n_mats, 1));
  std::memset(dm.data(), 0, sizeof(DevMaterial) * dm.size());
  for (int i = 0; i < n_mats; ++i) {
    for (int k = 0; k < 3; ++k) dm[i].albedo[k] = mats[i].albedo[k];
    dm[i].roughness = mats[i].roughness;
    dm[i].type = mats[i].type;
  }

  et_scene* s = new et_scene();
  s->n_tris = n; s->n_nodes = n_nodes; s->sah = sah; s->builder = builder;
  s->n_user = n_tris;
  s->refit_levels = refit_levels;
  for (int k = 0; k < 3; ++k) { s->box_lo[k] = box_lo[k]; s->box_hi[k] = box_hi[k]; }
  auto fail = [&](int code) { et_scene_free(s); return code; };
  cudaError_t e;
#define ET_SCENE_ALLOC(ptr, bytes)                                   \
  e = cudaMalloc((void**)&(ptr), (bytes));                           \
  if (e != cudaSuccess) { et_set_last_cuda_error(e); return fail(e == cudaErrorMemoryAllocation ? ET_ERR_OOM : ET_ERR_CUDA); }
  ET_SCENE_ALLOC(s->d_tris, sizeof(float4) * ht.size());
  ET_SCENE_ALLOC(s->d_nodes, sizeof(BvhNode) * hn.size());
  ET_SCENE_ALLOC(s->d_mats, sizeof(DevMaterial) * dm.size());
  ET_SCENE_ALLOC(s->d_lights, sizeof(DevLight) * dl.size());
  s->cam_cap = 1024;
  ET_SCENE_ALLOC(s->d_cams, sizeof(et_camera) * s->cam_cap);
  ET_SCENE_ALLOC(s->d_perm, sizeof(int32_t) * slot_tri.size());
  ET_SCENE_ALLOC(s->d_refit, sizeof(int32_t) * std::max<size_t>(refit_order.size(), 1));
#undef ET_SCENE_ALLOC
#define ET_SCENE_COPY(dst, src, bytes)                                           \
  e = cudaMemcpyAsync((dst), (src), (bytes), cudaMemcpyHostToDevice, stream);    \
  if (e != cudaSuccess) { et_set_last_cuda_error(e); return fail(ET_ERR_CUDA); }
  ET_SCENE_COPY(s->d_tris, ht.data(), sizeof(float4) * ht.size());
  ET_SCENE_COPY(s->d_nodes, hn.data(), sizeof(BvhNode) * hn.size());
  ET_SCENE_COPY(s->d_mats, dm.data(), sizeof(DevMaterial) * dm.size());
  ET_SCENE_COPY(s->d_lights, dl.data(), sizeof(DevLight) * dl.size());
  ET_SCENE_COPY(s->d_perm, slot_tri.data(), sizeof(int32_t) * slot_tri.size());
  if (!refit_order.empty())
    ET_SCENE_COPY(s->d_refit, refit_order.data(), sizeof(int32_t) * refit_order.size());
#undef ET_SCENE_COPY
  e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) { et_set_last_cuda_error(e); return fail(ET_ERR_CUDA); }
  s->dev.tris = s->d_tris;
  s->dev.nodes = s->d_nodes;
  s->dev.mats = s->d_mats;
  s->dev.lights = s->d_lights;
  s->dev.n_lights = n_lights;
  s->dev.root_ref = root_ref;
  s->dev.env = env;
  s->dev.n_tris = n;
  *out = s;
  return ET_OK;
}

extern "C" void et_scene_free(et_scene* s) {
  if (!s) return;
  cudaFree(s->d_tris); cudaFree(s->d_nodes); cudaFree(s->d_mats); cudaFree(s->d_lights);
  cudaFree(s->d_cams);
  cudaFree(s->wf_mem);
  cudaFree(s->wf_sort_mem);
  cudaFree(s->d_perm);
  cudaFree(s->d_refit);
  cudaFree(s->d_upd);
  for (cudaEvent_t e : s->prof.pool) cudaEventDestroy(e);
  if (s->prof.h_len) cudaFreeHost(s->prof.h_len);
  delete s;
}

extern "C" int et_scene_builder(const et_scene* s) { return s ? s->builder : -1; }

extern "C" int et_scene_info(const et_scene* s, int64_t* n_tris, int64_t* n_nodes, double* sah) {
  if (!s) return ET_ERR_ARG;
  if (n_tris) *n_tris = s->n_tris;
  if (n_nodes) *n_nodes = s->n_nodes;
  if (sah) *sah = s->sah;
  return ET_OK;
}

extern "C" const char* et_status_str(int st) {
  switch (st) {
    case ET_OK: return "ok";
    case ET_ERR_ARG: return "invalid argument";
    case ET_ERR_CUDA: return g_last_cuda != cudaSuccess ? cudaGetErrorString(g_last_cuda) : "CUDA error";
    case ET_ERR_OOM: return "out of device memory";
    case ET_ERR_CAPACITY: return "output buffer too small";
    case ET_ERR_TIMEOUT: return "device-side wait timed out";
    case ET_ERR_UNIMPLEMENTED: return "configuration not supported";
    default: return "unknown status";
  }
}
