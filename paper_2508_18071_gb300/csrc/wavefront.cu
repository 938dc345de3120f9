// Wavefront schedule of the path tracer (same per-path arithmetic as the
// one-kernel schedule, pt_common.cuh).
//
// The paths of a batch (whole frames, or sample slices of one frame when the
// sample count is large) advance one segment at a time:
//   raygen          camera rays for every path -> ray queue
//   trace_closest   persistent warps pull rays from the queue; a lane whose ray
//                   is finished gets a new ray as soon as enough lanes are idle,
//                   so warps stay full despite very different traversal lengths
//   shade           emission / environment, next-event estimation (appends a
//                   shadow ray with its would-be contribution), BSDF sampling
//                   (appends the continuation ray to the next queue)
//   trace_shadow    persistent any-hit warps; visible -> the path's radiance
//                   receives the contribution
// and finally `accumulate` sums each pixel's path radiances in sample order
// (the same order as the one-kernel schedule) and writes RGB and Eq. 1 log
// luminance.  Queues are compacted with one atomic per warp.
#include <algorithm>
#include <cub/device/device_radix_sort.cuh>
#include "et_internal.cuh"
#include "pt_common.cuh"
#include "scene_internal.h"
#include "render_internal.h"

namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int kLeafBatch = 24;       // lanes waiting at leaves that end a node phase
constexpr int kNodeSteps = 3;        // node visits per lane between two warp votes
constexpr int64_t kPathCap = 8 << 20;
// et_render_profile kinds (the order of the ms / launches / items arrays)
enum { kProfRaygen = 0, kProfTrace = 1, kProfShade = 2, kProfShadow = 3, kProfAccumulate = 4 };
#define ET_TRY(expr)                 \
  do {                               \
    const int rc_ = (expr);          \
    if (rc_ != ET_OK) return rc_;    \
  } while (0)

enum { C_NRAY0 = 0, C_NRAY1 = 1, C_NSH = 2, C_FETCH = 3, C_FETCH_SH = 4, C_N = 8 };

struct Batch {
  int f0, nf;          // frames of the call in this batch (relative to the call)
  int s0, ns;          // samples of each frame in this batch
  int64_t npix;        // W * H
  int64_t paths;       // nf * ns * npix
  int W;               // image width (the slot -> pixel map)
  int tiled;           // slots visit 8 x 4 pixel tiles (needs W % 8 == 0 and rows % 4 == 0)
};

// pixel of slot i of a frame's sample plane: raster order, or 8 x 4 tiles in
// raster order of tiles (a warp's 32 primary rays then cover a compact tile).
// Index arithmetic is 32-bit: the host keeps a batch below 2^31 paths.
__host__ __device__ __forceinline__ uint32_t slot_pixel(const Batch& bt, uint32_t i) {
  if (!bt.tiled) return i;
  const uint32_t tw = (uint32_t)bt.W >> 3, tile = i >> 5;
  const uint32_t ty = tile / tw, tx = tile - ty * tw;
  return (ty * 4 + ((i >> 3) & 3)) * (uint32_t)bt.W + tx * 8 + (i & 7);
}

// Extension rays reordered between bounces (ET_RENDER_WAVEFRONT_SORTED): the
// shading kernel writes a 24-bit key for every continuation ray it appends,
// the queue is sorted by key (stable radix sort) and the next closest-hit
// trace takes its rays through the sorted permutation.  Key: the direction's
// cell on an 8 x 8 octahedral map above (or below) a Morton code of the
// origin's cell on a 64^3 grid over the scene's box.  The order of a queue
// changes no path's arithmetic.
#ifndef ET_SORT_DIR_MAJOR
#define ET_SORT_DIR_MAJOR 1
#endif
constexpr int kSortBits = 24;

struct SortBox { float lo[3], scale[3]; };

__host__ __device__ __forceinline__ uint32_t spread3(uint32_t v) {   // 6 bits -> every third bit
  v &= 0x3Fu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

__device__ __forceinline__ uint32_t ray_key(const SortBox& B, f3 o, f3 d) {
  const float sx = fabsf(d.x) + fabsf(d.y) + fabsf(d.z);
  float u = d.x / sx, v = d.y / sx;
  if (d.z < 0.0f) {
    const float uu = (1.0f - fabsf(v)) * (u < 0.0f ? -1.0f : 1.0f);
    v = (1.0f - fabsf(u)) * (v < 0.0f ? -1.0f : 1.0f);
    u = uu;
  }
  const uint32_t du = (uint32_t)min(7, max(0, (int)((u + 1.0f) * 4.0f)));
  const uint32_t dv = (uint32_t)min(7, max(0, (int)((v + 1.0f) * 4.0f)));
  const uint32_t dir = (dv << 3) | du;
  const float c[3] = {o.x, o.y, o.z};
  uint32_t m = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int q = (int)((c[k] - B.lo[k]) * B.scale[k]);
    m |= spread3((uint32_t)min(63, max(0, q))) << k;
  }
  return ET_SORT_DIR_MAJOR ? (dir << 18) | m : (m << 6) | dir;
}

struct Args {
  et_scene_dev S;
  const et_camera* cams;
  int W, H, spp, max_depth;
  int y0;              // first image row of the rendered band (pixel ids are band-relative)
  uint32_t first_frame, k0, k1;
  Batch bt;
  float4* beta_pdf;
  float4* L;
  float4* qo[2];
  float4* qd[2];
  int2* hit;
  float4* sho;
  float4* shd;
  float4* shc;
  uint32_t* ctr;
  int32_t* records;
  uint32_t* skey;       // sorted mode: keys and queue indices the shading kernel appends
  uint32_t* sval;
  const uint32_t* perm; // sorted mode: queue index of the i-th ray the trace takes
  SortBox box;
};

// path q of the batch -> (frame of the call, sample, pixel)
__device__ __forceinline__ void path_ids(const Batch& bt, uint32_t q, int& f, int& s, int64_t& pix) {
  const uint32_t npix = (uint32_t)bt.npix, ns = (uint32_t)bt.ns;
  const uint32_t plane = q / npix;
  pix = slot_pixel(bt, q - plane * npix);
  const uint32_t fo = plane / ns;
  s = bt.s0 + (int)(plane - fo * ns);
  f = bt.f0 + (int)fo;
}

__device__ __forceinline__ int32_t* rec_of(const Args& A, int f, int s, int64_t pix) {
  if (!A.records) return nullptr;
  return A.records + (((int64_t)f * A.bt.npix + pix) * A.spp + s) * A.max_depth * 2;
}

// one atomic per warp: returns this lane's slot (valid only where want is true)
__device__ __forceinline__ uint32_t warp_append(uint32_t* counter, bool want) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned m = __ballot_sync(FULL, want);
  if (!m) return 0;
  const int leader = __ffs(m) - 1;
  uint32_t base = 0;
  if ((int)lane == leader) base = atomicAdd(counter, (uint32_t)__popc(m));
  base = __shfl_sync(FULL, base, leader);
  return base + (uint32_t)__popc(m & ((1u << lane) - 1u));
}

__global__ void __launch_bounds__(256) wf_raygen(Args A) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q == 0) A.ctr[C_NRAY0] = (uint32_t)A.bt.paths;
  if (q >= A.bt.paths) return;
  int f, s;
  int64_t pix;
  path_ids(A.bt, (uint32_t)q, f, s, pix);
  const uint32_t py = (uint32_t)pix / (uint32_t)A.W;
  const int x = (int)((uint32_t)pix - py * (uint32_t)A.W), y = (int)py + A.y0;
  const pt::Cam cam = pt::load_cam(A.cams[f]);
  f3 o, d;
  pt::camera_ray(cam, A.W, A.H, x, y, (uint32_t)s, A.first_frame + (uint32_t)f, A.k0, A.k1, o, d);
  A.qo[0][q] = make_float4(o.x, o.y, o.z, __uint_as_float((uint32_t)q));
  A.qd[0][q] = make_float4(d.x, d.y, d.z, 0.0f);
  A.beta_pdf[q] = make_float4(1.0f, 1.0f, 1.0f, 0.0f);
  A.L[q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  if (int32_t* rec = rec_of(A, f, s, pix))
    for (int i = 0; i < 2 * A.max_depth; ++i) rec[i] = (i & 1) ? -1 : -2;
}

// Persistent traversal with dynamic ray fetch.  kShadow: any-hit shadow rays
// (queue sho/shd/shc), else closest-hit extension rays (queue qo/qd -> hit).
// resident blocks of 128 threads per SM the register allocation aims for
#ifndef ET_TRACE_MIN_BLOCKS
#define ET_TRACE_MIN_BLOCKS 12
#endif
template <bool kShadow>
__global__ void __launch_bounds__(128, ET_TRACE_MIN_BLOCKS) wf_trace(Args A, int cur, int b) {
  const uint32_t n = A.ctr[kShadow ? C_NSH : (C_NRAY0 + cur)];
  uint32_t* fetch = A.ctr + (kShadow ? C_FETCH_SH : C_FETCH);
  const unsigned lane = threadIdx.x & 31u;
  pt::Traversal<kShadow> tr;
  pt::Ray ray;
  int idx = -1;                       // -1: wants a ray, -2: queue exhausted
  while (true) {
    const unsigned want = __ballot_sync(FULL, idx == -1);
    if (want) {
      const int leader = __ffs(want) - 1;
      uint32_t base = 0;
      if ((int)lane == leader) base = atomicAdd(fetch, (uint32_t)__popc(want));
      base = __shfl_sync(FULL, base, leader);
      if (idx == -1) {
        const uint32_t my = base + (uint32_t)__popc(want & ((1u << lane) - 1u));
        if (my < n) {
          idx = (int)my;
          float4 o, d;
          if (kShadow) { o = A.sho[my]; d = A.shd[my]; }
          else {
            if (A.perm) idx = (int)A.perm[my];
            o = A.qo[cur][idx]; d = A.qd[cur][idx];
          }
          pt::ray_setup(ray, mk(o.x, o.y, o.z), mk(d.x, d.y, d.z));
          tr.start(A.S, kShadow ? d.w : FLT_MAX);
        } else {
          idx = -2;
        }
      }
    }
    if (__all_sync(FULL, idx == -2)) break;
    // node phase: lanes at inner nodes descend together; it ends when no lane
    // has node work left or when enough lanes are waiting at a leaf
    while (true) {
      const bool node = idx >= 0 && tr.at_node();
      const unsigned nodes = __ballot_sync(FULL, node);
      if (!nodes) break;
      const unsigned leaves = __ballot_sync(FULL, idx >= 0 && tr.at_leaf());
      if (__popc(leaves) >= kLeafBatch) break;
      // up to kNodeSteps steps per vote: a lane keeps descending while it is at
      // an inner node (its own sequence of visits is unchanged)
      if (node) {
#pragma unroll
        for (int r = 0; r < kNodeSteps; ++r)
          if (tr.at_node()) tr.visit_node(A.S, ray);
      }
    }
    // leaf phase: lanes at a leaf test its triangles together
    if (idx >= 0 && tr.at_leaf()) tr.visit_leaf(A.S, ray);
    {
      if (idx >= 0 && tr.ref == pt::Traversal<kShadow>::kDone) {
        if (kShadow) {
          const bool vis = tr.h.slot < 0;
          const float4 c = A.shc[idx];
          const uint32_t q = __float_as_uint(A.sho[idx].w);
          if (vis) {
            float4 l = A.L[q];
            l.x = l.x + c.x; l.y = l.y + c.y; l.z = l.z + c.z;
            A.L[q] = l;
          }
          if (A.records) {
            int f, s;
            int64_t pix;
            path_ids(A.bt, q, f, s, pix);
            rec_of(A, f, s, pix)[2 * (b - 1) + 1] = 2 * (int)__float_as_uint(c.w) + (vis ? 1 : 0);
          }
        } else {
          A.hit[idx] = make_int2(__float_as_int(tr.h.t), tr.h.slot);
        }
        idx = -1;
      }
    }
  }
}

__global__ void __launch_bounds__(256) wf_shade(Args A, int cur, int b) {
  const uint32_t n = A.ctr[C_NRAY0 + cur];
  const int nxt = cur ^ 1;
  // whole warps iterate together so that the appends can use warp ballots
  const uint32_t warp_id = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t wbase = warp_id * 32u; wbase < n; wbase += n_warps * 32u) {
    const uint32_t i = wbase + (threadIdx.x & 31u);
    const bool live = i < n;
    bool want_sh = false, want_ray = false;
    f3 sh_dir = mk(0, 0, 0), contrib = mk(0, 0, 0), d_next = mk(0, 0, 0);
    float sh_tmax = 0.0f, pdf = 0.0f;
    int light = 0;
    uint32_t q = 0;
    pt::Vertex v;
    f3 beta = mk(0, 0, 0);
    if (live) {
      const float4 o4 = A.qo[cur][i], d4 = A.qd[cur][i];
      q = __float_as_uint(o4.w);
      const int2 hh = A.hit[i];
      pt::Hit h;
      h.t = __int_as_float(hh.x);
      h.slot = hh.y;
      h.prim = h.slot >= 0 ? __float_as_uint(A.S.tris[3 * (int64_t)h.slot].w) : 0xFFFFFFFFu;
      int f, s;
      int64_t pix;
      path_ids(A.bt, q, f, s, pix);
      if (int32_t* rec = rec_of(A, f, s, pix)) rec[2 * (b - 1)] = h.slot < 0 ? -1 : (int32_t)h.prim;
      const float4 bp = A.beta_pdf[q];
      beta = mk(bp.x, bp.y, bp.z);
      const float4 l4 = A.L[q];
      f3 L = mk(l4.x, l4.y, l4.z);
      const f3 o = mk(o4.x, o4.y, o4.z), d = mk(d4.x, d4.y, d4.z);
      const bool cont = pt::arrive(A.S, o, d, h, b, A.max_depth, bp.w, beta, L, v);
      A.L[q] = make_float4(L.x, L.y, L.z, 0.0f);
      if (cont) {
        const uint32_t pixu = (uint32_t)(pix + (int64_t)A.y0 * A.W), frame = A.first_frame + (uint32_t)f;
        if (A.S.n_lights > 0)
          want_sh = pt::nee(A.S, v, pixu, (uint32_t)s, frame, b, A.k0, A.k1, beta, sh_dir, sh_tmax,
                            contrib, light);
        want_ray = pt::continue_path(v, pixu, (uint32_t)s, frame, b, A.k0, A.k1, beta, d_next, pdf);
        if (want_ray) A.beta_pdf[q] = make_float4(beta.x, beta.y, beta.z, pdf);
      }
    }
    const uint32_t js = warp_append(A.ctr + C_NSH, want_sh);
    if (want_sh) {
      A.sho[js] = make_float4(v.on.x, v.on.y, v.on.z, __uint_as_float(q));
      A.shd[js] = make_float4(sh_dir.x, sh_dir.y, sh_dir.z, sh_tmax);
      A.shc[js] = make_float4(contrib.x, contrib.y, contrib.z, __uint_as_float((uint32_t)light));
    }
    const uint32_t jr = warp_append(A.ctr + C_NRAY0 + nxt, want_ray);
    if (want_ray) {
      A.qo[nxt][jr] = make_float4(v.on.x, v.on.y, v.on.z, __uint_as_float(q));
      A.qd[nxt][jr] = make_float4(d_next.x, d_next.y, d_next.z, 0.0f);
      if (A.skey) {
        A.skey[jr] = ray_key(A.box, v.on, d_next);
        A.sval[jr] = jr;
      }
    }
  }
}

// Sum the batch's path radiances into the per-pixel accumulators in sample
// order; after a frame's last sample write its mean RGB and log luminance.
__global__ void __launch_bounds__(256)
wf_accumulate(Args A, float4* acc, bool first_slice, bool last_slice, float* rgb, float* logl,
              int log_mode, float log_param) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)A.bt.nf * A.bt.npix) return;
  const uint32_t npix = (uint32_t)A.bt.npix;
  const int fb = (int)((uint32_t)i / npix);
  const int64_t slot = (uint32_t)i - (uint32_t)fb * npix;
  f3 a = mk(0.0f, 0.0f, 0.0f);
  if (!first_slice) { const float4 t = acc[i]; a = mk(t.x, t.y, t.z); }
  for (int sb = 0; sb < A.bt.ns; ++sb) {
    const float4 l = A.L[((int64_t)fb * A.bt.ns + sb) * A.bt.npix + slot];
    a = a + mk(l.x, l.y, l.z);
  }
  if (!last_slice) { acc[i] = make_float4(a.x, a.y, a.z, 0.0f); return; }
  const f3 m = a * (1.0f / (float)A.spp);
  const int64_t o = (int64_t)(A.bt.f0 + fb) * A.bt.npix + slot_pixel(A.bt, (uint32_t)slot);
  if (rgb) { rgb[3 * o] = m.x; rgb[3 * o + 1] = m.y; rgb[3 * o + 2] = m.z; }
  if (logl) logl[o] = pt::log_luminance(m, log_mode, log_param);
}

int ensure_workspace(et_scene* s, int64_t paths, int64_t acc_pix) {
  if (s->wf_cap >= paths && s->wf_acc_cap >= acc_pix) return ET_OK;
  cudaFree(s->wf_mem);
  s->wf_mem = nullptr;
  s->wf_cap = s->wf_acc_cap = 0;
  const int64_t cap = std::max<int64_t>(paths, 1), acap = std::max<int64_t>(acc_pix, 1);
  const size_t bytes = (size_t)cap * (16 * 2 + 16 * 4 + 8 + 16 * 3) + (size_t)acap * 16 + 256;
  ET_CHECK_CUDA(cudaMalloc(&s->wf_mem, bytes));
  s->wf_cap = cap;
  s->wf_acc_cap = acap;
  return ET_OK;
}

// keys, key copies, indices and the permutation (4 x 4 B per path) plus the
// radix sort's scratch, grown on demand
int ensure_sort_workspace(et_scene* s, int64_t paths, uint32_t** key, uint32_t** key_alt, uint32_t** val,
                          uint32_t** perm, void** tmp, size_t* tmp_bytes) {
  if (s->wf_sort_cap < paths) {
    cudaFree(s->wf_sort_mem);
    s->wf_sort_mem = nullptr;
    s->wf_sort_cap = 0;
    size_t tb = 0;
    ET_CHECK_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tb, (const uint32_t*)nullptr, (uint32_t*)nullptr,
                                                  (const uint32_t*)nullptr, (uint32_t*)nullptr,
                                                  (int)paths, 0, kSortBits));
    tb = (tb + 255) & ~(size_t)255;
    ET_CHECK_CUDA(cudaMalloc(&s->wf_sort_mem, (size_t)paths * 16 + tb));
    s->wf_sort_cap = paths;
    s->wf_sort_tmp = tb;
  }
  char* p = static_cast<char*>(s->wf_sort_mem);
  const int64_t cap = s->wf_sort_cap;
  *tmp = p; p += s->wf_sort_tmp;
  *tmp_bytes = s->wf_sort_tmp;
  *key = reinterpret_cast<uint32_t*>(p); p += 4 * cap;
  *key_alt = reinterpret_cast<uint32_t*>(p); p += 4 * cap;
  *val = reinterpret_cast<uint32_t*>(p); p += 4 * cap;
  *perm = reinterpret_cast<uint32_t*>(p);
  return ET_OK;
}

}  // namespace

int et_render_wavefront(et_scene* s, int n_frames, int first_frame, int W, int H, int y0, int y1,
                        int spp, int max_depth, uint64_t seed, float* rgb, float* logl, int log_mode,
                        float log_param, int32_t* records, cudaStream_t stream) {
  const int64_t npix = (int64_t)W * (y1 - y0);
  if (npix >= ((int64_t)1 << 31)) return ET_ERR_UNIMPLEMENTED;   // 32-bit path indices
  const int64_t planes = std::max<int64_t>(1, kPathCap / npix);
  Batch proto{};
  proto.npix = npix;
  proto.W = W;
  proto.tiled = (s->render_mode == ET_RENDER_WAVEFRONT_TILES || s->render_mode == ET_RENDER_WAVEFRONT_SORTED) &&
                W % 8 == 0 && (y1 - y0) % 4 == 0;
  int frames_per_batch, samples_per_batch;
  if (spp <= planes) {
    samples_per_batch = spp;
    frames_per_batch = (int)std::min<int64_t>(n_frames, planes / spp);
  } else {
    samples_per_batch = (int)planes;
    frames_per_batch = 1;
  }
  const int64_t cap_paths = (int64_t)frames_per_batch * samples_per_batch * npix;
  int rc = ensure_workspace(s, cap_paths, (int64_t)frames_per_batch * npix);
  if (rc != ET_OK) return rc;
  char* p = static_cast<char*>(s->wf_mem);
  const int64_t cap = s->wf_cap;
  Args A{};
  A.S = s->dev;
  A.cams = s->d_cams;
  A.W = W; A.H = H; A.spp = spp; A.max_depth = max_depth; A.y0 = y0;
  A.first_frame = (uint32_t)first_frame;
  A.k0 = (uint32_t)seed; A.k1 = (uint32_t)(seed >> 32);
  A.records = records;
  A.beta_pdf = reinterpret_cast<float4*>(p); p += 16 * cap;
  A.L = reinterpret_cast<float4*>(p); p += 16 * cap;
  A.qo[0] = reinterpret_cast<float4*>(p); p += 16 * cap;
  A.qd[0] = reinterpret_cast<float4*>(p); p += 16 * cap;
  A.qo[1] = reinterpret_cast<float4*>(p); p += 16 * cap;
  A.qd[1] = reinterpret_cast<float4*>(p); p += 16 * cap;
  A.sho = reinterpret_cast<float4*>(p); p += 16 * cap;
  A.shd = reinterpret_cast<float4*>(p); p += 16 * cap;
  A.shc = reinterpret_cast<float4*>(p); p += 16 * cap;
  float4* acc = reinterpret_cast<float4*>(p); p += 16 * s->wf_acc_cap;
  A.hit = reinterpret_cast<int2*>(p); p += 8 * cap;
  A.ctr = reinterpret_cast<uint32_t*>(p);
  int dev = 0, nsm = 0, occ_c = 0, occ_s = 0;
  ET_CHECK_CUDA(cudaGetDevice(&dev));
  ET_CHECK_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  ET_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_c, wf_trace<false>, 128, 0));
  ET_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_s, wf_trace<true>, 128, 0));
  const int grid_c = nsm * std::max(occ_c, 1), grid_s = nsm * std::max(occ_s, 1);
  const bool sorted = s->render_mode == ET_RENDER_WAVEFRONT_SORTED && max_depth > 1;
  uint32_t *skey = nullptr, *skey_alt = nullptr, *sval = nullptr, *sperm = nullptr;
  void* stmp = nullptr;
  size_t stmp_bytes = 0;
  if (sorted) {
    ET_TRY(ensure_sort_workspace(s, cap, &skey, &skey_alt, &sval, &sperm, &stmp, &stmp_bytes));
    for (int k = 0; k < 3; ++k) {
      const float ext = s->box_hi[k] - s->box_lo[k];
      A.box.lo[k] = s->box_lo[k];
      A.box.scale[k] = ext > 0.0f ? 64.0f / ext : 0.0f;
    }
  }
  const int grid_shade = nsm * 8;
  for (int f0 = 0; f0 < n_frames; f0 += frames_per_batch) {
    const int nf = std::min(frames_per_batch, n_frames - f0);
    for (int s0 = 0; s0 < spp; s0 += samples_per_batch) {
      Batch bt = proto;
      bt.f0 = f0; bt.nf = nf; bt.s0 = s0; bt.ns = std::min(samples_per_batch, spp - s0);
      bt.paths = (int64_t)nf * bt.ns * npix;
      A.bt = bt;
      ET_CHECK_CUDA(cudaMemsetAsync(A.ctr, 0, sizeof(uint32_t) * C_N, stream));
      size_t pe = 0;   // profiling marks (et_render_profile; no-ops when off)
      ET_TRY(prof_begin(s, kProfRaygen, stream, &pe));
      wf_raygen<<<(unsigned)((bt.paths + 255) / 256), 256, 0, stream>>>(A);
      ET_CHECK_LAUNCH();
      ET_TRY(prof_end(s, kProfRaygen, pe, bt.paths, nullptr, stream));
      int cur = 0;
      for (int b = 1; b <= max_depth; ++b) {
        const int nxt = cur ^ 1;
        ET_CHECK_CUDA(cudaMemsetAsync(A.ctr + C_NRAY0 + nxt, 0, sizeof(uint32_t), stream));
        ET_CHECK_CUDA(cudaMemsetAsync(A.ctr + C_NSH, 0, sizeof(uint32_t) * 3, stream));
        const bool sort_next = sorted && b < max_depth;
        Args At = A, Ash = A;
        At.perm = sorted && b > 1 ? sperm : nullptr;
        if (sort_next) {
          Ash.skey = skey;
          Ash.sval = sval;
          ET_CHECK_CUDA(cudaMemsetAsync(skey, 0xFF, sizeof(uint32_t) * bt.paths, stream));
        }
        ET_TRY(prof_begin(s, kProfTrace, stream, &pe));
        wf_trace<false><<<grid_c, 128, 0, stream>>>(At, cur, b);
        ET_CHECK_LAUNCH();
        ET_TRY(prof_end(s, kProfTrace, pe, 0, A.ctr + C_NRAY0 + cur, stream));
        ET_TRY(prof_begin(s, kProfShade, stream, &pe));
        wf_shade<<<grid_shade, 256, 0, stream>>>(Ash, cur, b);
        ET_CHECK_LAUNCH();
        if (sort_next) {
          // the continuation queue's live entries hold keys below or equal to
          // the all-ones filler of the rest, and the sort is stable: the
          // first n entries of the permutation are the queue's n rays
          ET_CHECK_CUDA(cub::DeviceRadixSort::SortPairs(stmp, stmp_bytes, skey, skey_alt, sval, sperm,
                                                        (int)bt.paths, 0, kSortBits, stream));
        }
        ET_TRY(prof_end(s, kProfShade, pe, 0, A.ctr + C_NRAY0 + cur, stream));
        if (s->dev.n_lights > 0 && b < max_depth) {
          ET_TRY(prof_begin(s, kProfShadow, stream, &pe));
          wf_trace<true><<<grid_s, 128, 0, stream>>>(A, cur, b);
          ET_CHECK_LAUNCH();
          ET_TRY(prof_end(s, kProfShadow, pe, 0, A.ctr + C_NSH, stream));
        }
        cur = nxt;
      }
      const int64_t np = (int64_t)nf * npix;
      ET_TRY(prof_begin(s, kProfAccumulate, stream, &pe));
      wf_accumulate<<<(unsigned)((np + 255) / 256), 256, 0, stream>>>(
          A, acc, s0 == 0, s0 + bt.ns >= spp, rgb, logl, log_mode, log_param);
      ET_CHECK_LAUNCH();
      ET_TRY(prof_end(s, kProfAccumulate, pe, np, nullptr, stream));
    }
  }
  return ET_OK;
}
