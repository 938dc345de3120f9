// Full-sweep SAH BVH construction on the GPU (the library's default builder).
//
// The same algorithm as the host sweep (scene.cu): at every node all n - 1
// splits of the centroid order along each axis are evaluated with the surface
// area heuristic C = 1 + (A_L N_L + A_R N_R) / A (areas in double, of float
// boxes), the first minimum in (axis, position) order is taken, a node of at
// most 4 triangles becomes a leaf when splitting is not cheaper, and the
// triangle indices are kept sorted by centroid along all three axes: a split
// stably partitions the two other orders by side.
//
// GPU schedule: the three orders come from one stable radix sort per axis
// (keys: the centroid coordinate made orderable; equal keys keep the index
// order).  The tree is then built one level at a time: one CTA per node of the
// level runs the reverse scan of box unions that gives the right-hand areas,
// the forward scan that gives the costs, the arg-min, and -- in a second kernel
// -- the stable partition of the other two orders.  The host keeps the per-node
// records, forms the next level and finally numbers the nodes in the order the
// host builder allocates them (depth first, children in pairs), so the
// flattened hierarchy has the same layout.
#include <algorithm>
#include <cfloat>
#include <cstring>
#include <cub/device/device_radix_sort.cuh>
#include "et_internal.cuh"
#include "bvh_build.h"

namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;

struct Seg { int first, count; };
// per node of a level: split axis (-1: leaf), split position, cost, box
struct Dec { int axis, split; double cost; float lo[3], hi[3]; };

struct B6 { float lo[3], hi[3]; };

__device__ __forceinline__ B6 empty6() {
  B6 b;
#pragma unroll
  for (int k = 0; k < 3; ++k) { b.lo[k] = FLT_MAX; b.hi[k] = -FLT_MAX; }
  return b;
}
__device__ __forceinline__ B6 join(const B6& a, const B6& b) {
  B6 r;
#pragma unroll
  for (int k = 0; k < 3; ++k) { r.lo[k] = fminf(a.lo[k], b.lo[k]); r.hi[k] = fmaxf(a.hi[k], b.hi[k]); }
  return r;
}
// the host builder's area: 2 (dx dy + dy dz + dz dx) in double, each product
// and sum rounded on its own (no fused multiply-add)
__device__ __forceinline__ double area6(const B6& b) {
  const double dx = __dsub_rn((double)b.hi[0], (double)b.lo[0]);
  const double dy = __dsub_rn((double)b.hi[1], (double)b.lo[1]);
  const double dz = __dsub_rn((double)b.hi[2], (double)b.lo[2]);
  if (dx < 0 || dy < 0 || dz < 0) return 0.0;
  return __dmul_rn(2.0, __dadd_rn(__dadd_rn(__dmul_rn(dx, dy), __dmul_rn(dy, dz)), __dmul_rn(dz, dx)));
}
__device__ __forceinline__ B6 shfl_up6(const B6& b, int d) {
  B6 r;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    r.lo[k] = __shfl_up_sync(0xFFFFFFFFu, b.lo[k], d);
    r.hi[k] = __shfl_up_sync(0xFFFFFFFFu, b.hi[k], d);
  }
  return r;
}

// inclusive block scan of box unions in thread order; `carry` (the union of
// everything before this chunk) is joined in and updated to the chunk's total
__device__ B6 block_scan(B6 v, B6& carry, B6* wsum) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const B6 u = shfl_up6(v, d);
    if (lane >= d) v = join(v, u);
  }
  if (lane == 31) wsum[w] = v;
  __syncthreads();
  B6 pre = carry;
  for (int j = 0; j < w; ++j) pre = join(pre, wsum[j]);
  v = join(v, pre);
  __syncthreads();
  B6 tot = carry;
  for (int j = 0; j < kWarps; ++j) tot = join(tot, wsum[j]);
  carry = tot;
  __syncthreads();
  return v;
}

__device__ __forceinline__ B6 load_box(const float* __restrict__ tb, int t) {
  B6 b;
#pragma unroll
  for (int k = 0; k < 3; ++k) { b.lo[k] = tb[6 * t + k]; b.hi[k] = tb[6 * t + 3 + k]; }
  return b;
}

__global__ void prim_boxes(const float* __restrict__ v, int64_t n, float* __restrict__ tb,
                           unsigned* __restrict__ keys) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float* p = v + 9 * i;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    tb[6 * i + k] = fminf(fminf(p[k], p[3 + k]), p[6 + k]);
    tb[6 * i + 3 + k] = fmaxf(fmaxf(p[k], p[3 + k]), p[6 + k]);
    // centroid as the host computes it, made orderable for the radix sort
    // (-0 and +0 compare equal there: both map to the key of +0)
    float c = (p[k] + p[3 + k] + p[6 + k]) * (1.0f / 3.0f);
    if (c == 0.0f) c = 0.0f;
    const unsigned u = __float_as_uint(c);
    keys[(int64_t)k * n + i] = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
  }
}

__global__ void iota3(int* __restrict__ vals, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 3 * n) vals[i] = (int)(i % n);
}

// one CTA per node of the level: box, the best split over all axes and positions
__global__ void __launch_bounds__(kThreads)
sweep_eval(const Seg* __restrict__ segs, const float* __restrict__ tb, const int* __restrict__ ord,
           int64_t n, double* __restrict__ rarea, Dec* __restrict__ dec) {
  __shared__ B6 wsum[kWarps];
  __shared__ double wcost[kWarps];
  __shared__ int wkey[kWarps];
  const Seg sg = segs[blockIdx.x];
  const int first = sg.first, count = sg.count, tid = threadIdx.x;
  // node box (the union over the order of axis 0)
  B6 carry = empty6();
  for (int c0 = 0; c0 < count; c0 += kThreads) {
    const int i = c0 + tid;
    const B6 v = i < count ? load_box(tb, ord[first + i]) : empty6();
    block_scan(v, carry, wsum);
  }
  const B6 box = carry;
  const double sa = area6(box);
  const double inv = sa > 0 ? sa : 1.0;
  double best = DBL_MAX;
  int key = INT_MAX;                   // axis * 2^27 + split: the order of the host's scan
  if (count > 1) {
    for (int a = 0; a < 3; ++a) {
      const int* o = ord + (int64_t)a * n + first;
      double* ra = rarea + first;
      // right-hand areas: union of positions i .. count-1, for i >= 1
      B6 rc = empty6();
      for (int c0 = count - 1; c0 >= 1; c0 -= kThreads) {
        const int i = c0 - tid;        // descending within the chunk
        const B6 v = i >= 1 ? load_box(tb, o[i]) : empty6();
        const B6 s = block_scan(v, rc, wsum);
        if (i >= 1) ra[i] = area6(s);
      }
      __syncthreads();
      // left-hand unions of positions 0 .. i-1 and the costs
      B6 lc = empty6();
      for (int c0 = 1; c0 < count; c0 += kThreads) {
        const int i = c0 + tid;
        const B6 v = i < count ? load_box(tb, o[i - 1]) : empty6();
        const B6 s = block_scan(v, lc, wsum);
        if (i < count) {
          const double c = __dadd_rn(1.0, __ddiv_rn(__dadd_rn(__dmul_rn(area6(s), (double)i),
                                                              __dmul_rn(ra[i], (double)(count - i))),
                                                    inv));
          const int k = (a << 27) | i;
          if (c < best || (c == best && k < key)) { best = c; key = k; }
        }
      }
      __syncthreads();
    }
  }
  // arg-min over the block: lowest cost, then lowest (axis, position)
  for (int d = 16; d > 0; d >>= 1) {
    const double oc = __shfl_down_sync(0xFFFFFFFFu, best, d);
    const int ok = __shfl_down_sync(0xFFFFFFFFu, key, d);
    if (oc < best || (oc == best && ok < key)) { best = oc; key = ok; }
  }
  if ((tid & 31) == 0) { wcost[tid >> 5] = best; wkey[tid >> 5] = key; }
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < kWarps; ++w)
      if (wcost[w] < best || (wcost[w] == best && wkey[w] < key)) { best = wcost[w]; key = wkey[w]; }
    Dec d;
    const bool leaf = count == 1 || (count <= kLeafMax && best >= count);
    d.axis = leaf ? -1 : (key >> 27);
    d.split = leaf ? 0 : (key & ((1 << 27) - 1));
    d.cost = best;
#pragma unroll
    for (int k = 0; k < 3; ++k) { d.lo[k] = box.lo[k]; d.hi[k] = box.hi[k]; }
    dec[blockIdx.x] = d;
  }
}

// one CTA per split node: side of every triangle, then the stable partition of
// the two other orders (left part first, each part in its old order)
__global__ void __launch_bounds__(kThreads)
sweep_partition(const Seg* __restrict__ segs, const Dec* __restrict__ dec, int* __restrict__ ord,
                int64_t n, unsigned char* __restrict__ side, int* __restrict__ tmp) {
  __shared__ int wcnt[kWarps];
  const Dec d = dec[blockIdx.x];
  if (d.axis < 0) return;
  const Seg sg = segs[blockIdx.x];
  const int first = sg.first, count = sg.count, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int* oa = ord + (int64_t)d.axis * n + first;
  for (int i = tid; i < count; i += kThreads) side[oa[i]] = i < d.split ? 1 : 0;
  __syncthreads();
  for (int b = 0; b < 3; ++b) {
    if (b == d.axis) continue;
    int* o = ord + (int64_t)b * n + first;
    int* t = tmp + first;
    int nl = 0;                           // left elements before this chunk
    for (int c0 = 0; c0 < count; c0 += kThreads) {
      const int i = c0 + tid;
      const int e = i < count ? o[i] : 0;
      const int isl = i < count ? (int)side[e] : 0;
      const unsigned m = __ballot_sync(0xFFFFFFFFu, isl);
      const int before = __popc(m & ((1u << lane) - 1u));
      if (lane == 31) wcnt[w] = __popc(m);
      __syncthreads();
      int pre = 0, tot = 0;
      for (int j = 0; j < kWarps; ++j) { if (j < w) pre += wcnt[j]; tot += wcnt[j]; }
      if (i < count) {
        const int lpos = nl + pre + before;          // left elements before i
        t[isl ? lpos : d.split + (i - lpos)] = e;
      }
      nl += tot;
      __syncthreads();
    }
    __syncthreads();
    for (int i = tid; i < count; i += kThreads) o[i] = t[i];
    __syncthreads();
  }
}

}  // namespace

int gpu_sweep_sah(const float* tris, int64_t n, cudaStream_t st, std::vector<BuildNode>& nodes,
                  std::vector<int>& perm, int& max_depth) {
  nodes.clear();
  perm.assign((size_t)n, 0);
  max_depth = 0;
  if (n <= 0 || n >= (1LL << 27)) return ET_ERR_ARG;
  DevBuf<float> v, tb;
  DevBuf<unsigned> keys, keys_out;
  DevBuf<int> vals, ord, tmp;
  DevBuf<double> rarea;
  DevBuf<unsigned char> side, cub_tmp;
  DevBuf<Seg> segs_d;
  DevBuf<Dec> dec_d;
  int rc;
  if ((rc = v.ensure(9 * (size_t)n)) || (rc = tb.ensure(6 * (size_t)n)) || (rc = keys.ensure(3 * (size_t)n)) ||
      (rc = keys_out.ensure((size_t)n)) || (rc = vals.ensure(3 * (size_t)n)) || (rc = ord.ensure(3 * (size_t)n)) ||
      (rc = tmp.ensure((size_t)n)) || (rc = rarea.ensure((size_t)n)) || (rc = side.ensure((size_t)n)))
    return rc;
  ET_CHECK_CUDA(cudaMemcpyAsync(v.p, tris, sizeof(float) * 9 * (size_t)n, cudaMemcpyHostToDevice, st));
  prim_boxes<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(v.p, n, tb.p, keys.p);
  ET_CHECK_LAUNCH();
  iota3<<<(unsigned)((3 * n + 255) / 256), 256, 0, st>>>(vals.p, n);
  ET_CHECK_LAUNCH();
  // the three centroid orders (stable: equal keys keep the index order)
  size_t tmp_bytes = 0;
  ET_CHECK_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, keys.p, keys_out.p, vals.p, ord.p, (int)n,
                                                0, 32, st));
  if ((rc = cub_tmp.ensure(tmp_bytes))) return rc;
  for (int a = 0; a < 3; ++a) {
    ET_CHECK_CUDA(cub::DeviceRadixSort::SortPairs(cub_tmp.p, tmp_bytes, keys.p + (size_t)a * n, keys_out.p,
                                                  vals.p + (size_t)a * n, ord.p + (size_t)a * n, (int)n, 0, 32,
                                                  st));
  }
  // level by level; the tree is kept with provisional node ids
  struct TNode { Dec d; int first, count, left, right; };
  std::vector<TNode> tn;
  struct Item { int id, first, count, depth; };
  std::vector<Item> level = {{0, 0, (int)n, 0}};
  tn.push_back(TNode());
  std::vector<Seg> sh;
  std::vector<Dec> dh;
  while (!level.empty()) {
    const int T = (int)level.size();
    sh.resize(T);
    for (int i = 0; i < T; ++i) {
      sh[i] = {level[i].first, level[i].count};
      max_depth = std::max(max_depth, level[i].depth);
    }
    if ((rc = segs_d.ensure((size_t)T)) || (rc = dec_d.ensure((size_t)T))) return rc;
    ET_CHECK_CUDA(cudaMemcpyAsync(segs_d.p, sh.data(), sizeof(Seg) * T, cudaMemcpyHostToDevice, st));
    sweep_eval<<<T, kThreads, 0, st>>>(segs_d.p, tb.p, ord.p, n, rarea.p, dec_d.p);
    ET_CHECK_LAUNCH();
    sweep_partition<<<T, kThreads, 0, st>>>(segs_d.p, dec_d.p, ord.p, n, side.p, tmp.p);
    ET_CHECK_LAUNCH();
    dh.resize(T);
    ET_CHECK_CUDA(cudaMemcpyAsync(dh.data(), dec_d.p, sizeof(Dec) * T, cudaMemcpyDeviceToHost, st));
    ET_CHECK_CUDA(cudaStreamSynchronize(st));
    std::vector<Item> next;
    for (int i = 0; i < T; ++i) {
      // by index: the vector grows below
      const int id = level[i].id;
      tn[id].d = dh[i];
      tn[id].first = level[i].first;
      tn[id].count = level[i].count;
      tn[id].left = tn[id].right = -1;
      if (dh[i].axis < 0) continue;
      if (max_depth + 1 > kMaxBvhDepth) return ET_ERR_UNIMPLEMENTED;   // deeper than the traversal stack
      if (dh[i].split < 1 || dh[i].split >= level[i].count) return ET_ERR_UNIMPLEMENTED;
      const int L = (int)tn.size();
      tn.push_back(TNode());
      tn.push_back(TNode());
      tn[id].left = L;
      tn[id].right = L + 1;
      next.push_back({L, level[i].first, dh[i].split, level[i].depth + 1});
      next.push_back({L + 1, level[i].first + dh[i].split, level[i].count - dh[i].split, level[i].depth + 1});
    }
    level.swap(next);
  }
  ET_CHECK_CUDA(cudaMemcpyAsync(perm.data(), ord.p, sizeof(int) * (size_t)n, cudaMemcpyDeviceToHost, st));
  ET_CHECK_CUDA(cudaStreamSynchronize(st));
  // number the nodes as the host builder allocates them: a stack, the left
  // child popped first, both children allocated when their parent splits
  nodes.resize(tn.size());
  std::vector<std::pair<int, int>> stack = {{0, 0}};   // (provisional id, final id)
  int next_id = 1;
  while (!stack.empty()) {
    const auto [pid, fid] = stack.back();
    stack.pop_back();
    if (pid < 0 || pid >= (int)tn.size() || fid >= (int)nodes.size()) return ET_ERR_UNIMPLEMENTED;
    const TNode& t = tn[pid];
    // a leaf holds 1 .. kLeafMax triangles (the leaf reference keeps 3 bits of count)
    if (t.left < 0 && (t.count < 1 || t.count > kLeafMax)) return ET_ERR_UNIMPLEMENTED;
    BuildNode& b = nodes[fid];
    for (int k = 0; k < 3; ++k) { b.box.lo[k] = t.d.lo[k]; b.box.hi[k] = t.d.hi[k]; }
    b.first = t.first;
    if (t.left < 0) {
      b.left = b.right = -1;
      b.count = t.count;
      continue;
    }
    b.count = 0;
    b.left = next_id;
    b.right = next_id + 1;
    next_id += 2;
    stack.push_back({t.right, b.right});
    stack.push_back({t.left, b.left});
  }
  return ET_OK;
}
