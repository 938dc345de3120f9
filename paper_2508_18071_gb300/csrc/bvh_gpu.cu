// Binned-SAH BVH construction on the GPU.
//
// The hierarchy is built top-down one level at a time.  For every node
// (task) of the current level the device
//   * reduces the bounds of its triangles and of their centroids,
//   * bins the centroids into 32 slabs per axis (counts and bounds per bin),
//     each block accumulating a 1024-triangle chunk in shared memory first,
//   * evaluates the surface-area heuristic C = 1 + (A_L N_L + A_R N_R) / A at
//     the 31 bin boundaries of each axis and keeps the cheapest split (a node
//     of at most 4 triangles becomes a leaf when that is cheaper; a node whose
//     centroids coincide is halved by position),
//   * partitions its triangle indices with per-node atomic cursors.
// The host keeps only the per-node records (a few numbers per node) and
// launches the next level; leaves copy their index range to the final
// permutation as soon as they are decided.
#include <cstring>
#include "et_internal.cuh"
#include "bvh_build.h"

namespace {

constexpr int kChunk = 1024;
constexpr int kThreads = 256;
constexpr int kBinInts = 3 * kSahBins * 7;   // per task: axis x bin x (count, lo3, hi3)

__host__ __device__ inline int fenc(float f) {
  int i;
#ifdef __CUDA_ARCH__
  i = __float_as_int(f);
#else
  std::memcpy(&i, &f, 4);
#endif
  return i >= 0 ? i : i ^ 0x7FFFFFFF;
}
__host__ __device__ inline float fdec(int i) {
  const int j = i >= 0 ? i : i ^ 0x7FFFFFFF;
#ifdef __CUDA_ARCH__
  return __int_as_float(j);
#else
  float f;
  std::memcpy(&f, &j, 4);
  return f;
#endif
}

struct Task { int first, count; };

// empty accumulators: bounds (12 ints per task: box lo/hi, centroid lo/hi) and
// bins (count 0, lo = +max, hi = -max)
__global__ void init_acc(int* __restrict__ tbox, int* __restrict__ bins, int n_tasks) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lo = fenc(FLT_MAX), hi = fenc(-FLT_MAX);
  if (i < 12LL * n_tasks) tbox[i] = (i % 6) < 3 ? lo : hi;
  if (i < (int64_t)kBinInts * n_tasks) {
    const int f = (int)(i % 7);
    bins[i] = f == 0 ? 0 : (f <= 3 ? lo : hi);
  }
}

// triangle bounds (lo, hi) and centroids from the vertices
__global__ void prim_bounds(const float* __restrict__ v, int64_t n, float* __restrict__ tb,
                            float* __restrict__ cen) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float* p = v + 9 * i;
  for (int k = 0; k < 3; ++k) {
    const float a = p[k], b = p[3 + k], c = p[6 + k];
    tb[6 * i + k] = fminf(a, fminf(b, c));
    tb[6 * i + 3 + k] = fmaxf(a, fmaxf(b, c));
    cen[3 * i + k] = (a + b + c) * (1.0f / 3.0f);
  }
}

// per task: bounds of the triangles (6 ints) and of the centroids (6 ints)
__global__ void __launch_bounds__(kThreads)
task_bounds(const int2* __restrict__ chunks, const Task* __restrict__ tasks, const int* __restrict__ idx,
            const float* __restrict__ tb, const float* __restrict__ cen, int* __restrict__ tbox) {
  __shared__ int s[12];
  const int2 ch = chunks[blockIdx.x];
  const Task t = tasks[ch.x];
  if (threadIdx.x < 12) s[threadIdx.x] = (threadIdx.x % 6) < 3 ? fenc(FLT_MAX) : fenc(-FLT_MAX);
  __syncthreads();
  const int end = min(t.count, ch.y + kChunk);
  int loc[12];
  for (int k = 0; k < 12; ++k) loc[k] = (k % 6) < 3 ? fenc(FLT_MAX) : fenc(-FLT_MAX);
  for (int i = ch.y + threadIdx.x; i < end; i += kThreads) {
    const int p = idx[t.first + i];
    for (int k = 0; k < 3; ++k) {
      loc[k] = min(loc[k], fenc(tb[6 * p + k]));
      loc[3 + k] = max(loc[3 + k], fenc(tb[6 * p + 3 + k]));
      loc[6 + k] = min(loc[6 + k], fenc(cen[3 * p + k]));
      loc[9 + k] = max(loc[9 + k], fenc(cen[3 * p + k]));
    }
  }
  for (int k = 0; k < 12; ++k) {
    if ((k % 6) < 3) atomicMin(&s[k], loc[k]);
    else atomicMax(&s[k], loc[k]);
  }
  __syncthreads();
  if (threadIdx.x < 12) {
    const int k = threadIdx.x;
    if ((k % 6) < 3) atomicMin(&tbox[12 * ch.x + k], s[k]);
    else atomicMax(&tbox[12 * ch.x + k], s[k]);
  }
}

__device__ __forceinline__ int bin_of(float c, float lo, float ext) {
  return min(kSahBins - 1, max(0, (int)((c - lo) * ((float)kSahBins / ext))));
}

// per task, axis and bin: triangle count and bounds
__global__ void __launch_bounds__(kThreads)
task_bins(const int2* __restrict__ chunks, const Task* __restrict__ tasks, const int* __restrict__ idx,
          const float* __restrict__ tb, const float* __restrict__ cen, const int* __restrict__ tbox,
          int* __restrict__ bins) {
  __shared__ int s[kBinInts];
  const int2 ch = chunks[blockIdx.x];
  const Task t = tasks[ch.x];
  for (int i = threadIdx.x; i < kBinInts; i += kThreads) {
    const int f = i % 7;
    s[i] = f == 0 ? 0 : (f <= 3 ? fenc(FLT_MAX) : fenc(-FLT_MAX));
  }
  __syncthreads();
  float clo[3], cext[3];
  for (int k = 0; k < 3; ++k) {
    clo[k] = fdec(tbox[12 * ch.x + 6 + k]);
    cext[k] = fdec(tbox[12 * ch.x + 9 + k]) - clo[k];
  }
  const int end = min(t.count, ch.y + kChunk);
  for (int i = ch.y + threadIdx.x; i < end; i += kThreads) {
    const int p = idx[t.first + i];
    for (int a = 0; a < 3; ++a) {
      if (!(cext[a] > 0.0f)) continue;
      int* b = s + (a * kSahBins + bin_of(cen[3 * p + a], clo[a], cext[a])) * 7;
      atomicAdd(b, 1);
      for (int k = 0; k < 3; ++k) {
        atomicMin(b + 1 + k, fenc(tb[6 * p + k]));
        atomicMax(b + 4 + k, fenc(tb[6 * p + 3 + k]));
      }
    }
  }
  __syncthreads();
  int* g = bins + (int64_t)ch.x * kBinInts;
  for (int i = threadIdx.x; i < kBinInts; i += kThreads) {
    const int f = i % 7;
    if (f == 0) { if (s[i]) atomicAdd(g + i, s[i]); }
    else if (f <= 3) atomicMin(g + i, s[i]);
    else atomicMax(g + i, s[i]);
  }
}

__device__ __forceinline__ double box_area(const float* lo, const float* hi) {
  const double dx = (double)hi[0] - lo[0], dy = (double)hi[1] - lo[1], dz = (double)hi[2] - lo[2];
  if (dx < 0 || dy < 0 || dz < 0) return 0.0;
  return 2.0 * (dx * dy + dy * dz + dz * dx);
}

// per task: the cheapest split.  dec = (kind, axis, bin, left count):
// kind 0 leaf, 1 SAH split (left = bin < split bin), 2 split by position.
__global__ void task_split(const Task* __restrict__ tasks, int n_tasks, const int* __restrict__ tbox,
                           const int* __restrict__ bins, int4* __restrict__ dec) {
  const int ti = blockIdx.x * blockDim.x + threadIdx.x;
  if (ti >= n_tasks) return;
  const Task t = tasks[ti];
  float lo[3], hi[3];
  for (int k = 0; k < 3; ++k) { lo[k] = fdec(tbox[12 * ti + k]); hi[k] = fdec(tbox[12 * ti + 3 + k]); }
  const double sa = box_area(lo, hi);
  double best = 1e300;
  int best_axis = -1, best_bin = -1, best_left = 0;
  const int* B = bins + (int64_t)ti * kBinInts;
  for (int a = 0; a < 3; ++a) {
    // suffix areas / counts
    double rarea[kSahBins];
    int rcnt[kSahBins];
    float rl[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, rh[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    int rc = 0;
    for (int b = kSahBins - 1; b > 0; --b) {
      const int* e = B + (a * kSahBins + b) * 7;
      if (e[0]) {
        for (int k = 0; k < 3; ++k) { rl[k] = fminf(rl[k], fdec(e[1 + k])); rh[k] = fmaxf(rh[k], fdec(e[4 + k])); }
        rc += e[0];
      }
      rarea[b] = box_area(rl, rh);
      rcnt[b] = rc;
    }
    float ll[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, lh[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    int lc = 0;
    for (int b = 1; b < kSahBins; ++b) {
      const int* e = B + (a * kSahBins + b - 1) * 7;
      if (e[0]) {
        for (int k = 0; k < 3; ++k) { ll[k] = fminf(ll[k], fdec(e[1 + k])); lh[k] = fmaxf(lh[k], fdec(e[4 + k])); }
        lc += e[0];
      }
      if (lc == 0 || rcnt[b] == 0) continue;
      const double c = 1.0 + (box_area(ll, lh) * lc + rarea[b] * rcnt[b]) / (sa > 0 ? sa : 1.0);
      if (c < best) { best = c; best_axis = a; best_bin = b; best_left = lc; }
    }
  }
  int4 d;
  if (t.count == 1 || (t.count <= kLeafMax && (best_axis < 0 || best >= (double)t.count))) {
    d = make_int4(0, 0, 0, 0);
  } else if (best_axis >= 0) {
    d = make_int4(1, best_axis, best_bin, best_left);
  } else {
    d = make_int4(2, 0, 0, t.count / 2);
  }
  dec[ti] = d;
}

// scatter each task's indices to its children's ranges (or to the final
// permutation when the task is a leaf)
__global__ void __launch_bounds__(kThreads)
task_partition(const int2* __restrict__ chunks, const Task* __restrict__ tasks, const int* __restrict__ idx,
               const float* __restrict__ cen, const int* __restrict__ tbox, const int4* __restrict__ dec,
               int* __restrict__ cursors, int* __restrict__ idx_out, int* __restrict__ final_perm) {
  const int2 ch = chunks[blockIdx.x];
  const Task t = tasks[ch.x];
  const int4 d = dec[ch.x];
  const int end = min(t.count, ch.y + kChunk);
  float clo = 0.0f, cext = 0.0f;
  if (d.x == 1) {
    clo = fdec(tbox[12 * ch.x + 6 + d.y]);
    cext = fdec(tbox[12 * ch.x + 9 + d.y]) - clo;
  }
  for (int i = ch.y + threadIdx.x; i < end; i += kThreads) {
    const int p = idx[t.first + i];
    if (d.x == 0) { final_perm[t.first + i] = p; continue; }
    bool left;
    if (d.x == 1) left = bin_of(cen[3 * p + d.y], clo, cext) < d.z;
    else left = i < d.w;
    const int slot = left ? atomicAdd(&cursors[2 * ch.x], 1) : d.w + atomicAdd(&cursors[2 * ch.x + 1], 1);
    idx_out[t.first + slot] = p;
  }
}



}  // namespace

int gpu_binned_sah(const float* tris, int64_t n, cudaStream_t st, std::vector<BuildNode>& nodes,
                   std::vector<int>& perm, int& max_depth) {
  nodes.clear();
  perm.assign((size_t)n, 0);
  max_depth = 0;
  if (n <= 0) return ET_ERR_ARG;
  DevBuf<float> v, tb, cen;
  DevBuf<int> idx[2], fin, tbox, bins, cursors;
  DevBuf<Task> tasks_d;
  DevBuf<int2> chunks_d;
  DevBuf<int4> dec_d;
  int rc;
  if ((rc = v.ensure(9 * (size_t)n)) || (rc = tb.ensure(6 * (size_t)n)) || (rc = cen.ensure(3 * (size_t)n)) ||
      (rc = idx[0].ensure((size_t)n)) || (rc = idx[1].ensure((size_t)n)) || (rc = fin.ensure((size_t)n)))
    return rc;
  ET_CHECK_CUDA(cudaMemcpyAsync(v.p, tris, sizeof(float) * 9 * (size_t)n, cudaMemcpyHostToDevice, st));
  prim_bounds<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(v.p, n, tb.p, cen.p);
  ET_CHECK_LAUNCH();
  {
    std::vector<int> iota((size_t)n);
    for (int64_t i = 0; i < n; ++i) iota[i] = (int)i;
    ET_CHECK_CUDA(cudaMemcpyAsync(idx[0].p, iota.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, st));
    ET_CHECK_CUDA(cudaStreamSynchronize(st));
  }
  struct HostTask { int node, first, count, depth; };
  std::vector<HostTask> level = {{0, 0, (int)n, 0}};
  nodes.push_back(BuildNode());
  int cur = 0;
  std::vector<Task> th;
  std::vector<int2> chh;
  std::vector<int4> dech;
  std::vector<int> boxh;
  while (!level.empty()) {
    const int T = (int)level.size();
    th.resize(T);
    chh.clear();
    for (int i = 0; i < T; ++i) {
      th[i] = {level[i].first, level[i].count};
      max_depth = std::max(max_depth, level[i].depth);
      for (int c = 0; c < level[i].count; c += kChunk) chh.push_back(make_int2(i, c));
    }
    const int nch = (int)chh.size();
    if ((rc = tasks_d.ensure(T)) || (rc = chunks_d.ensure(nch)) || (rc = dec_d.ensure(T)) ||
        (rc = tbox.ensure(12 * (size_t)T)) || (rc = bins.ensure((size_t)T * kBinInts)) ||
        (rc = cursors.ensure(2 * (size_t)T)))
      return rc;
    boxh.resize(12 * (size_t)T);
    ET_CHECK_CUDA(cudaMemcpyAsync(tasks_d.p, th.data(), sizeof(Task) * T, cudaMemcpyHostToDevice, st));
    ET_CHECK_CUDA(cudaMemcpyAsync(chunks_d.p, chh.data(), sizeof(int2) * nch, cudaMemcpyHostToDevice, st));
    init_acc<<<(unsigned)(((int64_t)kBinInts * T + 255) / 256), 256, 0, st>>>(tbox.p, bins.p, T);
    ET_CHECK_LAUNCH();
    ET_CHECK_CUDA(cudaMemsetAsync(cursors.p, 0, sizeof(int) * 2 * (size_t)T, st));
    task_bounds<<<nch, kThreads, 0, st>>>(chunks_d.p, tasks_d.p, idx[cur].p, tb.p, cen.p, tbox.p);
    ET_CHECK_LAUNCH();
    task_bins<<<nch, kThreads, 0, st>>>(chunks_d.p, tasks_d.p, idx[cur].p, tb.p, cen.p, tbox.p, bins.p);
    ET_CHECK_LAUNCH();
    task_split<<<(T + 127) / 128, 128, 0, st>>>(tasks_d.p, T, tbox.p, bins.p, dec_d.p);
    ET_CHECK_LAUNCH();
    task_partition<<<nch, kThreads, 0, st>>>(chunks_d.p, tasks_d.p, idx[cur].p, cen.p, tbox.p, dec_d.p,
                                             cursors.p, idx[cur ^ 1].p, fin.p);
    ET_CHECK_LAUNCH();
    dech.resize(T);
    ET_CHECK_CUDA(cudaMemcpyAsync(dech.data(), dec_d.p, sizeof(int4) * T, cudaMemcpyDeviceToHost, st));
    ET_CHECK_CUDA(cudaMemcpyAsync(boxh.data(), tbox.p, sizeof(int) * 12 * (size_t)T, cudaMemcpyDeviceToHost, st));
    ET_CHECK_CUDA(cudaStreamSynchronize(st));
    std::vector<HostTask> next;
    for (int i = 0; i < T; ++i) {
      const HostTask& ht = level[i];
      BuildNode& nd = nodes[ht.node];
      for (int k = 0; k < 3; ++k) { nd.box.lo[k] = fdec(boxh[12 * i + k]); nd.box.hi[k] = fdec(boxh[12 * i + 3 + k]); }
      nd.first = ht.first;
      if (dech[i].x == 0) {
        nd.left = nd.right = -1;
        nd.count = ht.count;
        continue;
      }
      const int left = dech[i].w;
      const int L = (int)nodes.size();
      nodes.push_back(BuildNode());
      const int R = (int)nodes.size();
      nodes.push_back(BuildNode());
      BuildNode& nd2 = nodes[ht.node];   // the vector may have moved
      nd2.left = L; nd2.right = R; nd2.count = 0;
      next.push_back({L, ht.first, left, ht.depth + 1});
      next.push_back({R, ht.first + left, ht.count - left, ht.depth + 1});
    }
    level.swap(next);
    cur ^= 1;
  }
  ET_CHECK_CUDA(cudaMemcpyAsync(perm.data(), fin.p, sizeof(int) * (size_t)n, cudaMemcpyDeviceToHost, st));
  ET_CHECK_CUDA(cudaStreamSynchronize(st));
  return ET_OK;
}
