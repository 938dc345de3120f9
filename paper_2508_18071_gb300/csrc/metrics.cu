// Event-stream F1 support: maximum matching of two event lists (host code),
// and the same count on two dense spike tensors (device kernel).
//
// Two events match when they share pixel and polarity and their frame
// indices differ by at most `delta`.  Keys (y, x, p, t) are packed into 64-bit
// integers and sorted; within one (y, x, p) the admissible pairs form an
// interval graph on the time line, for which the earliest-first greedy scan
// of both sorted lists is a maximum matching.
#include <algorithm>
#include <vector>
#include "et_internal.cuh"

namespace {
inline uint64_t pack(const et_event& e) {
  const uint64_t pol = e.p > 0 ? 1u : 0u;
  return ((uint64_t)e.y << 48) | ((uint64_t)e.x << 32) | (pol << 31) | (uint64_t)(e.t & 0x7FFFFFFFu);
}
}  // namespace

extern "C" int et_event_matches(const et_event* a, int64_t na, const et_event* b, int64_t nb,
                                int32_t delta, int64_t* matches) {
  if (na < 0 || nb < 0 || delta < 0 || !matches || (na > 0 && !a) || (nb > 0 && !b)) return ET_ERR_ARG;
  std::vector<uint64_t> ka((size_t)na), kb((size_t)nb);
  for (int64_t i = 0; i < na; ++i) ka[i] = pack(a[i]);
  for (int64_t i = 0; i < nb; ++i) kb[i] = pack(b[i]);
  std::sort(ka.begin(), ka.end());
  std::sort(kb.begin(), kb.end());
  const uint64_t kmask = ~(uint64_t)0x7FFFFFFFu;
  int64_t i = 0, j = 0, m = 0;
  while (i < na && j < nb) {
    const uint64_t ga = ka[i] & kmask, gb = kb[j] & kmask;
    if (ga != gb) { if (ga < gb) ++i; else ++j; continue; }
    const int64_t ta = (int64_t)(ka[i] & 0x7FFFFFFFu), tb = (int64_t)(kb[j] & 0x7FFFFFFFu);
    if (ta - tb <= delta && tb - ta <= delta) { ++m; ++i; ++j; }
    else if (ta < tb) ++i;
    else ++j;
  }
  *matches = m;
  return ET_OK;
}

// Dense form: one thread per pixel walks the K steps of both spike trains.
// Per polarity, bit i of a mask marks an unmatched event i steps old; events
// older than delta leave the mask.  After each step's events enter, the
// oldest pending event of one train is paired with the oldest pending event
// of the other while both exist: both lie within delta of the current step,
// hence of each other.  This is the earliest-first scan of the host function,
// run forward in time, so it finds a maximum matching too.
namespace {
__global__ void spike_match_kernel(const int8_t* __restrict__ a, const int8_t* __restrict__ b, int64_t K,
                                   int64_t npix, int delta, unsigned long long* out) {
  const int64_t px = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long m = 0;
  if (px < npix) {
    const uint32_t keep = delta >= 31 ? 0xFFFFFFFFu : ((1u << (delta + 1)) - 1u);
    uint32_t pa[2] = {0, 0}, pb[2] = {0, 0};
    for (int64_t t = 0; t < K; ++t) {
      const int8_t sa = a[t * npix + px], sb = b[t * npix + px];
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const int8_t want = p ? (int8_t)1 : (int8_t)-1;
        pa[p] = ((pa[p] << 1) | (sa == want ? 1u : 0u)) & keep;
        pb[p] = ((pb[p] << 1) | (sb == want ? 1u : 0u)) & keep;
        while (pa[p] && pb[p]) {
          pa[p] &= ~(1u << (31 - __clz(pa[p])));
          pb[p] &= ~(1u << (31 - __clz(pb[p])));
          ++m;
        }
      }
    }
  }
  // warp sum, one atomic per warp
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m += __shfl_down_sync(0xFFFFFFFFu, m, o);
  if ((threadIdx.x & 31) == 0 && m) atomicAdd(out, m);
}
}  // namespace

extern "C" int et_spike_matches(const int8_t* a, const int8_t* b, int64_t K, int64_t npix, int32_t delta,
                                int64_t* matches, void* stream) {
  if (K < 0 || npix < 0 || delta < 0 || delta > 30 || !matches || (K * npix > 0 && (!a || !b)))
    return ET_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ET_CHECK_CUDA(cudaMemsetAsync(matches, 0, sizeof(int64_t), st));
  if (K * npix == 0) return ET_OK;
  const int64_t blocks = (npix + 255) / 256;
  if (blocks > 0x7FFFFFFF) return ET_ERR_ARG;
  spike_match_kernel<<<(unsigned)blocks, 256, 0, st>>>(a, b, K, npix, delta,
                                                        reinterpret_cast<unsigned long long*>(matches));
  ET_CHECK_LAUNCH();
  return ET_OK;
}
