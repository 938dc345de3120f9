// Event-stream F1 support: maximum matching of two event lists (host code).
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
