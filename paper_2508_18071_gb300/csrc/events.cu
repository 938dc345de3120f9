// Contrast-threshold event generator (paper Sec. 3.1) and event compaction.
//
// One thread per pixel walks the frames in order with its reference level in a
// register.  The decision is taken in FP64 with explicitly rounded operations
// (no contraction), so it is reproducible bit for bit by any IEEE FP64
// implementation fed the same float32 log frames.  Events are appended with one
// atomic per warp and step: an inclusive warp scan of the per-thread counts
// gives each thread its slot.
#include "et_internal.cuh"
#include "event_emit.cuh"

namespace {

__global__ void __launch_bounds__(256)
threshold_kernel(const float* __restrict__ logl, int F, int H, int W, double C, int t0,
                 double* __restrict__ ref, int initialized, et_event* events, int64_t cap,
                 unsigned long long* n_events) {
  const int64_t npix = (int64_t)H * W;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = q < npix;
  double r = 0.0;
  int f0 = 0;
  if (live) {
    if (!initialized) r = (double)__ldg(logl + q);
    else r = ref[q];
  }
  if (!initialized) f0 = 1;
  const uint32_t x = live ? (uint32_t)(q % W) : 0u, y = live ? (uint32_t)(q / W) : 0u;
  for (int f = f0; f < F; ++f) {
    uint32_t n = 0;
    int p = 0;
    if (live) {
      const double d = __dsub_rn((double)__ldg(logl + (int64_t)f * npix + q), r);
      const double k = floor(__ddiv_rn(fabs(d), C));
      if (k > 0.0) {
        p = d > 0.0 ? 1 : -1;
        n = (uint32_t)k;
        r = __dadd_rn(r, __dmul_rn(__dmul_rn((double)p, k), C));
      }
    }
    emit_events_warp(events, cap, n_events, n, x, y, (uint32_t)(t0 + f), p);
  }
  if (live && F > 0) ref[q] = r;
}

}  // namespace

extern "C" int et_threshold_events(const float* logl, int32_t F, int32_t H, int32_t W, float C,
                                   int32_t t0, double* ref, int32_t initialized, et_event* events,
                                   int64_t cap, int64_t* n_events, void* stream_) {
  if (F < 0 || H < 1 || W < 1 || H > 65535 || W > 65535 || !(C > 0.0f) || cap < 0) return ET_ERR_ARG;
  if (!ref || !n_events || (F > 0 && !logl) || (cap > 0 && !events)) return ET_ERR_ARG;
  cudaStream_t stream = (cudaStream_t)stream_;
  ET_CHECK_CUDA(cudaMemsetAsync(n_events, 0, sizeof(int64_t), stream));
  if (F == 0) return ET_OK;
  const int64_t npix = (int64_t)H * W;
  const int threads = 256;
  const int64_t blocks = (npix + threads - 1) / threads;
  threshold_kernel<<<(unsigned)blocks, threads, 0, stream>>>(
      logl, F, H, W, (double)C, t0, ref, initialized, events, cap,
      reinterpret_cast<unsigned long long*>(n_events));
  ET_CHECK_LAUNCH();
  return ET_OK;
}
