// Warp-aggregated event append shared by the event-producing kernels.
#pragma once
#include "et_internal.cuh"

// Every lane of the warp must call this (lanes without events pass n = 0).
// Lane i appends n_i copies of (x, y, t, p); one atomicAdd per warp reserves
// the slots.  Slots at or beyond `cap` are counted but not written.
__device__ __forceinline__ void emit_events_warp(et_event* events, int64_t cap,
                                                 unsigned long long* counter, uint32_t n,
                                                 uint32_t x, uint32_t y, uint32_t t, int p) {
  const unsigned lane = threadIdx.x & 31u;
  uint32_t incl = n;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= (unsigned)o) incl += v;
  }
  const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
  if (total == 0) return;
  unsigned long long base = 0;
  if (lane == 31) base = atomicAdd(counter, (unsigned long long)total);
  base = __shfl_sync(0xFFFFFFFFu, base, 31);
  const unsigned long long start = base + (incl - n);
  uint32_t* out = reinterpret_cast<uint32_t*>(events);
  // slots at or beyond cap are counted only: the loop stops there
  for (uint32_t i = 0; i < n && start + i < (unsigned long long)cap; ++i) {
    const unsigned long long slot = start + i;
    out[3 * slot] = x | (y << 16);
    out[3 * slot + 1] = t;
    out[3 * slot + 2] = (uint32_t)(uint8_t)(int8_t)p;
  }
}
