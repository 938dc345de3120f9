// Tensor-core (tcgen05, BF16 in / FP32 accumulate) EvSNet forward.
#include "et_internal.cuh"
#include "evsnet_common.h"

int et_evsnet_forward_bf16(const float*, int32_t, const et_evsnet_weights*, et_evsnet_state*,
                           int32_t, et_event*, int64_t, int64_t*, float*, int8_t*, cudaStream_t) {
  return ET_ERR_UNIMPLEMENTED;
}
