// tc_maps.cu -- tensor-core (tcgen05) forms of the lambda / nu sums.
#include "squeeze_internal.cuh"

int sq_launch_step_tc(const squeeze_handle *, const uint8_t *, uint8_t *, cudaStream_t) {
  return SQUEEZE_ERR_UNSUPPORTED;
}

int sq_launch_map_tc(const squeeze_handle *, int, const void *, void *, uint64_t, cudaStream_t) {
  return SQUEEZE_ERR_UNSUPPORTED;
}
