// Car-among-pedestrians kernels (placeholder until the car path lands).
#include "model.hpp"

namespace dsp {
cudaError_t launch_car_expand(dsp_model*, const dsp_leaf_job*, const int4*, int, unsigned int*, cudaStream_t) {
  return cudaErrorNotSupported;
}
cudaError_t launch_car_step(const DevModel*, int, const uint32_t*, int, int, const int32_t*, int, uint32_t*, int,
                            uint64_t*, float*, uint32_t, cudaStream_t) {
  return cudaErrorNotSupported;
}
cudaError_t launch_car_rollout(const DevModel*, int, DevWork*, const uint32_t*, int, int, int, float*, uint32_t,
                               cudaStream_t) {
  return cudaErrorNotSupported;
}
}  // namespace dsp
