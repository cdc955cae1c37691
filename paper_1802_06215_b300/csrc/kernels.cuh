// Host-side launchers of the device kernels (one per .cu file).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace dsp {

size_t rs_expand_smem();
int rs_items_per_unit();
cudaError_t launch_rs_expand(const DevModel* gm, int robots, DevWork* work, const dsp_leaf_job* jobs,
                             const int4* units, int n_units, unsigned int* head, uint32_t plan_step, int grid,
                             int block, cudaStream_t st);
cudaError_t launch_rs_step(const DevModel* gm, int robots, const uint32_t* in, int in_cap, int count,
                           const int32_t* actions, int depth, uint32_t* out, int out_cap, uint64_t* keys,
                           float* rewards, uint32_t plan_step, cudaStream_t st);
cudaError_t launch_rs_rollout(const DevModel* gm, int robots, DevWork* work, const uint32_t* block, int cap,
                              int count, const int8_t* hist, int start_depth, float* value, uint32_t plan_step,
                              cudaStream_t st);
int rs_expand_blocks_per_sm(int robots, int block);

}  // namespace dsp
