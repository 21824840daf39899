// Launchers of the two-steps-per-launch (temporally blocked) kernels, see step2.cu.
#pragma once

#include "common.cuh"
#include "step_f16.cuh"

namespace lbmem {

// Allow the kernels' dynamic shared memory (call once per device, outside stream capture).
cudaError_t step2_prepare();
cudaError_t launch_step2_f32(const StepArgs<float> &a, const float *fin, float *fout, const long long *t_in,
                             long long *t_out, bool accumulate, cudaStream_t s);
cudaError_t launch_step2_f16(const F16Args &a, const long long *t_in, long long *t_out, bool accumulate,
                             cudaStream_t s);

}  // namespace lbmem
