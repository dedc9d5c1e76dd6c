// FP32 base-state-deviation form of the fused pass.
#include "sweep.cuh"

namespace ppm {
void launch_sweep_f32(const SweepArgs<float> &a, dim3 grid, dim3 block, cudaStream_t st) {
    sweep_kernel<float, false><<<grid, block, 0, st>>>(a);
}
}  // namespace ppm
