// FP64 plain form of the fused pass (full rho and E in storage).
#include "sweep.cuh"

namespace ppm {
void launch_sweep_f64(const SweepArgs<double> &a, dim3 grid, dim3 block, cudaStream_t st) {
    sweep_kernel<double, true><<<grid, block, 0, st>>>(a);
}
}  // namespace ppm
