// FP32 base-state-deviation form of the fused pass (approximate division
// and square root: this unit is compiled with -prec-div=false -prec-sqrt=false).
#include "sweep.cuh"

namespace ppm {
// Raise the dynamic shared-memory limit of both variants (once per device,
// called when a context is created).
cudaError_t prepare_sweep_f32() {
    cudaError_t e = cudaFuncSetAttribute(sweep_kernel<float, false, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         sweep_smem_bytes<float, true>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(sweep_kernel<float, false, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             sweep_smem_bytes<float, false>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(sweep_kernel<float, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                sweep_smem_bytes<float, false>());
}

void launch_sweep_f32(const SweepArgs<float> &a, dim3 grid, dim3 block, cudaStream_t st) {
    if (a.confine_r > 0.0)
        sweep_kernel<float, false, false, true><<<grid, block, sweep_smem_bytes<float, false>(), st>>>(a);
    else if (a.vec_x)
        sweep_kernel<float, false, true><<<grid, block, sweep_smem_bytes<float, true>(), st>>>(a);
    else
        sweep_kernel<float, false, false><<<grid, block, sweep_smem_bytes<float, false>(), st>>>(a);
}
}  // namespace ppm
