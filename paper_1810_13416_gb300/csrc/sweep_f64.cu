// FP64 plain form of the fused pass (full rho and E in storage).
#include "sweep.cuh"

namespace ppm {
cudaError_t prepare_sweep_f64() {
    cudaError_t e = cudaFuncSetAttribute(sweep_kernel<double, true, false, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         sweep_smem_bytes<double, false>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(sweep_kernel<double, true, false, false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, sweep_smem_bytes<double, false, SWEEP_NB, 15>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(sweep_kernel<double, true, false, false, false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, sweep_smem_bytes<double, false>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(sweep_kernel<double, true, false, false, false, false, SWEEP_NB, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, sweep_smem_bytes<double, false>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(sweep_kernel<double, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                sweep_smem_bytes<double, false>());
}

void launch_sweep_f64(const SweepArgs<double> &a, dim3 grid, dim3 block, cudaStream_t st) {
    if (a.halo_lo || a.halo_hi)
        sweep_kernel<double, true, false, false, false, false, SWEEP_NB, true>
            <<<grid, block, sweep_smem_bytes<double, false>(), st>>>(a);
    else if (a.divg)
        sweep_kernel<double, true, false, false, false, true><<<grid, block, sweep_smem_bytes<double, false>(), st>>>(a);
    else if (a.ten)
        sweep_kernel<double, true, false, false, true>
            <<<grid, block, sweep_smem_bytes<double, false, SWEEP_NB, 15>(), st>>>(a);
    else if (a.confine_r > 0.0)
        sweep_kernel<double, true, false, true><<<grid, block, sweep_smem_bytes<double, false>(), st>>>(a);
    else
        sweep_kernel<double, true, false><<<grid, block, sweep_smem_bytes<double, false>(), st>>>(a);
}
}  // namespace ppm
