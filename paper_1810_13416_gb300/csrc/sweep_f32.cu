// FP32 base-state-deviation form of the fused pass (approximate division
// and square root: this unit is compiled with -prec-div=false -prec-sqrt=false).
#include "sweep.cuh"

namespace ppm {
constexpr int TEN_VEC_NB = 64;
// Raise the dynamic shared-memory limit of every variant (once per device,
// called when a context is created).
cudaError_t prepare_sweep_f32() {
    cudaError_t e = cudaFuncSetAttribute(sweep_kernel<float, false, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         sweep_smem_bytes<float, true>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(sweep_kernel<float, false, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             sweep_smem_bytes<float, false>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(sweep_kernel<float, false, false, false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, sweep_smem_bytes<float, false, SWEEP_NB, 15>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(sweep_kernel<float, false, false, false, false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, sweep_smem_bytes<float, false>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(sweep_kernel<float, false, true, false, false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, sweep_smem_bytes<float, true>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(sweep_kernel<float, false, true, false, true, false, TEN_VEC_NB>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, sweep_smem_bytes<float, true, TEN_VEC_NB, 15>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(sweep_kernel<float, false, false, false, false, false, SWEEP_NB, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, sweep_smem_bytes<float, false>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(sweep_kernel<float, false, true, false, false, false, SWEEP_NB, false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, sweep_smem_bytes<float, true>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(sweep_kernel<float, false, false, false, false, false, SWEEP_NB, false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, sweep_smem_bytes<float, false>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(sweep_kernel<float, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                sweep_smem_bytes<float, false>());
}

void launch_sweep_f32(const SweepArgs<float> &a, dim3 grid, dim3 block, cudaStream_t st) {
    if (a.halo_lo || a.halo_hi) {
        // z pass of a slab with halo planes (no other feature combines with it)
        sweep_kernel<float, false, false, false, false, false, SWEEP_NB, true>
            <<<grid, block, sweep_smem_bytes<float, false>(), st>>>(a);
    } else if (a.divg) {
        if (a.vec_x)
            sweep_kernel<float, false, true, false, false, true><<<grid, block, sweep_smem_bytes<float, true>(), st>>>(a);
        else
            sweep_kernel<float, false, false, false, false, true><<<grid, block, sweep_smem_bytes<float, false>(), st>>>(a);
    } else if (a.ten && a.vec_x) {
        // 64-thread blocks: three fit with their 15-value 16-byte rings
        const dim3 g((a.nlane + TEN_VEC_NB - 1) / TEN_VEC_NB, a.nblk);
        sweep_kernel<float, false, true, false, true, false, TEN_VEC_NB>
            <<<g, dim3(TEN_VEC_NB), sweep_smem_bytes<float, true, TEN_VEC_NB, 15>(), st>>>(a);
    } else if (a.ten)
        sweep_kernel<float, false, false, false, true>
            <<<grid, block, sweep_smem_bytes<float, false, SWEEP_NB, 15>(), st>>>(a);
    else if (a.confine_r > 0.0)
        sweep_kernel<float, false, false, true><<<grid, block, sweep_smem_bytes<float, false>(), st>>>(a);
    // passes without sources and CFL maximum: their own instantiation
    // (measured 1.6% faster than the shared one)
    else if (a.vec_x && !a.sources && !a.cfl)
        sweep_kernel<float, false, true, false, false, false, SWEEP_NB, false, true>
            <<<grid, block, sweep_smem_bytes<float, true>(), st>>>(a);
    else if (!a.vec_x && !a.sources && !a.cfl)
        sweep_kernel<float, false, false, false, false, false, SWEEP_NB, false, true>
            <<<grid, block, sweep_smem_bytes<float, false>(), st>>>(a);
    else if (a.vec_x)
        sweep_kernel<float, false, true><<<grid, block, sweep_smem_bytes<float, true>(), st>>>(a);
    else
        sweep_kernel<float, false, false><<<grid, block, sweep_smem_bytes<float, false>(), st>>>(a);
}
}  // namespace ppm
