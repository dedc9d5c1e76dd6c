// FP32 base-state-deviation form of the fused pass (approximate division
// and square root: this unit is compiled with -prec-div=false -prec-sqrt=false).
#include "sweep.cuh"

namespace ppm {
constexpr int TEN_VEC_NB = 64;

// Every feature instantiation comes twice: for passes with sources or the
// CFL maximum, and without that code (NSRC) for the others (four of the six
// passes of a step; measured 1.6% faster on the plain pass).
template <bool VEC, bool CONF, bool TEN, bool DISS, int NB, bool HALO = false>
static cudaError_t set_smem(int bytes) {
    cudaError_t e = cudaFuncSetAttribute(sweep_kernel<float, false, VEC, CONF, TEN, DISS, NB, HALO, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(sweep_kernel<float, false, VEC, CONF, TEN, DISS, NB, HALO, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}
template <bool VEC, bool CONF, bool TEN, bool DISS, int NB, bool HALO = false>
static void launch_one(const SweepArgs<float> &a, dim3 grid, dim3 block, int bytes, cudaStream_t st) {
    if (a.sources || a.cfl)
        sweep_kernel<float, false, VEC, CONF, TEN, DISS, NB, HALO, false><<<grid, block, bytes, st>>>(a);
    else
        sweep_kernel<float, false, VEC, CONF, TEN, DISS, NB, HALO, true><<<grid, block, bytes, st>>>(a);
}

// Raise the dynamic shared-memory limit of every variant (once per device,
// called when a context is created).
cudaError_t prepare_sweep_f32() {
    cudaError_t e;
    if ((e = set_smem<true, false, false, false, SWEEP_NB>(sweep_smem_bytes<float, true>())) != cudaSuccess) return e;
    if ((e = set_smem<false, false, false, false, SWEEP_NB>(sweep_smem_bytes<float, false>())) != cudaSuccess) return e;
    if ((e = set_smem<false, true, false, false, SWEEP_NB>(sweep_smem_bytes<float, false>())) != cudaSuccess) return e;
    if ((e = set_smem<false, false, true, false, SWEEP_NB>(sweep_smem_bytes<float, false, SWEEP_NB, 15>())) !=
        cudaSuccess)
        return e;
    if ((e = set_smem<true, false, true, false, TEN_VEC_NB>(sweep_smem_bytes<float, true, TEN_VEC_NB, 15>())) !=
        cudaSuccess)
        return e;
    if ((e = set_smem<false, false, false, true, SWEEP_NB>(sweep_smem_bytes<float, false>())) != cudaSuccess) return e;
    if ((e = set_smem<true, false, false, true, SWEEP_NB>(sweep_smem_bytes<float, true>())) != cudaSuccess) return e;
    return cudaFuncSetAttribute(sweep_kernel<float, false, false, false, false, false, SWEEP_NB, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, sweep_smem_bytes<float, false>());
}

void launch_sweep_f32(const SweepArgs<float> &a, dim3 grid, dim3 block, cudaStream_t st) {
    if (a.halo_lo || a.halo_hi) {
        // z pass of a slab with halo planes (no other feature combines with it)
        sweep_kernel<float, false, false, false, false, false, SWEEP_NB, true>
            <<<grid, block, sweep_smem_bytes<float, false>(), st>>>(a);
    } else if (a.divg) {
        if (a.vec_x)
            launch_one<true, false, false, true, SWEEP_NB>(a, grid, block, sweep_smem_bytes<float, true>(), st);
        else
            launch_one<false, false, false, true, SWEEP_NB>(a, grid, block, sweep_smem_bytes<float, false>(), st);
    } else if (a.ten && a.vec_x) {
        // 64-thread blocks: three fit with their 15-value 16-byte rings
        const dim3 g((a.nlane + TEN_VEC_NB - 1) / TEN_VEC_NB, a.nblk);
        launch_one<true, false, true, false, TEN_VEC_NB>(a, g, dim3(TEN_VEC_NB),
                                                         sweep_smem_bytes<float, true, TEN_VEC_NB, 15>(), st);
    } else if (a.ten)
        launch_one<false, false, true, false, SWEEP_NB>(a, grid, block, sweep_smem_bytes<float, false, SWEEP_NB, 15>(),
                                                        st);
    else if (a.confine_r > 0.0)
        launch_one<false, true, false, false, SWEEP_NB>(a, grid, block, sweep_smem_bytes<float, false>(), st);
    else if (a.vec_x)
        launch_one<true, false, false, false, SWEEP_NB>(a, grid, block, sweep_smem_bytes<float, true>(), st);
    else
        launch_one<false, false, false, false, SWEEP_NB>(a, grid, block, sweep_smem_bytes<float, false>(), st);
}
}  // namespace ppm
