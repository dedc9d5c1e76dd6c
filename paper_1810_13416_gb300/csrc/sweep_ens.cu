// Ensemble passes: the fused pass body over a work list of many boxes.
// FP32 variants: 64- and 128-thread blocks (scalar loads), 128-thread blocks
// with the x-pass vector path; FP64: 128-thread blocks.  Compiled with
// approximate FP32 division and square root like the single-grid FP32 pass.
#include "sweep.cuh"

namespace ppm {

template <bool VEC, int NB>
static cudaError_t set_smem_f32() {
    cudaError_t e = cudaFuncSetAttribute(sweep_ensemble_kernel<float, false, VEC, NB, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, sweep_smem_bytes<float, VEC, NB>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(sweep_ensemble_kernel<float, false, VEC, NB, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, sweep_smem_bytes<float, VEC, NB>());
}

cudaError_t prepare_sweep_ensemble() {
    cudaError_t e;
    if ((e = set_smem_f32<false, 32>()) != cudaSuccess) return e;
    if ((e = set_smem_f32<false, 64>()) != cudaSuccess) return e;
    if ((e = set_smem_f32<false, 128>()) != cudaSuccess) return e;
    if ((e = set_smem_f32<true, 32>()) != cudaSuccess) return e;
    if ((e = set_smem_f32<true, 64>()) != cudaSuccess) return e;
    if ((e = set_smem_f32<true, 128>()) != cudaSuccess) return e;
    return cudaFuncSetAttribute(sweep_ensemble_kernel<double, true, false, 128>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, sweep_smem_bytes<double, false, 128>());
}

// Resident blocks per SM of a variant (for sizing a persistent grid).
template <bool VEC, int NB>
static int bps_f32() {
    int nblk = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nblk, sweep_ensemble_kernel<float, false, VEC, NB, false>, NB,
                                                  sweep_smem_bytes<float, VEC, NB>());
    return nblk;
}
int ensemble_blocks_per_sm(int f32, int vec, int nb) {
    int nblk = 0;
    if (!f32)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nblk, sweep_ensemble_kernel<double, true, false, 128>, 128,
                                                      sweep_smem_bytes<double, false, 128>());
    else if (vec)
        nblk = (nb == 32) ? bps_f32<true, 32>() : (nb == 64) ? bps_f32<true, 64>() : bps_f32<true, 128>();
    else
        nblk = (nb == 32) ? bps_f32<false, 32>() : (nb == 64) ? bps_f32<false, 64>() : bps_f32<false, 128>();
    return nblk > 0 ? nblk : 1;
}

// nsrc: no box of this pass has sources or the CFL maximum (the
// instantiation without that code; four of the six passes of a step)
template <bool VEC, int NB>
static void launch_f32(bool nsrc, const void *args, const WorkItem *work, int nwork, int *counter, int persistent,
                       int grid, cudaStream_t st) {
    const SweepArgs<float> *a = static_cast<const SweepArgs<float> *>(args);
    if (nsrc)
        sweep_ensemble_kernel<float, false, VEC, NB, true><<<grid, NB, sweep_smem_bytes<float, VEC, NB>(), st>>>(
            a, work, nwork, counter, persistent);
    else
        sweep_ensemble_kernel<float, false, VEC, NB, false><<<grid, NB, sweep_smem_bytes<float, VEC, NB>(), st>>>(
            a, work, nwork, counter, persistent);
}

void launch_sweep_ensemble(int f32, int vec, int nb, int nsrc, const void *args, const WorkItem *work, int nwork,
                           int *counter, int persistent, int grid, cudaStream_t st) {
    if (!f32) {
        sweep_ensemble_kernel<double, true, false, 128><<<grid, 128, sweep_smem_bytes<double, false, 128>(), st>>>(
            static_cast<const SweepArgs<double> *>(args), work, nwork, counter, persistent);
    } else if (vec) {
        if (nb == 32) launch_f32<true, 32>(nsrc != 0, args, work, nwork, counter, persistent, grid, st);
        else if (nb == 64) launch_f32<true, 64>(nsrc != 0, args, work, nwork, counter, persistent, grid, st);
        else launch_f32<true, 128>(nsrc != 0, args, work, nwork, counter, persistent, grid, st);
    } else if (nb == 32) {
        launch_f32<false, 32>(nsrc != 0, args, work, nwork, counter, persistent, grid, st);
    } else if (nb == 64) {
        launch_f32<false, 64>(nsrc != 0, args, work, nwork, counter, persistent, grid, st);
    } else {
        launch_f32<false, 128>(nsrc != 0, args, work, nwork, counter, persistent, grid, st);
    }
}

// The whole-step kernel (one launch per double step): shared memory for
// either copy path of its items.
template <typename R, bool PLAIN>
constexpr int step_smem_bytes() {
    return PLAIN ? sweep_smem_bytes<R, false, 128>()
                 : (sweep_smem_bytes<R, true, 128>() > sweep_smem_bytes<R, false, 128>() ? sweep_smem_bytes<R, true, 128>()
                                                                                       : sweep_smem_bytes<R, false, 128>());
}

cudaError_t prepare_ensemble_step() {
    cudaError_t e = cudaFuncSetAttribute(sweep_ensemble_step_kernel<float, false, 128>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, step_smem_bytes<float, false>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(sweep_ensemble_step_kernel<double, true, 128>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, step_smem_bytes<double, true>());
}

int ensemble_step_blocks_per_sm(int f32) {
    int nblk = 0;
    if (f32)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nblk, sweep_ensemble_step_kernel<float, false, 128>, 128,
                                                      step_smem_bytes<float, false>());
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nblk, sweep_ensemble_step_kernel<double, true, 128>, 128,
                                                      step_smem_bytes<double, true>());
    return nblk > 0 ? nblk : 1;
}

void launch_ensemble_step(int f32, const void *args, int nbox, const WorkItem *work, int nwork, int *ticket,
                          int *done, const int *need, int wait_test, int grid, cudaStream_t st) {
    if (f32)
        sweep_ensemble_step_kernel<float, false, 128><<<grid, 128, step_smem_bytes<float, false>(), st>>>(
            static_cast<const SweepArgs<float> *>(args), nbox, work, nwork, ticket, done, need, wait_test);
    else
        sweep_ensemble_step_kernel<double, true, 128><<<grid, 128, step_smem_bytes<double, true>(), st>>>(
            static_cast<const SweepArgs<double> *>(args), nbox, work, nwork, ticket, done, need, wait_test);
}

}  // namespace ppm
