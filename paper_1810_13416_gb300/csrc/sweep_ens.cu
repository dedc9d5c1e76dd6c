// Ensemble passes: the fused pass body over a work list of many boxes.
// FP32 variants: 64- and 128-thread blocks (scalar loads), 128-thread blocks
// with the x-pass vector path; FP64: 128-thread blocks.  Compiled with
// approximate FP32 division and square root like the single-grid FP32 pass.
#include "sweep.cuh"

namespace ppm {

cudaError_t prepare_sweep_ensemble() {
    cudaError_t e;
    e = cudaFuncSetAttribute(sweep_ensemble_kernel<float, false, false, 64>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, sweep_smem_bytes<float, false, 64>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(sweep_ensemble_kernel<float, false, false, 128>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, sweep_smem_bytes<float, false, 128>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(sweep_ensemble_kernel<float, false, true, 128>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, sweep_smem_bytes<float, true, 128>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(sweep_ensemble_kernel<double, true, false, 128>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, sweep_smem_bytes<double, false, 128>());
}

// Resident blocks per SM of a variant (for sizing a persistent grid).
int ensemble_blocks_per_sm(int f32, int vec, int nb) {
    int nblk = 0;
    if (!f32)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nblk, sweep_ensemble_kernel<double, true, false, 128>, 128,
                                                      sweep_smem_bytes<double, false, 128>());
    else if (vec)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nblk, sweep_ensemble_kernel<float, false, true, 128>, 128,
                                                      sweep_smem_bytes<float, true, 128>());
    else if (nb == 64)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nblk, sweep_ensemble_kernel<float, false, false, 64>, 64,
                                                      sweep_smem_bytes<float, false, 64>());
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nblk, sweep_ensemble_kernel<float, false, false, 128>, 128,
                                                      sweep_smem_bytes<float, false, 128>());
    return nblk > 0 ? nblk : 1;
}

void launch_sweep_ensemble(int f32, int vec, int nb, const void *args, const WorkItem *work, int nwork,
                           int *counter, int persistent, int grid, cudaStream_t st) {
    if (!f32) {
        sweep_ensemble_kernel<double, true, false, 128><<<grid, 128, sweep_smem_bytes<double, false, 128>(), st>>>(
            static_cast<const SweepArgs<double> *>(args), work, nwork, counter, persistent);
    } else if (vec) {
        sweep_ensemble_kernel<float, false, true, 128><<<grid, 128, sweep_smem_bytes<float, true, 128>(), st>>>(
            static_cast<const SweepArgs<float> *>(args), work, nwork, counter, persistent);
    } else if (nb == 64) {
        sweep_ensemble_kernel<float, false, false, 64><<<grid, 64, sweep_smem_bytes<float, false, 64>(), st>>>(
            static_cast<const SweepArgs<float> *>(args), work, nwork, counter, persistent);
    } else {
        sweep_ensemble_kernel<float, false, false, 128><<<grid, 128, sweep_smem_bytes<float, false, 128>(), st>>>(
            static_cast<const SweepArgs<float> *>(args), work, nwork, counter, persistent);
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
