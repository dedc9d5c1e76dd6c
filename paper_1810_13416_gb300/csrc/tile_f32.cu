// tile_f32.cu -- the cell-parallel tile form of the FP32 pass (tile.cuh),
// compiled with the FP32 pass flags (approximate division and square root,
// denormals flushed to zero), and the TMA tensor maps it reads and writes.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "tile.cuh"

namespace ppm {

cudaError_t prepare_tile_f32() {
    const int sm = (int)tile::SMEM_BYTES;
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(tile::tile_pass_kernel<0, true>, at, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(tile::tile_pass_kernel<1, true>, at, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(tile::tile_pass_kernel<2, true>, at, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(tile::tile_pass_kernel<0, false>, at, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(tile::tile_pass_kernel<1, false>, at, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(tile::tile_pass_kernel<2, false>, at, sm);
    return e;
}

size_t tile_smem_bytes() { return tile::SMEM_BYTES; }

// Tensor map of the FP32 state (9 arrays of nx*ny*nz floats, x fastest) with
// the box of one chunk of the pass along `axis`: 32 x 8 rows (x pass, 128-byte
// swizzle) or 8 x-columns x 32 cells (y, z).  0 on success, else a CUresult
// (or -1 when the driver entry point is missing).
int tile_encode_map(CUtensorMap *m, void *state, int nx, int ny, int nz, int axis) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return -1;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const cuuint64_t ncell = (cuuint64_t)nx * ny * nz;
    const cuuint64_t dims[4] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz, 9};
    const cuuint64_t strides[3] = {(cuuint64_t)nx * 4, (cuuint64_t)nx * ny * 4, ncell * 4};
    cuuint32_t box[4] = {(cuuint32_t)tile::P, 1, 1, 9};
    if (axis == 0) {
        box[0] = tile::S;
        box[1] = tile::P;
    } else if (axis == 1) {
        box[1] = tile::S;
    } else {
        box[2] = tile::S;
    }
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, state, dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE,
                              axis == 0 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return (int)r;
}

void launch_tile_f32(const SweepArgs<float> &a, const CUtensorMap *m, cudaStream_t st) {
    const dim3 grid((a.nlane + tile::P - 1) / tile::P, a.nblk);
    const bool full = a.sources || a.cfl;   // else the instantiation without that code
    if (a.axis == 0) {
        if (full) tile::tile_pass_kernel<0, true><<<grid, tile::NT, tile::SMEM_BYTES, st>>>(a, *m);
        else tile::tile_pass_kernel<0, false><<<grid, tile::NT, tile::SMEM_BYTES, st>>>(a, *m);
    } else if (a.axis == 1) {
        if (full) tile::tile_pass_kernel<1, true><<<grid, tile::NT, tile::SMEM_BYTES, st>>>(a, *m);
        else tile::tile_pass_kernel<1, false><<<grid, tile::NT, tile::SMEM_BYTES, st>>>(a, *m);
    } else {
        if (full) tile::tile_pass_kernel<2, true><<<grid, tile::NT, tile::SMEM_BYTES, st>>>(a, *m);
        else tile::tile_pass_kernel<2, false><<<grid, tile::NT, tile::SMEM_BYTES, st>>>(a, *m);
    }
}

}  // namespace ppm
