// noalloc.cu -- conserved totals of a caller-owned state without any device
// allocation.
//
// Some callers cannot let a library call cudaMalloc: a host code whose own
// pool allocator owns all device memory and budgets it in advance (a 1024^3
// FP64 state already takes 77 GB), or a time-step loop that cannot afford the
// device-wide synchronisation an allocation may cause.  ppm_totals_noalloc
// serves them: it reads nine FP64 arrays the caller already holds on the
// device, writes seven doubles the caller provides, and keeps its partial
// sums in the fixed static array below, which every GPU that loads this
// library holds until the process exits.
#include <cuda_runtime.h>

#include <cstdio>

#include "../../include/ppm.h"

namespace ppm {
void set_global_error(const char *msg);
}

namespace {

constexpr int NOALLOC_MAX_PLANES = PPM_NOALLOC_MAX_PLANES;
constexpr int NOALLOC_THREADS = 256;

// One row of 8 doubles per z-plane: the plane's 7 partial totals (+1 pad).
// Shared by every call on a device; the last call's contents stay behind.
static __device__ __align__(256) double g_plane_sums[NOALLOC_MAX_PLANES * 8];

// The nine state pointers, passed by value as a kernel argument.
struct StatePtrs {
    const double *q[9];
};

// Sums of one z-plane: (rho, rho*u, rho*v, rho*w, E, rho*FV, FV).
__global__ void plane_sums_kernel(const StatePtrs S, long long plane, double *sums) {
    const double *const *q = S.q;
    __shared__ double red[7][NOALLOC_THREADS / 32];
    const long long base = (long long)blockIdx.x * plane;
    double t[7] = {0, 0, 0, 0, 0, 0, 0};
    for (long long i = threadIdx.x; i < plane; i += blockDim.x) {
        const long long c = base + i;
        const double rho = q[0][c];
        t[0] += rho;
        t[1] += q[1][c];
        t[2] += q[2][c];
        t[3] += q[3][c];
        t[4] += q[4][c];
        t[5] += rho * q[5][c];
        t[6] += q[5][c];
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int m = 0; m < 7; ++m) {
        double v = t[m];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (l == 0) red[m][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < 7) {
        double v = 0.0;
        for (int k = 0; k < NOALLOC_THREADS / 32; ++k) v += red[threadIdx.x][k];
        sums[(long long)blockIdx.x * 8 + threadIdx.x] = v;   // written, never accumulated
    }
}

// Planes summed in order, so the result does not depend on scheduling.
__global__ void total_kernel(const double *sums, int nz, double dV, double *out) {
    const int m = threadIdx.x;
    if (m < 7) {
        double v = 0.0;
        for (int k = 0; k < nz; ++k) v += sums[(long long)k * 8 + m];
        out[m] = v * dV;
    }
}

// Device address of the static array in the current device's context.  It
// is looked up on every call (the lookup allocates nothing and queues no
// work), so a device reset or a new context on the same ordinal never leaves
// a stale address behind.
int scratch_for_current_device(double **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_plane_sums);
    if (e != cudaSuccess) {
        char msg[256];
        snprintf(msg, sizeof(msg), "ppm_totals_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        ppm::set_global_error(msg);
        return PPM_ECUDA;
    }
    *out = static_cast<double *>(p);
    return PPM_OK;
}

int launch_failed(const char *which) {
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) return PPM_OK;
    char msg[256];
    snprintf(msg, sizeof(msg), "ppm_totals_noalloc: launch of %s: %s", which, cudaGetErrorString(e));
    ppm::set_global_error(msg);
    return PPM_ECUDA;
}

}  // namespace

extern "C" int ppm_totals_noalloc(const double *const *q_dev, int nx, int ny, int nz, double dx,
                                  double *totals_dev, void *stream) {
    if (!q_dev || !totals_dev) {
        ppm::set_global_error("ppm_totals_noalloc: null pointer argument");
        return PPM_EINVAL;
    }
    for (int v = 0; v < 9; ++v)
        if (!q_dev[v]) {
            ppm::set_global_error("ppm_totals_noalloc: a state pointer is NULL");
            return PPM_EINVAL;
        }
    if (nx < 1 || ny < 1 || nz < 1 || !(dx > 0.0)) {
        ppm::set_global_error("ppm_totals_noalloc: extents must be >= 1 and dx > 0");
        return PPM_EINVAL;
    }
    if (nz > NOALLOC_MAX_PLANES) {
        char msg[160];
        snprintf(msg, sizeof(msg), "ppm_totals_noalloc: nz = %d exceeds the fixed scratch of %d z-planes",
                 nz, NOALLOC_MAX_PLANES);
        ppm::set_global_error(msg);
        return PPM_EINVAL;
    }
    {
        // an error left behind by earlier, unrelated work is reported as such
        // and not cleared, so that its owner can still see it
        const cudaError_t pe = cudaPeekAtLastError();
        if (pe != cudaSuccess) {
            char msg[256];
            snprintf(msg, sizeof(msg), "ppm_totals_noalloc: an earlier CUDA error is pending: %s",
                     cudaGetErrorString(pe));
            ppm::set_global_error(msg);
            return PPM_ECUDA;
        }
    }
    double *scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc != PPM_OK) return rc;
    StatePtrs S;
    for (int v = 0; v < 9; ++v) S.q[v] = q_dev[v];
    cudaStream_t st = (cudaStream_t)stream;
    const long long plane = (long long)nx * ny;
    plane_sums_kernel<<<nz, NOALLOC_THREADS, 0, st>>>(S, plane, scratch);
    if ((rc = launch_failed("plane_sums_kernel")) != PPM_OK) return rc;
    total_kernel<<<1, 32, 0, st>>>(scratch, nz, dx * dx * dx, totals_dev);
    if ((rc = launch_failed("total_kernel")) != PPM_OK) return rc;
    return PPM_OK;
}
