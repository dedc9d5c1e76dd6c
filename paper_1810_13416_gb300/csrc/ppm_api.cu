// ppm_api.cu -- the C ABI of libppm.so (include/ppm.h): context, state
// conversion, CFL and diagnostic reductions, and the CUDA-graph double step.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ppm.h"
#include "sweep.cuh"

namespace ppm {
void launch_sweep_f32(const SweepArgs<float> &a, dim3 grid, dim3 block, cudaStream_t st);
void launch_sweep_f64(const SweepArgs<double> &a, dim3 grid, dim3 block, cudaStream_t st);
cudaError_t prepare_sweep_f32();
cudaError_t prepare_sweep_f64();
cudaError_t prepare_sweep_ensemble();
int ensemble_blocks_per_sm(int f32, int vec, int nb);
void launch_sweep_ensemble(int f32, int vec, int nb, int nsrc, const void *args, const WorkItem *work, int nwork,
                           int *counter, int persistent, int grid, cudaStream_t st);
cudaError_t prepare_tile_f32();
cudaError_t prepare_ensemble_step();
int ensemble_step_blocks_per_sm(int f32);
void launch_ensemble_step(int f32, const void *args, int nbox, const WorkItem *work, int nwork, int *ticket,
                          int *done, const int *need, int wait_test, int grid, cudaStream_t st);
int tile_encode_map(CUtensorMap *m, void *state, int nx, int ny, int nz, int axis);
void launch_tile_f32(const SweepArgs<float> &a, const CUtensorMap *m, cudaStream_t st);
}  // namespace ppm

using namespace ppm;

namespace {

constexpr int NVAR_MAX = 15;   // with the ten-value PPB
constexpr int SWEEP_BLOCK = ppm::SWEEP_NB;
constexpr int MAX_BINS = 1024;

// Device scalars shared by the kernels of one context.
struct DevScal {
    double dt;                 // time step used by the passes
    double dt_user;            // > 0: explicit dt for the next step
    unsigned long long smax;   // bits of the running max of (max_d|u_d| + c)
    double cfl;                // CFL number for the device dt
    int flags;                 // FLAG_NONPHYS ...
    int pad;
};

thread_local std::string g_create_error;

}  // namespace

namespace ppm {
// Message for calls that have no context (read back by ppm_last_error(NULL)).
void set_global_error(const char *msg) { g_create_error = msg; }
}  // namespace ppm

struct ppm_ctx {
    int n[3];
    long long ncell;
    double gamma;
    int bc[6];
    int grav;
    int prec;
    double org[3], dx;
    int ntab;
    double s0, ds;
    double rho0c, p0c;         // uniform base (no gravity)
    double confine_r;          // > 0: confining sphere about the coordinate origin
    double domega;             // rotation increment per double step (0 = none)
    int nmom;                  // FV moments carried: 3 or 9 (ten-value PPB)
    int nvar;                  // stored values per cell: 6 + nmom
    double shock_k;            // 3-D shock dissipation coefficient (0 = off)
    long long graph_kernels;   // kernels in the step graph
    void *divg;                // its per-pass cell divergence (ncell values)
    void *vel;                 // FP32: the cell velocities the y/z passes of a step leave (3 x ncell)
    int has_heat, has_damp;
    int device;
    cudaStream_t stream;
    bool own_stream;
    void *state;               // 9 * ncell values (float or double)
    double *t64;               // FP64 tables: rho0, p0, g, heat, damp (5 * ntab)
    float *t32;                // FP32 copies
    float4 *t4;                // FP32 AoS tables for the passes: base[ntab4], sources[ntab4]
    int ntab4;
    float s4_0, inv_ds4;
    DevScal *ds_dev;
    double *stage;             // FP64 staging for host regions (two buffers)
    cudaStream_t xstream;      // host-region copies (created on first use)
    cudaEvent_t ev_copy[2], ev_kern[2];
    long long stage_cells;
    double *diag_acc;          // diagnostics accumulators
    float *base32;             // FP32 form, made by the first diagnostics call (NULL: not yet, or
                               // no memory for it): per cell rho0 as two floats hi + lo, and p0
    bool base32_tried;
    double base_sum[2];        // FP64 grid sums of rho0 and p0/(gamma-1) (with base32)
    cudaGraph_t graph;
    cudaGraphExec_t gexec;
    cudaGraphNode_t dt_node;   // first node of the step graph (dt_kernel)
    cudaEvent_t pev[7];        // recorded inside the step graph around its six passes
    bool have_speed;           // a valid device max speed exists for dt <= 0
    long long launches;
    int design[3];             // per pass axis: PPM_PASS_MARCH or PPM_PASS_TILE
    int halo_z;                // bit 0 / bit 1: the low / high z face takes halo planes
    int z_index0;              // global index of plane 0 (slab of a larger grid)
    void *halo[2];             // their buffers: nvar x 4 planes each, storage format
    bool tile_ok;              // the tile form applies to this context
    CUtensorMap tmap[3];       // its TMA maps of the state, one box shape per pass axis
    std::string err;
};

namespace {

int fail(ppm_ctx *c, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c)
        c->err = buf;
    else
        g_create_error = buf;
    return code;
}

#define CK(ctx, call)                                                                          \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail((ctx), PPM_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),      \
                        __FILE__, __LINE__);                                                   \
    } while (0)

// ---------------------------------------------------------------------------
// Argument structs for the passes
// ---------------------------------------------------------------------------
template <typename R>
SweepArgs<R> make_args(ppm_ctx *c, int axis) {
    SweepArgs<R> a;
    memset(&a, 0, sizeof(a));
    const int nx = c->n[0], ny = c->n[1], nz = c->n[2];
    a.q = static_cast<R *>(c->state);
    a.vs = c->ncell;
    a.axis = axis;
    a.n = c->n[axis];
    const long long sx = 1, sy = nx, sz = (long long)nx * ny;
    if (axis == 0) {  // pencils along x: lanes over y, blocks over z
        a.s_axis = sx; a.nlane = ny; a.s_lane = sy; a.lane_dim = 1; a.nblk = nz; a.s_blk = sz; a.blk_dim = 2;
    } else if (axis == 1) {  // along y: lanes over x, blocks over z
        a.s_axis = sy; a.nlane = nx; a.s_lane = sx; a.lane_dim = 0; a.nblk = nz; a.s_blk = sz; a.blk_dim = 2;
    } else {  // along z: lanes over x, blocks over y
        a.s_axis = sz; a.nlane = nx; a.s_lane = sx; a.lane_dim = 0; a.nblk = ny; a.s_blk = sy; a.blk_dim = 1;
    }
    a.bc_lo = c->bc[2 * axis];
    a.bc_hi = c->bc[2 * axis + 1];
    if (axis == 2 && c->halo_z) {
        const long long plane = (long long)nx * ny;
        a.halo_vs = 4 * plane;
        if (c->halo_z & 1) {
            a.bc_lo = BC_HALO;
            a.halo_lo = static_cast<const R *>(c->halo[0]);
        }
        if (c->halo_z & 2) {
            a.bc_hi = BC_HALO;
            a.halo_hi = static_cast<const R *>(c->halo[1]);
        }
    }
    a.grav = c->grav;
    for (int d = 0; d < 3; ++d) a.org[d] = c->org[d];
    a.ioff[0] = a.ioff[1] = 0;
    a.ioff[2] = c->z_index0;
    a.dx = c->dx;
    const R *t = std::is_same<R, float>::value ? (const R *)c->t32 : (const R *)c->t64;
    a.t_rho0 = t;
    a.t_p0 = t + c->ntab;
    a.t_g = t + 2 * c->ntab;
    a.t_heat = c->has_heat ? t + 3 * c->ntab : nullptr;
    a.t_damp = c->has_damp ? t + 4 * c->ntab : nullptr;
    a.ntab = c->ntab;
    a.t4_base = c->t4;
    a.t4_src = c->t4 + c->ntab4;
    a.ntab4 = c->ntab4;
    a.s4_0 = c->s4_0;
    a.inv_ds4 = c->inv_ds4;
    a.confine_r = c->confine_r;
    a.ten = (c->nmom == 9) ? 1 : 0;
    a.divg = static_cast<const R *>(c->divg);
    a.shock_k = c->shock_k;
    a.vec_x = (std::is_same<R, float>::value && axis == 0 && (c->n[0] % 8) == 0 && !(c->confine_r > 0.0)) ? 1 : 0;
    a.rho0_c = (R)c->rho0c;
    a.p0_c = (R)c->p0c;
    a.s0 = c->s0;
    a.ds = c->ds;
    a.gamma = c->gamma;
    a.dt = &c->ds_dev->dt;
    a.smax = &c->ds_dev->smax;
    a.flags = &c->ds_dev->flags;
    return a;
}

int launch_divergence(ppm_ctx *c, bool from_vel);

// vel: (shock dissipation, FP32) 1 = this pass leaves the cell velocities
// for the next pass's divergence, 2 = its divergence takes them from the pass
// before, 3 = both (a step's passes Y Z Z Y write, Z Z Y X read); 0 for a
// single pass
int launch_sweep(ppm_ctx *c, int axis, int sources, int cfl, int vel) {
    if (c->divg) {
        const int r = launch_divergence(c, (vel & 2) && c->vel);
        if (r != PPM_OK) return r;
    }
    dim3 block(SWEEP_BLOCK);
    if (c->prec == PPM_FP32_DEVIATION) {
        SweepArgs<float> a = make_args<float>(c, axis);
        a.sources = sources;
        a.cfl = cfl;
        if ((vel & 1) && c->vel && !a.vec_x) a.vel_out = static_cast<float *>(c->vel);
        dim3 grid((a.nlane + SWEEP_BLOCK - 1) / SWEEP_BLOCK, a.nblk);
        if (c->design[axis] == PPM_PASS_TILE && c->tile_ok)
            launch_tile_f32(a, &c->tmap[axis], c->stream);
        else
            launch_sweep_f32(a, grid, block, c->stream);
    } else {
        SweepArgs<double> a = make_args<double>(c, axis);
        a.sources = sources;
        a.cfl = cfl;
        dim3 grid((a.nlane + SWEEP_BLOCK - 1) / SWEEP_BLOCK, a.nblk);
        launch_sweep_f64(a, grid, block, c->stream);
    }
    c->launches++;
    CK(c, cudaGetLastError());
    return PPM_OK;
}

// ---------------------------------------------------------------------------
// Small kernels
// ---------------------------------------------------------------------------
// dt for the next step: explicit value, or CFL * dx / (max speed of the state
// left by the previous step); then clear the running maximum.
__global__ void dt_kernel(DevScal *s, double dx, double dt_user) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const double smax = __longlong_as_double((long long)s->smax);
        s->dt = (dt_user > 0.0) ? dt_user : s->cfl * dx / smax;
        s->smax = 0ull;
    }
}

// Write one device scalar from a kernel argument (no host buffer involved).
__global__ void set_scalar_kernel(double *dst, double v) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *dst = v;
}

// Base state of a grid cell (FP64 tables, non-contracted as in the passes).
template <typename R>
__device__ __forceinline__ Base<R> cell_base(const SweepArgs<R> &A, int i, int j, int k) {
    R xyz[3] = {coord(A, 0, i), coord(A, 1, j), coord(A, 2, k)};
    return base_at(A, xyz);
}

// The per-variable arrays of a region transfer, passed by value.
struct RegionPtrs {
    double *p[NVAR_MAX];
};

// FP64 full variables (a (hi-lo) box, x fastest) -> internal state.
template <typename R, bool PLAIN>
__global__ void set_region_kernel(SweepArgs<double> A64, R *st, long long ncell, int nx, int ny,
                                  int lo0, int lo1, int lo2, int bx, int by, int bz,
                                  const RegionPtrs src, long long src_off, int nvar) {
    const long long nb = (long long)bx * by * bz;
    const double gm1 = A64.gamma - 1.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nb;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % bx), j = (int)((t / bx) % by), k = (int)(t / ((long long)bx * by));
        const int gi = lo0 + i, gj = lo1 + j, gk = lo2 + k;
        const long long cidx = ((long long)gk * ny + gj) * nx + gi;
        double v[NVAR_MAX];
        for (int q = 0; q < nvar; ++q) v[q] = src.p[q][src_off + t];
        if (!PLAIN) {
            const Base<double> b = cell_base(A64, gi, gj, gk);
            v[0] = xsub(v[0], b.rho0);
            v[4] = xsub(v[4], xdiv(b.p0, gm1));
            // FV in [0,1], stored folded; moments within the FP32 bound
            const double fv = fmin(fmax(v[5], 0.0), 1.0);
            const float s = (fv > 0.5) ? (float)(-fabs(fv - 1.0)) : (float)fv;
            const float bnd = fv_moment_bound(s);
            for (int q = 0; q < 5; ++q) st[q * ncell + cidx] = (R)v[q];
            st[5 * ncell + cidx] = (R)s;
            for (int q = 6; q < 9; ++q) st[q * ncell + cidx] = (R)fminf(fmaxf((float)v[q], -bnd), bnd);
            if (nvar > 9) {
                // second and mixed moments within their bounds (as the passes clamp)
                const float g = bnd * (1.0f / 6.0f), f = (float)fv;
                const float qlo = -15.0f * g * (1.0f + f), qhi = 15.0f * g * (2.0f - f), bc = 36.0f * g;
                for (int q = 9; q < 12; ++q) st[q * ncell + cidx] = (R)fminf(fmaxf((float)v[q], qlo), qhi);
                for (int q = 12; q < 15; ++q) st[q * ncell + cidx] = (R)fminf(fmaxf((float)v[q], -bc), bc);
            }
        } else {
            for (int q = 0; q < nvar; ++q) st[q * ncell + cidx] = (R)v[q];
        }
    }
}

template <typename R, bool PLAIN>
__global__ void get_region_kernel(SweepArgs<double> A64, const R *st, long long ncell, int nx, int ny,
                                  int lo0, int lo1, int lo2, int bx, int by, int bz,
                                  const RegionPtrs dst, long long dst_off, int nvar) {
    const long long nb = (long long)bx * by * bz;
    const double gm1 = A64.gamma - 1.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nb;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % bx), j = (int)((t / bx) % by), k = (int)(t / ((long long)bx * by));
        const int gi = lo0 + i, gj = lo1 + j, gk = lo2 + k;
        const long long cidx = ((long long)gk * ny + gj) * nx + gi;
        double v[NVAR_MAX];
        for (int q = 0; q < nvar; ++q) v[q] = (double)st[q * ncell + cidx];
        if (!PLAIN) {
            const Base<double> b = cell_base(A64, gi, gj, gk);
            v[0] = xadd(b.rho0, v[0]);
            v[4] = xadd(xdiv(b.p0, gm1), v[4]);
            v[5] = signbit(v[5]) ? 1.0 + v[5] : v[5];
        }
        for (int q = 0; q < nvar; ++q) dst.p[q][dst_off + t] = v[q];
    }
}

__device__ __forceinline__ void block_max_atomic(double v, unsigned long long *out) {
    __shared__ double sm[32];
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sm[w] = v;
    __syncthreads();
    if (w == 0) {
        v = (l < (int)(blockDim.x >> 5)) ? sm[l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (l == 0) atomicMax(out, (unsigned long long)__double_as_longlong(v));
    }
}

// max over cells of (max_d |u_d| + c), in the precision of the state.
template <typename R, bool PLAIN>
__global__ void cfl_kernel(SweepArgs<R> A, const R *st, long long ncell, int nx, int ny,
                           unsigned long long *out) {
    const R gam = (R)A.gamma, gm1 = (R)(A.gamma - 1.0);
    R smax = 0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < ncell;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % nx), j = (int)((t / nx) % ny), k = (int)(t / ((long long)nx * ny));
        if (A.confine_r > 0.0 &&
            !fluid_point(cell_centre(A.org[0], A.dx, i), cell_centre(A.org[1], A.dx, j),
                         cell_centre(A.org[2], A.dx, k), A.confine_r))
            continue;  // solid cell of the confining sphere
        const Base<R> b = cell_base(A, i, j, k);
        const R rd = PLAIN ? xsub(st[t], b.rho0) : st[t];
        const R ed = PLAIN ? xsub(st[4 * ncell + t], xdiv(b.p0, gm1)) : st[4 * ncell + t];
        const R rho = b.rho0 + rd;
        const R ri = (R)1 / rho;
        const R mx = st[ncell + t], my = st[2 * ncell + t], mz = st[3 * ncell + t];
        const R u = mx * ri, v = my * ri, w = mz * ri;
        const R ke = (R)0.5 * (mx * u + (my * v + mz * w));
        const R p = b.p0 + gm1 * (ed - ke);
        const R s = rmax(rmax(rabs(u), rabs(v)), rabs(w)) + rsq(gam * p * ri);
        smax = rmax(smax, s);
    }
    block_max_atomic((double)smax, out);
}

// Rotation ramp (Sec. 3): every fluid cell gains the velocity
// domega * (-y, x, 0) (about the z axis through the coordinate origin), E the
// kinetic energy this adds (m.du + rho|du|^2/2, summed in x, y, z order); then,
// unless smax_out is NULL, the max over fluid cells of (max_d |u_d| + c) of
// the new state (the CFL maximum of the step, as the last pass would give).
// Launched after the step's last pass only while an increment is set, so the
// passes themselves carry none of it.
template <typename R, bool PLAIN>
__global__ void rotate_kernel(SweepArgs<R> A, R *st, long long ncell, int nx, int ny, double domega,
                              unsigned long long *smax_out) {
    const R gam = (R)A.gamma, gm1 = (R)(A.gamma - 1.0);
    const R w = (R)domega;
    R smax = 0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < ncell;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % nx), j = (int)((t / nx) % ny), k = (int)(t / ((long long)nx * ny));
        if (A.confine_r > 0.0 &&
            !fluid_point(cell_centre(A.org[0], A.dx, i), cell_centre(A.org[1], A.dx, j),
                         cell_centre(A.org[2], A.dx, k), A.confine_r))
            continue;  // solid cell of the confining sphere
        const Base<R> b = cell_base(A, i, j, k);
        const R rho = PLAIN ? st[t] : b.rho0 + st[t];
        R mx = st[ncell + t], my = st[2 * ncell + t];
        const R mz = st[3 * ncell + t];
        const R dux = -(w * coord(A, 1, j)), duy = w * coord(A, 0, i), duz = (R)0;
        const R dE = (mx * dux + (my * duy + mz * duz)) + (R)0.5 * rho * (dux * dux + (duy * duy + duz * duz));
        mx = mx + rho * dux;
        my = my + rho * duy;
        const R E = st[4 * ncell + t] + dE;
        st[ncell + t] = mx;
        st[2 * ncell + t] = my;
        st[4 * ncell + t] = E;
        if (smax_out) {
            const R rd = PLAIN ? xsub(st[t], b.rho0) : st[t];
            const R ed = PLAIN ? xsub(E, xdiv(b.p0, gm1)) : E;
            const R rh = b.rho0 + rd;
            const R ri = (R)1 / rh;
            const R u = mx * ri, v = my * ri, ww = mz * ri;
            const R ke = (R)0.5 * (mx * u + (my * v + mz * ww));
            const R p = b.p0 + gm1 * (ed - ke);
            smax = rmax(smax, rmax(rmax(rabs(u), rabs(v)), rabs(ww)) + rsq(gam * p * ri));
        }
    }
    if (smax_out) block_max_atomic((double)smax, smax_out);
}

// FP64 diagnostics: totals and shell averages.  acc layout: [0..6] totals,
// [8..8+6*nbins) per bin (count, rho, p, FV, |u|, u_r^2), [7] max Mach bits.

// Base state of every cell for the diagnostics of the FP32 form: rho0 as an
// unevaluated sum hi + lo of two floats (hi = rho0 rounded to float, lo = the
// remainder rounded: 48 significant bits together), p0 rounded to float (the
// Mach number and shell pressures only), and the FP64 grid sums of rho0 and
// of p0/(gamma-1) as the state download forms them (sums[0], sums[1]).
__global__ void base_fill_kernel(SweepArgs<double> A64, float *hi, float *lo, float *p0f, double *sums,
                                 long long ncell, int nx, int ny) {
    const double gm1 = A64.gamma - 1.0;
    double sr = 0.0, se = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < ncell;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % nx), j = (int)((t / nx) % ny), k = (int)(t / ((long long)nx * ny));
        const Base<double> bb = cell_base(A64, i, j, k);
        const float h = (float)bb.rho0;
        hi[t] = h;
        lo[t] = (float)(bb.rho0 - (double)h);
        p0f[t] = (float)bb.p0;
        sr += bb.rho0;
        se += xdiv(bb.p0, gm1);
    }
    __shared__ double red[2][32];
    for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        se += __shfl_xor_sync(0xffffffffu, se, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        red[0][w] = sr;
        red[1][w] = se;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double v = 0.0;
        for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) v += red[threadIdx.x][ww];
        atomicAdd(sums + threadIdx.x, v);
    }
}

// A float pair (s, c) standing for s + c, summed with Knuth's TwoSum: the
// rounding error of every addition is kept exactly and collected in c.
struct Sum2 {
    float s, c;
};
__device__ __forceinline__ void sum2_add(Sum2 &a, float x) {
    const float t = a.s + x;
    const float bp = t - a.s;
    a.c += (a.s - (t - bp)) + (x - bp);
    a.s = t;
}

// Totals of every cell's bin (shell averages): FP64 per cell, shared by both
// diagnostics kernels.
__device__ __forceinline__ void bin_cell(double *sbin, int nbins, double rmax_, double x, double y, double z,
                                         double r, double rho, double p, double fv, double mx, double my,
                                         double mz) {
    if (r < 0.0) r = sqrt(x * x + y * y + z * z);
    const int bin = (int)floor(r / rmax_ * nbins);
    if (bin >= 0 && bin < nbins) {
        const double rinv = 1.0 / rho;
        const double spd = sqrt(mx * mx + my * my + mz * mz) * rinv;
        const double ur = r > 0.0 ? (mx * x + my * y + mz * z) * rinv / r : 0.0;
        double *a = sbin + 6 * bin;
        atomicAdd(a + 0, 1.0);
        atomicAdd(a + 1, rho);
        atomicAdd(a + 2, p);
        atomicAdd(a + 3, fv);
        atomicAdd(a + 4, spd);
        atomicAdd(a + 5, ur * ur);
    }
}

// Block reduction of the seven totals, the Mach maximum and the bins into acc.
__device__ __forceinline__ void diag_flush_block(const double tot[7], double m2max, double *sbin, int nbins,
                                                 double *acc) {
    __shared__ double stot[7][32];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int m = 0; m < 7; ++m) {
        double v = tot[m];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (l == 0) stot[m][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < 7) {
        double v = 0.0;
        for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) v += stot[threadIdx.x][ww];
        atomicAdd(acc + threadIdx.x, v);
    }
    for (int b = threadIdx.x; b < 6 * nbins; b += blockDim.x)
        if (sbin[b] != 0.0) atomicAdd(acc + 8 + b, sbin[b]);
    block_max_atomic(m2max, reinterpret_cast<unsigned long long *>(acc + 7));
}

// Diagnostics of the FP32 form with the cached base state.  The totals keep
// FP64 accuracy without FP64 arithmetic per cell (FP64 is slow on this part):
// each thread sums its cells in float pairs (Sum2), products of two floats
// enter as exact pairs (p = a*b rounded, e = fma(a, b, -p)), and every 32
// cells the pairs are added into FP64.  Totals 0 and 4 are the sums of rho'
// and E': the host adds the base sums.  FV near 1 is stored as FV - 1 (a
// negative value s): FV = a + s with a = 1 for such a cell, 0 otherwise, so
// that both FV sums keep the folded value's precision.  The Mach number is
// taken in FP32; shell averages (nbins > 0) stay FP64 per cell.
__global__ void diag32_kernel(SweepArgs<double> A64, const float *st, long long ncell, int nx, int ny,
                              int nbins, double rmax_, double *acc, const float *bhi, const float *blo,
                              const float *bp0) {
    extern __shared__ double sbin[];
    for (int b = threadIdx.x; b < 6 * nbins; b += blockDim.x) sbin[b] = 0.0;
    __syncthreads();
    const double gm1 = A64.gamma - 1.0;
    const float gm1f = (float)gm1, gamf = (float)A64.gamma;
    double tot[7] = {0, 0, 0, 0, 0, 0, 0};
    Sum2 s[7];
    for (int m = 0; m < 7; ++m) s[m] = Sum2{0.0f, 0.0f};
    float small5 = 0.0f, ones6 = 0.0f;   // tiny product terms of rho*FV; folded-cell count
    float m2max = 0.0f;
    auto flush = [&]() {
        for (int m = 0; m < 7; ++m) {
            tot[m] += (double)s[m].s + (double)s[m].c;
            s[m] = Sum2{0.0f, 0.0f};
        }
        tot[5] += (double)small5;
        tot[6] += (double)ones6;
        small5 = ones6 = 0.0f;
    };
    int k = 0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < ncell;
         t += (long long)gridDim.x * blockDim.x) {
        const float rd = st[t], mx = st[ncell + t], my = st[2 * ncell + t], mz = st[3 * ncell + t];
        const float ed = st[4 * ncell + t], fs = st[5 * ncell + t];
        const float h = bhi[t], l = blo[t], p0 = bp0[t];
        sum2_add(s[0], rd);
        sum2_add(s[1], mx);
        sum2_add(s[2], my);
        sum2_add(s[3], mz);
        sum2_add(s[4], ed);
        const float a = signbit(fs) ? 1.0f : 0.0f;
        sum2_add(s[6], fs);
        ones6 += a;
        // rho FV = a (h + l + rho') + (h + l + rho') s
        const float p1 = h * fs, e1 = fmaf(h, fs, -p1);
        const float p2 = rd * fs, e2 = fmaf(rd, fs, -p2);
        sum2_add(s[5], a * h);
        sum2_add(s[5], a * rd);
        sum2_add(s[5], p1);
        sum2_add(s[5], p2);
        small5 += (e1 + e2) + l * (a + fs);
        const float rf = h + rd;
        const float m2 = fmaf(mx, mx, fmaf(my, my, mz * mz));
        const float pf = p0 + gm1f * (ed - 0.5f * __fdividef(m2, rf));
        m2max = fmaxf(m2max, __fdividef(m2, gamf * pf * rf));
        if (nbins > 0) {
            const int i = (int)(t % nx), j = (int)((t / nx) % ny), kz = (int)(t / ((long long)nx * ny));
            const double x = coord(A64, 0, i), y = coord(A64, 1, j), z = coord(A64, 2, kz);
            const double rho = ((double)h + (double)l) + (double)rd;
            const double md[3] = {(double)mx, (double)my, (double)mz};
            const double p = (double)p0 +
                             gm1 * ((double)ed - 0.5 * (md[0] * md[0] + md[1] * md[1] + md[2] * md[2]) / rho);
            bin_cell(sbin, nbins, rmax_, x, y, z, -1.0, rho, p, (double)a + (double)fs, md[0], md[1], md[2]);
        }
        if (++k == 32) {
            flush();
            k = 0;
        }
    }
    flush();
    diag_flush_block(tot, (double)m2max, sbin, nbins, acc);
}

// Diagnostics with the base state looked up per cell: the FP64 form, and
// the FP32 form when there was no room for the cached base state.  FP64 is
// slow on this part: per cell one square root (r, central gravity only) and
// two divisions; the table lookup multiplies by 1/ds and the Mach number is
// maximised as its square.  Results agree with the exact-lookup formulas to
// rounding.
template <typename R, bool PLAIN>
__global__ void diag_kernel(SweepArgs<double> A64, const R *st, long long ncell, int nx, int ny,
                            int nbins, double rmax_, double *acc) {
    extern __shared__ double sbin[];
    for (int b = threadIdx.x; b < 6 * nbins; b += blockDim.x) sbin[b] = 0.0;
    __syncthreads();
    const double gam = A64.gamma, gm1 = A64.gamma - 1.0, igm1 = 1.0 / gm1;
    const double inv_ds = 1.0 / A64.ds;
    const double *t_r = A64.t_rho0, *t_p = A64.t_p0;
    double tot[7] = {0, 0, 0, 0, 0, 0, 0};
    double m2max = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < ncell;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % nx), j = (int)((t / nx) % ny), k = (int)(t / ((long long)nx * ny));
        const double x = coord(A64, 0, i), y = coord(A64, 1, j), z = coord(A64, 2, k);
        double rho0, p0, r = -1.0;
        if (A64.grav == 0) {
            rho0 = A64.rho0_c;
            p0 = A64.p0_c;
        } else {
            double sv = z;
            if (A64.grav == 2) {
                r = sqrt(x * x + y * y + z * z);
                sv = r;
            }
            const double u = (sv - A64.s0) * inv_ds;
            const double fl = fmin(fmax(floor(u), 0.0), (double)(A64.ntab - 2));
            const int ii = (int)fl;
            const double wt = u - fl;
            rho0 = fma(wt, t_r[ii + 1] - t_r[ii], t_r[ii]);
            p0 = fma(wt, t_p[ii + 1] - t_p[ii], t_p[ii]);
        }
        double rho, E, Ed;
        if (PLAIN) {
            rho = (double)st[t];
            E = (double)st[4 * ncell + t];
            Ed = E - p0 * igm1;
        } else {
            rho = rho0 + (double)st[t];
            Ed = (double)st[4 * ncell + t];
            E = p0 * igm1 + Ed;
        }
        const double mx = st[ncell + t], my = st[2 * ncell + t], mz = st[3 * ncell + t];
        double fv = st[5 * ncell + t];
        if (!PLAIN) fv = signbit(fv) ? 1.0 + fv : fv;
        tot[0] += rho;
        tot[1] += mx;
        tot[2] += my;
        tot[3] += mz;
        tot[4] += E;
        tot[5] += rho * fv;
        tot[6] += fv;
        const double m2 = mx * mx + my * my + mz * mz;
        const double p = p0 + gm1 * (Ed - 0.5 * m2 / rho);
        if (PLAIN) {
            m2max = fmax(m2max, m2 / (gam * p * rho));   // |u|^2 / c^2
        } else {
            // FP32 state: its Mach number to FP32 accuracy
            const float rf = (float)rho, m2f = (float)m2;
            const float pf = (float)p0 + (float)gm1 * ((float)Ed - 0.5f * m2f / rf);
            m2max = fmax(m2max, (double)(m2f / ((float)gam * pf * rf)));
        }
        if (nbins > 0) bin_cell(sbin, nbins, rmax_, x, y, z, r, rho, p, fv, mx, my, mz);
    }
    diag_flush_block(tot, m2max, sbin, nbins, acc);
}

int grid_for(long long n, int block) {
    long long g = (n + block - 1) / block;
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    return (int)g;
}

// Velocity divergence of every cell for the 3-D shock dissipation: central
// differences of u_d = (rho u_d)/rho along each axis, summed in x, y, z order;
// ghost neighbours by the boundary conditions (periodic wrap; at a wall the
// mirror cell with its normal velocity reversed).
template <typename R, bool PLAIN>
__global__ void divergence_kernel(SweepArgs<R> A, const R *st, R *D, long long ncell, int nx, int ny, int nz,
                                  int bx0, int bx1, int by0, int by1, int bz0, int bz1) {
    const int n[3] = {nx, ny, nz};
    const int bl[3] = {bx0, by0, bz0}, bh[3] = {bx1, by1, bz1};
    const R h = (R)(0.5 / A.dx);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < ncell;
         t += (long long)gridDim.x * blockDim.x) {
        const int ijk[3] = {(int)(t % nx), (int)((t / nx) % ny), (int)(t / ((long long)nx * ny))};
        R diff[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            R u[2];
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                int idx[3] = {ijk[0], ijk[1], ijk[2]};
                bool flip;
                idx[d] = map_cell(ijk[d] + (s ? 1 : -1), n[d], bl[d], bh[d], flip);
                const long long cc = ((long long)idx[2] * ny + idx[1]) * nx + idx[0];
                R rho = st[cc];
                if (!PLAIN) rho = cell_base(A, idx[0], idx[1], idx[2]).rho0 + rho;
                const R v = st[(1 + d) * ncell + cc] / rho;
                u[s] = flip ? -v : v;
            }
            diff[d] = u[1] - u[0];
        }
        D[t] = ((diff[0] + diff[1]) + diff[2]) * h;
    }
}

// The same divergence for the FP32 form, tiled: a block of 32 x 16 threads
// owns a 32 x 16 column of cells in x-y and marches up a run of DIV_ZRUN
// z-planes.  Each cell's velocity (rho u_d / (rho0 + rho'), rho0 from the
// pass kernels' FP32 tables) is computed once; u_x and u_y of a plane, with a
// one-cell halo, sit in shared memory (two planes, one barrier per plane),
// u_z of the planes below and above stay in registers.  Ghost neighbours as
// in the passes: periodic wrap, or the mirror cell with the normal velocity
// reversed (applied as a sign-bit mask).  Differences summed in x, y, z
// order, times 1/(2 dx).
constexpr int DIV_TX = 32, DIV_TY = 16, DIV_ZRUN = 64;

// Loads: each thread copies the stored values its cells need (rho', three
// momenta and the two base-state table rows of its own cell; rho', one
// momentum and two rows of its halo cell) DIV_PF planes ahead into a private
// ring in shared memory with cp.async, so that DIV_PF planes of loads per
// thread are in flight without holding them in registers (an earlier form
// kept one plane of loads in registers and was bound by the memory latency:
// 1.5 ms more per launch at 1024^3).
constexpr int DIV_PF = 4;                      // planes in flight per thread
constexpr int DIV_NT = DIV_TX * DIV_TY;
constexpr int DIV_RV = 10;                     // ring values per thread and plane
constexpr int div_ring_smem() { return DIV_PF * DIV_RV * DIV_NT * (int)sizeof(float); }

__global__ void __launch_bounds__(DIV_NT, 2) divergence_ring_kernel(SweepArgs<float> A, const float *st, float *D,
                                                                    long long ncell, int nx, int ny, int nz, int bx0,
                                                                    int bx1, int by0, int by1, int bz0, int bz1) {
    extern __shared__ __align__(16) float ring[];   // [DIV_PF][DIV_RV][DIV_NT]
    __shared__ float ux[2][DIV_TY + 2][DIV_TX + 2];
    __shared__ float uy[2][DIV_TY + 2][DIV_TX + 2];
    const int tx = threadIdx.x, ty = threadIdx.y, t = ty * DIV_TX + tx;
    const int i = blockIdx.x * DIV_TX + tx, j = blockIdx.y * DIV_TY + ty;
    const int k0 = blockIdx.z * DIV_ZRUN, k1 = min(nz, k0 + DIV_ZRUN);
    const float h = (float)(0.5 / A.dx);
    const float ox = (float)A.org[0], oy = (float)A.org[1], oz = (float)A.org[2], dxf = (float)A.dx;
    const bool tab = (A.grav != 0);
    struct Col {
        long long xy;     // x-y offset of the mapped cell in a plane
        float x2y2;       // x^2 + y^2 of the mapped cell (central gravity)
        unsigned sx, sy;  // sign-bit masks of u and v
    };
    auto column = [&](int gi, int gj) -> Col {
        Col c;
        bool fx = false, fy = false;
        const int ii = map_cell(gi, nx, bx0, bx1, fx), jj = map_cell(gj, ny, by0, by1, fy);
        c.xy = (long long)jj * nx + ii;
        const float x = ox + ((float)ii + 0.5f) * dxf, y = oy + ((float)jj + 0.5f) * dxf;
        c.x2y2 = fmaf(y, y, x * x);
        c.sx = fx ? 0x80000000u : 0u;
        c.sy = fy ? 0x80000000u : 0u;
        return c;
    };
    auto flipf = [](float v, unsigned m) { return __uint_as_float(__float_as_uint(v) ^ m); };
    // table coordinate of plane kk of a column: row index and weight
    auto tab_u = [&](const Col &cl, int kk) {
        const float z = oz + ((float)kk + 0.5f) * dxf;
        const float sv = (A.grav == 1) ? z : fmaf(z, z, cl.x2y2);
        return (sv - A.s4_0) * A.inv_ds4;
    };
    auto tab_fl = [&](float uu) { return fminf(fmaxf(floorf(uu), 0.0f), (float)(A.ntab4 - 2)); };
    const long long plane_cells = (long long)nx * ny;
    // this thread's slot of a plane and, for threads 0..95, one halo slot
    // (rows j = -1 and j = DIV_TY across the tile need v; columns i = -1 and
    // i = DIV_TX along it need u; the corners are never used).  Just past the
    // grid edge (i == nx or j == ny) the slot is the ghost neighbour of the
    // last cell.
    const bool own = (i < nx && j < ny);
    const bool slot_ok = i <= nx && j <= ny && !(i == nx && j == ny);
    int hx = -1, hy = -1;
    if (t < 2 * DIV_TX) {
        hx = (t % DIV_TX) + 1;
        hy = (t < DIV_TX) ? 0 : DIV_TY + 1;
    } else if (t < 2 * DIV_TX + 2 * DIV_TY) {
        const int r = t - 2 * DIV_TX;
        hy = (r % DIV_TY) + 1;
        hx = (r < DIV_TY) ? 0 : DIV_TX + 1;
    }
    const bool halo_u = (t >= 2 * DIV_TX);
    const int gi = blockIdx.x * DIV_TX + hx - 1, gj = blockIdx.y * DIV_TY + hy - 1;
    const bool halo_ok = hx >= 0 && gi >= -1 && gi <= nx && gj >= -1 && gj <= ny;
    const Col col_own = column(slot_ok ? i : 0, slot_ok ? j : 0);
    const Col col_halo = column(halo_ok ? gi : 0, halo_ok ? gj : 0);
    // copies of plane gk into ring slot sl: the own cell for gk in
    // [k0-1, k1] (the planes just below and above the run give u_z), the halo
    // cell for gk in [k0, k1); one commit group per call, empty or not
    auto issue = [&](int gk, int sl) {
        if (gk <= k1) {
            float *r = ring + (sl * DIV_RV) * DIV_NT + t;
            if (slot_ok) {
                bool fz = false;
                const int kk = map_cell(gk, nz, bz0, bz1, fz);
                const float *p = st + (long long)kk * plane_cells + col_own.xy;
                cp_async<4>(r, p);
                cp_async<4>(r + DIV_NT, p + ncell);
                cp_async<4>(r + 2 * DIV_NT, p + 2 * ncell);
                cp_async<4>(r + 3 * DIV_NT, p + 3 * ncell);
                if (tab) {
                    const int row = (int)tab_fl(tab_u(col_own, kk));
                    cp_async<4>(r + 4 * DIV_NT, reinterpret_cast<const float *>(A.t4_base + row));
                    cp_async<4>(r + 5 * DIV_NT, reinterpret_cast<const float *>(A.t4_base + row + 1));
                }
            }
            if (halo_ok && gk >= k0 && gk < k1) {
                const float *p = st + (long long)gk * plane_cells + col_halo.xy;
                cp_async<4>(r + 6 * DIV_NT, p);
                cp_async<4>(r + 7 * DIV_NT, p + (halo_u ? 1 : 2) * ncell);
                if (tab) {
                    const int row = (int)tab_fl(tab_u(col_halo, gk));
                    cp_async<4>(r + 8 * DIV_NT, reinterpret_cast<const float *>(A.t4_base + row));
                    cp_async<4>(r + 9 * DIV_NT, reinterpret_cast<const float *>(A.t4_base + row + 1));
                }
            }
        }
        cp_commit();
    };
    // 1 / rho of a cell from its ring values (rho' at r[0], rows at r[a], r[b])
    auto rinv = [&](const float *r, int a, const Col &cl, int kk) {
        float rho0 = (float)A.rho0_c;
        if (tab) {
            const float uu = tab_u(cl, kk);
            const float ta = r[a * DIV_NT], tb = r[(a + 1) * DIV_NT];
            rho0 = fmaf(uu - tab_fl(uu), tb - ta, ta);
        }
        return qdiv(1.0f, rho0 + r[0]);
    };
#pragma unroll
    for (int sl = 0; sl < DIV_PF; ++sl) issue(k0 - 1 + sl, sl);
    float wm = 0.0f, w0 = 0.0f;   // u_z of planes q-2 and q-1
    for (int q = k0 - 1; q <= k1; ++q) {
        const int sl = (q - (k0 - 1)) & (DIV_PF - 1);
        cp_wait<DIV_PF - 1>();   // this thread's copies of plane q have landed
        const float *r = ring + (sl * DIV_RV) * DIV_NT + t;
        float u = 0.0f, v = 0.0f, w = 0.0f, hv = 0.0f;
        if (slot_ok) {
            bool fz = false;
            const int kk = map_cell(q, nz, bz0, bz1, fz);
            const float ri = rinv(r, 4, col_own, kk);
            u = flipf(r[DIV_NT] * ri, col_own.sx);
            v = flipf(r[2 * DIV_NT] * ri, col_own.sy);
            w = flipf(r[3 * DIV_NT] * ri, fz ? 0x80000000u : 0u);
        }
        const bool hq = halo_ok && q >= k0 && q < k1;
        if (hq) {
            const float ri = rinv(r + 6 * DIV_NT, 8 - 6, col_halo, q);
            hv = flipf(r[7 * DIV_NT] * ri, halo_u ? col_halo.sx : col_halo.sy);
        }
        issue(q + DIV_PF, sl);   // the slot is free again
        if (q >= k0 && q < k1) {
            const int b = q & 1;
            ux[b][ty + 1][tx + 1] = u;
            uy[b][ty + 1][tx + 1] = v;
            if (hq) {
                if (halo_u)
                    ux[b][hy][hx] = hv;
                else
                    uy[b][hy][hx] = hv;
            }
        }
        if (q > k0 && own) {   // plane q-1: u_x, u_y written last iteration, u_z of q-2 and q
            const int b = (q - 1) & 1;
            const float dxu = ux[b][ty + 1][tx + 2] - ux[b][ty + 1][tx];
            const float dyv = uy[b][ty + 2][tx + 1] - uy[b][ty][tx + 1];
            D[((long long)(q - 1) * ny + j) * nx + i] = ((dxu + dyv) + (w - wm)) * h;
        }
        wm = w0;
        w0 = w;
        __syncthreads();
    }
    cp_wait<0>();
}

// The same divergence from the cell velocities the pass before left
// (`SweepArgs::vel_out`: u_x, u_y, u_z arrays, the quotient and products of
// the full form above taken in that pass): no table lookup and no quotient
// here; a halo cell needs one component.  Ghosts as above.
constexpr int DV_RV = 4;   // ring values per thread and plane: u, v, w; the halo component
constexpr int div_vel_smem() { return DIV_PF * DV_RV * DIV_NT * (int)sizeof(float); }

__global__ void __launch_bounds__(DIV_NT, 2) divergence_vel_kernel(const float *vel, float *D, double dx,
                                                                   long long ncell, int nx, int ny, int nz, int bx0,
                                                                   int bx1, int by0, int by1, int bz0, int bz1) {
    extern __shared__ __align__(16) float ring[];   // [DIV_PF][DV_RV][DIV_NT]
    __shared__ float ux[2][DIV_TY + 2][DIV_TX + 2];
    __shared__ float uy[2][DIV_TY + 2][DIV_TX + 2];
    const int tx = threadIdx.x, ty = threadIdx.y, t = ty * DIV_TX + tx;
    const int i = blockIdx.x * DIV_TX + tx, j = blockIdx.y * DIV_TY + ty;
    const int k0 = blockIdx.z * DIV_ZRUN, k1 = min(nz, k0 + DIV_ZRUN);
    const float h = (float)(0.5 / dx);
    struct Col {
        long long xy;     // x-y offset of the mapped cell in a plane
        unsigned sx, sy;  // sign-bit masks of u and v
    };
    auto column = [&](int gi, int gj) -> Col {
        Col c;
        bool fx = false, fy = false;
        const int ii = map_cell(gi, nx, bx0, bx1, fx), jj = map_cell(gj, ny, by0, by1, fy);
        c.xy = (long long)jj * nx + ii;
        c.sx = fx ? 0x80000000u : 0u;
        c.sy = fy ? 0x80000000u : 0u;
        return c;
    };
    auto flipf = [](float v, unsigned m) { return __uint_as_float(__float_as_uint(v) ^ m); };
    const long long plane_cells = (long long)nx * ny;
    // slots and halo as in the full form
    const bool own = (i < nx && j < ny);
    const bool slot_ok = i <= nx && j <= ny && !(i == nx && j == ny);
    int hx = -1, hy = -1;
    if (t < 2 * DIV_TX) {
        hx = (t % DIV_TX) + 1;
        hy = (t < DIV_TX) ? 0 : DIV_TY + 1;
    } else if (t < 2 * DIV_TX + 2 * DIV_TY) {
        const int r = t - 2 * DIV_TX;
        hy = (r % DIV_TY) + 1;
        hx = (r < DIV_TY) ? 0 : DIV_TX + 1;
    }
    const bool halo_u = (t >= 2 * DIV_TX);
    const int gi = blockIdx.x * DIV_TX + hx - 1, gj = blockIdx.y * DIV_TY + hy - 1;
    const bool halo_ok = hx >= 0 && gi >= -1 && gi <= nx && gj >= -1 && gj <= ny;
    const Col col_own = column(slot_ok ? i : 0, slot_ok ? j : 0);
    const Col col_halo = column(halo_ok ? gi : 0, halo_ok ? gj : 0);
    auto issue = [&](int gk, int sl) {
        if (gk <= k1) {
            float *r = ring + (sl * DV_RV) * DIV_NT + t;
            if (slot_ok) {
                bool fz = false;
                const int kk = map_cell(gk, nz, bz0, bz1, fz);
                const float *p = vel + (long long)kk * plane_cells + col_own.xy;
                cp_async<4>(r, p);
                cp_async<4>(r + DIV_NT, p + ncell);
                cp_async<4>(r + 2 * DIV_NT, p + 2 * ncell);
            }
            if (halo_ok && gk >= k0 && gk < k1)
                cp_async<4>(r + 3 * DIV_NT, vel + (halo_u ? 0 : ncell) + (long long)gk * plane_cells + col_halo.xy);
        }
        cp_commit();
    };
#pragma unroll
    for (int sl = 0; sl < DIV_PF; ++sl) issue(k0 - 1 + sl, sl);
    float wm = 0.0f, w0 = 0.0f;   // u_z of planes q-2 and q-1
    for (int q = k0 - 1; q <= k1; ++q) {
        const int sl = (q - (k0 - 1)) & (DIV_PF - 1);
        cp_wait<DIV_PF - 1>();
        const float *r = ring + (sl * DV_RV) * DIV_NT + t;
        float u = 0.0f, v = 0.0f, w = 0.0f, hv = 0.0f;
        if (slot_ok) {
            bool fz = false;
            (void)map_cell(q, nz, bz0, bz1, fz);
            u = flipf(r[0], col_own.sx);
            v = flipf(r[DIV_NT], col_own.sy);
            w = flipf(r[2 * DIV_NT], fz ? 0x80000000u : 0u);
        }
        const bool hq = halo_ok && q >= k0 && q < k1;
        if (hq) hv = flipf(r[3 * DIV_NT], halo_u ? col_halo.sx : col_halo.sy);
        issue(q + DIV_PF, sl);
        if (q >= k0 && q < k1) {
            const int b = q & 1;
            ux[b][ty + 1][tx + 1] = u;
            uy[b][ty + 1][tx + 1] = v;
            if (hq) {
                if (halo_u)
                    ux[b][hy][hx] = hv;
                else
                    uy[b][hy][hx] = hv;
            }
        }
        if (q > k0 && own) {
            const int b = (q - 1) & 1;
            const float dxu = ux[b][ty + 1][tx + 2] - ux[b][ty + 1][tx];
            const float dyv = uy[b][ty + 2][tx + 1] - uy[b][ty][tx + 1];
            D[((long long)(q - 1) * ny + j) * nx + i] = ((dxu + dyv) + (w - wm)) * h;
        }
        wm = w0;
        w0 = w;
        __syncthreads();
    }
    cp_wait<0>();
}

int launch_divergence(ppm_ctx *c, bool from_vel) {
    const int g = grid_for(c->ncell, 256);
    const int *b = c->bc;
    if (c->prec == PPM_FP32_DEVIATION) {
        const dim3 grid((c->n[0] + DIV_TX - 1) / DIV_TX, (c->n[1] + DIV_TY - 1) / DIV_TY,
                        (c->n[2] + DIV_ZRUN - 1) / DIV_ZRUN);
        if (from_vel)
            divergence_vel_kernel<<<grid, dim3(DIV_TX, DIV_TY), div_vel_smem(), c->stream>>>(
                (const float *)c->vel, (float *)c->divg, c->dx, c->ncell, c->n[0], c->n[1], c->n[2], b[0], b[1],
                b[2], b[3], b[4], b[5]);
        else
            divergence_ring_kernel<<<grid, dim3(DIV_TX, DIV_TY), div_ring_smem(), c->stream>>>(
                make_args<float>(c, 0), (const float *)c->state, (float *)c->divg, c->ncell, c->n[0], c->n[1],
                c->n[2], b[0], b[1], b[2], b[3], b[4], b[5]);
    } else
        divergence_kernel<double, true><<<g, 256, 0, c->stream>>>(make_args<double>(c, 0), (const double *)c->state,
                                                                  (double *)c->divg, c->ncell, c->n[0], c->n[1], c->n[2],
                                                                  b[0], b[1], b[2], b[3], b[4], b[5]);
    c->launches++;
    CK(c, cudaGetLastError());
    return PPM_OK;
}

static int launch_rotate(ppm_ctx *c, bool with_cfl) {
    const int g = grid_for(c->ncell, 256);
    unsigned long long *so = nullptr;
    if (with_cfl) {
        CK(c, cudaMemsetAsync(&c->ds_dev->smax, 0, sizeof(unsigned long long), c->stream));
        so = &c->ds_dev->smax;
    }
    if (c->prec == PPM_FP32_DEVIATION)
        rotate_kernel<float, false><<<g, 256, 0, c->stream>>>(make_args<float>(c, 0), (float *)c->state, c->ncell,
                                                               c->n[0], c->n[1], c->domega, so);
    else
        rotate_kernel<double, true><<<g, 256, 0, c->stream>>>(make_args<double>(c, 0), (double *)c->state, c->ncell,
                                                               c->n[0], c->n[1], c->domega, so);
    c->launches++;
    CK(c, cudaGetLastError());
    return PPM_OK;
}


SweepArgs<double> args64(ppm_ctx *c) { return make_args<double>(c, 0); }

int check_flags(ppm_ctx *c) {
    int fl = 0;
    CK(c, cudaMemcpyAsync(&fl, &c->ds_dev->flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (fl & FLAG_TIMEOUT) {
        CK(c, cudaMemsetAsync(&c->ds_dev->flags, 0, sizeof(int), c->stream));
        return fail(c, PPM_ETIMEOUT, "a bounded device wait gave up (a TMA copy did not complete)");
    }
    if (fl & FLAG_NONPHYS) {
        CK(c, cudaMemsetAsync(&c->ds_dev->flags, 0, sizeof(int), c->stream));
        return fail(c, PPM_ENONPHYS, "a pass produced rho<=0, p<=0 or a non-finite value");
    }
    return PPM_OK;
}

// Device address of a host array of `count` doubles that lies in page-locked
// memory this device can address (cudaHostAlloc / cudaHostRegister), or NULL.
// The first and the last element must both be in such memory, at device
// addresses `count - 1` doubles apart.
double *mapped_host(const ppm_ctx *c, double *p, long long count) {
    cudaPointerAttributes a, b;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer || a.device != c->device) return nullptr;
    if (cudaPointerGetAttributes(&b, p + (count - 1)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (b.type != cudaMemoryTypeHost || !b.devicePointer) return nullptr;
    const long long span = (const char *)b.devicePointer - (const char *)a.devicePointer;
    if (span != (count - 1) * (long long)sizeof(double)) return nullptr;
    return static_cast<double *>(a.devicePointer);
}

// Host regions in page-locked memory are read or written in place by the
// conversion kernel over the host link (at the link's rate, with no staging
// pass and no copy engine).  Other host regions go through two device
// staging buffers in turn: the copies of one chunk (on the context's copy
// stream) overlap the conversion kernel of the previous chunk (on the
// context's stream), ordered by events.  Device regions are converted in
// place by one kernel.  All return when done.
int region_io(ppm_ctx *c, const int lo[3], const int hi[3], double *const *arrs, int mem, bool to_dev) {
    if (!c || !lo || !hi || !arrs) return fail(c, PPM_EINVAL, "null argument");
    int b[3];
    for (int d = 0; d < 3; ++d) {
        if (lo[d] < 0 || hi[d] > c->n[d] || lo[d] >= hi[d])
            return fail(c, PPM_EINVAL, "region [%d,%d) outside axis %d of extent %d", lo[d], hi[d], d, c->n[d]);
        b[d] = hi[d] - lo[d];
    }
    const int nv = c->nvar;
    for (int q = 0; q < nv; ++q)
        if (!arrs[q]) return fail(c, PPM_EINVAL, "q[%d] is NULL", q);
    if (mem != PPM_MEM_HOST && mem != PPM_MEM_DEVICE) return fail(c, PPM_EINVAL, "bad mem kind %d", mem);
    const SweepArgs<double> A = args64(c);
    const long long plane = (long long)b[0] * b[1];
    auto convert = [&](const RegionPtrs &ptrs, int lz, int nk, long long cnt) -> int {
        const int g = grid_for(cnt, 256);
        if (to_dev) {
            if (c->prec == PPM_FP32_DEVIATION)
                set_region_kernel<float, false><<<g, 256, 0, c->stream>>>(A, (float *)c->state, c->ncell, c->n[0], c->n[1], lo[0], lo[1], lz, b[0], b[1], nk, ptrs, 0, nv);
            else
                set_region_kernel<double, true><<<g, 256, 0, c->stream>>>(A, (double *)c->state, c->ncell, c->n[0], c->n[1], lo[0], lo[1], lz, b[0], b[1], nk, ptrs, 0, nv);
        } else {
            if (c->prec == PPM_FP32_DEVIATION)
                get_region_kernel<float, false><<<g, 256, 0, c->stream>>>(A, (const float *)c->state, c->ncell, c->n[0], c->n[1], lo[0], lo[1], lz, b[0], b[1], nk, ptrs, 0, nv);
            else
                get_region_kernel<double, true><<<g, 256, 0, c->stream>>>(A, (const double *)c->state, c->ncell, c->n[0], c->n[1], lo[0], lo[1], lz, b[0], b[1], nk, ptrs, 0, nv);
        }
        c->launches++;
        CK(c, cudaGetLastError());
        return PPM_OK;
    };
    RegionPtrs mapped;
    bool direct = (mem == PPM_MEM_DEVICE);
    bool host_mapped = false;
    if (direct) {
        for (int q = 0; q < nv; ++q) mapped.p[q] = arrs[q];
    } else {
        host_mapped = true;
        for (int q = 0; q < nv && host_mapped; ++q) {
            mapped.p[q] = mapped_host(c, arrs[q], plane * b[2]);
            host_mapped = mapped.p[q] != nullptr;
        }
        direct = host_mapped;
    }
    if (direct) {
        // host memory in slabs of about 2^26 cells per launch (one launch
        // over a 77 GB download ran at a fifth of the link's rate, slabs at
        // the full rate); device memory in one launch
        const long long kstep = host_mapped ? std::max(1LL, (1LL << 26) / plane) : (long long)b[2];
        for (long long k0 = 0; k0 < b[2]; k0 += kstep) {
            const long long nk = std::min(kstep, (long long)b[2] - k0);
            RegionPtrs part;
            for (int q = 0; q < nv; ++q) part.p[q] = mapped.p[q] + k0 * plane;
            const int r = convert(part, lo[2] + (int)k0, (int)nk, plane * nk);
            if (r != PPM_OK) return r;
        }
        CK(c, cudaStreamSynchronize(c->stream));
        if (to_dev) c->have_speed = false;
        return PPM_OK;
    }
    if (plane > c->stage_cells)
        return fail(c, PPM_EINVAL, "region plane of %lld cells exceeds the staging buffer", plane);
    if (!c->stage) {
        if (cudaMalloc(&c->stage, 2 * (size_t)nv * c->stage_cells * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            c->stage = nullptr;
            return fail(c, PPM_ENOMEM, "cannot allocate the host-transfer staging buffers");
        }
    }
    if (!c->xstream) {
        CK(c, cudaStreamCreateWithFlags(&c->xstream, cudaStreamNonBlocking));
        for (int i = 0; i < 2; ++i) {
            CK(c, cudaEventCreateWithFlags(&c->ev_copy[i], cudaEventDisableTiming));
            CK(c, cudaEventCreateWithFlags(&c->ev_kern[i], cudaEventDisableTiming));
        }
    }
    const long long kchunk = std::max(1LL, c->stage_cells / plane);
    int chunk = 0;
    for (long long k0 = 0; k0 < b[2]; k0 += kchunk, ++chunk) {
        const int h = chunk & 1;
        double *stage = c->stage + (long long)h * nv * c->stage_cells;
        const long long nk = std::min(kchunk, (long long)b[2] - k0);
        const long long cnt = plane * nk;
        RegionPtrs ptrs;
        for (int q = 0; q < nv; ++q) ptrs.p[q] = stage + (long long)q * c->stage_cells;
        if (to_dev) {
            if (chunk >= 2) CK(c, cudaStreamWaitEvent(c->xstream, c->ev_kern[h], 0));   // stage h converted
            for (int q = 0; q < nv; ++q)
                CK(c, cudaMemcpyAsync(ptrs.p[q], arrs[q] + k0 * plane, cnt * sizeof(double),
                                      cudaMemcpyHostToDevice, c->xstream));
            CK(c, cudaEventRecord(c->ev_copy[h], c->xstream));
            CK(c, cudaStreamWaitEvent(c->stream, c->ev_copy[h], 0));
            const int r = convert(ptrs, lo[2] + (int)k0, (int)nk, cnt);
            if (r != PPM_OK) return r;
            CK(c, cudaEventRecord(c->ev_kern[h], c->stream));
        } else {
            if (chunk >= 2) CK(c, cudaStreamWaitEvent(c->stream, c->ev_copy[h], 0));    // stage h drained
            const int r = convert(ptrs, lo[2] + (int)k0, (int)nk, cnt);
            if (r != PPM_OK) return r;
            CK(c, cudaEventRecord(c->ev_kern[h], c->stream));
            CK(c, cudaStreamWaitEvent(c->xstream, c->ev_kern[h], 0));
            for (int q = 0; q < nv; ++q)
                CK(c, cudaMemcpyAsync(arrs[q] + k0 * plane, ptrs.p[q], cnt * sizeof(double),
                                      cudaMemcpyDeviceToHost, c->xstream));
            CK(c, cudaEventRecord(c->ev_copy[h], c->xstream));
        }
    }
    CK(c, cudaStreamSynchronize(c->xstream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (to_dev) c->have_speed = false;
    return PPM_OK;
}

void release(ppm_ctx *c) {
    if (!c) return;
    for (int e = 0; e < 7; ++e)
        if (c->pev[e]) cudaEventDestroy(c->pev[e]);
    for (int h = 0; h < 2; ++h)
        if (c->halo[h]) cudaFree(c->halo[h]);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    if (c->state) cudaFree(c->state);
    if (c->divg) cudaFree(c->divg);
    if (c->vel) cudaFree(c->vel);
    if (c->t64) cudaFree(c->t64);
    if (c->t32) cudaFree(c->t32);
    if (c->t4) cudaFree(c->t4);
    if (c->ds_dev) cudaFree(c->ds_dev);
    if (c->xstream) {
        cudaStreamSynchronize(c->xstream);
        for (int i = 0; i < 2; ++i) {
            if (c->ev_copy[i]) cudaEventDestroy(c->ev_copy[i]);
            if (c->ev_kern[i]) cudaEventDestroy(c->ev_kern[i]);
        }
        cudaStreamDestroy(c->xstream);
    }
    if (c->stage) cudaFree(c->stage);
    if (c->diag_acc) cudaFree(c->diag_acc);
    if (c->base32) cudaFree(c->base32);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
}

}  // namespace

extern "C" {

int ppm_create(ppm_ctx **out, int nx, int ny, int nz, double gamma, const int bc[6],
               const ppm_gravity *grav, const ppm_options *opt) {
    if (!out || !bc || !grav || !opt) return fail(nullptr, PPM_EINVAL, "null argument");
    *out = nullptr;
    if (nx < 4 || ny < 4 || nz < 4) return fail(nullptr, PPM_EINVAL, "every extent must be >= 4 (got %d %d %d)", nx, ny, nz);
    if (!(gamma > 1.0)) return fail(nullptr, PPM_EINVAL, "gamma must exceed 1");
    for (int d = 0; d < 3; ++d) {
        if (d == 2 && opt->halo_z) continue;   // z faces checked with the halo planes below
        for (int s = 0; s < 2; ++s)
            if (bc[2 * d + s] != PPM_BC_PERIODIC && bc[2 * d + s] != PPM_BC_REFLECT)
                return fail(nullptr, PPM_EINVAL, "bad boundary kind on face %d", 2 * d + s);
        if ((bc[2 * d] == PPM_BC_PERIODIC) != (bc[2 * d + 1] == PPM_BC_PERIODIC))
            return fail(nullptr, PPM_EINVAL, "periodic faces must come in pairs (axis %d)", d);
    }
    if (grav->kind < 0 || grav->kind > 2) return fail(nullptr, PPM_EINVAL, "bad gravity kind");
    if (grav->ntab < 2 || !grav->rho0 || !grav->p0 || !grav->g || !(grav->ds > 0.0))
        return fail(nullptr, PPM_EINVAL, "base-state tables need ntab >= 2, ds > 0 and rho0, p0, g");
    if (opt->precision != PPM_FP64_PLAIN && opt->precision != PPM_FP32_DEVIATION)
        return fail(nullptr, PPM_EINVAL, "bad precision");
    if (!(opt->dx > 0.0)) return fail(nullptr, PPM_EINVAL, "dx must be positive");
    if (grav->kind == PPM_GRAV_NONE && (opt->heat || opt->damp))
        return fail(nullptr, PPM_EINVAL, "heating/damping tables need a gravity coordinate (plane or central)");
    if (!(opt->confine_r >= 0.0) || !std::isfinite(opt->confine_r))
        return fail(nullptr, PPM_EINVAL, "confine_r must be finite and >= 0");
    const int nmom = (opt->nmom == 0) ? 3 : opt->nmom;
    if (nmom != 3 && nmom != 9) return fail(nullptr, PPM_EINVAL, "nmom must be 3 or 9 (got %d)", opt->nmom);
    if (nmom == 9 && opt->confine_r > 0.0)
        return fail(nullptr, PPM_EINVAL, "the ten-value PPB (nmom 9) is not combined with a confining sphere");
    if (opt->halo_z < 0 || opt->halo_z > 3) return fail(nullptr, PPM_EINVAL, "halo_z must be 0..3");
    if (opt->halo_z) {
        if (opt->confine_r > 0.0 || opt->nmom == 9 || opt->shock_k > 0.0)
            return fail(nullptr, PPM_EINVAL, "halo planes are not combined with a confining sphere, nmom 9 or "
                                             "shock dissipation");
        // a z face without halo planes needs a wall (a periodic pair cannot be split)
        for (int s2 = 0; s2 < 2; ++s2)
            if (!(opt->halo_z & (1 << s2)) && bc[4 + s2] != PPM_BC_REFLECT)
                return fail(nullptr, PPM_EINVAL, "a z face without halo planes must be reflecting when the other "
                                                 "takes halo planes");
    }
    if (!(opt->shock_k >= 0.0) || !std::isfinite(opt->shock_k))
        return fail(nullptr, PPM_EINVAL, "shock_k must be finite and >= 0");
    if (opt->shock_k > 0.0 && (opt->confine_r > 0.0 || nmom == 9))
        return fail(nullptr, PPM_EINVAL, "shock dissipation is not combined with a confining sphere or nmom 9");
    if (opt->confine_r > 0.0)
        for (int f = 0; f < 6; ++f)
            if (bc[f] != PPM_BC_REFLECT)
                return fail(nullptr, PPM_EINVAL, "a confining sphere needs reflecting walls on all six faces");

    ppm_ctx *c = new ppm_ctx();
    c->n[0] = nx; c->n[1] = ny; c->n[2] = nz;
    c->ncell = (long long)nx * ny * nz;
    c->gamma = gamma;
    for (int i = 0; i < 6; ++i) c->bc[i] = bc[i];
    c->grav = grav->kind;
    c->prec = opt->precision;
    c->org[0] = opt->x0; c->org[1] = opt->y0; c->org[2] = opt->z0;
    c->dx = opt->dx;
    c->ntab = grav->ntab;
    c->rho0c = grav->rho0[0];
    c->p0c = grav->p0[0];
    c->s0 = grav->s0;
    c->ds = grav->ds;
    c->has_heat = opt->heat != nullptr;
    c->has_damp = opt->damp != nullptr;
    c->confine_r = opt->confine_r;
    c->nmom = nmom;
    c->nvar = 6 + nmom;
    c->shock_k = opt->shock_k;
    c->device = opt->device;
    c->halo_z = opt->halo_z;
    c->z_index0 = opt->z_index0;

    auto bail = [&](int code) {
        std::string m = c->err;
        release(c);
        delete c;
        g_create_error = m;
        return code;
    };
    cudaError_t e = cudaSetDevice(opt->device);
    if (e != cudaSuccess) {
        fail(c, PPM_ECUDA, "cudaSetDevice(%d): %s", opt->device, cudaGetErrorString(e));
        return bail(PPM_ECUDA);
    }
    if (opt->stream) {
        c->stream = (cudaStream_t)opt->stream;
        c->own_stream = false;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            fail(c, PPM_ECUDA, "cudaStreamCreate failed");
            return bail(PPM_ECUDA);
        }
        c->own_stream = true;
    }
    const size_t es = (c->prec == PPM_FP32_DEVIATION) ? sizeof(float) : sizeof(double);
    const size_t sbytes = (size_t)c->nvar * (size_t)c->ncell * es;
    if (cudaMalloc(&c->state, sbytes) != cudaSuccess) {
        cudaGetLastError();
        fail(c, PPM_ENOMEM, "cannot allocate %zu bytes of state", sbytes);
        return bail(PPM_ENOMEM);
    }
    for (int h = 0; h < 2; ++h)
        if ((c->halo_z & (1 << h)) &&
            cudaMalloc(&c->halo[h], (size_t)c->nvar * 4 * (size_t)nx * ny * es) != cudaSuccess) {
            cudaGetLastError();
            c->halo[h] = nullptr;
            fail(c, PPM_ENOMEM, "cannot allocate the halo planes");
            return bail(PPM_ENOMEM);
        }
    if (c->shock_k > 0.0 && cudaMalloc(&c->divg, (size_t)c->ncell * es) != cudaSuccess) {
        cudaGetLastError();
        c->divg = nullptr;
        fail(c, PPM_ENOMEM, "cannot allocate the divergence buffer");
        return bail(PPM_ENOMEM);
    }
    if (c->shock_k > 0.0 && c->prec == PPM_FP32_DEVIATION &&
        cudaMalloc(&c->vel, (size_t)3 * c->ncell * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        c->vel = nullptr;
        fail(c, PPM_ENOMEM, "cannot allocate the velocity buffer");
        return bail(PPM_ENOMEM);
    }
    const int nt = grav->ntab;
    std::vector<double> h64((size_t)5 * nt, 0.0);
    std::vector<float> h32((size_t)5 * nt, 0.0f);
    for (int i = 0; i < nt; ++i) {
        h64[i] = grav->rho0[i];
        h64[nt + i] = grav->p0[i];
        h64[2 * nt + i] = grav->g[i];
        h64[3 * nt + i] = opt->heat ? opt->heat[i] : 0.0;
        h64[4 * nt + i] = opt->damp ? opt->damp[i] : 0.0;
    }
    for (size_t i = 0; i < h64.size(); ++i) h32[i] = (float)h64[i];
    // FP32 pass tables, one float4 per point: {rho0, p0, g, 0} and {heat, damp, 0, 0}
    // on the z grid (plane-parallel) or on a uniform grid in r^2 (central; g/r
    // stored, so a pass needs neither a square root nor a division)
    std::vector<float4> h4;
    {
        auto lerp = [&](const double *t, double s) {
            const double u = (s - grav->s0) / grav->ds;
            const double fl = std::min(std::max(std::floor(u), 0.0), (double)(nt - 2));
            const int i = (int)fl;
            const double w = u - fl;
            return t[i] + w * (t[i + 1] - t[i]);
        };
        const double *heat = opt->heat, *damp = opt->damp;
        if (grav->kind == PPM_GRAV_CENTRAL) {
            const int n4 = 16384;
            const double r_end = grav->s0 + (nt - 1) * grav->ds;
            const double ds4 = r_end * r_end / (n4 - 1);
            c->ntab4 = n4;
            c->s4_0 = 0.0f;
            c->inv_ds4 = (float)(1.0 / ds4);
            h4.resize(2 * (size_t)n4);
            for (int j = 0; j < n4; ++j) {
                const double r = std::sqrt(j * ds4);
                const double rr = (j == 0) ? std::sqrt(ds4) : r;
                h4[j] = make_float4((float)lerp(grav->rho0, r), (float)lerp(grav->p0, r),
                                    (float)(lerp(grav->g, rr) / rr), 0.0f);
                h4[n4 + j] = make_float4(heat ? (float)lerp(heat, r) : 0.0f, damp ? (float)lerp(damp, r) : 0.0f,
                                         0.0f, 0.0f);
            }
        } else {
            c->ntab4 = nt;
            c->s4_0 = (float)grav->s0;
            c->inv_ds4 = (float)(1.0 / grav->ds);
            h4.resize(2 * (size_t)nt);
            for (int j = 0; j < nt; ++j) {
                h4[j] = make_float4((float)grav->rho0[j], (float)grav->p0[j], (float)grav->g[j], 0.0f);
                h4[nt + j] = make_float4(heat ? (float)heat[j] : 0.0f, damp ? (float)damp[j] : 0.0f, 0.0f, 0.0f);
            }
        }
    }
    // stage (allocated on the first host transfer): up to 2^24 cells per
    // variable (9 x 128 MiB), or the whole grid if smaller
    c->stage_cells = std::min<long long>(c->ncell, 1LL << 24);
    if (cudaMalloc(&c->t64, h64.size() * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->t4, h4.size() * sizeof(float4)) != cudaSuccess ||
        cudaMalloc(&c->t32, h32.size() * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&c->ds_dev, sizeof(DevScal)) != cudaSuccess ||
        cudaMalloc(&c->diag_acc, (8 + 6 * MAX_BINS + 2) * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        fail(c, PPM_ENOMEM, "cannot allocate tables / accumulators");
        return bail(PPM_ENOMEM);
    }
    if (cudaMemcpy(c->t64, h64.data(), h64.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->t32, h32.data(), h32.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->t4, h4.data(), h4.size() * sizeof(float4), cudaMemcpyHostToDevice) != cudaSuccess ||
        prepare_sweep_f32() != cudaSuccess || prepare_sweep_f64() != cudaSuccess ||
        prepare_sweep_ensemble() != cudaSuccess ||
        cudaFuncSetAttribute(divergence_ring_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             div_ring_smem()) != cudaSuccess ||
        cudaFuncSetAttribute(divergence_vel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             div_vel_smem()) != cudaSuccess ||
        cudaMemset(c->ds_dev, 0, sizeof(DevScal)) != cudaSuccess ||
        cudaMemset(c->state, 0, sbytes) != cudaSuccess) {
        fail(c, PPM_ECUDA, "initialising device buffers failed");
        return bail(PPM_ECUDA);
    }
    // the tile form of the pass: FP32 four-value state, no confining sphere
    // or shock dissipation, and rows of whole 16-byte groups for TMA
    c->design[0] = c->design[1] = c->design[2] = PPM_PASS_MARCH;
    c->tile_ok = false;
    for (int h = 0; h < 2; ++h)
        if (c->halo[h] && cudaMemset(c->halo[h], 0, (size_t)c->nvar * 4 * (size_t)nx * ny * es) != cudaSuccess) {
            fail(c, PPM_ECUDA, "initialising the halo planes failed");
            return bail(PPM_ECUDA);
        }
    if (c->prec == PPM_FP32_DEVIATION && c->nmom == 3 && !(c->confine_r > 0.0) && !(c->shock_k > 0.0) &&
        nx % 4 == 0 && !c->halo_z) {
        bool ok = prepare_tile_f32() == cudaSuccess;
        for (int a = 0; a < 3 && ok; ++a) ok = tile_encode_map(&c->tmap[a], c->state, nx, ny, nz, a) == 0;
        if (!ok) cudaGetLastError();
        c->tile_ok = ok;
    }
    *out = c;
    return PPM_OK;
}

int ppm_set_pass_designs(ppm_ctx *c, const int design[3]) {
    if (!c || !design) return fail(c, PPM_EINVAL, "null argument");
    for (int a = 0; a < 3; ++a) {
        if (design[a] != PPM_PASS_MARCH && design[a] != PPM_PASS_TILE)
            return fail(c, PPM_EINVAL, "unknown pass design %d (axis %d)", design[a], a);
        if (design[a] == PPM_PASS_TILE && !c->tile_ok)
            return fail(c, PPM_EINVAL, "the tile pass needs the FP32 four-value form, no confining sphere or shock "
                                       "dissipation, and nx %% 4 == 0");
    }
    if (design[0] != c->design[0] || design[1] != c->design[1] || design[2] != c->design[2]) {
        // the step graph holds the pass kernels: capture it again
        if (c->gexec) cudaGraphExecDestroy(c->gexec);
        if (c->graph) cudaGraphDestroy(c->graph);
        c->gexec = nullptr;
        c->graph = nullptr;
        for (int a = 0; a < 3; ++a) c->design[a] = design[a];
    }
    return PPM_OK;
}

int ppm_set_pass_design(ppm_ctx *c, int design) {
    const int d[3] = {design, design, design};
    return ppm_set_pass_designs(c, d);
}

int ppm_get_pass_design(const ppm_ctx *c, int design[3], int *tile_available) {
    if (!c) return PPM_EINVAL;
    if (design)
        for (int a = 0; a < 3; ++a) design[a] = c->design[a];
    if (tile_available) *tile_available = c->tile_ok ? 1 : 0;
    return PPM_OK;
}

// Signature of what the pass timing depends on: GPU, extents, precision,
// gravity kind, boundaries, sources, PPB form.
static std::string ctx_signature(const ppm_ctx *c) {
    cudaDeviceProp prop;
    char name[256] = "gpu";
    if (cudaGetDeviceProperties(&prop, c->device) == cudaSuccess) snprintf(name, sizeof(name), "%s", prop.name);
    else cudaGetLastError();
    char buf[512];
    snprintf(buf, sizeof(buf), "%s|%d %d %d|prec %d|grav %d|bc %d%d%d%d%d%d|src %d%d|nmom %d", name, c->n[0], c->n[1],
             c->n[2], c->prec, c->grav, c->bc[0], c->bc[1], c->bc[2], c->bc[3], c->bc[4], c->bc[5], c->has_heat,
             c->has_damp, c->nmom);
    for (char *q = buf; *q; ++q)
        if (*q == '\t' || *q == '\n') *q = ' ';
    return buf;
}

int ppm_tune(ppm_ctx *c, const char *cache_path, int *from_cache) {
    if (!c) return PPM_EINVAL;
    if (from_cache) *from_cache = 0;
    if (!c->tile_ok) return PPM_OK;   // one design applies: nothing to choose
    const std::string key = ctx_signature(c);
    if (cache_path) {
        FILE *f = fopen(cache_path, "r");
        if (f) {
            char line[1024];
            while (fgets(line, sizeof(line), f)) {
                char *tab = strchr(line, '\t');
                if (!tab) continue;
                *tab = 0;
                if (key != line) continue;
                int d[3];
                if (sscanf(tab + 1, "%d %d %d", &d[0], &d[1], &d[2]) == 3) {
                    fclose(f);
                    if (from_cache) *from_cache = 1;
                    return ppm_set_pass_designs(c, d);
                }
            }
            fclose(f);
        }
    }
    // snapshot the state, time each design's pass along each axis on the real
    // data (three launches, the first a warm-up), restore after every launch
    const size_t bytes = (size_t)c->nvar * c->ncell * (c->prec == PPM_FP32_DEVIATION ? 4 : 8);
    void *snap = nullptr;
    if (cudaMalloc(&snap, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, PPM_ENOMEM, "the tuner needs a copy of the state (%zu bytes)", bytes);
    }
    int rc = PPM_OK;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (cudaMemcpyAsync(snap, c->state, bytes, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess ||
        cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess)
        rc = fail(c, PPM_ECUDA, "tuner set-up failed");
    double dtc = 0.0;
    if (rc == PPM_OK && ppm_cfl_dt(c, 0.5, &dtc) != PPM_OK)
        rc = fail(c, PPM_ENONPHYS, "no valid state to tune on");
    if (rc == PPM_OK) set_scalar_kernel<<<1, 32, 0, c->stream>>>(&c->ds_dev->dt, 0.5 * dtc);
    const int saved[3] = {c->design[0], c->design[1], c->design[2]};
    int best_d[3] = {PPM_PASS_MARCH, PPM_PASS_MARCH, PPM_PASS_MARCH};
    for (int a = 0; a < 3 && rc == PPM_OK; ++a) {
        float best = 1e30f;
        for (int d = PPM_PASS_MARCH; d <= PPM_PASS_TILE && rc == PPM_OK; ++d) {
            c->design[a] = d;
            float ms = 0.0f;
            for (int rep = 0; rep < 3 && rc == PPM_OK; ++rep) {
                cudaEventRecord(t0, c->stream);
                rc = launch_sweep(c, a, 0, 0, 0);
                cudaEventRecord(t1, c->stream);
                if (rc == PPM_OK && cudaMemcpyAsync(c->state, snap, bytes, cudaMemcpyDeviceToDevice, c->stream) !=
                                        cudaSuccess)
                    rc = fail(c, PPM_ECUDA, "tuner restore failed");
                if (rc == PPM_OK && cudaEventSynchronize(t1) != cudaSuccess)
                    rc = fail(c, PPM_ECUDA, "tuner event sync failed");
                float m = 0.0f;
                if (rc == PPM_OK) cudaEventElapsedTime(&m, t0, t1);
                if (rep > 0) ms += m;
            }
            if (rc == PPM_OK && ms < best) {
                best = ms;
                best_d[a] = d;
            }
        }
        c->design[a] = saved[a];
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    cudaStreamSynchronize(c->stream);
    cudaMemsetAsync(&c->ds_dev->flags, 0, sizeof(int), c->stream);
    cudaStreamSynchronize(c->stream);
    cudaFree(snap);
    c->have_speed = false;
    if (rc != PPM_OK) return rc;
    rc = check_flags(c);
    if (rc != PPM_OK) return rc;
    rc = ppm_set_pass_designs(c, best_d);
    if (rc == PPM_OK && cache_path) {
        FILE *f = fopen(cache_path, "a");
        if (f) {
            fprintf(f, "%s\t%d %d %d\n", key.c_str(), best_d[0], best_d[1], best_d[2]);
            fclose(f);
        }
    }
    return rc;
}

int ppm_slab_halo(ppm_ctx *c, int side, void **dev_ptr, size_t *bytes) {
    if (!c || !dev_ptr) return fail(c, PPM_EINVAL, "null argument");
    if (side < 0 || side > 1) return fail(c, PPM_EINVAL, "side must be 0 (low z) or 1 (high z)");
    if (!(c->halo_z & (1 << side))) return fail(c, PPM_EINVAL, "this z face takes no halo planes (halo_z)");
    *dev_ptr = c->halo[side];
    if (bytes)
        *bytes = (size_t)c->nvar * 4 * (size_t)c->n[0] * c->n[1] *
                 (c->prec == PPM_FP32_DEVIATION ? sizeof(float) : sizeof(double));
    return PPM_OK;
}

int ppm_slab_pack(ppm_ctx *c, int side, void *dst_dev) {
    if (!c || !dst_dev) return fail(c, PPM_EINVAL, "null argument");
    if (side < 0 || side > 1) return fail(c, PPM_EINVAL, "side must be 0 (low z) or 1 (high z)");
    const size_t es = (c->prec == PPM_FP32_DEVIATION) ? sizeof(float) : sizeof(double);
    const size_t plane = (size_t)c->n[0] * c->n[1];
    const size_t k0 = side == 0 ? 0 : (size_t)c->n[2] - 4;
    for (int v = 0; v < c->nvar; ++v) {
        const char *src = static_cast<const char *>(c->state) + ((size_t)v * c->ncell + k0 * plane) * es;
        char *dst = static_cast<char *>(dst_dev) + (size_t)v * 4 * plane * es;
        CK(c, cudaMemcpyAsync(dst, src, 4 * plane * es, cudaMemcpyDeviceToDevice, c->stream));
    }
    return PPM_OK;
}

int ppm_pass_times(ppm_ctx *c, double ms[6]) {
    if (!c || !ms) return fail(c, PPM_EINVAL, "null argument");
    if (!c->gexec || !c->pev[0]) return fail(c, PPM_ESTATE, "no double step has run yet");
    CK(c, cudaEventSynchronize(c->pev[6]));
    for (int s = 0; s < 6; ++s) {
        float t = 0.0f;
        CK(c, cudaEventElapsedTime(&t, c->pev[s], c->pev[s + 1]));
        ms[s] = t;
    }
    return PPM_OK;
}


int ppm_set_region(ppm_ctx *c, const int lo[3], const int hi[3], const double *const q[], int mem) {
    return region_io(c, lo, hi, const_cast<double *const *>(q), mem, true);
}

int ppm_get_region(ppm_ctx *c, const int lo[3], const int hi[3], double *const q[], int mem) {
    if (!c) return PPM_EINVAL;
    int r = region_io(c, lo, hi, q, mem, false);
    if (r != PPM_OK) return r;
    return check_flags(c);
}

int ppm_set_state(ppm_ctx *c, const double *const q[]) {
    if (!c) return PPM_EINVAL;
    const int lo[3] = {0, 0, 0};
    return ppm_set_region(c, lo, c->n, q, PPM_MEM_HOST);
}

int ppm_get_state(ppm_ctx *c, double *const q[]) {
    if (!c) return PPM_EINVAL;
    const int lo[3] = {0, 0, 0};
    return ppm_get_region(c, lo, c->n, q, PPM_MEM_HOST);
}

int ppm_cfl_dt(ppm_ctx *c, double cfl, double *dt_out) {
    if (!c) return PPM_EINVAL;
    if (!(cfl > 0.0)) return fail(c, PPM_EINVAL, "cfl must be positive");
    if (cfl > 1.0) return fail(c, PPM_ECFL, "cfl %.3g exceeds 1", cfl);
    set_scalar_kernel<<<1, 32, 0, c->stream>>>(&c->ds_dev->cfl, cfl);
    c->launches++;
    // After a double step the last pass (or the rotation increment) has
    // already taken the maximum signal speed of the new state, and nothing
    // has changed the state since: no pass over the grid is needed.
    if (!c->have_speed) {
        CK(c, cudaMemsetAsync(&c->ds_dev->smax, 0, sizeof(unsigned long long), c->stream));
        const int g = grid_for(c->ncell, 256);
        if (c->prec == PPM_FP32_DEVIATION)
            cfl_kernel<float, false><<<g, 256, 0, c->stream>>>(make_args<float>(c, 0), (const float *)c->state, c->ncell, c->n[0], c->n[1], &c->ds_dev->smax);
        else
            cfl_kernel<double, true><<<g, 256, 0, c->stream>>>(make_args<double>(c, 0), (const double *)c->state, c->ncell, c->n[0], c->n[1], &c->ds_dev->smax);
        c->launches++;
        CK(c, cudaGetLastError());
        c->have_speed = true;
    }
    if (dt_out) {
        int r = check_flags(c);
        if (r != PPM_OK) return r;
        unsigned long long bits = 0;
        CK(c, cudaMemcpyAsync(&bits, &c->ds_dev->smax, sizeof(bits), cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
        double smax;
        memcpy(&smax, &bits, sizeof(double));
        if (!(smax > 0.0) || !std::isfinite(smax)) return fail(c, PPM_ENONPHYS, "max signal speed %g", smax);
        *dt_out = cfl * c->dx / smax;
    }
    return PPM_OK;
}

static int capture_step(ppm_ctx *c) {
    for (int e = 0; e < 7; ++e)
        if (!c->pev[e]) CK(c, cudaEventCreate(&c->pev[e]));
    CK(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    const long long before = c->launches;
    dt_kernel<<<1, 32, 0, c->stream>>>(c->ds_dev, c->dx, -1.0);
    c->launches++;
    const int order[6] = {0, 1, 2, 2, 1, 0};
    int rc = PPM_OK;
    // external event nodes (a plain record inside a capture would only be a
    // dependency marker of the capture)
    cudaError_t er = cudaEventRecordWithFlags(c->pev[0], c->stream, cudaEventRecordExternal);
    for (int s = 0; s < 6 && rc == PPM_OK && er == cudaSuccess; ++s) {
        const int src = (s == 2 || s == 5) ? ((c->has_heat || c->has_damp) ? 1 : 0) : 0;
        // the y and z passes leave the cell velocities for the divergence
        // before the next pass (passes 2..5 take them)
        const int vel = (s >= 1 && s <= 4 ? 1 : 0) | (s >= 2 ? 2 : 0);
        rc = launch_sweep(c, order[s], src, s == 5 ? 1 : 0, vel);
        if (rc == PPM_OK) er = cudaEventRecordWithFlags(c->pev[s + 1], c->stream, cudaEventRecordExternal);
    }
    if (rc == PPM_OK && er != cudaSuccess) rc = fail(c, PPM_ECUDA, "event record in capture: %s", cudaGetErrorString(er));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    c->graph_kernels = c->launches - before;  // captured, not yet launched
    c->launches = before;
    if (rc != PPM_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(c, PPM_ECUDA, "stream capture: %s", cudaGetErrorString(e));
    c->graph = g;
    // the dt kernel is the only node without dependencies
    size_t nn = 0;
    CK(c, cudaGraphGetRootNodes(c->graph, nullptr, &nn));
    if (nn != 1) return fail(c, PPM_ECUDA, "unexpected step graph shape (%zu roots)", nn);
    CK(c, cudaGraphGetRootNodes(c->graph, &c->dt_node, &nn));
    CK(c, cudaGraphInstantiate(&c->gexec, c->graph, 0));
    return PPM_OK;
}

int ppm_step(ppm_ctx *c, double dt) {
    if (!c) return PPM_EINVAL;
    if (!(dt > 0.0) && !c->have_speed)
        return fail(c, PPM_ESTATE, "ppm_step with dt <= 0 needs a device dt (call ppm_cfl_dt first)");
    if (!std::isfinite(dt)) return fail(c, PPM_EINVAL, "dt is not finite");
    if (!c->gexec) {
        int r = capture_step(c);
        if (r != PPM_OK) return r;
    }
    // the explicit dt travels as an argument of the graph's first kernel;
    // updating it does not touch launches already in flight
    {
        DevScal *dsp = c->ds_dev;
        double dxv = c->dx;
        double dtu = dt > 0.0 ? dt : -1.0;
        void *args[3] = {&dsp, &dxv, &dtu};
        cudaKernelNodeParams kp;
        memset(&kp, 0, sizeof(kp));
        kp.func = (void *)dt_kernel;
        kp.gridDim = dim3(1);
        kp.blockDim = dim3(32);
        kp.sharedMemBytes = 0;
        kp.kernelParams = args;
        CK(c, cudaGraphExecKernelNodeSetParams(c->gexec, c->dt_node, &kp));
    }
    CK(c, cudaGraphLaunch(c->gexec, c->stream));
    c->launches += c->graph_kernels;
    c->have_speed = true;
    if (c->domega != 0.0) return launch_rotate(c, true);
    return PPM_OK;
}

int ppm_sweep(ppm_ctx *c, int axis, double dt, int sources) {
    if (!c) return PPM_EINVAL;
    if (axis < 0 || axis > 2) return fail(c, PPM_EINVAL, "axis must be 0, 1 or 2");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, PPM_EINVAL, "dt must be positive");
    set_scalar_kernel<<<1, 32, 0, c->stream>>>(&c->ds_dev->dt, dt);
    c->launches++;
    CK(c, cudaGetLastError());
    if (sources < 0 || sources > 3) return fail(c, PPM_EINVAL, "sources must be 0..3");
    int r = launch_sweep(c, axis, (sources & 1) && (c->has_heat || c->has_damp) ? 1 : 0, 0, 0);
    c->have_speed = false;
    if (r == PPM_OK && (sources & 2) && c->domega != 0.0) r = launch_rotate(c, false);
    return r;
}

int ppm_set_rotation(ppm_ctx *c, double domega) {
    if (!c) return PPM_EINVAL;
    if (!std::isfinite(domega)) return fail(c, PPM_EINVAL, "domega is not finite");
    c->domega = domega;
    return PPM_OK;
}

int ppm_diagnostics(ppm_ctx *c, double totals[7], int nbins, double rmax, double *profiles, double *max_mach) {
    if (!c || !totals) return fail(c, PPM_EINVAL, "null argument");
    if (nbins < 0 || nbins > MAX_BINS) return fail(c, PPM_EINVAL, "nbins must be in [0, %d]", MAX_BINS);
    if (nbins > 0 && (!profiles || !(rmax > 0.0))) return fail(c, PPM_EINVAL, "profiles need rmax > 0 and an output array");
    const size_t nacc = 8 + 6 * (size_t)nbins;
    CK(c, cudaMemsetAsync(c->diag_acc, 0, nacc * sizeof(double), c->stream));
    const int g = grid_for(c->ncell, 256);
    const size_t shm = 6 * (size_t)nbins * sizeof(double);
    const SweepArgs<double> A = args64(c);
    bool cached = false;
    if (c->prec == PPM_FP32_DEVIATION) {
        if (!c->base32 && !c->base32_tried) {
            c->base32_tried = true;
            if (cudaMalloc(&c->base32, 3 * (size_t)c->ncell * sizeof(float)) != cudaSuccess) {
                cudaGetLastError();   // no room: the kernel looks the base state up instead
                c->base32 = nullptr;
            } else {
                double *sums = c->diag_acc + 8 + 6 * MAX_BINS;
                CK(c, cudaMemsetAsync(sums, 0, 2 * sizeof(double), c->stream));
                base_fill_kernel<<<g, 256, 0, c->stream>>>(A, c->base32, c->base32 + c->ncell,
                                                           c->base32 + 2 * c->ncell, sums, c->ncell, c->n[0],
                                                           c->n[1]);
                c->launches++;
                CK(c, cudaGetLastError());
                CK(c, cudaMemcpyAsync(c->base_sum, sums, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
                CK(c, cudaStreamSynchronize(c->stream));
            }
        }
        cached = c->base32 != nullptr;
        if (cached) {
            if (shm > 48 * 1024) CK(c, cudaFuncSetAttribute(diag32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
            diag32_kernel<<<g, 256, shm, c->stream>>>(A, (const float *)c->state, c->ncell, c->n[0], c->n[1], nbins,
                                                      rmax, c->diag_acc, c->base32, c->base32 + c->ncell,
                                                      c->base32 + 2 * c->ncell);
        } else {
            if (shm > 48 * 1024) CK(c, cudaFuncSetAttribute(diag_kernel<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
            diag_kernel<float, false><<<g, 256, shm, c->stream>>>(A, (const float *)c->state, c->ncell, c->n[0], c->n[1], nbins, rmax, c->diag_acc);
        }
    } else {
        if (shm > 48 * 1024) CK(c, cudaFuncSetAttribute(diag_kernel<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
        diag_kernel<double, true><<<g, 256, shm, c->stream>>>(A, (const double *)c->state, c->ncell, c->n[0], c->n[1], nbins, rmax, c->diag_acc);
    }
    c->launches++;
    CK(c, cudaGetLastError());
    std::vector<double> h(nacc);
    CK(c, cudaMemcpyAsync(h.data(), c->diag_acc, nacc * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    const double dV = c->dx * c->dx * c->dx;
    if (cached) {   // the kernel summed rho' and E'
        h[0] += c->base_sum[0];
        h[4] += c->base_sum[1];
    }
    for (int m = 0; m < 7; ++m) totals[m] = h[m] * dV;
    for (int b = 0; b < nbins; ++b) {
        const double *a = &h[8 + 6 * b];
        for (int m = 0; m < 5; ++m) profiles[5 * b + m] = a[0] > 0.0 ? a[1 + m] / a[0] : 0.0;
    }
    if (max_mach) *max_mach = std::sqrt(h[7]);   // the kernel maximises Mach^2
    return check_flags(c);
}

int ppm_sync(ppm_ctx *c) {
    if (!c) return PPM_EINVAL;
    CK(c, cudaStreamSynchronize(c->stream));
    return check_flags(c);
}

long long ppm_launch_count(const ppm_ctx *c) { return c ? c->launches : 0; }

const char *ppm_last_error(const ppm_ctx *c) { return c ? c->err.c_str() : g_create_error.c_str(); }

void ppm_destroy(ppm_ctx *c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    release(c);
    delete c;
}

}  // extern "C"

// ===========================================================================
// Ensembles of independent boxes (one launch per pass for all boxes)
// ===========================================================================
struct ppm_ens {
    int nbox = 0;
    int prec = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<ppm_ctx *> box;
    void *d_args = nullptr;         // SweepArgs<R>[6 passes][nbox]
    size_t args_bytes = 0;
    WorkItem *d_work = nullptr;     // work lists, [axis][variant] slices
    int work_off[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    int nwork[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    int *d_counters = nullptr;      // [6 passes][2 variants], then ticket, sentinel, done[6][nbox]
    bool one_launch = false;        // the whole double step in one launch (besides the dt kernel)
    int wait_test = 0;              // tests only: the first item of each block waits for nothing that comes
    WorkItem *d_work1 = nullptr;    // one-launch work list: all passes in order, pad = pass * 2 + vec
    int nwork1 = 0;
    int *d_need = nullptr;          // items per (pass, box)
    int bps1 = 1;                   // resident blocks per SM of the one-launch kernel
    DevScal **d_ds = nullptr;
    double *d_dx = nullptr;
    int cfg_nb[3] = {128, 128, 128};
    int cfg_pers[3] = {1, 1, 1};
    int cfg_vec = 1;
    int bps[2][3] = {{1, 1, 1}, {1, 1, 1}};   // resident blocks per SM: [vec][32, 64, 128 pencils]
    int nsm = 152;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaGraphNode_t dt_node = nullptr;
    bool have_speed = false;
    long long launches = 0;
    std::string err;
};

namespace {

constexpr int ENS_PASS_AXIS[6] = {0, 1, 2, 2, 1, 0};

int efail(ppm_ens *e, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (e)
        e->err = buf;
    else
        g_create_error = buf;
    return code;
}

#define ECK(ens, call)                                                                         \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return efail((ens), PPM_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),     \
                         __FILE__, __LINE__);                                                  \
    } while (0)

// dt of every box for the next step, clearing the running maxima and the
// work counters of the persistent passes.
__global__ void ens_dt_kernel(DevScal *const *ds, const double *dx, int nbox, int *counters, int ncounters,
                              double dt_user) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nbox; b += gridDim.x * blockDim.x) {
        DevScal *s = ds[b];
        const double smax = __longlong_as_double((long long)s->smax);
        s->dt = (dt_user > 0.0) ? dt_user : s->cfl * dx[b] / smax;
        s->smax = 0ull;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncounters; i += gridDim.x * blockDim.x) counters[i] = 0;
}

__global__ void zero_ints_kernel(int *p, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = 0;
}

int pencils_along(const ppm_ctx *c, int axis, int *nlane, int *nblk) {
    if (axis == 0) {
        *nlane = c->n[1];
        *nblk = c->n[2];
    } else if (axis == 1) {
        *nlane = c->n[0];
        *nblk = c->n[2];
    } else {
        *nlane = c->n[0];
        *nblk = c->n[1];
    }
    return c->n[axis];
}

bool box_vec_ok(const ppm_ens *e, int b) { return e->prec == PPM_FP32_DEVIATION && (e->box[b]->n[0] % 8) == 0; }

// Work lists for the current configuration: longest pencils first.
int build_work(ppm_ens *e) {
    std::vector<WorkItem> all;
    for (int a = 0; a < 3; ++a) {
        for (int var = 0; var < 2; ++var) {
            std::vector<WorkItem> items;
            for (int b = 0; b < e->nbox; ++b) {
                const bool v = (a == 0) && e->cfg_vec && box_vec_ok(e, b);
                if ((var == 1) != v) continue;
                const int nb = e->cfg_nb[a];
                int nlane, nblk;
                pencils_along(e->box[b], a, &nlane, &nblk);
                const int nlb = (nlane + nb - 1) / nb;
                for (int k = 0; k < nblk; ++k)
                    for (int l = 0; l < nlb; ++l) items.push_back(WorkItem{b, l, k, 0});
            }
            std::stable_sort(items.begin(), items.end(), [&](const WorkItem &x, const WorkItem &y) {
                return e->box[x.box]->n[a] > e->box[y.box]->n[a];
            });
            e->work_off[a][var] = (int)all.size();
            e->nwork[a][var] = (int)items.size();
            all.insert(all.end(), items.begin(), items.end());
        }
    }
    if (e->d_work) cudaFree(e->d_work);
    e->d_work = nullptr;
    ECK(e, cudaMalloc(&e->d_work, std::max<size_t>(1, all.size()) * sizeof(WorkItem)));
    ECK(e, cudaMemcpy(e->d_work, all.data(), all.size() * sizeof(WorkItem), cudaMemcpyHostToDevice));
    // one-launch list: the six passes in order, 128-pencil blocks, longest
    // pencils first within a pass; need[s][b] = items of pass s of box b
    {
        std::vector<WorkItem> list;
        std::vector<int> need((size_t)6 * e->nbox, 0);
        for (int s = 0; s < 6; ++s) {
            const int a = ENS_PASS_AXIS[s];
            std::vector<WorkItem> items;
            for (int b = 0; b < e->nbox; ++b) {
                const int v = ((a == 0) && e->cfg_vec && box_vec_ok(e, b)) ? 1 : 0;
                int nlane, nblk;
                pencils_along(e->box[b], a, &nlane, &nblk);
                const int nlb = (nlane + 127) / 128;
                for (int k = 0; k < nblk; ++k)
                    for (int l = 0; l < nlb; ++l) items.push_back(WorkItem{b, l, k, s * 2 + v});
                need[(size_t)s * e->nbox + b] = nblk * nlb;
            }
            std::stable_sort(items.begin(), items.end(), [&](const WorkItem &x, const WorkItem &y) {
                return e->box[x.box]->n[a] > e->box[y.box]->n[a];
            });
            list.insert(list.end(), items.begin(), items.end());
        }
        if (e->d_work1) cudaFree(e->d_work1);
        e->d_work1 = nullptr;
        e->nwork1 = (int)list.size();
        ECK(e, cudaMalloc(&e->d_work1, std::max<size_t>(1, list.size()) * sizeof(WorkItem)));
        ECK(e, cudaMemcpy(e->d_work1, list.data(), list.size() * sizeof(WorkItem), cudaMemcpyHostToDevice));
        if (!e->d_need) ECK(e, cudaMalloc(&e->d_need, need.size() * sizeof(int)));
        ECK(e, cudaMemcpy(e->d_need, need.data(), need.size() * sizeof(int), cudaMemcpyHostToDevice));
    }
    if (e->gexec) cudaGraphExecDestroy(e->gexec);
    if (e->graph) cudaGraphDestroy(e->graph);
    e->gexec = nullptr;
    e->graph = nullptr;
    return PPM_OK;
}

// Launch one pass (both variants) of every box.
int ens_launch_pass(ppm_ens *e, int pass) {
    const int a = ENS_PASS_AXIS[pass];
    const int f32 = e->prec == PPM_FP32_DEVIATION;
    const size_t asz = f32 ? sizeof(SweepArgs<float>) : sizeof(SweepArgs<double>);
    const void *args = static_cast<const char *>(e->d_args) + (size_t)pass * e->nbox * asz;
    for (int var = 1; var >= 0; --var) {
        const int nw = e->nwork[a][var];
        if (nw == 0) continue;
        const int vec = var;
        const int nb = f32 ? e->cfg_nb[a] : 128;
        const int pers = e->cfg_pers[a];
        int grid = nw;
        if (pers) grid = std::min(nw, e->nsm * e->bps[vec][nb == 32 ? 0 : (nb == 64 ? 1 : 2)]);
        // passes 2 and 5 carry the sources, pass 5 the CFL maximum
        const int nsrc = (pass != 2 && pass != 5) ? 1 : 0;
        launch_sweep_ensemble(f32, vec, nb, nsrc, args, e->d_work + e->work_off[a][var], nw,
                              e->d_counters + pass * 2 + var, pers, grid, e->stream);
        e->launches++;
        ECK(e, cudaGetLastError());
    }
    return PPM_OK;
}

int ens_ncounters(const ppm_ens *e) { return 14 + 6 * e->nbox; }

// The whole double step of every box as one launch of the step kernel.
int ens_launch_step(ppm_ens *e) {
    const int f32 = e->prec == PPM_FP32_DEVIATION;
    const int grid = std::max(1, std::min(e->nwork1, e->nsm * e->bps1));
    int *ctr = e->d_counters + 12;
    launch_ensemble_step(f32, e->d_args, e->nbox, e->d_work1, e->nwork1, ctr, ctr + 2, e->d_need, e->wait_test, grid,
                         e->stream);
    e->launches++;
    ECK(e, cudaGetLastError());
    return PPM_OK;
}

int ens_capture(ppm_ens *e) {
    ECK(e, cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal));
    ens_dt_kernel<<<1, 256, 0, e->stream>>>(e->d_ds, e->d_dx, e->nbox, e->d_counters, ens_ncounters(e), -1.0);
    int rc = PPM_OK;
    const long long l0 = e->launches;
    if (e->one_launch)
        rc = ens_launch_step(e);
    else
        for (int s = 0; s < 6 && rc == PPM_OK; ++s) rc = ens_launch_pass(e, s);
    e->launches = l0;
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(e->stream, &g);
    if (rc != PPM_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (ce != cudaSuccess) return efail(e, PPM_ECUDA, "stream capture: %s", cudaGetErrorString(ce));
    e->graph = g;
    size_t nn = 0;
    ECK(e, cudaGraphGetRootNodes(e->graph, nullptr, &nn));
    if (nn != 1) return efail(e, PPM_ECUDA, "unexpected ensemble graph shape (%zu roots)", nn);
    ECK(e, cudaGraphGetRootNodes(e->graph, &e->dt_node, &nn));
    ECK(e, cudaGraphInstantiate(&e->gexec, e->graph, 0));
    return PPM_OK;
}

int graph_launches_per_step(const ppm_ens *e) {
    if (e->one_launch) return 2;
    int n = 1;
    for (int s = 0; s < 6; ++s)
        for (int var = 0; var < 2; ++var) n += e->nwork[ENS_PASS_AXIS[s]][var] > 0 ? 1 : 0;
    return n;
}

void ens_release(ppm_ens *e) {
    if (e->stream) cudaStreamSynchronize(e->stream);
    if (e->gexec) cudaGraphExecDestroy(e->gexec);
    if (e->graph) cudaGraphDestroy(e->graph);
    for (ppm_ctx *c : e->box) ppm_destroy(c);
    e->box.clear();
    if (e->d_args) cudaFree(e->d_args);
    if (e->d_work) cudaFree(e->d_work);
    if (e->d_counters) cudaFree(e->d_counters);
    if (e->d_work1) cudaFree(e->d_work1);
    if (e->d_need) cudaFree(e->d_need);
    if (e->d_ds) cudaFree(e->d_ds);
    if (e->d_dx) cudaFree(e->d_dx);
    if (e->own_stream && e->stream) cudaStreamDestroy(e->stream);
}

std::string ens_signature(const ppm_ens *e) {
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, e->device);
    std::vector<std::string> shapes;
    for (const ppm_ctx *c : e->box) {
        char b[64];
        snprintf(b, sizeof(b), "%dx%dx%d", c->n[0], c->n[1], c->n[2]);
        shapes.push_back(b);
    }
    std::sort(shapes.begin(), shapes.end());
    std::string key = std::string(prop.name) + "|prec" + std::to_string(e->prec) + "|";
    for (size_t i = 0; i < shapes.size(); ++i) key += (i ? "," : "") + shapes[i];
    for (char &ch : key)
        if (ch == ' ' || ch == '\t') ch = '_';
    return key;
}

}  // namespace

extern "C" {

int ppm_ensemble_create(ppm_ens **out, int nbox, const ppm_box *boxes, double gamma, int precision, void *stream,
                        int device) {
    if (!out || !boxes) return efail(nullptr, PPM_EINVAL, "null argument");
    *out = nullptr;
    if (nbox < 1 || nbox > 4096) return efail(nullptr, PPM_EINVAL, "nbox must be in [1, 4096]");
    if (precision != PPM_FP64_PLAIN && precision != PPM_FP32_DEVIATION)
        return efail(nullptr, PPM_EINVAL, "bad precision");
    ppm_ens *e = new ppm_ens();
    e->nbox = nbox;
    e->prec = precision;
    e->device = device;
    auto bail = [&](int code) {
        std::string m = e->err;
        ens_release(e);
        delete e;
        g_create_error = m;
        return code;
    };
    if (cudaSetDevice(device) != cudaSuccess) {
        efail(e, PPM_ECUDA, "cudaSetDevice(%d) failed", device);
        return bail(PPM_ECUDA);
    }
    if (stream) {
        e->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking) != cudaSuccess) {
            efail(e, PPM_ECUDA, "cudaStreamCreate failed");
            return bail(PPM_ECUDA);
        }
        e->own_stream = true;
    }
    for (int b = 0; b < nbox; ++b) {
        const ppm_box &B = boxes[b];
        ppm_options opt;
        memset(&opt, 0, sizeof(opt));
        opt.x0 = B.x0;
        opt.y0 = B.y0;
        opt.z0 = B.z0;
        opt.dx = B.dx;
        opt.precision = precision;
        opt.heat = B.heat;
        opt.damp = B.damp;
        opt.stream = e->stream;
        opt.device = device;
        ppm_ctx *c = nullptr;
        const int rc = ppm_create(&c, B.n[0], B.n[1], B.n[2], gamma, B.bc, &B.grav, &opt);
        if (rc != PPM_OK) {
            efail(e, rc, "box %d: %s", b, g_create_error.c_str());
            return bail(rc);
        }
        e->box.push_back(c);
    }
    // per-pass argument arrays
    const int f32 = precision == PPM_FP32_DEVIATION;
    const size_t asz = f32 ? sizeof(SweepArgs<float>) : sizeof(SweepArgs<double>);
    std::vector<char> h((size_t)6 * nbox * asz);
    for (int s = 0; s < 6; ++s)
        for (int b = 0; b < nbox; ++b) {
            ppm_ctx *c = e->box[b];
            const int src = (s == 2 || s == 5) ? ((c->has_heat || c->has_damp) ? 1 : 0) : 0;
            char *dst = h.data() + ((size_t)s * nbox + b) * asz;
            if (f32) {
                SweepArgs<float> a = make_args<float>(c, ENS_PASS_AXIS[s]);
                a.sources = src;
                a.cfl = (s == 5);
                memcpy(dst, &a, asz);
            } else {
                SweepArgs<double> a = make_args<double>(c, ENS_PASS_AXIS[s]);
                a.sources = src;
                a.cfl = (s == 5);
                memcpy(dst, &a, asz);
            }
        }
    std::vector<DevScal *> hds(nbox);
    std::vector<double> hdx(nbox);
    for (int b = 0; b < nbox; ++b) {
        hds[b] = e->box[b]->ds_dev;
        hdx[b] = e->box[b]->dx;
    }
    if (cudaMalloc(&e->d_args, h.size()) != cudaSuccess ||
        cudaMalloc(&e->d_counters, (size_t)(14 + 6 * nbox) * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&e->d_ds, nbox * sizeof(DevScal *)) != cudaSuccess ||
        cudaMalloc(&e->d_dx, nbox * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        efail(e, PPM_ENOMEM, "cannot allocate ensemble tables");
        return bail(PPM_ENOMEM);
    }
    e->args_bytes = h.size();
    if (cudaMemcpy(e->d_args, h.data(), h.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(e->d_ds, hds.data(), nbox * sizeof(DevScal *), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(e->d_dx, hdx.data(), nbox * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(e->d_counters, 0, (size_t)(14 + 6 * nbox) * sizeof(int)) != cudaSuccess ||
        prepare_ensemble_step() != cudaSuccess) {
        efail(e, PPM_ECUDA, "initialising ensemble tables failed");
        return bail(PPM_ECUDA);
    }
    {
        int nsm = 0;
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
        e->nsm = nsm > 0 ? nsm : 152;
        for (int v = 0; v < 2; ++v)
            for (int i = 0; i < 3; ++i) e->bps[v][i] = ensemble_blocks_per_sm(f32, v, 32 << i);
        e->bps1 = ensemble_step_blocks_per_sm(f32);
    }
    const int rc = build_work(e);
    if (rc != PPM_OK) return bail(rc);
    *out = e;
    return PPM_OK;
}

int ppm_ensemble_set_state(ppm_ens *e, int b, const double *const q[9]) {
    if (!e || b < 0 || b >= e->nbox) return efail(e, PPM_EINVAL, "bad ensemble or box index");
    const int rc = ppm_set_state(e->box[b], q);
    if (rc != PPM_OK) return efail(e, rc, "box %d: %s", b, e->box[b]->err.c_str());
    e->have_speed = false;
    return PPM_OK;
}

int ppm_ensemble_set_region(ppm_ens *e, int b, const int lo[3], const int hi[3], const double *const q[9], int mem) {
    if (!e || b < 0 || b >= e->nbox) return efail(e, PPM_EINVAL, "bad ensemble or box index");
    const int rc = ppm_set_region(e->box[b], lo, hi, q, mem);
    if (rc != PPM_OK) return efail(e, rc, "box %d: %s", b, e->box[b]->err.c_str());
    e->have_speed = false;
    return PPM_OK;
}

int ppm_ensemble_get_state(ppm_ens *e, int b, double *const q[9]) {
    if (!e || b < 0 || b >= e->nbox) return efail(e, PPM_EINVAL, "bad ensemble or box index");
    const int rc = ppm_get_state(e->box[b], q);
    if (rc != PPM_OK) return efail(e, rc, "box %d: %s", b, e->box[b]->err.c_str());
    return PPM_OK;
}

int ppm_ensemble_cfl_dt(ppm_ens *e, double cfl, double *dt_out) {
    if (!e) return PPM_EINVAL;
    for (int b = 0; b < e->nbox; ++b) {
        const int rc = ppm_cfl_dt(e->box[b], cfl, dt_out ? dt_out + b : nullptr);
        if (rc != PPM_OK) return efail(e, rc, "box %d: %s", b, e->box[b]->err.c_str());
        e->launches += 2;
    }
    e->have_speed = true;
    return PPM_OK;
}

int ppm_ensemble_step(ppm_ens *e, double dt) {
    if (!e) return PPM_EINVAL;
    if (!(dt > 0.0) && !e->have_speed)
        return efail(e, PPM_ESTATE, "ppm_ensemble_step with dt <= 0 needs device dts (call ppm_ensemble_cfl_dt)");
    if (!std::isfinite(dt)) return efail(e, PPM_EINVAL, "dt is not finite");
    if (!e->gexec) {
        const int rc = ens_capture(e);
        if (rc != PPM_OK) return rc;
    }
    DevScal **dsp = e->d_ds;
    const double *dxp = e->d_dx;
    int nb = e->nbox, *ctr = e->d_counters, nctr = ens_ncounters(e);
    double dtu = dt > 0.0 ? dt : -1.0;
    void *args[6] = {&dsp, &dxp, &nb, &ctr, &nctr, &dtu};
    cudaKernelNodeParams kp;
    memset(&kp, 0, sizeof(kp));
    kp.func = (void *)ens_dt_kernel;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(256);
    kp.kernelParams = args;
    ECK(e, cudaGraphExecKernelNodeSetParams(e->gexec, e->dt_node, &kp));
    ECK(e, cudaGraphLaunch(e->gexec, e->stream));
    e->launches += graph_launches_per_step(e);
    e->have_speed = true;
    return PPM_OK;
}

int ppm_ensemble_diagnostics(ppm_ens *e, int b, double totals[7], double *max_mach) {
    if (!e || b < 0 || b >= e->nbox) return efail(e, PPM_EINVAL, "bad ensemble or box index");
    const int rc = ppm_diagnostics(e->box[b], totals, 0, 1.0, nullptr, max_mach);
    if (rc != PPM_OK) return efail(e, rc, "box %d: %s", b, e->box[b]->err.c_str());
    e->launches += 1;
    return PPM_OK;
}

int ppm_ensemble_sync(ppm_ens *e) {
    if (!e) return PPM_EINVAL;
    // every box's flags are read and cleared; the first error is reported
    int first = PPM_OK;
    for (int b = 0; b < e->nbox; ++b) {
        const int rc = ppm_sync(e->box[b]);
        if (rc != PPM_OK && first == PPM_OK) {
            first = rc;
            efail(e, rc, "box %d: %s", b, e->box[b]->err.c_str());
        }
    }
    return first;
}

int ppm_ensemble_set_config(ppm_ens *e, int axis, int block, int persistent, int vec) {
    if (!e || axis < 0 || axis > 2) return efail(e, PPM_EINVAL, "bad axis");
    if (block != 32 && block != 64 && block != 128) return efail(e, PPM_EINVAL, "block must be 32, 64 or 128");
    if (e->prec != PPM_FP32_DEVIATION && block != 128) return efail(e, PPM_EINVAL, "FP64 passes use 128-thread blocks");
    e->cfg_nb[axis] = block;
    e->cfg_pers[axis] = persistent ? 1 : 0;
    if (axis == 0) e->cfg_vec = vec ? 1 : 0;
    return build_work(e);
}

int ppm_ensemble_set_launch_mode(ppm_ens *e, int mode) {
    if (!e) return PPM_EINVAL;
    if (mode != PPM_ENS_PER_PASS && mode != PPM_ENS_ONE_LAUNCH) return efail(e, PPM_EINVAL, "unknown launch mode %d", mode);
    if ((mode == PPM_ENS_ONE_LAUNCH) != e->one_launch) {
        if (e->gexec) cudaGraphExecDestroy(e->gexec);
        if (e->graph) cudaGraphDestroy(e->graph);
        e->gexec = nullptr;
        e->graph = nullptr;
        e->one_launch = (mode == PPM_ENS_ONE_LAUNCH);
    }
    return PPM_OK;
}

int ppm_ensemble_get_launch_mode(const ppm_ens *e) {
    return e ? (e->one_launch ? PPM_ENS_ONE_LAUNCH : PPM_ENS_PER_PASS) : PPM_EINVAL;
}

int ppm_ensemble_set_wait_test(ppm_ens *e, int on) {
    if (!e) return PPM_EINVAL;
    if ((on != 0) != (e->wait_test != 0)) {
        if (e->gexec) cudaGraphExecDestroy(e->gexec);
        if (e->graph) cudaGraphDestroy(e->graph);
        e->gexec = nullptr;
        e->graph = nullptr;
        e->wait_test = on ? 1 : 0;
    }
    return PPM_OK;
}

int ppm_ensemble_get_config(const ppm_ens *e, int cfg[7]) {
    if (!e || !cfg) return PPM_EINVAL;
    for (int a = 0; a < 3; ++a) {
        cfg[2 * a] = e->cfg_nb[a];
        cfg[2 * a + 1] = e->cfg_pers[a];
    }
    cfg[6] = e->cfg_vec;
    return PPM_OK;
}

int ppm_ensemble_tune(ppm_ens *e, const char *cache_path, int *from_cache) {
    if (!e) return PPM_EINVAL;
    if (from_cache) *from_cache = 0;
    const std::string key = ens_signature(e);
    if (cache_path) {
        FILE *f = fopen(cache_path, "r");
        if (f) {
            char line[8192];
            while (fgets(line, sizeof(line), f)) {
                char *tab = strchr(line, '\t');
                if (!tab) continue;
                *tab = 0;
                if (key != line) continue;
                int v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                const int nv = sscanf(tab + 1, "%d %d %d %d %d %d %d %d", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5],
                                      &v[6], &v[7]);
                if (nv == 7 || nv == 8) {
                    fclose(f);
                    for (int a = 0; a < 3; ++a) {
                        e->cfg_nb[a] = v[2 * a];
                        e->cfg_pers[a] = v[2 * a + 1];
                    }
                    e->cfg_vec = v[6];
                    if (from_cache) *from_cache = 1;
                    const int rc = build_work(e);
                    return rc != PPM_OK ? rc : ppm_ensemble_set_launch_mode(e, v[7] ? PPM_ENS_ONE_LAUNCH : PPM_ENS_PER_PASS);
                }
            }
            fclose(f);
        }
    }
    // snapshot the states, time every candidate on the real data, restore
    std::vector<void *> snap(e->nbox, nullptr);
    size_t total = 0;
    for (ppm_ctx *c : e->box) total += (size_t)c->nvar * c->ncell * (e->prec == PPM_FP32_DEVIATION ? 4 : 8);
    char *scratch = nullptr;
    ECK(e, cudaMalloc(&scratch, total));
    auto copy_all = [&](bool save) -> int {
        size_t off = 0;
        for (ppm_ctx *c : e->box) {
            const size_t bytes = (size_t)c->nvar * c->ncell * (e->prec == PPM_FP32_DEVIATION ? 4 : 8);
            ECK(e, cudaMemcpyAsync(save ? scratch + off : c->state, save ? c->state : scratch + off, bytes,
                                   cudaMemcpyDeviceToDevice, e->stream));
            off += bytes;
        }
        return PPM_OK;
    };
    int rc = copy_all(true);
    // a valid dt for every box: half the CFL-0.5 step of the current state
    for (int b = 0; b < e->nbox && rc == PPM_OK; ++b) {
        double dtb = 0.0;
        if (ppm_cfl_dt(e->box[b], 0.5, &dtb) != PPM_OK) rc = efail(e, PPM_ENONPHYS, "box %d has no valid state to tune on", b);
        else set_scalar_kernel<<<1, 32, 0, e->stream>>>(&e->box[b]->ds_dev->dt, 0.5 * dtb);
    }
    const bool f32 = e->prec == PPM_FP32_DEVIATION;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (rc == PPM_OK && (cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess))
        rc = efail(e, PPM_ECUDA, "cudaEventCreate failed");
    for (int a = 0; a < 3 && rc == PPM_OK; ++a) {
        float best = 1e30f;
        int bnb = 128, bpers = 1, bvec = e->cfg_vec;
        const int nbs[3] = {32, 64, 128};
        for (int vec = (a == 0 && f32) ? 1 : e->cfg_vec; vec >= 0 && rc == PPM_OK; --vec) {
            for (int ib = (f32 ? 0 : 2); ib < 3 && rc == PPM_OK; ++ib) {
                for (int pers = 0; pers < 2 && rc == PPM_OK; ++pers) {
                    e->cfg_nb[a] = nbs[ib];
                    e->cfg_pers[a] = pers;
                    if (a == 0) e->cfg_vec = vec;
                    if ((rc = build_work(e)) != PPM_OK) break;
                    const int pass = a;  // passes 0, 1, 2 are x, y, z
                    float ms = 0.0f;
                    for (int rep = 0; rep < 3 && rc == PPM_OK; ++rep) {
                        zero_ints_kernel<<<1, 32, 0, e->stream>>>(e->d_counters, 12);
                        cudaEventRecord(t0, e->stream);
                        rc = ens_launch_pass(e, pass);
                        cudaEventRecord(t1, e->stream);
                        if (rc == PPM_OK) rc = copy_all(false);
                        if (cudaEventSynchronize(t1) != cudaSuccess) rc = efail(e, PPM_ECUDA, "event sync failed");
                        float m = 0.0f;
                        cudaEventElapsedTime(&m, t0, t1);
                        if (rep > 0) ms += m;  // first repetition warms up
                    }
                    if (rc == PPM_OK && ms < best) {
                        best = ms;
                        bnb = nbs[ib];
                        bpers = pers;
                        bvec = (a == 0) ? vec : e->cfg_vec;
                    }
                }
            }
        }
        e->cfg_nb[a] = bnb;
        e->cfg_pers[a] = bpers;
        if (a == 0) e->cfg_vec = bvec;
    }
    // launch mode: one double step per mode with that configuration (after a
    // warm-up step), the states restored after each
    int best_mode = e->one_launch ? PPM_ENS_ONE_LAUNCH : PPM_ENS_PER_PASS;
    if (rc == PPM_OK) rc = build_work(e);
    double dt_min = 0.0;
    for (int b = 0; b < e->nbox && rc == PPM_OK; ++b) {
        double dtb = 0.0;
        if (ppm_cfl_dt(e->box[b], 0.5, &dtb) != PPM_OK) rc = efail(e, PPM_ENONPHYS, "box %d has no valid state to tune on", b);
        dt_min = (b == 0 || dtb < dt_min) ? dtb : dt_min;
    }
    if (rc == PPM_OK) rc = copy_all(false);
    float best_step = 1e30f;
    for (int mode = PPM_ENS_PER_PASS; mode <= PPM_ENS_ONE_LAUNCH && rc == PPM_OK; ++mode) {
        rc = ppm_ensemble_set_launch_mode(e, mode);
        float ms = 0.0f;
        for (int rep = 0; rep < 2 && rc == PPM_OK; ++rep) {
            cudaEventRecord(t0, e->stream);
            rc = ppm_ensemble_step(e, 0.5 * dt_min);
            cudaEventRecord(t1, e->stream);
            if (rc == PPM_OK) rc = copy_all(false);
            if (rc == PPM_OK && cudaEventSynchronize(t1) != cudaSuccess) rc = efail(e, PPM_ECUDA, "event sync failed");
            if (rc == PPM_OK && rep == 1) cudaEventElapsedTime(&ms, t0, t1);
        }
        if (rc == PPM_OK && ms < best_step) {
            best_step = ms;
            best_mode = mode;
        }
    }
    if (rc == PPM_OK) rc = ppm_ensemble_set_launch_mode(e, best_mode);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    cudaStreamSynchronize(e->stream);
    for (ppm_ctx *c : e->box) cudaMemsetAsync(&c->ds_dev->flags, 0, sizeof(int), e->stream);
    cudaStreamSynchronize(e->stream);
    cudaFree(scratch);
    e->have_speed = false;
    if (rc != PPM_OK) return rc;
    rc = build_work(e);
    if (rc != PPM_OK) return rc;
    if (cache_path) {
        FILE *f = fopen(cache_path, "a");
        if (f) {
            fprintf(f, "%s\t%d %d %d %d %d %d %d %d\n", key.c_str(), e->cfg_nb[0], e->cfg_pers[0], e->cfg_nb[1],
                    e->cfg_pers[1], e->cfg_nb[2], e->cfg_pers[2], e->cfg_vec, e->one_launch ? 1 : 0);
            fclose(f);
        }
    }
    return PPM_OK;
}

long long ppm_ensemble_launch_count(const ppm_ens *e) {
    if (!e) return 0;
    long long n = e->launches;
    for (const ppm_ctx *c : e->box) n += c->launches;
    return n;
}

const char *ppm_ensemble_last_error(const ppm_ens *e) { return e ? e->err.c_str() : g_create_error.c_str(); }

void ppm_ensemble_destroy(ppm_ens *e) {
    if (!e) return;
    ens_release(e);
    delete e;
}

}  // extern "C"
