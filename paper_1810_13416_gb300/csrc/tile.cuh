// tile.cuh -- the fused 1-D PPM + PPB pass as a cell-parallel tile march
// (FP32 base-state-deviation form, four-value PPB).
//
// A block of 256 threads owns P = 8 neighbouring grid pencils and walks along
// them S = 32 cells at a time.  Each step every thread takes one cell (or
// face) of the 8 x 32 tile through each stage of the pass, and the stages
// hand their results to the next through small rings in shared memory, so a
// thread carries no multi-cell window in registers (the register-window form
// in sweep.cuh needs ~240 registers per pencil; here the limit is 128, which
// lets two blocks, 16 warps, share an SM).  The stencil reaches 4 cells
// (Sec. 4), and every quantity is still computed once per cell: each stage
// lags the one before by the cells it needs ahead.  With t the cells loaded
// in a step:
//   A  primitives of cell t                          (steps a1 of the pass)
//   B  interface values, detector, flattening,       (a2-a5)
//      parabolas and tracing of cell t-2, and its PPB profile
//   C  Riemann solve, fluxes and PPB transfers       (a6, a7, a9)
//      at face (t-3)+1/2
//   D  hydro update, sources, CFL of cell t-3,       (a8, a10)
//      FCT factors
//   E  FCT limits and the FV / moment update of t-4  (a9)
// The state moves by TMA: a producer thread loads each 8 x 32 x 9 tile of
// the next chunk (cp.async.bulk.tensor, completion on an mbarrier) while the
// block works on the current one, and stores each finished chunk the same
// way, in place.  For the y and z passes the box is 8 cells along x (32 B)
// by 32 cells along the pass; for the x pass it is 32 cells along x by 8
// rows, read through the 128-byte swizzle so that a warp's 8 rows x 4 cells
// fall in 32 different banks.
//
// The arithmetic of each stage is the one of sweep.cuh (the same
// expressions, in the same order), so both forms agree with the FP64 oracle
// at the FP32 tolerances.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "sweep.cuh"

namespace ppm {
namespace tile {

constexpr int S = 32;          // cells per pencil and step
constexpr int P = 8;           // pencils per block
constexpr int NT = S * P;      // threads per block
constexpr int R = 40;          // ring slots per pencil (>= S + the 8 cells of lag)
constexpr int NIN = 3;         // input chunk buffers (two read, one in flight)
constexpr int NOUT = 2;        // output chunk buffers
constexpr int CHUNK_FLOATS = 9 * S * P;          // one chunk of the 9 values
constexpr unsigned CHUNK_BYTES = CHUNK_FLOATS * 4u;
constexpr int NX1 = 8, NX2 = 12, NX3 = 16, NX4 = 3;
constexpr long long WAIT_LIMIT = 1ll << 26;      // bounded mbarrier wait (iterations)
constexpr int FLAG_TIMEOUT = 2;

// Shared memory of one block (offsets from a 1024-byte aligned base).
struct Smem {
    float in[NIN][CHUNK_FLOATS];   // TMA destinations (9216 B each: 1024-byte multiples)
    float out[NOUT][CHUNK_FLOATS]; // TMA sources
    float x1[NX1][R * P];          // A -> B, D, E: rho', u, v, w, p', rho0, p0, g
    float x2[NX2][R * P];          // B -> C: left state (5), right state (5), PPB profile (2)
    float x3[NX3][R * P];          // C -> D, E: fluxes (7), PPB transfers (9)
    float x4[NX4][R * P];          // D -> E: FCT factors R+, R-, new density
    float stash[9][4 * P];         // cells 0..3 (high-side ghosts of periodic pencils)
    unsigned long long bar[NIN];
    int abort;
};
constexpr size_t SMEM_BYTES = sizeof(Smem) + 1024;   // + alignment slack

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long *b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(b)), "r"(bytes)
                 : "memory");
}
// Bounded wait for phase `parity` of barrier b; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(unsigned long long *b, unsigned parity) {
    const unsigned a = smem_u32(b);
    for (long long it = 0; it < WAIT_LIMIT; ++it) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
__device__ __forceinline__ void tma_load4(void *dst, const CUtensorMap *tm, int c0, int c1, int c2, int c3,
                                          unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(smem_u32(dst)),
        "l"(tm), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_store4(const CUtensorMap *tm, int c0, int c1, int c2, int c3, const void *src) {
    asm volatile(
        "cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4}], [%5];\n" ::"l"(tm),
        "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(src))
        : "memory");
    asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }

// Position of (pencil p, row r of a chunk) inside one value's 256 floats of a
// chunk buffer.  y / z passes: row-major [r][p] (8 floats = 32 B per row).
// x pass: [p][r] (128 B per row) under the 128-byte swizzle, i.e. the 16-byte
// group r/4 of row p sits at group (r/4) ^ p.
template <bool XP>
__device__ __forceinline__ int chunk_pos(int p, int r) {
    if constexpr (XP)
        return p * S + ((((r >> 2) ^ p) & 7) << 2) + (r & 3);
    else
        return r * P + p;
}

// Ring slot of cell c (c >= -2R).
__device__ __forceinline__ int slot_of(int c) { return (c + 2 * R) % R; }
__device__ __forceinline__ int slot_add(int s, int d) {
    int t = s + d;
    t = (t >= R) ? t - R : t;
    return (t < 0) ? t + R : t;
}

// ---------------------------------------------------------------------------
// The kernel.  XP: x pass (pencils are rows along x); otherwise the y or z
// pass (A.axis), pencils along it, 8 neighbouring x columns per block.
// Grid: (ceil(nlane / 8), nblk).  Needs nx % 4 == 0 (TMA strides), no
// confining sphere, four-value PPB, no shock dissipation.
// ---------------------------------------------------------------------------
template <bool XP>
__global__ void __launch_bounds__(NT, 2) tile_pass_kernel(const SweepArgs<float> A,
                                                         const __grid_constant__ CUtensorMap tmap) {
    extern __shared__ unsigned char smem_raw[];
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u));
    const int tid = threadIdx.x;
    const int p = tid & (P - 1);          // pencil of this thread
    const int l = tid >> 3;               // cell of this thread within a step
    const int ax = XP ? 0 : A.axis, t1d = (ax + 1) % 3, t2d = (ax + 2) % 3;
    const int n = A.n, bcl = A.bc_lo, bch = A.bc_hi;
    const int lane = blockIdx.x * P + p, blk = blockIdx.y;
    const bool pen_ok = lane < A.nlane;
    const bool lane_t1 = (A.lane_dim == t1d);
    // variables in the pass frame: normal and transverse momenta / moments
    const int pn = 1 + ax, p1 = 1 + t1d, p2 = 1 + t2d;
    const int on_ = 6 + ax, o1_ = 6 + t1d, o2_ = 6 + t2d;

    const float gam = (float)A.gamma, gm1 = (float)(A.gamma - 1.0);
    const float kk = (float)((A.gamma + 1.0) / (2.0 * A.gamma));
    const float gg1 = (float)(A.gamma / (A.gamma - 1.0));
    const double dtd = *A.dt;
    const float dt = (float)dtd;
    const float dtdx = (float)(dtd / A.dx);
    const float hdt = 0.5f * dt;

    // transverse position of this thread's pencil
    const float xt1 = (float)coord(A, t1d, lane_t1 ? lane : blk);
    const float xt2 = (float)coord(A, t2d, lane_t1 ? blk : lane);
    const float zt = (t1d == 2) ? xt1 : xt2;
    const float rt2 = xt1 * xt1 + xt2 * xt2;
    float4 bconst = make_float4(0.f, 0.f, 0.f, 0.f);
    if (A.grav == 0) bconst = make_float4((float)A.rho0_c, (float)A.p0_c, 0.f, 0.f);
    else if (A.grav == 1 && ax != 2) {
        bconst = tab4(A.t4_base, A.ntab4, A.s4_0, A.inv_ds4, zt);
        bconst.z = 0.0f;
    }
    const bool bvar = (A.grav == 2 || (A.grav == 1 && ax == 2));
    const float orgf = (float)A.org[ax], dxf = (float)A.dx;
    // base state (rho0, p0, g along the pass) at coordinate xa along the pass
    auto base_at_x = [&](float xa) -> float4 {
        if (!bvar) return bconst;
        const float sv = (A.grav == 1) ? xa : fmaf(xa, xa, rt2);
        float4 r = tab4(A.t4_base, A.ntab4, A.s4_0, A.inv_ds4, sv);
        r.w = 0.0f;
        if (A.grav == 2) r.z *= xa;
        return r;
    };
    auto xcell32 = [&](int mm) { return orgf + ((float)mm + 0.5f) * dxf; };
    auto xface32 = [&](int j) { return orgf + (float)map_face(j, n, bcl, bch) * dxf; };

    // raw (stored) value v of cell c of this thread's pencil
    auto in_idx = [&](int c) {
        const int k = (c - 4 + S) / S - 1;          // chunk of cell c (c >= -8)
        const int b = (k + 1) % NIN;
        return b * CHUNK_FLOATS + chunk_pos<XP>(p, c - 4 - k * S);
    };
    auto raw = [&](int v, int c) -> float { return (&sm.in[0][0])[in_idx(c) + v * (S * P)]; };
    auto out_ref = [&](int v, int c) -> float & {
        const int j = (c + S) / S - 1;              // output chunk of cell c (c >= -S)
        const int b = (j + NOUT) % NOUT;
        return sm.out[b][v * (S * P) + chunk_pos<XP>(p, c - j * S)];
    };
    auto X = [&](float (*ring)[R * P], int v, int slot) -> float & { return ring[v][slot * P + p]; };

    // tile coordinates of a chunk: cells [c0, c0 + S) along the pass
    auto coords = [&](int c0, int &k0, int &k1, int &k2) {
        if constexpr (XP) {
            k0 = c0; k1 = blockIdx.x * P; k2 = blk;
        } else if (A.axis == 1) {
            k0 = blockIdx.x * P; k1 = c0; k2 = blk;
        } else {
            k0 = blockIdx.x * P; k1 = blk; k2 = c0;
        }
    };
    const int klast = (n + S - 1) / S - 1;         // last step (stores cells up to n - 1)

    // ---- set-up: barriers, rings cleared, periodic low-side ghosts --------
    if (tid == 0) {
        for (int b = 0; b < NIN; ++b) mbar_init(&sm.bar[b], 1);
        sm.abort = 0;
        fence_mbar_init();
    }
    for (int i = tid; i < NX1 * R * P; i += NT) (&sm.x1[0][0])[i] = 0.0f;
    for (int i = tid; i < NX2 * R * P; i += NT) (&sm.x2[0][0])[i] = 0.0f;
    for (int i = tid; i < NX3 * R * P; i += NT) (&sm.x3[0][0])[i] = 0.0f;
    for (int i = tid; i < NX4 * R * P; i += NT) (&sm.x4[0][0])[i] = 0.0f;
    // periodic pencils: cells n-4..n-1 are the low-side ghosts; read them now,
    // before any store of this block can overwrite them (thread tid < 4 P
    // holds ghost (tid / P) of pencil tid % P)
    float gpre[9];
    const bool gthr = (bcl == 0) && tid < 4 * P;
    if (gthr) {
        const int gp = tid % P, gc = tid / P;      // ghost cell -4 + gc <- cell n - 4 + gc
        const int gl = blockIdx.x * P + gp;
        if (gl < A.nlane) {
            const float *q = A.q + (long long)gl * A.s_lane + (long long)blk * A.s_blk +
                             (long long)(n - 4 + gc) * A.s_axis;
            for (int v = 0; v < 9; ++v) gpre[v] = q[(long long)v * A.vs];
        } else {
            for (int v = 0; v < 9; ++v) gpre[v] = 0.0f;
        }
    }
    __syncthreads();
    if (tid == 0) {
        // first chunk (step -1: cells [-S+4, 4), ghosts and cells 0..3)
        int k0, k1, k2;
        coords(-S + 4, k0, k1, k2);
        mbar_expect_tx(&sm.bar[0], CHUNK_BYTES);
        tma_load4(&sm.in[0][0], &tmap, k0, k1, k2, 0, &sm.bar[0]);
    }

    float smax_local = 0.0f;
    bool bad = false;
}  // namespace tile
}  // namespace ppm
