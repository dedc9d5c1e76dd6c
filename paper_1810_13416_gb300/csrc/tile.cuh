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
// way, in place.  Stage A reads each cell's nine stored values once, maps the
// ghost cells (periodic wrap, or the mirror image with the normal components
// reversed) and puts them in a ring of their own for the later stages.  For the y and z passes the box is 8 cells along x (32 B)
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
constexpr int NIN = 2;         // input chunk buffers (one read, one in flight)
constexpr int NOUT = 2;        // output chunk buffers
constexpr int CHUNK_FLOATS = 9 * S * P;          // one chunk of the 9 values
constexpr unsigned CHUNK_BYTES = CHUNK_FLOATS * 4u;
constexpr int NX1 = 8, NX2 = 12, NX3 = 16, NX4 = 3;
constexpr long long WAIT_LIMIT = 1ll << 26;      // bounded mbarrier wait (iterations)

// Shared memory of one block (offsets from a 1024-byte aligned base).
struct Smem {
    float in[NIN][CHUNK_FLOATS];   // TMA destinations (9216 B each: 1024-byte multiples)
    float out[NOUT][CHUNK_FLOATS]; // TMA sources
    float x0[9][R * P];            // A -> B..E: the stored values (ghosts mapped and mirrored)
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
// The kernel for the pass along axis AX.  AX = 0: pencils are rows along x,
// 8 neighbouring rows per block; AX = 1, 2: pencils along y or z, 8
// neighbouring x columns per block.
// Grid: (ceil(nlane / 8), nblk).  Needs nx % 4 == 0 (TMA strides), no
// confining sphere, four-value PPB, no shock dissipation.
//
// Step k (k = -1 .. klast) loads chunk k = cells [kS + 4, kS + S + 4) of
// every pencil; thread (p, l) takes cell kS + 4 + l in stage A, the cell or
// face l - 2, l - 3, l - 3, l - 4 behind it in stages B to E, and the block
// stores cells [kS, kS + S) at the end of the step.
// ---------------------------------------------------------------------------
// FULL = false: a pass without sources and without the CFL maximum (its own
// instantiation, without that code)
template <int AX, bool FULL = true>
__global__ void __launch_bounds__(NT, 2) tile_pass_kernel(const SweepArgs<float> A,
                                                         const __grid_constant__ CUtensorMap tmap) {
    constexpr bool XP = (AX == 0);
    extern __shared__ unsigned char smem_raw[];
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u));
    const int tid = threadIdx.x;
    const int p = tid & (P - 1);          // pencil of this thread
    const int l = tid >> 3;               // cell of this thread within a step
    constexpr int ax = AX, t1d = (AX + 1) % 3, t2d = (AX + 2) % 3;
    const int n = A.n, bcl = A.bc_lo, bch = A.bc_hi;
    const int lane = blockIdx.x * P + p, blk = blockIdx.y;
    const bool pen_ok = lane < A.nlane;
    const bool lane_t1 = (A.lane_dim == t1d);
    // variables in the pass frame: normal and transverse momenta / moments
    constexpr int pn = 1 + ax, p1 = 1 + t1d, p2 = 1 + t2d;
    constexpr int on_ = 6 + ax, o1_ = 6 + t1d, o2_ = 6 + t2d;

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
    // The same lookup split in two, so that the two rows can be fetched a
    // stage before they are needed (the latency then overlaps other work)
    struct Rows {
        float4 a, b;
        float w;
    };
    auto rows_issue = [&](float xa) -> Rows {
        Rows r;
        if (!bvar) {
            r.a = r.b = bconst;
            r.w = 0.0f;
            return r;
        }
        const float sv = (A.grav == 1) ? xa : fmaf(xa, xa, rt2);
        const float u = (sv - A.s4_0) * A.inv_ds4;
        const float fl = fminf(fmaxf(floorf(u), 0.0f), (float)(A.ntab4 - 2));
        const int i = (int)fl;
        r.a = __ldg(A.t4_base + i);
        r.b = __ldg(A.t4_base + i + 1);
        r.w = u - fl;
        return r;
    };
    auto rows_finish = [&](const Rows &t, float xa) -> float4 {
        if (!bvar) return bconst;
        float4 r = make_float4(fmaf(t.w, t.b.x - t.a.x, t.a.x), fmaf(t.w, t.b.y - t.a.y, t.a.y),
                               fmaf(t.w, t.b.z - t.a.z, t.a.z), 0.0f);
        if (A.grav == 2) r.z *= xa;
        return r;
    };
    // cell centres and faces from float cell indices: k S + (small integer)
    // is exact in FP32, so these equal the register-window form's values
    auto xcell_f = [&](float fm) { return orgf + (fm + 0.5f) * dxf; };

    auto X = [&](float (*ring)[R * P], int v, int slot) -> float & { return ring[v][slot * P + p]; };
    // this thread's row in a chunk buffer: stage A reads row l of chunk k;
    // stage E writes row l of output chunk k, stage D row l + 1 (or row 0 of
    // chunk k + 1 for l = S - 1)
    const int posA = chunk_pos<XP>(p, l);
    const int posD = chunk_pos<XP>(p, (l + 1) & (S - 1));

    // tile coordinates of a chunk: cells [c0, c0 + S) along the pass
    auto coords = [&](int c0, int &k0, int &k1, int &k2) {
        if constexpr (XP) {
            k0 = c0; k1 = blockIdx.x * P; k2 = blk;
        } else if constexpr (AX == 1) {
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
    for (int i = tid; i < 9 * R * P; i += NT) (&sm.x0[0][0])[i] = 0.0f;
    for (int i = tid; i < NX1 * R * P; i += NT) (&sm.x1[0][0])[i] = 0.0f;
    for (int i = tid; i < NX2 * R * P; i += NT) (&sm.x2[0][0])[i] = 0.0f;
    for (int i = tid; i < NX3 * R * P; i += NT) (&sm.x3[0][0])[i] = 0.0f;
    for (int i = tid; i < NX4 * R * P; i += NT) (&sm.x4[0][0])[i] = 0.0f;
    // periodic pencils: cells n-4..n-1 are the low-side ghosts -4..-1, which
    // the threads l = S-8 .. S-5 take in stage A of step -1; they read them
    // now, before any store of this block can overwrite them
    float gpre[9];
    const int c_first = -S + 4 + l;                 // stage A cell of step -1
    if (bcl == 0 && c_first >= -4 && c_first < 0 && pen_ok) {
        const float *q = A.q + (long long)lane * A.s_lane + (long long)blk * A.s_blk +
                         (long long)(n + c_first) * A.s_axis;
#pragma unroll
        for (int v = 0; v < 9; ++v) gpre[v] = q[(long long)v * A.vs];
    } else {
#pragma unroll
        for (int v = 0; v < 9; ++v) gpre[v] = 0.0f;
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
    int kstop = klast + 1;                          // step at which a wait gave up
    int sA = (l + 12) % R;                          // ring slot of the stage A cell (-S + 4 + l)
    const float flA = (float)(4 + l);
    Rows rowsA = rows_issue(xcell_f((float)(-S) + flA));   // stage A of step -1

    for (int k = -1; k <= klast; ++k) {
        const int cA = k * S + 4 + l;               // stage A cell of this thread
        const float fk = (float)(k * S);
        if (k > -1) sA = (sA + S >= R) ? sA + S - R : sA + S;
        // ---- producer: chunk k+1 into the buffer of chunk k-1 -------------
        if (tid == 0 && k + 1 <= klast) {
            const int b = (k + 2) & 1;
            fence_async_smem();   // the block's reads of chunk k-1 came first
            int k0, k1, k2;
            coords((k + 1) * S + 4, k0, k1, k2);
            mbar_expect_tx(&sm.bar[b], CHUNK_BYTES);
            tma_load4(&sm.in[b][0], &tmap, k0, k1, k2, 0, &sm.bar[b]);
        }
        // ---- wait for chunk k (its buffer's use (k+1)/2, parity & 1) -------
        const float *inb = &sm.in[(k + 1) & 1][0];
        if (!mbar_wait(&sm.bar[(k + 1) & 1], (unsigned)(((k + 1) >> 1) & 1))) sm.abort = 1;
        __syncthreads();
        if (sm.abort) {
            kstop = k;
            break;
        }

        // ================= A: stored values and primitives of cell cA ========
        {
            const int c = cA;
            float q[9];
            bool flip = false;
            int m = c;
            if (c >= 0 && c < n) {
#pragma unroll
                for (int v = 0; v < 9; ++v) q[v] = inb[v * (S * P) + posA];
                if (k == -1 && bch == 0) {
                    // cells 0..3 of periodic pencils, before they are overwritten
#pragma unroll
                    for (int v = 0; v < 9; ++v) sm.stash[v][c * P + p] = q[v];
                }
            } else if (c < -4 || c >= n + 4) {
#pragma unroll
                for (int v = 0; v < 9; ++v) q[v] = 0.0f;   // beyond the ghosts: never used
                m = 0;
            } else {
                // ghost: periodic image or mirror image (normal components reversed)
                m = map_cell(c, n, bcl, bch, flip);
                if (c < 0 && bcl == 0) {
#pragma unroll
                    for (int v = 0; v < 9; ++v) q[v] = gpre[v];
                } else if (c < 0) {
                    const int pos = chunk_pos<XP>(p, m + S - 4);   // row of cell m in chunk -1
#pragma unroll
                    for (int v = 0; v < 9; ++v) q[v] = inb[v * (S * P) + pos];
                } else if (bch == 0) {
#pragma unroll
                    for (int v = 0; v < 9; ++v) q[v] = sm.stash[v][m * P + p];
                } else if (m >= k * S + 4) {
                    const int pos = chunk_pos<XP>(p, m - k * S - 4);
#pragma unroll
                    for (int v = 0; v < 9; ++v) q[v] = inb[v * (S * P) + pos];
                } else {
                    const int sm_ = slot_of(m);
#pragma unroll
                    for (int v = 0; v < 9; ++v) q[v] = X(sm.x0, v, sm_);
                }
                if (flip) {
                    q[pn] = -q[pn];
                    q[on_] = -q[on_];
                }
            }
            // base state: the rows fetched a step ahead hold cell c itself
            const float4 bb = (m == c) ? rows_finish(rowsA, xcell_f(fk + flA)) : base_at_x(xcell_f((float)m));
            const float sg = flip ? -1.0f : 1.0f;
            const float rd = q[0];
            const float mn = q[pn], m1 = q[p1], m2 = q[p2];
            const float ed = q[4];
            const float rho = bb.x + rd;
            const float rinv = qdiv(1.0f, rho);
            const float u = mn * rinv, v = m1 * rinv, w = m2 * rinv;
            const float ke = 0.5f * (mn * u + (m1 * v + m2 * w));
            const float pd = gm1 * (ed - ke);
#pragma unroll
            for (int vv = 0; vv < 9; ++vv) X(sm.x0, vv, sA) = q[vv];
            X(sm.x1, 0, sA) = rd;
            X(sm.x1, 1, sA) = u;
            X(sm.x1, 2, sA) = v;
            X(sm.x1, 3, sA) = w;
            X(sm.x1, 4, sA) = pd;
            X(sm.x1, 5, sA) = bb.x;
            X(sm.x1, 6, sA) = bb.y;
            X(sm.x1, 7, sA) = sg * bb.z;
        }
        __syncthreads();

        // face j+1/2 of stage C (j = cA - 3): its position, and its table rows
        // fetched now so that stage B covers their latency
        const int jC = cA - 3;
        const bool plain_face = (jC + 1 >= 0 && jC + 1 <= n && !(jC + 1 == n && bch == 0));
        const float xfC = orgf + (plain_face ? fk + (float)(l + 2) : (float)map_face(jC, n, bcl, bch)) * dxf;
        const Rows rowsC = rows_issue(xfC);

        // ================= B: cell cA-2 ======================================
        {
            const int s0 = slot_add(sA, -2);
            const int sm2 = slot_add(sA, -4), sm1 = slot_add(sA, -3), sp1 = slot_add(sA, -1);
            const int sl5[5] = {sm2, sm1, s0, sp1, sA};
            float wrd[5], wu[5], wv[5], ww[5], wpd[5];
#pragma unroll
            for (int d = 0; d < 5; ++d) {
                wrd[d] = X(sm.x1, 0, sl5[d]);
                wu[d] = X(sm.x1, 1, sl5[d]);
                wv[d] = X(sm.x1, 2, sl5[d]);
                ww[d] = X(sm.x1, 3, sl5[d]);
                wpd[d] = X(sm.x1, 4, sl5[d]);
            }
            const float r0c = X(sm.x1, 5, s0), p0c = X(sm.x1, 6, s0), gc = X(sm.x1, 7, s0);
            const float p0m = X(sm.x1, 6, sm1), p0p = X(sm.x1, 6, sp1);
            // interface values of faces c-1/2 and c+1/2 (a2)
            float afp[5], afn[5];
            afp[0] = iface(wrd[0], wrd[1], wrd[2], wrd[3]);
            afp[1] = iface(wu[0], wu[1], wu[2], wu[3]);
            afp[2] = iface(wv[0], wv[1], wv[2], wv[3]);
            afp[3] = iface(ww[0], ww[1], ww[2], ww[3]);
            afp[4] = iface(wpd[0], wpd[1], wpd[2], wpd[3]);
            afn[0] = iface(wrd[1], wrd[2], wrd[3], wrd[4]);
            afn[1] = iface(wu[1], wu[2], wu[3], wu[4]);
            afn[2] = iface(wv[1], wv[2], wv[3], wv[4]);
            afn[3] = iface(ww[1], ww[2], ww[3], ww[4]);
            afn[4] = iface(wpd[1], wpd[2], wpd[3], wpd[4]);
            float WLn[5], WRc[5];
            const float rho2 = r0c + wrd[2];
            const float p2 = p0c + wpd[2];
            const float c2 = qdiv(gam * p2, rho2);
            const float cs = rsq<true>(c2);
            // flattening coefficient (a3)
            float f = 0.0f;
            {
                const float dp1 = wpd[3] - wpd[1];
                const float dp2 = wpd[4] - wpd[0];
                const float pmin = rmin<true>(p0p + wpd[3], p0m + wpd[1]);
                if (rabs(dp1) > 0.33f * pmin && wu[1] - wu[3] > 0.0f) {
                    const float r = (dp2 != 0.0f) ? qdiv(dp1, dp2) : 1.0f;
                    f = rsat<true>(10.0f * (r - 0.75f));
                }
            }
            // parabolas of the five variables (a3, a4)
            float aL[5], aR[5], a6[5];
            {
                const float q0 = smooth5<float, true>(wrd[0], wrd[1], wrd[2], wrd[3], wrd[4], rho2);
                parabola<float, true>(wrd[1], wrd[2], wrd[3], afp[0], afn[0], f, q0, aL[0], aR[0], a6[0]);
                const float q1 = smooth5<float, true>(wu[0], wu[1], wu[2], wu[3], wu[4], cs);
                parabola<float, true>(wu[1], wu[2], wu[3], afp[1], afn[1], f, q1, aL[1], aR[1], a6[1]);
                const float q2 = smooth5<float, true>(wv[0], wv[1], wv[2], wv[3], wv[4], cs);
                parabola<float, true>(wv[1], wv[2], wv[3], afp[2], afn[2], f, q2, aL[2], aR[2], a6[2]);
                const float q3 = smooth5<float, true>(ww[0], ww[1], ww[2], ww[3], ww[4], cs);
                parabola<float, true>(ww[1], ww[2], ww[3], afp[3], afn[3], f, q3, aL[3], aR[3], a6[3]);
                const float q4 = smooth5<float, true>(wpd[0], wpd[1], wpd[2], wpd[3], wpd[4], p2);
                parabola<float, true>(wpd[1], wpd[2], wpd[3], afp[4], afn[4], f, q4, aL[4], aR[4], a6[4]);
            }
            // characteristic tracing (waves u-c, u, u+c) + buoyancy (a5)
            const float uc = wu[2];
            const float C = rho2 * cs;
            const float lm = uc - cs, l0 = uc, lp = uc + cs;
            const float hg = hdt * (qdiv(wrd[2], rho2) * gc);
            {   // right edge -> left state of face c+1/2
                const float sp = rmax<true>(lp, 0.0f) * dtdx;
                float st[5];
#pragma unroll
                for (int q = 0; q < 5; ++q) st[q] = fR(aL[q], aR[q], a6[q], sp);
                const float rr = st[0], ru = st[1], rv = st[2], rw = st[3], rp = st[4];
                if (l0 > 0.0f) {
                    const float sq = l0 * dtdx;
                    const float dr = rr - fR(aL[0], aR[0], a6[0], sq);
                    const float dp = rp - fR(aL[4], aR[4], a6[4], sq);
                    st[0] = st[0] - (dr - qdiv(dp, c2));
                    st[2] = st[2] - (rv - fR(aL[2], aR[2], a6[2], sq));
                    st[3] = st[3] - (rw - fR(aL[3], aR[3], a6[3], sq));
                }
                if (lm > 0.0f) {
                    const float sq = lm * dtdx;
                    const float du = ru - fR(aL[1], aR[1], a6[1], sq);
                    const float dp = rp - fR(aL[4], aR[4], a6[4], sq);
                    const float Aa = 0.5f * (dp - C * du);
                    st[0] = st[0] - qdiv(Aa, c2);
                    st[1] = st[1] + qdiv(Aa, C);
                    st[4] = st[4] - Aa;
                }
                st[1] = st[1] + hg;
#pragma unroll
                for (int q = 0; q < 5; ++q) WLn[q] = st[q];
            }
            {   // left edge -> right state of face c-1/2
                const float sq0 = rmax<true>(-lm, 0.0f) * dtdx;
                float st[5];
#pragma unroll
                for (int q = 0; q < 5; ++q) st[q] = fL(aL[q], aR[q], a6[q], sq0);
                const float rr = st[0], ru = st[1], rv = st[2], rw = st[3], rp = st[4];
                if (l0 < 0.0f) {
                    const float sq = -l0 * dtdx;
                    const float dr = rr - fL(aL[0], aR[0], a6[0], sq);
                    const float dp = rp - fL(aL[4], aR[4], a6[4], sq);
                    st[0] = st[0] - (dr - qdiv(dp, c2));
                    st[2] = st[2] - (rv - fL(aL[2], aR[2], a6[2], sq));
                    st[3] = st[3] - (rw - fL(aL[3], aR[3], a6[3], sq));
                }
                if (lp < 0.0f) {
                    const float sq = -lp * dtdx;
                    const float du = ru - fL(aL[1], aR[1], a6[1], sq);
                    const float dp = rp - fL(aL[4], aR[4], a6[4], sq);
                    const float Aa = 0.5f * (dp + C * du);
                    st[0] = st[0] - qdiv(Aa, c2);
                    st[1] = st[1] - qdiv(Aa, C);
                    st[4] = st[4] - Aa;
                }
                st[1] = st[1] + hg;
#pragma unroll
                for (int q = 0; q < 5; ++q) WRc[q] = st[q];
            }
            // PPB profile of cell c: f = FV + m xi + a2 (xi^2 - 1/12), bound-limited (a9)
            float me2, ae2;
            {
                const float fs = X(sm.x0, 5, s0);
                const float F = fv_unfold(fs), mm = X(sm.x0, on_, s0);
                const float a2 = 0.25f * (X(sm.x0, on_, sp1) - X(sm.x0, on_, sm1));
                const float ep = 0.5f * mm + a2 * (1.0f / 6.0f);
                const float em = a2 * (1.0f / 6.0f) - 0.5f * mm;
                float gmax = rmax<true>(ep, em), gmin = rmin<true>(ep, em);
                const bool nz = (a2 != 0.0f);
                const float xv = qdiv(-mm, 2.0f * (nz ? a2 : 1.0f));
                const float gv = mm * xv + a2 * (xv * xv - (1.0f / 12.0f));
                const bool in = nz && (rabs(xv) < 0.5f);
                gmax = in ? rmax<true>(gmax, gv) : gmax;
                gmin = in ? rmin<true>(gmin, gv) : gmin;
                float th = 1.0f;
                const float omf = fv_complement(fs);
                const bool hi = gmax > omf, lo = -gmin > F;
                const float t1 = qdiv(omf, hi ? gmax : 1.0f), t2 = qdiv(F, lo ? -gmin : 1.0f);
                th = hi ? rmin<true>(th, t1) : th;
                th = lo ? rmin<true>(th, t2) : th;
                me2 = th * mm;
                ae2 = th * a2;
            }
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                X(sm.x2, q, s0) = WLn[q];
                X(sm.x2, 5 + q, s0) = WRc[q];
            }
            X(sm.x2, 10, s0) = me2;
            X(sm.x2, 11, s0) = ae2;
        }
        __syncthreads();

        // heating and damping rows of stage D's cell, fetched before stage C
        // (same index and weight as a lookup of the source table; measured
        // 3% faster on the pass with sources)
        float2 hsa = make_float2(0.f, 0.f), hsb = hsa;
        float hsw = 0.0f;
        if (FULL && A.sources) {
            const float xa = xcell_f(fk + (float)(l + 1));
            const float sv = (A.grav == 1) ? (ax == 2 ? xa : zt) : fmaf(xa, xa, rt2);
            const float u = (sv - A.s4_0) * A.inv_ds4;
            const float fl = fminf(fmaxf(floorf(u), 0.0f), (float)(A.ntab4 - 2));
            const int r = (int)fl;
            const float2 *t2 = reinterpret_cast<const float2 *>(A.t4_src);
            hsa = __ldg(t2 + 2 * r);
            hsb = __ldg(t2 + 2 * r + 2);
            hsw = u - fl;
        }
        // ================= C: face (cA-3)+1/2 ================================
        {
            const int j = cA - 3;                    // face j+1/2 between cells j and j+1
            const int sj = slot_add(sA, -3), sr = slot_add(sA, -2);
            float WLp[5], WRc[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                WLp[q] = X(sm.x2, q, sj);            // left state: right edge of cell j
                WRc[q] = X(sm.x2, 5 + q, sr);        // right state: left edge of cell j+1
            }
            const float4 bf = rows_finish(rowsC, xfC);
            const float r0 = bf.x, p0 = bf.y;
            const float rdL = WLp[0], uL = WLp[1], pdL = WLp[4];
            const float rdR = WRc[0], uR = WRc[1], pdR = WRc[4];
            const float rL = r0 + rdL, pL = p0 + pdL;
            const float rR = r0 + rdR, pR = p0 + pdR;
            const float CL = rsq<true>(gam * pL * rL), CR = rsq<true>(gam * pR * rR);
            const float pfl = 1e-10f * rmin<true>(pL, pR);
            float den = CL + CR;
            float iden = qdiv(1.0f, den);
            float pst = pdL + CL * (CR * (uL - uR) + (pdR - pdL)) * iden;
            float ust = uL + (CR * (uR - uL) + (pdL - pdR)) * iden;
            if (p0 + pst < pfl) pst = pfl - p0;
            const float WLi = CL * rsq<true>(1.0f + qdiv(kk * (pst - pdL), pL));
            const float WRi = CR * rsq<true>(1.0f + qdiv(kk * (pst - pdR), pR));
            den = WLi + WRi;
            iden = qdiv(1.0f, den);
            pst = pdL + WLi * (WRi * (uL - uR) + (pdR - pdL)) * iden;
            ust = uL + (WRi * (uR - uL) + (pdL - pdR)) * iden;
            if (p0 + pst < pfl) pst = pfl - p0;
            const bool wall = (j == -1 && bcl == 1) || (j == n - 1 && bch == 1);
            if (wall) ust = 0.0f;
            const bool left = (ust >= 0.0f);
            const float rds = left ? rdL : rdR;
            const float pds = left ? pdL : pdR;
            const float rs = left ? rL : rR;
            const float pss = left ? pL : pR;
            float vst = left ? WLp[2] : WRc[2];
            float wst = left ? WLp[3] : WRc[3];
            const float dps = pst - pds;
            float rdst = rds + qdiv(rs * dps, gam * pss + 0.5f * gm1 * dps);
            {
                // the two-shock solution at x/t = 0: upwind traced state where
                // both waves move to one side
                const bool supL = !wall && (uL * rL >= WLi);
                const bool supR = !wall && !supL && (uR * rR <= -WRi);
                ust = supL ? uL : (supR ? uR : ust);
                pst = supL ? pdL : (supR ? pdR : pst);
                rdst = supL ? rdL : (supR ? rdR : rdst);
                vst = supL ? WLp[2] : (supR ? WRc[2] : vst);
                wst = supL ? WLp[3] : (supR ? WRc[3] : wst);
            }
            const float h0 = gg1 * p0;
            const float kin = 0.5f * (ust * ust + (vst * vst + wst * wst));
            // mass and energy fluxes carry their base-state parts (rho0 u*,
            // h0 u*) as exact hi + lo pairs (a7)
            float Frc, Frlc, FEc, FElc;
            {
                float hi, e;
                two_prod(r0, ust, hi, e);
                Frc = hi;
                Frlc = e + rdst * ust;
            }
            const float Fr = Frc + Frlc;
            {
                float hE, eE;
                two_prod(ust, h0, hE, eE);
                FEc = hE;
                FElc = eE + (ust * (gg1 * pst) + kin * Fr);
            }
            // PPB transfers across the face: donor j (from the left) or j+1
            {
                const float sig = ust * dtdx;
                const float phi = dtdx * Fr;
                const bool fromleft = (sig >= 0.0f);
                const float sabs = fromleft ? sig : -sig;
                float M1 = 0.5f - 0.5f * sabs;
                const float M2 = 0.25f - 0.5f * sabs + sabs * sabs * (1.0f / 3.0f);
                float M3 = 0.125f - 0.375f * sabs + 0.5f * sabs * sabs - 0.25f * sabs * sabs * sabs;
                if (!fromleft) {
                    M1 = -M1;
                    M3 = -M3;
                }
                const int sd = fromleft ? sj : sr;
                const float F = fv_unfold(X(sm.x0, 5, sd));
                const float me = X(sm.x2, 10, sd);
                const float ae = X(sm.x2, 11, sd);
                const float ot1 = X(sm.x0, o1_, sd), ot2 = X(sm.x0, o2_, sd);
                const float phibar = F + me * M1 + ae * (M2 - (1.0f / 12.0f));
                const float psibar = F * M1 + me * M2 + ae * (M3 - M1 * (1.0f / 12.0f));
                const float GLc = phi * F;
                X(sm.x3, 7, sj) = GLc;
                X(sm.x3, 8, sj) = phi * phibar - GLc;
                X(sm.x3, 9, sj) = phi * F * M1;
                X(sm.x3, 10, sj) = phi * psibar;
                X(sm.x3, 11, sj) = phi * ot1;
                X(sm.x3, 12, sj) = phi * ot2;
                X(sm.x3, 13, sj) = phi;
                X(sm.x3, 14, sj) = phi * M1;
                X(sm.x3, 15, sj) = sig;
            }
            X(sm.x3, 0, sj) = Frc;
            X(sm.x3, 1, sj) = Frlc;
            X(sm.x3, 2, sj) = Fr * ust + pst;
            X(sm.x3, 3, sj) = Fr * vst;
            X(sm.x3, 4, sj) = Fr * wst;
            X(sm.x3, 5, sj) = FEc;
            X(sm.x3, 6, sj) = FElc;
        }
        if (tid == 0) bulk_wait_read_all();   // the last store has read its buffer
        __syncthreads();

        // ================= D: cell cA-3 ======================================
        {
            const int c = cA - 3;
            const int sc = slot_add(sA, -3), sl = slot_add(sA, -4);
            const float g = X(sm.x1, 7, sc), r0c = X(sm.x1, 5, sc), p0c = X(sm.x1, 6, sc);
            const float rd3 = X(sm.x0, 0, sc), mn3 = X(sm.x0, pn, sc), m13 = X(sm.x0, p1, sc);
            const float m23 = X(sm.x0, p2, sc), ed3 = X(sm.x0, 4, sc);
            const float Frc = X(sm.x3, 0, sc), Frlc = X(sm.x3, 1, sc), Frp = X(sm.x3, 0, sl), Frlp = X(sm.x3, 1, sl);
            const float FEc = X(sm.x3, 5, sc), FElc = X(sm.x3, 6, sc), FEp = X(sm.x3, 5, sl), FElp = X(sm.x3, 6, sl);
            float sE, eE;
            two_sum(Frc, -Frp, sE, eE);
            const float dFr = sE + (eE + (Frlc - Frlp));
            const float rdn = rd3 - dtdx * dFr;
            two_sum(FEc, -FEp, sE, eE);
            const float dFE = sE + (eE + (FElc - FElp));
            float edo = ed3 - dtdx * dFE + dt * g * (0.5f * ((Frp + Frlp) + (Frc + Frlc)));
            float mno = mn3 - dtdx * (X(sm.x3, 2, sc) - X(sm.x3, 2, sl)) + dt * g * (0.5f * (rd3 + rdn));
            float m1o = m13 - dtdx * (X(sm.x3, 3, sc) - X(sm.x3, 3, sl));
            float m2o = m23 - dtdx * (X(sm.x3, 4, sc) - X(sm.x3, 4, sl));
            const float rnew = r0c + rdn;
            // FCT factors of cell c, bounds [0, 1]
            {
                const float rold = r0c + rd3;
                const float GLc = X(sm.x3, 7, sc), GLp = X(sm.x3, 7, sl);
                const float Ac = X(sm.x3, 8, sc), Ap = X(sm.x3, 8, sl);
                const float cL = rold * fv_unfold(X(sm.x0, 5, sc)) - (GLc - GLp);
                const float FVL = qdiv(cL, rnew);
                const float Pp = rmax<true>(0.0f, Ap) - rmin<true>(0.0f, Ac);
                const float Pm = rmax<true>(0.0f, Ac) - rmin<true>(0.0f, Ap);
                const float Qp = (1.0f - FVL) * rnew;
                const float Qm = FVL * rnew;
                X(sm.x4, 0, sc) = (Pp > 0.0f) ? rsat<true>(qdiv(Qp, Pp)) : 0.0f;
                X(sm.x4, 1, sc) = (Pm > 0.0f) ? rsat<true>(qdiv(Qm, Pm)) : 0.0f;
                X(sm.x4, 2, sc) = rnew;
            }
            // heating and damping after the pass (fused), checks and CFL
            if (FULL && A.sources) {
                const float2 hs = make_float2(fmaf(hsw, hsb.x - hsa.x, hsa.x), fmaf(hsw, hsb.y - hsa.y, hsa.y));
                if (A.t_heat) edo = edo + dt * hs.x;
                if (A.t_damp) {
                    const float fd = rmax<true>(0.0f, 1.0f - dt * hs.y);
                    const float kin = qdiv(0.5f * (mno * mno + (m1o * m1o + m2o * m2o)), rnew);
                    mno = mno * fd;
                    m1o = m1o * fd;
                    m2o = m2o * fd;
                    edo = edo - (1.0f - fd * fd) * kin;
                }
            }
            if (c >= 0 && c < n && pen_ok) {
                const float ri = qdiv(1.0f, rnew);
                const float uu = mno * ri, vv = m1o * ri, wv_ = m2o * ri;
                const float kin = 0.5f * (mno * uu + (m1o * vv + m2o * wv_));
                const float pr = p0c + gm1 * (edo - kin);
                if (!(rnew > 0.0f) || !(pr > 0.0f)) bad = true;
                if (FULL && A.cfl) {
                    const float spd = rmax<true>(rmax<true>(rabs(uu), rabs(vv)), rabs(wv_)) + rsq<true>(gam * pr * ri);
                    smax_local = rmax<true>(smax_local, spd);
                }
            }
            float *o = &sm.out[(l == S - 1 ? k + 1 : k) & 1][posD];
            o[0] = rdn;
            o[pn * (S * P)] = mno;
            o[p1 * (S * P)] = m1o;
            o[p2 * (S * P)] = m2o;
            o[4 * (S * P)] = edo;
        }
        __syncthreads();

        // rows of the next step's stage A cell (cA + S), fetched during stage E
        rowsA = rows_issue(xcell_f(fk + (float)S + flA));

        // ================= E: cell cA-4 ======================================
        {
            const int sc = slot_add(sA, -4), sl = slot_add(sA, -5), sr = slot_add(sA, -3);
            const float Rpl = X(sm.x4, 0, sl), Rml = X(sm.x4, 1, sl);
            const float Rpc = X(sm.x4, 0, sc), Rmc = X(sm.x4, 1, sc);
            const float Rpr = X(sm.x4, 0, sr), Rmr = X(sm.x4, 1, sr);
            // limited transfers of the right face (c+1/2) and the left face (c-1/2)
            const float Ar = X(sm.x3, 8, sc), Al = X(sm.x3, 8, sl);
            const float Cfr = (Ar >= 0.0f) ? rmin<true>(Rpr, Rmc) : rmin<true>(Rpc, Rmr);
            const float Cfl = (Al >= 0.0f) ? rmin<true>(Rpc, Rml) : rmin<true>(Rpl, Rmc);
            const float KLr = X(sm.x3, 9, sc), KLl = X(sm.x3, 9, sl);
            const float Gc4 = X(sm.x3, 7, sc) + Cfr * Ar;
            const float Kc4 = KLr + Cfr * (X(sm.x3, 10, sc) - KLr);
            const float Gq = X(sm.x3, 7, sl) + Cfl * Al;
            const float Kq = KLl + Cfl * (X(sm.x3, 10, sl) - KLl);
            const float PHIp = X(sm.x3, 13, sc), PHIq = X(sm.x3, 13, sl);
            const float KMp = X(sm.x3, 14, sc), KMq = X(sm.x3, 14, sl);
            const float sp = X(sm.x3, 15, sc), smm = X(sm.x3, 15, sl);
            const float T1p = X(sm.x3, 11, sc), T1q = X(sm.x3, 11, sl);
            const float T2p = X(sm.x3, 12, sc), T2q = X(sm.x3, 12, sl);
            const float rold = X(sm.x1, 5, sc) + X(sm.x0, 0, sc);
            const float rnew = X(sm.x4, 2, sc);
            const float fs0 = X(sm.x0, 5, sc);
            const float fv0 = fv_unfold(fs0);
            const float on0 = X(sm.x0, on_, sc), o10 = X(sm.x0, o1_, sc), o20 = X(sm.x0, o2_, sc);
            const float cold = rold * fv0;
            float c_out = 0, z_out = 0, z_in = 0, m_out = 0, zr_out = 0, zr_in = 0;
            if (sp >= 0.0f) {
                c_out = c_out + Gc4;
                z_out = z_out + Kc4;
                m_out = m_out + PHIp;
                zr_out = zr_out + KMp;
            } else {
                const float sh = sp + 1.0f;
                z_in = z_in + (-Kc4 - Gc4 * sh);
                zr_in = zr_in + (-KMp - PHIp * sh);
            }
            if (smm >= 0.0f) {
                const float sh = smm - 1.0f;
                z_in = z_in + (Kq + Gq * sh);
                zr_in = zr_in + (KMq + PHIq * sh);
            } else {
                c_out = c_out - Gq;
                z_out = z_out - Kq;
                m_out = m_out - PHIq;
                zr_out = zr_out - KMq;
            }
            const float sbar = 0.5f * (smm + sp);
            const float dZc = (cold - c_out) * sbar + z_in - z_out;
            const float Zr = (rold - m_out) * sbar + zr_in - zr_out;
            const float dPhi = PHIp - PHIq;
            const float dG = Gc4 - Gq;
            const float rinvn = qdiv(1.0f, rnew);
            const float fvs = fv_add(fs0, (fv0 * dPhi - dG) * rinvn);
            const float fvn = fv_unfold(fvs);
            const float bnd = fv_moment_bound(fvs);
            float onn = on0 + (on0 * dPhi + 12.0f * (dZc - fvn * Zr)) * rinvn;
            float o1 = o10 + (o10 * dPhi - (T1p - T1q)) * rinvn;
            float o2 = o20 + (o20 * dPhi - (T2p - T2q)) * rinvn;
            onn = rclamp<true>(onn, -bnd, bnd);
            o1 = rclamp<true>(o1, -bnd, bnd);
            o2 = rclamp<true>(o2, -bnd, bnd);
            float *o = &sm.out[k & 1][posA];
            o[5 * (S * P)] = fvs;
            o[on_ * (S * P)] = onn;
            o[o1_ * (S * P)] = o1;
            o[o2_ * (S * P)] = o2;
        }
        fence_async_smem();        // this thread's output writes, seen by the TMA store
        __syncthreads();
        if (tid == 0 && k >= 0) {
            int k0, k1, k2;
            coords(k * S, k0, k1, k2);
            tma_store4(&tmap, k0, k1, k2, 0, &sm.out[k & 1][0]);
        }
    }

    if (tid == 0) {
        if (kstop <= klast) {
            // the loads still in flight (chunks kstop and kstop + 1) land
            // before the block leaves; each wait is bounded
            for (int kk2 = kstop; kk2 <= kstop + 1 && kk2 <= klast; ++kk2)
                (void)mbar_wait(&sm.bar[(kk2 + 1) & 1], (unsigned)(((kk2 + 1) >> 1) & 1));
            atomicOr(A.flags, FLAG_TIMEOUT);
        }
        bulk_wait_all();
    }
    if (bad && pen_ok) atomicOr(A.flags, FLAG_NONPHYS);
    if (FULL && A.cfl) {
        double smx = (double)smax_local;
        for (int o = 16; o > 0; o >>= 1) smx = fmax(smx, __shfl_xor_sync(0xffffffffu, smx, o));
        if ((threadIdx.x & 31) == 0) atomicMax(A.smax, dbits(smx));
    }
}

}  // namespace tile
}  // namespace ppm
