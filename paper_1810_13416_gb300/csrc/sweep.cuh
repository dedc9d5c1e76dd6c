// sweep.cuh -- the fused 1-D PPM + PPB pass (one kernel per axis and precision).
//
// One thread owns one grid pencil and marches along it cell by cell, keeping a
// five-cell window of the state in registers, the way the paper keeps three
// 32-word vectors per quantity on chip and barrel-shifts them (Sec. 4, Fig. 7):
// every quantity of the pass is computed exactly once per cell, with no halo
// recomputation.  Neighbouring threads own neighbouring pencils, so for the y
// and z passes every load and store of a warp is one contiguous 128-byte
// segment along x.
//
// At step c (the newest cell loaded is c) the pipeline does, with fixed lags:
//   load + primitives            cell c                       (step a1)
//   interface value              face (c-2)+1/2               (a2)
//   detector, flattening,        cell c-2                     (a3, a4)
//   parabola, characteristic
//   tracing of both edges                                     (a5)
//   Riemann solve and fluxes     face (c-3)+1/2               (a6, a7)
//   hydro update                 cell c-3                     (a8)
//   PPB profile                  cell c-2                     (a9)
//   PPB transfers                face (c-3)+1/2
//   FCT factors                  cell c-3; limit face (c-4)+1/2
//   FV / moment update, sources, cell c-4 -> stored in place
//   CFL maximum
// so the cell written (c-4) is never read again by this pencil; the four
// cells needed as high-side ghosts are kept in a per-thread stash before they
// are overwritten.
//
// The formulas are the ones of the method description (perturbation form
// about the hydrostatic base state, Sec. 1; fourth-order interface values,
// Sec. 1; five-cell smoothness test, Sec. 1; Colella-Woodward parabolas,
// flattening and tracing; acoustic + two-shock Riemann solver in difference
// form; PPB advection of FV with three first moments and FCT to [0,1],
// Sec. 1 and Sec. 4).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <climits>

#include <type_traits>

namespace ppm {

constexpr int G = 4;  // ghost width (Sec. 4: the difference stencil reaches 4 cells)

// status flags (device int, OR-ed)
constexpr int FLAG_NONPHYS = 1;
constexpr int FLAG_TIMEOUT = 2;   // a bounded device wait gave up

template <typename R>
struct SweepArgs {
    R *q;                 // state: 9 arrays of ncell values, var stride vs
    long long vs;
    int n;                // cells along the pass
    int nlane, nblk;      // pencils: lane index (fast) x block index
    long long s_axis, s_lane, s_blk;  // element strides
    int lane_dim, blk_dim;            // physical axis of lane / block index
    int axis;
    int bc_lo, bc_hi;     // 0 periodic, 1 reflect, 2 halo planes from halo_lo / halo_hi (along the pass)
    const R *halo_lo, *halo_hi;   // BC_HALO sides: 4 ghost planes, [var][plane 0..3][pencil offset]
    long long halo_vs;            // their variable stride (4 x cells per plane)
    int grav;             // 0 none, 1 plane z, 2 central
    double org[3];
    int ioff[3];          // global index of cell 0 along each axis (a slab of a larger grid; else 0)
    double dx;
    // tables in precision R (FP64 plain: the FP64 tables themselves)
    const R *t_rho0, *t_p0, *t_g, *t_heat, *t_damp;
    int ntab;
    double s0, ds;
    R rho0_c, p0_c;       // uniform base (grav == 0)
    // FP32 form: AoS tables {rho0, p0, g (plane) or g/r (central), 0} and
    // {heat, damp, 0, 0} on s_j = s4_0 + j*ds4, s = z (plane) or r^2 (central)
    const float4 *t4_base, *t4_src;
    int ntab4;
    float s4_0, inv_ds4;
    int vec_x;            // x pass with 16-byte copies (n % 4 == 0)
    double confine_r;     // > 0: confining sphere; each pencil updates its fluid run only
    int ten;              // ten-value PPB (15 stored values per cell)
    const R *divg;        // 3-D shock dissipation: cell velocity divergence (NULL: off)
    R *vel_out;           // FP32 y/z passes with it: the final cell velocities (x, y, z arrays), else NULL
    double shock_k;       // its coefficient K
    double gamma;
    const double *dt;     // device time step
    int sources;          // apply heating/damping after the pass
    int cfl;              // accumulate max(|u_d|)+c into *smax
    unsigned long long *smax;
    int *flags;
};

// ---------------------------------------------------------------------------
// Exact (non-contracted) arithmetic for the base-state lookups, so that the
// FP64 form reproduces the base state of the reference arithmetic bit for bit
// and a state at rest stays at rest exactly.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double xadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double xsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double xmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double xdiv(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double xsqrt(double a) { return __dsqrt_rn(a); }
__device__ __forceinline__ float xadd(float a, float b) { return a + b; }
__device__ __forceinline__ float xsub(float a, float b) { return a - b; }
__device__ __forceinline__ float xmul(float a, float b) { return a * b; }
__device__ __forceinline__ float xdiv(float a, float b) { return a / b; }
__device__ __forceinline__ float xsqrt(float a) { return sqrtf(a); }

// Quotients of the pass.  FP32: the reciprocal-based approximate quotient
// (2 ulp for denominators of magnitude 2^-126 .. 2^126, the range of every
// denominator in the pass: densities, pressures, sound speeds, impedances,
// limiter sums); the full-range form costs a range test and a scaling per
// division (measured: the FP32 passes 4% faster with this one).  FP64: the
// IEEE quotient.
__device__ __forceinline__ double qdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float qdiv(float a, float b) { return __fdividef(a, b); }

// Minimum, maximum, clamp and square root in two instruction forms, chosen
// per kernel design (FF = false: compare-and-select and sqrtf; FF = true:
// fminf / fmaxf, saturation and x * rsqrt(x)).  They agree on every finite
// positive-argument input (up to the sign of a zero); which one schedules
// better depends on the kernel around it (measured: the register-window march
// is 5% slower with the second form, the tile form 6% faster).  FP64 has one
// form.
template <bool FF = false>
__device__ __forceinline__ double rsq(double a) { return sqrt(a); }
template <bool FF = false>
__device__ __forceinline__ float rsq(float a) { return FF ? a * rsqrtf(a) : sqrtf(a); }
__device__ __forceinline__ double rabs(double a) { return fabs(a); }
__device__ __forceinline__ float rabs(float a) { return fabsf(a); }
template <bool FF = false>
__device__ __forceinline__ double rmax(double a, double b) { return a > b ? a : b; }
template <bool FF = false>
__device__ __forceinline__ double rmin(double a, double b) { return a < b ? a : b; }
template <bool FF = false>
__device__ __forceinline__ float rmax(float a, float b) { return FF ? fmaxf(a, b) : (a > b ? a : b); }
template <bool FF = false>
__device__ __forceinline__ float rmin(float a, float b) { return FF ? fminf(a, b) : (a < b ? a : b); }
template <bool FF = false, typename R>
__device__ __forceinline__ R rclamp(R x, R lo, R hi) { return rmin<FF>(rmax<FF>(x, lo), hi); }
template <bool FF = false>
__device__ __forceinline__ double rsat(double x) { return rclamp(x, 0.0, 1.0); }
template <bool FF = false>
__device__ __forceinline__ float rsat(float x) { return FF ? __saturatef(x) : rclamp(x, 0.0f, 1.0f); }

template <typename R>
__device__ __forceinline__ R lerp_tab(const SweepArgs<R> &A, const R *__restrict__ tab, R s) {
    const R u = xdiv(xsub(s, (R)A.s0), (R)A.ds);
    R fl = floor(u);
    int i = (int)rmin(rmax(fl, (R)0), (R)(A.ntab - 2));
    const R w = xsub(u, (R)i);
    const R t0 = __ldg(tab + i), t1 = __ldg(tab + i + 1);
    return xadd(t0, xmul(w, xsub(t1, t0)));
}

template <typename R>
struct Base {
    R rho0, p0, g[3];
};

// Hydrostatic base state and gravity at a point (Sec. 1).
template <typename R>
__device__ __forceinline__ Base<R> base_at(const SweepArgs<R> &A, const R xyz[3]) {
    Base<R> b;
    b.g[0] = b.g[1] = b.g[2] = (R)0;
    if (A.grav == 0) {
        b.rho0 = A.rho0_c;
        b.p0 = A.p0_c;
    } else if (A.grav == 1) {
        b.rho0 = lerp_tab(A, A.t_rho0, xyz[2]);
        b.p0 = lerp_tab(A, A.t_p0, xyz[2]);
        b.g[2] = lerp_tab(A, A.t_g, xyz[2]);
    } else {
        const R r = xsqrt(xadd(xadd(xmul(xyz[0], xyz[0]), xmul(xyz[1], xyz[1])), xmul(xyz[2], xyz[2])));
        b.rho0 = lerp_tab(A, A.t_rho0, r);
        b.p0 = lerp_tab(A, A.t_p0, r);
        if (r > (R)0) {
            const R gor = xdiv(lerp_tab(A, A.t_g, r), r);
            b.g[0] = xmul(gor, xyz[0]);
            b.g[1] = xmul(gor, xyz[1]);
            b.g[2] = xmul(gor, xyz[2]);
        }
    }
    return b;
}

// The same base state from the three coordinates as scalars, with gravity
// only along the pass axis ax (no per-axis array in the pass kernel).
template <typename R>
struct BaseAx {
    R rho0, p0, g;
};
template <typename R>
__device__ __forceinline__ BaseAx<R> base_along(const SweepArgs<R> &A, R x, R y, R z, int ax) {
    BaseAx<R> b;
    b.g = (R)0;
    if (A.grav == 0) {
        b.rho0 = A.rho0_c;
        b.p0 = A.p0_c;
    } else if (A.grav == 1) {
        b.rho0 = lerp_tab(A, A.t_rho0, z);
        b.p0 = lerp_tab(A, A.t_p0, z);
        if (ax == 2) b.g = lerp_tab(A, A.t_g, z);
    } else {
        const R r = xsqrt(xadd(xadd(xmul(x, x), xmul(y, y)), xmul(z, z)));
        b.rho0 = lerp_tab(A, A.t_rho0, r);
        b.p0 = lerp_tab(A, A.t_p0, r);
        if (r > (R)0) b.g = xmul(xdiv(lerp_tab(A, A.t_g, r), r), ax == 0 ? x : (ax == 1 ? y : z));
    }
    return b;
}

template <typename R>
__device__ __forceinline__ R coord(const SweepArgs<R> &A, int d, int idx) {
    return xadd((R)A.org[d], xmul(xadd((R)(idx + A.ioff[d]), (R)0.5), (R)A.dx));
}

// ---------------------------------------------------------------------------
// Pass building blocks (one cell / one face at a time)
// ---------------------------------------------------------------------------

// a2: fourth-order interface value between a1 and a2 (Sec. 1).
template <typename R>
__device__ __forceinline__ R iface(R a0, R a1, R a2, R a3) {
    return ((R)7 * (a1 + a2) - (a0 + a3)) * (R)(1.0 / 12.0);
}

// a3: smoothness on the 5-cell stencil (Sec. 1).  Returns the constraint
// weight: 0 where T <= S/2 + 1e-9 scale (smooth: no constraint), rising
// linearly to 1 at T >= S + 2e-9 scale, with T the largest third difference
// and S the largest first or second difference of the stencil.
template <typename R, bool FF = false>
__device__ __forceinline__ R smooth5(R am2, R am1, R a0, R ap1, R ap2, R scale) {
    const R d1m2 = am1 - am2, d1m1 = a0 - am1, d10 = ap1 - a0, d1p1 = ap2 - ap1;
    const R d2m = d1m1 - d1m2, d20 = d10 - d1m1, d2p = d1p1 - d10;
    const R T = rmax<FF>(rabs(d20 - d2m), rabs(d2p - d20));
    const R S = rmax<FF>(rmax<FF>(rabs(d1m1), rabs(d10)), rmax<FF>(rmax<FF>(rabs(d2m), rabs(d20)), rabs(d2p)));
    const R fl = (R)1e-9 * scale;
    const R x = T - (R)0.5 * S - fl;
    if constexpr (std::is_same<R, float>::value) {
        // FP32: no branch (non-smooth cells are scattered, so it would
        // diverge in almost every warp)
        return rsat<FF>(qdiv(x, (R)0.5 * S + fl));
    } else {
        // FP64: keep the division (slow on this part) off the smooth path
        R w = (R)0;
        if (x > (R)0) w = rmin<FF>((R)1, x / ((R)0.5 * S + fl));
        return w;
    }
}

// a4: parabola of one variable; returns aL, aR, a6 (da = aR - aL).  The
// Colella-Woodward constraints are blended in with the detector weight w.
template <typename R, bool FF = false>
__device__ __forceinline__ void parabola(R am, R a, R ap, R aL, R aR, R f, R w, R &oL, R &oR,
                                         R &o6) {
    if (f > (R)0) {
        aL = aL + f * (a - aL);
        aR = aR + f * (a - aR);
    }
    // Constrained edges, evaluated without branches (non-smooth cells are
    // scattered, so a branch would diverge in almost every warp); w = 0
    // leaves aL, aR unchanged.
    {
        const R cL = rclamp<FF>(aL, rmin<FF>(am, a), rmax<FF>(am, a));
        const R cR = rclamp<FF>(aR, rmin<FF>(a, ap), rmax<FF>(a, ap));
        const bool ext = (cR - a) * (a - cL) <= (R)0;   // local extremum: flat
        const R da = cR - cL;
        const R dm = a - (R)0.5 * (cL + cR);
        const R d6 = da * da * (R)(1.0 / 6.0);
        const R x = da * dm;
        const bool fixL = x > d6;                        // overshoot on the left
        const bool fixR = !fixL && (-d6 > x);            // overshoot on the right
        R nL = fixL ? (R)3 * a - (R)2 * cR : cL;
        R nR = fixR ? (R)3 * a - (R)2 * cL : cR;
        nL = ext ? a : nL;
        nR = ext ? a : nR;
        aL = aL + w * (nL - aL);
        aR = aR + w * (nR - aR);
    }
    oL = aL;
    oR = aR;
    o6 = (R)6 * (a - (R)0.5 * (aL + aR));
}

// Averages of the parabola over a domain of dependence of width s (cells)
// at the right / left edge.
template <typename R>
__device__ __forceinline__ R fR(R aL, R aR, R a6, R s) {
    return aR - (R)0.5 * s * ((aR - aL) - ((R)1 - (R)(2.0 / 3.0) * s) * a6);
}
template <typename R>
__device__ __forceinline__ R fL(R aL, R aR, R a6, R s) {
    return aL + (R)0.5 * s * ((aR - aL) + ((R)1 - (R)(2.0 / 3.0) * s) * a6);
}

// Error-free transforms for the compensated FP32 update.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = a * b;
    e = fmaf(a, b, -p);
}

// Map a ghost index onto the pencil (periodic wrap or mirror).  With walls
// at both ends the pencil and its mirror images repeat with period 2n, so a
// ghost deeper than n cells (a short fluid run inside a confining sphere) is
// an image of an image: same orientation, no flip.
__device__ __forceinline__ int map_cell(int i, int n, int bl, int bh, bool &flip) {
    flip = false;
    if (i >= 0 && i < n) return i;
    if ((i < 0 && bl == 0) || (i >= n && bh == 0)) {
        const int k = i % n;
        return k < 0 ? k + n : k;
    }
    int k = i % (2 * n);
    if (k < 0) k += 2 * n;
    if (k < n) return k;
    flip = true;
    return 2 * n - 1 - k;
}
constexpr int BC_HALO = 2;   // ghost cells come from caller-supplied halo planes

// Position (cells from the low end) of face j+1/2 after the same mapping
// (faces beyond a halo side keep their own position).
__device__ __forceinline__ int map_face(int j, int n, int bl, int bh) {
    const int P = j + 1;
    if (P >= 0 && P <= n) return (P == n && bh == 0) ? 0 : P;
    if ((P < 0 && bl == BC_HALO) || (P > n && bh == BC_HALO)) return P;
    if ((P < 0 && bl == 0) || (P > n && bh == 0)) {
        const int k = P % n;
        return k < 0 ? k + n : k;
    }
    int k = P % (2 * n);
    if (k < 0) k += 2 * n;
    return k <= n ? k : 2 * n - k;
}

// Confining sphere (Sec. 3): a cell is fluid when its centre lies strictly
// inside the sphere of radius r about the coordinate origin.  Evaluated in
// FP64 without contraction, with the centre at org + (idx + 1/2) dx and the
// squares summed in x, y, z order, so every kernel classifies a cell alike.
__device__ __forceinline__ double cell_centre(double org, double dx, int idx) {
    return __dadd_rn(org, __dmul_rn(__dadd_rn((double)idx, 0.5), dx));
}
__device__ __forceinline__ bool fluid_point(double x, double y, double z, double r) {
    return __dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z)) < __dmul_rn(r, r);
}

// ---------------------------------------------------------------------------
// Asynchronous global -> shared copies (each thread copies and later reads
// only its own data, so a per-thread wait is enough: no block barrier).
// ---------------------------------------------------------------------------
template <int BYTES>
__device__ __forceinline__ void cp_async(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// FP32 table lookup: one index for all four columns.
__device__ __forceinline__ float4 tab4(const float4 *__restrict__ t, int ntab, float s0, float inv_ds, float s) {
    const float u = (s - s0) * inv_ds;
    const float fl = fminf(fmaxf(floorf(u), 0.0f), (float)(ntab - 2));
    const int i = (int)fl;
    const float w = u - fl;
    const float4 a = __ldg(t + i), b = __ldg(t + i + 1);
    return make_float4(fmaf(w, b.x - a.x, a.x), fmaf(w, b.y - a.y, a.y), fmaf(w, b.z - a.z, a.z),
                       fmaf(w, b.w - a.w, a.w));
}

__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }

// FP32 storage of FV is folded: s = FV for FV <= 1/2 and s = FV - 1 (<= -0.0)
// above, so both small concentrations and small complements (1 - FV) keep
// their significant bits; updates act on s directly (FV + d <=> s + d).
__device__ __forceinline__ float fv_unfold(float s) { return signbit(s) ? 1.0f + s : s; }
__device__ __forceinline__ float fv_complement(float s) { return signbit(s) ? -s : 1.0f - s; }
// s + d, clamped to FV in [0, 1] and refolded (all conversions are exact).
__device__ __forceinline__ float fv_add(float s, float d) {
    if (!signbit(s)) {
        const float f = s + d;
        if (!(f > 0.0f)) return 0.0f;
        if (f <= 0.5f) return f;
        if (f < 1.0f) return f - 1.0f;
        return -0.0f;
    }
    const float t = s + d;
    if (t >= 0.0f) return -0.0f;
    if (t > -0.5f) return t;
    if (t > -1.0f) return 1.0f + t;
    return 0.0f;
}
// realisability bound of a first moment: 6 FV (1 - FV), from the folded value
__device__ __forceinline__ float fv_moment_bound(float s) {
    const float a = fabsf(s);
    return 6.0f * a * (1.0f - a);
}

// ---------------------------------------------------------------------------
// The kernel.  PLAIN: FP64 storage of full rho and E (subtracting the base
// state on load and adding it back on store); otherwise deviation storage.
// ---------------------------------------------------------------------------
#ifndef PPM_SWEEP_MINB
#define PPM_SWEEP_MINB 1
#endif

#ifndef PPM_SWEEP_NB
#define PPM_SWEEP_NB 128
#endif
constexpr int SWEEP_NB = PPM_SWEEP_NB;   // threads per block
constexpr int RING = 8;         // scalar prefetch ring slots per thread
constexpr int PREF = 4;         // scalar prefetch distance (cells)

// x pass (VEC): groups of 4 cells in flight per thread (the one being read
// and two ahead; a fourth slot for 9 values), and cells staged per output
// flush (8 = one 32-byte sector per value; 4 for 15 values, so that three
// 64-thread blocks fit on an SM instead of two).
__host__ __device__ constexpr int vec_slots(int NV) { return NV > 9 ? 3 : 4; }
__host__ __device__ constexpr int vec_stage(int NV) { return NV > 9 ? 4 : 8; }

// Dynamic shared memory of one block of the pass (NV stored values per cell:
// 9, or 15 with the ten-value PPB).
// FP32 scalar path: heating and damping table rows of each cell to be
// updated, copied with the state (two 8-byte rows and the weight per slot;
// measured: the pass with sources 48.6 -> 45.7 ms at 1024^3, where a
// synchronous lookup exposed the table latency and a prefetch into
// registers cost more than it saved)
constexpr int SRC_SLOTS = 8;
template <typename R, bool VEC>
constexpr int src_ring_bytes(int NB, int NV) {
    return (!VEC && sizeof(R) == 4 && NV == 9) ? SRC_SLOTS * NB * (2 * 8 + 4) : 0;
}
template <typename R, bool VEC, int NB = SWEEP_NB, int NV = 9>
constexpr int sweep_smem_bytes() {
    return VEC ? (vec_slots(NV) * NV * NB * 16 + NV * NB * 4 * vec_stage(NV))
               : (RING * NV * NB * (int)sizeof(R) + src_ring_bytes<R, VEC>(NB, NV));
}

#ifndef PPM_SWEEP_UNROLL
#define PPM_SWEEP_UNROLL 1
#endif
constexpr int SWEEP_UNROLL = PPM_SWEEP_UNROLL;  // unroll factor of the march loop

// ---------------------------------------------------------------------------
// The kernel.  PLAIN: FP64 storage of full rho and E (subtracting the base
// state on load and adding it back on store); otherwise deviation storage.
// VEC (FP32 x pass, n % 8 == 0): each thread copies 4 consecutive cells of
// its row per variable with one 16-byte asynchronous copy, and writes its
// results back 8 cells (one whole 32-byte sector) at a time, instead of 9
// scalar accesses per cell that touch 32 different cache lines per warp.
// ---------------------------------------------------------------------------
// One block of the pass: NB consecutive pencils (lane_block) of pencil row
// blk.  Called by the single-grid kernel and by the work-list kernel.
// TEN: the ten-value PPB (FV, 3 first, 3 second and 3 mixed moments; 15
// stored values per cell), with a purely local parabola along the pass.
// DISS: 3-D shock dissipation (momentum and E' diffuse across faces where the
// cell velocity divergence marks a shock).
// HALO: the pass along z of a slab of a larger grid, a side with bc BC_HALO
// taking its 4 ghost planes from A.halo_lo / A.halo_hi (no wall there, ghost
// cells at their own position).
template <typename R, bool PLAIN, bool VEC, int NB, bool CONF = false, bool TEN = false, bool DISS = false,
          bool HALO = false, bool NSRC = false>
__device__ __forceinline__ void sweep_body(const SweepArgs<R> &A, int lane_block, int blk,
                                           unsigned char *smem_raw) {
    constexpr int SWEEP_NB = NB;
    constexpr bool F32 = std::is_same<R, float>::value;
    // instruction forms of min / max (measured in this kernel: the second
    // form pays in the detector and costs in the parabola constraints)
    constexpr bool MFS = true, MFP = false;
    static_assert(!VEC || F32, "vector path is FP32 only");
    constexpr int NV = TEN ? 15 : 9;
    const int tid = threadIdx.x;
    const int lane = lane_block * NB + threadIdx.x;
    // threads past the edge take part in the final warp reduction only
    bool active = (lane < A.nlane) && (blk < A.nblk);
    R smax_local = 0;
    bool bad = false;
    const int ax = VEC ? 0 : A.axis, t1d = (ax + 1) % 3, t2d = (ax + 2) % 3;
    const bool lane_t1 = (A.lane_dim == t1d);
    // The cells this pencil updates: [i0, i0 + n) with boundary kinds bcl,
    // bch.  Without a confining sphere that is the whole pencil; with one, it
    // is the pencil's run of fluid cells (a line meets a ball in one segment,
    // and the fluid test is monotone in the distance from the cell nearest
    // the centre), found by bisection on each side, with walls at both ends.
    int i0 = 0, n = A.n, bcl = A.bc_lo, bch = A.bc_hi;
    if (CONF && active) {
        const double c1 = cell_centre(A.org[t1d], A.dx, lane_t1 ? lane : blk);
        const double c2 = cell_centre(A.org[t2d], A.dx, lane_t1 ? blk : lane);
        auto inside = [&](int i) {
            const double ca = cell_centre(A.org[ax], A.dx, i);
            const double x = (ax == 0) ? ca : (t1d == 0 ? c1 : c2);
            const double y = (ax == 1) ? ca : (t1d == 1 ? c1 : c2);
            const double z = (ax == 2) ? ca : (t1d == 2 ? c1 : c2);
            return fluid_point(x, y, z, A.confine_r);
        };
        const int N = A.n;
        int ic = min(max((int)floor(-A.org[ax] / A.dx), 0), N - 1);
        if (!inside(ic)) {  // (a neighbour at the same distance up to rounding)
            if (ic > 0 && inside(ic - 1)) --ic;
            else if (ic + 1 < N && inside(ic + 1)) ++ic;
        }
        if (!inside(ic)) {
            active = false;
        } else {
            int lo = 0, hi = ic;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (inside(mid)) hi = mid; else lo = mid + 1;
            }
            i0 = lo;
            lo = ic;
            hi = N - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (inside(mid)) lo = mid; else hi = mid - 1;
            }
            n = lo + 1 - i0;
            bcl = bch = 1;
        }
    }
    // The lanes of a warp march over the same global cell index, each
    // taking part while it is inside its own run (plus ghosts), so that
    // their loads and stores stay coalesced when the runs start at
    // different cells.  Without a confining sphere every lane has the
    // whole pencil and this is the plain march.
    int w_lo = 0, w_hi = n;
    if constexpr (CONF) {
        w_lo = __reduce_min_sync(0xffffffffu, active ? i0 : INT_MAX);
        w_hi = __reduce_max_sync(0xffffffffu, active ? i0 + n : INT_MIN);
    }
    if (active) {
    R *__restrict__ q = A.q + (long long)lane * A.s_lane + (long long)blk * A.s_blk + (long long)i0 * A.s_axis;
    const R *__restrict__ dvp = DISS ? A.divg + (long long)lane * A.s_lane + (long long)blk * A.s_blk : nullptr;
    const long long vs = A.vs, sa = A.s_axis;
    // Cells are held in the pass frame: slot k of a cell is stored variable
    // vslot(k) (normal momentum and moment first, then the two transverse
    // ones in cyclic order), so that no per-cell array is indexed by the
    // run-time axis.
    // Ten-value form: slots 9..11 = second moments (normal, t1, t2), 12 =
    // the mixed moment of the two transverse axes, 13 / 14 = the mixed
    // moments of the normal with t1 / t2 (stored at 12 + the remaining axis).
    const int pn = 1 + ax, p1 = 1 + t1d, p2 = 1 + t2d;
    auto voff = [&](int k) -> long long {
        const int v = (k == 1) ? pn : (k == 2) ? p1 : (k == 3) ? p2
                    : (k == 6) ? pn + 5 : (k == 7) ? p1 + 5 : (k == 8) ? p2 + 5
                    : (k == 9) ? 9 + ax : (k == 10) ? 9 + t1d : (k == 11) ? 9 + t2d
                    : (k == 12) ? 12 + ax : (k == 13) ? 12 + t2d : (k == 14) ? 12 + t1d : k;
        return (long long)v * vs;
    };

    const R gam = (R)A.gamma, gm1 = (R)(A.gamma - 1.0);
    const R kk = (R)((A.gamma + 1.0) / (2.0 * A.gamma));
    const R gg1 = (R)(A.gamma / (A.gamma - 1.0));
    const double dtd = *A.dt;
    const R dt = (R)dtd;
    const R dtdx = (R)(dtd / A.dx);
    const R hdt = (R)0.5 * dt;

    // transverse position of this pencil (the lane and block indices run
    // over the two transverse axes)
    const R xt1 = coord(A, t1d, lane_t1 ? lane : blk);
    const R xt2 = coord(A, t2d, lane_t1 ? blk : lane);
    // physical coordinates of a point at coordinate `along` on the pencil
    auto point = [&](R along, R &x, R &y, R &z) {
        x = (ax == 0) ? along : (t1d == 0 ? xt1 : xt2);
        y = (ax == 1) ? along : (t1d == 1 ? xt1 : xt2);
        z = (ax == 2) ? along : (t1d == 2 ? xt1 : xt2);
    };
    const R zt = (t1d == 2) ? xt1 : xt2;  // z of the pencil when ax != 2
    const R lo = (R)A.org[ax];

    // FP32 base state: squared transverse radius, and the base state of a
    // pencil on which it does not vary (plane-parallel gravity, x/y pass)
    const float rt2 = F32 ? (float)(xt1 * xt1 + xt2 * xt2) : 0.0f;
    float4 bconst = make_float4(0.f, 0.f, 0.f, 0.f);
    if constexpr (F32) {
        if (A.grav == 0) bconst = make_float4((float)A.rho0_c, (float)A.p0_c, 0.f, 0.f);
        else if (A.grav == 1 && ax != 2) {
            bconst = tab4(A.t4_base, A.ntab4, A.s4_0, A.inv_ds4, (float)zt);
            bconst.z = 0.0f;  // vertical gravity has no component along x or y
        }
    }
    // FP32 base state (rho0, p0, g along the pass) at coordinate xa along the
    // pass.  Where it varies along the pencil the two table rows are fetched
    // one step before they are needed (issue / finish), so the table load
    // latency is off the step's dependency chain.
    const float orgf = (float)A.org[ax], dxf = (float)A.dx;
    const bool bvar = F32 && (A.grav == 2 || (A.grav == 1 && ax == 2));
    struct TabFetch {
        float4 a, b;
        float w, xa;
    };
    auto tab_issue = [&](float xa) -> TabFetch {
        TabFetch t;
        t.xa = xa;
        if (!bvar) {
            t.a = t.b = bconst;
            t.w = 0.0f;
            return t;
        }
        const float sv = (A.grav == 1) ? xa : fmaf(xa, xa, rt2);
        const float u = (sv - A.s4_0) * A.inv_ds4;
        const float fl = fminf(fmaxf(floorf(u), 0.0f), (float)(A.ntab4 - 2));
        const int i = (int)fl;
        t.a = __ldg(A.t4_base + i);
        t.b = __ldg(A.t4_base + i + 1);
        t.w = u - fl;
        return t;
    };
    auto tab_finish = [&](const TabFetch &t) -> float4 {
        if (!bvar) return bconst;
        float4 r = make_float4(fmaf(t.w, t.b.x - t.a.x, t.a.x), fmaf(t.w, t.b.y - t.a.y, t.a.y),
                               fmaf(t.w, t.b.z - t.a.z, t.a.z), 0.0f);
        if (A.grav == 2) r.z *= t.xa;  // (g/r) * x_axis
        return r;
    };
    const int io = A.ioff[ax];
    auto xcell32 = [&](int mm) { return orgf + ((float)(i0 + io + mm) + 0.5f) * dxf; };
    auto xface32 = [&](int j) { return orgf + (float)(i0 + io + map_face(j, n, bcl, bch)) * dxf; };
    // a cell beyond a halo side is its own ghost (no wrap, no mirror)
    auto halo_cell = [&](int cc) {
        return HALO && ((cc < 0 && bcl == BC_HALO) || (cc >= n && bch == BC_HALO));
    };
    auto mapc = [&](int cc, bool &fl) -> int {
        if (halo_cell(cc)) {
            fl = false;
            return cc;
        }
        return map_cell(cc, n, bcl, bch, fl);
    };
    TabFetch cell_next, face_next;
    if constexpr (F32) {
        bool fl0;
        cell_next = tab_issue(xcell32(mapc(-G, fl0)));
        face_next = tab_issue(xface32(-G - 3));
    }

    // per-thread stash of the 4 cells that serve as high-side ghosts
    // (every entry is written before it is read, since n >= 4)
    R stash[4][NV];
    // stash slot of cell m: cells 0..3 (periodic) or the last four cells
    // (walls; all cells of a run shorter than 4)
    const int stash_lo = (bch == 0) ? 0 : max(0, n - 4);

    // prefetch rings (shared memory, private to each thread)
    R *ring = reinterpret_cast<R *>(smem_raw);
    float *ringv = reinterpret_cast<float *>(smem_raw);
    constexpr int VSLOT = vec_slots(NV), VSTAGE = vec_stage(NV);
    auto vslot = [](int g) { return VSLOT == 4 ? (g & 3) : (g % VSLOT); };
    float *outv = reinterpret_cast<float *>(smem_raw) + VSLOT * NV * SWEEP_NB * 4;
    // (not in the ten-value and confined instantiations: measured slower
    // there, 65.0 -> 74.2 and 42.9 -> 43.7 ms per pass at 1024^3)
    constexpr bool SRING = F32 && !VEC && !NSRC && !TEN && !CONF;
    float2 *srow = reinterpret_cast<float2 *>(smem_raw + RING * NV * SWEEP_NB * sizeof(R));
    float *sw = reinterpret_cast<float *>(srow + SRC_SLOTS * 2 * SWEEP_NB);
    // table rows of cell cs (issued with the state copies of cell cs + PREF,
    // so they have landed when cell cs is updated, PREF iterations later)
    auto fetch_src = [&](int cs) {
        if (cs < 0 || cs >= n) return;
        const float xa = xcell32(cs);
        const float sv = (A.grav == 1) ? (ax == 2 ? xa : (float)zt) : fmaf(xa, xa, rt2);
        const float u = (sv - A.s4_0) * A.inv_ds4;
        const float fl = fminf(fmaxf(floorf(u), 0.0f), (float)(A.ntab4 - 2));
        const int r = (int)fl;
        const float2 *t2 = reinterpret_cast<const float2 *>(A.t4_src);
        const int sl = cs & (SRC_SLOTS - 1);
        cp_async<8>(srow + (sl * 2) * SWEEP_NB + tid, t2 + 2 * r);
        cp_async<8>(srow + (sl * 2 + 1) * SWEEP_NB + tid, t2 + 2 * r + 2);
        sw[sl * SWEEP_NB + tid] = u - fl;
    };
    auto fetch = [&](int cf) {
        if constexpr (SRING)
            if (A.sources) fetch_src(cf - PREF);
        if (HALO && halo_cell(cf) && cf < n + G) {
            // ghost plane of a halo side: [var][plane][pencil offset]
            const R *hb = (cf < 0) ? A.halo_lo + (long long)(cf + G) * sa : A.halo_hi + (long long)(cf - n) * sa;
            const R *src = hb + (long long)lane * A.s_lane + (long long)blk * A.s_blk;
            R *dst = ring + ((cf + G) & (RING - 1)) * NV * SWEEP_NB + tid;
#pragma unroll
            for (int v = 0; v < NV; ++v)
                cp_async<(int)sizeof(R)>(dst + v * SWEEP_NB, src + voff(v) / vs * A.halo_vs);
        } else if (cf < n) {
            bool fl;
            const int mm = map_cell(cf, n, bcl, bch, fl);
            const R *src = q + (long long)mm * sa;
            R *dst = ring + ((cf + G) & (RING - 1)) * NV * SWEEP_NB + tid;
#pragma unroll
            for (int v = 0; v < NV; ++v) cp_async<(int)sizeof(R)>(dst + v * SWEEP_NB, src + voff(v));
        }
        cp_commit();
    };
    auto fetchg = [&](int g) {  // group of cells 4g-G .. 4g-G+3 (x pass, FP32)
        const int c0 = 4 * g - G;
        if (c0 < n) {
            const int m0 = (c0 < 0) ? ((bcl == 0) ? n - 4 : 0) : c0;
            const float *src = reinterpret_cast<const float *>(q) + m0;
            float *dst = ringv + ((vslot(g) * NV) * SWEEP_NB + tid) * 4;
#pragma unroll
            for (int v = 0; v < NV; ++v) cp_async<16>(dst + v * SWEEP_NB * 4, src + voff(v));
        }
        cp_commit();
    };
    if constexpr (VEC) {
        fetchg(0);
        fetchg(1);
    } else {
#pragma unroll
        for (int k = 0; k < PREF; ++k) fetch(-G + k);
    }

    // ---- windows: slot s holds cell c-4+s --------------------------------
    R wrd[5], wu[5], wv[5], ww[5], wpd[5];     // primitives for interpolation
    R wfv[5], won[5], wo1[5], wo2[5];          // FV and moments
    R wro[5];                                  // full old density
    R wp0[5], wr0[5];                          // base state at the cell
    R wg[5];                                   // gravity along the pass
    R wfs[5];                                  // stored (FP32: folded) FV
    R wmn[5], wm1[5], wm2[5], wed[5];          // conserved momenta and E'
    R wqn[5], wq1[5], wq2[5], wc12[5], wcn1[5], wcn2[5];  // ten-value form only
    R wdv[5] = {0, 0, 0, 0, 0};                // cell divergence (shock dissipation only)
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        wrd[s] = wu[s] = wv[s] = ww[s] = wpd[s] = (R)0;
        wfv[s] = won[s] = wo1[s] = wo2[s] = (R)0;
        wro[s] = wr0[s] = wp0[s] = (R)1;
        wg[s] = wfs[s] = (R)0;
        wmn[s] = wm1[s] = wm2[s] = wed[s] = (R)0;
        wqn[s] = wq1[s] = wq2[s] = wc12[s] = wcn1[s] = wcn2[s] = (R)0;
    }
    // interface values of face (c-3)+1/2 (from the previous step)
    R afp[5] = {0, 0, 0, 0, 0};
    // traced left state of face (c-3)+1/2 (right edge of cell c-3)
    R WLp[5] = {0, 0, 0, 0, 0};
    // fluxes of face (c-4)+1/2
    R Frp = 0, Frlp = 0, Fnp = 0, Ft1p = 0, Ft2p = 0, FEp = 0, FElp = 0;
    // PPB: profile of cell c-3, face (c-4)+1/2 transfers, FCT factors of cell c-4
    R me3 = 0, ae3 = 0;
    R GLp = 0, Ap = 0, KLp = 0, KHp = 0, T1p = 0, T2p = 0, PHIp = 0, KMp = 0, sgp = 0;
    R Rp4 = 0, Rm4 = 0;
    // limited transfers of face (c-5)+1/2
    R Gq = 0, Kq = 0, T1q = 0, T2q = 0, PHIq = 0, KMq = 0, sgq = 0;
    // ten-value form: second moments of content (low / high order) and of
    // mass, transverse xi-moments, transverse second and mixed moments of
    // face (c-4)+1/2, and the same (content limited) of face (c-5)+1/2
    R K2Lp = 0, K2Hp = 0, KM2p = 0, U1p = 0, U2p = 0, Q1p = 0, Q2p = 0, C12p = 0;
    R K2q = 0, KM2q = 0, U1q = 0, U2q = 0, Q1q = 0, Q2q = 0, C12q = 0;
    // hydro update of cell c-4 (computed one step earlier)
    R rdn4 = 0, mnn4 = 0, m1n4 = 0, m2n4 = 0, edn4 = 0;

#pragma unroll SWEEP_UNROLL
    for (int cg = w_lo - G; cg < w_hi + G; ++cg) {
        const int c = CONF ? cg - i0 : cg;  // this lane's cell (index within its run)
        if (CONF && (c < -G || c >= n + G)) continue;
        // ================= a1: load cell c ==================================
        if constexpr (VEC) {
            if (((c + G) & 3) == 0) {
                fetchg(((c + G) >> 2) + 2);
                cp_wait<2>();
            }
        } else {
            fetch(c + PREF);
            cp_wait<PREF>();
        }
        R raw[NV];
        bool flip = false;
        const int m = mapc(c, flip);
        if (c >= n && !halo_cell(c)) {
            const int si = m - stash_lo;
#pragma unroll
            for (int v = 0; v < NV; ++v) raw[v] = stash[si][v];
        } else {
            if constexpr (VEC) {
                const int sub = (c + G) & 3;
                const int idx = (c < 0 && bcl == 1) ? 3 - sub : sub;
                const float *src = ringv + ((vslot((c + G) >> 2) * NV) * SWEEP_NB + tid) * 4 + idx;
#pragma unroll
                for (int v = 0; v < NV; ++v) raw[v] = src[v * SWEEP_NB * 4];
            } else {
                const R *src = ring + ((c + G) & (RING - 1)) * NV * SWEEP_NB + tid;
#pragma unroll
                for (int v = 0; v < NV; ++v) raw[v] = src[v * SWEEP_NB];
            }
            if (c >= 0) {
                const int si = c - stash_lo;
                if (si >= 0 && si < 4) {
#pragma unroll
                    for (int v = 0; v < NV; ++v) stash[si][v] = raw[v];
                }
            }
        }
        R b_rho0, b_p0, b_g;
        if constexpr (F32) {
            const float4 bb = tab_finish(cell_next);
            b_rho0 = bb.x;
            b_p0 = bb.y;
            b_g = bb.z;
            bool fln;
            cell_next = tab_issue(xcell32(mapc(c + 1, fln)));
        } else {
            R cx, cy, cz;
            point(coord(A, ax, i0 + m), cx, cy, cz);
            const BaseAx<R> b = base_along(A, cx, cy, cz, ax);
            b_rho0 = b.rho0;
            b_p0 = b.p0;
            b_g = b.g;
        }
        const R sg = flip ? (R)-1 : (R)1;
        // rotate into the pass frame and subtract the base state
        const R rd = PLAIN ? xsub(raw[0], b_rho0) : raw[0];
        const R mn = sg * raw[1];
        const R m1 = raw[2];
        const R m2 = raw[3];
        const R ed = PLAIN ? xsub(raw[4], xdiv(b_p0, gm1)) : raw[4];
        const R rho = b_rho0 + rd;
        const R rinv = qdiv((R)1, rho);
        const R u = mn * rinv, v = m1 * rinv, w = m2 * rinv;
        const R ke = (R)0.5 * (mn * u + (m1 * v + m2 * w));
        const R pd = gm1 * (ed - ke);
        // shift windows and insert cell c at slot 4
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            wrd[s] = wrd[s + 1]; wu[s] = wu[s + 1]; wv[s] = wv[s + 1]; ww[s] = ww[s + 1];
            wpd[s] = wpd[s + 1]; wfv[s] = wfv[s + 1]; won[s] = won[s + 1]; wo1[s] = wo1[s + 1];
            wo2[s] = wo2[s + 1]; wro[s] = wro[s + 1]; wp0[s] = wp0[s + 1]; wr0[s] = wr0[s + 1];
            wg[s] = wg[s + 1]; wfs[s] = wfs[s + 1];
            wmn[s] = wmn[s + 1]; wm1[s] = wm1[s + 1]; wm2[s] = wm2[s + 1]; wed[s] = wed[s + 1];
            if constexpr (DISS) wdv[s] = wdv[s + 1];
            if constexpr (TEN) {
                wqn[s] = wqn[s + 1]; wq1[s] = wq1[s + 1]; wq2[s] = wq2[s + 1];
                wc12[s] = wc12[s + 1]; wcn1[s] = wcn1[s + 1]; wcn2[s] = wcn2[s + 1];
            }
        }
        wrd[4] = rd; wu[4] = u; wv[4] = v; ww[4] = w; wpd[4] = pd;
        if constexpr (F32) {
            wfv[4] = fv_unfold(raw[5]);
        } else {
            wfv[4] = raw[5];
        }
        wfs[4] = raw[5];
        won[4] = sg * raw[6];
        wo1[4] = raw[7];
        wo2[4] = raw[8];
        wro[4] = rho; wp0[4] = b_p0; wr0[4] = b_rho0;
        wg[4] = sg * b_g;
        wmn[4] = mn; wm1[4] = m1; wm2[4] = m2; wed[4] = ed;
        if constexpr (DISS) wdv[4] = __ldg(dvp + (long long)m * sa);   // even under a mirror
        if constexpr (TEN) {
            wqn[4] = raw[9]; wq1[4] = raw[10]; wq2[4] = raw[11];
            wc12[4] = raw[12]; wcn1[4] = sg * raw[13]; wcn2[4] = sg * raw[14];
        }

        // ================= a2: interface values of face (c-2)+1/2 ==========
        R afn[5];
        afn[0] = iface(wrd[1], wrd[2], wrd[3], wrd[4]);
        afn[1] = iface(wu[1], wu[2], wu[3], wu[4]);
        afn[2] = iface(wv[1], wv[2], wv[3], wv[4]);
        afn[3] = iface(ww[1], ww[2], ww[3], ww[4]);
        afn[4] = iface(wpd[1], wpd[2], wpd[3], wpd[4]);

        // ================= a3-a5: cell c-2 (slot 2) ========================
        R WLn[5], WRc[5];
        {
            const R rho2 = wro[2];
            const R p2 = wp0[2] + wpd[2];
            const R c2 = qdiv(gam * p2, rho2);
            const R cs = rsq(c2);
            // flattening coefficient
            R f = (R)0;
            {
                const R dp1 = wpd[3] - wpd[1];
                const R dp2 = wpd[4] - wpd[0];
                const R pmin = rmin(wp0[3] + wpd[3], wp0[1] + wpd[1]);
                if (rabs(dp1) > (R)0.33 * pmin && wu[1] - wu[3] > (R)0) {
                    const R r = (dp2 != (R)0) ? qdiv(dp1, dp2) : (R)1;
                    f = rsat((R)10 * (r - (R)0.75));
                }
            }
            // parabolas of the five variables
            R aL[5], aR[5], a6[5];
            {
                const R s0 = smooth5<R, MFS>(wrd[0], wrd[1], wrd[2], wrd[3], wrd[4], rho2);
                parabola<R, MFP>(wrd[1], wrd[2], wrd[3], afp[0], afn[0], f, s0, aL[0], aR[0], a6[0]);
                const R s1 = smooth5<R, MFS>(wu[0], wu[1], wu[2], wu[3], wu[4], cs);
                parabola<R, MFP>(wu[1], wu[2], wu[3], afp[1], afn[1], f, s1, aL[1], aR[1], a6[1]);
                const R s2 = smooth5<R, MFS>(wv[0], wv[1], wv[2], wv[3], wv[4], cs);
                parabola<R, MFP>(wv[1], wv[2], wv[3], afp[2], afn[2], f, s2, aL[2], aR[2], a6[2]);
                const R s3 = smooth5<R, MFS>(ww[0], ww[1], ww[2], ww[3], ww[4], cs);
                parabola<R, MFP>(ww[1], ww[2], ww[3], afp[3], afn[3], f, s3, aL[3], aR[3], a6[3]);
                const R s4 = smooth5<R, MFS>(wpd[0], wpd[1], wpd[2], wpd[3], wpd[4], p2);
                parabola<R, MFP>(wpd[1], wpd[2], wpd[3], afp[4], afn[4], f, s4, aL[4], aR[4], a6[4]);
            }
            // characteristic tracing (waves u-c, u, u+c) + buoyancy
            const R uc = wu[2];
            const R C = rho2 * cs;
            const R lm = uc - cs, l0 = uc, lp = uc + cs;
            const R hg = hdt * (qdiv(wrd[2], rho2) * wg[2]);
            {   // right edge -> left state of face (c-2)+1/2
                const R sp = rmax(lp, (R)0) * dtdx;
                R st[5];
#pragma unroll
                for (int k = 0; k < 5; ++k) st[k] = fR(aL[k], aR[k], a6[k], sp);
                const R rr = st[0], ru = st[1], rv = st[2], rw = st[3], rp = st[4];
                if (l0 > (R)0) {
                    const R s0 = l0 * dtdx;
                    const R dr = rr - fR(aL[0], aR[0], a6[0], s0);
                    const R dp = rp - fR(aL[4], aR[4], a6[4], s0);
                    st[0] = st[0] - (dr - qdiv(dp, c2));
                    st[2] = st[2] - (rv - fR(aL[2], aR[2], a6[2], s0));
                    st[3] = st[3] - (rw - fR(aL[3], aR[3], a6[3], s0));
                }
                if (lm > (R)0) {
                    const R sm = lm * dtdx;
                    const R du = ru - fR(aL[1], aR[1], a6[1], sm);
                    const R dp = rp - fR(aL[4], aR[4], a6[4], sm);
                    const R Aa = (R)0.5 * (dp - C * du);
                    st[0] = st[0] - qdiv(Aa, c2);
                    st[1] = st[1] + qdiv(Aa, C);
                    st[4] = st[4] - Aa;
                }
                st[1] = st[1] + hg;
#pragma unroll
                for (int k = 0; k < 5; ++k) WLn[k] = st[k];
            }
            {   // left edge -> right state of face (c-3)+1/2
                const R sm = rmax(-lm, (R)0) * dtdx;
                R st[5];
#pragma unroll
                for (int k = 0; k < 5; ++k) st[k] = fL(aL[k], aR[k], a6[k], sm);
                const R rr = st[0], ru = st[1], rv = st[2], rw = st[3], rp = st[4];
                if (l0 < (R)0) {
                    const R s0 = -l0 * dtdx;
                    const R dr = rr - fL(aL[0], aR[0], a6[0], s0);
                    const R dp = rp - fL(aL[4], aR[4], a6[4], s0);
                    st[0] = st[0] - (dr - qdiv(dp, c2));
                    st[2] = st[2] - (rv - fL(aL[2], aR[2], a6[2], s0));
                    st[3] = st[3] - (rw - fL(aL[3], aR[3], a6[3], s0));
                }
                if (lp < (R)0) {
                    const R s1 = -lp * dtdx;
                    const R du = ru - fL(aL[1], aR[1], a6[1], s1);
                    const R dp = rp - fL(aL[4], aR[4], a6[4], s1);
                    const R Aa = (R)0.5 * (dp + C * du);
                    st[0] = st[0] - qdiv(Aa, c2);
                    st[1] = st[1] - qdiv(Aa, C);
                    st[4] = st[4] - Aa;
                }
                st[1] = st[1] + hg;
#pragma unroll
                for (int k = 0; k < 5; ++k) WRc[k] = st[k];
            }
        }

        // ================= a6-a7: Riemann + fluxes at face (c-3)+1/2 =======
        R Frc, Frlc, Fnc, Ft1c, Ft2c, FEc, FElc, usc;
        {
            const int j = c - 3;
            R r0, p0;
            if constexpr (F32) {
                const float4 bf = tab_finish(face_next);
                r0 = bf.x;
                p0 = bf.y;
                face_next = tab_issue(xface32(j + 1));
            } else {
                const R xf = xadd(lo, xmul((R)(i0 + io + map_face(j, n, bcl, bch)), (R)A.dx));
                R fx, fy, fz;
                point(xf, fx, fy, fz);
                const BaseAx<R> bf = base_along(A, fx, fy, fz, ax);
                r0 = bf.rho0;
                p0 = bf.p0;
            }
            const R rdL = WLp[0], uL = WLp[1], pdL = WLp[4];
            const R rdR = WRc[0], uR = WRc[1], pdR = WRc[4];
            const R rL = r0 + rdL, pL = p0 + pdL;
            const R rR = r0 + rdR, pR = p0 + pdR;
            const R CL = rsq(gam * pL * rL), CR = rsq(gam * pR * rR);
            const R pfl = (R)1e-10 * rmin(pL, pR);
            // FP32: one reciprocal per denominator, and the supersonic tests
            // below as products (the FP64 form keeps the oracle's quotients)
            R den = CL + CR;
            R pst, ust;
            if constexpr (F32) {
                const R iden = qdiv((R)1, den);
                pst = pdL + CL * (CR * (uL - uR) + (pdR - pdL)) * iden;
                ust = uL + (CR * (uR - uL) + (pdL - pdR)) * iden;
            } else {
                pst = pdL + qdiv(CL * (CR * (uL - uR) + (pdR - pdL)), den);
                ust = uL + qdiv(CR * (uR - uL) + (pdL - pdR), den);
            }
            if (p0 + pst < pfl) pst = pfl - p0;
            const R WLi = CL * rsq((R)1 + qdiv(kk * (pst - pdL), pL));
            const R WRi = CR * rsq((R)1 + qdiv(kk * (pst - pdR), pR));
            den = WLi + WRi;
            if constexpr (F32) {
                const R iden = qdiv((R)1, den);
                pst = pdL + WLi * (WRi * (uL - uR) + (pdR - pdL)) * iden;
                ust = uL + (WRi * (uR - uL) + (pdL - pdR)) * iden;
            } else {
                pst = pdL + qdiv(WLi * (WRi * (uL - uR) + (pdR - pdL)), den);
                ust = uL + qdiv(WRi * (uR - uL) + (pdL - pdR), den);
            }
            if (p0 + pst < pfl) pst = pfl - p0;
            const bool wall = (j == -1 && bcl == 1) || (j == n - 1 && bch == 1);
            if (wall) ust = (R)0;
            const bool left = (ust >= (R)0);
            const R rds = left ? rdL : rdR;
            const R pds = left ? pdL : pdR;
            const R rs = left ? rL : rR;
            const R pss = left ? pL : pR;
            R vst = left ? WLp[2] : WRc[2];
            R wst = left ? WLp[3] : WRc[3];
            const R dps = pst - pds;
            R rdst = rds + qdiv(rs * dps, gam * pss + (R)0.5 * gm1 * dps);
            {
                // the interface state is the two-shock solution at x/t = 0:
                // where both waves move to one side (supersonic flow through
                // the face) it is the upwind traced state itself; wave speeds
                // from the Lagrangian impedances (selects: no divergence)
                const bool supL = !wall && (F32 ? (uL * rL >= WLi) : (uL - qdiv(WLi, rL) >= (R)0));
                const bool supR = !wall && !supL && (F32 ? (uR * rR <= -WRi) : (uR + qdiv(WRi, rR) <= (R)0));
                ust = supL ? uL : (supR ? uR : ust);
                pst = supL ? pdL : (supR ? pdR : pst);
                rdst = supL ? rdL : (supR ? rdR : rdst);
                vst = supL ? WLp[2] : (supR ? WRc[2] : vst);
                wst = supL ? WLp[3] : (supR ? WRc[3] : wst);
            }
            const R h0 = gg1 * p0;
            const R kin = (R)0.5 * (ust * ust + (vst * vst + wst * wst));
            if constexpr (F32) {
                // mass and energy fluxes carry their large base-state parts
                // (rho0 u*, h0 u*) as exact hi+lo pairs
                float hi, e;
                two_prod(r0, ust, hi, e);
                Frc = hi;
                Frlc = e + rdst * ust;
                const float Fr = Frc + Frlc;
                float hE, eE;
                two_prod(ust, h0, hE, eE);
                FEc = hE;
                FElc = eE + (ust * (gg1 * pst) + kin * Fr);
                Fnc = Fr * ust + pst;
                Ft1c = Fr * vst;
                Ft2c = Fr * wst;
            } else {
                const R Fr = (r0 + rdst) * ust;
                Frc = Fr;
                Frlc = 0;
                Fnc = Fr * ust + pst;
                Ft1c = Fr * vst;
                Ft2c = Fr * wst;
                FEc = ust * (gg1 * pst + h0) + kin * Fr;
                FElc = 0;
            }
            if constexpr (DISS) {
                // 3-D dissipation inside shocks (Sec. 1): momentum and E'
                // diffuse with nu = K max(0, -div(u) dx - 0.05 c), the cell
                // divergences averaged to the face and c the mean sound speed
                // of the two traced states; no mass diffusion
                const R dface = (R)0.5 * (wdv[1] + wdv[2]);
                const R cface = (R)0.5 * (qdiv(CL, rL) + qdiv(CR, rR));
                const R nu = (R)A.shock_k * rmax((R)0, -(dface * (R)A.dx) - (R)0.05 * cface);
                Fnc = Fnc - nu * (wmn[2] - wmn[1]);
                Ft1c = Ft1c - nu * (wm1[2] - wm1[1]);
                Ft2c = Ft2c - nu * (wm2[2] - wm2[1]);
                if constexpr (F32)
                    FElc = FElc - nu * (wed[2] - wed[1]);
                else
                    FEc = FEc - nu * (wed[2] - wed[1]);
            }
            usc = ust;
        }

        // ================= a8: hydro update of cell c-3 (slot 1) ===========
        R rdn3, mnn3, m1n3, m2n3, edn3;
        {
            const R g = wg[1];
            const R mn3 = wmn[1], m13 = wm1[1], m23 = wm2[1], ed3 = wed[1];
            if constexpr (F32) {
                float s, e;
                two_sum(Frc, -Frp, s, e);
                const float dFr = s + (e + (Frlc - Frlp));
                rdn3 = wrd[1] - dtdx * dFr;
                two_sum(FEc, -FEp, s, e);
                const float dFE = s + (e + (FElc - FElp));
                edn3 = ed3 - dtdx * dFE + dt * g * ((R)0.5 * ((Frp + Frlp) + (Frc + Frlc)));
            } else {
                rdn3 = wrd[1] - dtdx * (Frc - Frp);
                edn3 = ed3 - dtdx * (FEc - FEp) + dt * g * ((R)0.5 * (Frp + Frc));
            }
            mnn3 = mn3 - dtdx * (Fnc - Fnp) + dt * g * ((R)0.5 * (wrd[1] + rdn3));
            m1n3 = m13 - dtdx * (Ft1c - Ft1p);
            m2n3 = m23 - dtdx * (Ft2c - Ft2p);
        }
        const R rnew3 = wr0[1] + rdn3;

        // ================= a9: PPB ==========================================
        // profile of cell c-2 (slot 2): f = FV + m xi + a2 (xi^2 - 1/12), bound-limited
        R me2, ae2;
        {
            const R F = wfv[2], mm = won[2];
            // curvature: the cell's own second moment (ten-value form), else
            // from the neighbours' slopes
            const R a2 = TEN ? wqn[2] : (R)0.25 * (won[3] - won[1]);
            const R ep = (R)0.5 * mm + a2 * (R)(1.0 / 6.0);
            const R em = a2 * (R)(1.0 / 6.0) - (R)0.5 * mm;
            R gmax = rmax(ep, em), gmin = rmin(ep, em);
            if constexpr (F32) {
                // selects, not branches: bound-limited profiles are scattered
                const bool nz = (a2 != (R)0);
                const R xv = qdiv(-mm, (R)2 * (nz ? a2 : (R)1));   // interior extremum
                const R gv = mm * xv + a2 * (xv * xv - (R)(1.0 / 12.0));
                const bool in = nz && (rabs(xv) < (R)0.5);
                gmax = in ? rmax(gmax, gv) : gmax;
                gmin = in ? rmin(gmin, gv) : gmin;
            } else if (a2 != (R)0) {
                const R xv = -mm / ((R)2 * a2);
                if (rabs(xv) < (R)0.5) {
                    const R gv = mm * xv + a2 * (xv * xv - (R)(1.0 / 12.0));
                    gmax = rmax(gmax, gv);
                    gmin = rmin(gmin, gv);
                }
            }
            R th = (R)1;
            if constexpr (F32) {
                const float omf = fv_complement(wfs[2]);
                const bool hi = gmax > omf, lo = -gmin > F;
                const float t1 = qdiv(omf, hi ? gmax : 1.0f), t2 = qdiv(F, lo ? -gmin : 1.0f);
                th = hi ? rmin(th, t1) : th;
                th = lo ? rmin(th, t2) : th;
            } else {
                if (F + gmax > (R)1) th = rmin(th, ((R)1 - F) / gmax);
                if (F + gmin < (R)0) th = rmin(th, F / (-gmin));
            }
            me2 = th * mm;
            ae2 = th * a2;
        }
        // transfers across face (c-3)+1/2: donor c-3 (slot 1) or c-2 (slot 2)
        R GLc, Ac, KLc, KHc, T1c, T2c, PHIc, KMc, sgc;
        R K2Lc = 0, K2Hc = 0, KM2c = 0, U1c = 0, U2c = 0, Q1c = 0, Q2c = 0, C12c = 0;
        {
            const R Fr = Frc + Frlc;
            const R sig = usc * dtdx;
            const R phi = dtdx * Fr;
            const bool fromleft = (sig >= (R)0);
            const R s = fromleft ? sig : -sig;
            R M1 = (R)0.5 - (R)0.5 * s;
            const R M2 = (R)0.25 - (R)0.5 * s + s * s * (R)(1.0 / 3.0);
            R M3 = (R)0.125 - (R)0.375 * s + (R)0.5 * s * s - (R)0.25 * s * s * s;
            if (!fromleft) {
                M1 = -M1;
                M3 = -M3;
            }
            const R F = fromleft ? wfv[1] : wfv[2];
            const R me = fromleft ? me3 : me2;
            const R ae = fromleft ? ae3 : ae2;
            const R ot1 = fromleft ? wo1[1] : wo1[2];
            const R ot2 = fromleft ? wo2[1] : wo2[2];
            const R phibar = F + me * M1 + ae * (M2 - (R)(1.0 / 12.0));
            const R psibar = F * M1 + me * M2 + ae * (M3 - M1 * (R)(1.0 / 12.0));
            GLc = phi * F;
            Ac = phi * phibar - GLc;
            KLc = phi * F * M1;
            KHc = phi * psibar;
            T1c = phi * ot1;
            T2c = phi * ot2;
            PHIc = phi;
            KMc = phi * M1;
            sgc = sig;
            if constexpr (TEN) {
                // second moments about the donor's centre (mean of xi^4 over
                // the slab: even power, same for both donors); transverse
                // moments with their linear variation along the pass
                const R M4 = (R)0.0625 - (R)0.25 * s + (R)0.5 * s * s - (R)0.5 * s * s * s + (R)0.2 * s * s * s * s;
                const R chibar = F * M2 + me * M3 + ae * (M4 - M2 * (R)(1.0 / 12.0));
                const R cn1 = fromleft ? wcn1[1] : wcn1[2];
                const R cn2 = fromleft ? wcn2[1] : wcn2[2];
                K2Lc = phi * F * M2;
                K2Hc = phi * chibar;
                KM2c = phi * M2;
                T1c = phi * (ot1 + cn1 * M1);
                T2c = phi * (ot2 + cn2 * M1);
                U1c = phi * (ot1 * M1 + cn1 * M2);
                U2c = phi * (ot2 * M1 + cn2 * M2);
                Q1c = phi * (fromleft ? wq1[1] : wq1[2]);
                Q2c = phi * (fromleft ? wq2[1] : wq2[2]);
                C12c = phi * (fromleft ? wc12[1] : wc12[2]);
            }
        }
        // FCT factors of cell c-3 (slot 1), bounds [0,1]
        R Rp3, Rm3;
        {
            const R rold = wro[1];
            const R cL = rold * wfv[1] - (GLc - GLp);
            const R FVL = qdiv(cL, rnew3);
            const R Pp = rmax((R)0, Ap) - rmin((R)0, Ac);
            const R Pm = rmax((R)0, Ac) - rmin((R)0, Ap);
            const R Qp = ((R)1 - FVL) * rnew3;
            const R Qm = FVL * rnew3;
            Rp3 = (Pp > (R)0) ? rsat(qdiv(Qp, Pp)) : (R)0;
            Rm3 = (Pm > (R)0) ? rsat(qdiv(Qm, Pm)) : (R)0;
        }
        // limit face (c-4)+1/2 with the factors of cells c-4 and c-3
        R Gc4, Kc4, K2c4 = 0;
        {
            const R Cf = (Ap >= (R)0) ? rmin(Rp3, Rm4) : rmin(Rp4, Rm3);
            Gc4 = GLp + Cf * Ap;
            Kc4 = KLp + Cf * (KHp - KLp);
            if constexpr (TEN) K2c4 = K2Lp + Cf * (K2Hp - K2Lp);
        }

        // ================= final update of cell c-4 (slot 0) ===============
        if (c >= G) {
            const int i = c - G;
            const R rold = wro[0];
            const R rnew = wr0[0] + rdn4;
            const R sm = sgq, sp = sgp;
            const R cold = rold * wfv[0];
            R c_out = 0, z_out = 0, z_in = 0, m_out = 0, zr_out = 0, zr_in = 0;
            if (sp >= (R)0) {
                c_out = c_out + Gc4;
                z_out = z_out + Kc4;
                m_out = m_out + PHIp;
                zr_out = zr_out + KMp;
            } else {
                const R sh = sp + (R)1;
                z_in = z_in + (-Kc4 - Gc4 * sh);
                zr_in = zr_in + (-KMp - PHIp * sh);
            }
            if (sm >= (R)0) {
                const R sh = sm - (R)1;
                z_in = z_in + (Kq + Gq * sh);
                zr_in = zr_in + (KMq + PHIq * sh);
            } else {
                c_out = c_out - Gq;
                z_out = z_out - Kq;
                m_out = m_out - PHIq;
                zr_out = zr_out - KMq;
            }
            const R sbar = (R)0.5 * (sm + sp);
            const R dZc = (cold - c_out) * sbar + z_in - z_out;
            const R Zr = (rold - m_out) * sbar + zr_in - zr_out;
            const R dPhi = PHIp - PHIq;
            const R dG = Gc4 - Gq;
            const R rinvn = qdiv((R)1, rnew);
            R fvn, fvs, bnd;
            if constexpr (F32) {
                fvs = fv_add(wfs[0], (wfv[0] * dPhi - dG) * rinvn);
                fvn = fv_unfold(fvs);
                bnd = fv_moment_bound(fvs);
            } else {
                fvn = rclamp(wfv[0] + (wfv[0] * dPhi - dG) * rinvn, (R)0, (R)1);
                fvs = fvn;
                bnd = (R)6 * fvn * ((R)1 - fvn);
            }
            R onn = won[0] + (won[0] * dPhi + (R)12 * (dZc - fvn * Zr)) * rinvn;
            R o1 = wo1[0] + (wo1[0] * dPhi - (T1p - T1q)) * rinvn;
            R o2 = wo2[0] + (wo2[0] * dPhi - (T2p - T2q)) * rinvn;
            R qnn = 0, q1n = 0, q2n = 0, c12n = 0, cn1n = 0, cn2n = 0;
            if constexpr (TEN) {
                // second moments of the content and mass pieces about this
                // cell's centre after the move, transverse xi-moments; then
                // the moments relative to the new mass distribution, in
                // difference form (the reading of the ten-value update)
                R z2_out = 0, z2_in = 0, zr2_out = 0, zr2_in = 0;
                R t1_out = 0, u1_out = 0, u1_in = 0, t2_out = 0, u2_out = 0, u2_in = 0;
                if (sp >= (R)0) {
                    z2_out = z2_out + K2c4;
                    zr2_out = zr2_out + KM2p;
                    t1_out = t1_out + T1p;
                    u1_out = u1_out + U1p;
                    t2_out = t2_out + T2p;
                    u2_out = u2_out + U2p;
                } else {
                    const R h = sp + (R)1;
                    z2_in = z2_in - (K2c4 + (R)2 * h * Kc4 + h * h * Gc4);
                    zr2_in = zr2_in - (KM2p + (R)2 * h * KMp + h * h * PHIp);
                    u1_in = u1_in - (U1p + T1p * h);
                    u2_in = u2_in - (U2p + T2p * h);
                }
                if (sm >= (R)0) {
                    const R h = sm - (R)1;
                    z2_in = z2_in + (K2q + (R)2 * h * Kq + h * h * Gq);
                    zr2_in = zr2_in + (KM2q + (R)2 * h * KMq + h * h * PHIq);
                    u1_in = u1_in + (U1q + T1q * h);
                    u2_in = u2_in + (U2q + T2q * h);
                } else {
                    z2_out = z2_out - K2q;
                    zr2_out = zr2_out - KM2q;
                    t1_out = t1_out - T1q;
                    u1_out = u1_out - U1q;
                    t2_out = t2_out - T2q;
                    u2_out = u2_out - U2q;
                }
                const R S0 = cold - c_out;
                const R S1 = rold * won[0] * (R)(1.0 / 12.0) - z_out;
                const R dZc2 = (R)2 * sbar * S1 + sbar * sbar * S0 + z2_in - z2_out;
                const R Zr2 = (R)-2 * sbar * zr_out + sbar * sbar * (rold - m_out) + zr2_in - zr2_out +
                              (rold - rnew) * (R)(1.0 / 12.0);
                const R dC2p = dZc2 + dG * (R)(1.0 / 12.0);
                qnn = wqn[0] + (wqn[0] * dPhi + (R)180 * (dC2p - fvn * Zr2) - (R)12 * onn * Zr) * rinvn;
                const R dY1 = (rold * wo1[0] - t1_out) * sbar + u1_in - u1_out;
                const R dY2 = (rold * wo2[0] - t2_out) * sbar + u2_in - u2_out;
                cn1n = wcn1[0] + (wcn1[0] * dPhi + (R)12 * (dY1 - o1 * Zr)) * rinvn;
                cn2n = wcn2[0] + (wcn2[0] * dPhi + (R)12 * (dY2 - o2 * Zr)) * rinvn;
                q1n = wq1[0] + (wq1[0] * dPhi - (Q1p - Q1q)) * rinvn;
                q2n = wq2[0] + (wq2[0] * dPhi - (Q2p - Q2q)) * rinvn;
                c12n = wc12[0] + (wc12[0] * dPhi - (C12p - C12q)) * rinvn;
                // realisability: all content at the centre / at the ends /
                // in one corner
                const R g = bnd * (R)(1.0 / 6.0);
                const R qlo = (R)-15 * g * ((R)1 + fvn), qhi = (R)15 * g * ((R)2 - fvn);
                const R bc = (R)36 * g;
                qnn = rclamp(qnn, qlo, qhi);
                q1n = rclamp(q1n, qlo, qhi);
                q2n = rclamp(q2n, qlo, qhi);
                cn1n = rclamp(cn1n, -bc, bc);
                cn2n = rclamp(cn2n, -bc, bc);
                c12n = rclamp(c12n, -bc, bc);
            }
            onn = rclamp(onn, -bnd, bnd);
            o1 = rclamp(o1, -bnd, bnd);
            o2 = rclamp(o2, -bnd, bnd);

            R rdo = rdn4, mno = mnn4, m1o = m1n4, m2o = m2n4, edo = edn4;
            if (!NSRC && A.sources) {
                R heat = 0, kd = 0;
                if constexpr (F32) {
                    if constexpr (SRING) {
                        const int sl = i & (SRC_SLOTS - 1);
                        const float2 ra = srow[(sl * 2) * SWEEP_NB + tid], rb = srow[(sl * 2 + 1) * SWEEP_NB + tid];
                        const float w = sw[sl * SWEEP_NB + tid];
                        heat = fmaf(w, rb.x - ra.x, ra.x);
                        kd = fmaf(w, rb.y - ra.y, ra.y);
                    } else {
                        const float xa = xcell32(i);
                        const float s = (A.grav == 1) ? (ax == 2 ? xa : (float)zt) : fmaf(xa, xa, rt2);
                        const float4 hs = tab4(A.t4_src, A.ntab4, A.s4_0, A.inv_ds4, s);
                        heat = hs.x;
                        kd = hs.y;
                    }
                } else {
                    R cx, cy, cz;
                    point(coord(A, ax, i0 + i), cx, cy, cz);
                    const R s = (A.grav == 1) ? cz
                                              : xsqrt(xadd(xadd(xmul(cx, cx), xmul(cy, cy)), xmul(cz, cz)));
                    if (A.t_heat) heat = lerp_tab(A, A.t_heat, s);
                    if (A.t_damp) kd = lerp_tab(A, A.t_damp, s);
                }
                if (A.t_heat) edo = edo + dt * heat;
                if (A.t_damp) {
                    const R fd = rmax((R)0, (R)1 - dt * kd);
                    const R kin = qdiv((R)0.5 * (mno * mno + (m1o * m1o + m2o * m2o)), rnew);
                    mno = mno * fd;
                    m1o = m1o * fd;
                    m2o = m2o * fd;
                    edo = edo - ((R)1 - fd * fd) * kin;
                }
            }
            // physical checks and CFL maximum on the final values
            {
                const R ri = qdiv((R)1, rnew);
                const R uu = mno * ri, vv = m1o * ri, wv_ = m2o * ri;
                if constexpr (DISS && F32 && !VEC) {
                    // the final velocities of the cell, for the next pass's
                    // divergence (the same quotient and products it would take)
                    if (A.vel_out) {
                        R *vp = A.vel_out + (q - A.q) + (long long)i * sa;
                        vp[(long long)ax * vs] = uu;
                        vp[(long long)t1d * vs] = vv;
                        vp[(long long)t2d * vs] = wv_;
                    }
                }
                const R kin = (R)0.5 * (mno * uu + (m1o * vv + m2o * wv_));
                const R pr = wp0[0] + gm1 * (edo - kin);
                if (!(rnew > (R)0) || !(pr > (R)0)) bad = true;
                if (!NSRC && A.cfl) {
                    const R spd = rmax(rmax(rabs(uu), rabs(vv)), rabs(wv_)) + rsq(gam * pr * ri);
                    smax_local = rmax(smax_local, spd);
                }
            }
            R outc[NV];
            outc[0] = PLAIN ? xadd(wr0[0], rdo) : rdo;
            outc[1] = mno;
            outc[2] = m1o;
            outc[3] = m2o;
            outc[4] = PLAIN ? xadd(xdiv(wp0[0], gm1), edo) : edo;
            outc[5] = fvs;
            outc[6] = onn;
            outc[7] = o1;
            outc[8] = o2;
            if constexpr (TEN) {
                outc[9] = qnn;
                outc[10] = q1n;
                outc[11] = q2n;
                outc[12] = c12n;
                outc[13] = cn1n;
                outc[14] = cn2n;
            }
            if constexpr (VEC) {
                // stage VSTAGE cells ([var][cell][thread]: conflict-free), then
                // VSTAGE / 4 16-byte stores per variable
                float *st = outv + (size_t)(i & (VSTAGE - 1)) * SWEEP_NB + tid;
#pragma unroll
                for (int vv = 0; vv < NV; ++vv) st[vv * SWEEP_NB * VSTAGE] = outc[vv];
                if ((i & (VSTAGE - 1)) == VSTAGE - 1) {
                    float *g = reinterpret_cast<float *>(q) + (i - (VSTAGE - 1));
                    const float *sv = outv + tid;
#pragma unroll
                    for (int vv = 0; vv < NV; ++vv) {
                        const float *r = sv + vv * SWEEP_NB * VSTAGE;
                        float4 *d = reinterpret_cast<float4 *>(g + voff(vv));
                        d[0] = make_float4(r[0], r[SWEEP_NB], r[2 * SWEEP_NB], r[3 * SWEEP_NB]);
                        if constexpr (VSTAGE == 8)
                            d[1] = make_float4(r[4 * SWEEP_NB], r[5 * SWEEP_NB], r[6 * SWEEP_NB], r[7 * SWEEP_NB]);
                    }
                }
            } else {
                R *p = q + (long long)i * sa;
#pragma unroll
                for (int vv = 0; vv < NV; ++vv) p[voff(vv)] = outc[vv];
            }
        }

        // ================= carry to the next step ===========================
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            afp[k] = afn[k];
            WLp[k] = WLn[k];
        }
        Frp = Frc; Frlp = Frlc; Fnp = Fnc; Ft1p = Ft1c; Ft2p = Ft2c; FEp = FEc; FElp = FElc;
        me3 = me2; ae3 = ae2;
        Gq = Gc4; Kq = Kc4; T1q = T1p; T2q = T2p; PHIq = PHIp; KMq = KMp; sgq = sgp;
        GLp = GLc; Ap = Ac; KLp = KLc; KHp = KHc; T1p = T1c; T2p = T2c; PHIp = PHIc; KMp = KMc; sgp = sgc;
        if constexpr (TEN) {
            K2q = K2c4; KM2q = KM2p; U1q = U1p; U2q = U2p; Q1q = Q1p; Q2q = Q2p; C12q = C12p;
            K2Lp = K2Lc; K2Hp = K2Hc; KM2p = KM2c; U1p = U1c; U2p = U2c; Q1p = Q1c; Q2p = Q2c; C12p = C12c;
        }
        Rp4 = Rp3; Rm4 = Rm3;
        rdn4 = rdn3; mnn4 = mnn3; m1n4 = m1n3; m2n4 = m2n3; edn4 = edn3;
    }
    }  // active

    if (bad) atomicOr(A.flags, FLAG_NONPHYS);
    if (!NSRC && A.cfl) {
        // warp max, then one atomic per warp (double bits of positive values
        // order like unsigned integers)
        double sm = (double)smax_local;
        for (int o = 16; o > 0; o >>= 1) sm = fmax(sm, __shfl_xor_sync(0xffffffffu, sm, o));
        if ((threadIdx.x & 31) == 0) atomicMax(A.smax, dbits(sm));
    }
}

// CONF: grid with a confining sphere (per-pencil fluid runs, lanes marching
// on the global cell index); a separate instantiation so that the plain
// grid's kernel carries none of it.
// NB: threads per block (the ten-value x pass uses 64, so that two blocks
// with their 16-byte rings fit in shared memory).
template <typename R, bool PLAIN, bool VEC, bool CONF = false, bool TEN = false, bool DISS = false,
          int NB = SWEEP_NB, bool HALO = false, bool NSRC = false>
__global__ void __launch_bounds__(NB, PPM_SWEEP_MINB) sweep_kernel(const SweepArgs<R> A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    sweep_body<R, PLAIN, VEC, NB, CONF, TEN, DISS, HALO, NSRC>(A, blockIdx.x, blockIdx.y, smem_raw);
}

// ---------------------------------------------------------------------------
// Ensemble pass: one launch walks a work list of (box, lane block, pencil row)
// items of many independent boxes; each box has its own arguments (shape,
// tables, dt, CFL accumulator).  persistent != 0: a grid of resident blocks
// takes items from a counter in list order (longest pencils first); else one
// block per item.
// ---------------------------------------------------------------------------
struct WorkItem {
    int box, lane_block, blk, pad;
};

template <typename R, bool PLAIN, bool VEC, int NB, bool NSRC = false>
__global__ void __launch_bounds__(NB, 1) sweep_ensemble_kernel(const SweepArgs<R> *__restrict__ args,
                                                               const WorkItem *__restrict__ work, int nwork,
                                                               int *counter, int persistent) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ SweepArgs<R> sA;
    __shared__ int s_item;
    int item = blockIdx.x;
    if (persistent) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        item = s_item;
    }
    while (item < nwork) {
        const WorkItem w = work[item];
        if (threadIdx.x == 0) sA = args[w.box];
        __syncthreads();
        sweep_body<R, PLAIN, VEC, NB, false, false, false, false, NSRC>(sA, w.lane_block, w.blk, smem_raw);
        __syncthreads();
        if (!persistent) break;
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        item = s_item;
    }
}

// ---------------------------------------------------------------------------
// Whole double step of an ensemble in one launch.  The work list holds the
// items of the six passes X Y Z Z Y X of every box in pass order (item.pad =
// pass * 2 + vec); a resident grid takes items from a ticket counter in list
// order.  An item of pass s > 0 of box b first waits until every item of pass
// s-1 of box b is done (done[(s-1) nbox + b] == need[...]), so the pass
// reads a complete state; as items are handed out in list order, an item
// only ever waits for items already held by running blocks, and the earliest
// unfinished item has nothing to wait for.  Ordering across SMs: the block
// that finishes an item fences and then counts it (release); the waiting
// thread reads the count with acquire semantics and the block's loads follow
// it through a block barrier.  Each wait is bounded: after ENS_WAIT_NS of
// polling the block sets FLAG_TIMEOUT in its box's flags and leaves (every
// item depending on it then gives up the same way), so the host reports
// PPM_ETIMEOUT and the context stays usable.  wait_test != 0 (tests of that
// path only): the first item of every block waits for a count that no item
// ever reaches.
// ---------------------------------------------------------------------------
constexpr unsigned long long ENS_WAIT_NS = 2000000000ull;   // a wait gives up after 2 s
constexpr long long ENS_WAIT_POLLS = 1ll << 26;            // and after this many polls in any case

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}

__device__ __forceinline__ int ld_acquire_gpu(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <typename R, bool PLAIN, int NB>
__global__ void __launch_bounds__(NB, 1) sweep_ensemble_step_kernel(const SweepArgs<R> *__restrict__ args, int nbox,
                                                                    const WorkItem *__restrict__ work, int nwork,
                                                                    int *ticket, int *done, const int *need,
                                                                    int wait_test) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ SweepArgs<R> sA;
    __shared__ int s_item, s_fail;
    bool first = true;
    for (;;) {
        if (threadIdx.x == 0) {
            s_item = atomicAdd(ticket, 1);
            s_fail = 0;
        }
        __syncthreads();
        const int item = s_item;
        if (item >= nwork) break;
        const WorkItem w = work[item];
        const int pass = w.pad >> 1, vec = w.pad & 1;
        if (threadIdx.x == 0) {
            const bool test = wait_test && first;
            if (pass > 0 || test) {
                const int *cnt = test ? ticket + 1 : done + (pass - 1) * nbox + w.box;
                const int want = test ? INT_MAX : need[(pass - 1) * nbox + w.box];
                long long it = 0;
                const unsigned long long t0 = global_ns();
                while (ld_acquire_gpu(cnt) < want) {
                    if (++it > ENS_WAIT_POLLS || global_ns() - t0 > ENS_WAIT_NS) {
                        s_fail = 1;
                        break;
                    }
                    __nanosleep(256);
                }
            }
            if (!s_fail) sA = args[pass * nbox + w.box];
        }
        first = false;
        __syncthreads();
        if (s_fail) {
            if (threadIdx.x == 0) atomicOr(args[pass * nbox + w.box].flags, FLAG_TIMEOUT);
            return;
        }
        if (vec) {
            if constexpr (!PLAIN) sweep_body<R, PLAIN, true, NB>(sA, w.lane_block, w.blk, smem_raw);
        } else {
            sweep_body<R, PLAIN, false, NB>(sA, w.lane_block, w.blk, smem_raw);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(done + pass * nbox + w.box, 1);
        }
    }
}

}  // namespace ppm
