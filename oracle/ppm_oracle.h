/*
 * ppm_oracle.h -- plain FP64 CPU oracle for the PPM+PPB 1-D sweeps.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, obviously-correct statement of
 * what the directionally split PPM gas dynamics + PPB fractional-volume sweep
 * computes (Woodward et al., Sec. 1 and Sec. 4).  Only the tests, the
 * package's smoke check and the benchmark's CPU-baseline leg may load it; the
 * CUDA library never includes, links or calls it, and the two share no code.
 *
 * Every function works on full (not base-subtracted) FP64 state arrays
 * q[9] = (rho, rho*u, rho*v, rho*w, E, FV, m_x, m_y, m_z), each nx*ny*nz with
 * x fastest (q[15] with the second and mixed moments when nmom == 9).
 * Internally each 1-D pass gathers one pencil at a time, subtracts the
 * hydrostatic base state (Sec. 1: the stored initial state is removed from
 * the scheme with care), runs the pass step by step on whole-pencil arrays,
 * and scatters back.
 *
 * Parity status of each step (what pins it, besides the CUDA path agreeing):
 *   interface values, parabolas, tracing, Riemann, fluxes, update: pinned by
 *     exact Riemann solutions (Sod, Lax), exact preservation of uniform and
 *     hydrostatic states, conservation, axis-permutation symmetry, and the
 *     measured convergence order on smooth advection;
 *   PPB advection: pinned by bounds, conservation, exact transport of linear
 *     and quadratic profiles and of the first moment at constant velocity;
 *   the pencil machinery (gather, ghost and face mapping, base state at
 *     faces, stencil offsets): pinned bit for bit by a separately written
 *     whole-grid, array-at-a-time statement of one four-value pass;
 *   smoothness-detector constants, flattening constants, PPB curvature and
 *     FCT limiter details: parity unpinned against the paper (it prints no
 *     formulas for them); pinned only through the invariants above.
 */
#ifndef PPM_ORACLE_H
#define PPM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int nx, ny, nz;
    double x0, y0, z0;      /* low corner of the grid */
    double dx;              /* uniform cubic cells (Sec. 1: uniform Cartesian grid) */
    double gamma;           /* gamma-law gas */
    int bc[6];              /* -x,+x,-y,+y,-z,+z : 0 periodic, 1 reflecting */
    int grav;               /* 0 none (uniform base), 1 plane-parallel in z, 2 central */
    int ntab;               /* profile tables on s_i = s0 + i*ds, i < ntab (ntab >= 2) */
    double s0, ds;
    const double *rho0, *p0, *g;   /* base density, pressure, signed acceleration along +s */
    const double *heat, *damp;     /* optional (NULL): heating rate, damping rate */
    double confine_r;       /* > 0: confining sphere of this radius about the coordinate
                               origin (Sec. 3); cells whose centre is not strictly inside
                               are solid: never updated, not part of the CFL maximum, and
                               every fluid run of a pencil has reflecting walls at its ends.
                               Requires reflecting walls on all six cube faces. */
    double domega;          /* rotation ramp (Sec. 3): velocity domega * (-y, x, 0) added to
                               every fluid cell once per double step (0 = none) */
    int nmom;               /* FV moments carried: 3 (or 0: first moments only, q[9]) or 9
                               (the ten-value PPB of Sec. 1/4, q[15]: after the first moments
                               q[9..11] = second moments along x, y, z and q[12..14] = the mixed
                               moments yz, xz, xy) */
    double shock_k;         /* > 0: 3-D dissipation inside shocks (Sec. 1) with this coefficient
                               K: in each pass, momentum and E' diffuse across a face with
                               nu = K max(0, -div(u) dx - 0.05 c), div(u) the 3-D velocity
                               divergence of the pass's input state averaged to the face
                               (grid passes only; not with a confining sphere) */
} oracle_problem;

/* One 1-D pass along axis (0=x,1=y,2=z) over the whole grid, in place.
 * sources: bit 0 applies heating/damping to every updated cell after the
 * pass, bit 1 the rotation increment domega. */
void oracle_sweep(const oracle_problem *pb, double *q[9], int axis, double dt, int sources);

/* One Strang double step: X Y Z [heat/damp] Z Y X [heat/damp, rotation], same dt. */
void oracle_double_step(const oracle_problem *pb, double *q[9], double dt);

/* dt = cfl * dx / max over cells of (max_d |u_d| + c). */
double oracle_cfl_dt(const oracle_problem *pb, double *const q[9], double cfl);

/* One pass of a single pencil: in[v][i], out[v][i] for i < n (n = extent of
 * the grid along axis); (ja, jb) are the pencil's transverse cell indices in
 * cyclic order (axis+1, axis+2). */
void oracle_sweep_pencil(const oracle_problem *pb, int axis, int ja, int jb,
                         double *const in[9], double *out[9], double dt, int sources);

/* One z pass of the slab of global planes [k0, k0+nzl) of the grid of pb
 * (no confining sphere),
 * for a domain decomposition into z slabs: q[v] holds nx*ny*(nzl+8) values,
 * plane 0 = global plane k0-4, i.e. 4 halo planes on each side filled by the
 * caller (neighbours' planes, or the wrapped / mirrored planes of the global
 * boundary, raw: normal components are flipped here as for any ghost).
 * Only planes 4 .. 4+nzl-1 are updated.  With correct halos the result is
 * identical to the same planes of oracle_sweep over the whole grid. */
void oracle_sweep_z_slab(const oracle_problem *pb, double *q[9], int k0, int nzl, double dt, int sources);

/* Conserved totals (x dV) M, Px, Py, Pz, E, sum rho*FV, sum FV; spherical
 * shell averages (nbins bins of width rmax/nbins; per bin rho, p, FV, |u|,
 * u_r^2, volume-weighted; empty bins 0); max Mach number. */
void oracle_diagnostics(const oracle_problem *pb, double *const q[9], double totals[7],
                        int nbins, double rmax, double *profiles, double *max_mach);

/* The cell velocity divergence the shock dissipation uses (out: ncell). */
void oracle_divergence(const oracle_problem *pb, double *const q[9], double *out);

/* Event counters since the last reset: [0] cells with a non-smooth hydro
 * variable, [1] cells flattened, [2] PPB profiles bound-limited, [3] faces
 * FCT-limited (C<1), [4] moment-bound clamps, [5] cells visited, [6] faces
 * with shock dissipation, [7] faces where both two-shock waves move to one
 * side (supersonic flow; the upwind traced state is the interface state). */
void oracle_counters(long long out[8]);
void oracle_reset_counters(void);

/* Counted arithmetic: runs one pass along axis on a copy of q with every
 * add/sub/mul/div/sqrt counted.  out[0] = flops per cell, out[1] = selects
 * (min/max/abs/compare) per cell. */
void oracle_count_flops(const oracle_problem *pb, double *const q[9], int axis, double dt,
                        double out[2]);

/* Threads used by the OpenMP loops (0 = library default). */
void oracle_set_threads(int n);
int oracle_get_threads(void);

#ifdef __cplusplus
}
#endif
#endif
