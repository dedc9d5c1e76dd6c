/*
 * ppm.h -- C ABI of libppm.so: directionally split PPM gas dynamics with PPB
 * fractional-volume advection on a uniform 3-D Cartesian grid, on one GPU.
 *
 * The method is the one summarised by Woodward, Lin, Mao, Andrassy & Herwig,
 * "Simulating 3-D Stellar Hydrodynamics using PPM and PPB Multifluid Gas
 * Dynamics on CPU and CPU+GPU Nodes": Sec. 1 (high-order interface values,
 * constraints only where the 5-cell smoothness test fails, subtraction of the
 * hydrostatic initial state, PPB advection of the fractional volume FV),
 * Sec. 4 (1-D passes over grid pencils, stencil reaching 4 cells).
 *
 * Conventions shared by every call
 *   - Return value: PPM_OK (0) or a negative ppm_status.  After an error the
 *     context stays usable unless the status is PPM_ECUDA; ppm_last_error()
 *     gives a one-line message.
 *   - State: 9 arrays q[0..8] = (rho, rho*u, rho*v, rho*w, E, FV, m_x, m_y,
 *     m_z), each nx*ny*nz doubles with x fastest (index (k*ny + j)*nx + i).
 *     rho and E are full values (the base state is never subtracted in the
 *     caller's arrays).  FV is the volume fraction of the tracked fluid and
 *     m_d = 12 * integral over the cell of xi_d * FV (xi in [-1/2,1/2]).
 *     With nmom = 9 (ten-value PPB) 15 arrays: q[9..11] = q_d = 180 *
 *     integral of (xi_d^2 - 1/12) FV, q[12..14] = 144 * integral of
 *     (xi_y xi_z, xi_x xi_z, xi_x xi_y) FV.  The q[] parameters below have
 *     6 + nmom entries.
 *   - Memory: the library owns all device memory; caller arrays are read or
 *     written only during the call and never retained.  Host pointers may
 *     be pageable or pinned.
 *   - Threads: one context per host thread at a time.  Work is queued on the
 *     context's stream (given at creation, or created by the library).
 */
#ifndef PPM_H
#define PPM_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ppm_ctx ppm_ctx;

typedef enum {
    PPM_OK = 0,
    PPM_EINVAL = -1,     /* bad argument (sizes, pointers, ranges) */
    PPM_ENOMEM = -2,     /* device or host allocation failed */
    PPM_ECUDA = -3,      /* CUDA runtime error: the context must be destroyed */
    PPM_ENONPHYS = -4,   /* a pass produced rho<=0, p<=0 or a non-finite value */
    PPM_ECFL = -5,       /* requested time step exceeds the CFL limit (cfl > 1) */
    PPM_ETIMEOUT = -6,   /* a bounded device wait gave up (tile pass: a TMA copy never completed) */
    PPM_ESTATE = -7      /* call out of order (e.g. step with device dt before any cfl_dt) */
} ppm_status;

typedef enum { PPM_BC_PERIODIC = 0, PPM_BC_REFLECT = 1 } ppm_bc;

typedef enum {
    PPM_GRAV_NONE = 0,     /* uniform base state (rho0[0], p0[0]), no gravity */
    PPM_GRAV_PLANE_Z = 1,  /* base state and gravity g(z) along +z, tables in z */
    PPM_GRAV_CENTRAL = 2   /* spherically symmetric base, g(r) radial, tables in r */
} ppm_grav_kind;

typedef enum {
    PPM_FP64_PLAIN = 0,     /* FP64 storage of full rho, E and FP64 arithmetic */
    PPM_FP32_DEVIATION = 1  /* FP32 storage of rho-rho0, E-p0/(gamma-1); FP32 arithmetic,
                               FP64 base tables, conversions and reductions */
} ppm_precision;

typedef enum { PPM_MEM_HOST = 0, PPM_MEM_DEVICE = 1 } ppm_mem;

/* Hydrostatic base state (Sec. 1: the initial, spherically symmetric state is
 * kept and removed from the scheme) on a uniform coordinate grid
 * s_i = s0 + i*ds, i < ntab (ntab >= 2); s = z (PLANE_Z) or r (CENTRAL),
 * linear interpolation, ends extrapolated from the last interval.
 * g is the signed acceleration along +s.  Arrays are host FP64 and copied. */
typedef struct {
    int kind;              /* ppm_grav_kind */
    int ntab;
    double s0, ds;
    const double *rho0, *p0, *g;
} ppm_gravity;

typedef struct {
    double x0, y0, z0;     /* low corner of the grid */
    double dx;             /* cell size (cubic cells) */
    int precision;         /* ppm_precision */
    const double *heat;    /* optional: heating rate per unit volume on the gravity grid (NULL) */
    const double *damp;    /* optional: velocity damping rate on the gravity grid (NULL) */
    void *stream;          /* cudaStream_t to queue work on, or NULL for a private stream */
    int device;            /* CUDA device ordinal */
    double confine_r;      /* > 0: confining sphere of this radius about the coordinate
                              origin (Sec. 3: the star is enclosed in an impenetrable,
                              immovable sphere inscribed in the cube).  A cell is fluid
                              when its centre (x0 + (i+1/2) dx, ...) lies strictly inside,
                              tested in FP64 as x*x + y*y + z*z < r*r.  Each pass updates
                              every pencil's run of fluid cells with reflecting walls at its
                              ends; solid cells are never read or written by a pass and are
                              left out of the CFL maximum (diagnostics still sum them).  The
                              tapered gravity of Sec. 3 is the caller's g table.  Needs
                              PPM_BC_REFLECT on all six faces (else EINVAL); 0 = off. */
    int nmom;              /* FV moments carried per cell: 3 (or 0) = first moments only;
                              9 = the ten-value PPB of Sec. 1/4 (first, second and mixed
                              moments; each pass uses the cell's own parabola).  With 9 the
                              state has 15 arrays (below); not combined with confine_r
                              (EINVAL). */
    double shock_k;        /* > 0: 3-D dissipation inside shocks (Sec. 1) with coefficient K:
                              before each pass a kernel takes the velocity divergence of
                              every cell (central differences, boundary ghosts as in the
                              passes), and the pass diffuses momentum and E' across each face
                              with nu = K max(0, -div(u) dx - 0.05 c) (divergence averaged to
                              the face, c the mean sound speed of the traced states); mass is
                              not diffused.  0 = off; not combined with confine_r or nmom 9
                              (EINVAL).  Device memory: 4 B per cell for the divergence, and in
                              FP32 12 B per cell more for the cell velocities that the y and z
                              passes of ppm_step leave for the divergence before the next pass
                              (equal to the one taken from the state up to FP32 rounding). */
    int halo_z;            /* z slab of a larger grid (domain decomposition, Sec. 4/5: a grid
                              brick is updated from its neighbours' boundary planes): bit 0 /
                              bit 1 = the low / high z face takes 4 halo planes from the caller
                              (ppm_slab_halo) instead of a boundary condition; its bc entry is
                              ignored, and a z face without halo planes must be reflecting.  The
                              halo planes must hold the neighbouring cells' current values before
                              each z pass, so a slab is advanced pass by pass (ppm_sweep), not by
                              ppm_step; give z0 of the whole grid and the slab's z_index0.  Not
                              combined with confine_r, nmom 9 or shock_k (EINVAL).  0 = off. */
    int z_index0;          /* global index of the context's first z plane: cell centres are at
                              z0 + (z_index0 + k + 1/2) dx, so that a slab whose z0 is the
                              global grid's computes every position exactly as the whole grid
                              does (bit-equal base states); 0 for a whole grid. */
} ppm_options;

/* Create a context: nx, ny, nz >= 4; gamma > 1; bc[6] per face
 * (-x,+x,-y,+y,-z,+z), periodic faces must come in pairs; grav, opt not NULL.
 * Allocates the state (6 + nmom values per cell in the chosen precision) and
 * copies the tables to the device.  EINVAL / ENOMEM / ECUDA. */
int ppm_create(ppm_ctx **out, int nx, int ny, int nz, double gamma, const int bc[6],
               const ppm_gravity *grav, const ppm_options *opt);

/* Upload the whole state from host FP64 arrays (full variables, layout above;
 * 6 + nmom arrays).  FP32 form: rho - rho0 and E - p0/(gamma-1) are formed in
 * FP64 on the device before rounding; FV and the moments are clipped to their
 * bounds.  Host arrays in page-locked memory that the device can address
 * (cudaHostAlloc / cudaHostRegister) are read in place by the conversion
 * kernel, in slabs of about 2^26 cells; other host arrays go through two
 * device staging buffers in turn (copies overlapping the conversion).  The
 * call returns when done.  Invalidates the device time step (call
 * ppm_cfl_dt). */
int ppm_set_state(ppm_ctx *ctx, const double *const q[]);

/* Download the whole state to host FP64 arrays (full variables); page-locked
 * host arrays are written in place, others through the staging buffers. */
int ppm_get_state(ppm_ctx *ctx, double *const q[]);

/* Same for the sub-box lo <= (i,j,k) < hi; arrays are (hi-lo) boxes with x
 * fastest, on the host (mem = PPM_MEM_HOST) or on the context's device
 * (PPM_MEM_DEVICE).  EINVAL for an empty or out-of-range box, a NULL array,
 * or (host) a box whose x-y plane exceeds 2^24 cells. */
int ppm_set_region(ppm_ctx *ctx, const int lo[3], const int hi[3], const double *const q[], int mem);
int ppm_get_region(ppm_ctx *ctx, const int lo[3], const int hi[3], double *const q[], int mem);

/* CFL time step: dt = cfl * dx / max over cells of
 * (max_d |u_d| + c), c = sqrt(gamma p / rho), reduced in FP64 on the device.
 * After ppm_step the maximum taken by the step's last pass (or rotation
 * increment) on the final values is used; after an upload, a single pass or
 * context creation one grid pass takes it afresh.  0 < cfl <= 1 (else ECFL).
 * dt_out may be NULL: the value then stays on the device for
 * ppm_step(ctx, 0).  Returns ENONPHYS if a previous pass flagged a
 * non-physical cell. */
int ppm_cfl_dt(ppm_ctx *ctx, double cfl, double *dt_out);

/* One Strang double step (Sec. 1 / Sec. 4 directional splitting):
 * passes X Y Z [heating/damping] Z Y X [heating/damping, rotation increment],
 * all with the same dt, as one CUDA graph launch.  dt > 0 uses that value;
 * dt <= 0 uses the device value from the last ppm_cfl_dt or, after a step,
 * the CFL maximum fused into that step's last pass (ESTATE if there is
 * none).  Never waits for the device. */
int ppm_step(ppm_ctx *ctx, double dt);

/* One 1-D pass along axis (0=x, 1=y, 2=z) with time step dt > 0.
 * sources (0..3, else EINVAL): bit 0 applies heating/damping after the
 * pass, bit 1 the rotation increment of ppm_set_rotation. */
int ppm_sweep(ppm_ctx *ctx, int axis, double dt, int sources);

/* Rotation ramp (Sec. 3: a solid-body rotational flow is added gradually
 * over the first several thousand steps, until the wanted rate is reached).
 * Every ppm_step queued after this call adds, after its last X pass, the
 * velocity domega * (-y, x, 0) (rotation about the z axis through the
 * coordinate origin) to every fluid cell, E gaining the kinetic energy it
 * adds: new momentum m + rho*du, new E = E + m.du + rho|du|^2/2; the device
 * CFL maximum for the next step is then taken on the rotated state.  One
 * extra kernel per step while domega != 0; call with 0 to end the ramp.
 * ppm_sweep applies it with sources bit 1.  Host state only (no device
 * work, no wait); EINVAL if not finite. */
int ppm_set_rotation(ppm_ctx *ctx, double domega);

/* Form of the FP32 pass kernel (the arithmetic of a pass, Sec. 1 and Sec. 4,
 * is the same in both; results agree with the FP64 oracle at the FP32
 * tolerances, not bit for bit with each other):
 *   PPM_PASS_MARCH: one thread per pencil marching along it with a five-cell
 *     register window (every context; the FP64 form always uses it);
 *   PPM_PASS_TILE: 256 threads per 8 pencils, each taking one cell of a
 *     32-cell chunk through every stage, stages joined by shared-memory
 *     rings, chunks moved by TMA in both directions.  Needs the FP32
 *     four-value form without a confining sphere or shock dissipation, and
 *     nx % 4 == 0 (else EINVAL).
 * The choice holds for later steps and passes of the context (the step
 * graph is captured again). */
enum { PPM_PASS_MARCH = 0, PPM_PASS_TILE = 1 };
int ppm_set_pass_design(ppm_ctx *ctx, int design);
/* The same per pass axis (design[3] for the x, y, z passes). */
int ppm_set_pass_designs(ppm_ctx *ctx, const int design[3]);
/* The current design of each axis and whether PPM_PASS_TILE applies (either
 * may be NULL). */
int ppm_get_pass_design(const ppm_ctx *ctx, int design[3], int *tile_available);
/* Autotuner of the single-box pass: when the tile form applies, times one
 * pass of each design along each axis on the current state (a copy of the
 * state is saved in device memory and restored after every timed pass, so
 * the state is unchanged; ENOMEM when the copy does not fit) and keeps the
 * faster design per axis.  cache_path (may be NULL): text file of
 * "signature<TAB>design_x design_y design_z" lines, signature = GPU name,
 * extents, precision, gravity kind, boundaries, sources and PPB form; a
 * matching line is used without timing (*from_cache = 1).  Needs a valid
 * state; the device time step must be recomputed afterwards (ppm_cfl_dt). */
int ppm_tune(ppm_ctx *ctx, const char *cache_path, int *from_cache);

/* Halo planes of a slab context (halo_z).  ppm_slab_halo: the device buffer
 * of the low (side 0) or high (side 1) halo planes, layout [var][plane 0..3,
 * outward order from the slab: planes k0-4..k0-1 below, k0+nz..k0+nz+3
 * above][ny][nx] in the context's storage format (FP32 deviations or FP64
 * full values), and its size; EINVAL for a face without halo planes.
 * ppm_slab_pack: copies the context's own 4 boundary planes of that side
 * (planes 0..3 or nz-4..nz-1, same layout) into a device buffer, e.g. the
 * neighbouring slab's halo buffer, queued on the context's stream.  Both
 * contexts must share precision and base state; the caller orders the copy
 * against the two contexts' streams.  These carry no arithmetic of the
 * method: the exchange step of a decomposition into z slabs. */
int ppm_slab_halo(ppm_ctx *ctx, int side, void **dev_ptr, size_t *bytes);
int ppm_slab_pack(ppm_ctx *ctx, int side, void *dst_dev);

/* Device durations (ms) of the six passes X Y Z Z Y X of the most recent
 * ppm_step, from CUDA events recorded inside the step graph between its pass
 * launches (with the 3-D shock dissipation a pass includes its divergence
 * kernel).  Waits for that step to finish.  ESTATE before the first step. */
int ppm_pass_times(ppm_ctx *ctx, double ms[6]);

/* Reductions of the current state to FP64 accuracy:
 * totals[7] = (M, Px, Py, Pz, E, sum rho*FV, sum FV), each times dx^3 (FP32
 * form: each thread sums its cells as float pairs with exact error terms,
 * added into FP64 every 32 cells, plus the FP64 sums of the base state; the
 * first call builds the cached base state, 12 bytes per cell);
 * profiles (may be NULL when nbins == 0): nbins x 5 volume averages of
 * (rho, p, FV, |u|, u_r^2) over shells of width rmax/nbins about the
 * coordinate origin (Sec. 1: averages on spherical surfaces), 0 <= nbins <= 1024;
 * max_mach (may be NULL): max |u|/c.  Synchronises with the device. */
int ppm_diagnostics(ppm_ctx *ctx, double totals[7], int nbins, double rmax, double *profiles,
                    double *max_mach);

/* Wait for all queued work; returns ENONPHYS if a pass flagged a
 * non-physical cell since the last check (the flag is then cleared). */
int ppm_sync(ppm_ctx *ctx);

/* Number of kernel launches queued by this context so far (for accounting). */
long long ppm_launch_count(const ppm_ctx *ctx);

/* Largest nz accepted by ppm_totals_noalloc (size of its fixed scratch). */
#define PPM_NOALLOC_MAX_PLANES 8192

/* Conserved totals of a state the caller keeps on the device, without any
 * device allocation.  The paper has no counterpart: this entry point exists
 * for callers that cannot let a library call cudaMalloc -- a code whose own
 * pool allocator owns (and budgets in advance) all device memory, or a step
 * loop that cannot take the device-wide synchronisation an allocation may
 * cause.  It does not need a context.
 *   q_dev[9]   device pointers to the FP64 full variables (rho, rho*u, rho*v,
 *              rho*w, E, FV, m_x, m_y, m_z; the moments are not read), each
 *              nx*ny*nz with x fastest; read only.
 *   dx         cell size; the totals are multiplied by dx^3.
 *   totals_dev device pointer to 7 doubles written with (M, Px, Py, Pz, E,
 *              sum rho*FV, sum FV) * dx^3, the same quantities as the
 *              totals of ppm_diagnostics; plane sums are added in z order, so
 *              repeated calls give identical results.
 *   stream     cudaStream_t to queue on (NULL: the legacy default stream);
 *              returns without waiting for the device.
 * Limits: nz <= PPM_NOALLOC_MAX_PLANES (else EINVAL with a message from
 * ppm_last_error(NULL)).  Scratch: a fixed static device array of
 * PPM_NOALLOC_MAX_PLANES x 8 doubles (512 KiB), held by every GPU that loads
 * the library until the process exits.  All calls on a device share that one
 * array and it keeps the last call's contents; each call overwrites the rows
 * it uses before reading them (nothing needs clearing), and calls that
 * overlap on the GPU (for example on two streams) race on it.  Each call
 * looks up the array's device address in the current context
 * (cudaGetSymbolAddress, which allocates nothing once the library's device
 * code is loaded), so a device reset between calls leaves no stale address.
 * The first call on each device is its set-up: CUDA loads device code lazily
 * by default, so that call may load this library's module and map the array,
 * which can allocate device memory.  Make the first call once, outside any
 * budgeted step loop and before any stream capture.  Errors: EINVAL (NULL
 * pointers, extents, nz too large), ECUDA (an earlier CUDA error still
 * pending -- reported, not cleared -- or the lookup or a launch failed; the
 * message names which). */
int ppm_totals_noalloc(const double *const q_dev[9], int nx, int ny, int nz, double dx,
                       double *totals_dev, void *stream);

/* ---------------------------------------------------------------------------
 * Ensembles: many independent boxes of uneven shapes advanced together, one
 * kernel launch per pass for all boxes (a work list of pencil blocks, longest
 * pencils first), the whole double step captured as one CUDA graph.  Each
 * box keeps its own time step from its own CFL maximum.  This is the batched
 * form of the same passes (Sec. 4: the grid-pencil updates are nearly
 * independent of one another).
 * ------------------------------------------------------------------------- */
typedef struct ppm_ens ppm_ens;

typedef struct {
    int n[3];              /* nx, ny, nz >= 4 */
    int bc[6];             /* as for ppm_create */
    ppm_gravity grav;      /* this box's base-state tables */
    double x0, y0, z0, dx; /* low corner and cell size */
    const double *heat;    /* optional source tables on grav's grid (NULL) */
    const double *damp;
} ppm_box;

/* Create nbox (1..4096) boxes sharing gamma, precision, device and stream
 * (NULL: private stream).  Each box is a ppm_ctx internally; EINVAL names the
 * offending box. */
int ppm_ensemble_create(ppm_ens **out, int nbox, const ppm_box *boxes, double gamma, int precision,
                        void *stream, int device);
/* Per-box state transfers (same layout and semantics as ppm_set_state etc.). */
int ppm_ensemble_set_state(ppm_ens *e, int box, const double *const q[9]);
int ppm_ensemble_set_region(ppm_ens *e, int box, const int lo[3], const int hi[3], const double *const q[9],
                            int mem);
int ppm_ensemble_get_state(ppm_ens *e, int box, double *const q[9]);
/* CFL time step of every box (dt_out: nbox doubles, or NULL to keep them on
 * the device). */
int ppm_ensemble_cfl_dt(ppm_ens *e, double cfl, double *dt_out);
/* One Strang double step of every box as one graph launch; dt > 0: that dt
 * for all boxes; dt <= 0: each box's device dt (ESTATE before any cfl). */
int ppm_ensemble_step(ppm_ens *e, double dt);
/* Totals (to FP64 accuracy) and max Mach of one box (as ppm_diagnostics). */
int ppm_ensemble_diagnostics(ppm_ens *e, int box, double totals[7], double *max_mach);
/* Wait for the ensemble's work; ENONPHYS if any box flagged a bad cell. */
int ppm_ensemble_sync(ppm_ens *e);
/* Tile configuration per axis: block = pencils per block (32, 64 or 128;
 * FP64: 128; small boxes leave fewer lanes idle in smaller blocks), persistent != 0: a resident grid takes work items from a counter
 * instead of one block per item; vec (axis 0 only): 16-byte x-pass copies for
 * boxes with nx % 8 == 0 (FP32). */
int ppm_ensemble_set_config(ppm_ens *e, int axis, int block, int persistent, int vec);
/* Launch mode of a double step.  PPM_ENS_PER_PASS: one launch per pass (as
 * configured above).  PPM_ENS_ONE_LAUNCH: the six passes of every box in one
 * launch of a resident grid taking 128-pencil items of all passes in order
 * from a counter; an item of a box's pass waits (bounded: two seconds)
 * until that box's previous pass is complete, so the passes of different
 * boxes overlap; results are bit for bit those of PPM_ENS_PER_PASS.  A wait
 * that gives up makes ppm_ensemble_sync return PPM_ETIMEOUT (the states are
 * then undefined; the context stays usable).  The step graph is then the dt
 * kernel plus one launch. */
enum { PPM_ENS_PER_PASS = 0, PPM_ENS_ONE_LAUNCH = 1 };
int ppm_ensemble_set_launch_mode(ppm_ens *e, int mode);
int ppm_ensemble_get_launch_mode(const ppm_ens *e);
/* For tests of the failure path only: with on != 0, the first item each
 * block takes in PPM_ENS_ONE_LAUNCH mode waits for a count that no item ever
 * reaches, so every wait runs out and the step ends with PPM_ETIMEOUT. */
int ppm_ensemble_set_wait_test(ppm_ens *e, int on);
/* cfg[7] = {block_x, persistent_x, block_y, persistent_y, block_z, persistent_z, vec}. */
int ppm_ensemble_get_config(const ppm_ens *e, int cfg[7]);
/* Autotuner: times every configuration of each axis on the current states
 * (saved and restored around the timing, so they are unchanged) and keeps the
 * fastest.  cache_path (may be NULL): text file of "signature	config" lines,
 * signature = GPU name, precision and the sorted box shapes; a matching line
 * is used without timing (*from_cache = 1).  Needs valid states; the device
 * time steps must be recomputed afterwards (ppm_ensemble_cfl_dt). */
int ppm_ensemble_tune(ppm_ens *e, const char *cache_path, int *from_cache);
long long ppm_ensemble_launch_count(const ppm_ens *e);
const char *ppm_ensemble_last_error(const ppm_ens *e);
void ppm_ensemble_destroy(ppm_ens *e);

/* Last error message of this context (or of the last failed ppm_create when
 * ctx is NULL). */
const char *ppm_last_error(const ppm_ctx *ctx);

/* Release all device memory, the graph and (if private) the stream. */
void ppm_destroy(ppm_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* PPM_H */
