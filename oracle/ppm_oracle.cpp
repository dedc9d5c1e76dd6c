/*
 * ppm_oracle.cpp -- plain FP64 CPU oracle for the PPM+PPB 1-D sweeps.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg; never by the CUDA library.  See ppm_oracle.h
 * for what pins each step.
 *
 * The paper (Woodward et al., Sec. 1 and Sec. 4) names the ingredients of the
 * pass but prints no formulas; each step below states the published method it
 * restates and the reading taken where the paper is silent:
 *   - perturbation form about a hydrostatic base state (Sec. 1, the stored
 *     initial state removed from the scheme): rho' = rho - rho0,
 *     E' = E - p0/(gamma-1), p' = p - p0;
 *   - interface values one order higher than the parabola (Sec. 1): the
 *     fourth-order centred formula of Colella & Woodward (1984);
 *   - smoothness judged on the 5-cell stencil centred on the cell, no
 *     monotonicity constraints where smooth (Sec. 1): third differences
 *     compared against first and second differences (a reading);
 *   - parabola, monotonicity constraints, flattening and characteristic
 *     tracing: Colella & Woodward (1984);
 *   - approximate Riemann solver: acoustic guess plus one two-shock update,
 *     written in difference form so equal states give back exactly p' and u;
 *   - PPB fractional-volume advection (Sec. 1, Sec. 4; van Leer's scheme VI
 *     lineage): FV with its three first moments, parabolic sub-cell profile,
 *     exact swept-region integrals, Zalesak (1979) flux-corrected transport
 *     for 0 <= FV <= 1;
 *   - directional splitting (Sec. 1, Sec. 4), ghost width 4 (Sec. 4).
 * Compile with -ffp-contract=off: no fused multiply-adds.
 */
#include "ppm_oracle.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr int G = 4;                     // ghost cells per side (Sec. 4: stencil reaches 4 cells)
constexpr double C_SMOOTH = 0.5;         // detector: smooth iff T <= C_SMOOTH * S + EPS_SMOOTH * scale
constexpr double EPS_SMOOTH = 1e-9;      // detector floor, relative to rho / c / p of the cell
constexpr double EPS_SHOCK = 0.33;       // flattening: relative pressure jump
constexpr double OMEGA1 = 0.75, OMEGA2 = 10.0;
constexpr double P_FLOOR = 1e-10;        // Riemann: p* >= P_FLOOR * min(pL, pR)
constexpr double SHOCK_EPS = 0.05;       // 3-D dissipation acts where -div(u) dx > SHOCK_EPS c

std::atomic<long long> g_cnt[8];
int g_threads = 0;

// --------------------------------------------------------------------------
// Scalar types: plain double, and a counted double for the flop census.
// --------------------------------------------------------------------------
struct Counted {
    double v;
    static thread_local long long flops;
    static thread_local long long selects;
    Counted() : v(0.0) {}
    Counted(double x) : v(x) {}  // NOLINT: implicit by design
};
thread_local long long Counted::flops = 0;
thread_local long long Counted::selects = 0;

inline Counted operator+(Counted a, Counted b) { ++Counted::flops; return Counted(a.v + b.v); }
inline Counted operator-(Counted a, Counted b) { ++Counted::flops; return Counted(a.v - b.v); }
inline Counted operator*(Counted a, Counted b) { ++Counted::flops; return Counted(a.v * b.v); }
inline Counted operator/(Counted a, Counted b) { ++Counted::flops; return Counted(a.v / b.v); }
inline Counted operator-(Counted a) { return Counted(-a.v); }
inline Counted &operator+=(Counted &a, Counted b) { a = a + b; return a; }
inline Counted &operator-=(Counted &a, Counted b) { a = a - b; return a; }
inline Counted &operator*=(Counted &a, Counted b) { a = a * b; return a; }
inline bool operator<(Counted a, Counted b) { ++Counted::selects; return a.v < b.v; }
inline bool operator>(Counted a, Counted b) { ++Counted::selects; return a.v > b.v; }
inline bool operator<=(Counted a, Counted b) { ++Counted::selects; return a.v <= b.v; }
inline bool operator>=(Counted a, Counted b) { ++Counted::selects; return a.v >= b.v; }
inline bool operator!=(Counted a, Counted b) { ++Counted::selects; return a.v != b.v; }

inline double val(double x) { return x; }
inline double val(Counted x) { return x.v; }
inline double Sqrt(double x) { return std::sqrt(x); }
inline Counted Sqrt(Counted x) { ++Counted::flops; return Counted(std::sqrt(x.v)); }
inline double Abs(double x) { return std::fabs(x); }
inline Counted Abs(Counted x) { ++Counted::selects; return Counted(std::fabs(x.v)); }
inline double Max(double a, double b) { return a > b ? a : b; }
inline Counted Max(Counted a, Counted b) { ++Counted::selects; return a.v > b.v ? a : b; }
inline double Min(double a, double b) { return a < b ? a : b; }
inline Counted Min(Counted a, Counted b) { ++Counted::selects; return a.v < b.v ? a : b; }

template <class R> inline R Clamp(R x, R lo, R hi) { return Min(Max(x, lo), hi); }

// --------------------------------------------------------------------------
// Base state and source tables: linear interpolation on a uniform grid.
// --------------------------------------------------------------------------
template <class R>
R lerp_tab(const oracle_problem *pb, const double *tab, R s) {
    R u = (s - R(pb->s0)) / R(pb->ds);
    double fl = std::floor(val(u));
    int i = (int)std::min(std::max(fl, 0.0), (double)(pb->ntab - 2));
    R w = u - R((double)i);
    return R(tab[i]) + w * (R(tab[i + 1]) - R(tab[i]));
}

template <class R>
struct BasePoint {
    R rho0, p0, g[3];
};

// Hydrostatic base state and gravity at a point (Sec. 1: the initial,
// spherically symmetric state saved on the grid).
template <class R>
BasePoint<R> base_at(const oracle_problem *pb, const R xyz[3]) {
    BasePoint<R> b;
    b.g[0] = b.g[1] = b.g[2] = R(0.0);
    if (pb->grav == 0) {
        b.rho0 = R(pb->rho0[0]);
        b.p0 = R(pb->p0[0]);
    } else if (pb->grav == 1) {
        b.rho0 = lerp_tab(pb, pb->rho0, xyz[2]);
        b.p0 = lerp_tab(pb, pb->p0, xyz[2]);
        b.g[2] = lerp_tab(pb, pb->g, xyz[2]);
    } else {
        R r = Sqrt(xyz[0] * xyz[0] + xyz[1] * xyz[1] + xyz[2] * xyz[2]);
        b.rho0 = lerp_tab(pb, pb->rho0, r);
        b.p0 = lerp_tab(pb, pb->p0, r);
        if (r > R(0.0)) {
            R gor = lerp_tab(pb, pb->g, r) / r;
            for (int d = 0; d < 3; ++d) b.g[d] = gor * xyz[d];
        }
    }
    return b;
}

// Table coordinate of a point for the heating / damping profiles.
template <class R>
R source_coord(const oracle_problem *pb, const R xyz[3]) {
    if (pb->grav == 1) return xyz[2];
    return Sqrt(xyz[0] * xyz[0] + xyz[1] * xyz[1] + xyz[2] * xyz[2]);
}

inline int extent(const oracle_problem *pb, int a) { return a == 0 ? pb->nx : (a == 1 ? pb->ny : pb->nz); }
inline double origin(const oracle_problem *pb, int a) { return a == 0 ? pb->x0 : (a == 1 ? pb->y0 : pb->z0); }

// Ghost-cell index mapping along a pencil (periodic wrap or mirror).  A
// pencil with walls at both ends and its mirror images repeat with period 2n,
// so a ghost deeper than n cells (a short fluid run inside a confining
// sphere) is an image of an image: same orientation, no flip.
inline int map_cell(int i, int n, int bc_lo, int bc_hi, bool *flip) {
    *flip = false;
    if (i >= 0 && i < n) return i;
    if ((i < 0 && bc_lo == 0) || (i >= n && bc_hi == 0)) {
        int k = i % n;
        return k < 0 ? k + n : k;
    }
    int k = i % (2 * n);
    if (k < 0) k += 2 * n;
    if (k < n) return k;
    *flip = true;
    return 2 * n - 1 - k;
}

// Position (in cells from the low boundary) of face j+1/2 after mapping
// through the boundary conditions (same images as map_cell).
inline int map_face(int j, int n, int bc_lo, int bc_hi) {
    const int P = j + 1;
    if (P >= 0 && P <= n) return (P == n && bc_hi == 0) ? 0 : P;
    if ((P < 0 && bc_lo == 0) || (P > n && bc_hi == 0)) {
        int k = P % n;
        return k < 0 ? k + n : k;
    }
    int k = P % (2 * n);
    if (k < 0) k += 2 * n;
    return k <= n ? k : 2 * n - k;
}

inline size_t cell_index(const oracle_problem *pb, int axis, int i, int ja, int jb) {
    int ijk[3];
    ijk[axis] = i;
    ijk[(axis + 1) % 3] = ja;
    ijk[(axis + 2) % 3] = jb;
    return ((size_t)ijk[2] * pb->ny + ijk[1]) * pb->nx + ijk[0];
}

template <class R>
void cell_position(const oracle_problem *pb, int axis, int i, int ja, int jb, R xyz[3]) {
    int ijk[3];
    ijk[axis] = i;
    ijk[(axis + 1) % 3] = ja;
    ijk[(axis + 2) % 3] = jb;
    for (int d = 0; d < 3; ++d) xyz[d] = R(origin(pb, d)) + (R((double)ijk[d]) + R(0.5)) * R(pb->dx);
}

// Confining sphere (Sec. 3: the star sits inside an impenetrable, immovable
// sphere inscribed in the cube): a cell is fluid when its centre lies
// strictly inside the sphere of radius confine_r about the coordinate origin.
inline bool fluid_cell(const oracle_problem *pb, const double xyz[3]) {
    if (!(pb->confine_r > 0.0)) return true;
    return xyz[0] * xyz[0] + xyz[1] * xyz[1] + xyz[2] * xyz[2] < pb->confine_r * pb->confine_r;
}

// The fluid cells of a pencil, [i0, i0 + n): the whole pencil without a
// confining sphere.  A line meets a ball in one segment, so they are
// contiguous (checked); false when the pencil has none.
bool pencil_run(const oracle_problem *pb, int axis, int ja, int jb, int *i0, int *n) {
    const int N = extent(pb, axis);
    if (!(pb->confine_r > 0.0)) {
        *i0 = 0;
        *n = N;
        return true;
    }
    int a = -1, b = -1, count = 0;
    for (int i = 0; i < N; ++i) {
        double xyz[3];
        cell_position<double>(pb, axis, i, ja, jb, xyz);
        if (fluid_cell(pb, xyz)) {
            if (a < 0) a = i;
            b = i + 1;
            ++count;
        }
    }
    if (a < 0) return false;
    if (count != b - a) {
        std::fprintf(stderr, "oracle: fluid cells of a pencil are not contiguous\n");
        std::abort();
    }
    *i0 = a;
    *n = b - a;
    return true;
}

// --------------------------------------------------------------------------
// One pencil: all per-cell and per-face arrays of one 1-D pass.
// Cell i lives at [i+G] for i in [-G, n+G); face j+1/2 lives at [j+G].
// --------------------------------------------------------------------------
enum { V_R = 0, V_U = 1, V_V = 2, V_W = 3, V_P = 4, NH = 5 };

template <class R>
struct Pencil {
    int n = 0, axis = 0, ja = 0, jb = 0;
    int i0 = 0;                 // global index (along the pass) of local cell 0
    bool confined = false;      // a fluid run inside a confining sphere: walls at both ends
    bool wall_lo = false, wall_hi = false;
    // conserved, deviation form, rotated frame (n = along the pass)
    std::vector<R> rd, mn, mt1, mt2, ed, fv, on, ot1, ot2;
    // base state at cells and faces
    std::vector<R> rho0c, p0c, gn, rho0f, p0f;
    // primitives
    std::vector<R> rho, cs, c2, pfull;
    std::vector<R> W[NH];                       // rho', u, v, w, p'
    std::vector<R> af[NH];                      // interface values
    std::vector<R> wgt[NH];                     // constraint weight, 0 = smooth
    std::vector<R> flat;
    std::vector<R> PL[NH], PR[NH], PD[NH], P6[NH];
    std::vector<R> WL[NH], WR[NH];              // traced states left/right of face j+1/2
    std::vector<R> us, ps, Fr, Fn, Ft1, Ft2, FE; // Riemann + fluxes at faces
    std::vector<R> rdn, mnn, mt1n, mt2n, edn;   // hydro update
    std::vector<R> meff, aeff;                  // PPB bound-limited profile coefficients
    std::vector<R> GL, GH, KL, KH, T1, T2;      // PPB face transfers
    std::vector<R> PHI, KM;                     // mass transfer and its first moment
    std::vector<R> Rp, Rm, Gf, Kf;              // FCT
    std::vector<R> fvn, onn, ot1n, ot2n;
    // ten-value PPB (nmom == 9): second moments along the pass (qn) and across
    // it (q1, q2), mixed moments across (c12) and with the pass axis (cn1, cn2)
    bool ten = false;
    std::vector<R> qn, q1, q2, c12, cn1, cn2, qnn, q1n, q2n, c12n, cn1n, cn2n;
    // 3-D shock dissipation: velocity divergence of each cell (pass start)
    const double *divg = nullptr;
    std::vector<R> dv;
    long long c_diss = 0;
    long long c_sup = 0;       // faces sampled on the upwind side (supersonic)
    std::vector<R> K2L, K2H, K2f, KM2, U1, U2, Q1, Q2, C12;
    long long c_nonsmooth = 0, c_flat = 0, c_theta = 0, c_fct = 0, c_clamp = 0;

    void alloc(int n_) {
        n = n_;
        size_t m = (size_t)n + 2 * G;
        for (auto *v : {&rd, &mn, &mt1, &mt2, &ed, &fv, &on, &ot1, &ot2, &rho0c, &p0c, &gn,
                        &rho0f, &p0f, &rho, &cs, &c2, &pfull, &flat, &us, &ps, &Fr, &Fn, &Ft1,
                        &Ft2, &FE, &rdn, &mnn, &mt1n, &mt2n, &edn, &meff, &aeff, &GL, &GH, &KL,
                        &KH, &T1, &T2, &PHI, &KM, &Rp, &Rm, &Gf, &Kf, &fvn, &onn, &ot1n, &ot2n,
                        &qn, &q1, &q2, &c12, &cn1, &cn2, &qnn, &q1n, &q2n, &c12n, &cn1n, &cn2n,
                        &K2L, &K2H, &K2f, &KM2, &U1, &U2, &Q1, &Q2, &C12, &dv})
            v->assign(m, R(0.0));
        for (int k = 0; k < NH; ++k) {
            for (auto *v : {&W[k], &af[k], &PL[k], &PR[k], &PD[k], &P6[k], &WL[k], &WR[k]})
                v->assign(m, R(0.0));
            wgt[k].assign(m, R(0.0));
        }
    }
    static int at(int i) { return i + G; }
};

// Step a1: gather one pencil with ghosts, subtract the base state.
template <class R>
void gather(const oracle_problem *pb, Pencil<R> &P, double *const q[9]) {
    const int a = P.axis, n = P.n;
    const int bl = P.confined ? 1 : pb->bc[2 * a], bh = P.confined ? 1 : pb->bc[2 * a + 1];
    P.wall_lo = (bl == 1);
    P.wall_hi = (bh == 1);
    const R gm1 = R(pb->gamma - 1.0);
    const int t1 = (a + 1) % 3, t2 = (a + 2) % 3;
    for (int i = -G; i < n + G; ++i) {
        bool flip;
        int m = P.i0 + map_cell(i, n, bl, bh, &flip);
        size_t c = cell_index(pb, a, m, P.ja, P.jb);
        R xyz[3];
        cell_position(pb, a, m, P.ja, P.jb, xyz);
        BasePoint<R> b = base_at(pb, xyz);
        const int k = Pencil<R>::at(i);
        R sgn = flip ? R(-1.0) : R(1.0);
        P.rho0c[k] = b.rho0;
        P.p0c[k] = b.p0;
        P.gn[k] = flip ? -b.g[a] : b.g[a];
        P.rd[k] = R(q[0][c]) - b.rho0;
        P.mn[k] = flip ? -R(q[1 + a][c]) : R(q[1 + a][c]);
        P.mt1[k] = R(q[1 + t1][c]);
        P.mt2[k] = R(q[1 + t2][c]);
        P.ed[k] = R(q[4][c]) - b.p0 / gm1;
        P.fv[k] = R(q[5][c]);
        P.on[k] = flip ? -R(q[6 + a][c]) : R(q[6 + a][c]);
        P.ot1[k] = R(q[6 + t1][c]);
        P.ot2[k] = R(q[6 + t2][c]);
        if (P.divg) P.dv[k] = R(P.divg[c]);   // even under a mirror
        if (P.ten) {
            // q[9+d]: second moment along d; q[12+e]: mixed moment of the two
            // axes other than e.  A mirror flips the moments odd in the normal.
            P.qn[k] = R(q[9 + a][c]);
            P.q1[k] = R(q[9 + t1][c]);
            P.q2[k] = R(q[9 + t2][c]);
            P.c12[k] = R(q[12 + a][c]);
            P.cn1[k] = flip ? -R(q[12 + t2][c]) : R(q[12 + t2][c]);
            P.cn2[k] = flip ? -R(q[12 + t1][c]) : R(q[12 + t1][c]);
        }
        (void)sgn;
    }
    // base state at faces j+1/2, j in [-G, n+G-1]
    const R lo = R(origin(pb, a));
    for (int j = -G; j < n + G; ++j) {
        int Pf = map_face(j, n, bl, bh);
        R xyz[3];
        cell_position(pb, a, 0, P.ja, P.jb, xyz);
        xyz[a] = lo + R((double)(P.i0 + Pf)) * R(pb->dx);
        BasePoint<R> b = base_at(pb, xyz);
        P.rho0f[Pencil<R>::at(j)] = b.rho0;
        P.p0f[Pencil<R>::at(j)] = b.p0;
    }
}

// Step a1 (cont.): primitive variables in perturbation form; p' from E'
// with the base energy cancelled exactly (Sec. 1).
template <class R>
void primitives(const oracle_problem *pb, Pencil<R> &P) {
    const R gam = R(pb->gamma), gm1 = R(pb->gamma - 1.0);
    for (int i = -G; i < P.n + G; ++i) {
        const int k = Pencil<R>::at(i);
        R rho = P.rho0c[k] + P.rd[k];
        R u = P.mn[k] / rho, v = P.mt1[k] / rho, w = P.mt2[k] / rho;
        R ke = R(0.5) * (P.mn[k] * u + (P.mt1[k] * v + P.mt2[k] * w));
        R pd = gm1 * (P.ed[k] - ke);
        R p = P.p0c[k] + pd;
        R c2 = gam * p / rho;
        P.rho[k] = rho;
        P.pfull[k] = p;
        P.c2[k] = c2;
        P.cs[k] = Sqrt(c2);
        P.W[V_R][k] = P.rd[k];
        P.W[V_U][k] = u;
        P.W[V_V][k] = v;
        P.W[V_W][k] = w;
        P.W[V_P][k] = pd;
    }
}

// Step a2: interface values, fourth order (one order above the parabola, Sec. 1).
template <class R>
void interface_values(Pencil<R> &P) {
    for (int v = 0; v < NH; ++v)
        for (int j = -G + 1; j <= P.n + G - 3; ++j) {
            const auto &a = P.W[v];
            const int k = Pencil<R>::at(j);
            P.af[v][k] = (R(7.0) * (a[k] + a[k + 1]) - (a[k - 1] + a[k + 2])) * R(1.0 / 12.0);
        }
}

// Step a3: smoothness on the 5-cell stencil centred on the cell (Sec. 1).
// Reading: third differences T against first/second differences S.  The
// judgment is made continuous so that it does not amplify round-off: the
// constraint weight is w = 0 where T <= C_SMOOTH*S + EPS_SMOOTH*scale (smooth:
// no constraint at all), rising linearly to w = 1 (full constraints) at
// T >= S + 2*EPS_SMOOTH*scale; scale is the cell's full density (for rho'),
// sound speed (velocities) or full pressure (p'), so that round-off noise on
// flat data counts as smooth.
template <class R>
void smoothness(Pencil<R> &P) {
    for (int v = 0; v < NH; ++v)
        for (int i = -G + 2; i <= P.n + G - 3; ++i) {
            const auto &a = P.W[v];
            const int k = Pencil<R>::at(i);
            const R scale = (v == V_R) ? P.rho[k] : ((v == V_P) ? P.pfull[k] : P.cs[k]);
            R d1m2 = a[k - 1] - a[k - 2];
            R d1m1 = a[k] - a[k - 1];
            R d10 = a[k + 1] - a[k];
            R d1p1 = a[k + 2] - a[k + 1];
            R d2m = d1m1 - d1m2, d20 = d10 - d1m1, d2p = d1p1 - d10;
            R T = Max(Abs(d20 - d2m), Abs(d2p - d20));
            R S = Max(Max(Abs(d1m1), Abs(d10)), Max(Max(Abs(d2m), Abs(d20)), Abs(d2p)));
            R fl = R(EPS_SMOOTH) * scale;
            R x = T - R(C_SMOOTH) * S - fl;
            R w = R(0.0);
            if (x > R(0.0)) w = Min(R(1.0), x / (R(1.0 - C_SMOOTH) * S + fl));
            P.wgt[v][k] = w;
        }
    for (int i = 0; i < P.n; ++i) {
        const int k = Pencil<R>::at(i);
        bool any = false;
        for (int v = 0; v < NH; ++v) any = any || (val(P.wgt[v][k]) > 0.0);
        if (any) ++P.c_nonsmooth;
    }
}

// Step a3 (cont.): shock flattening coefficient (Colella & Woodward 1984),
// without the neighbour maximum so the stencil stays within +-2 cells.
template <class R>
void flattening(Pencil<R> &P) {
    for (int i = -G + 2; i <= P.n + G - 3; ++i) {
        const int k = Pencil<R>::at(i);
        const auto &pd = P.W[V_P];
        const auto &u = P.W[V_U];
        R dp1 = pd[k + 1] - pd[k - 1];
        R dp2 = pd[k + 2] - pd[k - 2];
        R pmin = Min(P.pfull[k + 1], P.pfull[k - 1]);
        R f = R(0.0);
        if (Abs(dp1) > R(EPS_SHOCK) * pmin && u[k - 1] - u[k + 1] > R(0.0)) {
            R r = (dp2 != R(0.0)) ? dp1 / dp2 : R(1.0);
            f = Clamp(R(OMEGA2) * (r - R(OMEGA1)), R(0.0), R(1.0));
        }
        P.flat[k] = f;
        if (i >= 0 && i < P.n && val(f) > 0.0) ++P.c_flat;
    }
}

// Step a4: parabolas; constraints only where the detector found the cell
// non-smooth (Sec. 1), in the form of Colella & Woodward (1984), blended in
// with the detector's weight w (w = 1: fully constrained edges).
template <class R>
void parabolas(Pencil<R> &P) {
    for (int v = 0; v < NH; ++v)
        for (int i = -G + 2; i <= P.n + G - 3; ++i) {
            const int k = Pencil<R>::at(i);
            const auto &A = P.W[v];
            R a = A[k];
            R aL = P.af[v][k - 1], aR = P.af[v][k];
            R f = P.flat[k];
            if (f > R(0.0)) {
                aL = aL + f * (a - aL);
                aR = aR + f * (a - aR);
            }
            const R w = P.wgt[v][k];
            if (w > R(0.0)) {
                R cL = Clamp(aL, Min(A[k - 1], a), Max(A[k - 1], a));
                R cR = Clamp(aR, Min(a, A[k + 1]), Max(a, A[k + 1]));
                if ((cR - a) * (a - cL) <= R(0.0)) {
                    cL = a;
                    cR = a;
                } else {
                    R da = cR - cL;
                    R dm = a - R(0.5) * (cL + cR);
                    R d6 = da * da * R(1.0 / 6.0);
                    if (da * dm > d6)
                        cL = R(3.0) * a - R(2.0) * cR;
                    else if (-d6 > da * dm)
                        cR = R(3.0) * a - R(2.0) * cL;
                }
                aL = aL + w * (cL - aL);
                aR = aR + w * (cR - aR);
            }
            P.PL[v][k] = aL;
            P.PR[v][k] = aR;
            P.PD[v][k] = aR - aL;
            P.P6[v][k] = R(6.0) * (a - R(0.5) * (aL + aR));
        }
}

// Average of the parabola over a domain of dependence of width sigma (in
// cells) next to the right edge (fR) or the left edge (fL) of the cell.
template <class R>
inline R fR(const Pencil<R> &P, int v, int k, R s) {
    return P.PR[v][k] - R(0.5) * s * (P.PD[v][k] - (R(1.0) - R(2.0 / 3.0) * s) * P.P6[v][k]);
}
template <class R>
inline R fL(const Pencil<R> &P, int v, int k, R s) {
    return P.PL[v][k] + R(0.5) * s * (P.PD[v][k] + (R(1.0) - R(2.0 / 3.0) * s) * P.P6[v][k]);
}

// Step a5: characteristic tracing of the three wave families u-c, u, u+c
// (Colella & Woodward 1984), plus half a step of the buoyancy acceleration
// (rho'/rho) g (Sec. 1 perturbation form).
template <class R>
void trace(const oracle_problem *pb, Pencil<R> &P, R dt) {
    const R dtdx = dt / R(pb->dx);
    for (int i = -G + 2; i <= P.n + G - 3; ++i) {
        const int k = Pencil<R>::at(i);
        const R u = P.W[V_U][k], c = P.cs[k], c2 = P.c2[k];
        const R C = P.rho[k] * c;
        const R lm = u - c, l0 = u, lp = u + c;
        const R gp = (P.rd[k] / P.rho[k]) * P.gn[k];
        const R hg = R(0.5) * dt * gp;
        // right edge -> left state of face i+1/2
        {
            R st[NH];
            R sp = Max(lp, R(0.0)) * dtdx;
            for (int v = 0; v < NH; ++v) st[v] = fR(P, v, k, sp);
            R ref_r = st[V_R], ref_u = st[V_U], ref_p = st[V_P], ref_v = st[V_V], ref_w = st[V_W];
            if (l0 > R(0.0)) {
                R s0 = l0 * dtdx;
                R dr = ref_r - fR(P, V_R, k, s0);
                R dp = ref_p - fR(P, V_P, k, s0);
                st[V_R] = st[V_R] - (dr - dp / c2);
                st[V_V] = st[V_V] - (ref_v - fR(P, V_V, k, s0));
                st[V_W] = st[V_W] - (ref_w - fR(P, V_W, k, s0));
            }
            if (lm > R(0.0)) {
                R sm = lm * dtdx;
                R du = ref_u - fR(P, V_U, k, sm);
                R dp = ref_p - fR(P, V_P, k, sm);
                R A = R(0.5) * (dp - C * du);
                st[V_R] = st[V_R] - A / c2;
                st[V_U] = st[V_U] + A / C;
                st[V_P] = st[V_P] - A;
            }
            st[V_U] = st[V_U] + hg;
            for (int v = 0; v < NH; ++v) P.WL[v][k] = st[v];
        }
        // left edge -> right state of face i-1/2
        {
            R st[NH];
            R sm = Max(-lm, R(0.0)) * dtdx;
            for (int v = 0; v < NH; ++v) st[v] = fL(P, v, k, sm);
            R ref_r = st[V_R], ref_u = st[V_U], ref_p = st[V_P], ref_v = st[V_V], ref_w = st[V_W];
            if (l0 < R(0.0)) {
                R s0 = -l0 * dtdx;
                R dr = ref_r - fL(P, V_R, k, s0);
                R dp = ref_p - fL(P, V_P, k, s0);
                st[V_R] = st[V_R] - (dr - dp / c2);
                st[V_V] = st[V_V] - (ref_v - fL(P, V_V, k, s0));
                st[V_W] = st[V_W] - (ref_w - fL(P, V_W, k, s0));
            }
            if (lp < R(0.0)) {
                R s1 = -lp * dtdx;
                R du = ref_u - fL(P, V_U, k, s1);
                R dp = ref_p - fL(P, V_P, k, s1);
                R A = R(0.5) * (dp + C * du);
                st[V_R] = st[V_R] - A / c2;
                st[V_U] = st[V_U] - A / C;
                st[V_P] = st[V_P] - A;
            }
            st[V_U] = st[V_U] + hg;
            for (int v = 0; v < NH; ++v) P.WR[v][k - 1] = st[v];
        }
    }
}

// Steps a6-a7: approximate Riemann solver and fluxes at face j+1/2.
template <class R>
void riemann_fluxes(const oracle_problem *pb, Pencil<R> &P) {
    const R gam = R(pb->gamma), gm1 = R(pb->gamma - 1.0);
    const R kk = R((pb->gamma + 1.0) / (2.0 * pb->gamma));
    const R gg1 = R(pb->gamma / (pb->gamma - 1.0));
    for (int j = -G + 2; j <= P.n + G - 4; ++j) {
        const int k = Pencil<R>::at(j);
        const R r0 = P.rho0f[k], p0 = P.p0f[k];
        const R rdL = P.WL[V_R][k], uL = P.WL[V_U][k], pdL = P.WL[V_P][k];
        const R rdR = P.WR[V_R][k], uR = P.WR[V_U][k], pdR = P.WR[V_P][k];
        const R rL = r0 + rdL, pL = p0 + pdL;
        const R rR = r0 + rdR, pR = p0 + pdR;
        const R CL = Sqrt(gam * pL * rL), CR = Sqrt(gam * pR * rR);
        const R pfl = R(P_FLOOR) * Min(pL, pR);
        // acoustic guess, difference form
        R den = CL + CR;
        R pst = pdL + CL * (CR * (uL - uR) + (pdR - pdL)) / den;
        R ust = uL + (CR * (uR - uL) + (pdL - pdR)) / den;
        if (p0 + pst < pfl) pst = pfl - p0;
        // one two-shock impedance update
        const R WLi = CL * Sqrt(R(1.0) + kk * (pst - pdL) / pL);
        const R WRi = CR * Sqrt(R(1.0) + kk * (pst - pdR) / pR);
        den = WLi + WRi;
        pst = pdL + WLi * (WRi * (uL - uR) + (pdR - pdL)) / den;
        ust = uL + (WRi * (uR - uL) + (pdL - pdR)) / den;
        if (p0 + pst < pfl) pst = pfl - p0;
        const bool wall = (j == -1 && P.wall_lo) || (j == P.n - 1 && P.wall_hi);
        if (wall) ust = R(0.0);
        // upwind side of the contact
        const bool left = (ust >= R(0.0));
        const R rds = left ? rdL : rdR;
        const R pds = left ? pdL : pdR;
        const R rs = left ? rL : rR;
        const R pss = left ? pL : pR;
        R vst = left ? P.WL[V_V][k] : P.WR[V_V][k];
        R wst = left ? P.WL[V_W][k] : P.WR[V_W][k];
        const R dps = pst - pds;
        R rdst = rds + rs * dps / (gam * pss + R(0.5) * gm1 * dps);
        // The interface state is the two-shock solution at x/t = 0: where both
        // waves move to the same side (supersonic flow through the face), it
        // is the traced state on the upwind side itself.  Wave speeds from the
        // Lagrangian shock impedances: S_L = u_L - W_L/rho_L, S_R = u_R + W_R/rho_R.
        if (!wall) {
            const R SL = uL - WLi / rL, SR = uR + WRi / rR;
            if (SL >= R(0.0) || SR <= R(0.0)) {
                if (j >= -1 && j <= P.n - 1) ++P.c_sup;
            }
            if (SL >= R(0.0)) {
                ust = uL; pst = pdL; rdst = rdL;
                vst = P.WL[V_V][k]; wst = P.WL[V_W][k];
            } else if (SR <= R(0.0)) {
                ust = uR; pst = pdR; rdst = rdR;
                vst = P.WR[V_V][k]; wst = P.WR[V_W][k];
            }
        }
        // fluxes (Sec. 1 perturbation form)
        const R rst = r0 + rdst;
        const R Fr = rst * ust;
        const R h0 = gg1 * p0;
        P.us[k] = ust;
        P.ps[k] = pst;
        P.Fr[k] = Fr;
        P.Fn[k] = Fr * ust + pst;
        P.Ft1[k] = Fr * vst;
        P.Ft2[k] = Fr * wst;
        P.FE[k] = ust * (gg1 * pst + h0) + R(0.5) * (ust * ust + (vst * vst + wst * wst)) * Fr;
        if (P.divg && pb->shock_k > 0.0) {
            // 3-D dissipation inside shocks (Sec. 1): momentum and E' diffuse
            // across the face with nu = K max(0, -div(u) dx - eps c), div(u)
            // the full 3-D divergence averaged to the face, c the mean sound
            // speed of the two traced states.  Mass is not diffused.
            const R dface = R(0.5) * (P.dv[k] + P.dv[k + 1]);
            const R cface = R(0.5) * (CL / rL + CR / rR);
            const R nu = R(pb->shock_k) * Max(R(0.0), -(dface * R(pb->dx)) - R(SHOCK_EPS) * cface);
            if (val(nu) > 0.0) {
                if (j >= -1 && j <= P.n - 1) ++P.c_diss;
                P.Fn[k] = P.Fn[k] - nu * (P.mn[k + 1] - P.mn[k]);
                P.Ft1[k] = P.Ft1[k] - nu * (P.mt1[k + 1] - P.mt1[k]);
                P.Ft2[k] = P.Ft2[k] - nu * (P.mt2[k + 1] - P.mt2[k]);
                P.FE[k] = P.FE[k] - nu * (P.ed[k + 1] - P.ed[k]);
            }
        }
    }
}

// Step a8: conservative update with the gravity sources of the perturbation
// equations: momentum += dt rho' g (time-centred rho'), energy += dt g times
// the time-centred mass flux.
template <class R>
void hydro_update(const oracle_problem *pb, Pencil<R> &P, R dt) {
    const R dtdx = dt / R(pb->dx);
    for (int i = -1; i <= P.n; ++i) {
        const int k = Pencil<R>::at(i);
        const R g = P.gn[k];
        const R rdn = P.rd[k] - dtdx * (P.Fr[k] - P.Fr[k - 1]);
        P.rdn[k] = rdn;
        P.mnn[k] = P.mn[k] - dtdx * (P.Fn[k] - P.Fn[k - 1]) + dt * g * (R(0.5) * (P.rd[k] + rdn));
        P.mt1n[k] = P.mt1[k] - dtdx * (P.Ft1[k] - P.Ft1[k - 1]);
        P.mt2n[k] = P.mt2[k] - dtdx * (P.Ft2[k] - P.Ft2[k - 1]);
        P.edn[k] = P.ed[k] - dtdx * (P.FE[k] - P.FE[k - 1]) + dt * g * (R(0.5) * (P.Fr[k - 1] + P.Fr[k]));
    }
}

// Step a9a: PPB sub-cell profile along the pass,
// f(xi) = FV + m xi + a2 (xi^2 - 1/12), a2 = (m_{i+1} - m_{i-1})/4,
// scaled by theta in [0,1] when it would leave [0,1] on the cell.
template <class R>
void ppb_profiles(Pencil<R> &P) {
    for (int i = -G + 1; i <= P.n + G - 2; ++i) {
        const int k = Pencil<R>::at(i);
        const R F = P.fv[k], m = P.on[k];
        const R a2 = R(0.25) * (P.on[k + 1] - P.on[k - 1]);
        const R ep = R(0.5) * m + a2 * R(1.0 / 6.0);
        const R em = a2 * R(1.0 / 6.0) - R(0.5) * m;
        R gmax = Max(ep, em), gmin = Min(ep, em);
        if (a2 != R(0.0)) {
            const R xv = -m / (R(2.0) * a2);
            if (Abs(xv) < R(0.5)) {
                const R gv = m * xv + a2 * (xv * xv - R(1.0 / 12.0));
                gmax = Max(gmax, gv);
                gmin = Min(gmin, gv);
            }
        }
        R th = R(1.0);
        if (F + gmax > R(1.0)) th = Min(th, (R(1.0) - F) / gmax);
        if (F + gmin < R(0.0)) th = Min(th, F / (-gmin));
        if (i >= 0 && i < P.n && val(th) < 1.0) ++P.c_theta;
        P.meff[k] = th * m;
        P.aeff[k] = th * a2;
    }
}

// Step a9b: PPB transfers across face j+1/2: exact integrals of the donor's
// profile over the swept region of width |u*| dt/dx (content and first
// moment about the donor's centre), their donor-cell counterparts, and the
// donor-cell transfer of the transverse moments.  Signed: positive = to +x.
template <class R>
void ppb_fluxes(const oracle_problem *pb, Pencil<R> &P, R dt) {
    const R dtdx = dt / R(pb->dx);
    for (int j = -G + 2; j <= P.n + G - 4; ++j) {
        const int k = Pencil<R>::at(j);
        const R sig = P.us[k] * dtdx;
        const R phi = dtdx * P.Fr[k];
        const bool fromleft = (sig >= R(0.0));
        const int d = fromleft ? k : k + 1;
        const R s = fromleft ? sig : -sig;
        R M1 = R(0.5) - R(0.5) * s;
        const R M2 = R(0.25) - R(0.5) * s + s * s * R(1.0 / 3.0);
        R M3 = R(0.125) - R(0.375) * s + R(0.5) * s * s - R(0.25) * s * s * s;
        if (!fromleft) {
            M1 = -M1;
            M3 = -M3;
        }
        const R F = P.fv[d], me = P.meff[d], ae = P.aeff[d];
        const R phibar = F + me * M1 + ae * (M2 - R(1.0 / 12.0));
        const R psibar = F * M1 + me * M2 + ae * (M3 - M1 * R(1.0 / 12.0));
        P.GL[k] = phi * F;
        P.GH[k] = phi * phibar;
        P.KL[k] = phi * F * M1;
        P.KH[k] = phi * psibar;
        P.T1[k] = phi * P.ot1[d];
        P.T2[k] = phi * P.ot2[d];
        P.PHI[k] = phi;
        P.KM[k] = phi * M1;
    }
}

// Step a9c: Zalesak (1979) flux-corrected transport of rho*FV: the donor-cell
// transfer plus the limited antidiffusive part.  Reading: the bounds are the
// physical ones, 0 <= FV <= 1, not local extrema, so smooth extrema are never
// clipped (Sec. 1: the PPB representation is almost never constrained).
template <class R>
void ppb_fct(Pencil<R> &P) {
    for (int i = -1; i <= P.n; ++i) {
        const int k = Pencil<R>::at(i);
        const R rold = P.rho0c[k] + P.rd[k];
        const R rnew = P.rho0c[k] + P.rdn[k];
        const R cL = rold * P.fv[k] - (P.GL[k] - P.GL[k - 1]);
        const R FVL = cL / rnew;
        const R fmax = R(1.0);
        const R fmin = R(0.0);
        const R Ap = P.GH[k] - P.GL[k];
        const R Am = P.GH[k - 1] - P.GL[k - 1];
        const R Pp = Max(R(0.0), Am) - Min(R(0.0), Ap);
        const R Pm = Max(R(0.0), Ap) - Min(R(0.0), Am);
        const R Qp = (fmax - FVL) * rnew;
        const R Qm = (FVL - fmin) * rnew;
        P.Rp[k] = (Pp > R(0.0)) ? Clamp(Qp / Pp, R(0.0), R(1.0)) : R(0.0);
        P.Rm[k] = (Pm > R(0.0)) ? Clamp(Qm / Pm, R(0.0), R(1.0)) : R(0.0);
    }
    for (int j = -1; j <= P.n - 1; ++j) {
        const int k = Pencil<R>::at(j);
        const R A = P.GH[k] - P.GL[k];
        const R C = (A >= R(0.0)) ? Min(P.Rp[k + 1], P.Rm[k]) : Min(P.Rp[k], P.Rm[k + 1]);
        if (val(A) != 0.0 && val(C) < 1.0) ++P.c_fct;
        P.Gf[k] = P.GL[k] + C * A;
        P.Kf[k] = P.KL[k] + C * (P.KH[k] - P.KL[k]);
    }
}

// Step a9d: new FV and moments.  Content staying in the cell moves by the
// mean of its two face displacements, content crossing a face by that
// face's displacement; first moments are re-taken about the receiving
// cell's centre.  The same rules move the mass (uniform density in each
// piece), and the FV moment is the fluid-2 content moment minus FV times
// the mass moment (so a uniform FV keeps a zero moment in compressing
// flow).  Then each |m_d| <= 6 FV (1-FV): the largest first moment any
// sub-cell profile with values in [0,1] can have (a step inside the cell).
template <class R>
void ppb_update(const oracle_problem *pb, Pencil<R> &P, R dt) {
    const R dtdx = dt / R(pb->dx);
    for (int i = 0; i < P.n; ++i) {
        const int k = Pencil<R>::at(i);
        const R rold = P.rho0c[k] + P.rd[k];
        const R rnew = P.rho0c[k] + P.rdn[k];
        const R sm = P.us[k - 1] * dtdx, sp = P.us[k] * dtdx;
        const R cold = rold * P.fv[k];
        R c_out = R(0.0), z_out = R(0.0), z_in = R(0.0);
        R m_out = R(0.0), zr_out = R(0.0), zr_in = R(0.0);
        if (sp >= R(0.0)) {
            c_out = c_out + P.Gf[k];
            z_out = z_out + P.Kf[k];
            m_out = m_out + P.PHI[k];
            zr_out = zr_out + P.KM[k];
        } else {
            const R sh = sp + R(1.0);
            z_in = z_in + (-P.Kf[k] - P.Gf[k] * sh);
            zr_in = zr_in + (-P.KM[k] - P.PHI[k] * sh);
        }
        if (sm >= R(0.0)) {
            const R sh = sm - R(1.0);
            z_in = z_in + (P.Kf[k - 1] + P.Gf[k - 1] * sh);
            zr_in = zr_in + (P.KM[k - 1] + P.PHI[k - 1] * sh);
        } else {
            c_out = c_out - P.Gf[k - 1];
            z_out = z_out - P.Kf[k - 1];
            m_out = m_out - P.PHI[k - 1];
            zr_out = zr_out - P.KM[k - 1];
        }
        // difference form: X_new = X + (X dPhi - dQ) / rho_new, with dPhi the
        // net mass outflow and dQ the net outflow of rho*X, so that a cell
        // with no net transfer keeps its values bit for bit
        const R sbar = R(0.5) * (sm + sp);
        const R dZc = (cold - c_out) * sbar + z_in - z_out;
        const R Zr = (rold - m_out) * sbar + zr_in - zr_out;
        const R dPhi = P.PHI[k] - P.PHI[k - 1];
        const R dG = P.Gf[k] - P.Gf[k - 1];
        R fvn = Clamp(P.fv[k] + (P.fv[k] * dPhi - dG) / rnew, R(0.0), R(1.0));
        R onn = P.on[k] + (P.on[k] * dPhi + R(12.0) * (dZc - fvn * Zr)) / rnew;
        R o1 = P.ot1[k] + (P.ot1[k] * dPhi - (P.T1[k] - P.T1[k - 1])) / rnew;
        R o2 = P.ot2[k] + (P.ot2[k] * dPhi - (P.T2[k] - P.T2[k - 1])) / rnew;
        const R bnd = R(6.0) * fvn * (R(1.0) - fvn);
        if (Abs(onn) > bnd || Abs(o1) > bnd || Abs(o2) > bnd) {
            onn = Clamp(onn, -bnd, bnd);
            o1 = Clamp(o1, -bnd, bnd);
            o2 = Clamp(o2, -bnd, bnd);
            ++P.c_clamp;
        }
        P.fvn[k] = fvn;
        P.onn[k] = onn;
        P.ot1n[k] = o1;
        P.ot2n[k] = o2;
    }
}

// --------------------------------------------------------------------------
// Ten-value PPB (Sec. 1 and Sec. 4: the production form carries the average
// and 9 moments of FV per cell, so that each 1-D pass has a purely local
// parabola and constraints are almost never needed).  On the unit cell
// (xi, eta, zeta in [-1/2, 1/2]) the sub-cell profile is
//   f = FV + sum_d m_d P1(xi_d) + sum_d q_d P2(xi_d) + sum_{d<e} c_de xi_d xi_e,
// P1 = xi, P2 = xi^2 - 1/12, with m_d = 12 int xi_d f, q_d = 180 int P2(xi_d) f,
// c_de = 144 int xi_d xi_e f (the L2 projection on these polynomials).  In a
// pass along xi (transverse eta, zeta) the profile integrated across is the
// local parabola FV + m_n xi + q_n P2(xi); the eta-moment density along xi is
// (m_1 + c_n1 xi)/12, the zeta one (m_2 + c_n2 xi)/12, and the P2(eta),
// P2(zeta) and eta*zeta densities are the constants q_1/180, q_2/180,
// c_12/144.  Pieces of content and of mass are moved rigidly as in the
// four-value form, and every moment of the new cell is re-taken about its
// centre, relative to the mass distribution to first order.
// --------------------------------------------------------------------------

// Step a9a': the local parabola along the pass, bound-limited (theta) as in
// the four-value form, with the cell's own second moment as curvature.
template <class R>
void ppb10_profiles(Pencil<R> &P) {
    for (int i = -G + 1; i <= P.n + G - 2; ++i) {
        const int k = Pencil<R>::at(i);
        const R F = P.fv[k], m = P.on[k], a2 = P.qn[k];
        const R ep = R(0.5) * m + a2 * R(1.0 / 6.0);
        const R em = a2 * R(1.0 / 6.0) - R(0.5) * m;
        R gmax = Max(ep, em), gmin = Min(ep, em);
        if (a2 != R(0.0)) {
            const R xv = -m / (R(2.0) * a2);
            if (Abs(xv) < R(0.5)) {
                const R gv = m * xv + a2 * (xv * xv - R(1.0 / 12.0));
                gmax = Max(gmax, gv);
                gmin = Min(gmin, gv);
            }
        }
        R th = R(1.0);
        if (F + gmax > R(1.0)) th = Min(th, (R(1.0) - F) / gmax);
        if (F + gmin < R(0.0)) th = Min(th, F / (-gmin));
        if (i >= 0 && i < P.n && val(th) < 1.0) ++P.c_theta;
        P.meff[k] = th * m;
        P.aeff[k] = th * a2;
    }
}

// Step a9b': transfers across face j+1/2 (signed, positive = to +x): the
// four-value ones (content, first moments of content and mass about the
// donor's centre) plus the second moments of content and mass about that
// centre, the transverse first moments with their xi-moments, and the
// transverse second and mixed moments (constant across the swept slab).
template <class R>
void ppb10_fluxes(const oracle_problem *pb, Pencil<R> &P, R dt) {
    const R dtdx = dt / R(pb->dx);
    for (int j = -G + 2; j <= P.n + G - 4; ++j) {
        const int k = Pencil<R>::at(j);
        const R sig = P.us[k] * dtdx;
        const R phi = dtdx * P.Fr[k];
        const bool fromleft = (sig >= R(0.0));
        const int d = fromleft ? k : k + 1;
        const R s = fromleft ? sig : -sig;
        // means of xi^p over the swept slab [1/2 - s, 1/2] of a left donor
        // (odd powers change sign for the slab [-1/2, -1/2 + s] of a right one)
        R M1 = R(0.5) - R(0.5) * s;
        const R M2 = R(0.25) - R(0.5) * s + s * s * R(1.0 / 3.0);
        R M3 = R(0.125) - R(0.375) * s + R(0.5) * s * s - R(0.25) * s * s * s;
        const R M4 = R(0.0625) - R(0.25) * s + R(0.5) * s * s - R(0.5) * s * s * s + R(0.2) * s * s * s * s;
        if (!fromleft) {
            M1 = -M1;
            M3 = -M3;
        }
        const R F = P.fv[d], me = P.meff[d], ae = P.aeff[d];
        const R phibar = F + me * M1 + ae * (M2 - R(1.0 / 12.0));
        const R psibar = F * M1 + me * M2 + ae * (M3 - M1 * R(1.0 / 12.0));
        const R chibar = F * M2 + me * M3 + ae * (M4 - M2 * R(1.0 / 12.0));
        P.GL[k] = phi * F;
        P.GH[k] = phi * phibar;
        P.KL[k] = phi * F * M1;
        P.KH[k] = phi * psibar;
        P.K2L[k] = phi * F * M2;
        P.K2H[k] = phi * chibar;
        P.PHI[k] = phi;
        P.KM[k] = phi * M1;
        P.KM2[k] = phi * M2;
        P.T1[k] = phi * (P.ot1[d] + P.cn1[d] * M1);
        P.T2[k] = phi * (P.ot2[d] + P.cn2[d] * M1);
        P.U1[k] = phi * (P.ot1[d] * M1 + P.cn1[d] * M2);
        P.U2[k] = phi * (P.ot2[d] * M1 + P.cn2[d] * M2);
        P.Q1[k] = phi * P.q1[d];
        P.Q2[k] = phi * P.q2[d];
        P.C12[k] = phi * P.c12[d];
    }
}

// Step a9c': the same FCT; the limited second moment of content follows the
// content with the same factor.
template <class R>
void ppb10_fct(Pencil<R> &P) {
    ppb_fct(P);
    for (int j = -1; j <= P.n - 1; ++j) {
        const int k = Pencil<R>::at(j);
        const R A = P.GH[k] - P.GL[k];
        const R C = (A >= R(0.0)) ? Min(P.Rp[k + 1], P.Rm[k]) : Min(P.Rp[k], P.Rm[k + 1]);
        P.K2f[k] = P.K2L[k] + C * (P.K2H[k] - P.K2L[k]);
    }
}

// Step a9d': new FV and its nine moments.  Raw moments (about the new cell's
// centre) of the staying piece (shifted by the mean face displacement) and of
// the incoming pieces (shifted by their face's displacement); the old cell's
// mass is uniform.  With rho = rho_bar (1 + r1 xi + ...) the content moments
// relative to the mass give, to first order in the mass moments,
//   rho m_n / 12   = C1 - FV R1,
//   rho q_n / 180  = C2' - FV R2' - m_n R1 / 15      (C2', R2': P2-moments),
//   rho c_n1 / 12  = Y1 - m_1 R1                      (Y1 = 12 int xi eta c),
// and the transverse moments are conserved contents (rho m_1, rho q_1, ...).
// All in difference form (X_new = X + (X dPhi - dQ)/rho_new), so a cell with
// no transfer keeps its values bit for bit.  Then realisability bounds for a
// profile in [0,1] with mean FV: |m| <= 6 FV(1-FV), -15 FV(1-FV)(1+FV) <= q
// <= 15 FV(1-FV)(2-FV) (all content at the centre / at the two ends), and
// |c| <= 36 FV(1-FV) (all content in one corner).
template <class R>
void ppb10_update(const oracle_problem *pb, Pencil<R> &P, R dt) {
    const R dtdx = dt / R(pb->dx);
    for (int i = 0; i < P.n; ++i) {
        const int k = Pencil<R>::at(i);
        const R rold = P.rho0c[k] + P.rd[k];
        const R rnew = P.rho0c[k] + P.rdn[k];
        const R sm = P.us[k - 1] * dtdx, sp = P.us[k] * dtdx;
        const R cold = rold * P.fv[k];
        // outgoing amounts and moments about this cell's centre; incoming
        // moments about it after the move
        R c_out = R(0.0), z_out = R(0.0), z2_out = R(0.0), z_in = R(0.0), z2_in = R(0.0);
        R m_out = R(0.0), zr_out = R(0.0), zr2_out = R(0.0), zr_in = R(0.0), zr2_in = R(0.0);
        R t1_out = R(0.0), u1_out = R(0.0), u1_in = R(0.0);
        R t2_out = R(0.0), u2_out = R(0.0), u2_in = R(0.0);
        if (sp >= R(0.0)) {
            c_out = c_out + P.Gf[k];
            z_out = z_out + P.Kf[k];
            z2_out = z2_out + P.K2f[k];
            m_out = m_out + P.PHI[k];
            zr_out = zr_out + P.KM[k];
            zr2_out = zr2_out + P.KM2[k];
            t1_out = t1_out + P.T1[k];
            u1_out = u1_out + P.U1[k];
            t2_out = t2_out + P.T2[k];
            u2_out = u2_out + P.U2[k];
        } else {
            const R h = sp + R(1.0);
            z_in = z_in - (P.Kf[k] + P.Gf[k] * h);
            z2_in = z2_in - (P.K2f[k] + R(2.0) * h * P.Kf[k] + h * h * P.Gf[k]);
            zr_in = zr_in - (P.KM[k] + P.PHI[k] * h);
            zr2_in = zr2_in - (P.KM2[k] + R(2.0) * h * P.KM[k] + h * h * P.PHI[k]);
            u1_in = u1_in - (P.U1[k] + P.T1[k] * h);
            u2_in = u2_in - (P.U2[k] + P.T2[k] * h);
        }
        if (sm >= R(0.0)) {
            const R h = sm - R(1.0);
            z_in = z_in + (P.Kf[k - 1] + P.Gf[k - 1] * h);
            z2_in = z2_in + (P.K2f[k - 1] + R(2.0) * h * P.Kf[k - 1] + h * h * P.Gf[k - 1]);
            zr_in = zr_in + (P.KM[k - 1] + P.PHI[k - 1] * h);
            zr2_in = zr2_in + (P.KM2[k - 1] + R(2.0) * h * P.KM[k - 1] + h * h * P.PHI[k - 1]);
            u1_in = u1_in + (P.U1[k - 1] + P.T1[k - 1] * h);
            u2_in = u2_in + (P.U2[k - 1] + P.T2[k - 1] * h);
        } else {
            c_out = c_out - P.Gf[k - 1];
            z_out = z_out - P.Kf[k - 1];
            z2_out = z2_out - P.K2f[k - 1];
            m_out = m_out - P.PHI[k - 1];
            zr_out = zr_out - P.KM[k - 1];
            zr2_out = zr2_out - P.KM2[k - 1];
            t1_out = t1_out - P.T1[k - 1];
            u1_out = u1_out - P.U1[k - 1];
            t2_out = t2_out - P.T2[k - 1];
            u2_out = u2_out - P.U2[k - 1];
        }
        const R sbar = R(0.5) * (sm + sp);
        const R dPhi = P.PHI[k] - P.PHI[k - 1];
        const R dG = P.Gf[k] - P.Gf[k - 1];
        // staying content: amount S0, first moment S1 (about the old centre)
        const R S0 = cold - c_out;
        const R S1 = rold * P.on[k] * R(1.0 / 12.0) - z_out;
        const R dZc = S0 * sbar + z_in - z_out;                                   // C1 change
        const R dZc2 = R(2.0) * sbar * S1 + sbar * sbar * S0 + z2_in - z2_out;   // C2 change
        const R Zr = (rold - m_out) * sbar + zr_in - zr_out;                      // R1 (old: 0)
        const R Zr2 = R(-2.0) * sbar * zr_out + sbar * sbar * (rold - m_out) + zr2_in - zr2_out
                      + (rold - rnew) * R(1.0 / 12.0);                            // R2' = R2 - rnew/12
        const R fvn = Clamp(P.fv[k] + (P.fv[k] * dPhi - dG) / rnew, R(0.0), R(1.0));
        R onn = P.on[k] + (P.on[k] * dPhi + R(12.0) * (dZc - fvn * Zr)) / rnew;
        // P2-moment change of content: C2 change minus (content change)/12
        const R dC2p = dZc2 + dG * R(1.0 / 12.0);
        R qnn = P.qn[k] + (P.qn[k] * dPhi + R(180.0) * (dC2p - fvn * Zr2) - R(12.0) * onn * Zr) / rnew;
        R o1 = P.ot1[k] + (P.ot1[k] * dPhi - (P.T1[k] - P.T1[k - 1])) / rnew;
        R o2 = P.ot2[k] + (P.ot2[k] * dPhi - (P.T2[k] - P.T2[k - 1])) / rnew;
        const R dY1 = (rold * P.ot1[k] - t1_out) * sbar + u1_in - u1_out;
        const R dY2 = (rold * P.ot2[k] - t2_out) * sbar + u2_in - u2_out;
        R cn1 = P.cn1[k] + (P.cn1[k] * dPhi + R(12.0) * (dY1 - o1 * Zr)) / rnew;
        R cn2 = P.cn2[k] + (P.cn2[k] * dPhi + R(12.0) * (dY2 - o2 * Zr)) / rnew;
        R q1 = P.q1[k] + (P.q1[k] * dPhi - (P.Q1[k] - P.Q1[k - 1])) / rnew;
        R q2 = P.q2[k] + (P.q2[k] * dPhi - (P.Q2[k] - P.Q2[k - 1])) / rnew;
        R c12 = P.c12[k] + (P.c12[k] * dPhi - (P.C12[k] - P.C12[k - 1])) / rnew;
        const R g = fvn * (R(1.0) - fvn);
        const R bm = R(6.0) * g, bc = R(36.0) * g;
        const R qlo = R(-15.0) * g * (R(1.0) + fvn), qhi = R(15.0) * g * (R(2.0) - fvn);
        bool clamped = false;
        auto cl = [&](R &x, R lo, R hi) {
            if (x < lo || x > hi) {
                x = Clamp(x, lo, hi);
                clamped = true;
            }
        };
        cl(onn, -bm, bm);
        cl(o1, -bm, bm);
        cl(o2, -bm, bm);
        cl(qnn, qlo, qhi);
        cl(q1, qlo, qhi);
        cl(q2, qlo, qhi);
        cl(cn1, -bc, bc);
        cl(cn2, -bc, bc);
        cl(c12, -bc, bc);
        if (clamped) ++P.c_clamp;
        P.fvn[k] = fvn;
        P.onn[k] = onn;
        P.ot1n[k] = o1;
        P.ot2n[k] = o2;
        P.qnn[k] = qnn;
        P.q1n[k] = q1;
        P.q2n[k] = q2;
        P.cn1n[k] = cn1;
        P.cn2n[k] = cn2;
        P.c12n[k] = c12;
    }
}

// Sources, after the pass update of each cell of the run.  flags & 1:
// heating and damping (after the Z pass of X Y Z and the X pass of Z Y X):
// E' += dt*heat(s); velocities scaled by max(0, 1 - dt*damp(s)) with the
// kinetic energy removed from E'.  flags & 2: the rotation ramp of Sec. 3, a
// solid-body flow added gradually: once per double step (after the X pass of
// Z Y X) every fluid cell gains the velocity domega * (-y, x, 0) about the z
// axis through the origin, E' gaining the kinetic energy this adds.
template <class R>
void sources(const oracle_problem *pb, Pencil<R> &P, R dt, int flags) {
    const bool heatdamp = (flags & 1) && (pb->heat || pb->damp);
    const bool rotate = (flags & 2) && pb->domega != 0.0;
    if (!heatdamp && !rotate) return;
    const int a = P.axis, t1 = (a + 1) % 3, t2 = (a + 2) % 3;
    for (int i = 0; i < P.n; ++i) {
        const int k = Pencil<R>::at(i);
        R xyz[3];
        cell_position(pb, P.axis, P.i0 + i, P.ja, P.jb, xyz);
        if (heatdamp) {
            const R s = source_coord(pb, xyz);
            if (pb->heat) P.edn[k] = P.edn[k] + dt * lerp_tab(pb, pb->heat, s);
            if (pb->damp) {
                const R kd = lerp_tab(pb, pb->damp, s);
                const R f = Max(R(0.0), R(1.0) - dt * kd);
                const R rho = P.rho0c[k] + P.rdn[k];
                const R ke = R(0.5) * (P.mnn[k] * P.mnn[k] + (P.mt1n[k] * P.mt1n[k] + P.mt2n[k] * P.mt2n[k])) / rho;
                P.mnn[k] = P.mnn[k] * f;
                P.mt1n[k] = P.mt1n[k] * f;
                P.mt2n[k] = P.mt2n[k] * f;
                P.edn[k] = P.edn[k] - (R(1.0) - f * f) * ke;
            }
        }
        if (rotate) {
            const R rho = P.rho0c[k] + P.rdn[k];
            const R w = R(pb->domega);
            R du[3];
            du[0] = -(w * xyz[1]);
            du[1] = w * xyz[0];
            du[2] = R(0.0);
            const R dn = du[a], d1 = du[t1], d2 = du[t2];
            const R dE = (P.mnn[k] * dn + (P.mt1n[k] * d1 + P.mt2n[k] * d2)) +
                         R(0.5) * rho * (dn * dn + (d1 * d1 + d2 * d2));
            P.mnn[k] = P.mnn[k] + rho * dn;
            P.mt1n[k] = P.mt1n[k] + rho * d1;
            P.mt2n[k] = P.mt2n[k] + rho * d2;
            P.edn[k] = P.edn[k] + dE;
        }
    }
}

// Whole pass on one gathered pencil.
template <class R>
void pass(const oracle_problem *pb, Pencil<R> &P, R dt, int with_sources) {
    primitives(pb, P);
    interface_values(P);
    smoothness(P);
    flattening(P);
    parabolas(P);
    trace(pb, P, dt);
    riemann_fluxes(pb, P);
    hydro_update(pb, P, dt);
    if (P.ten) {
        ppb10_profiles(P);
        ppb10_fluxes(pb, P, dt);
        ppb10_fct(P);
        ppb10_update(pb, P, dt);
    } else {
        ppb_profiles(P);
        ppb_fluxes(pb, P, dt);
        ppb_fct(P);
        ppb_update(pb, P, dt);
    }
    if (with_sources) sources(pb, P, dt, with_sources);
}

// Step a1 inverse: back to full variables in the unrotated frame.
template <class R>
void scatter(const oracle_problem *pb, const Pencil<R> &P, double *q[9]) {
    const int a = P.axis, t1 = (a + 1) % 3, t2 = (a + 2) % 3;
    const R gm1 = R(pb->gamma - 1.0);
    for (int i = 0; i < P.n; ++i) {
        const int k = Pencil<R>::at(i);
        size_t c = cell_index(pb, a, P.i0 + i, P.ja, P.jb);
        q[0][c] = val(P.rho0c[k] + P.rdn[k]);
        q[1 + a][c] = val(P.mnn[k]);
        q[1 + t1][c] = val(P.mt1n[k]);
        q[1 + t2][c] = val(P.mt2n[k]);
        q[4][c] = val(P.p0c[k] / gm1 + P.edn[k]);
        q[5][c] = val(P.fvn[k]);
        q[6 + a][c] = val(P.onn[k]);
        q[6 + t1][c] = val(P.ot1n[k]);
        q[6 + t2][c] = val(P.ot2n[k]);
        if (P.ten) {
            q[9 + a][c] = val(P.qnn[k]);
            q[9 + t1][c] = val(P.q1n[k]);
            q[9 + t2][c] = val(P.q2n[k]);
            q[12 + a][c] = val(P.c12n[k]);
            q[12 + t2][c] = val(P.cn1n[k]);
            q[12 + t1][c] = val(P.cn2n[k]);
        }
    }
}

template <class R>
void flush_counters(const Pencil<R> &P) {
    g_cnt[0] += P.c_nonsmooth;
    g_cnt[1] += P.c_flat;
    g_cnt[2] += P.c_theta;
    g_cnt[3] += P.c_fct;
    g_cnt[4] += P.c_clamp;
    g_cnt[5] += P.n;
    g_cnt[6] += P.c_diss;
    g_cnt[7] += P.c_sup;
}

// Velocity divergence of every cell for the 3-D shock dissipation: central
// differences of u_d = (rho u_d)/rho along each axis, summed in x, y, z order;
// ghost neighbours by the boundary conditions (periodic wrap; at a wall the
// mirror cell with its normal velocity reversed).
void divergence(const oracle_problem *pb, double *const q[], std::vector<double> &D) {
    const int n[3] = {pb->nx, pb->ny, pb->nz};
    const long long ncell = (long long)n[0] * n[1] * n[2];
    D.assign((size_t)ncell, 0.0);
    const double h = 0.5 / pb->dx;
#pragma omp parallel for num_threads(g_threads > 0 ? g_threads : omp_get_max_threads())
    for (long long c = 0; c < ncell; ++c) {
        const int ijk[3] = {(int)(c % n[0]), (int)((c / n[0]) % n[1]), (int)(c / ((long long)n[0] * n[1]))};
        double diff[3];
        for (int d = 0; d < 3; ++d) {
            double u[2];
            for (int s = 0; s < 2; ++s) {
                int idx[3] = {ijk[0], ijk[1], ijk[2]};
                bool flip;
                idx[d] = map_cell(ijk[d] + (s ? 1 : -1), n[d], pb->bc[2 * d], pb->bc[2 * d + 1], &flip);
                const long long cc = ((long long)idx[2] * n[1] + idx[1]) * n[0] + idx[0];
                const double v = q[1 + d][cc] / q[0][cc];
                u[s] = flip ? -v : v;
            }
            diff[d] = u[1] - u[0];
        }
        D[(size_t)c] = ((diff[0] + diff[1]) + diff[2]) * h;
    }
}

template <class R>
void sweep_all(const oracle_problem *pb, double *q[9], int axis, double dt, int with_sources,
               bool parallel) {
    const int n = extent(pb, axis);
    const int na = extent(pb, (axis + 1) % 3), nb = extent(pb, (axis + 2) % 3);
    const long long npen = (long long)na * nb;
    std::vector<double> D;
    if (pb->shock_k > 0.0) divergence(pb, q, D);
    auto body = [&](Pencil<R> &P, long long p) {
        P.divg = D.empty() ? nullptr : D.data();
        P.ja = (int)(p % na);
        P.jb = (int)(p / na);
        P.c_nonsmooth = P.c_flat = P.c_theta = P.c_fct = P.c_clamp = P.c_diss = P.c_sup = 0;
        if (!pencil_run(pb, axis, P.ja, P.jb, &P.i0, &P.n)) return;
        P.confined = pb->confine_r > 0.0;
        P.ten = pb->nmom == 9;
        gather(pb, P, q);
        pass(pb, P, R(dt), with_sources);
        scatter(pb, P, q);
        flush_counters(P);
    };
    if (parallel) {
#pragma omp parallel num_threads(g_threads > 0 ? g_threads : omp_get_max_threads())
        {
            Pencil<R> P;
            P.alloc(n);
            P.axis = axis;
#pragma omp for schedule(static)
            for (long long p = 0; p < npen; ++p) body(P, p);
        }
    } else {
        Pencil<R> P;
        P.alloc(n);
        P.axis = axis;
        for (long long p = 0; p < npen; ++p) body(P, p);
    }
}

bool has_sources(const oracle_problem *pb) { return pb->heat || pb->damp; }

// Source flags a pass actually applies: bit 0 heating/damping (when tables
// exist), bit 1 the rotation increment (when domega != 0).
int source_flags(const oracle_problem *pb, int requested) {
    return ((requested & 1) && has_sources(pb) ? 1 : 0) | ((requested & 2) && pb->domega != 0.0 ? 2 : 0);
}

}  // namespace

extern "C" {

void oracle_sweep(const oracle_problem *pb, double *q[9], int axis, double dt, int with_sources) {
    sweep_all<double>(pb, q, axis, dt, source_flags(pb, with_sources), true);
}

void oracle_double_step(const oracle_problem *pb, double *q[9], double dt) {
    oracle_sweep(pb, q, 0, dt, 0);
    oracle_sweep(pb, q, 1, dt, 0);
    oracle_sweep(pb, q, 2, dt, 1);
    oracle_sweep(pb, q, 2, dt, 0);
    oracle_sweep(pb, q, 1, dt, 0);
    oracle_sweep(pb, q, 0, dt, 1 | 2);
}

double oracle_cfl_dt(const oracle_problem *pb, double *const q[9], double cfl) {
    const double gam = pb->gamma, gm1 = pb->gamma - 1.0;
    double smax = 0.0;
    const long long ncell = (long long)pb->nx * pb->ny * pb->nz;
#pragma omp parallel for reduction(max : smax) num_threads(g_threads > 0 ? g_threads : omp_get_max_threads())
    for (long long c = 0; c < ncell; ++c) {
        int i = (int)(c % pb->nx), j = (int)((c / pb->nx) % pb->ny), k = (int)(c / ((long long)pb->nx * pb->ny));
        double xyz[3];
        cell_position<double>(pb, 0, i, j, k, xyz);
        if (!fluid_cell(pb, xyz)) continue;   // solid cells of a confining sphere
        BasePoint<double> b = base_at<double>(pb, xyz);
        double rho = q[0][c];
        double u = q[1][c] / rho, v = q[2][c] / rho, w = q[3][c] / rho;
        double ke = 0.5 * (q[1][c] * u + q[2][c] * v + q[3][c] * w);
        double ed = q[4][c] - b.p0 / gm1;
        double p = b.p0 + gm1 * (ed - ke);
        double cs = std::sqrt(gam * p / rho);
        double s = std::max(std::max(std::fabs(u), std::fabs(v)), std::fabs(w)) + cs;
        smax = std::max(smax, s);
    }
    return cfl * pb->dx / smax;
}

void oracle_sweep_pencil(const oracle_problem *pb, int axis, int ja, int jb, double *const in[9],
                         double *out[9], double dt, int with_sources) {
    // The same pass on one pencil given as separate arrays (positions are
    // those of pencil (ja, jb) of the grid); solid cells are copied through.
    const int N = extent(pb, axis);
    const int nv = pb->nmom == 9 ? 15 : 9;
    for (int v = 0; v < nv; ++v)
        for (int i = 0; i < N; ++i) out[v][i] = in[v][i];
    Pencil<double> P;
    P.alloc(N);
    P.axis = axis;
    P.ja = ja;
    P.jb = jb;
    P.ten = pb->nmom == 9;
    if (!pencil_run(pb, axis, ja, jb, &P.i0, &P.n)) return;
    P.confined = pb->confine_r > 0.0;
    const int n = P.n;
    const int bl = P.confined ? 1 : pb->bc[2 * axis], bh = P.confined ? 1 : pb->bc[2 * axis + 1];
    P.wall_lo = (bl == 1);
    P.wall_hi = (bh == 1);
    const double gm1 = pb->gamma - 1.0;
    const int t1 = (axis + 1) % 3, t2 = (axis + 2) % 3;
    for (int i = -G; i < n + G; ++i) {
        bool flip;
        const int m = P.i0 + map_cell(i, n, bl, bh, &flip);
        double xyz[3];
        cell_position<double>(pb, axis, m, ja, jb, xyz);
        BasePoint<double> b = base_at<double>(pb, xyz);
        const int k = Pencil<double>::at(i);
        P.rho0c[k] = b.rho0;
        P.p0c[k] = b.p0;
        P.gn[k] = flip ? -b.g[axis] : b.g[axis];
        P.rd[k] = in[0][m] - b.rho0;
        P.mn[k] = flip ? -in[1 + axis][m] : in[1 + axis][m];
        P.mt1[k] = in[1 + t1][m];
        P.mt2[k] = in[1 + t2][m];
        P.ed[k] = in[4][m] - b.p0 / gm1;
        P.fv[k] = in[5][m];
        P.on[k] = flip ? -in[6 + axis][m] : in[6 + axis][m];
        P.ot1[k] = in[6 + t1][m];
        P.ot2[k] = in[6 + t2][m];
        if (P.ten) {
            P.qn[k] = in[9 + axis][m];
            P.q1[k] = in[9 + t1][m];
            P.q2[k] = in[9 + t2][m];
            P.c12[k] = in[12 + axis][m];
            P.cn1[k] = flip ? -in[12 + t2][m] : in[12 + t2][m];
            P.cn2[k] = flip ? -in[12 + t1][m] : in[12 + t1][m];
        }
    }
    const double lo = origin(pb, axis);
    for (int j = -G; j < n + G; ++j) {
        int Pf = map_face(j, n, bl, bh);
        double xyz[3];
        cell_position<double>(pb, axis, 0, ja, jb, xyz);
        xyz[axis] = lo + (double)(P.i0 + Pf) * pb->dx;
        BasePoint<double> b = base_at<double>(pb, xyz);
        P.rho0f[Pencil<double>::at(j)] = b.rho0;
        P.p0f[Pencil<double>::at(j)] = b.p0;
    }
    pass(pb, P, dt, source_flags(pb, with_sources));
    for (int i = 0; i < n; ++i) {
        const int k = Pencil<double>::at(i);
        const int m = P.i0 + i;
        out[0][m] = P.rho0c[k] + P.rdn[k];
        out[1 + axis][m] = P.mnn[k];
        out[1 + t1][m] = P.mt1n[k];
        out[1 + t2][m] = P.mt2n[k];
        out[4][m] = P.p0c[k] / gm1 + P.edn[k];
        out[5][m] = P.fvn[k];
        out[6 + axis][m] = P.onn[k];
        out[6 + t1][m] = P.ot1n[k];
        out[6 + t2][m] = P.ot2n[k];
        if (P.ten) {
            out[9 + axis][m] = P.qnn[k];
            out[9 + t1][m] = P.q1n[k];
            out[9 + t2][m] = P.q2n[k];
            out[12 + axis][m] = P.c12n[k];
            out[12 + t2][m] = P.cn1n[k];
            out[12 + t1][m] = P.cn2n[k];
        }
    }
    flush_counters(P);
}

void oracle_sweep_z_slab(const oracle_problem *pb, double *q[9], int k0, int nzl, double dt, int with_sources) {
    const int axis = 2, n = pb->nz;
    const int bl = pb->bc[4], bh = pb->bc[5];
    const double gm1 = pb->gamma - 1.0;
    const long long plane = (long long)pb->nx * pb->ny;
    const int src = source_flags(pb, with_sources);
#pragma omp parallel num_threads(g_threads > 0 ? g_threads : omp_get_max_threads())
    {
        Pencil<double> P;
        P.alloc(nzl);
        P.axis = axis;
#pragma omp for schedule(static)
        for (long long pidx = 0; pidx < plane; ++pidx) {
            const int ja = (int)(pidx % pb->nx), jb = (int)(pidx / pb->nx);  // (x, y) of the z pencil
            P.ja = ja;
            P.jb = jb;
            P.c_nonsmooth = P.c_flat = P.c_theta = P.c_fct = P.c_clamp = P.c_sup = 0;
            P.wall_lo = (k0 == 0 && bl == 1);
            P.wall_hi = (k0 + nzl == n && bh == 1);
            for (int i = -G; i < nzl + G; ++i) {
                const int kg = k0 + i;                 // global plane
                bool flip;
                const int m = map_cell(kg, n, bl, bh, &flip);
                double xyz[3];
                cell_position<double>(pb, axis, m, ja, jb, xyz);
                BasePoint<double> b = base_at<double>(pb, xyz);
                const int k = Pencil<double>::at(i);
                const long long c = (long long)(i + G) * plane + pidx;
                P.rho0c[k] = b.rho0;
                P.p0c[k] = b.p0;
                P.gn[k] = flip ? -b.g[axis] : b.g[axis];
                P.rd[k] = q[0][c] - b.rho0;
                P.mn[k] = flip ? -q[3][c] : q[3][c];
                P.mt1[k] = q[1][c];
                P.mt2[k] = q[2][c];
                P.ed[k] = q[4][c] - b.p0 / gm1;
                P.fv[k] = q[5][c];
                P.on[k] = flip ? -q[8][c] : q[8][c];
                P.ot1[k] = q[6][c];
                P.ot2[k] = q[7][c];
            }
            const double lo = origin(pb, axis);
            for (int j = -G; j < nzl + G; ++j) {
                const int Pf = map_face(k0 + j, n, bl, bh);
                double xyz[3];
                cell_position<double>(pb, axis, 0, ja, jb, xyz);
                xyz[axis] = lo + (double)Pf * pb->dx;
                BasePoint<double> b = base_at<double>(pb, xyz);
                P.rho0f[Pencil<double>::at(j)] = b.rho0;
                P.p0f[Pencil<double>::at(j)] = b.p0;
            }
            P.i0 = k0;   // sources use the global position of each updated cell
            pass(pb, P, dt, src);
            for (int i = 0; i < nzl; ++i) {
                const int k = Pencil<double>::at(i);
                const long long c = (long long)(i + G) * plane + pidx;
                q[0][c] = P.rho0c[k] + P.rdn[k];
                q[3][c] = P.mnn[k];
                q[1][c] = P.mt1n[k];
                q[2][c] = P.mt2n[k];
                q[4][c] = P.p0c[k] / gm1 + P.edn[k];
                q[5][c] = P.fvn[k];
                q[8][c] = P.onn[k];
                q[6][c] = P.ot1n[k];
                q[7][c] = P.ot2n[k];
            }
            flush_counters(P);
        }
    }
}

void oracle_diagnostics(const oracle_problem *pb, double *const q[9], double totals[7], int nbins,
                        double rmax, double *profiles, double *max_mach) {
    const double gam = pb->gamma, gm1 = pb->gamma - 1.0;
    const double dV = pb->dx * pb->dx * pb->dx;
    const long long ncell = (long long)pb->nx * pb->ny * pb->nz;
    double t[7] = {0, 0, 0, 0, 0, 0, 0};
    std::vector<double> acc((size_t)(nbins > 0 ? nbins : 0) * 6, 0.0);
    double mmax = 0.0;
    for (long long c = 0; c < ncell; ++c) {
        int i = (int)(c % pb->nx), j = (int)((c / pb->nx) % pb->ny), k = (int)(c / ((long long)pb->nx * pb->ny));
        double xyz[3];
        cell_position<double>(pb, 0, i, j, k, xyz);
        BasePoint<double> b = base_at<double>(pb, xyz);
        const double rho = q[0][c];
        t[0] += rho;
        t[1] += q[1][c];
        t[2] += q[2][c];
        t[3] += q[3][c];
        t[4] += q[4][c];
        t[5] += rho * q[5][c];
        t[6] += q[5][c];
        const double u = q[1][c] / rho, v = q[2][c] / rho, w = q[3][c] / rho;
        const double ke = 0.5 * (q[1][c] * u + q[2][c] * v + q[3][c] * w);
        const double p = b.p0 + gm1 * ((q[4][c] - b.p0 / gm1) - ke);
        const double cs = std::sqrt(gam * p / rho);
        const double speed = std::sqrt(u * u + v * v + w * w);
        mmax = std::max(mmax, speed / cs);
        if (nbins > 0) {
            const double r = std::sqrt(xyz[0] * xyz[0] + xyz[1] * xyz[1] + xyz[2] * xyz[2]);
            const int bin = (int)std::floor(r / rmax * nbins);
            if (bin >= 0 && bin < nbins) {
                const double ur = r > 0.0 ? (u * xyz[0] + v * xyz[1] + w * xyz[2]) / r : 0.0;
                double *a = &acc[(size_t)bin * 6];
                a[0] += 1.0;
                a[1] += rho;
                a[2] += p;
                a[3] += q[5][c];
                a[4] += speed;
                a[5] += ur * ur;
            }
        }
    }
    for (int m = 0; m < 7; ++m) totals[m] = t[m] * dV;
    for (int b = 0; b < nbins; ++b) {
        const double *a = &acc[(size_t)b * 6];
        for (int m = 0; m < 5; ++m) profiles[b * 5 + m] = a[0] > 0.0 ? a[1 + m] / a[0] : 0.0;
    }
    if (max_mach) *max_mach = mmax;
}

void oracle_divergence(const oracle_problem *pb, double *const q[9], double *out) {
    std::vector<double> D;
    divergence(pb, q, D);
    std::memcpy(out, D.data(), sizeof(double) * D.size());
}

void oracle_counters(long long out[8]) {
    for (int i = 0; i < 8; ++i) out[i] = g_cnt[i].load();
}

void oracle_reset_counters(void) {
    for (int i = 0; i < 8; ++i) g_cnt[i] = 0;
}

void oracle_count_flops(const oracle_problem *pb, double *const q[9], int axis, double dt, double out[2]) {
    const long long ncell = (long long)pb->nx * pb->ny * pb->nz;
    const int nv = pb->nmom == 9 ? 15 : 9;
    std::vector<std::vector<double>> copy(nv, std::vector<double>((size_t)ncell));
    double *qc[15];
    for (int v = 0; v < nv; ++v) {
        std::memcpy(copy[v].data(), q[v], sizeof(double) * (size_t)ncell);
        qc[v] = copy[v].data();
    }
    Counted::flops = 0;
    Counted::selects = 0;
    // count only the pass itself (gather/scatter excluded)
    const int n = extent(pb, axis);
    const int na = extent(pb, (axis + 1) % 3), nb = extent(pb, (axis + 2) % 3);
    Pencil<Counted> P;
    P.alloc(n);
    P.axis = axis;
    long long fl = 0, se = 0;
    for (long long p = 0; p < (long long)na * nb; ++p) {
        P.ja = (int)(p % na);
        P.jb = (int)(p / na);
        if (!pencil_run(pb, axis, P.ja, P.jb, &P.i0, &P.n)) continue;
        P.confined = pb->confine_r > 0.0;
        P.ten = pb->nmom == 9;
        gather(pb, P, qc);
        Counted::flops = 0;
        Counted::selects = 0;
        pass(pb, P, Counted(dt), 0);
        fl += Counted::flops;
        se += Counted::selects;
    }
    out[0] = (double)fl / (double)ncell;
    out[1] = (double)se / (double)ncell;
}

void oracle_set_threads(int n) { g_threads = n; }

int oracle_get_threads(void) {
#ifdef _OPENMP
    return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
    return 1;
#endif
}

}  // extern "C"
