/*
 * dg2_oracle.c -- plain, slow FP64 CPU statement of the slope-decoupled DG2
 * shallow-water scheme of Ayog et al., "Second-order discontinuous Galerkin
 * flood model" (Sec. 2.1, Eqs. 1-7; diagnostics Eq. 11).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA path is
 * checked against.  Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference legs may load it.  It shares no code, header,
 * table or constant with the CUDA library, and the product never calls it.
 *
 * Style: one cell at a time, every face flux recomputed by each cell that
 * needs it, no blocking or fusion, so that each function can be read against
 * the paper.  Compiled with -ffp-contract=off (no fused multiply-add).
 *
 * Readings where the paper is silent:
 *   - Riemann solver: HLL with Toro's wet/dry wave speeds by default (the
 *     paper uses Roe, Sec. 2.1.2, available as an option).
 *   - z* revision uses the cell's own limit at each of its faces (Sec. 2.1.2).
 *   - Friction: point-implicit backward Euler of S_f, once per time step
 *     before stage 1 (Sec. 2.1.3).
 *   - Local limiter: Jacobi (all cells read the pre-limit state), directional
 *     wet-dry guard over {W,c,E} / {S,c,N}, no limiting normal to a domain
 *     edge, Eq. 6 tested in the division-free form J > thresh * den, with the
 *     magnitude in den floored at tol_dry (so round-off in still water, where
 *     the discharge magnitude vanishes, never counts as a shock).
 *   - RK2: two-stage SSP form; after each stage a wet-dry treatment (dry cells
 *     keep only h0; a wet cell drops to first order in a direction where a face
 *     depth reaches tol_dry at a non-wall face); averages are never clipped.
 *   - Boundary ghosts: wall (normal discharge negated), transmissive (copy,
 *     without an inward normal discharge), inflow segment (critical-depth ghost
 *     carrying Q(t) per unit width).
 *   - Sources (rain, point inflow) add to L0 of h; the paper has none.
 *
 * Parity pins and what each one fixes are in tests/test_oracle_*.py.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef ORC_REAL
typedef double real;
#else
typedef ORC_REAL real;
#endif

/* Plane index of variable v (0 h, 1 qx, 2 qy) and mode m (0 average,
 * 1 x-slope, 2 y-slope) in the 9-plane state array (Eq. 2). */
#define PL(v, m) ((v) * 3 + (m))

enum { EW = 0, EE = 1, ES = 2, EN = 3 };    /* domain edges west, east, south, north */
enum { BC_WALL = 0, BC_OPEN = 1 };

#define MAX_INFLOW 8
#define MAX_KNOTS 4096

typedef struct {
    int edge;              /* EW..EN */
    double s0, len;        /* segment [s0, s0+len] along the edge (m) */
    int nk;
    double tk[MAX_KNOTS];  /* piecewise-linear hydrograph Q(t), m^3/s */
    real qk[MAX_KNOTS];
} inflow_t;

typedef struct {
    int nx, ny;
    double dx, dy;
    double g, cfl, tol_dry, ds_thresh, dt_max;
    int limiter;           /* 0: DG2-NL, 1: DG2-LL */
    int flux;              /* Riemann solver: 0 HLL, 1 Roe */
    int scheme;            /* 0 DG2, 1 MUSCL-FV2, 2 FV1 (Sec. 2.2 comparators) */
    int wd;                /* DG2 face revision: 1 (default) positivity-consistent depths
                              in partially wet cells, 0 Sec. 2.1.2 as printed */
    int bc[4];
    int n_in;
    inflow_t in[MAX_INFLOW];
    double rain, rain_t0, rain_t1;   /* m/s over [t0, t1) */
    double px, py, qp;               /* point inflow (m^3/s) at (px, py) */
    real *z;               /* 3 planes: z0, z1x, z1y (Eq. 3 applied to the DEM) */
    real *nm;              /* Manning n per cell */
    real *U;               /* 9 planes (Eq. 2) */
    real *U1, *L, *Ls;     /* stage state, operator output, limiter scratch */
    real *bnd;             /* mass fluxes of the edge faces of the last operator call:
                              west [ny], east [ny], south [nx], north [nx] */
    double t;
    real ledger;           /* initial mass + boundary and source volumes */
    real last_bflux;       /* boundary + source volume rate of the last operator call */
} orc_t;

/* ------------------------------------------------------------------ */
/* Point values of U = [h, hu, hv] (Eq. 1)                             */
/* ------------------------------------------------------------------ */

typedef struct { real h, qx, qy; } st3;

static st3 mk(real h, real qx, real qy) { st3 s; s.h = h; s.qx = qx; s.qy = qy; return s; }

/* Velocities of a point state: q/h above tol_dry, zero otherwise (Sec. 2.1.2). */
static void velocities(const orc_t *o, st3 s, real *u, real *v)
{
    if (s.h > o->tol_dry) { *u = s.qx / s.h; *v = s.qy / s.h; }
    else { *u = 0.0; *v = 0.0; }
}

/* Physical flux F(U) = [hu, hu^2 + g h^2 / 2, huv] (Eq. 1). */
static st3 flux_x(const orc_t *o, st3 s)
{
    real u, v;
    velocities(o, s, &u, &v);
    return mk(s.h * u, s.h * u * u + 0.5 * o->g * s.h * s.h, s.h * u * v);
}

/* Physical flux G(U) = [hv, huv, hv^2 + g h^2 / 2] (Eq. 1). */
static st3 flux_y(const orc_t *o, st3 s)
{
    real u, v;
    velocities(o, s, &u, &v);
    return mk(s.h * v, s.h * u * v, s.h * v * v + 0.5 * o->g * s.h * s.h);
}

/* Depth-positivity revision of a face limit (Sec. 2.1.2):
 * h* = max(0, h), q* = h* u, with u zeroed at or below tol_dry. */
static st3 revise(const orc_t *o, st3 s)
{
    real u, v;
    velocities(o, s, &u, &v);
    real hs = s.h > 0.0 ? s.h : (real)0.0;
    return mk(hs, hs * u, hs * v);
}

/* HLL flux across a face normal to x, left state L, right state R.
 * Wave speeds (not printed in the paper, which names Roe): Toro's estimates,
 * with the dry-bed forms when one side is at or below tol_dry. */
static st3 hll_x(const orc_t *o, st3 Ls, st3 Rs)
{
    const real tol = o->tol_dry, g = o->g;
    if (Ls.h <= tol && Rs.h <= tol) return mk(0.0, 0.0, 0.0);
    real uL, vL, uR, vR;
    velocities(o, Ls, &uL, &vL);
    velocities(o, Rs, &uR, &vR);
    real cL = sqrt(g * Ls.h), cR = sqrt(g * Rs.h);
    real sL, sR;
    if (Ls.h <= tol) {
        sL = uR - 2.0 * cR;
        sR = uR + cR;
    } else if (Rs.h <= tol) {
        sL = uL - cL;
        sR = uL + 2.0 * cL;
    } else {
        real us = 0.5 * (uL + uR) + cL - cR;
        real cs = 0.5 * (cL + cR) + 0.25 * (uL - uR);
        real a = uL - cL, b = us - cs;
        sL = a < b ? a : b;
        real c = uR + cR, d = us + cs;
        sR = c > d ? c : d;
    }
    st3 FL = flux_x(o, Ls), FR = flux_x(o, Rs);
    if (sL >= 0.0) return FL;
    if (sR <= 0.0) return FR;
    real den = sR - sL;
    return mk((sR * FL.h - sL * FR.h + sL * sR * (Rs.h - Ls.h)) / den,
              (sR * FL.qx - sL * FR.qx + sL * sR * (Rs.qx - Ls.qx)) / den,
              (sR * FL.qy - sL * FR.qy + sL * sR * (Rs.qy - Ls.qy)) / den);
}

/* Acoustic-wave speed magnitude with Harten's entropy fix: |lam| is
 * replaced by (lam^2 + d^2) / (2 d) when |lam| < d, d = max(0, lam - lamL,
 * lamR - lam) (the spread of the characteristic speeds across the face). */
static real harten(real lam, real lamL, real lamR)
{
    real d = lam - lamL;
    if (lamR - lam > d) d = lamR - lam;
    if (d < 0.0) d = 0.0;
    real a = fabs(lam);
    if (a < d) a = (lam * lam + d * d) / (2.0 * d);
    return a;
}

/* Roe flux across a face normal to x (Sec. 2.1.2 names Roe's solver): the
 * average of the two physical fluxes minus the upwinding of the three waves of
 * the Roe-linearised system, with Roe averages u^ = (sqrt(hL) uL +
 * sqrt(hR) uR) / (sqrt(hL) + sqrt(hR)) (v^ alike), h^ = sqrt(hL hR),
 * c^ = sqrt(g (hL + hR) / 2), eigenvalues u^ - c^, u^, u^ + c^, wave
 * strengths a1,3 = (dh -+ h^ du / c^) / 2, a2 = h^ dv, eigenvectors
 * (1, u^ -+ c^, v^) and (0, 0, 1); Harten's entropy fix on the acoustic
 * waves; zero flux between two dry limits. */
static st3 roe_x(const orc_t *o, st3 Ls, st3 Rs)
{
    const real tol = o->tol_dry, g = o->g;
    if (Ls.h <= tol && Rs.h <= tol) return mk(0.0, 0.0, 0.0);
    real uL, vL, uR, vR;
    velocities(o, Ls, &uL, &vL);
    velocities(o, Rs, &uR, &vR);
    real sL = sqrt(Ls.h), sR = sqrt(Rs.h);
    real uh = (sL * uL + sR * uR) / (sL + sR);
    real vh = (sL * vL + sR * vR) / (sL + sR);
    real hh = sL * sR;
    real ch = sqrt(0.5 * g * (Ls.h + Rs.h));
    real dh = Rs.h - Ls.h, du = uR - uL, dv = vR - vL;
    real a1 = 0.5 * (dh - hh * du / ch), a2 = hh * dv, a3 = 0.5 * (dh + hh * du / ch);
    real l1 = uh - ch, l3 = uh + ch;
    real cL = sqrt(g * Ls.h), cR = sqrt(g * Rs.h);
    real e1 = harten(l1, uL - cL, uR - cR), e2 = fabs(uh), e3 = harten(l3, uL + cL, uR + cR);
    st3 FL = flux_x(o, Ls), FR = flux_x(o, Rs);
    real w1 = e1 * a1, w2 = e2 * a2, w3 = e3 * a3;
    return mk(0.5 * (FL.h + FR.h) - 0.5 * (w1 + w3),
              0.5 * (FL.qx + FR.qx) - 0.5 * (w1 * l1 + w3 * l3),
              0.5 * (FL.qy + FR.qy) - 0.5 * (w1 * vh + w2 + w3 * vh));
}

/* The Riemann solver of the run across a face normal to x. */
static st3 riemann_x(const orc_t *o, st3 Ls, st3 Rs)
{
    return o->flux == 1 ? roe_x(o, Ls, Rs) : hll_x(o, Ls, Rs);
}

/* Flux across a face normal to y: the x-solver in the frame where y is
 * the normal direction (qy normal, qx tangential), rotated back. */
static st3 hll_y(const orc_t *o, st3 Ss, st3 Ns)
{
    st3 r = riemann_x(o, mk(Ss.h, Ss.qy, Ss.qx), mk(Ns.h, Ns.qy, Ns.qx));
    return mk(r.h, r.qy, r.qx);
}

/* ------------------------------------------------------------------ */
/* Boundary ghost states                                               */
/* ------------------------------------------------------------------ */

/* Piecewise-linear hydrograph, held constant outside its knots. */
static real hydrograph(const inflow_t *f, double t)
{
    if (f->nk <= 0) return 0.0;
    if (t <= f->tk[0]) return f->qk[0];
    for (int k = 0; k + 1 < f->nk; ++k) {
        if (t <= f->tk[k + 1]) {
            double w = (t - f->tk[k]) / (f->tk[k + 1] - f->tk[k]);
            return f->qk[k] + w * (f->qk[k + 1] - f->qk[k]);
        }
    }
    return f->qk[f->nk - 1];
}

/* Number of faces of edge e whose centre lies in the segment of inflow f. */
static int inflow_nfaces(const orc_t *o, const inflow_t *f)
{
    int n = (f->edge == EW || f->edge == EE) ? o->ny : o->nx;
    double d = (f->edge == EW || f->edge == EE) ? o->dy : o->dx;
    int cnt = 0;
    for (int k = 0; k < n; ++k) {
        double s = (k + 0.5) * d;
        if (s >= f->s0 && s <= f->s0 + f->len) ++cnt;
    }
    return cnt;
}

/* The state outside edge `edge` at the face whose centre has edge coordinate
 * s, given the cell's own (unrevised) limit `in` at that face. */
static st3 ghost(const orc_t *o, int edge, double s, st3 in, double t)
{
    for (int k = 0; k < o->n_in; ++k) {
        const inflow_t *f = &o->in[k];
        if (f->edge != edge || s < f->s0 || s > f->s0 + f->len) continue;
        int nf = inflow_nfaces(o, f);
        double d = (edge == EW || edge == EE) ? o->dy : o->dx;
        real qin = hydrograph(f, t) / (nf * d);          /* discharge per unit width */
        real hin = in.h > 0.0 ? in.h : (real)0.0;
        real hc = cbrt(qin * qin / o->g);                /* critical depth of qin */
        real hg = hin > hc ? hin : hc;
        real qn = (edge == EW || edge == ES) ? qin : -qin;   /* pointing into the domain */
        if (edge == EW || edge == EE) return mk(hg, qn, 0.0);
        return mk(hg, 0.0, qn);
    }
    if (o->bc[edge] == BC_OPEN) {
        /* transmissive edge read as free outflow: the state is copied, but a
         * normal discharge pointing into the domain is not */
        if (edge == EW && in.qx > 0.0) return mk(in.h, 0.0, in.qy);
        if (edge == EE && in.qx < 0.0) return mk(in.h, 0.0, in.qy);
        if (edge == ES && in.qy > 0.0) return mk(in.h, in.qx, 0.0);
        if (edge == EN && in.qy < 0.0) return mk(in.h, in.qx, 0.0);
        return in;
    }
    /* wall: reflect the normal discharge */
    if (edge == EW || edge == EE) return mk(in.h, -in.qx, in.qy);
    return mk(in.h, in.qx, -in.qy);
}

/* ------------------------------------------------------------------ */
/* Face limits of the planar solution (Eq. 2 evaluated at E, W, N, S)  */
/* ------------------------------------------------------------------ */

static st3 limit_at(const orc_t *o, const real *U, int i, int j, int face)
{
    size_t N = (size_t)o->nx * o->ny, c = (size_t)j * o->nx + i;
    int m = (face == EE || face == EW) ? 1 : 2;
    real sg = (face == EE || face == EN) ? 1.0 : -1.0;
    return mk(U[PL(0, 0) * N + c] + sg * U[PL(0, m) * N + c],
              U[PL(1, 0) * N + c] + sg * U[PL(1, m) * N + c],
              U[PL(2, 0) * N + c] + sg * U[PL(2, m) * N + c]);
}

static real zlimit_at(const orc_t *o, int i, int j, int face)
{
    size_t N = (size_t)o->nx * o->ny, c = (size_t)j * o->nx + i;
    int m = (face == EE || face == EW) ? 1 : 2;
    real sg = (face == EE || face == EN) ? 1.0 : -1.0;
    return o->z[0 * N + c] + sg * o->z[m * N + c];
}

/* Limit on the far side of face `face` of cell (i, j): the neighbour's
 * opposite limit, or the boundary ghost built from the cell's own limit. */
static st3 outer_limit(const orc_t *o, const real *U, int i, int j, int face, double t)
{
    switch (face) {
    case EE: return i + 1 < o->nx ? limit_at(o, U, i + 1, j, EW)
                                  : ghost(o, EE, (j + 0.5) * o->dy, limit_at(o, U, i, j, EE), t);
    case EW: return i > 0 ? limit_at(o, U, i - 1, j, EE)
                          : ghost(o, EW, (j + 0.5) * o->dy, limit_at(o, U, i, j, EW), t);
    case EN: return j + 1 < o->ny ? limit_at(o, U, i, j + 1, ES)
                                  : ghost(o, EN, (i + 0.5) * o->dx, limit_at(o, U, i, j, EN), t);
    default: return j > 0 ? limit_at(o, U, i, j - 1, EN)
                          : ghost(o, ES, (i + 0.5) * o->dx, limit_at(o, U, i, j, ES), t);
    }
}

/* ------------------------------------------------------------------ */
/* Revised face states (Sec. 2.1.2), and the positivity-consistent      */
/* variant for partially wet cells                                      */
/* ------------------------------------------------------------------ */

/* One side of a face: its planar limit, the depth the face may draw on, the
 * side's own bed level and free surface there. */
typedef struct { st3 lim; real hs, zo, eta, u, v; int pw; } frec;

/* Velocity of a face limit under the default revision: q/h by the tol rule,
 * except at a limit thinner than eps = h0 / 10 in a cell whose mean depth h0
 * is above 10 tol_dry, where the planar discharge is not a resolved velocity
 * (a 6e-5 m limit carrying 1.2 m^2/s beside a 1 m deep average moves at
 * 20 km/s).  There the velocity is desingularised as in Kurganov and Petrova
 * (2007), u = 2 h q / (h^2 + eps^2) with h clipped at 0, which equals q/h at
 * h = eps and falls to 0 with h: continuous in h and q. */
static void face_velocity(const orc_t *o, st3 lim, real h0, real *u, real *v)
{
    const real eps = 0.1 * h0;
    if (eps > o->tol_dry && lim.h < eps) {
        const real hp = lim.h > 0.0 ? lim.h : (real)0.0;
        const real den = lim.h * lim.h + eps * eps;
        *u = 2.0 * hp * lim.qx / den;
        *v = 2.0 * hp * lim.qy / den;
        return;
    }
    velocities(o, lim, u, v);
}

/* The four face records of cell (i, j).  A wet cell (h0 > tol_dry) whose planar
 * depth is negative at a face is partially wet: its clipped face depths
 * max(0, h_f) average to more than h0, so they are scaled to average h0, and
 * each face gets the bed level under the planar free surface at that depth
 * (z_f raised by the depth removed).  Every other cell keeps max(0, h_f) over
 * the continuous bed. */
static void cell_recs(const orc_t *o, const real *U, int i, int j, frec r[4])
{
    const size_t c = (size_t)j * o->nx + i;
    const real h0 = U[c];
    real sum = 0.0;
    int neg = 0;
    for (int f = 0; f < 4; ++f) {
        r[f].lim = limit_at(o, U, i, j, f);
        real hf = r[f].lim.h;
        if (hf < 0.0) neg = 1;
        sum += hf > 0.0 ? hf : (real)0.0;
    }
    const int pw = h0 > o->tol_dry && neg;
    const real sc = pw ? h0 / (0.25 * sum) : (real)1.0;
    for (int f = 0; f < 4; ++f) {
        real hf = r[f].lim.h, zf = zlimit_at(o, i, j, f);
        real hp = hf > 0.0 ? hf : (real)0.0;
        face_velocity(o, r[f].lim, h0, &r[f].u, &r[f].v);
        r[f].pw = pw;
        if (pw) {
            r[f].hs = sc * hp;
            r[f].eta = hf + zf;
            r[f].zo = r[f].eta - r[f].hs;
        } else {
            r[f].hs = hp;
            r[f].zo = zf;
            r[f].eta = zf + hp;
        }
    }
}

/* Record of the far side of face f of cell (i, j): the neighbour's, or the
 * boundary ghost of the own planar limit over the own face bed. */
static frec outer_rec(const orc_t *o, const real *U, int i, int j, int f, double t)
{
    int ni = i + (f == EE) - (f == EW), nj = j + (f == EN) - (f == ES);
    int opp = f == EE ? EW : f == EW ? EE : f == EN ? ES : EN;
    frec r;
    if (ni >= 0 && ni < o->nx && nj >= 0 && nj < o->ny) {
        frec nr[4];
        cell_recs(o, U, ni, nj, nr);
        return nr[opp];
    }
    r.lim = outer_limit(o, U, i, j, f, t);
    real zf = zlimit_at(o, i, j, f);
    velocities(o, r.lim, &r.u, &r.v);
    r.hs = r.lim.h > 0.0 ? r.lim.h : (real)0.0;
    r.zo = zf;
    r.eta = zf + r.hs;
    r.pw = 0;
    return r;
}

/* Revised states of the face between lower side a and upper side b, and the
 * bed level each side's own bed term uses.  Neither side partially wet: the
 * revision of Sec. 2.1.2 over the continuous bed.  Otherwise the free-surface
 * revision of Sec. 2.2.2 on the sides' own bed levels: z* = max(za, zb),
 * h* = max(0, eta - z*), q* = h* u, and each side's bed term takes z* lowered
 * by the amount its free surface lies below it. */
static void face_revise(const orc_t *o, frec a, frec b, st3 *ra, st3 *rb, real *za, real *zb)
{
    if (!a.pw && !b.pw) {
        *ra = mk(a.hs, a.hs * a.u, a.hs * a.v);
        *rb = mk(b.hs, b.hs * b.u, b.hs * b.v);
        *za = a.zo - (a.lim.h < 0.0 ? -a.lim.h : (real)0.0);
        *zb = b.zo - (b.lim.h < 0.0 ? -b.lim.h : (real)0.0);
        return;
    }
    real zs = a.zo > b.zo ? a.zo : b.zo;
    real ha = a.eta - zs, hb = b.eta - zs;
    if (ha < 0.0) ha = 0.0;
    if (hb < 0.0) hb = 0.0;
    *ra = mk(ha, ha * a.u, ha * a.v);
    *rb = mk(hb, hb * b.u, hb * b.v);
    real da = a.eta - zs, db = b.eta - zs;
    *za = zs - (da < 0.0 ? -da : (real)0.0);
    *zb = zs - (db < 0.0 ? -db : (real)0.0);
}

/* ------------------------------------------------------------------ */
/* Spatial operators L0, L1x, L1y (Eqs. 4a-c with Eq. 5)               */
/* ------------------------------------------------------------------ */

static int source_cell(const orc_t *o)
{
    if (o->qp == 0.0) return -1;
    int i = (int)floor(o->px / o->dx), j = (int)floor(o->py / o->dy);
    if (i < 0) i = 0;
    if (i >= o->nx) i = o->nx - 1;
    if (j < 0) j = 0;
    if (j >= o->ny) j = o->ny - 1;
    return j * o->nx + i;
}

/* Writes the 9 operator planes of state U at time t into Lout and returns
 * the rate (m^3/s) at which boundary fluxes and sources add water. */
static real spatial_operator(const orc_t *o, const real *U, double t, real *Lout)
{
    const int nx = o->nx, ny = o->ny;
    const size_t N = (size_t)nx * ny;
    const real g = o->g, dx = o->dx, dy = o->dy, s3 = sqrt(3.0);
    const int csrc = source_cell(o);
    const int raining = (o->rain != 0.0 && t >= o->rain_t0 && t < o->rain_t1);
    real bsum = 0.0;
    real *bw = o->bnd, *be = o->bnd + ny, *bs = o->bnd + 2 * ny, *bn = o->bnd + 2 * ny + nx;

    /* every cell writes only its own outputs (rows may run in parallel when built
     * with OpenMP: the results do not depend on it) */
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t c = (size_t)j * nx + i;
            st3 Es, Ws, Ns, Ss;
            real zE, zW, zN, zS;
            st3 FE, FW, GN, GS;
            if (!o->wd) {
                /* own limits and their revision */
                st3 E = limit_at(o, U, i, j, EE), W = limit_at(o, U, i, j, EW);
                st3 Nn = limit_at(o, U, i, j, EN), S = limit_at(o, U, i, j, ES);
                Es = revise(o, E); Ws = revise(o, W); Ns = revise(o, Nn); Ss = revise(o, S);
                /* topography limits, revised with the own depth limit at each face */
                zE = zlimit_at(o, i, j, EE) - (E.h < 0.0 ? -E.h : (real)0.0);
                zW = zlimit_at(o, i, j, EW) - (W.h < 0.0 ? -W.h : (real)0.0);
                zN = zlimit_at(o, i, j, EN) - (Nn.h < 0.0 ? -Nn.h : (real)0.0);
                zS = zlimit_at(o, i, j, ES) - (S.h < 0.0 ? -S.h : (real)0.0);
                /* inter-elemental fluxes */
                FE = riemann_x(o, Es, revise(o, outer_limit(o, U, i, j, EE, t)));
                FW = riemann_x(o, revise(o, outer_limit(o, U, i, j, EW, t)), Ws);
                GN = hll_y(o, Ns, revise(o, outer_limit(o, U, i, j, EN, t)));
                GS = hll_y(o, revise(o, outer_limit(o, U, i, j, ES, t)), Ss);
            } else {
                frec r[4];
                cell_recs(o, U, i, j, r);
                st3 oE, oW, oN, oS;
                real zx;
                face_revise(o, r[EE], outer_rec(o, U, i, j, EE, t), &Es, &oE, &zE, &zx);
                face_revise(o, outer_rec(o, U, i, j, EW, t), r[EW], &oW, &Ws, &zx, &zW);
                face_revise(o, r[EN], outer_rec(o, U, i, j, EN, t), &Ns, &oN, &zN, &zx);
                face_revise(o, outer_rec(o, U, i, j, ES, t), r[ES], &oS, &Ss, &zx, &zS);
                FE = riemann_x(o, Es, oE);
                FW = riemann_x(o, oW, Ws);
                GN = hll_y(o, Ns, oN);
                GS = hll_y(o, oS, Ss);
            }
            if (i == 0) bw[j] = FW.h;
            if (i == nx - 1) be[j] = FE.h;
            if (j == 0) bs[i] = GS.h;
            if (j == ny - 1) bn[i] = GN.h;
            /* dummy modes, Eq. 5 (Eq. 5b read as the 0y mode) */
            st3 U0x = mk(0.5 * (Es.h + Ws.h), 0.5 * (Es.qx + Ws.qx), 0.5 * (Es.qy + Ws.qy));
            st3 U1x = mk(0.5 * (Es.h - Ws.h), 0.5 * (Es.qx - Ws.qx), 0.5 * (Es.qy - Ws.qy));
            st3 U0y = mk(0.5 * (Ns.h + Ss.h), 0.5 * (Ns.qx + Ss.qx), 0.5 * (Ns.qy + Ss.qy));
            st3 U1y = mk(0.5 * (Ns.h - Ss.h), 0.5 * (Ns.qx - Ss.qx), 0.5 * (Ns.qy - Ss.qy));
            real z1x = 0.5 * (zE - zW), z1y = 0.5 * (zN - zS);
            /* physical fluxes at the two Gauss points of each centreline */
            st3 Fp = flux_x(o, mk(U0x.h + U1x.h / s3, U0x.qx + U1x.qx / s3, U0x.qy + U1x.qy / s3));
            st3 Fm = flux_x(o, mk(U0x.h - U1x.h / s3, U0x.qx - U1x.qx / s3, U0x.qy - U1x.qy / s3));
            st3 Gp = flux_y(o, mk(U0y.h + U1y.h / s3, U0y.qx + U1y.qx / s3, U0y.qy + U1y.qy / s3));
            st3 Gm = flux_y(o, mk(U0y.h - U1y.h / s3, U0y.qx - U1y.qx / s3, U0y.qy - U1y.qy / s3));
            /* Eq. 4a */
            real L0h = -(FE.h - FW.h) / dx - (GN.h - GS.h) / dy;
            real L0x = -(FE.qx - FW.qx) / dx - (GN.qx - GS.qx) / dy - 2.0 * g * U0x.h * z1x / dx;
            real L0y = -(FE.qy - FW.qy) / dx - (GN.qy - GS.qy) / dy - 2.0 * g * U0y.h * z1y / dy;
            if (raining) L0h += o->rain;
            if ((int)c == csrc) L0h += o->qp / (dx * dy);
            /* Eq. 4b */
            real L1xh = -(3.0 / dx) * ((FE.h + FW.h) - (Fp.h + Fm.h));
            real L1xx = -(3.0 / dx) * ((FE.qx + FW.qx) - (Fp.qx + Fm.qx) + (2.0 * g / 3.0) * U1x.h * z1x);
            real L1xy = -(3.0 / dx) * ((FE.qy + FW.qy) - (Fp.qy + Fm.qy));
            /* Eq. 4c */
            real L1yh = -(3.0 / dy) * ((GN.h + GS.h) - (Gp.h + Gm.h));
            real L1yx = -(3.0 / dy) * ((GN.qx + GS.qx) - (Gp.qx + Gm.qx));
            real L1yy = -(3.0 / dy) * ((GN.qy + GS.qy) - (Gp.qy + Gm.qy) + (2.0 * g / 3.0) * U1y.h * z1y);

            Lout[PL(0, 0) * N + c] = L0h;
            Lout[PL(1, 0) * N + c] = L0x;
            Lout[PL(2, 0) * N + c] = L0y;
            Lout[PL(0, 1) * N + c] = L1xh;
            Lout[PL(1, 1) * N + c] = L1xx;
            Lout[PL(2, 1) * N + c] = L1xy;
            Lout[PL(0, 2) * N + c] = L1yh;
            Lout[PL(1, 2) * N + c] = L1yx;
            Lout[PL(2, 2) * N + c] = L1yy;
        }
    /* volume rate through the domain edges, summed in cell order */
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            if (i == 0) bsum += bw[j] * dy;
            if (i == nx - 1) bsum -= be[j] * dy;
            if (j == 0) bsum += bs[i] * dx;
            if (j == ny - 1) bsum -= bn[i] * dx;
        }
    if (raining) bsum += o->rain * dx * dy * (double)N;
    if (csrc >= 0) bsum += o->qp;
    return bsum;
}

/* ------------------------------------------------------------------ */
/* Friction (Sec. 2.1.3): implicit splitting of S_f at the centre and   */
/* at the Gauss points of both centrelines                              */
/* ------------------------------------------------------------------ */

/* dq/dt = -g n^2 q |q| / h^(7/3) (S_f of Eq. 1 written in q, h), advanced
 * one step by backward Euler with |q| frozen at the old value. */
static void friction_point(const orc_t *o, real n, real dt, real h, real *qx, real *qy)
{
    if (h <= o->tol_dry || n == 0.0) return;
    real qm = sqrt((*qx) * (*qx) + (*qy) * (*qy));
    real d = 1.0 + dt * o->g * n * n * qm / (h * h * cbrt(h));
    *qx = *qx / d;
    *qy = *qy / d;
}

static void apply_friction(orc_t *o, real *U, double dt)
{
    const size_t N = (size_t)o->nx * o->ny;
    const real s3 = sqrt(3.0);
#pragma omp parallel for schedule(static)
    for (size_t c = 0; c < N; ++c) {
        real n = o->nm[c];
        real h0 = U[PL(0, 0) * N + c], x0 = U[PL(1, 0) * N + c], y0 = U[PL(2, 0) * N + c];
        /* centre point -> average discharges */
        real cx = x0, cy = y0;
        friction_point(o, n, dt, h0, &cx, &cy);
        /* Gauss points of each centreline -> slope discharges by differencing */
        real nq[2][2];
        for (int d = 1; d <= 2; ++d) {
            real h1 = U[PL(0, d) * N + c], x1 = U[PL(1, d) * N + c], y1 = U[PL(2, d) * N + c];
            real hp = h0 + h1 / s3, xp = x0 + x1 / s3, yp = y0 + y1 / s3;
            real hm = h0 - h1 / s3, xm = x0 - x1 / s3, ym = y0 - y1 / s3;
            friction_point(o, n, dt, hp, &xp, &yp);
            friction_point(o, n, dt, hm, &xm, &ym);
            nq[d - 1][0] = 0.5 * s3 * (xp - xm);
            nq[d - 1][1] = 0.5 * s3 * (yp - ym);
        }
        U[PL(1, 0) * N + c] = cx;
        U[PL(2, 0) * N + c] = cy;
        U[PL(1, 1) * N + c] = nq[0][0];
        U[PL(2, 1) * N + c] = nq[0][1];
        U[PL(1, 2) * N + c] = nq[1][0];
        U[PL(2, 2) * N + c] = nq[1][1];
    }
}

/* ------------------------------------------------------------------ */
/* Local limiting (Sec. 2.1.3, Eqs. 6-7)                               */
/* ------------------------------------------------------------------ */

static real minmod3(real a, real b, real c)
{
    if (a > 0.0 && b > 0.0 && c > 0.0) {
        real m = a < b ? a : b;
        return m < c ? m : c;
    }
    if (a < 0.0 && b < 0.0 && c < 0.0) {
        real m = a > b ? a : b;
        return m > c ? m : c;
    }
    return 0.0;
}

/* One component along one direction.  k0w,k1w / k0,k1 / k0e,k1e are the
 * average and slope of the component in the lower neighbour, the cell and
 * the upper neighbour; half = dx/2 (or dy/2).  Returns the (possibly
 * limited) slope. */
static real limit_component(const orc_t *o, real half, real k0w, real k1w, real k0, real k1,
                            real k0e, real k1e)
{
    const real s3 = sqrt(3.0);
    real jE = fabs((k0e - k1e) - (k0 + k1));           /* |U_E^+ - U_E^-| */
    real jW = fabs((k0 - k1) - (k0w + k1w));           /* |U_W^+ - U_W^-| */
    real a = fabs(k0 - k1 / s3), b = fabs(k0 + k1 / s3);
    real m = a > b ? a : b;
    if (m < o->tol_dry) m = o->tol_dry;       /* still water: round-off cannot trigger */
    real den = half * m;
    real jm = jE > jW ? jE : jW;
    if (!(jm > o->ds_thresh * den)) return k1;          /* Eq. 6 detector: no shock */
    return minmod3(k1, k0e - k0, k0 - k0w);             /* Eq. 7 */
}

/* Jacobi sweep: Uout = limited copy of Uin. */
static void apply_limiter(const orc_t *o, const real *Uin, real *Uout)
{
    const int nx = o->nx, ny = o->ny;
    const size_t N = (size_t)nx * ny;
    memcpy(Uout, Uin, 9 * N * sizeof(real));
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t c = (size_t)j * nx + i;
            for (int d = 1; d <= 2; ++d) {
                int has_lo = d == 1 ? i > 0 : j > 0;
                int has_hi = d == 1 ? i + 1 < nx : j + 1 < ny;
                if (!has_lo || !has_hi) continue;               /* no limiting normal to an edge */
                size_t cl = d == 1 ? c - 1 : c - nx, ch = d == 1 ? c + 1 : c + nx;
                const real tol = o->tol_dry;
                if (Uin[cl] <= tol || Uin[c] <= tol || Uin[ch] <= tol) continue;   /* wet-dry front */
                real half = 0.5 * (d == 1 ? o->dx : o->dy);
                /* free-surface elevation eta = h + z instead of h */
                const real *z0 = o->z, *z1 = o->z + d * N;
                real e1 = limit_component(o, half,
                                          Uin[cl] + z0[cl], Uin[PL(0, d) * N + cl] + z1[cl],
                                          Uin[c] + z0[c], Uin[PL(0, d) * N + c] + z1[c],
                                          Uin[ch] + z0[ch], Uin[PL(0, d) * N + ch] + z1[ch]);
                if (e1 != Uin[PL(0, d) * N + c] + z1[c])
                    Uout[PL(0, d) * N + c] = e1 - z1[c];
                for (int v = 1; v <= 2; ++v) {
                    const real *k0 = Uin + PL(v, 0) * N, *k1 = Uin + PL(v, d) * N;
                    Uout[PL(v, d) * N + c] = limit_component(o, half, k0[cl], k1[cl], k0[c], k1[c],
                                                             k0[ch], k1[ch]);
                }
            }
        }
}

/* ------------------------------------------------------------------ */
/* Time step (Sec. 2.1.2: explicit RK2 under a Courant number)         */
/* ------------------------------------------------------------------ */

/* Wet-dry treatment applied to every stage result (readings of Sec. 2.1.2-2.1.3,
 * which promise depth positivity and flag dry elements by h0 alone):
 *  - a dry cell (h0 <= tol_dry) keeps its average depth only: every slope and
 *    every discharge mode is zeroed;
 *  - in a wet cell, a direction in which a face limit of h is at or below
 *    tol_dry at a face that is not a wall face drops to first order: its h,
 *    qx and qy slopes are zeroed.  A wall face is one whose bed stands above the
 *    cell's mean free surface h0 + z0 -- there the planar solution is kept, so
 *    still water blocked by high ground stays balanced through z*.
 * Averages are never changed, so mass is untouched. */
static void dry_reset(const orc_t *o, real *U)
{
    const size_t N = (size_t)o->nx * o->ny;
#pragma omp parallel for schedule(static)
    for (size_t c = 0; c < N; ++c) {
        real h0 = U[c];
        if (h0 <= o->tol_dry) {
            for (int k = 1; k < 9; ++k) U[k * N + c] = 0.0;
            continue;
        }
        real eta0 = h0 + o->z[c];
        for (int d = 1; d <= 2; ++d) {
            int front = 0;
            for (int sg = -1; sg <= 1; sg += 2) {
                real hp = h0 + sg * U[PL(0, d) * N + c];
                real zp = o->z[c] + sg * o->z[d * N + c];
                if (hp <= o->tol_dry && !(zp > eta0)) front = 1;
            }
            if (front) {
                U[PL(0, d) * N + c] = 0.0;
                U[PL(1, d) * N + c] = 0.0;
                U[PL(2, d) * N + c] = 0.0;
            }
        }
    }
}

double orc_cfl_dt(const orc_t *o)
{
    const size_t N = (size_t)o->nx * o->ny;
    double best = -1.0;
    for (size_t c = 0; c < N; ++c) {
        real h = o->U[c];
        if (h <= o->tol_dry) continue;
        real u = o->U[3 * N + c] / h, v = o->U[6 * N + c] / h, a = sqrt(o->g * h);
        real tx = o->dx / (fabs(u) + a), ty = o->dy / (fabs(v) + a);
        real tc = tx < ty ? tx : ty;
        if (best < 0.0 || tc < best) best = tc;
    }
    if (best < 0.0) return o->dt_max;
    double dt = o->cfl * best;
    return dt < o->dt_max ? dt : o->dt_max;
}

/* ------------------------------------------------------------------ */
/* MUSCL-FV2 and FV1 comparators (Sec. 2.2, Eqs. 8-10)                 */
/* ------------------------------------------------------------------ */

/* Sweby's symmetric limiter with parameter beta (Sec. 2.2.3, beta = 1.25). */
static real sweby(real r, real beta)
{
    real a = beta * r < 1.0 ? beta * r : (real)1.0;
    real b = r < beta ? r : (real)beta;
    real m = a > b ? a : b;
    return m > 0.0 ? m : (real)0.0;
}

/* Component k of cell c for the reconstruction: 0 eta = h + z, 1 h, 2 qx, 3 qy. */
static real fv_val(const orc_t *o, const real *U, size_t c, int k)
{
    const size_t N = (size_t)o->nx * o->ny;
    switch (k) {
    case 0: return U[c] + o->z[c];
    case 1: return U[c];
    case 2: return U[3 * N + c];
    default: return U[6 * N + c];
    }
}

/* Limited MUSCL slope of component k of cell (i, j) along dir (Eq. 10, read
 * with r = forward / backward difference so that the slope stays in Sweby's
 * TVD region); zero without both neighbours, at a wet-dry front (the cell or a
 * neighbour along dir at or below tol_dry, as the DG2 limiter's guard) and for
 * FV1. */
static real fv_slope(const orc_t *o, const real *U, int i, int j, int dir, int k)
{
    if (o->scheme != 1) return 0.0;
    const int nx = o->nx, ny = o->ny;
    if (dir == 1 ? (i == 0 || i == nx - 1) : (j == 0 || j == ny - 1)) return 0.0;
    size_t c = (size_t)j * nx + i;
    size_t lo = dir == 1 ? c - 1 : c - nx, hi = dir == 1 ? c + 1 : c + nx;
    if (U[lo] <= o->tol_dry || U[c] <= o->tol_dry || U[hi] <= o->tol_dry) return 0.0;
    real vc = fv_val(o, U, c, k);
    real db = vc - fv_val(o, U, lo, k), df = fv_val(o, U, hi, k) - vc;
    if (db == 0.0) return 0.0;
    return sweby(df / db, 1.25) * db;
}

typedef struct { real eta, h, qx, qy; } st4;

/* Limit of cell (i, j) at its face (EE, EW, EN, ES): average + / - half the
 * slope (Eq. 9). */
static st4 fv_limit(const orc_t *o, const real *U, int i, int j, int face)
{
    const int dir = (face == EE || face == EW) ? 1 : 2;
    const real sg = (face == EE || face == EN) ? 0.5 : -0.5;
    size_t c = (size_t)j * o->nx + i;
    st4 r;
    r.eta = fv_val(o, U, c, 0) + sg * fv_slope(o, U, i, j, dir, 0);
    r.h = fv_val(o, U, c, 1) + sg * fv_slope(o, U, i, j, dir, 1);
    r.qx = fv_val(o, U, c, 2) + sg * fv_slope(o, U, i, j, dir, 2);
    r.qy = fv_val(o, U, c, 3) + sg * fv_slope(o, U, i, j, dir, 3);
    return r;
}

/* The limit beyond face `face` of cell (i, j): the neighbour's limit, or the
 * boundary ghost of the own limit over the same bed. */
static st4 fv_outer(const orc_t *o, const real *U, int i, int j, int face, double t)
{
    int ni = i + (face == EE) - (face == EW), nj = j + (face == EN) - (face == ES);
    int opp = face == EE ? EW : face == EW ? EE : face == EN ? ES : EN;
    if (ni >= 0 && ni < o->nx && nj >= 0 && nj < o->ny) return fv_limit(o, U, ni, nj, opp);
    st4 own = fv_limit(o, U, i, j, face);
    double s = (face == EE || face == EW) ? (j + 0.5) * o->dy : (i + 0.5) * o->dx;
    st3 g = ghost(o, face, s, mk(own.h, own.qx, own.qy), t);
    st4 r;
    r.eta = g.h + (own.eta - own.h);
    r.h = g.h;
    r.qx = g.qx;
    r.qy = g.qy;
    return r;
}

/* Revised states of a face from its lower (a) and upper (b) limits
 * (Sec. 2.2.2): z+- = eta+- - h+-, z* = max(z-, z+), h*+- = max(0, eta+- - z*),
 * q*+- = h*+- u+- with u by the tol_dry rule; returns z*. */
static real fv_face(const orc_t *o, st4 a, st4 b, st3 *ra, st3 *rb)
{
    real za = a.eta - a.h, zb = b.eta - b.h;
    real zs = za > zb ? za : zb;
    real ha = a.eta - zs, hb = b.eta - zs;
    if (ha < 0.0) ha = 0.0;
    if (hb < 0.0) hb = 0.0;
    real ua, va, ub, vb;
    velocities(o, mk(a.h, a.qx, a.qy), &ua, &va);
    velocities(o, mk(b.h, b.qx, b.qy), &ub, &vb);
    *ra = mk(ha, ha * ua, ha * va);
    *rb = mk(hb, hb * ub, hb * vb);
    return zs;
}

/* Eq. 8 at every cell (bed term read with the factor 2 / dx of Eq. 4a, which
 * balances the face fluxes at rest); returns the boundary + source rate. */
static real fv_operator(const orc_t *o, const real *U, double t, real *Lout)
{
    const int nx = o->nx, ny = o->ny;
    const size_t N = (size_t)nx * ny;
    const real g = o->g, dx = o->dx, dy = o->dy;
    const int csrc = source_cell(o);
    const int raining = (o->rain != 0.0 && t >= o->rain_t0 && t < o->rain_t1);
    real bsum = 0.0;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t c = (size_t)j * nx + i;
            st3 aE, bE, aW, bW, aN, bN, aS, bS;
            st4 own_e = fv_limit(o, U, i, j, EE), own_w = fv_limit(o, U, i, j, EW);
            st4 own_n = fv_limit(o, U, i, j, EN), own_s = fv_limit(o, U, i, j, ES);
            real zE = fv_face(o, own_e, fv_outer(o, U, i, j, EE, t), &aE, &bE);
            real zW = fv_face(o, fv_outer(o, U, i, j, EW, t), own_w, &aW, &bW);
            real zN = fv_face(o, own_n, fv_outer(o, U, i, j, EN, t), &aN, &bN);
            real zS = fv_face(o, fv_outer(o, U, i, j, ES, t), own_s, &aS, &bS);
            st3 FE = riemann_x(o, aE, bE), FW = riemann_x(o, aW, bW);
            st3 GN = hll_y(o, aN, bN), GS = hll_y(o, aS, bS);
            if (i == 0) bsum += FW.h * dy;
            if (i == nx - 1) bsum -= FE.h * dy;
            if (j == 0) bsum += GS.h * dx;
            if (j == ny - 1) bsum -= GN.h * dx;
            /* own-side bed limits, lowered where the own free surface is below
             * z* (water held by a higher wall) */
            real dE = own_e.eta - zE, dW = own_w.eta - zW, dN = own_n.eta - zN, dS = own_s.eta - zS;
            zE = zE - (dE < 0.0 ? -dE : (real)0.0);
            zW = zW - (dW < 0.0 ? -dW : (real)0.0);
            zN = zN - (dN < 0.0 ? -dN : (real)0.0);
            zS = zS - (dS < 0.0 ? -dS : (real)0.0);
            real h0x = 0.5 * (aE.h + bW.h), z1x = 0.5 * (zE - zW);
            real h0y = 0.5 * (aN.h + bS.h), z1y = 0.5 * (zN - zS);
            real Lh = -(FE.h - FW.h) / dx - (GN.h - GS.h) / dy;
            real Lx = -(FE.qx - FW.qx) / dx - (GN.qx - GS.qx) / dy - 2.0 * g * h0x * z1x / dx;
            real Ly = -(FE.qy - FW.qy) / dx - (GN.qy - GS.qy) / dy - 2.0 * g * h0y * z1y / dy;
            if (raining) Lh += o->rain;
            if ((int)c == csrc) Lh += o->qp / (dx * dy);
            for (int k = 0; k < 9; ++k) Lout[k * N + c] = 0.0;
            Lout[c] = Lh;
            Lout[3 * N + c] = Lx;
            Lout[6 * N + c] = Ly;
        }
    if (raining) bsum += o->rain * dx * dy * (double)N;
    if (csrc >= 0) bsum += o->qp;
    return bsum;
}

/* After a stage: a dry cell keeps no discharge. */
static void fv_dry(const orc_t *o, real *U)
{
    const size_t N = (size_t)o->nx * o->ny;
    for (size_t c = 0; c < N; ++c)
        if (U[c] <= o->tol_dry) { U[3 * N + c] = 0.0; U[6 * N + c] = 0.0; }
}

/* One step of the FV comparators: friction on the averages (the DG2
 * procedure at the centre point, Sec. 2.2.3), then RK2 (MUSCL-FV2) or forward
 * Euler (FV1) on Eq. 8. */
static void fv_step(orc_t *o, double dt)
{
    const size_t N = (size_t)o->nx * o->ny;
    real *Un = o->U, *U1 = o->U1, *L = o->L;
    for (size_t c = 0; c < N; ++c) {
        real qx = Un[3 * N + c], qy = Un[6 * N + c];
        friction_point(o, o->nm[c], dt, Un[c], &qx, &qy);
        Un[3 * N + c] = qx;
        Un[6 * N + c] = qy;
    }
    real b1 = fv_operator(o, Un, o->t, L);
    if (o->scheme == 2) {
        for (size_t k = 0; k < 9 * N; ++k) Un[k] = Un[k] + dt * L[k];
        fv_dry(o, Un);
        o->last_bflux = b1;
        o->ledger += dt * b1;
        o->t += dt;
        return;
    }
    for (size_t k = 0; k < 9 * N; ++k) U1[k] = Un[k] + dt * L[k];
    fv_dry(o, U1);
    real b2 = fv_operator(o, U1, o->t + dt, L);
    for (size_t k = 0; k < 9 * N; ++k) Un[k] = 0.5 * (Un[k] + U1[k] + dt * L[k]);
    fv_dry(o, Un);
    o->last_bflux = 0.5 * (b1 + b2);
    o->ledger += dt * 0.5 * (b1 + b2);
    o->t += dt;
}

/* One RK2 step of size dt: friction, [limit], stage 1, [limit], stage 2. */
void orc_step(orc_t *o, double dt)
{
    if (o->scheme != 0) {
        fv_step(o, dt);
        return;
    }
    const size_t N = (size_t)o->nx * o->ny;
    real *Un = o->U, *U1 = o->U1, *L = o->L;
    apply_friction(o, Un, dt);
    if (o->limiter) {
        apply_limiter(o, Un, o->Ls);
        memcpy(Un, o->Ls, 9 * N * sizeof(real));
    }
    real b1 = spatial_operator(o, Un, o->t, L);
#pragma omp parallel for schedule(static)
    for (size_t k = 0; k < 9 * N; ++k) U1[k] = Un[k] + dt * L[k];
    dry_reset(o, U1);
    if (o->limiter) {
        apply_limiter(o, U1, o->Ls);
        memcpy(U1, o->Ls, 9 * N * sizeof(real));
    }
    real b2 = spatial_operator(o, U1, o->t + dt, L);
#pragma omp parallel for schedule(static)
    for (size_t k = 0; k < 9 * N; ++k) Un[k] = 0.5 * (Un[k] + U1[k] + dt * L[k]);
    dry_reset(o, Un);
    o->last_bflux = 0.5 * (b1 + b2);
    o->ledger += dt * 0.5 * (b1 + b2);
    o->t += dt;
}

/* ------------------------------------------------------------------ */
/* Initialisation from corner data (Eq. 3 and the DEM rule of Sec. 2.1.1) */
/* ------------------------------------------------------------------ */

/* Modes of a field given at the (nx+1) x (ny+1) corner nodes: face-centre
 * values are averages of the two corners of each face, then Eq. 3. */
static void corner_modes(int nx, int ny, const double *f, real *m0, real *m1x, real *m1y)
{
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            const double *r0 = f + (size_t)j * (nx + 1), *r1 = f + (size_t)(j + 1) * (nx + 1);
            double fE = 0.5 * (r0[i + 1] + r1[i + 1]), fW = 0.5 * (r0[i] + r1[i]);
            double fN = 0.5 * (r1[i] + r1[i + 1]), fS = 0.5 * (r0[i] + r0[i + 1]);
            size_t c = (size_t)j * nx + i;
            m0[c] = 0.5 * (fE + fW);
            m1x[c] = 0.5 * (fE - fW);
            m1y[c] = 0.5 * (fN - fS);
        }
}

double orc_mass(const orc_t *o)
{
    const size_t N = (size_t)o->nx * o->ny;
    double s = 0.0;
    for (size_t c = 0; c < N; ++c) s += o->U[c];
    return s * o->dx * o->dy;
}

/* ------------------------------------------------------------------ */
/* Public entry points (ctypes)                                         */
/* ------------------------------------------------------------------ */

orc_t *orc_create(int nx, int ny, double dx, double dy, double g, double cfl, double tol_dry,
                  double ds_thresh, double dt_max, int limiter, const int *bc)
{
    if (nx < 1 || ny < 1) return NULL;
    orc_t *o = (orc_t *)calloc(1, sizeof(orc_t));
    size_t N = (size_t)nx * ny;
    o->nx = nx; o->ny = ny; o->dx = dx; o->dy = dy;
    o->g = g; o->cfl = cfl; o->tol_dry = tol_dry; o->ds_thresh = ds_thresh; o->dt_max = dt_max;
    o->limiter = limiter;
    o->wd = 1;
    for (int k = 0; k < 4; ++k) o->bc[k] = bc[k];
    o->z = (real *)calloc(3 * N, sizeof(real));
    o->nm = (real *)calloc(N, sizeof(real));
    o->U = (real *)calloc(9 * N, sizeof(real));
    o->U1 = (real *)calloc(9 * N, sizeof(real));
    o->L = (real *)calloc(9 * N, sizeof(real));
    o->Ls = (real *)calloc(9 * N, sizeof(real));
    o->bnd = (real *)calloc(2 * ((size_t)nx + ny), sizeof(real));
    return o;
}

void orc_destroy(orc_t *o)
{
    if (!o) return;
    free(o->z); free(o->nm); free(o->U); free(o->U1); free(o->L); free(o->Ls); free(o->bnd);
    free(o);
}

/* z_corner, eta_corner: (ny+1) x (nx+1) row-major corner nodes; eta_corner
 * NULL means dry.  manning: nx*ny per cell, or NULL for n_uniform. */
void orc_set_dem(orc_t *o, const double *z_corner, const double *manning, double n_uniform,
                 const double *eta_corner)
{
    int nx = o->nx, ny = o->ny;
    size_t N = (size_t)nx * ny, NC = (size_t)(nx + 1) * (ny + 1);
    corner_modes(nx, ny, z_corner, o->z, o->z + N, o->z + 2 * N);
    for (size_t c = 0; c < N; ++c) o->nm[c] = manning ? manning[c] : n_uniform;
    memset(o->U, 0, 9 * N * sizeof(real));
    if (eta_corner) {
        /* corner depths eta - z, left unclipped so the planar depth keeps the
         * free surface flat; a cell whose average depth is not positive is dry */
        double *hc = (double *)malloc(NC * sizeof(double));
        for (size_t k = 0; k < NC; ++k) hc[k] = eta_corner[k] - z_corner[k];
        corner_modes(nx, ny, hc, o->U, o->U + N, o->U + 2 * N);
        free(hc);
        for (size_t c = 0; c < N; ++c)
            if (o->U[c] <= 0.0) { o->U[c] = 0.0; o->U[N + c] = 0.0; o->U[2 * N + c] = 0.0; }
    }
    if (o->scheme != 0) {
        /* the FV schemes hold cell averages only (Eq. 3a) */
        for (int k = 0; k < 9; ++k)
            if (k % 3) memset(o->U + k * N, 0, N * sizeof(real));
    }
    o->t = 0.0;
    o->ledger = orc_mass(o);
}

int orc_add_inflow(orc_t *o, int edge, double s0, double len, const double *tk, const double *qk,
                   int nk)
{
    if (o->n_in >= MAX_INFLOW || nk < 1 || nk > MAX_KNOTS) return -1;
    inflow_t *f = &o->in[o->n_in++];
    f->edge = edge; f->s0 = s0; f->len = len; f->nk = nk;
    for (int k = 0; k < nk; ++k) { f->tk[k] = tk[k]; f->qk[k] = qk[k]; }
    return 0;
}

void orc_set_sources(orc_t *o, double rain, double t0, double t1, double px, double py, double qp)
{
    o->rain = rain; o->rain_t0 = t0; o->rain_t1 = t1;
    o->px = px; o->py = py; o->qp = qp;
}

/* Copies between the caller's double arrays and the oracle's `real` arrays. */
static void to_double(double *dst, const real *src, size_t n)
{
    for (size_t k = 0; k < n; ++k) dst[k] = src[k];
}

static real *from_double(const double *src, size_t n)
{
    real *dst = (real *)calloc(n, sizeof(real));
    for (size_t k = 0; k < n; ++k) dst[k] = src[k];
    return dst;
}

void orc_get_state(const orc_t *o, double *planes, double *t)
{
    to_double(planes, o->U, 9 * (size_t)o->nx * o->ny);
    if (t) *t = o->t;
}

void orc_set_state(orc_t *o, const double *planes, double t)
{
    for (size_t k = 0; k < 9 * (size_t)o->nx * o->ny; ++k) o->U[k] = planes[k];
    o->t = t;
    o->ledger = orc_mass(o);
}

void orc_get_topo(const orc_t *o, double *planes3)
{
    to_double(planes3, o->z, 3 * (size_t)o->nx * o->ny);
}

double orc_time(const orc_t *o) { return o->t; }
double orc_ledger(const orc_t *o) { return o->ledger; }

/* Exposed pieces for the pin tests. */
double orc_operator(orc_t *o, const double *U, double t, double *Lout)
{
    const size_t n = 9 * (size_t)o->nx * o->ny;
    real *u = from_double(U, n), *l = (real *)calloc(n, sizeof(real));
    double b = spatial_operator(o, u, t, l);
    to_double(Lout, l, n);
    free(u);
    free(l);
    return b;
}

void orc_friction(orc_t *o, double *U, double dt)
{
    const size_t n = 9 * (size_t)o->nx * o->ny;
    real *u = from_double(U, n);
    apply_friction(o, u, dt);
    to_double(U, u, n);
    free(u);
}

void orc_limit(const orc_t *o, const double *Uin, double *Uout)
{
    const size_t n = 9 * (size_t)o->nx * o->ny;
    real *u = from_double(Uin, n), *v = (real *)calloc(n, sizeof(real));
    apply_limiter(o, u, v);
    to_double(Uout, v, n);
    free(u);
    free(v);
}
void orc_hll(const orc_t *o, int dir, const double *l3, const double *r3, double *f3)
{
    st3 a = mk(l3[0], l3[1], l3[2]), b = mk(r3[0], r3[1], r3[2]);
    st3 f = dir == 0 ? riemann_x(o, a, b) : hll_y(o, a, b);
    f3[0] = f.h; f3[1] = f.qx; f3[2] = f.qy;
}
double orc_minmod(double a, double b, double c) { return minmod3(a, b, c); }
/* Riemann solver of the run: 0 HLL (default), 1 Roe. */
void orc_set_flux(orc_t *o, int flux) { o->flux = flux; }
/* Scheme of the run: 0 DG2 (default), 1 MUSCL-FV2, 2 FV1 (set before orc_set_dem). */
void orc_set_scheme(orc_t *o, int scheme) { o->scheme = scheme; }
void orc_set_wetdry(orc_t *o, int wd) { o->wd = wd; }

/* Threads of the rows-parallel loops: effective only in a build with OpenMP
 * (the results are the same for any count); returns the count in use. */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* Depth at (x, y) from the planar solution of the containing cell, clipped at 0. */
double orc_gauge_h(const orc_t *o, double x, double y)
{
    int i = (int)floor(x / o->dx), j = (int)floor(y / o->dy);
    if (i < 0) i = 0;
    if (i >= o->nx) i = o->nx - 1;
    if (j < 0) j = 0;
    if (j >= o->ny) j = o->ny - 1;
    size_t N = (size_t)o->nx * o->ny, c = (size_t)j * o->nx + i;
    double xi = (x - (i + 0.5) * o->dx) / (0.5 * o->dx), et = (y - (j + 0.5) * o->dy) / (0.5 * o->dy);
    double h = o->U[c] + xi * o->U[N + c] + et * o->U[2 * N + c];
    return h > 0.0 ? h : 0.0;
}

/* Advances to t_end with CFL steps, landing exactly on every multiple of
 * sample_every (if > 0) and on t_end; records gauge depths at each landing.
 * Returns the number of steps; writes at most cap samples. */
long orc_run_to(orc_t *o, double t_end, double sample_every, int ngauge, const double *gxy,
                double *t_out, double *h_out, int cap, int *nsamp)
{
    long steps = 0;
    int ns = 0;
    double next = sample_every > 0.0 ? (floor(o->t / sample_every + 1e-9) + 1.0) * sample_every : 0.0;
    while (o->t < t_end) {
        double dt = orc_cfl_dt(o);
        double target = t_end;
        int at_sample = 0;
        if (sample_every > 0.0 && next <= t_end) { target = next; at_sample = 1; }
        int land = 0;
        if (o->t + dt >= target) { dt = target - o->t; land = 1; }
        orc_step(o, dt);
        if (land) o->t = target;
        ++steps;
        if (land && at_sample) {
            if (ns < cap) {
                t_out[ns] = o->t;
                for (int k = 0; k < ngauge; ++k)
                    h_out[(size_t)ns * ngauge + k] = orc_gauge_h(o, gxy[2 * k], gxy[2 * k + 1]);
            }
            ++ns;
            next += sample_every;
        }
    }
    if (nsamp) *nsamp = ns;
    return steps;
}
