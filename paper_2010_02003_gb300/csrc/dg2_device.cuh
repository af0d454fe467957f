// dg2_device.cuh -- device code of the GB300 DG2 solver (sm_103a).
//
// One RK2 step of the slope-decoupled DG2 scheme (Sec. 2.1 of Ayog et al.)
// is three launches on the caller's stream:
//   friction_kernel   implicit Manning friction at the centre and the four
//                     Gauss points of every cell (Sec. 2.1.3), in place;
//   stage_kernel<1>   [local limiting, Eqs. 6-7] + spatial operator
//                     (Eqs. 4-5) + U1 = Un + dt L(Un) + wet-dry treatment;
//   stage_kernel<2>   [limiting] + operator + Un+1 = (Un + U1 + dt L(U1)) / 2
//                     + wet-dry treatment, then the Courant-number reduction
//                     for the next step; its last block to finish advances t,
//                     the mass ledger and the gauges (no host round trip).
//
// Layout: structure of arrays, one FP64 plane per coefficient, row pitch a
// multiple of 32 elements.  A block owns a TX x TY tile of cells; it computes
// every revised face limit once (Sec. 2.1.2), keeps the east/north limits in
// shared memory so each interior face flux is evaluated once per tile, and
// evaluates the halo limits (and ghost states on domain edges) itself.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dg2 {

// FP64 tile of TX x TY cells.  Measured on GB300 with the weight-class lists
// (floodplain 2000 x 1000 from t = 1 h, ms per step, 32 -> 16 wide): DG2-LL
// 0.421 -> 0.422, DG2-NL 0.345 -> 0.335; 32 x 8 is kept.
#ifndef DG2_TX64
#define DG2_TX64 32
#endif
constexpr int TX = DG2_TX64;
constexpr int TY = 8;

// A warp of the FP64 tile kernels covers a WX x WY block of cells (lane l:
// column l % WX, row l / WX of the block); a 32 x 8 tile is 4 x 2 such blocks,
// warp w the block (w % 4, w / 4).  Wet regions are compact, so square-ish
// blocks hold fewer dry lanes than rows of 32.  The tile cell of the calling
// thread:
constexpr int WX = 8, WY = 4, TBX = TX / WX, TBY = TY / WY;
static_assert(WX * WY == 32 && TBX * WX == TX && TBY * WY == TY, "warp blocks tile the tile");
__device__ __forceinline__ void warp_cell(int& tx, int& ty) {
  const int t = threadIdx.y * TX + threadIdx.x, w = t >> 5, l = t & 31;
  tx = (w % TBX) * WX + (l % WX);
  ty = (w / TBX) * WY + (l / WX);
}

constexpr int kMaxInflow = 8;
constexpr int kMaxGauges = 256;

// Plane indices of the 9 flow coefficients (Eq. 2): variable * 3 + mode.
enum { H0 = 0, H1X, H1Y, QX0, QX1X, QX1Y, QY0, QY1X, QY1Y };

struct InflowDesc {
  int edge;        // 0 W, 1 E, 2 S, 3 N
  int nk;          // knots
  int koff;        // offset into the knot arrays
  int nfaces;      // faces whose centre lies in the segment
  double s0, s1;   // segment [s0, s1] along the edge
  double width;    // nfaces * face length
};

// The step's list of computed tiles is kept in kListClasses weight classes, by
// the count of non-quiescent cells of each tile when the list is built
// (heaviest class first), so the blocks of long tiles start first and short
// ones fill the end of a stage.  The order of the entries does not change the
// result (lists_kernel).
#ifndef DG2_LIST_CLASSES
#define DG2_LIST_CLASSES 8
#endif
constexpr int kListClasses = DG2_LIST_CLASSES;

// Device-resident scalars of a context (one per context, in the workspace).
struct Scalars {
  double t;            // simulated time
  double dt;           // step size of the next step (capped)
  double dt_cfl;       // Courant-number step of the current state (uncapped)
  double t_end;        // run_to target (+inf outside run_to)
  double next_sample;  // next gauge sample time (+inf if none)
  double sample_every;
  double ledger;       // initial mass + boundary / source volumes
  double mass;         // last dg2_mass result
  unsigned long long lam_bits;  // max wave speed / cell size, as FP64 bits
  unsigned int count;  // blocks finished (last-block-done pattern)
  int done;            // t reached t_end during run_to
  int land;            // the capped dt lands exactly on the target
  int fixed_dt;        // dg2_step with a caller-forced dt: no landing logic
  int nonfinite;       // a non-finite value or h0 < -1 appeared
  int nsamp;           // samples recorded (may exceed capacity)
  int ledger_init;     // mass kernel: also reset the ledger
  int pad;
  long long steps;     // completed steps (count of stage-2 finalisations)
  double last_dt;      // size of the last completed step
  int n_act;           // tiles computed in the current step (entries of tiles.list)
  int n_b[kListClasses];  // of these, the entries of each weight class
  int n_front;         // frontier tiles copied in stage 1 (entries of tiles.front)
  int list_all;        // every tile is computed: list entry e is tile e
  int skip_lists;      // the step was not taken (run already done): keep the lists
  long long tiles_done;  // tiles computed by the stage kernels of all completed steps
};

// Exact skipping of quiescent dry tiles.  A cell is quiescent when its depth
// average is at or below tol_dry and every other mode is zero (FP64 form) or
// its free-surface slopes equal the topography slopes and its discharges are
// zero (FP32 form) -- the state the wet-dry treatment leaves in dry cells.  A
// quiescent cell whose neighbours are quiescent is a fixed point of a stage:
// every face between dry limits carries zero flux, the depth modes do not
// change and the treatment re-zeroes the discharges.  Water moves at most one
// cell per stage (Courant number < 1), two per step, fewer than a 32 x 8 tile,
// so a tile whose 3 x 3 tile neighbourhood holds no non-quiescent or forced
// (inflow, point source, rain) tile is left untouched, bit for bit as if it
// had been computed.
//
// The FP64 DG2 stage kernels refine this to single cells of a computed tile.
// Each stage records, one bit per cell, which cells of its output are
// non-quiescent (qm: plane 0 for Un, written by stage 2; plane 1 for U1,
// written by stage 1).  A cell whose input and four face neighbours are
// quiescent is a fixed point of the stage (a dry cell's limited slopes are its
// own, so the records of a quiescent cell depend on it alone, in DG2-LL too):
// stage 1 copies it to U1, stage 2 leaves Un as it is when the cell was also a
// fixed point of stage 1 (qm plane 2 holds stage 1's computed cells).  The
// computed cells of a tile are handed to the first threads (classify_cells),
// records and faces are evaluated only where a computed cell uses them, and
// friction skips 8 x 4 warp blocks of quiescent cells.  Forced tiles, rain and
// skip = 0 compute every cell.
struct Tiles {
  unsigned char* flag;          // [ntiles] tile held a non-quiescent cell after the last stage 2
  unsigned char* act;           // [ntiles] tile computed in the current step
  const unsigned char* forced;  // [ntiles] tile must be computed (inflow, source); set on the host
  int* list;                    // [kListClasses * ntiles] computed tiles of the step, by weight class
  int* front;                   // [ntiles] frontier tiles of the step (stage-1 copy), ascending
  int ntx, nty, ntiles;         // tile grid
  int all_forced;               // every tile must be computed (rain)
  int skip;                     // 0: compute every tile
};

// Tile of entry e of the step's list: the weight classes' entries in turn.
template <class S>
__device__ __forceinline__ int list_tile(const Tiles& T, const S* sc, int e) {
  int k = 0;
  for (; k < kListClasses - 1; ++k) {
    const int n = sc->n_b[k];
    if (e < n) break;
    e -= n;
  }
  return T.list[k * T.ntiles + e];
}

struct Dev {
  // grid
  int nx, ny, pitch;
  long long plane;           // elements per plane
  double dx, dy, inv_dx, inv_dy;
  // parameters
  double g, cfl, tol, ds, dt_max;
  int bc[4];
  int flux;                  // 0 HLL, 1 Roe
  int scheme;                // 0 DG2, 1 MUSCL-FV2, 2 FV1 (Sec. 2.2)
  int wd;                    // 1: positivity-consistent revision of partially wet cells
  // inflows
  int n_in;
  InflowDesc in[kMaxInflow];
  const double* knot_t;
  const double* knot_q;
  // sources
  double rain, rain_t0, rain_t1;
  double qp;                 // point inflow, m^3/s
  long long src_idx;         // plane index of the point-source cell, -1 if none
  // buffers
  double* S;                 // 9 planes: state Un
  double* T;                 // 9 planes: stage state U1
  double* Q;                 // 6 planes: limited slopes of Un (DG2-LL)
  const double* Z;           // 3 planes: z0, z1x, z1y
  const double* N;           // 1 plane: Manning n
  double* bpart;             // [2][nblocks] boundary mass-rate partials
  double* mpart;             // [nblocks] mass partials
  Scalars* sc;
  // gauges
  int ngauge, max_samples;
  const long long* g_idx;    // plane index of each gauge cell
  const double* g_xi;        // local coordinates in [-1, 1]
  const double* g_eta;
  double* samp_t;            // [max_samples]
  double* samp_h;            // [max_samples][ngauge]
  int nblocks;               // blocks of the stage grid
  Tiles tiles;
  // FP64 DG2 cell skipping: [3][nby][nbx] words, one per 8 x 4 warp block (bit l
  // of word (Y, X): cell (8 X + l % 8, 4 Y + l / 8)): the non-quiescence of Un
  // (plane 0, written by stage 2) and of U1 (plane 1, by stage 1), and the
  // cells stage 1 computed (plane 2)
  unsigned int* qm;
  int nbx, nby;              // warp blocks per row / column (whole tiles)
  long long qplane;          // words per qm plane
};

// ---------------------------------------------------------------------------
// FP64 comparisons on the integer units
// ---------------------------------------------------------------------------
// GB300 runs every FP64 instruction, comparisons and min / max included, on a
// pipe 64 times narrower than FP32, and the FP64 stage kernels are bound by
// it.  Comparisons against zero and against a non-negative constant are taken
// on the IEEE bit patterns instead, which order like the values: for x not a
// NaN, x > 0 exactly when the pattern read as int64 is positive, x < 0 when
// it is above the -0 pattern read as uint64, and, for c >= +0, x > c exactly
// when bits(x) > bits(c) as int64.  A comparison of two values of any sign
// uses the key (magnitude, negated for a set sign bit), which ranks -0 and +0
// equal.  Every result equals the IEEE comparison for non-NaN operands.
__device__ __forceinline__ long long fbits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ bool is_pos(double x) { return fbits(x) > 0; }  // x > 0
__device__ __forceinline__ bool is_neg(double x) {                        // x < 0
  return (unsigned long long)fbits(x) > 0x8000000000000000ull;
}
// x > c for c >= +0
__device__ __forceinline__ bool above(double x, double c) { return fbits(x) > fbits(c); }
__device__ __forceinline__ double pos_part(double x) { return is_pos(x) ? x : 0.0; }  // max(x, 0)
__device__ __forceinline__ long long order_key(double x) {
  const long long b = fbits(x), m = b & 0x7fffffffffffffffll;
  return b < 0 ? -m : m;
}
__device__ __forceinline__ bool gt(double a, double b) { return order_key(a) > order_key(b); }
__device__ __forceinline__ double min2(double a, double b) { return gt(a, b) ? b : a; }
__device__ __forceinline__ double max2(double a, double b) { return gt(b, a) ? b : a; }
// comparisons of values known non-negative (sign bit clear or +0 after fabs)
__device__ __forceinline__ double max_nn(double a, double b) { return fbits(b) > fbits(a) ? b : a; }
__device__ __forceinline__ double min_nn(double a, double b) { return fbits(b) < fbits(a) ? b : a; }
// x != 0 (either zero)
__device__ __forceinline__ bool nonzero(double x) { return (fbits(x) << 1) != 0; }

// ---------------------------------------------------------------------------
// Point-state helpers
// ---------------------------------------------------------------------------

// A revised face limit (Sec. 2.1.2): h* = max(0, h), velocities q/h above
// tol_dry and zero otherwise, q* = h* u.  The velocities are kept for the flux.
struct Lim {
  double h, qx, qy, u, v;
};

struct F3 {
  double h, x, y;
};

__device__ __forceinline__ Lim revise(double h, double qx, double qy, double tol) {
  Lim r;
  if (above(h, tol)) {
    const double ih = 1.0 / h;
    r.u = qx * ih;
    r.v = qy * ih;
  } else {
    r.u = 0.0;
    r.v = 0.0;
  }
  r.h = pos_part(h);
  r.qx = r.h * r.u;
  r.qy = r.h * r.v;
  return r;
}

// HLL flux normal to a face (Toro's wave-speed estimates with the dry-bed
// forms).  n = normal, t = tangential component; (un, ut) are the limit's
// velocities.  Returns (mass, normal momentum, tangential momentum).
__device__ __forceinline__ F3 hll(double hL, double qnL, double qtL, double unL, double utL,
                                  double hR, double qnR, double qtR, double unR, double utR,
                                  double g, double tol) {
  F3 f;
  const bool dL = !above(hL, tol), dR = !above(hR, tol);
  if (dL && dR) {
    f.h = 0.0; f.x = 0.0; f.y = 0.0;
    return f;
  }
  const double cL = sqrt(g * hL), cR = sqrt(g * hR);
  double sL, sR;
  if (dL) {
    sL = unR - 2.0 * cR;
    sR = unR + cR;
  } else if (dR) {
    sL = unL - cL;
    sR = unL + 2.0 * cL;
  } else {
    const double us = 0.5 * (unL + unR) + cL - cR;
    const double cs = 0.5 * (cL + cR) + 0.25 * (unL - unR);
    sL = min2(unL - cL, us - cs);
    sR = max2(unR + cR, us + cs);
  }
  // physical normal flux [h un, h un^2 + g h^2 / 2, h un ut] of each side
  const double fLh = hL * unL, fLn = hL * unL * unL + 0.5 * g * hL * hL, fLt = hL * unL * utL;
  const double fRh = hR * unR, fRn = hR * unR * unR + 0.5 * g * hR * hR, fRt = hR * unR * utR;
  if (!is_neg(sL)) {
    f.h = fLh; f.x = fLn; f.y = fLt;
    return f;
  }
  if (!is_pos(sR)) {
    f.h = fRh; f.x = fRn; f.y = fRt;
    return f;
  }
  const double inv = 1.0 / (sR - sL), sLR = sL * sR;
  f.h = (sR * fLh - sL * fRh + sLR * (hR - hL)) * inv;
  f.x = (sR * fLn - sL * fRn + sLR * (qnR - qnL)) * inv;
  f.y = (sR * fLt - sL * fRt + sLR * (qtR - qtL)) * inv;
  return f;
}

// |lam| with Harten's entropy fix: (lam^2 + d^2) / (2 d) below d = max(0,
// lam - lamL, lamR - lam), the spread of the characteristic speeds at the face.
__device__ __forceinline__ double harten(double lam, double lamL, double lamR) {
  double d = lam - lamL;
  if (lamR - lam > d) d = lamR - lam;
  if (d < 0.0) d = 0.0;
  double a = fabs(lam);
  if (a < d) a = (lam * lam + d * d) / (2.0 * d);
  return a;
}

// Roe flux normal to a face (Sec. 2.1.2 names Roe's solver): the average of
// the physical fluxes minus the upwinding of the waves of the Roe-linearised
// system (Roe averages, eigenvalues u^ -+ c^ and u^, wave strengths
// (dh -+ h^ du / c^) / 2 and h^ dt), Harten's entropy fix on the acoustic waves.
__device__ __forceinline__ F3 roe(double hL, double qnL, double qtL, double unL, double utL,
                                  double hR, double qnR, double qtR, double unR, double utR,
                                  double g, double tol) {
  F3 f;
  if (hL <= tol && hR <= tol) {
    f.h = 0.0; f.x = 0.0; f.y = 0.0;
    return f;
  }
  const double sL = sqrt(hL), sR = sqrt(hR);
  const double isum = 1.0 / (sL + sR);
  const double uh = (sL * unL + sR * unR) * isum;
  const double vh = (sL * utL + sR * utR) * isum;
  const double hh = sL * sR;
  const double ch = sqrt(0.5 * g * (hL + hR));
  const double dh = hR - hL, du = unR - unL, dv = utR - utL;
  const double a1 = 0.5 * (dh - hh * du / ch), a2 = hh * dv, a3 = 0.5 * (dh + hh * du / ch);
  const double l1 = uh - ch, l3 = uh + ch;
  const double cL = sqrt(g * hL), cR = sqrt(g * hR);
  const double e1 = harten(l1, unL - cL, unR - cR), e2 = fabs(uh);
  const double e3 = harten(l3, unL + cL, unR + cR);
  const double w1 = e1 * a1, w2 = e2 * a2, w3 = e3 * a3;
  const double fLh = hL * unL, fLn = hL * unL * unL + 0.5 * g * hL * hL, fLt = hL * unL * utL;
  const double fRh = hR * unR, fRn = hR * unR * unR + 0.5 * g * hR * hR, fRt = hR * unR * utR;
  f.h = 0.5 * (fLh + fRh) - 0.5 * (w1 + w3);
  f.x = 0.5 * (fLn + fRn) - 0.5 * (w1 * l1 + w3 * l3);
  f.y = 0.5 * (fLt + fRt) - 0.5 * (w1 * vh + w2 + w3 * vh);
  return f;
}

// x-face flux: returns [F^h, F^qx, F^qy].
__device__ __forceinline__ F3 flux_x(const Lim& L, const Lim& R, double g, double tol,
                                     int flux = 0) {
  if (flux == 1) return roe(L.h, L.qx, L.qy, L.u, L.v, R.h, R.qx, R.qy, R.u, R.v, g, tol);
  return hll(L.h, L.qx, L.qy, L.u, L.v, R.h, R.qx, R.qy, R.u, R.v, g, tol);
}

// y-face flux in the rotated frame, mapped back: returns [G^h, G^qx, G^qy].
__device__ __forceinline__ F3 flux_y(const Lim& S, const Lim& N, double g, double tol,
                                     int flux = 0) {
  F3 r = flux == 1 ? roe(S.h, S.qy, S.qx, S.v, S.u, N.h, N.qy, N.qx, N.v, N.u, g, tol)
                   : hll(S.h, S.qy, S.qx, S.v, S.u, N.h, N.qy, N.qx, N.v, N.u, g, tol);
  F3 o;
  o.h = r.h; o.x = r.y; o.y = r.x;
  return o;
}

// Face flux along x or y by a run-time flag: the normal and tangential
// components selected, so a warp holding both kinds of faces evaluates one flux
// (the same arithmetic as flux_x / flux_y).
__device__ __forceinline__ F3 flux_dir(const Lim& A, const Lim& B, bool ydir, double g, double tol,
                                       int flux) {
  const double an = ydir ? A.qy : A.qx, at = ydir ? A.qx : A.qy;
  const double aun = ydir ? A.v : A.u, aut = ydir ? A.u : A.v;
  const double bn = ydir ? B.qy : B.qx, bt = ydir ? B.qx : B.qy;
  const double bun = ydir ? B.v : B.u, but = ydir ? B.u : B.v;
  const F3 r = flux == 1 ? roe(A.h, an, at, aun, aut, B.h, bn, bt, bun, but, g, tol)
                         : hll(A.h, an, at, aun, aut, B.h, bn, bt, bun, but, g, tol);
  F3 o;
  o.h = r.h;
  o.x = ydir ? r.y : r.x;
  o.y = ydir ? r.x : r.y;
  return o;
}

// Physical flux F (x) or G (y) of a point state, velocities by the tol rule.
__device__ __forceinline__ F3 phys_flux(double h, double qx, double qy, double g, double tol,
                                        bool ydir) {
  double u = 0.0, v = 0.0;
  if (above(h, tol)) {
    const double ih = 1.0 / h;
    u = qx * ih;
    v = qy * ih;
  }
  F3 f;
  const double p = 0.5 * g * h * h;
  if (!ydir) {
    f.h = h * u; f.x = h * u * u + p; f.y = h * u * v;
  } else {
    f.h = h * v; f.x = h * u * v; f.y = h * v * v + p;
  }
  return f;
}

// ---------------------------------------------------------------------------
// Boundary ghosts
// ---------------------------------------------------------------------------

static __device__ double hydrograph(const Dev& d, const InflowDesc& f, double t) {
  const double* tk = d.knot_t + f.koff;
  const double* qk = d.knot_q + f.koff;
  if (t <= tk[0]) return qk[0];
  for (int k = 0; k + 1 < f.nk; ++k) {
    if (t <= tk[k + 1]) {
      const double w = (t - tk[k]) / (tk[k + 1] - tk[k]);
      return qk[k] + w * (qk[k + 1] - qk[k]);
    }
  }
  return qk[f.nk - 1];
}

// Outside state at a face of `edge` whose centre has edge coordinate s,
// built from the cell's own unrevised limit (h, qx, qy).
static __device__ void ghost(const Dev& d, int edge, double s, double t, double& h, double& qx,
                      double& qy) {
  for (int k = 0; k < d.n_in; ++k) {
    const InflowDesc& f = d.in[k];
    if (f.edge != edge || s < f.s0 || s > f.s1) continue;
    const double qin = hydrograph(d, f, t) / f.width;
    const double hin = h > 0.0 ? h : 0.0;
    const double hc = cbrt(qin * qin / d.g);
    const double hg = hin > hc ? hin : hc;
    const double qn = (edge == 0 || edge == 2) ? qin : -qin;
    h = hg;
    if (edge <= 1) { qx = qn; qy = 0.0; } else { qx = 0.0; qy = qn; }
    return;
  }
  if (d.bc[edge] == 1) {
    // free outflow: copy, without an inward normal discharge
    if (edge == 0 && qx > 0.0) qx = 0.0;
    if (edge == 1 && qx < 0.0) qx = 0.0;
    if (edge == 2 && qy > 0.0) qy = 0.0;
    if (edge == 3 && qy < 0.0) qy = 0.0;
    return;
  }
  if (edge <= 1) qx = -qx; else qy = -qy;  // wall
}

// ---------------------------------------------------------------------------
// Local limiting (Eqs. 6-7)
// ---------------------------------------------------------------------------

__device__ __forceinline__ double minmod3(double a, double b, double c) {
  // same-signed operands: the bit patterns order the magnitudes
  if (is_pos(a) && is_pos(b) && is_pos(c)) return min_nn(min_nn(a, b), c);
  if (is_neg(a) && is_neg(b) && is_neg(c)) {
    const double m = fbits(b) < fbits(a) ? b : a;  // the smaller magnitude
    return fbits(c) < fbits(m) ? c : m;
  }
  return 0.0;
}

// Detector (Eq. 6, tested as J > thresh * den, the magnitude in den floored at
// tol_dry) and generalised minmod (Eq. 7) for one component along one direction.
__device__ __forceinline__ double limit_component(double thresh, double tol, double half,
                                                  double k0w, double k1w, double k0, double k1,
                                                  double k0e, double k1e) {
  // k1 / sqrt(3) as a product with 1 / sqrt(3) rounded to nearest (one FP64
  // division fewer per component; within an ulp of the quotient)
  const double q = k1 * 0.57735026918962576;
  const double jE = fabs((k0e - k1e) - (k0 + k1));
  const double jW = fabs((k0 - k1) - (k0w + k1w));
  // max(|k0 - q|, |k0 + q|) = |k0| + |q|: the larger is the one whose terms
  // share a sign, a sum of magnitudes, rounded alike
  double mag = fabs(k0) + fabs(q);
  if (fbits(mag) < fbits(tol)) mag = tol;  // still water: round-off never counts as a shock
  const double den = half * mag;
  const double jm = max_nn(jE, jW);
  if (!gt(jm, thresh * den)) return k1;
  return minmod3(k1, k0e - k0, k0 - k0w);
}

// Slopes (h, qx, qy) of cell (i, j) along `dir` (1 = x, 2 = y) from buffer U,
// limited by Eqs. 6-7 when the cell and both neighbours are wet and the cell
// is not on the edge normal to `dir`; eta = h + z is limited instead of h.
static __device__ void limited_slopes(const Dev& d, const double* __restrict__ U, int i, int j, int dir,
                               double& sh, double& sqx, double& sqy) {
  const long long P = d.plane;
  const long long c = (long long)j * d.pitch + i;
  sh = U[(dir)*P + c];
  sqx = U[(3 + dir) * P + c];
  sqy = U[(6 + dir) * P + c];
  const bool lo = dir == 1 ? i > 0 : j > 0;
  const bool hi = dir == 1 ? i + 1 < d.nx : j + 1 < d.ny;
  if (!lo || !hi) return;
  const long long cl = dir == 1 ? c - 1 : c - d.pitch;
  const long long ch = dir == 1 ? c + 1 : c + d.pitch;
  const double hl = U[cl], hc = U[c], hh = U[ch];
  if (!above(hl, d.tol) || !above(hc, d.tol) || !above(hh, d.tol)) return;
  const double half = 0.5 * (dir == 1 ? d.dx : d.dy);
  const double* z0 = d.Z;
  const double* z1 = d.Z + dir * P;
  const double e1c = sh + z1[c];
  const double e1 = limit_component(d.ds, d.tol, half, hl + z0[cl], U[dir * P + cl] + z1[cl],
                                    hc + z0[c], e1c, hh + z0[ch], U[dir * P + ch] + z1[ch]);
  if (e1 != e1c) sh = e1 - z1[c];
  {
    const double* k0 = U + 3 * P;
    const double* k1 = U + (3 + dir) * P;
    sqx = limit_component(d.ds, d.tol, half, k0[cl], k1[cl], k0[c], k1[c], k0[ch], k1[ch]);
  }
  {
    const double* k0 = U + 6 * P;
    const double* k1 = U + (6 + dir) * P;
    sqy = limit_component(d.ds, d.tol, half, k0[cl], k1[cl], k0[c], k1[c], k0[ch], k1[ch]);
  }
}

// ---------------------------------------------------------------------------
// Wet-dry treatment after each stage (mass-neutral; averages untouched)
// ---------------------------------------------------------------------------

__device__ __forceinline__ void wetdry(double* m, double z0, double z1x, double z1y, double tol) {
  const double h0 = m[H0];
  if (!above(h0, tol)) {
#pragma unroll
    for (int k = 1; k < 9; ++k) m[k] = 0.0;
    return;
  }
  const double eta0 = h0 + z0;
  // x direction
  {
    const bool fe = !above(h0 + m[H1X], tol) && !gt(z0 + z1x, eta0);
    const bool fw = !above(h0 - m[H1X], tol) && !gt(z0 - z1x, eta0);
    if (fe || fw) { m[H1X] = 0.0; m[QX1X] = 0.0; m[QY1X] = 0.0; }
  }
  {
    const bool fn = !above(h0 + m[H1Y], tol) && !gt(z0 + z1y, eta0);
    const bool fs = !above(h0 - m[H1Y], tol) && !gt(z0 - z1y, eta0);
    if (fn || fs) { m[H1Y] = 0.0; m[QX1Y] = 0.0; m[QY1Y] = 0.0; }
  }
}

// ---------------------------------------------------------------------------
// Block reductions
// ---------------------------------------------------------------------------

template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh) {
  const int lane = (threadIdx.y * blockDim.x + threadIdx.x) & 31;
  const int warp = (threadIdx.y * blockDim.x + threadIdx.x) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double r = 0.0;
  if (warp == 0) {
    r = lane < NT / 32 ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
  }
  return r;  // valid in thread 0
}

template <int NT>
__device__ __forceinline__ double block_max(double v, double* sh) {
  const int lane = (threadIdx.y * blockDim.x + threadIdx.x) & 31;
  const int warp = (threadIdx.y * blockDim.x + threadIdx.x) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double r = 0.0;
  if (warp == 0) {
    r = lane < NT / 32 ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_down_sync(0xffffffffu, r, o));
  }
  return r;
}

template <int NT>
__device__ __forceinline__ float block_max_f(float v, float* sh) {
  const int lane = (threadIdx.y * blockDim.x + threadIdx.x) & 31;
  const int warp = (threadIdx.y * blockDim.x + threadIdx.x) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  float r = 0.f;
  if (warp == 0) {
    r = lane < NT / 32 ? sh[lane] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r = fmaxf(r, __shfl_down_sync(0xffffffffu, r, o));
  }
  return r;
}

// Courant wave-speed rate of a cell: max((|u|+c)/dx, (|v|+c)/dy) if wet.
__device__ __forceinline__ double cell_rate(const Dev& d, double h0, double qx0, double qy0) {
  if (!above(h0, d.tol)) return 0.0;
  const double ih = 1.0 / h0;
  const double u = qx0 * ih, v = qy0 * ih, c = sqrt(d.g * h0);
  return max_nn((fabs(u) + c) * d.inv_dx, (fabs(v) + c) * d.inv_dy);
}

// Turns the reduced rate into the next step: Courant step (capped by dt_max,
// dt_max if nothing is wet) then capped to land on the next target time.
static __device__ void schedule_next_dt(const Dev& d, Scalars* sc, double lam) {
  double dt = d.dt_max;
  if (lam > 0.0) {
    dt = d.cfl / lam;
    if (dt > d.dt_max) dt = d.dt_max;
  }
  sc->dt_cfl = dt;
  sc->land = 0;
  if (!sc->fixed_dt) {
    double target = sc->t_end;
    if (sc->next_sample <= target) target = sc->next_sample;
    if (sc->t + dt >= target) {
      dt = target - sc->t;
      sc->land = 1;
    }
  }
  sc->dt = dt;
  sc->lam_bits = 0ull;
}

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------

// Initial modes from corner data (Eq. 3): corners staged in `zc` / `ec`
// ((ny+1) x (nx+1) dense); ec == nullptr for a dry start; man == nullptr for
// the uniform n.
static __global__ void init_kernel(Dev d, const double* __restrict__ zc, const double* __restrict__ ec,
                            const double* __restrict__ man, double n_uniform, double* Zw,
                            double* Nw) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= d.nx || j >= d.ny) return;
  const long long P = d.plane, c = (long long)j * d.pitch + i;
  const int W = d.nx + 1;
  const double* r0 = zc + (long long)j * W;
  const double* r1 = zc + (long long)(j + 1) * W;
  {
    const double fE = 0.5 * (r0[i + 1] + r1[i + 1]), fW = 0.5 * (r0[i] + r1[i]);
    const double fN = 0.5 * (r1[i] + r1[i + 1]), fS = 0.5 * (r0[i] + r0[i + 1]);
    Zw[c] = 0.5 * (fE + fW);
    Zw[P + c] = 0.5 * (fE - fW);
    Zw[2 * P + c] = 0.5 * (fN - fS);
  }
  double h0 = 0.0, h1x = 0.0, h1y = 0.0;
  if (ec) {
    const double* e0 = ec + (long long)j * W;
    const double* e1 = ec + (long long)(j + 1) * W;
    const double a = e0[i] - r0[i], b = e0[i + 1] - r0[i + 1];
    const double cc = e1[i] - r1[i], dd = e1[i + 1] - r1[i + 1];
    const double fE = 0.5 * (b + dd), fW = 0.5 * (a + cc);
    const double fN = 0.5 * (cc + dd), fS = 0.5 * (a + b);
    h0 = 0.5 * (fE + fW);
    h1x = 0.5 * (fE - fW);
    h1y = 0.5 * (fN - fS);
    if (h0 <= 0.0) { h0 = 0.0; h1x = 0.0; h1y = 0.0; }
    if (d.scheme != 0) { h1x = 0.0; h1y = 0.0; }  // the FV schemes hold averages only
  }
  double* S = d.S;
  S[H0 * P + c] = h0;
  S[H1X * P + c] = h1x;
  S[H1Y * P + c] = h1y;
#pragma unroll
  for (int k = 3; k < 9; ++k) S[k * P + c] = 0.0;
  Nw[c] = man ? man[(long long)j * d.nx + i] : n_uniform;
}

// Point-implicit friction (Sec. 2.1.3) at one point: q /= 1 + dt g n^2 |q| / h^(7/3).
// h^(-7/3) for h in (1e-30, 1e30): the inverse cube root r = h^(-1/3) by two
// Newton steps on f(r) = r^-3 - h, r <- r + r (1 - h r^3) / 3 (the error
// squares at each step), from the FP32 inverse cube root as the seed (relative
// error ~1e-7, so the second step reaches FP64 rounding), then r^7 = r (r^3)^2:
// no FP64 cube root and no division.  Outside that range, h^2 cbrt(h) divides.
__device__ __forceinline__ double h_m73(double h) {
  if (!(fbits(h) > fbits(1e-30) && fbits(h) < fbits(1e30))) return 1.0 / (h * h * cbrt(h));
  double r = (double)rcbrtf((float)h);
  const double third = 1.0 / 3.0;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const double e = fma(-h, r * r * r, 1.0);
    r = fma(r * third, e, r);
  }
  const double r3 = r * r * r;
  return r * (r3 * r3);
}

__device__ __forceinline__ void friction_point(double gn2dt, double tol, double h, double& qx,
                                               double& qy) {
  if (!above(h, tol)) return;
  const double qm = sqrt(qx * qx + qy * qy);
  const double den = 1.0 + gn2dt * qm * h_m73(h);
  const double iden = 1.0 / den;
  qx = qx * iden;
  qy = qy * iden;
}

// Friction on the cells of one 32 x 8 tile (threads 32 x 8).  A quiescent cell
// (every Gauss-point depth at h0 <= tol_dry, Un's qm bit clear) has no water to
// rub, and neither has a cell without roughness: the others are gathered and
// handed to the first threads, so the FP64 arithmetic runs on full warps.
// `cells` is shared memory for the tile's list, `cnt` for the per-warp counts.
__device__ __forceinline__ void friction_tile(const Dev& d, int bx, int by, unsigned short* cells,
                                              int* cnt) {
  const Scalars* sc = d.sc;
  const int t = threadIdx.y * TX + threadIdx.x, w = t >> 5, lane = t & 31;
  int tx, ty;
  warp_cell(tx, ty);
  const int i = bx * TX + tx, j = by * TY + ty;
  const long long P = d.plane;
  bool work = i < d.nx && j < d.ny;
  if (work && d.qm && d.tiles.skip && d.scheme == 0)
    work = (d.qm[(long long)(by * TBY + ty / WY) * d.nbx + bx * TBX + tx / WX] >> lane) & 1u;
  if (work) work = d.N[(long long)j * d.pitch + i] != 0.0;
  const unsigned bw = __ballot_sync(0xffffffffu, work);
  if (lane == 0) cnt[w] = __popc(bw);
  __syncthreads();
  int before = 0, total = 0;
#pragma unroll
  for (int k = 0; k < TX * TY / 32; ++k) {
    before += k < w ? cnt[k] : 0;
    total += cnt[k];
  }
  if (work) cells[before + __popc(bw & ((1u << lane) - 1u))] = (unsigned short)(ty * TX + tx);
  __syncthreads();
  if (t < total) {
    const int me = cells[t];
    const int ci = bx * TX + me % TX, cj = by * TY + me / TX;
    const long long c = (long long)cj * d.pitch + ci;
    const double n = d.N[c];
    const double dt = sc->dt;
    const double gn2dt = dt * d.g * n * n;
    double* S = d.S;
    const double h0 = S[H0 * P + c], x0 = S[QX0 * P + c], y0 = S[QY0 * P + c];
    double cx = x0, cy = y0;
    friction_point(gn2dt, d.tol, h0, cx, cy);
    const double r3 = 1.0 / 1.7320508075688772, hs3 = 0.5 * 1.7320508075688772;
    double nq[2][2];
#pragma unroll
    for (int dd = 1; dd <= 2; ++dd) {
      const double h1 = S[dd * P + c], x1 = S[(3 + dd) * P + c], y1 = S[(6 + dd) * P + c];
      double xp = x0 + x1 * r3, yp = y0 + y1 * r3, xm = x0 - x1 * r3, ym = y0 - y1 * r3;
      friction_point(gn2dt, d.tol, h0 + h1 * r3, xp, yp);
      friction_point(gn2dt, d.tol, h0 - h1 * r3, xm, ym);
      nq[dd - 1][0] = hs3 * (xp - xm);
      nq[dd - 1][1] = hs3 * (yp - ym);
    }
    S[QX0 * P + c] = cx;
    S[QY0 * P + c] = cy;
    S[QX1X * P + c] = nq[0][0];
    S[QY1X * P + c] = nq[0][1];
    S[QX1Y * P + c] = nq[1][0];
    S[QY1Y * P + c] = nq[1][1];
  }
  __syncthreads();  // the list is reused by the block's next tile
}

// Friction over the step's computed tiles (a quiescent tile has no water to rub).
static __global__ void __launch_bounds__(TX * TY) friction_kernel(Dev d) {
  __shared__ unsigned short cells[TX * TY];
  __shared__ int cnt[TX * TY / 32];
  const Scalars* sc = d.sc;
  if (sc->done) return;
  const int n_act = sc->n_act, ntx = d.tiles.ntx;
  const bool all = sc->list_all != 0;
  for (int e = blockIdx.x; e < n_act; e += gridDim.x) {
    const int tile = all ? e : list_tile(d.tiles, sc, e);
    friction_tile(d, tile % ntx, tile / ntx, cells, cnt);
  }
}

// Loads the 9 coefficients of cell c from buffer U.
__device__ __forceinline__ void load9(const double* __restrict__ U, long long P, long long c,
                                      double* m) {
#pragma unroll
  for (int k = 0; k < 9; ++k) m[k] = U[k * P + c];
}

// One side of a face (Sec. 2.1.2 and its positivity-consistent reading): the
// planar limit's depth h and velocities (u, v by the tol rule), the depth the
// face may draw on (hs), the continuous face bed zf, and whether the side's
// cell is partially wet (a wet cell whose planar depth is negative at a face).
struct Rec {
  double h, u, v, hs, zf;
  int pw;
};

// A revised face: its flux and the lower (west / south) side's revised depth
// and bed level for that side's own Eq. 5 and bed term.
struct FaceR {
  double fh, fx, fy, ha, za;
};

struct StageSmem {
  Rec e[TY][TX];     // east record of each cell (lower side of the face to its east)
  Rec n[TY][TX];     // north record of each cell
  Rec hw[TY];        // record west of the tile's first column (neighbour or ghost)
  Rec he[TY];        // record east of the tile's last column
  Rec hs[TX];        // record south of the tile's first row
  Rec hn[TX];        // record north of the tile's last row
  FaceR fx[TY][TX + 1];  // x faces; fx[ty][tx] is the west face of column tx
  FaceR fy[TY + 1][TX];  // y faces; fy[ty][tx] is the south face of row ty
  double red[32];
  unsigned char nq[TY + 2][TX + 2];   // the stage input's non-quiescence, tile and ring
  unsigned char cls[TY][TX];          // 0 outside the grid, 1 fixed point, 2 computed
  unsigned char nqo[TY][TX];          // the stage output's non-quiescence
  unsigned short perm[TX * TY];       // tile cell of each thread, computed cells first
  int wcnt[2][TX * TY / 32];          // computed / fixed-point cells of each warp block
};

// Record of a side whose planar limit is (h, qx, qy) over face bed zf; `sc` is
// the depth scale of a partially wet cell (pw), 1 otherwise.  Velocities by
// the tol rule; under the default revision (thin = wd), a limit thinner than
// eps = h0 / 10 in a cell deeper than 10 tol_dry has its velocity
// desingularised (Kurganov and Petrova, 2007): u = 2 max(h, 0) q / (h^2 +
// eps^2), equal to q/h at h = eps (the planar discharge is not a resolved
// velocity at such a face).
__device__ __forceinline__ Rec make_rec(double h, double qx, double qy, double zf, bool pw,
                                        double sc, double tol, bool thin = false, double h0 = 0.0) {
  Rec r;
  r.h = h;
  r.u = 0.0;
  r.v = 0.0;
  const double eps = 0.1 * h0;
  if (thin && above(eps, tol) && fbits(h) < fbits(eps)) {  // h < eps (eps > 0)
    const double hp = pos_part(h);
    const double den = h * h + eps * eps;
    const double k = 2.0 * hp / den;
    r.u = k * qx;
    r.v = k * qy;
  } else if (above(h, tol)) {
    const double ih = 1.0 / h;
    r.u = qx * ih;
    r.v = qy * ih;
  }
  const double hp = pos_part(h);
  r.hs = pw ? sc * hp : hp;
  r.zf = zf;
  r.pw = pw ? 1 : 0;
  return r;
}

// Partially wet test and depth scale of a cell from its four planar depth
// limits (W, E, S, N); `positive` = 0 keeps the printed revision (never pw).
__device__ __forceinline__ bool pw_scale(double h0, double hW, double hE, double hS, double hN,
                                         double tol, int positive, double& sc) {
  sc = 1.0;
  if (!positive || !above(h0, tol)) return false;
  if (!(is_neg(hW) || is_neg(hE) || is_neg(hS) || is_neg(hN))) return false;
  double sum = 0.0;
  sum += pos_part(hW);
  sum += pos_part(hE);
  sum += pos_part(hS);
  sum += pos_part(hN);
  sc = h0 / (0.25 * sum);
  return true;
}

// Revision of the face between lower side a and upper side b and its flux
// (normal y if ydir).  Neither side partially wet: h* = max(0, h) over the
// continuous bed, each side's bed term on zf - max(0, -h).  Otherwise the
// free-surface revision of Sec. 2.2.2 on the sides' own bed levels (zf raised
// by the depth a partially wet side does not offer): z* = max(za, zb),
// h* = max(0, eta - z*), q* = h* u, each side's bed term on z* lowered by the
// amount its free surface lies below it.
__device__ __forceinline__ F3 revise_face(const Rec& a, const Rec& b, bool ydir, double g, double tol,
                                          int flux, double& ha, double& za, double& hb, double& zb) {
  Lim ra, rb;
  if (!a.pw && !b.pw) {
    ha = a.hs;
    hb = b.hs;
    za = a.zf - (is_neg(a.h) ? -a.h : 0.0);
    zb = b.zf - (is_neg(b.h) ? -b.h : 0.0);
    // the flux's velocities follow the tol rule on the revised depth
    const bool wa = above(ha, tol), wb = above(hb, tol);
    ra.u = wa ? a.u : 0.0; ra.v = wa ? a.v : 0.0;
    rb.u = wb ? b.u : 0.0; rb.v = wb ? b.v : 0.0;
  } else {
    double ea, oa, eb, ob;  // free surface and own bed level of each side
    if (a.pw) { ea = a.h + a.zf; oa = ea - a.hs; } else { oa = a.zf; ea = a.zf + a.hs; }
    if (b.pw) { eb = b.h + b.zf; ob = eb - b.hs; } else { ob = b.zf; eb = b.zf + b.hs; }
    const double zs = gt(oa, ob) ? oa : ob;
    const double da = ea - zs, db = eb - zs;
    ha = pos_part(da);
    hb = pos_part(db);
    za = zs - (is_neg(da) ? -da : 0.0);
    zb = zs - (is_neg(db) ? -db : 0.0);
    const bool wa = above(ha, tol), wb = above(hb, tol);
    ra.u = wa ? a.u : 0.0; ra.v = wa ? a.v : 0.0;
    rb.u = wb ? b.u : 0.0; rb.v = wb ? b.v : 0.0;
  }
  ra.h = ha; ra.qx = ha * a.u; ra.qy = ha * a.v;
  rb.h = hb; rb.qx = hb * b.u; rb.qy = hb * b.v;
  return flux_dir(ra, rb, ydir, g, tol, flux);
}

// Planar depth slope of cell (i, j) along dir, limited (Eqs. 6-7 on eta) when
// LL: the h part of limited_slopes.
template <bool LL>
__device__ __forceinline__ double h_slope(const Dev& d, const double* __restrict__ U, int i, int j,
                                          int dir) {
  double sh, sx, sy;
  if (LL) {
    limited_slopes(d, U, i, j, dir, sh, sx, sy);
    return sh;
  }
  return U[dir * d.plane + (long long)j * d.pitch + i];
}

// Record, at the face it shares with a cell of the tile, of the neighbour
// (ni, nj) on side `side` of that face (0: the neighbour is west / south, its
// east / north limit; 1: east / north, its west / south limit), along dir.
template <bool LL>
__device__ __forceinline__ Rec neighbour_rec(const Dev& d, const double* __restrict__ In, int ni, int nj,
                                             int dir, int side) {
  const long long P = d.plane, c = (long long)nj * d.pitch + ni;
  double s1h, s1x, s1y;
  if (LL) limited_slopes(d, In, ni, nj, dir, s1h, s1x, s1y);
  else { s1h = In[dir * P + c]; s1x = In[(3 + dir) * P + c]; s1y = In[(6 + dir) * P + c]; }
  const double h0 = In[H0 * P + c];
  const double o1 = h_slope<LL>(d, In, ni, nj, 3 - dir);   // the other direction's slope
  const double hx1 = dir == 1 ? s1h : o1, hy1 = dir == 1 ? o1 : s1h;
  double sc;
  const bool pw = pw_scale(h0, h0 - hx1, h0 + hx1, h0 - hy1, h0 + hy1, d.tol, d.wd, sc);
  const double sg = side == 0 ? 1.0 : -1.0;
  const double zf = d.Z[c] + sg * d.Z[dir * P + c];
  const double qx0 = In[QX0 * P + c], qy0 = In[QY0 * P + c];
  return make_rec(h0 + sg * s1h, qx0 + sg * s1x, qy0 + sg * s1y, zf, pw, sc, d.tol, d.wd != 0, h0);
}

// Planar limit (h, qx, qy) of cell (i, j) at face f (0 E, 1 W, 2 N, 3 S), with
// the slopes limited when LL, and the face bed zf: what the cell's own thread
// forms, for a ghost built by another thread.
template <bool LL>
__device__ __forceinline__ void own_face_limit(const Dev& d, const double* __restrict__ In, int i,
                                               int j, int f, double& h, double& qx, double& qy,
                                               double& zf) {
  const long long P = d.plane, c = (long long)j * d.pitch + i;
  const int dir = f <= 1 ? 1 : 2;
  double s1h, s1x, s1y;
  if (LL) limited_slopes(d, In, i, j, dir, s1h, s1x, s1y);
  else { s1h = In[dir * P + c]; s1x = In[(3 + dir) * P + c]; s1y = In[(6 + dir) * P + c]; }
  const double h0 = In[H0 * P + c], x0 = In[QX0 * P + c], y0 = In[QY0 * P + c];
  const double z0 = d.Z[c], z1 = d.Z[dir * P + c];
  if (f == 0 || f == 2) { h = h0 + s1h; qx = x0 + s1x; qy = y0 + s1y; zf = z0 + z1; }
  else { h = h0 - s1h; qx = x0 - s1x; qy = y0 - s1y; zf = z0 - z1; }
}

// Ghost record beyond a domain edge, from the own planar limit (h, qx, qy) at
// that edge over the own face bed zf.
__device__ __forceinline__ Rec ghost_rec(const Dev& d, int edge, double s, double t, double h,
                                         double qx, double qy, double zf) {
  ghost(d, edge, s, t, h, qx, qy);
  return make_rec(h, qx, qy, zf, false, 1.0, d.tol);
}

// Per-cell classification of a tile for one stage.  A cell is "computed" when
// its stage input or one of its four face neighbours is non-quiescent (from the
// input's qm bits), or, in stage 2, when stage 1 computed it (its U1 may differ
// from Un): a cell that is not computed is a fixed point of the stage (it is
// quiescent, and so are the records of its faces, whose fluxes vanish), so
// stage 1 copies it to U1 and stage 2 leaves Un in place.  The tile's cells are
// then handed to the threads computed first: thread t takes the t-th cell of
// that order, so the expensive arithmetic runs on full warps and the fixed
// points (and the cells past a ragged grid edge) gather in the last warps,
// which also build the halo records.  Forced tiles, rain and skip = 0 compute
// every cell.  Returns the calling thread's cell in (tx, ty); sm.cls[y][x]
// holds each cell's class (0 outside the grid, 1 fixed point, 2 computed).
template <int STAGE>
__device__ __forceinline__ void classify_cells(const Dev& d, StageSmem& sm, int bx, int by,
                                               bool every, int& tx, int& ty) {
  const int t = threadIdx.y * TX + threadIdx.x, w = t >> 5, lane = t & 31;
  // the input's non-quiescence of the tile's cells and of the ring around it
  {
    int cx, cy;
    warp_cell(cx, cy);
    const int X = bx * TBX + cx / WX, Y = by * TBY + cy / WY;
    const unsigned* qm = STAGE == 1 ? d.qm : d.qm + d.qplane;
    const bool in = bx * TX + cx < d.nx && by * TY + cy < d.ny;
    sm.nq[cy + 1][cx + 1] = in ? (unsigned char)((qm[(long long)Y * d.nbx + X] >> lane) & 1u) : 0;
    if (t < 2 * (TX + TY) + 4) {
      // ring cell k: west / east columns (TY + 2 each, corners included), then south / north rows
      int rx, ry;
      if (t < 2 * (TY + 2)) { rx = t < TY + 2 ? -1 : TX; ry = (t < TY + 2 ? t : t - (TY + 2)) - 1; }
      else { const int q = t - 2 * (TY + 2); rx = q < TX ? q : q - TX; ry = q < TX ? -1 : TY; }
      const int gi = bx * TX + rx, gj = by * TY + ry;
      unsigned char v = 0;
      if (gi >= 0 && gj >= 0 && gi < d.nx && gj < d.ny) {
        const int Xr = gi / WX, Yr = gj / WY;
        const int l = (gj % WY) * WX + gi % WX;
        v = (unsigned char)((qm[(long long)Yr * d.nbx + Xr] >> l) & 1u);
      }
      sm.nq[ry + 1][rx + 1] = v;
    }
  }
  __syncthreads();
  int cx, cy;
  warp_cell(cx, cy);
  const bool act = bx * TX + cx < d.nx && by * TY + cy < d.ny;
  bool comp = false;
  if (act) {
    comp = every || sm.nq[cy + 1][cx + 1] || sm.nq[cy + 1][cx] || sm.nq[cy + 1][cx + 2] ||
           sm.nq[cy][cx + 1] || sm.nq[cy + 2][cx + 1];
    if (STAGE == 2 && !comp) {
      const int X = bx * TBX + cx / WX, Y = by * TBY + cy / WY;
      comp = (d.qm[2 * d.qplane + (long long)Y * d.nbx + X] >> lane) & 1u;
    }
  }
  sm.cls[cy][cx] = (unsigned char)(act ? (comp ? 2 : 1) : 0);
  // computed cells first, then fixed points, then cells outside the grid; each
  // group in the order of the 8 x 4 warp blocks
  const unsigned bc = __ballot_sync(0xffffffffu, comp), ba = __ballot_sync(0xffffffffu, act);
  if (lane == 0) {
    sm.wcnt[0][w] = __popc(bc);
    sm.wcnt[1][w] = __popc(ba & ~bc);
  }
  __syncthreads();
  int nc = 0, na = 0, before_c = 0, before_f = 0, before_o = 0;
#pragma unroll
  for (int k = 0; k < TX * TY / 32; ++k) {
    const int c1 = sm.wcnt[0][k], f1 = sm.wcnt[1][k];
    nc += c1;
    na += f1;
    if (k < w) { before_c += c1; before_f += f1; before_o += 32 - c1 - f1; }
  }
  const unsigned lt = (1u << lane) - 1u;
  int idx;
  if (comp) idx = before_c + __popc(bc & lt);
  else if (act) idx = nc + before_f + __popc(ba & ~bc & lt);
  else idx = nc + na + before_o + __popc(~ba & lt);
  sm.perm[idx] = (unsigned short)(cy * TX + cx);
  if (STAGE == 1 && lane == 0) {
    // stage 1's computed cells, for stage 2's rule
    const int X = bx * TBX + cx / WX, Y = by * TBY + cy / WY;
    d.qm[2 * d.qplane + (long long)Y * d.nbx + X] = bc;
  }
  __syncthreads();
  const int me = sm.perm[t];
  tx = me % TX;
  ty = me / TX;
}

// One RK stage on the 32 x 8 tile (bx, by): face records, one revision and
// one flux per face, Eqs. 4-5, the stage update and the wet-dry treatment.
// Accumulates the boundary inflow rate, the Courant rate and the non-finite /
// non-quiescent flags of the thread's cell into the caller's variables.  Cells
// that are fixed points of the stage (classify_cells) skip the faces and
// Eqs. 4-5.
template <bool LL, int STAGE>
__device__ __forceinline__ void stage_tile(const Dev& d, StageSmem& sm, int bx, int by,
                                           double& brate, double& lam, bool& bad, bool& nonq) {
  Scalars* sc = d.sc;
  const int tile = by * d.tiles.ntx + bx;
  const bool every = !d.tiles.skip || d.tiles.all_forced || d.tiles.forced[tile];
  int tx, ty;
  classify_cells<STAGE>(d, sm, bx, by, every, tx, ty);
  const int i = bx * TX + tx, j = by * TY + ty;
  const bool act = i < d.nx && j < d.ny;
  const long long P = d.plane;
  const long long c = (long long)j * d.pitch + i;
  const double dt = sc->dt;
  const double ts = STAGE == 1 ? sc->t : sc->t + dt;  // boundary-condition time
  const double* __restrict__ In = STAGE == 1 ? d.S : d.T;
  const double g = d.g, tol = d.tol;
  const bool b_me = sm.cls[ty][tx] == 2;
  const bool b_w = tx > 0 && sm.cls[ty][tx - 1] == 2, b_e = tx + 1 < TX && sm.cls[ty][tx + 1] == 2;
  const bool b_s = ty > 0 && sm.cls[ty - 1][tx] == 2, b_n = ty + 1 < TY && sm.cls[ty + 1][tx] == 2;
  double m[9];
  double z0 = 0.0, z1x = 0.0, z1y = 0.0;
  Rec rE, rW, rN, rS;  // own records
  // records: a computed cell's, and those of its neighbours (their limits make
  // the computed cell's faces)
  const bool recs = act && (b_me || b_w || b_e || b_s || b_n);
  if (recs) {
    load9(In, P, c, m);
    if (LL) {
      limited_slopes(d, In, i, j, 1, m[H1X], m[QX1X], m[QY1X]);
      limited_slopes(d, In, i, j, 2, m[H1Y], m[QX1Y], m[QY1Y]);
    }
    z0 = d.Z[c];
    z1x = d.Z[P + c];
    z1y = d.Z[2 * P + c];
    const double eh = m[H0] + m[H1X], wh = m[H0] - m[H1X];
    const double nh = m[H0] + m[H1Y], shh = m[H0] - m[H1Y];
    double scl;
    const bool pw = pw_scale(m[H0], wh, eh, shh, nh, tol, d.wd, scl);
    const bool thin = d.wd != 0;
    rE = make_rec(eh, m[QX0] + m[QX1X], m[QY0] + m[QY1X], z0 + z1x, pw, scl, tol, thin, m[H0]);
    rW = make_rec(wh, m[QX0] - m[QX1X], m[QY0] - m[QY1X], z0 - z1x, pw, scl, tol, thin, m[H0]);
    rN = make_rec(nh, m[QX0] + m[QX1Y], m[QY0] + m[QY1Y], z0 + z1y, pw, scl, tol, thin, m[H0]);
    rS = make_rec(shh, m[QX0] - m[QX1Y], m[QY0] - m[QY1Y], z0 - z1y, pw, scl, tol, thin, m[H0]);
    sm.e[ty][tx] = rE;
    sm.n[ty][tx] = rN;
  }
  // the records beyond the tile (a neighbour's, or the edge ghost), one per
  // thread of the last 2 (TX + TY) threads (the fixed-point cells' threads when
  // there are enough of them), so no warp runs them one lane at a time: west
  // column, east column, south row, north row, every thread on the same code
  // with its side's indices, so a warp holding several sides builds their
  // records together
  {
    const int t = TX * TY - 1 - (threadIdx.y * TX + threadIdx.x);
    const int i0 = bx * TX, j0 = by * TY;
    const int ni = d.nx - i0 < TX ? d.nx - i0 : TX, nj = d.ny - j0 < TY ? d.ny - j0 : TY;
    const int kind = t < TY ? 0 : t < 2 * TY ? 1 : t < 2 * TY + TX ? 2 : 3;
    const int q = kind == 0 ? t : kind == 1 ? t - TY : kind == 2 ? t - 2 * TY : t - 2 * TY - TX;
    // the tile cell beside the face
    const int ci = kind == 0 ? 0 : kind == 1 ? ni - 1 : q;
    const int cj = kind <= 1 ? q : kind == 2 ? 0 : nj - 1;
    if (t < 2 * (TX + TY) && q < (kind <= 1 ? nj : ni) && sm.cls[cj][ci] == 2) {
      const int dir = kind <= 1 ? 1 : 2, side = kind & 1;
      const int gi = i0 + ci, gj = j0 + cj;
      const bool at_edge = dir == 1 ? (side == 0 ? gi == 0 : gi == d.nx - 1)
                                    : (side == 0 ? gj == 0 : gj == d.ny - 1);
      Rec rec;
      if (at_edge) {
        // the ghost of the tile cell's own limit at that face
        const int fo = kind == 0 ? 1 : kind == 1 ? 0 : kind == 2 ? 3 : 2;
        double h, qx, qy, zf;
        own_face_limit<LL>(d, In, gi, gj, fo, h, qx, qy, zf);
        const double s = dir == 1 ? (gj + 0.5) * d.dy : (gi + 0.5) * d.dx;
        rec = ghost_rec(d, kind, s, ts, h, qx, qy, zf);
      } else {
        const int sx = dir == 1 ? (side == 0 ? -1 : 1) : 0, sy = dir == 2 ? (side == 0 ? -1 : 1) : 0;
        rec = neighbour_rec<LL>(d, In, gi + sx, gj + sy, dir, side);
      }
      Rec* dst = kind == 0 ? sm.hw : kind == 1 ? sm.he : kind == 2 ? sm.hs : sm.hn;
      dst[q] = rec;
    }
  }
  __syncthreads();

  // one revision and one flux per face: each thread its west and south faces
  // (the own, upper side stays in registers, the lower side's depth and bed go
  // to shared memory with the flux), then the tile's east and north edge
  // faces one per thread (again the last threads)
  double hWo = 0, zWo = 0, hSo = 0, zSo = 0;
  if (act && (b_me || b_w)) {
    double ha, za;
    const Rec& Lw = tx > 0 ? sm.e[ty][tx - 1] : sm.hw[ty];
    const F3 fw = revise_face(Lw, rW, false, g, tol, d.flux, ha, za, hWo, zWo);
    sm.fx[ty][tx] = FaceR{fw.h, fw.x, fw.y, ha, za};
    if (i == 0) brate += fw.h * d.dy;
  }
  if (act && (b_me || b_s)) {
    double ha, za;
    const Rec& Ls = ty > 0 ? sm.n[ty - 1][tx] : sm.hs[tx];
    const F3 fs = revise_face(Ls, rS, true, g, tol, d.flux, ha, za, hSo, zSo);
    sm.fy[ty][tx] = FaceR{fs.h, fs.x, fs.y, ha, za};
    if (j == 0) brate += fs.h * d.dx;
  }
  {
    const int t = TX * TY - 1 - (threadIdx.y * TX + threadIdx.x);
    const int ni = d.nx - bx * TX < TX ? d.nx - bx * TX : TX;
    const int nj = d.ny - by * TY < TY ? d.ny - by * TY : TY;
    double ha, za, hb, zb;
    // east edge faces (t < nj) and north edge faces (TY <= t < TY + ni) on one
    // code path: the north faces' normal is y
    const bool yf = t >= TY;
    const int q = yf ? t - TY : t;
    if ((yf ? q < ni : q < nj) && (yf ? sm.cls[nj - 1][q] : sm.cls[q][ni - 1]) == 2) {
      const F3 f = revise_face(yf ? sm.n[nj - 1][q] : sm.e[q][ni - 1], yf ? sm.hn[q] : sm.he[q], yf,
                               g, tol, d.flux, ha, za, hb, zb);
      FaceR* dst = yf ? &sm.fy[nj][q] : &sm.fx[q][ni];
      *dst = FaceR{f.h, f.x, f.y, ha, za};
      if (yf ? by * TY + nj == d.ny : bx * TX + ni == d.nx) brate -= f.h * (yf ? d.dx : d.dy);
    }
  }
  __syncthreads();
  bool nq_out = false;  // the cell's output is non-quiescent
  if (act && b_me) {
    const FaceR FW = sm.fx[ty][tx], FE = sm.fx[ty][tx + 1];
    const FaceR GS = sm.fy[ty][tx], GN = sm.fy[ty + 1][tx];
    // own side of the east / north faces: revised as their lower side
    const double hEo = FE.ha, zEo = FE.za, hNo = GN.ha, zNo = GN.za;
    // own revised states (Eq. 5 operands): q* = h* u
    const double Esh = hEo, Esx = hEo * rE.u, Esy = hEo * rE.v;
    const double Wsh = hWo, Wsx = hWo * rW.u, Wsy = hWo * rW.v;
    const double Nsh = hNo, Nsx = hNo * rN.u, Nsy = hNo * rN.v;
    const double Ssh = hSo, Ssx = hSo * rS.u, Ssy = hSo * rS.v;
    const double zb1x = 0.5 * (zEo - zWo), zb1y = 0.5 * (zNo - zSo);
    // dummy modes (Eq. 5; the second line read as the 0y mode)
    const double h0x = 0.5 * (Esh + Wsh), x0x = 0.5 * (Esx + Wsx), y0x = 0.5 * (Esy + Wsy);
    const double h1x_ = 0.5 * (Esh - Wsh), x1x = 0.5 * (Esx - Wsx), y1x = 0.5 * (Esy - Wsy);
    const double h0y = 0.5 * (Nsh + Ssh), x0y = 0.5 * (Nsx + Ssx), y0y = 0.5 * (Nsy + Ssy);
    const double h1y_ = 0.5 * (Nsh - Ssh), x1y = 0.5 * (Nsx - Ssx), y1y = 0.5 * (Nsy - Ssy);
    const double r3 = 1.0 / 1.7320508075688772;
    const F3 Fp = phys_flux(h0x + h1x_ * r3, x0x + x1x * r3, y0x + y1x * r3, g, tol, false);
    const F3 Fm = phys_flux(h0x - h1x_ * r3, x0x - x1x * r3, y0x - y1x * r3, g, tol, false);
    const F3 Gp = phys_flux(h0y + h1y_ * r3, x0y + x1y * r3, y0y + y1y * r3, g, tol, true);
    const F3 Gm = phys_flux(h0y - h1y_ * r3, x0y - x1y * r3, y0y - y1y * r3, g, tol, true);
    const double idx = d.inv_dx, idy = d.inv_dy;
    // Eq. 4a
    double L[9];
    L[H0] = -(FE.fh - FW.fh) * idx - (GN.fh - GS.fh) * idy;
    L[QX0] = -(FE.fx - FW.fx) * idx - (GN.fx - GS.fx) * idy - 2.0 * g * h0x * zb1x * idx;
    L[QY0] = -(FE.fy - FW.fy) * idx - (GN.fy - GS.fy) * idy - 2.0 * g * h0y * zb1y * idy;
    if (d.rain != 0.0 && ts >= d.rain_t0 && ts < d.rain_t1) L[H0] += d.rain;
    if (c == d.src_idx) L[H0] += d.qp * idx * idy;
    // Eq. 4b
    const double k3x = -3.0 * idx, k3y = -3.0 * idy, g23 = 2.0 * g / 3.0;
    L[H1X] = k3x * ((FE.fh + FW.fh) - (Fp.h + Fm.h));
    L[QX1X] = k3x * ((FE.fx + FW.fx) - (Fp.x + Fm.x) + g23 * h1x_ * zb1x);
    L[QY1X] = k3x * ((FE.fy + FW.fy) - (Fp.y + Fm.y));
    // Eq. 4c
    L[H1Y] = k3y * ((GN.fh + GS.fh) - (Gp.h + Gm.h));
    L[QX1Y] = k3y * ((GN.fx + GS.fx) - (Gp.x + Gm.x));
    L[QY1Y] = k3y * ((GN.fy + GS.fy) - (Gp.y + Gm.y) + g23 * h1y_ * zb1y);

    double out[9];
    if (STAGE == 1) {
#pragma unroll
      for (int k = 0; k < 9; ++k) out[k] = m[k] + dt * L[k];
      wetdry(out, z0, z1x, z1y, tol);
#pragma unroll
      for (int k = 0; k < 9; ++k) d.T[k * P + c] = out[k];
      nq_out = above(out[H0], tol);
#pragma unroll
      for (int k = 1; k < 9; ++k) nq_out = nq_out || nonzero(out[k]);
      if (LL) {
        d.Q[0 * P + c] = m[H1X]; d.Q[1 * P + c] = m[H1Y];
        d.Q[2 * P + c] = m[QX1X]; d.Q[3 * P + c] = m[QX1Y];
        d.Q[4 * P + c] = m[QY1X]; d.Q[5 * P + c] = m[QY1Y];
      }
    } else {
      double un[9];
      un[H0] = d.S[H0 * P + c]; un[QX0] = d.S[QX0 * P + c]; un[QY0] = d.S[QY0 * P + c];
      if (LL) {
        un[H1X] = d.Q[0 * P + c]; un[H1Y] = d.Q[1 * P + c];
        un[QX1X] = d.Q[2 * P + c]; un[QX1Y] = d.Q[3 * P + c];
        un[QY1X] = d.Q[4 * P + c]; un[QY1Y] = d.Q[5 * P + c];
      } else {
        un[H1X] = d.S[H1X * P + c]; un[H1Y] = d.S[H1Y * P + c];
        un[QX1X] = d.S[QX1X * P + c]; un[QX1Y] = d.S[QX1Y * P + c];
        un[QY1X] = d.S[QY1X * P + c]; un[QY1Y] = d.S[QY1Y * P + c];
      }
#pragma unroll
      for (int k = 0; k < 9; ++k) out[k] = 0.5 * (un[k] + m[k] + dt * L[k]);
      wetdry(out, z0, z1x, z1y, tol);
#pragma unroll
      for (int k = 0; k < 9; ++k) d.S[k * P + c] = out[k];
      lam = cell_rate(d, out[H0], out[QX0], out[QY0]);
      bad = bad || !(isfinite(out[H0]) && isfinite(out[QX0]) && isfinite(out[QY0])) ||
            out[H0] < -1.0;
      nq_out = above(out[H0], tol);
#pragma unroll
      for (int k = 1; k < 9; ++k) nq_out = nq_out || nonzero(out[k]);
    }
  } else if (act && STAGE == 1) {
    // a fixed point: U1 = Un as the computed stage writes it (a quiescent
    // cell's rate is zero and the wet-dry treatment zeroes its other modes;
    // its limited slopes are its own)
    if (!recs) load9(In, P, c, m);
    d.T[c] = m[H0];
#pragma unroll
    for (int k = 1; k < 9; ++k) d.T[k * P + c] = 0.0;
    if (LL) {
      d.Q[0 * P + c] = m[H1X]; d.Q[1 * P + c] = m[H1Y];
      d.Q[2 * P + c] = m[QX1X]; d.Q[3 * P + c] = m[QX1Y];
      d.Q[4 * P + c] = m[QY1X]; d.Q[5 * P + c] = m[QY1Y];
    }
  }
  // (a stage-2 fixed point keeps Un in place)
  nonq = nq_out;
  // the output's non-quiescence bits, one word per 8 x 4 warp block
  sm.nqo[ty][tx] = nq_out ? 1 : 0;
  __syncthreads();
  {
    int cx, cy;
    warp_cell(cx, cy);
    const unsigned bits = __ballot_sync(0xffffffffu, sm.nqo[cy][cx] != 0);
    if ((threadIdx.x & 31) == 0) {
      const int X = bx * TBX + cx / WX, Y = by * TBY + cy / WY;
      d.qm[(STAGE == 1 ? d.qplane : 0) + (long long)Y * d.nbx + X] = bits;
    }
  }
}

// Work distribution of the stage kernels over the step's tile lists:
// DG2_TILE_LOOP64 1 runs a fixed grid of resident blocks that loop over the
// entries; 0 launches one block per tile of the grid and a block takes the
// entry of its own index (blocks past the lists exit at once, and the
// hardware balances tiles of unequal cost over the SMs).  Measured on the
// 2000 x 1000 floodplain: FP64 tiles (tens of microseconds each, 1-2 blocks
// per SM) run faster one per block; the FP32 kernels (shared with ensembles)
// loop over the list in resident blocks.
#ifndef DG2_TILE_LOOP64
#define DG2_TILE_LOOP64 0
#endif
// minimum resident blocks per SM asked of the register allocator: 2 for both
// FP64 stages (128 registers; measured on the floodplain, DG2-LL 0.857 ms/step
// at 2 blocks against 0.955 at 1 block with 156 registers)
#ifndef DG2_MINB64_NL
#define DG2_MINB64_NL 2
#endif
#ifndef DG2_MINB64_LL
#define DG2_MINB64_LL 2
#endif

// Stage kernels run over the step's list of active tiles (and, in stage 1,
// the frontier tiles that only copy their state for a neighbour's halo),
// built at the end of the previous step.
template <bool LL, int STAGE>
static __global__ void __launch_bounds__(TX* TY, LL ? DG2_MINB64_LL : DG2_MINB64_NL) stage_kernel(Dev d) {
  extern __shared__ double stage_smem[];  // one StageSmem (dynamic: above 48 KB)
  StageSmem& sm = *reinterpret_cast<StageSmem*>(stage_smem);
  Scalars* sc = d.sc;
  if (sc->done) return;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int ntx = d.tiles.ntx;
  const int n_act = sc->n_act;
  const bool all = sc->list_all != 0;
  double lam = 0.0;
  bool bad = false;
#if DG2_TILE_LOOP64
  for (int e = blockIdx.x; e < n_act; e += gridDim.x) {
#else
  if (STAGE == 2 && (int)blockIdx.x >= n_act) return;
  for (int e = blockIdx.x; e < n_act; e = n_act) {
#endif
    const int tile = all ? e : list_tile(d.tiles, sc, e);
    const int bx = tile % ntx, by = tile / ntx;
    double brate = 0.0, lam_t = 0.0;
    bool nonq = false;
    stage_tile<LL, STAGE>(d, sm, bx, by, brate, lam_t, bad, nonq);
    lam = fmax(lam, lam_t);
    // boundary inflow rate of an edge tile, kept per tile (summed in tile order later)
    if (bx == 0 || by == 0 || bx == ntx - 1 || by == d.tiles.nty - 1) {
      const double bsum = block_sum<TX * TY>(brate, sm.red);
      if (tx == 0 && ty == 0) d.bpart[(STAGE - 1) * d.tiles.ntiles + tile] = bsum;
    }
    if (STAGE == 2) {
      const int any_nonq = __syncthreads_or(nonq);
      if (tx == 0 && ty == 0) d.tiles.flag[tile] = any_nonq ? 1 : 0;
    }
    __syncthreads();
  }
  if (STAGE == 1) {
    // frontier tiles: a computed neighbour reads their stage state as halo
    const int n_front = sc->n_front;
    const long long P = d.plane;
#if DG2_TILE_LOOP64
    for (int e = blockIdx.x; e < n_front; e += gridDim.x) {
#else
    for (int e = (int)blockIdx.x - n_act; e >= 0 && e < n_front; e = n_front) {
#endif
      const int tile = d.tiles.front[e];
      int cx, cy;
      warp_cell(cx, cy);
      const int i = (tile % ntx) * TX + cx, j = (tile / ntx) * TY + cy;
      bool nq = false;
      if (i < d.nx && j < d.ny) {
        const long long c = (long long)j * d.pitch + i;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          const double v = d.S[k * P + c];
          d.T[k * P + c] = v;
          nq = nq || (k == 0 ? above(v, d.tol) : nonzero(v));
        }
      }
      // U1's non-quiescence bits of the copied blocks, for a computed neighbour's stage 2
      const unsigned bits = __ballot_sync(0xffffffffu, nq);
      if ((threadIdx.x & 31) == 0) {
        const int X = (tile % ntx) * TBX + cx / WX, Y = (tile / ntx) * TBY + cy / WY;
        d.qm[d.qplane + (long long)Y * d.nbx + X] = bits;
      }
    }
    return;
  }
  if (__syncthreads_or(bad) && tx == 0 && ty == 0) sc->nonfinite = 1;
  const double bl = block_max<TX * TY>(lam, sm.red);
  if (tx == 0 && ty == 0 && bl > 0.0)
    atomicMax(&sc->lam_bits, (unsigned long long)__double_as_longlong(bl));
}

// ---------------------------------------------------------------------------
// End of step: one block of kFinThreads threads
// ---------------------------------------------------------------------------
constexpr int kFinThreads = 1024;

// Builds the next step's tile lists from the non-quiescence flags and the
// forced mask: a tile is computed if its 3 x 3 tile neighbourhood holds a
// flagged or forced tile; a tile that is not computed but has one in its 5 x 5
// neighbourhood copies its state in stage 1 (a computed neighbour reads it).
// One thread per tile, LTX x LTY tiles per block staged with a 2-tile halo in
// shared memory; one atomic per block reserves its list range.  The order of
// the list entries is not fixed, but every tile writes only its own cells,
// bpart slot and flag, and the step's reductions are exact (max) or summed
// per tile in a fixed order, so the step's result does not depend on it.
constexpr int LTX = 32, LTY = 8;
template <class D>
static __global__ void __launch_bounds__(LTX* LTY) lists_kernel(D d) {
  Scalars* sc = d.sc;
  if (sc->skip_lists) return;
  const Tiles& T = d.tiles;
  const int ntx = T.ntx, nty = T.nty;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * LTX + tx;
  const int bx = blockIdx.x * LTX + tx, by = blockIdx.y * LTY + ty;
  const bool in = bx < ntx && by < nty;
  const int t = by * ntx + bx;
  if (!T.skip || T.all_forced) {
    if (in) T.act[t] = 1;
    if (tid == 0 && blockIdx.x == 0 && blockIdx.y == 0) {
      sc->n_act = T.ntiles;
      sc->n_front = 0;
      sc->list_all = 1;
    }
    return;
  }
  __shared__ unsigned char busy[LTY + 4][LTX + 4];
  __shared__ int wa[LTY][kListClasses], wf[LTY], base[kListClasses + 1];
  for (int k = tid; k < (LTY + 4) * (LTX + 4); k += LTX * LTY) {
    const int ly = k / (LTX + 4), lx = k % (LTX + 4);
    const int gx = blockIdx.x * LTX + lx - 2, gy = blockIdx.y * LTY + ly - 2;
    unsigned char v = 0;
    if (gx >= 0 && gy >= 0 && gx < ntx && gy < nty) {
      const int q = gy * ntx + gx;
      v = (T.flag[q] | T.forced[q]) != 0;
    }
    busy[ly][lx] = v;
  }
  __syncthreads();
  bool a = false, f = false;
  if (in) {
#pragma unroll
    for (int oy = -2; oy <= 2; ++oy)
#pragma unroll
      for (int ox = -2; ox <= 2; ++ox) {
        if (!busy[ty + 2 + oy][tx + 2 + ox]) continue;
        if (ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1) a = true;
        else f = true;
      }
    if (a) f = false;
    T.act[t] = a ? 1 : 0;
  }
  // weight class of a computed tile: its count of non-quiescent cells (the DG2
  // cell masks of the new state) in kListClasses equal parts of the tile, the
  // fullest part first
  int cls = kListClasses - 1;
  if (a && d.qm && d.scheme == 0) {
    int nq = 0;
    for (int yy = 0; yy < TBY; ++yy)
      for (int xx = 0; xx < TBX; ++xx)
        nq += __popc(d.qm[(long long)(by * TBY + yy) * d.nbx + bx * TBX + xx]);
    cls = kListClasses - 1 - nq * kListClasses / (TX * TY + 1);
  }
  // warp = one row of LTX tiles: ballot prefix in the warp, warp offsets, one
  // atomic per class
  const int lane = tid & 31;
  const unsigned below = (1u << lane) - 1u;
  const unsigned bf = __ballot_sync(0xffffffffu, f);
  unsigned bk[kListClasses];
#pragma unroll
  for (int k = 0; k < kListClasses; ++k) bk[k] = __ballot_sync(0xffffffffu, a && cls == k);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < kListClasses; ++k) wa[ty][k] = __popc(bk[k]);
    wf[ty] = __popc(bf);
  }
  __syncthreads();
  if (tid == 0) {
    int sall = 0, sf = 0;
    for (int k = 0; k < kListClasses; ++k) {
      int sa = 0;
      for (int w = 0; w < LTY; ++w) {
        const int xa = wa[w][k];
        wa[w][k] = sa;
        sa += xa;
      }
      base[k] = sa ? atomicAdd(&sc->n_b[k], sa) : 0;
      sall += sa;
    }
    for (int w = 0; w < LTY; ++w) {
      const int xf = wf[w];
      wf[w] = sf;
      sf += xf;
    }
    if (sall) atomicAdd(&sc->n_act, sall);
    base[kListClasses] = sf ? atomicAdd(&sc->n_front, sf) : 0;
  }
  __syncthreads();
  if (a) T.list[cls * T.ntiles + base[cls] + wa[ty][cls] + __popc(bk[cls] & below)] = t;
  if (f) T.front[base[kListClasses] + wf[ty] + __popc(bf & below)] = t;
}

// Resets the list counters for lists_kernel (thread 0 of the finalize block).
__device__ __forceinline__ void open_lists(Scalars* sc) {
  sc->n_act = 0;
  sc->n_front = 0;
  sc->list_all = 0;
  sc->skip_lists = 0;
  for (int k = 0; k < kListClasses; ++k) sc->n_b[k] = 0;
}

// Sum over the boundary ring of tiles, in a fixed order, of the per-tile
// boundary inflow rates of both stages (only tiles computed this step).
template <class D>
static __device__ double ring_inflow(const D& d) {
  __shared__ double red[32];
  const Tiles& T = d.tiles;
  const int ntx = T.ntx, nty = T.nty, nt = T.ntiles;
  const int nring = nty == 1 ? ntx : (ntx == 1 ? nty : 2 * ntx + 2 * (nty - 2));
  double part = 0.0;
  for (int k = threadIdx.x; k < nring; k += kFinThreads) {
    int t;
    if (nty == 1) t = k;
    else if (ntx == 1) t = k * ntx;
    else if (k < ntx) t = k;                                       // south row
    else if (k < 2 * ntx) t = (nty - 1) * ntx + (k - ntx);         // north row
    else if (k < 2 * ntx + nty - 2) t = (k - 2 * ntx + 1) * ntx;   // west column
    else t = (k - 2 * ntx - nty + 3) * ntx + ntx - 1;              // east column
    if (T.act[t]) part += d.bpart[t] + d.bpart[nt + t];
  }
  return block_sum<kFinThreads>(part, red);
}

// Time, ledger, gauges and the next step; opens the next step's tile lists
// (built by lists_kernel).  `lists_only`: after a new DEM / state / forced
// mask, only open the lists.
static __global__ void __launch_bounds__(kFinThreads) finalize_kernel(Dev d, int lists_only) {
  Scalars* sc = d.sc;
  if (!lists_only) {
    if (sc->done) {
      if (threadIdx.x == 0) sc->skip_lists = 1;
      return;
    }
    const double btot = ring_inflow(d);
    if (threadIdx.x == 0) {
      const double t = sc->t, dt = sc->dt;
      double src1 = 0.0, src2 = 0.0;
      const double area = d.dx * d.dy * (double)d.nx * (double)d.ny;
      if (d.rain != 0.0 && t >= d.rain_t0 && t < d.rain_t1) src1 += d.rain * area;
      if (d.rain != 0.0 && t + dt >= d.rain_t0 && t + dt < d.rain_t1) src2 += d.rain * area;
      if (d.src_idx >= 0) { src1 += d.qp; src2 += d.qp; }
      if (d.scheme == 2) src2 = src1;  // FV1: one forward-Euler stage at time t
      sc->ledger += dt * 0.5 * (btot + src1 + src2);
      double tn;
      bool at_sample = false;
      if (sc->land && !sc->fixed_dt) {
        double target = sc->t_end;
        if (sc->next_sample <= target) { target = sc->next_sample; at_sample = true; }
        tn = target;
      } else {
        tn = t + dt;
      }
      sc->t = tn;
      if (at_sample) {
        const int r = sc->nsamp;
        if (r < d.max_samples) {
          d.samp_t[r] = tn;
          const long long P = d.plane;
          for (int k = 0; k < d.ngauge; ++k) {
            const long long gc = d.g_idx[k];
            const double h = d.S[gc] + d.g_xi[k] * d.S[P + gc] + d.g_eta[k] * d.S[2 * P + gc];
            d.samp_h[(long long)r * d.ngauge + k] = h > 0.0 ? h : 0.0;
          }
        }
        sc->nsamp = r + 1;
        sc->next_sample += sc->sample_every;
      }
      if (!(dt > 0.0) || !isfinite(tn)) sc->nonfinite = 1;
      sc->steps += 1;
      sc->last_dt = dt;
      schedule_next_dt(d, sc, __longlong_as_double((long long)sc->lam_bits));
      if (!sc->fixed_dt && sc->t >= sc->t_end) sc->done = 1;
      sc->tiles_done += sc->n_act;
    }
  }
  if (threadIdx.x == 0) open_lists(sc);
}

// Courant reduction of the current state alone (after set-up or set_state).
static __global__ void __launch_bounds__(256) rate_kernel(Dev d) {
  __shared__ double red[32];
  __shared__ bool last;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  double lam = 0.0;
  if (i < d.nx && j < d.ny) {
    const long long P = d.plane, c = (long long)j * d.pitch + i;
    lam = cell_rate(d, d.S[c], d.S[QX0 * P + c], d.S[QY0 * P + c]);
  }
  const double bl = block_max<256>(lam, red);
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  Scalars* sc = d.sc;
  if (tid == 0) {
    if (bl > 0.0) atomicMax(&sc->lam_bits, (unsigned long long)__double_as_longlong(bl));
    __threadfence();
    const unsigned int k = atomicAdd(&sc->count, 1u);
    last = (k == gridDim.x * gridDim.y - 1);
  }
  __syncthreads();
  if (last && tid == 0) {
    __threadfence();
    schedule_next_dt(d, sc, __longlong_as_double((long long)atomicAdd(&sc->lam_bits, 0ull)));
    sc->count = 0u;
  }
}

// Starts a run_to: sets the target, recomputes the next sample time from the
// current time and re-caps the pending Courant step to land on the targets.
static __device__ void begin_run_body(Scalars* sc, double t_end) {
  sc->t_end = t_end;
  sc->fixed_dt = 0;
  if (sc->sample_every > 0.0)
    sc->next_sample = (floor(sc->t / sc->sample_every + 1e-9) + 1.0) * sc->sample_every;
  double dt = sc->dt_cfl;
  sc->land = 0;
  double target = sc->t_end;
  if (sc->next_sample <= target) target = sc->next_sample;
  if (sc->t + dt >= target) {
    dt = target - sc->t;
    sc->land = 1;
  }
  sc->dt = dt;
  sc->done = sc->t >= sc->t_end ? 1 : 0;
}

static __global__ void begin_run_kernel(Dev d, double t_end) { begin_run_body(d.sc, t_end); }

// Starts a dg2_step: forced dt (> 0) or the pending Courant step, no landing.
static __global__ void begin_step_kernel(Dev d, double dt) {
  Scalars* sc = d.sc;
  sc->fixed_dt = 1;
  sc->done = 0;
  sc->land = 0;
  sc->dt = dt > 0.0 ? dt : sc->dt_cfl;
}

// Domain mass sum(h0) dx dy (Eq. 11): fixed-order block partials, then the
// last block sums them in block order (deterministic).
static __global__ void __launch_bounds__(256) mass_kernel(Dev d) {
  __shared__ double red[32];
  __shared__ bool last;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  double v = 0.0;
  if (i < d.nx && j < d.ny) v = d.S[(long long)j * d.pitch + i];
  const double s = block_sum<256>(v, red);
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nb = gridDim.x * gridDim.y;
  Scalars* sc = d.sc;
  if (tid == 0) {
    d.mpart[blockIdx.y * gridDim.x + blockIdx.x] = s;
    __threadfence();
    const unsigned int k = atomicAdd(&sc->count, 1u);
    last = (k == (unsigned int)nb - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double part = 0.0;
  for (int k = tid; k < nb; k += 256) part += __ldcg(&d.mpart[k]);
  const double tot = block_sum<256>(part, red);
  if (tid == 0) {
    sc->mass = tot * d.dx * d.dy;
    if (sc->ledger_init) {
      sc->ledger = sc->mass;
      sc->ledger_init = 0;
    }
    sc->count = 0u;
  }
}

}  // namespace dg2
