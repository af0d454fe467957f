// dg2_adj.cu -- discrete adjoint of the FP64 DG2-NL RK2 step (C ABI in
// include/dg2.h, dg2_adj_*).
//
// The problem: K steps of DG2-NL (friction, two RK stages with the wet-dry
// treatment of each stage) from a given state with a given sequence of step
// sizes (frozen: no derivative through the Courant step), and the misfit
//   J = sum over samples s and gauges g of (h_g(U^{k_s}) - obs_{s,g})^2
// of the sampled gauge depths h_g = max(0, h0 + xi h1x + eta h1y) (the gauge
// rule of the forward solver).  Gradients of J with respect to the Manning n
// of every cell and the discharges of the inflow hydrograph's knots.
//
// Reverse sweep written by hand: per step, the adjoint of stage 2, of stage 1
// and of friction, each a transposed stencil evaluated as one pass over the
// faces (the flux of each face, its two neighbouring cells' operator
// adjoints, the face Jacobian) and one pass over the cells (the cell's own
// terms of Eqs. 4-5 and the gather of its four faces).  The local Jacobians
// (one face flux with its revisions and boundary ghost; one cell's own terms;
// one cell's friction) come from forward-mode dual numbers run through the
// same templated point functions the forward kernels of this file use, so
// values and derivatives follow the same branches: the wet-dry, revision,
// HLL-regime and ghost branches of the forward state are frozen.  The
// wet-dry treatment is a frozen 0/1 mask per mode.
//
// Step states are kept by binomial checkpointing (Griewank's treeverse): with
// c snapshot slots, K steps are reversed with at most r extra forward sweeps,
// r the least integer with C(c + r, c) >= K.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/dg2.h"
#include "dg2_internal.h"

// Storage of this translation unit: FP64 by default (namespace dg2::adj);
// dg2_adj32.cu compiles the same file with FP32 storage (namespace dg2::adj32).
#ifndef DG2_ADJ_STORE
#define DG2_ADJ_STORE double
#define DG2_ADJ_NS adj
#endif

namespace dg2 {
namespace DG2_ADJ_NS {

// Arithmetic type (FP64 in both builds) and storage type of every device buffer:
// state, checkpoints, operator adjoints, face Jacobians, topography, Manning n,
// gauge tables and gradients -- double, or float for the FP32 adjoint (this file
// is compiled once for each).  Kernels load stored values into FP64 registers and
// round their results to the storage type; the hydrograph, the step times, the
// per-step discharge adjoint sums and the misfit stay FP64.
#ifndef DG2_ADJ_ARITH
#define DG2_ADJ_ARITH double
#endif
using real = DG2_ADJ_ARITH;
using store = DG2_ADJ_STORE;

// ---------------------------------------------------------------------------
// Forward-mode dual numbers
// ---------------------------------------------------------------------------

template <int N>
struct Dual {
  real v;
  real d[N];
};

template <int N>
__device__ __forceinline__ Dual<N> cst(real x) {
  Dual<N> r;
  r.v = x;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = 0.0;
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> var(real x, int k) {
  Dual<N> r = cst<N>(x);
  r.d[k] = 1.0;
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] - b.d[k];
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator-(const Dual<N>& a) {
  Dual<N> r;
  r.v = -a.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = -a.d[k];
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a.v / b.v;
  const real ib = 1.0 / b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator+(const Dual<N>& a, real b) { return a + cst<N>(b); }
template <int N>
__device__ __forceinline__ Dual<N> operator+(real a, const Dual<N>& b) { return cst<N>(a) + b; }
template <int N>
__device__ __forceinline__ Dual<N> operator-(const Dual<N>& a, real b) { return a - cst<N>(b); }
template <int N>
__device__ __forceinline__ Dual<N> operator-(real a, const Dual<N>& b) { return cst<N>(a) - b; }
template <int N>
__device__ __forceinline__ Dual<N> operator*(const Dual<N>& a, real b) {
  Dual<N> r;
  r.v = a.v * b;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * b;
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator*(real a, const Dual<N>& b) { return b * a; }
template <int N>
__device__ __forceinline__ Dual<N> operator/(const Dual<N>& a, real b) { return a / cst<N>(b); }
template <int N>
__device__ __forceinline__ Dual<N> operator/(real a, const Dual<N>& b) { return cst<N>(a) / b; }
// sqrt, cbrt and |.| with the derivative taken as 0 where the function has
// none (a zero argument: a dry limit's celerity, a still point's |q|).
template <int N>
__device__ __forceinline__ Dual<N> sqrt(const Dual<N>& a) {
  Dual<N> r;
  r.v = ::sqrt(a.v);
  const real s = r.v > 0.0 ? 0.5 / r.v : 0.0;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * s;
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> cbrt(const Dual<N>& a) {
  Dual<N> r;
  r.v = ::cbrt(a.v);
  const real s = r.v != 0.0 ? 1.0 / (3.0 * r.v * r.v) : 0.0;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * s;
  return r;
}
__device__ __forceinline__ real sqrt(real x) { return ::sqrt(x); }
__device__ __forceinline__ real cbrt(real x) { return ::cbrt(x); }
__device__ __forceinline__ real val(real x) { return x; }
template <int N>
__device__ __forceinline__ real val(const Dual<N>& x) { return x.v; }
// a if a <= b else b (and the max likewise), selecting the operand
template <class T>
__device__ __forceinline__ T tmin(const T& a, const T& b) { return val(b) < val(a) ? b : a; }
template <class T>
__device__ __forceinline__ T tmax(const T& a, const T& b) { return val(b) > val(a) ? b : a; }

// ---------------------------------------------------------------------------
// The scheme's point functions, templated on the scalar (real or Dual)
// ---------------------------------------------------------------------------

template <class T>
struct LimT {
  T h, qx, qy, u, v;
};
template <class T>
struct F3T {
  T h, x, y;
};

// Revised face limit (Sec. 2.1.2): h* = max(0, h), velocities q/h above tol.
template <class T>
__device__ __forceinline__ LimT<T> revise_t(const T& h, const T& qx, const T& qy, real tol) {
  LimT<T> r;
  const T zero = T(h - h);  // a zero of the right type
  if (val(h) > tol) {
    r.u = qx / h;
    r.v = qy / h;
  } else {
    r.u = zero;
    r.v = zero;
  }
  r.h = val(h) > 0.0 ? h : zero;
  r.qx = r.h * r.u;
  r.qy = r.h * r.v;
  return r;
}

// HLL normal flux with Toro's wave speeds (n normal, t tangential).
template <class T>
__device__ __forceinline__ F3T<T> hll_t(const T& hL, const T& qnL, const T& qtL, const T& unL,
                                        const T& utL, const T& hR, const T& qnR, const T& qtR,
                                        const T& unR, const T& utR, real g, real tol) {
  F3T<T> f;
  const T zero = T(hL - hL);
  if (val(hL) <= tol && val(hR) <= tol) {
    f.h = zero; f.x = zero; f.y = zero;
    return f;
  }
  const T cL = sqrt(g * hL), cR = sqrt(g * hR);
  T sL, sR;
  if (val(hL) <= tol) {
    sL = unR - 2.0 * cR;
    sR = unR + cR;
  } else if (val(hR) <= tol) {
    sL = unL - cL;
    sR = unL + 2.0 * cL;
  } else {
    const T us = 0.5 * (unL + unR) + cL - cR;
    const T cs = 0.5 * (cL + cR) + 0.25 * (unL - unR);
    sL = tmin(unL - cL, us - cs);
    sR = tmax(unR + cR, us + cs);
  }
  const T fLh = hL * unL, fLn = hL * unL * unL + 0.5 * g * hL * hL, fLt = hL * unL * utL;
  const T fRh = hR * unR, fRn = hR * unR * unR + 0.5 * g * hR * hR, fRt = hR * unR * utR;
  if (val(sL) >= 0.0) {
    f.h = fLh; f.x = fLn; f.y = fLt;
    return f;
  }
  if (val(sR) <= 0.0) {
    f.h = fRh; f.x = fRn; f.y = fRt;
    return f;
  }
  const T inv = 1.0 / (sR - sL), sLR = sL * sR;
  f.h = (sR * fLh - sL * fRh + sLR * (hR - hL)) * inv;
  f.x = (sR * fLn - sL * fRn + sLR * (qnR - qnL)) * inv;
  f.y = (sR * fLt - sL * fRt + sLR * (qtR - qtL)) * inv;
  return f;
}

template <class T>
__device__ __forceinline__ F3T<T> flux_face(const LimT<T>& L, const LimT<T>& R, bool ydir,
                                            real g, real tol) {
  if (!ydir) return hll_t(L.h, L.qx, L.qy, L.u, L.v, R.h, R.qx, R.qy, R.u, R.v, g, tol);
  const F3T<T> r = hll_t(L.h, L.qy, L.qx, L.v, L.u, R.h, R.qy, R.qx, R.v, R.u, g, tol);
  F3T<T> o;
  o.h = r.h; o.x = r.y; o.y = r.x;
  return o;
}

template <class T>
__device__ __forceinline__ F3T<T> phys_t(const T& h, const T& qx, const T& qy, real g, real tol,
                                         bool ydir) {
  const T zero = T(h - h);
  T u = zero, v = zero;
  if (val(h) > tol) {
    u = qx / h;
    v = qy / h;
  }
  F3T<T> f;
  const T p = 0.5 * g * h * h;
  if (!ydir) {
    f.h = h * u; f.x = h * u * u + p; f.y = h * u * v;
  } else {
    f.h = h * v; f.x = h * u * v; f.y = h * v * v + p;
  }
  return f;
}

// ---------------------------------------------------------------------------
// Face records and their revision (Sec. 2.1.2 and its positivity-consistent
// reading for partially wet cells, with the desingularised velocity of thin
// face limits), templated like the functions above; operation order as the
// CPU oracle's cell_recs / face_revise.
// ---------------------------------------------------------------------------

template <class T>
__device__ __forceinline__ T pos_t(const T& x) {
  const T zero = T(x - x);
  return val(x) > 0.0 ? x : zero;
}

// x with its value replaced by v (derivatives kept): the cell mean depth h0 is
// the mode the forward holds, its derivative that of (hE + hW) / 2.
__device__ __forceinline__ real with_value(real, real v) { return v; }
template <int N>
__device__ __forceinline__ Dual<N> with_value(Dual<N> x, real v) {
  x.v = v;
  return x;
}

template <class T>
struct RecT {
  T h, u, v, hs;  // planar depth limit, velocities, the depth the face may draw on
  real zf;      // continuous face bed
  bool pw;        // the side's cell is partially wet
};

// Partially wet test and depth scale from the cell's mean depth and its four
// planar depth limits (summed W, E, S, N); wd = 0 keeps the printed revision.
template <class T>
__device__ __forceinline__ bool pw_scale_t(const T& h0, const T& hW, const T& hE, const T& hS,
                                           const T& hN, real tol, int wd, T& sc) {
  const T zero = T(h0 - h0);
  sc = zero + 1.0;
  if (!wd || !(val(h0) > tol)) return false;
  if (!(val(hW) < 0.0 || val(hE) < 0.0 || val(hS) < 0.0 || val(hN) < 0.0)) return false;
  T sum = zero;
  sum = sum + pos_t(hW);
  sum = sum + pos_t(hE);
  sum = sum + pos_t(hS);
  sum = sum + pos_t(hN);
  sc = h0 / (0.25 * sum);
  return true;
}

// Record of a side with planar limit (h, qx, qy) over face bed zf; velocities by
// the tol rule, or desingularised below eps = h0 / 10 (thin: default revision).
template <class T>
__device__ __forceinline__ RecT<T> make_rec_t(const T& h, const T& qx, const T& qy, real zf,
                                              bool pw, const T& sc, real tol, bool thin,
                                              const T& h0) {
  const T zero = T(h - h);
  RecT<T> r;
  r.h = h;
  r.u = zero;
  r.v = zero;
  r.zf = zf;
  r.pw = pw;
  const T eps = 0.1 * h0;
  if (thin && val(eps) > tol && val(h) < val(eps)) {
    const T hp = pos_t(h);
    const T den = h * h + eps * eps;
    r.u = 2.0 * hp * qx / den;
    r.v = 2.0 * hp * qy / den;
  } else if (val(h) > tol) {
    r.u = qx / h;
    r.v = qy / h;
  }
  const T hp = pos_t(h);
  r.hs = pw ? sc * hp : hp;
  return r;
}

// Revision of the face between lower side a and upper side b: the flux's
// states and each side's revised depth and bed level for its own terms.
template <class T>
__device__ __forceinline__ void revise_face_t(const RecT<T>& a, const RecT<T>& b, real tol,
                                              LimT<T>& ra, LimT<T>& rb, T& ha, T& za, T& hb,
                                              T& zb) {
  const T zero = T(a.h - a.h);
  if (!a.pw && !b.pw) {
    ha = a.hs;
    hb = b.hs;
    za = a.zf - (val(a.h) < 0.0 ? -a.h : zero);
    zb = b.zf - (val(b.h) < 0.0 ? -b.h : zero);
  } else {
    const T ea = a.pw ? a.h + a.zf : a.zf + a.hs;
    const T eb = b.pw ? b.h + b.zf : b.zf + b.hs;
    const T oa = a.pw ? ea - a.hs : zero + a.zf;
    const T ob = b.pw ? eb - b.hs : zero + b.zf;
    const T zs = val(oa) > val(ob) ? oa : ob;
    const T da = ea - zs, db = eb - zs;
    ha = pos_t(da);
    hb = pos_t(db);
    za = zs - (val(da) < 0.0 ? -da : zero);
    zb = zs - (val(db) < 0.0 ? -db : zero);
  }
  // the flux's velocities follow the tol rule on the revised depth
  ra.h = ha; ra.qx = ha * a.u; ra.qy = ha * a.v;
  ra.u = val(ha) > tol ? a.u : zero; ra.v = val(ha) > tol ? a.v : zero;
  rb.h = hb; rb.qx = hb * b.u; rb.qy = hb * b.v;
  rb.u = val(hb) > tol ? b.u : zero; rb.v = val(hb) > tol ? b.v : zero;
}

// Reverse-mode adjoint of one face's revision and flux (revise_face_t, then
// flux_face): the gradient of S = wF . F + wha ha + wza za + whb hb + wzb zb
// (F the flux in x / y components, ha, za, hb, zb the revised depths and beds
// of the lower side a and the upper side b) with respect to each side's record
// fields (h, u, v, hs), added into ga and gb.  The forward values are formed
// by the same operations and value tests as the templated functions, so the
// same branches are taken: the wet-dry, revision, HLL-regime and partially
// wet branches are frozen, sqrt has derivative 0 at 0, and a tie in the wave
// speeds' min / max or the revision's bed level goes to the same operand.
// One forward and one backward sweep replace forward-mode derivatives in
// eight directions.
__device__ __noinline__ void revise_flux_adj(const RecT<real>& a, const RecT<real>& b, bool ydir,
                                             real gr, real tol, const real* wF, real wha,
                                             real wza, real whb, real wzb, real* ga, real* gb) {
  // ---- forward: the revision (revise_face_t) ----
  const bool np = !a.pw && !b.pw;
  // (the revised beds za, zb enter S linearly; their values are not needed)
  real ha, hb, ea = 0.0, eb = 0.0, zs = 0.0, da = 0.0, db = 0.0;
  bool zs_a = false;
  if (np) {
    ha = a.hs;
    hb = b.hs;
  } else {
    ea = a.pw ? a.h + a.zf : a.zf + a.hs;
    eb = b.pw ? b.h + b.zf : b.zf + b.hs;
    const real oa = a.pw ? ea - a.hs : a.zf;
    const real ob = b.pw ? eb - b.hs : b.zf;
    zs_a = oa > ob;
    zs = zs_a ? oa : ob;
    da = ea - zs;
    db = eb - zs;
    ha = da > 0.0 ? da : 0.0;
    hb = db > 0.0 ? db : 0.0;
  }
  // the flux's states in the face frame (normal n, tangential t)
  const bool wa = ha > tol, wb = hb > tol;
  const real an = ydir ? a.v : a.u, at = ydir ? a.u : a.v;
  const real bn = ydir ? b.v : b.u, bt = ydir ? b.u : b.v;
  const real hL = ha, qnL = ha * an, qtL = ha * at, unL = wa ? an : 0.0, utL = wa ? at : 0.0;
  const real hR = hb, qnR = hb * bn, qtR = hb * bt, unR = wb ? bn : 0.0, utR = wb ? bt : 0.0;
  // weights of the frame's components
  const real w[3] = {wF[0], ydir ? wF[2] : wF[1], ydir ? wF[1] : wF[2]};
  // adjoints of the HLL inputs
  real g_hL = 0.0, g_qnL = 0.0, g_qtL = 0.0, g_unL = 0.0, g_utL = 0.0;
  real g_hR = 0.0, g_qnR = 0.0, g_qtR = 0.0, g_unR = 0.0, g_utR = 0.0;
  if (!(hL <= tol && hR <= tol)) {
    // ---- forward: HLL (hll_t) ----
    const real cL = sqrt(gr * hL), cR = sqrt(gr * hR);
    real sL, sR, us = 0.0, cs = 0.0;
    int mode;
    bool sL_first = true, sR_first = true;
    if (hL <= tol) {
      mode = 1;
      sL = unR - 2.0 * cR;
      sR = unR + cR;
    } else if (hR <= tol) {
      mode = 2;
      sL = unL - cL;
      sR = unL + 2.0 * cL;
    } else {
      mode = 0;
      us = 0.5 * (unL + unR) + cL - cR;
      cs = 0.5 * (cL + cR) + 0.25 * (unL - unR);
      const real s1 = unL - cL, s2 = us - cs, r1 = unR + cR, r2 = us + cs;
      sL_first = !(s2 < s1);
      sR_first = !(r2 > r1);
      sL = sL_first ? s1 : s2;
      sR = sR_first ? r1 : r2;
    }
    const real fL[3] = {hL * unL, hL * unL * unL + 0.5 * gr * hL * hL, hL * unL * utL};
    const real fR[3] = {hR * unR, hR * unR * unR + 0.5 * gr * hR * hR, hR * unR * utR};
    real g_fL[3] = {0.0, 0.0, 0.0}, g_fR[3] = {0.0, 0.0, 0.0};
    // ---- backward: HLL ----
    if (sL >= 0.0) {
      for (int k = 0; k < 3; ++k) g_fL[k] = w[k];
    } else if (sR <= 0.0) {
      for (int k = 0; k < 3; ++k) g_fR[k] = w[k];
    } else {
      // F_k = (sR fL_k - sL fR_k + sL sR (qR_k - qL_k)) / (sR - sL)
      const real inv = 1.0 / (sR - sL), sLR = sL * sR;
      const real dq[3] = {hR - hL, qnR - qnL, qtR - qtL};
      real g_sL = 0.0, g_sR = 0.0, g_inv = 0.0, g_dq[3];
      for (int k = 0; k < 3; ++k) {
        const real nk = sR * fL[k] - sL * fR[k] + sLR * dq[k];
        const real gn = w[k] * inv;
        g_inv += w[k] * nk;
        g_fL[k] = gn * sR;
        g_fR[k] = -gn * sL;
        g_sR += gn * (fL[k] + sL * dq[k]);
        g_sL += gn * (sR * dq[k] - fR[k]);
        g_dq[k] = gn * sLR;
      }
      g_sR -= g_inv * inv * inv;
      g_sL += g_inv * inv * inv;
      g_hR += g_dq[0]; g_hL -= g_dq[0];
      g_qnR += g_dq[1]; g_qnL -= g_dq[1];
      g_qtR += g_dq[2]; g_qtL -= g_dq[2];
      // wave speeds
      real g_cL = 0.0, g_cR = 0.0;
      if (mode == 1) {
        g_unR += g_sL + g_sR;
        g_cR += -2.0 * g_sL + g_sR;
      } else if (mode == 2) {
        g_unL += g_sL + g_sR;
        g_cL += -g_sL + 2.0 * g_sR;
      } else {
        real g_us = 0.0, g_cs = 0.0;
        if (sL_first) { g_unL += g_sL; g_cL -= g_sL; } else { g_us += g_sL; g_cs -= g_sL; }
        if (sR_first) { g_unR += g_sR; g_cR += g_sR; } else { g_us += g_sR; g_cs += g_sR; }
        g_unL += 0.5 * g_us + 0.25 * g_cs;
        g_unR += 0.5 * g_us - 0.25 * g_cs;
        g_cL += g_us + 0.5 * g_cs;
        g_cR += -g_us + 0.5 * g_cs;
      }
      // c = sqrt(g h): dc/dh = g / (2 c), 0 at c = 0
      if (cL > 0.0) g_hL += g_cL * (0.5 * gr / cL);
      if (cR > 0.0) g_hR += g_cR * (0.5 * gr / cR);
    }
    // physical fluxes f = (h un, h un^2 + g h^2 / 2, h un ut)
    g_hL += g_fL[0] * unL + g_fL[1] * (unL * unL + gr * hL) + g_fL[2] * unL * utL;
    g_unL += g_fL[0] * hL + g_fL[1] * 2.0 * hL * unL + g_fL[2] * hL * utL;
    g_utL += g_fL[2] * hL * unL;
    g_hR += g_fR[0] * unR + g_fR[1] * (unR * unR + gr * hR) + g_fR[2] * unR * utR;
    g_unR += g_fR[0] * hR + g_fR[1] * 2.0 * hR * unR + g_fR[2] * hR * utR;
    g_utR += g_fR[2] * hR * unR;
  }
  // ---- backward: the flux states to the records and the revised depths ----
  const real g_ha = wha + g_hL + g_qnL * an + g_qtL * at;
  const real g_hb = whb + g_hR + g_qnR * bn + g_qtR * bt;
  const real g_an = g_qnL * ha + (wa ? g_unL : 0.0), g_at = g_qtL * ha + (wa ? g_utL : 0.0);
  const real g_bn = g_qnR * hb + (wb ? g_unR : 0.0), g_bt = g_qtR * hb + (wb ? g_utR : 0.0);
  ga[1] += ydir ? g_at : g_an;
  ga[2] += ydir ? g_an : g_at;
  gb[1] += ydir ? g_bt : g_bn;
  gb[2] += ydir ? g_bn : g_bt;
  // ---- backward: the revision ----
  if (np) {
    ga[3] += g_ha;
    gb[3] += g_hb;
    if (a.h < 0.0) ga[0] += wza;
    if (b.h < 0.0) gb[0] += wzb;
  } else {
    // ha = max(da, 0), za = zs + min(da, 0), da = ea - zs (and b's)
    const real g_da = (da > 0.0 ? g_ha : 0.0) + (da < 0.0 ? wza : 0.0);
    const real g_db = (db > 0.0 ? g_hb : 0.0) + (db < 0.0 ? wzb : 0.0);
    const real g_zs = wza + wzb - g_da - g_db;
    real g_ea = g_da, g_eb = g_db;
    // zs = max(oa, ob), oa = ea - hs (partially wet) or the face bed
    if (zs_a) {
      if (a.pw) { g_ea += g_zs; ga[3] -= g_zs; }
    } else {
      if (b.pw) { g_eb += g_zs; gb[3] -= g_zs; }
    }
    // ea = h + zf (partially wet) or zf + hs
    if (a.pw) ga[0] += g_ea; else ga[3] += g_ea;
    if (b.pw) gb[0] += g_eb; else gb[3] += g_eb;
  }
}

// ---------------------------------------------------------------------------
// Problem description
// ---------------------------------------------------------------------------

constexpr int kMaxKnotsAdj = 4096;

struct Prob {
  int nx, ny;
  long long N;                 // cells (dense planes, x fastest)
  real dx, dy, inv_dx, inv_dy, g, tol;
  int bc[4];
  // one inflow segment (edge < 0: none)
  int in_edge;
  real in_s0, in_s1, in_width;
  const store* Z;            // 3 planes z0, z1x, z1y
  const store* Nm;           // Manning n
  real rain, rain_t0, rain_t1;
  int wd;                      // 1: positivity-consistent revision (default), 0: printed
};

__device__ __forceinline__ bool on_inflow(const Prob& p, int edge, real s) {
  return p.in_edge == edge && s >= p.in_s0 && s <= p.in_s1;
}

// Outside state of an edge face from the own raw limit (h, qx, qy) and the
// hydrograph discharge Q (m^3/s) of the inflow segment at the stage time.
template <class T>
__device__ __forceinline__ void ghost_t(const Prob& p, int edge, real s, const T& Q, T& h, T& qx,
                                        T& qy) {
  const T zero = T(h - h);
  if (on_inflow(p, edge, s)) {
    const T qin = Q / p.in_width;
    const T hin = val(h) > 0.0 ? h : zero;
    const T hc = cbrt(qin * qin / p.g);
    const T hg = val(hin) > val(hc) ? hin : hc;
    const T qn = (edge == 0 || edge == 2) ? qin : -qin;
    h = hg;
    if (edge <= 1) { qx = qn; qy = zero; } else { qx = zero; qy = qn; }
    return;
  }
  if (p.bc[edge] == DG2_OPEN) {
    if (edge == 0 && val(qx) > 0.0) qx = zero;
    if (edge == 1 && val(qx) < 0.0) qx = zero;
    if (edge == 2 && val(qy) > 0.0) qy = zero;
    if (edge == 3 && val(qy) < 0.0) qy = zero;
    return;
  }
  if (edge <= 1) qx = -qx; else qy = -qy;
}

enum { H0 = 0, H1X, H1Y, QX0, QX1X, QX1Y, QY0, QY1X, QY1Y };

// Raw limit (h, qx, qy) of cell c at face f (0 E, 1 W, 2 N, 3 S).
__device__ __forceinline__ void raw_limit(const store* __restrict__ U, long long N, long long c,
                                          int f, real& h, real& qx, real& qy) {
  const int m = f <= 1 ? 1 : 2;
  const real sg = (f == 0 || f == 2) ? 1.0 : -1.0;
  h = U[c] + sg * U[m * N + c];
  qx = U[3 * N + c] + sg * U[(3 + m) * N + c];
  qy = U[6 * N + c] + sg * U[(6 + m) * N + c];
}

// The four face records of cell c (faces 0 E, 1 W, 2 N, 3 S) from its raw
// limits and mean depth h0.
template <class T>
__device__ __forceinline__ void cell_recs_t(const Prob& p, long long c, const T* E, const T* W,
                                            const T* Nn, const T* S, const T& h0, RecT<T>* r) {
  const real z0 = p.Z[c], z1x = p.Z[p.N + c], z1y = p.Z[2 * p.N + c];
  T sc;
  const bool pw = pw_scale_t(h0, W[0], E[0], S[0], Nn[0], p.tol, p.wd, sc);
  const bool thin = p.wd != 0;
  r[0] = make_rec_t(E[0], E[1], E[2], z0 + z1x, pw, sc, p.tol, thin, h0);
  r[1] = make_rec_t(W[0], W[1], W[2], z0 - z1x, pw, sc, p.tol, thin, h0);
  r[2] = make_rec_t(Nn[0], Nn[1], Nn[2], z0 + z1y, pw, sc, p.tol, thin, h0);
  r[3] = make_rec_t(S[0], S[1], S[2], z0 - z1y, pw, sc, p.tol, thin, h0);
}

// Cell's own terms of Eqs. 4-5 (fluxes excluded) from its revised face depths
// h*, bed levels z* and face velocities (u, v): dummy modes, Gauss-point
// fluxes and bed terms.
template <class T>
__device__ __forceinline__ void own_terms(const Prob& p, const T* hs, const T* zs, const T* u,
                                          const T* v, T* L) {
  const T zero = T(hs[0] - hs[0]);
  LimT<T> Es, Ws, Ns, Ss;
  Es.h = hs[0]; Es.qx = hs[0] * u[0]; Es.qy = hs[0] * v[0];
  Ws.h = hs[1]; Ws.qx = hs[1] * u[1]; Ws.qy = hs[1] * v[1];
  Ns.h = hs[2]; Ns.qx = hs[2] * u[2]; Ns.qy = hs[2] * v[2];
  Ss.h = hs[3]; Ss.qx = hs[3] * u[3]; Ss.qy = hs[3] * v[3];
  const T zb1x = 0.5 * (zs[0] - zs[1]), zb1y = 0.5 * (zs[2] - zs[3]);
  const T h0x = 0.5 * (Es.h + Ws.h), x0x = 0.5 * (Es.qx + Ws.qx), y0x = 0.5 * (Es.qy + Ws.qy);
  const T h1x = 0.5 * (Es.h - Ws.h), x1x = 0.5 * (Es.qx - Ws.qx), y1x = 0.5 * (Es.qy - Ws.qy);
  const T h0y = 0.5 * (Ns.h + Ss.h), x0y = 0.5 * (Ns.qx + Ss.qx), y0y = 0.5 * (Ns.qy + Ss.qy);
  const T h1y = 0.5 * (Ns.h - Ss.h), x1y = 0.5 * (Ns.qx - Ss.qx), y1y = 0.5 * (Ns.qy - Ss.qy);
  const real r3 = 1.0 / 1.7320508075688772;
  const F3T<T> Fp = phys_t(h0x + h1x * r3, x0x + x1x * r3, y0x + y1x * r3, p.g, p.tol, false);
  const F3T<T> Fm = phys_t(h0x - h1x * r3, x0x - x1x * r3, y0x - y1x * r3, p.g, p.tol, false);
  const F3T<T> Gp = phys_t(h0y + h1y * r3, x0y + x1y * r3, y0y + y1y * r3, p.g, p.tol, true);
  const F3T<T> Gm = phys_t(h0y - h1y * r3, x0y - x1y * r3, y0y - y1y * r3, p.g, p.tol, true);
  const real g = p.g, idx = p.inv_dx, idy = p.inv_dy;
  const real k3x = -3.0 * idx, k3y = -3.0 * idy, g23 = 2.0 * g / 3.0;
  L[H0] = zero;
  L[QX0] = -(2.0 * g * h0x * zb1x * idx);
  L[QY0] = -(2.0 * g * h0y * zb1y * idy);
  L[H1X] = k3x * (-(Fp.h + Fm.h));
  L[QX1X] = k3x * (-(Fp.x + Fm.x) + g23 * h1x * zb1x);
  L[QY1X] = k3x * (-(Fp.y + Fm.y));
  L[H1Y] = k3y * (-(Gp.h + Gm.h));
  L[QX1Y] = k3y * (-(Gp.x + Gm.x));
  L[QY1Y] = k3y * (-(Gp.y + Gm.y) + g23 * h1y * zb1y);
}

// Adjoint of a Gauss-point physical flux (phys_t) of state (h, qx, qy) along x
// or y: adds the gradient of gf . f into g_h, g_qx, g_qy (velocities by the
// tol rule, frozen below it).
__device__ __forceinline__ void phys_adj(real h, real qx, real qy, real gr, real tol, bool ydir,
                                         const real* gf, real& g_h, real& g_qx, real& g_qy) {
  const bool wet = h > tol;
  const real u = wet ? qx / h : 0.0, v = wet ? qy / h : 0.0;
  real gh, gu, gv;
  if (!ydir) {  // (h u, h u^2 + g h^2 / 2, h u v)
    gh = gf[0] * u + gf[1] * (u * u + gr * h) + gf[2] * u * v;
    gu = gf[0] * h + gf[1] * 2.0 * h * u + gf[2] * h * v;
    gv = gf[2] * h * u;
  } else {      // (h v, h u v, h v^2 + g h^2 / 2)
    gh = gf[0] * v + gf[1] * u * v + gf[2] * (v * v + gr * h);
    gu = gf[1] * h * v;
    gv = gf[0] * h + gf[1] * h * u + gf[2] * 2.0 * h * v;
  }
  if (wet) {  // u = qx / h, v = qy / h
    g_qx += gu / h;
    g_qy += gv / h;
    gh -= (gu * u + gv * v) / h;
  }
  g_h += gh;
}

// Reverse-mode adjoint of own_terms contracted with mu: the gradient of
// sum_k mu[k] L[k] with respect to the faces' revised depths hs, beds zs and
// velocities u, v (written to g_hs, g_zs, g_u, g_v; faces E, W, N, S).
__device__ __noinline__ void own_terms_adj(const Prob& p, const real* hs, const real* zs,
                                           const real* u, const real* v, const real* mu,
                                           real* g_hs, real* g_zs, real* g_u, real* g_v) {
  const real gr = p.g, idx = p.inv_dx, idy = p.inv_dy;
  const real k3x = -3.0 * idx, k3y = -3.0 * idy, g23 = 2.0 * gr / 3.0;
  const real r3 = 1.0 / 1.7320508075688772;
  // forward: the revised states (q* = h* u) and the dummy modes of both directions
  real sh[4], sx[4], sy[4];
  for (int f = 0; f < 4; ++f) {
    sh[f] = hs[f];
    sx[f] = hs[f] * u[f];
    sy[f] = hs[f] * v[f];
  }
  const real zb1x = 0.5 * (zs[0] - zs[1]), zb1y = 0.5 * (zs[2] - zs[3]);
  // mean and slope of (h, qx, qy) along x (faces E, W) and y (faces N, S)
  real m0[2][3], m1[2][3];
  for (int dd = 0; dd < 2; ++dd) {
    const int fp = 2 * dd, fm = 2 * dd + 1;
    m0[dd][0] = 0.5 * (sh[fp] + sh[fm]);
    m1[dd][0] = 0.5 * (sh[fp] - sh[fm]);
    m0[dd][1] = 0.5 * (sx[fp] + sx[fm]);
    m1[dd][1] = 0.5 * (sx[fp] - sx[fm]);
    m0[dd][2] = 0.5 * (sy[fp] + sy[fm]);
    m1[dd][2] = 0.5 * (sy[fp] - sy[fm]);
  }
  // backward: adjoints of the modes and of the bed slopes
  real g_m0[2][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
  real g_m1[2][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
  real g_zb1x = 0.0, g_zb1y = 0.0;
  // bed terms of the average and slope equations
  g_m0[0][0] += -2.0 * gr * idx * zb1x * mu[QX0];
  g_zb1x += -2.0 * gr * idx * m0[0][0] * mu[QX0];
  g_m0[1][0] += -2.0 * gr * idy * zb1y * mu[QY0];
  g_zb1y += -2.0 * gr * idy * m0[1][0] * mu[QY0];
  g_m1[0][0] += k3x * g23 * zb1x * mu[QX1X];
  g_zb1x += k3x * g23 * m1[0][0] * mu[QX1X];
  g_m1[1][0] += k3y * g23 * zb1y * mu[QY1Y];
  g_zb1y += k3y * g23 * m1[1][0] * mu[QY1Y];
  // Gauss-point fluxes: L = k3 (-(Fp + Fm)) in the slope equations
  for (int dd = 0; dd < 2; ++dd) {
    const real k3 = dd == 0 ? k3x : k3y;
    const real gf[3] = {-k3 * mu[dd == 0 ? H1X : H1Y], -k3 * mu[dd == 0 ? QX1X : QX1Y],
                        -k3 * mu[dd == 0 ? QY1X : QY1Y]};
    for (int sgn = 0; sgn < 2; ++sgn) {
      const real r = sgn == 0 ? r3 : -r3;
      real gh = 0.0, gx = 0.0, gy = 0.0;
      phys_adj(m0[dd][0] + m1[dd][0] * r, m0[dd][1] + m1[dd][1] * r, m0[dd][2] + m1[dd][2] * r,
               gr, p.tol, dd == 1, gf, gh, gx, gy);
      g_m0[dd][0] += gh;
      g_m1[dd][0] += gh * r;
      g_m0[dd][1] += gx;
      g_m1[dd][1] += gx * r;
      g_m0[dd][2] += gy;
      g_m1[dd][2] += gy * r;
    }
  }
  // modes to the faces' revised states, then to hs, u, v
  for (int dd = 0; dd < 2; ++dd) {
    const int fp = 2 * dd, fm = 2 * dd + 1;
    const real ghp = 0.5 * (g_m0[dd][0] + g_m1[dd][0]), ghm = 0.5 * (g_m0[dd][0] - g_m1[dd][0]);
    const real gxp = 0.5 * (g_m0[dd][1] + g_m1[dd][1]), gxm = 0.5 * (g_m0[dd][1] - g_m1[dd][1]);
    const real gyp = 0.5 * (g_m0[dd][2] + g_m1[dd][2]), gym = 0.5 * (g_m0[dd][2] - g_m1[dd][2]);
    g_hs[fp] = ghp + gxp * u[fp] + gyp * v[fp];
    g_hs[fm] = ghm + gxm * u[fm] + gym * v[fm];
    g_u[fp] = gxp * hs[fp];
    g_v[fp] = gyp * hs[fp];
    g_u[fm] = gxm * hs[fm];
    g_v[fm] = gym * hs[fm];
  }
  g_zs[0] = 0.5 * g_zb1x;
  g_zs[1] = -0.5 * g_zb1x;
  g_zs[2] = 0.5 * g_zb1y;
  g_zs[3] = -0.5 * g_zb1y;
}

// Records of cell (i, j) of state U in real.
__device__ __forceinline__ void recs_double(const Prob& p, const store* __restrict__ U, long long c,
                                            RecT<real>* r) {
  real E[3], W[3], Nn[3], S[3];
  raw_limit(U, p.N, c, 0, E[0], E[1], E[2]);
  raw_limit(U, p.N, c, 1, W[0], W[1], W[2]);
  raw_limit(U, p.N, c, 2, Nn[0], Nn[1], Nn[2]);
  raw_limit(U, p.N, c, 3, S[0], S[1], S[2]);
  cell_recs_t<real>(p, c, E, W, Nn, S, U[c], r);
}

// Record of one side of a face from the side's four depth limits (E, W, N, S),
// its discharge limits (qx, qy) at the face and its cell-mean depth h0v, over
// face bed zf; fo is the face as the side sees it.  The mean depth carries the
// derivative of (hE + hW) / 2 (with_value).
template <class T>
__device__ __forceinline__ RecT<T> side_rec(const Prob& p, const T* h4, const T& qx, const T& qy,
                                            real h0v, int fo, real zf) {
  const T h0 = with_value(0.5 * (h4[0] + h4[1]), h0v);
  T sc;
  const bool pw = pw_scale_t(h0, h4[1], h4[0], h4[3], h4[2], p.tol, p.wd, sc);
  const T& hf = fo == 0 ? h4[0] : fo == 1 ? h4[1] : fo == 2 ? h4[2] : h4[3];
  return make_rec_t(hf, qx, qy, zf, pw, sc, p.tol, p.wd != 0, h0);
}

// Reverse-mode adjoint of a record's velocities (make_rec_t): adds the
// gradient of gu u + gv v with respect to the planar limit (h, qx, qy) and the
// cell's mean depth h0 (through the thin-limit threshold eps = h0 / 10), the
// forward's branches frozen.
__device__ __forceinline__ void rec_uv_adj(real h, real qx, real qy, bool thin, real tol, real h0,
                                           real gu, real gv, real& g_h, real& g_qx, real& g_qy,
                                           real& g_h0) {
  const real eps = 0.1 * h0;
  if (thin && eps > tol && h < eps) {
    // u = k qx, v = k qy with k = 2 max(h, 0) / (h^2 + eps^2)
    const real hp = h > 0.0 ? h : 0.0;
    const real den = h * h + eps * eps;
    const real k = 2.0 * hp / den;
    g_qx += gu * k;
    g_qy += gv * k;
    const real g_k = gu * qx + gv * qy;
    if (h > 0.0) g_h += g_k * 2.0 / den;
    const real g_den = -g_k * k / den;
    g_h += g_den * 2.0 * h;
    g_h0 += g_den * 2.0 * eps * 0.1;
  } else if (h > tol) {
    const real u = qx / h, v = qy / h;
    g_qx += gu / h;
    g_qy += gv / h;
    g_h -= (gu * u + gv * v) / h;
  }
}

// Reverse-mode adjoint of side_rec: the gradient of gr . (h, u, v, hs) of the
// record with respect to the side's four depth limits (E, W, N, S) and its
// discharge limits (qx, qy), written to g[0..5].
__device__ __noinline__ void side_rec_adj(const Prob& p, const real* h4, real qx, real qy,
                                          real h0, int fo, const real* gr, real* g) {
  const real tol = p.tol;
  // the partially wet test and scale of pw_scale_t (limits W, E, S, N)
  bool pw = false;
  real sc = 1.0, sum = 0.0;
  if (p.wd && h0 > tol && (h4[1] < 0.0 || h4[0] < 0.0 || h4[3] < 0.0 || h4[2] < 0.0)) {
    pw = true;
    const int order[4] = {1, 0, 3, 2};
    for (int k = 0; k < 4; ++k) sum += h4[order[k]] > 0.0 ? h4[order[k]] : 0.0;
    sc = h0 / (0.25 * sum);
  }
  const real hf = fo == 0 ? h4[0] : fo == 1 ? h4[1] : fo == 2 ? h4[2] : h4[3];
  const real hp = hf > 0.0 ? hf : 0.0;
  real g_hf = gr[0], g_h0 = 0.0, g_qx = 0.0, g_qy = 0.0;
  // hs = sc max(h, 0) (partially wet) or max(h, 0)
  const real g_hp = pw ? gr[3] * sc : gr[3];
  const real g_sc = pw ? gr[3] * hp : 0.0;
  if (hf > 0.0) g_hf += g_hp;
  rec_uv_adj(hf, qx, qy, p.wd != 0, tol, h0, gr[1], gr[2], g_hf, g_qx, g_qy, g_h0);
  real g4[4] = {0.0, 0.0, 0.0, 0.0};
  if (pw) {  // sc = h0 / (sum / 4)
    g_h0 += g_sc / (0.25 * sum);
    const real g_sum = -g_sc * sc / sum;
    for (int k = 0; k < 4; ++k)
      if (h4[k] > 0.0) g4[k] += g_sum;
  }
  g4[fo] += g_hf;
  // h0 carries the derivative of (hE + hW) / 2
  g4[0] += 0.5 * g_h0;
  g4[1] += 0.5 * g_h0;
  for (int k = 0; k < 4; ++k) g[k] = g4[k];
  g[4] = g_qx;
  g[5] = g_qy;
}

// Face on side f (0 E, 1 W, 2 N, 3 S) of cell (i, j) of state U at stage time
// with hydrograph discharge Q, in real: its flux and the own side's revised
// depth and bed level.
__device__ void face_rev(const Prob& p, const store* __restrict__ U, int i, int j, int f, real Q,
                         const RecT<real>* own, F3T<real>& F, real& ho, real& zo) {
  const long long N = p.N, c = (long long)j * p.nx + i;
  RecT<real> oth;
  const bool edge = (f == 0 && i == p.nx - 1) || (f == 1 && i == 0) || (f == 2 && j == p.ny - 1) ||
                    (f == 3 && j == 0);
  if (edge) {
    real h, qx, qy;
    raw_limit(U, N, c, f, h, qx, qy);
    const int e = f == 0 ? 1 : f == 1 ? 0 : f == 2 ? 3 : 2;
    const real s = f <= 1 ? (j + 0.5) * p.dy : (i + 0.5) * p.dx;
    ghost_t<real>(p, e, s, Q, h, qx, qy);
    oth = make_rec_t<real>(h, qx, qy, own[f].zf, false, 1.0, p.tol, false, 0.0);
  } else {
    // the neighbour's record of this face alone (its four depth limits set
    // its partially wet scale)
    const long long cn = f == 0 ? c + 1 : f == 1 ? c - 1 : f == 2 ? c + p.nx : c - p.nx;
    const int fn = f == 0 ? 1 : f == 1 ? 0 : f == 2 ? 3 : 2;
    const int m = fn <= 1 ? 1 : 2;
    const real sg = (fn == 0 || fn == 2) ? 1.0 : -1.0;
    const real u0 = U[cn], u1x = U[N + cn], u1y = U[2 * N + cn];  // in real, as raw_limit
    real h4[4];
    h4[0] = u0 + u1x;
    h4[1] = u0 - u1x;
    h4[2] = u0 + u1y;
    h4[3] = u0 - u1y;
    const real qx = U[3 * N + cn] + sg * U[(3 + m) * N + cn];
    const real qy = U[6 * N + cn] + sg * U[(6 + m) * N + cn];
    oth = side_rec<real>(p, h4, qx, qy, U[cn], fn, p.Z[cn] + sg * p.Z[m * N + cn]);
  }
  LimT<real> ra, rb;
  real ha, za, hb, zb;
  const bool own_lower = f == 0 || f == 2;
  if (own_lower) revise_face_t(own[f], oth, p.tol, ra, rb, ha, za, hb, zb);
  else revise_face_t(oth, own[f], p.tol, ra, rb, ha, za, hb, zb);
  F = flux_face(ra, rb, f >= 2, p.g, p.tol);
  ho = own_lower ? ha : hb;
  zo = own_lower ? za : zb;
}

// L(U) at cell (i, j) in real (Eq. 4 with the fluxes of its four faces).  With
// rev, also writes the revised depth and bed of each face (planes 2f, 2f + 1 of
// faces E, W, N, S), which the reverse sweep's own-terms pass reads.
__device__ void cell_operator(const Prob& p, const store* __restrict__ U, int i, int j, real t,
                              real Q, real* L, store* __restrict__ rev = nullptr) {
  const long long c = (long long)j * p.nx + i;
  RecT<real> r[4];
  recs_double(p, U, c, r);
  F3T<real> F[4];
  real hs[4], zs[4], u[4], v[4];
  for (int f = 0; f < 4; ++f) {
    face_rev(p, U, i, j, f, Q, r, F[f], hs[f], zs[f]);
    u[f] = r[f].u;
    v[f] = r[f].v;
  }
  if (rev) {
    for (int f = 0; f < 4; ++f) {
      rev[(2 * f) * p.N + c] = hs[f];
      rev[(2 * f + 1) * p.N + c] = zs[f];
    }
  }
  own_terms<real>(p, hs, zs, u, v, L);
  const F3T<real> FE = F[0], FW = F[1], GN = F[2], GS = F[3];
  const real idx = p.inv_dx, idy = p.inv_dy, k3x = -3.0 * idx, k3y = -3.0 * idy;
  L[H0] += -(FE.h - FW.h) * idx - (GN.h - GS.h) * idy;
  L[QX0] += -(FE.x - FW.x) * idx - (GN.x - GS.x) * idy;
  L[QY0] += -(FE.y - FW.y) * idx - (GN.y - GS.y) * idy;
  L[H1X] += k3x * (FE.h + FW.h);
  L[QX1X] += k3x * (FE.x + FW.x);
  L[QY1X] += k3x * (FE.y + FW.y);
  L[H1Y] += k3y * (GN.h + GS.h);
  L[QX1Y] += k3y * (GN.x + GS.x);
  L[QY1Y] += k3y * (GN.y + GS.y);
  if (p.rain != 0.0 && t >= p.rain_t0 && t < p.rain_t1) L[H0] += p.rain;
}

// Wet-dry treatment after a stage (mass-neutral); returns the 9-bit mask of
// the modes it keeps.
__device__ __forceinline__ unsigned wetdry_mask(real* m, real z0, real z1x, real z1y,
                                                real tol) {
  const real h0 = m[H0];
  if (h0 <= tol) {
#pragma unroll
    for (int k = 1; k < 9; ++k) m[k] = 0.0;
    return 1u;
  }
  unsigned keep = 0x1FFu;
  const real eta0 = h0 + z0;
  {
    const bool fe = (h0 + m[H1X] <= tol) && !(z0 + z1x > eta0);
    const bool fw = (h0 - m[H1X] <= tol) && !(z0 - z1x > eta0);
    if (fe || fw) {
      m[H1X] = 0.0; m[QX1X] = 0.0; m[QY1X] = 0.0;
      keep &= ~((1u << H1X) | (1u << QX1X) | (1u << QY1X));
    }
  }
  {
    const bool fn = (h0 + m[H1Y] <= tol) && !(z0 + z1y > eta0);
    const bool fs = (h0 - m[H1Y] <= tol) && !(z0 - z1y > eta0);
    if (fn || fs) {
      m[H1Y] = 0.0; m[QX1Y] = 0.0; m[QY1Y] = 0.0;
      keep &= ~((1u << H1Y) | (1u << QX1Y) | (1u << QY1Y));
    }
  }
  return keep;
}

// Friction of one cell (Sec. 2.1.3, as the forward solver): modes m -> out.
template <class T>
__device__ __forceinline__ void friction_point_t(const T& gn2dt, real tol, const T& h, T& qx,
                                                 T& qy) {
  if (!(val(h) > tol)) return;
  const T qm = sqrt(qx * qx + qy * qy);
  const T den = 1.0 + gn2dt * qm / (h * h * cbrt(h));
  qx = qx / den;
  qy = qy / den;
}

template <class T>
__device__ __forceinline__ void friction_cell(const T* m, const T& n, real dt, real g, real tol,
                                              T* out) {
#pragma unroll
  for (int k = 0; k < 9; ++k) out[k] = m[k];
  const T gn2dt = dt * g * n * n;
  T cx = m[QX0], cy = m[QY0];
  friction_point_t(gn2dt, tol, m[H0], cx, cy);
  const real r3 = 1.0 / 1.7320508075688772, hs3 = 0.5 * 1.7320508075688772;
#pragma unroll
  for (int dd = 1; dd <= 2; ++dd) {
    const T h1 = m[dd], x1 = m[3 + dd], y1 = m[6 + dd];
    T xp = m[QX0] + x1 * r3, yp = m[QY0] + y1 * r3, xm = m[QX0] - x1 * r3, ym = m[QY0] - y1 * r3;
    friction_point_t(gn2dt, tol, m[H0] + h1 * r3, xp, yp);
    friction_point_t(gn2dt, tol, m[H0] - h1 * r3, xm, ym);
    out[3 + dd] = hs3 * (xp - xm);
    out[6 + dd] = hs3 * (yp - ym);
  }
  out[QX0] = cx;
  out[QY0] = cy;
}

// Reverse-mode adjoint of one friction point (friction_point_t): given the
// adjoints (wx, wy) of the updated discharges, adds the gradient into g_gn2dt,
// g_h, g_qx, g_qy (a dry point is the identity).
__device__ __forceinline__ void friction_point_adj(real gn2dt, real tol, real h, real qx, real qy,
                                                   real wx, real wy, real& g_gn2dt, real& g_h,
                                                   real& g_qx, real& g_qy) {
  if (!(h > tol)) {
    g_qx += wx;
    g_qy += wy;
    return;
  }
  const real qm = sqrt(qx * qx + qy * qy);
  const real D = h * h * cbrt(h);  // h^(7/3)
  const real den = 1.0 + gn2dt * qm / D;
  const real ox = qx / den, oy = qy / den;
  g_qx += wx / den;
  g_qy += wy / den;
  const real g_den = -(wx * ox + wy * oy) / den;
  g_gn2dt += g_den * qm / D;
  const real g_qm = g_den * gn2dt / D;
  const real g_D = -g_den * gn2dt * qm / (D * D);
  g_h += g_D * (7.0 / 3.0) * D / h;
  if (qm > 0.0) {
    g_qx += g_qm * qx / qm;
    g_qy += g_qm * qy / qm;
  }
}

// Reverse-mode adjoint of friction_cell: the gradient of ls . Fric(m; n) with
// respect to the modes m (g_m) and the Manning n (g_n).
__device__ __noinline__ void friction_cell_adj(const real* m, real n, real dt, real g, real tol,
                                               const real* ls, real* g_m, real& g_n) {
  const real gn2dt = dt * g * n * n;
  real g_gn2dt = 0.0;
  for (int k = 0; k < 9; ++k) g_m[k] = 0.0;
  // depth modes pass through
  g_m[H0] += ls[H0];
  g_m[H1X] += ls[H1X];
  g_m[H1Y] += ls[H1Y];
  // centre
  friction_point_adj(gn2dt, tol, m[H0], m[QX0], m[QY0], ls[QX0], ls[QY0], g_gn2dt, g_m[H0],
                     g_m[QX0], g_m[QY0]);
  const real r3 = 1.0 / 1.7320508075688772, hs3 = 0.5 * 1.7320508075688772;
  for (int dd = 1; dd <= 2; ++dd) {
    // out[3 + dd] = hs3 (xp - xm), out[6 + dd] = hs3 (yp - ym)
    const real wx = hs3 * ls[3 + dd], wy = hs3 * ls[6 + dd];
    const real h1 = m[dd], x1 = m[3 + dd], y1 = m[6 + dd];
    for (int sgn = 0; sgn < 2; ++sgn) {
      const real r = sgn == 0 ? r3 : -r3, w = sgn == 0 ? 1.0 : -1.0;
      real gh = 0.0, gx = 0.0, gy = 0.0;
      friction_point_adj(gn2dt, tol, m[H0] + h1 * r, m[QX0] + x1 * r, m[QY0] + y1 * r, w * wx,
                         w * wy, g_gn2dt, gh, gx, gy);
      g_m[H0] += gh;
      g_m[dd] += gh * r;
      g_m[QX0] += gx;
      g_m[3 + dd] += gx * r;
      g_m[QY0] += gy;
      g_m[6 + dd] += gy * r;
    }
  }
  // gn2dt = dt g n^2
  g_n = g_gn2dt * 2.0 * dt * g * n;
}

// ---------------------------------------------------------------------------
// Forward kernels (one thread per cell, dense planes)
// ---------------------------------------------------------------------------

__global__ void fwd_friction_kernel(Prob p, const store* __restrict__ U, store* __restrict__ Us,
                                    real dt) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p.N) return;
  real m[9], o[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) m[k] = U[k * p.N + c];
  friction_cell<real>(m, p.Nm[c], dt, p.g, p.tol, o);
#pragma unroll
  for (int k = 0; k < 9; ++k) Us[k * p.N + c] = o[k];
}

// Stage 1: U1 = W(Us + dt L(Us, t)); stage 2: Uo = W((Us + U1 + dt L(U1, t)) / 2).
template <int STAGE>
__global__ void fwd_stage_kernel(Prob p, const store* __restrict__ Us, const store* __restrict__ U1,
                                 store* __restrict__ Uo, unsigned short* __restrict__ mask, real dt,
                                 real t, real Q, store* __restrict__ rev) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p.N) return;
  const int i = (int)(c % p.nx), j = (int)(c / p.nx);
  const store* In = STAGE == 1 ? Us : U1;
  real L[9], o[9];
  cell_operator(p, In, i, j, t, Q, L, rev);
#pragma unroll
  for (int k = 0; k < 9; ++k)
    o[k] = STAGE == 1 ? Us[k * p.N + c] + dt * L[k]
                      : 0.5 * (Us[k * p.N + c] + U1[k * p.N + c] + dt * L[k]);
  const unsigned keep = wetdry_mask(o, p.Z[c], p.Z[p.N + c], p.Z[2 * p.N + c], p.tol);
  mask[c] = (unsigned short)keep;
#pragma unroll
  for (int k = 0; k < 9; ++k) Uo[k * p.N + c] = o[k];
}

// Sampled gauge depths max(0, planar h) of state U.
__global__ void gauge_kernel(const store* __restrict__ U, long long N, int ng,
                             const long long* __restrict__ gc, const store* __restrict__ gx,
                             const store* __restrict__ ge, store* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ng) return;
  const long long c = gc[k];
  const real h = U[c] + gx[k] * U[N + c] + ge[k] * U[2 * N + c];
  out[k] = h > 0.0 ? h : 0.0;
}

// lambda += dJ/dU for one sample: 2 (h - obs) (1, xi, eta) on the depth modes
// where the clipped depth is positive (one thread: gauges may share a cell).
__global__ void gauge_seed_kernel(store* __restrict__ lam, long long N, int ng,
                                  const long long* __restrict__ gc, const store* __restrict__ gx,
                                  const store* __restrict__ ge, const store* __restrict__ h,
                                  const store* __restrict__ obs) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int k = 0; k < ng; ++k) {
    if (!(h[k] > 0.0)) continue;
    const real r = 2.0 * (h[k] - obs[k]);
    const long long c = gc[k];
    lam[c] += r;
    lam[N + c] += r * gx[k];
    lam[2 * N + c] += r * ge[k];
  }
}

// ---------------------------------------------------------------------------
// Reverse kernels
// ---------------------------------------------------------------------------

// Adjoint mu of the operator output of a stage at cell c:
//   stage 2: mu = dt/2 * mask2 * lam2            (V2 = (Us + U1 + dt L) / 2)
//   stage 1: mu = dt * mask1 * lamU1             (V1 = Us + dt L)
__device__ __forceinline__ void stage_mu(const store* __restrict__ lam, const unsigned short* mask,
                                         long long N, long long c, real w, real* mu) {
  const unsigned m = mask[c];
#pragma unroll
  for (int k = 0; k < 9; ++k) mu[k] = ((m >> k) & 1u) ? w * lam[k * N + c] : 0.0;
}

// Per-cell pass of a stage, before the faces: the Jacobian of the cell's own
// terms (Eqs. 4-5 without the fluxes) with respect to its 12 raw limits
// (faces E, W, N, S; h, qx, qy each) and to the revised depth h* and bed z* of
// each of its four faces.  Writes OWN planes 0..11 (the raw limits' adjoints)
// and 12..19 (h*, z* of faces E, W, N, S).  rev holds the faces' revised
// depths and beds at this state, written by the stage's forward recomputation.
__global__ void adj_own_kernel(Prob p, const store* __restrict__ In, const store* __restrict__ lam,
                               const unsigned short* __restrict__ mask, real w,
                               const store* __restrict__ rev, store* __restrict__ OWN) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p.N) return;
  const long long N = p.N;
  real mu[9];
  stage_mu(lam, mask, N, c, w, mu);
  bool any = false;
#pragma unroll
  for (int k = 0; k < 9; ++k) any = any || mu[k] != 0.0;
  if (!any) {
    for (int q = 0; q < 20; ++q) OWN[q * N + c] = 0.0;
    return;
  }
  real lim[4][3];
  for (int f = 0; f < 4; ++f) raw_limit(In, N, c, f, lim[f][0], lim[f][1], lim[f][2]);
  // the faces' revised depths and beds (from the forward) and the records'
  // velocities at this state
  real hsv[4], zsv[4], ru[4], rv[4];
  {
    RecT<real> r[4];
    recs_double(p, In, c, r);
    for (int f = 0; f < 4; ++f) {
      hsv[f] = rev[(2 * f) * N + c];
      zsv[f] = rev[(2 * f + 1) * N + c];
      ru[f] = r[f].u;
      rv[f] = r[f].v;
    }
  }
  // The own terms depend on the raw limits only through the four face
  // velocities (u, v), and on the faces' h* and z* as inputs of their own: one
  // reverse sweep of the own terms gives the adjoints of all sixteen, and the
  // velocities' are taken to the 12 raw limits by a reverse sweep of the
  // records.
  real g_hs[4], g_zs[4], g_u[4], g_v[4];
  own_terms_adj(p, hsv, zsv, ru, rv, mu, g_hs, g_zs, g_u, g_v);
  for (int f = 0; f < 4; ++f) {
    OWN[(12 + 2 * f) * N + c] = g_hs[f];
    OWN[(13 + 2 * f) * N + c] = g_zs[f];
  }
  // the records' velocities depend on each face's limit and, through the
  // thin-limit threshold, on the mean depth (hE + hW) / 2
  real glim[4][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
  real g_h0 = 0.0;
  const real h0v = In[c];
  for (int f = 0; f < 4; ++f)
    rec_uv_adj(lim[f][0], lim[f][1], lim[f][2], p.wd != 0, p.tol, h0v, g_u[f], g_v[f], glim[f][0],
               glim[f][1], glim[f][2], g_h0);
  glim[0][0] += 0.5 * g_h0;
  glim[1][0] += 0.5 * g_h0;
  for (int f = 0; f < 4; ++f)
    for (int k = 0; k < 3; ++k) OWN[(3 * f + k) * N + c] = glim[f][k];
}

// One pass over the faces of a stage: face (left/lower cell a, right/upper cell
// b) of direction dir (0 x, 1 y); index f runs over (nx+1) * ny x-faces or
// nx * (ny+1) y-faces.  The face's outputs are its flux (adjoint phi from both
// cells' operator adjoints) and each side's revised depth and bed (adjoints
// from OWN); its inputs per side are the cell's four depth limits (E, W, N, S:
// they set the partially wet scale) and its discharge limits at this face.
// Writes the six input adjoints of each side (FL: a, FR: b; the boundary side
// folded into the own cell) and, for inflow faces, the adjoint of the
// hydrograph discharge.
__global__ void adj_face_kernel(Prob p, int dir, const store* __restrict__ In,
                                const store* __restrict__ lam, const unsigned short* __restrict__ mask,
                                real w, real Q, const store* __restrict__ OWN,
                                store* __restrict__ FL, store* __restrict__ FR,
                                store* __restrict__ gq_face) {
  const long long nfx = (long long)(p.nx + 1) * p.ny, nfy = (long long)p.nx * (p.ny + 1);
  const long long nf = dir == 0 ? nfx : nfy;
  const long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  int i, j;  // cell on the right / upper side (may be outside)
  if (dir == 0) { i = (int)(f % (p.nx + 1)); j = (int)(f / (p.nx + 1)); }
  else { i = (int)(f % p.nx); j = (int)(f / p.nx); }
  const long long N = p.N;
  const bool has_a = dir == 0 ? i > 0 : j > 0;
  const bool has_b = dir == 0 ? i < p.nx : j < p.ny;
  const long long cb = (long long)j * p.nx + i;
  const long long ca = dir == 0 ? cb - 1 : cb - p.nx;
  const real inv = dir == 0 ? p.inv_dx : p.inv_dy;
  const int l1 = dir == 0 ? 1 : 2;            // slope mode of the direction
  const int fa = dir == 0 ? 0 : 2, fb = dir == 0 ? 1 : 3;  // the face as seen from a and b
  // adjoints of the outputs: flux (3), a's h* and z*, b's h* and z*
  real phi[3] = {0.0, 0.0, 0.0}, pha = 0.0, pza = 0.0, phb = 0.0, pzb = 0.0;
  real mua[9], mub[9];
  if (has_a) {
    stage_mu(lam, mask, N, ca, w, mua);
    for (int v = 0; v < 3; ++v) phi[v] += -mua[3 * v] * inv - 3.0 * inv * mua[3 * v + l1];
    pha = OWN[(12 + 2 * fa) * N + ca];
    pza = OWN[(13 + 2 * fa) * N + ca];
  }
  if (has_b) {
    stage_mu(lam, mask, N, cb, w, mub);
    for (int v = 0; v < 3; ++v) phi[v] += mub[3 * v] * inv - 3.0 * inv * mub[3 * v + l1];
    phb = OWN[(12 + 2 * fb) * N + cb];
    pzb = OWN[(13 + 2 * fb) * N + cb];
  }
  real la[6] = {0, 0, 0, 0, 0, 0}, lb[6] = {0, 0, 0, 0, 0, 0}, gq = 0.0;
  const bool any = phi[0] != 0.0 || phi[1] != 0.0 || phi[2] != 0.0 || pha != 0.0 || pza != 0.0 ||
                   phb != 0.0 || pzb != 0.0;
  const bool y = dir == 1;
  if (any && has_a && has_b) {
    real ha4[4], hb4[4], qa[3], qb[3];
    for (int q = 0; q < 4; ++q) {
      real t1, t2;
      raw_limit(In, N, ca, q, ha4[q], t1, t2);
      raw_limit(In, N, cb, q, hb4[q], t1, t2);
    }
    raw_limit(In, N, ca, fa, qa[0], qa[1], qa[2]);
    raw_limit(In, N, cb, fb, qb[0], qb[1], qb[2]);
    const real za0 = p.Z[ca] + p.Z[l1 * N + ca], zb0 = p.Z[cb] - p.Z[l1 * N + cb];
    // The face's outputs depend on the inputs only through each side's record
    // (h, u, v, hs; its bed and partially wet flag are constants of the state).
    // Their adjoint is taken back to the eight record fields by one reverse
    // sweep of the revision and flux, then to each side's six inputs by a
    // reverse sweep of that side's record.
    const RecT<real> Ra = side_rec(p, ha4, qa[1], qa[2], In[ca], fa, za0);
    const RecT<real> Rb = side_rec(p, hb4, qb[1], qb[2], In[cb], fb, zb0);
    real grec[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    revise_flux_adj(Ra, Rb, y, p.g, p.tol, phi, pha, pza, phb, pzb, grec, grec + 4);
    side_rec_adj(p, ha4, qa[1], qa[2], In[ca], fa, grec, la);
    side_rec_adj(p, hb4, qb[1], qb[2], In[cb], fb, grec + 4, lb);
  } else if (!(has_a && has_b)) {
    // boundary face: the outside state is the ghost of the inside cell's limit
    const bool inside_b = has_b;
    const long long c = inside_b ? cb : ca;
    const int ci = inside_b ? i : (dir == 0 ? i - 1 : i);
    const int cj = inside_b ? j : (dir == 0 ? j : j - 1);
    const int fo = inside_b ? fb : fa;  // own face
    const int edge = dir == 0 ? (inside_b ? 0 : 1) : (inside_b ? 2 : 3);
    const real s = dir == 0 ? (cj + 0.5) * p.dy : (ci + 0.5) * p.dx;
    const real pho = inside_b ? phb : pha, pzo = inside_b ? pzb : pza;
    if (any) {
      real h4[4], qo[3];
      for (int q = 0; q < 4; ++q) {
        real t1, t2;
        raw_limit(In, N, c, q, h4[q], t1, t2);
      }
      raw_limit(In, N, c, fo, qo[0], qo[1], qo[2]);
      // seven inputs (the four depth limits, qx, qy, the discharge Q) in three
      // passes of three derivatives: boundary faces are few, and narrow duals
      // keep the kernel's registers for the interior faces
      const real sg = (fo == 0 || fo == 2) ? 1.0 : -1.0;
      const real zf = p.Z[c] + sg * p.Z[l1 * N + c];
      real lo7[9];
#pragma unroll 1
      for (int l0 = 0; l0 < 9; l0 += 3) {
        auto seed = [l0](real x, int input) {
          return input >= l0 && input < l0 + 3 ? var<3>(x, input - l0) : cst<3>(x);
        };
        Dual<3> O[4];
        for (int q = 0; q < 4; ++q) O[q] = seed(h4[q], q);
        const Dual<3> Qd = seed(Q, 6);
        const RecT<Dual<3>> Ro = side_rec(p, O, seed(qo[1], 4), seed(qo[2], 5), In[c], fo, zf);
        Dual<3> G[3] = {fo == 0 ? O[0] : fo == 1 ? O[1] : fo == 2 ? O[2] : O[3], seed(qo[1], 4),
                        seed(qo[2], 5)};
        ghost_t(p, edge, s, Qd, G[0], G[1], G[2]);
        const Dual<3> h0 = with_value(0.5 * (O[0] + O[1]), In[c]);
        const RecT<Dual<3>> Rg = make_rec_t(G[0], G[1], G[2], zf, false, h0 - h0 + 1.0, p.tol,
                                            false, h0);
        LimT<Dual<3>> ra, rb;
        Dual<3> ha, za, hb, zb;
        if (inside_b) revise_face_t(Rg, Ro, p.tol, ra, rb, ha, za, hb, zb);
        else revise_face_t(Ro, Rg, p.tol, ra, rb, ha, za, hb, zb);
        const F3T<Dual<3>> F = flux_face(ra, rb, y, p.g, p.tol);
        const Dual<3>& ho = inside_b ? hb : ha;
        const Dual<3>& zo = inside_b ? zb : za;
        for (int k = 0; k < 3; ++k)
          lo7[l0 + k] = phi[0] * F.h.d[k] + phi[1] * F.x.d[k] + phi[2] * F.y.d[k] +
                        pho * ho.d[k] + pzo * zo.d[k];
      }
      gq = lo7[6];
      for (int k = 0; k < 6; ++k) { if (inside_b) lb[k] = lo7[k]; else la[k] = lo7[k]; }
    }
    // fold into the edge slot index: along-edge position
    const int pos = dir == 0 ? cj : ci;
    const int slot = edge * (p.nx > p.ny ? p.nx : p.ny) + pos;
    gq_face[slot] = gq;
  }
  for (int k = 0; k < 6; ++k) {
    FL[k * nf + f] = la[k];
    FR[k * nf + f] = lb[k];
  }
}

// One pass over the cells of a stage.  Stage 2 writes lamU1 = mask2 lam2 / 2 +
// L'(U1)^T mu2.  Stage 1 writes lamUs = mask2 lam2 / 2 + mask1 lamU1 +
// L'(Us)^T mu1, then the friction adjoint: lam <- Fric'(U)^T lamUs and the
// Manning gradient.  The raw limits' adjoints are the own terms' (OWN) plus
// each of the four faces' for this side.
template <int STAGE>
__global__ void adj_cell_kernel(Prob p, const store* __restrict__ OWN,
                                const store* __restrict__ lam2, const unsigned short* __restrict__ mask2,
                                const unsigned short* __restrict__ mask1, const store* __restrict__ lamU1,
                                const store* __restrict__ FXL, const store* __restrict__ FXR,
                                const store* __restrict__ FYL, const store* __restrict__ FYR,
                                const store* __restrict__ U, real dt, store* __restrict__ out,
                                store* __restrict__ gn) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p.N) return;
  const long long N = p.N;
  const int i = (int)(c % p.nx), j = (int)(c / p.nx);
  const long long nfx = (long long)(p.nx + 1) * p.ny, nfy = (long long)p.nx * (p.ny + 1);
  real lr[4][3];
  for (int f = 0; f < 4; ++f)
    for (int k = 0; k < 3; ++k) lr[f][k] = OWN[(3 * f + k) * N + c];
  // faces: this cell is side a of its east and north faces, side b of its west and south
  const long long fe = (long long)j * (p.nx + 1) + i + 1, fw = (long long)j * (p.nx + 1) + i;
  const long long fn = (long long)(j + 1) * p.nx + i, fs = (long long)j * p.nx + i;
  const store* src[4] = {FXL, FXR, FYL, FYR};
  const long long fi[4] = {fe, fw, fn, fs};
  const long long fcount[4] = {nfx, nfx, nfy, nfy};
  for (int f = 0; f < 4; ++f) {
    const store* Fs = src[f];
    for (int q = 0; q < 4; ++q) lr[q][0] += Fs[q * fcount[f] + fi[f]];
    lr[f][1] += Fs[4 * fcount[f] + fi[f]];
    lr[f][2] += Fs[5 * fcount[f] + fi[f]];
  }
  // limits -> modes: E = U0 + U1x, W = U0 - U1x, N = U0 + U1y, S = U0 - U1y
  real a[9];
  for (int v = 0; v < 3; ++v) {
    a[3 * v] = lr[0][v] + lr[1][v] + lr[2][v] + lr[3][v];
    a[3 * v + 1] = lr[0][v] - lr[1][v];
    a[3 * v + 2] = lr[2][v] - lr[3][v];
  }
  // direct RK terms
  const unsigned m2 = mask2[c];
  real half2[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) half2[k] = ((m2 >> k) & 1u) ? 0.5 * lam2[k * N + c] : 0.0;
  if (STAGE == 2) {
#pragma unroll
    for (int k = 0; k < 9; ++k) out[k * N + c] = half2[k] + a[k];
    return;
  }
  const unsigned m1 = mask1[c];
  real ls[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) ls[k] = half2[k] + (((m1 >> k) & 1u) ? lamU1[k * N + c] : 0.0) + a[k];
  // friction: Us = Fric(U; n), its adjoint by one reverse sweep
  real m[9], gm[9], sn;
  for (int k = 0; k < 9; ++k) m[k] = U[k * N + c];
  friction_cell_adj(m, p.Nm[c], dt, p.g, p.tol, ls, gm, sn);
  for (int k = 0; k < 9; ++k) out[k * N + c] = gm[k];
  gn[c] += sn;
}

// Sum of the inflow faces' discharge adjoints in a fixed order into one slot:
// one block of kSumThreads threads, thread r summing entries r, r + kSumThreads,
// ... in turn, then a fixed pairwise tree over the threads (the same order on
// every call, so the gradient does not depend on scheduling).
constexpr int kSumThreads = 256;
__global__ void __launch_bounds__(kSumThreads) sum_gq_kernel(const store* __restrict__ gq_face,
                                                             int n, double* __restrict__ slot) {
  __shared__ double part[kSumThreads];
  const int r = threadIdx.x;
  double s = 0.0;
  for (int k = r; k < n; k += kSumThreads) s += gq_face[k];
  part[r] = s;
  __syncthreads();
  for (int w = kSumThreads / 2; w > 0; w >>= 1) {
    if (r < w) part[r] += part[r + w];
    __syncthreads();
  }
  if (r == 0) *slot = part[0];
}

}  // namespace DG2_ADJ_NS
}  // namespace dg2

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

namespace dg2 {
namespace DG2_ADJ_NS {
namespace {

int afail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  dg2::set_error_text(buf);
  return code;
}

#define ACU(call)                                                                       \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return afail(DG2_E_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));         \
  } while (0)

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct AdjLayout {
  size_t off_Z, off_Nm, off_U0, off_snap, off_work, off_Us, off_U1, off_m1, off_m2, off_lam,
      off_lamU1, off_tmp, off_own, off_rev, off_FXL, off_FXR, off_FYL, off_FYR, off_gq_face, off_gn, off_gidx,
      off_gxi, off_geta, off_gh, off_gq_step, total;
  long long N, nfx, nfy, plane9;
  int nsnap, ngq;
};

bool adj_layout(int nx, int ny, int nsnap, int max_gauges, int max_steps, AdjLayout& L) {
  if (nx < 1 || ny < 1 || nsnap < 1 || max_gauges < 0 || max_steps < 1) return false;
  L.N = (long long)nx * ny;
  L.nfx = (long long)(nx + 1) * ny;
  L.nfy = (long long)nx * (ny + 1);
  L.plane9 = 9 * L.N;
  L.nsnap = nsnap;
  L.ngq = 4 * (nx > ny ? nx : ny);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align_up(o + bytes);
    return at;
  };
  const size_t s9 = (size_t)L.plane9 * sizeof(store);
  L.off_Z = take(3 * (size_t)L.N * sizeof(store));
  L.off_Nm = take((size_t)L.N * sizeof(store));
  L.off_U0 = take(s9);
  L.off_snap = take((size_t)nsnap * s9);
  L.off_work = take(2 * s9);
  L.off_Us = take(s9);
  L.off_U1 = take(s9);
  L.off_m1 = take((size_t)L.N * sizeof(unsigned short));
  L.off_m2 = take((size_t)L.N * sizeof(unsigned short));
  L.off_lam = take(s9);
  L.off_lamU1 = take(s9);
  L.off_tmp = take(s9);
  L.off_own = take(20 * (size_t)L.N * sizeof(store));
  L.off_rev = take(16 * (size_t)L.N * sizeof(store));
  L.off_FXL = take(6 * (size_t)L.nfx * sizeof(store));
  L.off_FXR = take(6 * (size_t)L.nfx * sizeof(store));
  L.off_FYL = take(6 * (size_t)L.nfy * sizeof(store));
  L.off_FYR = take(6 * (size_t)L.nfy * sizeof(store));
  L.off_gq_face = take((size_t)L.ngq * sizeof(store));
  L.off_gn = take((size_t)L.N * sizeof(store));
  const size_t ng = max_gauges > 0 ? max_gauges : 1;
  L.off_gidx = take(ng * sizeof(long long));
  L.off_gxi = take(ng * sizeof(store));
  L.off_geta = take(ng * sizeof(store));
  L.off_gh = take(ng * sizeof(store));
  L.off_gq_step = take(2 * (size_t)max_steps * sizeof(double));
  L.total = o;
  return true;
}

}  // namespace

// An adjoint problem of this precision (the C ABI's dg2_adj wraps one).
struct Ctx {
  Prob p;
  AdjLayout lay;
  char* ws;
  cudaStream_t st;
  int max_gauges, max_steps;
  // problem
  std::vector<double> tk, qk;       // hydrograph knots (times, discharges)
  double t0;
  std::vector<double> dts;          // frozen step sizes
  std::vector<int> samp_step;       // step count after which each sample is taken
  std::vector<double> obs;          // [nsamp][ngauge]
  int ngauge;
  bool have_state, have_schedule;
  // per-run host results
  std::vector<double> gauge_h;      // [nsamp][ngauge] from the last forward
  int64_t fwd_steps, rev_steps;
};

namespace {

// Host FP64 values to device storage (converted on the host when it is FP32).
int upload(const double* src, size_t n, store* dst, cudaStream_t st) {
  if (sizeof(store) == sizeof(double)) {
    ACU(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyHostToDevice, st));
    return cudaStreamSynchronize(st) == cudaSuccess ? DG2_OK : afail(DG2_E_CUDA, "copy failed");
  }
  std::vector<store> tmp(src, src + n);
  ACU(cudaMemcpyAsync(dst, tmp.data(), n * sizeof(store), cudaMemcpyHostToDevice, st));
  ACU(cudaStreamSynchronize(st));
  return DG2_OK;
}

// Device storage to host FP64 values (synchronises the stream).
int download(const store* src, size_t n, double* dst, cudaStream_t st) {
  std::vector<store> tmp(n);
  ACU(cudaMemcpyAsync(tmp.data(), src, n * sizeof(store), cudaMemcpyDeviceToHost, st));
  ACU(cudaStreamSynchronize(st));
  for (size_t k = 0; k < n; ++k) dst[k] = (double)tmp[k];
  return DG2_OK;
}

store* dptr(Ctx* a, size_t off) { return (store*)(a->ws + off); }
store* snap(Ctx* a, int s) { return dptr(a, a->lay.off_snap) + (size_t)s * a->lay.plane9; }

double hydro(const Ctx* a, double t) {
  const std::vector<double>& tk = a->tk;
  const std::vector<double>& qk = a->qk;
  if (tk.empty()) return 0.0;
  if (t <= tk[0]) return qk[0];
  for (size_t k = 0; k + 1 < tk.size(); ++k)
    if (t <= tk[k + 1]) {
      const double w = (t - tk[k]) / (tk[k + 1] - tk[k]);
      return qk[k] + w * (qk[k + 1] - qk[k]);
    }
  return qk.back();
}

// dQ(t)/dq_k added into g with weight s
void hydro_grad(const Ctx* a, double t, double s, double* g) {
  const std::vector<double>& tk = a->tk;
  if (tk.empty()) return;
  if (t <= tk[0]) { g[0] += s; return; }
  for (size_t k = 0; k + 1 < tk.size(); ++k)
    if (t <= tk[k + 1]) {
      const double w = (t - tk[k]) / (tk[k + 1] - tk[k]);
      g[k] += s * (1.0 - w);
      g[k + 1] += s * w;
      return;
    }
  g[tk.size() - 1] += s;
}

double step_time(const Ctx* a, int k) {
  // t_k = t0 + dt_0 + ... + dt_{k-1}, summed in step order as the forward does
  double t = a->t0;
  for (int q = 0; q < k; ++q) t += a->dts[q];
  return t;
}

int launch_ok() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return afail(DG2_E_CUDA, "kernel launch failed: %s", cudaGetErrorString(e));
  return DG2_OK;
}

unsigned blocks(long long n) { return (unsigned)((n + 255) / 256); }

// One forward step k from Uin to Uout (Us, U1, masks left in the workspace;
// with keep_rev also each stage's revised face depths and beds).
int fwd_step(Ctx* a, int k, double t, const store* Uin, store* Uout, bool keep_rev = false) {
  const double dt = a->dts[k];
  store* Us = dptr(a, a->lay.off_Us);
  store* U1 = dptr(a, a->lay.off_U1);
  unsigned short* m1 = (unsigned short*)(a->ws + a->lay.off_m1);
  unsigned short* m2 = (unsigned short*)(a->ws + a->lay.off_m2);
  const unsigned nb = blocks(a->lay.N);
  fwd_friction_kernel<<<nb, 256, 0, a->st>>>(a->p, Uin, Us, dt);
  store* rev = dptr(a, a->lay.off_rev);
  const long long r8 = 8 * (long long)a->lay.N;
  fwd_stage_kernel<1><<<nb, 256, 0, a->st>>>(a->p, Us, nullptr, U1, m1, dt, t, hydro(a, t),
                                             keep_rev ? rev : nullptr);
  fwd_stage_kernel<2><<<nb, 256, 0, a->st>>>(a->p, Us, U1, Uout, m2, dt, t + dt, hydro(a, t + dt),
                                             keep_rev ? rev + r8 : nullptr);
  a->fwd_steps++;
  return launch_ok();
}

// Advances `buf` (the state after `from` steps) to the state after `to` steps.
int advance(Ctx* a, store* buf, int from, int to) {
  store* w = dptr(a, a->lay.off_work);
  double t = step_time(a, from);
  const size_t s9 = (size_t)a->lay.plane9 * sizeof(store);
  for (int k = from; k < to; ++k) {
    int r = fwd_step(a, k, t, buf, w);
    if (r) return r;
    ACU(cudaMemcpyAsync(buf, w, s9, cudaMemcpyDeviceToDevice, a->st));
    t += a->dts[k];
  }
  return DG2_OK;
}

// Reverse of step k from state Uk: lam (adjoint of the state after step k)
// becomes the adjoint of Uk; Manning gradient and discharge adjoints added.
int rev_step(Ctx* a, int k, const store* Uk) {
  const AdjLayout& L = a->lay;
  const double dt = a->dts[k];
  const double t = step_time(a, k);
  store* Us = dptr(a, L.off_Us);
  store* U1 = dptr(a, L.off_U1);
  store* w = dptr(a, L.off_work);
  unsigned short* m1 = (unsigned short*)(a->ws + L.off_m1);
  unsigned short* m2 = (unsigned short*)(a->ws + L.off_m2);
  int r = fwd_step(a, k, t, Uk, w, true);  // Us, U1, masks, revised faces of this step
  if (r) return r;
  a->fwd_steps--;                     // counted as part of the reverse step
  store* lam = dptr(a, L.off_lam);
  store* lamU1 = dptr(a, L.off_lamU1);
  store* tmp = dptr(a, L.off_tmp);
  store* OWN = dptr(a, L.off_own);
  store* FXL = dptr(a, L.off_FXL);
  store* FXR = dptr(a, L.off_FXR);
  store* FYL = dptr(a, L.off_FYL);
  store* FYR = dptr(a, L.off_FYR);
  store* gqf = dptr(a, L.off_gq_face);
  store* gn = dptr(a, L.off_gn);
  double* gqs = (double*)(a->ws + L.off_gq_step);
  const unsigned nb = blocks(L.N);
  // stage 2 at U1, time t + dt: mu2 = dt/2 mask2 lam
  ACU(cudaMemsetAsync(gqf, 0, (size_t)L.ngq * sizeof(store), a->st));
  const store* rev = dptr(a, L.off_rev);
  adj_own_kernel<<<nb, 256, 0, a->st>>>(a->p, U1, lam, m2, 0.5 * dt, rev + 8 * (long long)L.N, OWN);
  adj_face_kernel<<<blocks(L.nfx), 256, 0, a->st>>>(a->p, 0, U1, lam, m2, 0.5 * dt, hydro(a, t + dt),
                                                    OWN, FXL, FXR, gqf);
  adj_face_kernel<<<blocks(L.nfy), 256, 0, a->st>>>(a->p, 1, U1, lam, m2, 0.5 * dt, hydro(a, t + dt),
                                                    OWN, FYL, FYR, gqf);
  sum_gq_kernel<<<1, kSumThreads, 0, a->st>>>(gqf, L.ngq, gqs + 2 * (size_t)k + 1);
  adj_cell_kernel<2><<<nb, 256, 0, a->st>>>(a->p, OWN, lam, m2, m1, nullptr, FXL, FXR, FYL, FYR,
                                            nullptr, dt, lamU1, gn);
  // stage 1 at Us, time t: mu1 = dt mask1 lamU1
  ACU(cudaMemsetAsync(gqf, 0, (size_t)L.ngq * sizeof(store), a->st));
  adj_own_kernel<<<nb, 256, 0, a->st>>>(a->p, Us, lamU1, m1, dt, rev, OWN);
  adj_face_kernel<<<blocks(L.nfx), 256, 0, a->st>>>(a->p, 0, Us, lamU1, m1, dt, hydro(a, t), OWN, FXL,
                                                    FXR, gqf);
  adj_face_kernel<<<blocks(L.nfy), 256, 0, a->st>>>(a->p, 1, Us, lamU1, m1, dt, hydro(a, t), OWN, FYL,
                                                    FYR, gqf);
  sum_gq_kernel<<<1, kSumThreads, 0, a->st>>>(gqf, L.ngq, gqs + 2 * (size_t)k);
  adj_cell_kernel<1><<<nb, 256, 0, a->st>>>(a->p, OWN, lam, m2, m1, lamU1, FXL, FXR, FYL, FYR, Uk,
                                            dt, tmp, gn);
  ACU(cudaMemcpyAsync(lam, tmp, (size_t)L.plane9 * sizeof(store), cudaMemcpyDeviceToDevice, a->st));
  a->rev_steps++;
  return launch_ok();
}

// Adds dJ/dU of the samples taken after `k` steps into lam.
int seed_samples(Ctx* a, int k) {
  const AdjLayout& L = a->lay;
  const int ns = (int)a->samp_step.size();
  for (int s = 0; s < ns; ++s) {
    if (a->samp_step[s] != k) continue;
    store* gh = dptr(a, L.off_gh);
    int r = upload(a->gauge_h.data() + (size_t)s * a->ngauge, a->ngauge, gh, a->st);
    if (r) return r;
    // observed depths staged behind the gauge depths in the same small buffer is
    // not possible (max_gauges slots); stage them in the tmp plane instead
    store* ob = dptr(a, L.off_tmp);
    r = upload(a->obs.data() + (size_t)s * a->ngauge, a->ngauge, ob, a->st);
    if (r) return r;
    gauge_seed_kernel<<<1, 32, 0, a->st>>>(dptr(a, L.off_lam), L.N, a->ngauge,
                                           (const long long*)(a->ws + L.off_gidx), dptr(a, L.off_gxi),
                                           dptr(a, L.off_geta), gh, ob);
    r = launch_ok();
    if (r) return r;
  }
  return DG2_OK;
}

// Binomial checkpointing (treeverse): reverse steps s..e-1; the state after s
// steps is in snapshot `slot`; `free` further slots (slot+1 ..) are usable.
double binom(int c, int r) {
  double b = 1.0;
  for (int k = 1; k <= c; ++k) b = b * (r + k) / k;
  return b;
}

int reverse_range(Ctx* a, int s, int e, int slot, int free) {
  const size_t s9 = (size_t)a->lay.plane9 * sizeof(store);
  if (e - s == 1) {
    int r = rev_step(a, s, snap(a, slot));
    if (r) return r;
    return seed_samples(a, s);
  }
  if (free == 0) {
    // no slot left: recompute from s for each step
    store* w2 = dptr(a, a->lay.off_work) + a->lay.plane9;
    for (int k = e - 1; k >= s; --k) {
      ACU(cudaMemcpyAsync(w2, snap(a, slot), s9, cudaMemcpyDeviceToDevice, a->st));
      int r = advance(a, w2, s, k);
      if (!r) r = rev_step(a, k, w2);
      if (!r) r = seed_samples(a, k);
      if (r) return r;
    }
    return DG2_OK;
  }
  const int t = e - s;
  int rr = 1;
  while (binom(free, rr) < t) ++rr;
  // the right part takes the steps that free - 1 slots reverse with rr sweeps
  double right = binom(free - 1, rr);
  int nr = right >= t - 1 ? t - 1 : (int)right;
  if (nr < 1) nr = 1;
  const int m = e - nr;
  const int ns = slot + 1;
  ACU(cudaMemcpyAsync(snap(a, ns), snap(a, slot), s9, cudaMemcpyDeviceToDevice, a->st));
  int r = advance(a, snap(a, ns), s, m);
  if (!r) r = reverse_range(a, m, e, ns, free - 1);
  if (!r) r = reverse_range(a, s, m, slot, free);
  return r;
}

int check_adj(Ctx* a) {
  if (!a) return afail(DG2_E_ARG, "null adjoint context");
  if (!a->have_state) return afail(DG2_E_STATE, "dg2_adj_set_problem first");
  if (!a->have_schedule) return afail(DG2_E_STATE, "dg2_adj_set_schedule first");
  return DG2_OK;
}

// Forward over all steps from U0; gauge depths of every sample to the host;
// returns J.
int forward_all(Ctx* a, double* loss) {
  const AdjLayout& L = a->lay;
  const int K = (int)a->dts.size();
  const size_t s9 = (size_t)L.plane9 * sizeof(store);
  store* cur = snap(a, 0);
  ACU(cudaMemcpyAsync(cur, dptr(a, L.off_U0), s9, cudaMemcpyDeviceToDevice, a->st));
  const int ns = (int)a->samp_step.size();
  a->gauge_h.assign((size_t)ns * a->ngauge, 0.0);
  store* w = dptr(a, L.off_work);
  double t = a->t0;
  auto sample = [&](int k) -> int {
    for (int s = 0; s < ns; ++s) {
      if (a->samp_step[s] != k) continue;
      store* gh = dptr(a, L.off_gh);
      gauge_kernel<<<1, 256, 0, a->st>>>(cur, L.N, a->ngauge, (const long long*)(a->ws + L.off_gidx),
                                         dptr(a, L.off_gxi), dptr(a, L.off_geta), gh);
      int r = launch_ok();
      if (r) return r;
      r = download(gh, a->ngauge, a->gauge_h.data() + (size_t)s * a->ngauge, a->st);
      if (r) return r;
    }
    return DG2_OK;
  };
  int r = sample(0);
  for (int k = 0; k < K && !r; ++k) {
    r = fwd_step(a, k, t, cur, w);
    if (!r) {
      cudaError_t e = cudaMemcpyAsync(cur, w, s9, cudaMemcpyDeviceToDevice, a->st);
      if (e != cudaSuccess) r = afail(DG2_E_CUDA, "copy failed: %s", cudaGetErrorString(e));
    }
    t += a->dts[k];
    if (!r) r = sample(k + 1);
  }
  if (r) return r;
  ACU(cudaStreamSynchronize(a->st));
  double J = 0.0;
  for (size_t q = 0; q < a->gauge_h.size(); ++q) {
    const double d = a->gauge_h[q] - a->obs[q];
    J += d * d;
  }
  if (!std::isfinite(J)) return afail(DG2_E_NONFINITE, "non-finite misfit");
  *loss = J;
  return DG2_OK;
}

}  // namespace

// The entry points of this precision (the C ABI dispatches to them).


size_t workspace_bytes(int nx, int ny, int nsnap, int max_gauges, int max_steps) {
  AdjLayout L;
  if (!adj_layout(nx, ny, nsnap, max_gauges, max_steps, L)) return 0;
  return L.total;
}

int create(Ctx** out, int nx, int ny, double dx, double dy, const dg2_params* prm, int nsnap,
           int max_gauges, int max_steps, void* dev_workspace, size_t ws_bytes, void* cuda_stream) {
  if (!out) return afail(DG2_E_ARG, "out is null");
  *out = nullptr;
  if (!prm) return afail(DG2_E_ARG, "params is null");
  if (prm->variant != DG2_NL || prm->flux != DG2_HLL ||
      prm->scheme != DG2_SCHEME_DG2 ||
      (prm->wetdry != DG2_WD_POSITIVE && prm->wetdry != DG2_WD_PRINTED))
    return afail(DG2_E_ARG, "the adjoint is of the DG2-NL step with the HLL flux");
  if (!(dx > 0.0) || !(dy > 0.0)) return afail(DG2_E_ARG, "dx, dy must be > 0");
  AdjLayout L;
  if (!adj_layout(nx, ny, nsnap, max_gauges, max_steps, L))
    return afail(DG2_E_ARG, "bad sizes (nx, ny, nsnap, max_steps >= 1; max_gauges >= 0)");
  if (!dev_workspace || ((uintptr_t)dev_workspace % kAlign))
    return afail(DG2_E_ARG, "workspace must be non-null and 256-byte aligned");
  if (ws_bytes < L.total) return afail(DG2_E_NOMEM, "workspace too small: %zu < %zu", ws_bytes, L.total);
  Ctx* a = new Ctx();
  a->lay = L;
  a->ws = (char*)dev_workspace;
  a->st = (cudaStream_t)cuda_stream;
  a->max_gauges = max_gauges;
  a->max_steps = max_steps;
  Prob& p = a->p;
  memset(&p, 0, sizeof p);
  p.nx = nx; p.ny = ny; p.N = L.N;
  p.dx = dx; p.dy = dy; p.inv_dx = 1.0 / dx; p.inv_dy = 1.0 / dy;
  p.g = prm->g; p.tol = prm->tol_dry;
  p.wd = prm->wetdry == DG2_WD_POSITIVE ? 1 : 0;
  for (int k = 0; k < 4; ++k) p.bc[k] = prm->bc[k];
  p.in_edge = -1;
  p.Z = dptr(a, L.off_Z);
  p.Nm = dptr(a, L.off_Nm);
  a->t0 = 0.0;
  a->ngauge = 0;
  a->have_state = a->have_schedule = false;
  a->fwd_steps = a->rev_steps = 0;
  *out = a;
  return DG2_OK;
}

int set_problem(Ctx* a, const double* z3, const double* state9, double t0, const double* manning,
                int inflow_edge, double s0, double len, const double* t_knots,
                const double* q_knots, int nknots, const double* gauge_xy, int ngauge) {
  if (!a) return afail(DG2_E_ARG, "null adjoint context");
  if (!z3 || !state9 || !manning) return afail(DG2_E_ARG, "z3, state9 and manning are required");
  if (ngauge < 0 || ngauge > a->max_gauges) return afail(DG2_E_ARG, "ngauge must be 0..%d", a->max_gauges);
  if (ngauge > 0 && !gauge_xy) return afail(DG2_E_ARG, "gauge_xy is null");
  if (inflow_edge >= 0) {
    if (inflow_edge > 3 || !t_knots || !q_knots || nknots < 1 || nknots > kMaxKnotsAdj)
      return afail(DG2_E_ARG, "inflow needs edge 0..3 and 1..%d knots", kMaxKnotsAdj);
    for (int k = 1; k < nknots; ++k)
      if (!(t_knots[k] > t_knots[k - 1])) return afail(DG2_E_ARG, "t_knots must increase");
  }
  const AdjLayout& L = a->lay;
  Prob& p = a->p;
  const size_t N = (size_t)L.N;
  int r = upload(z3, 3 * N, dptr(a, L.off_Z), a->st);
  if (!r) r = upload(state9, 9 * N, dptr(a, L.off_U0), a->st);
  if (!r) r = upload(manning, N, dptr(a, L.off_Nm), a->st);
  if (r) return r;
  a->t0 = t0;
  p.in_edge = inflow_edge;
  a->tk.clear();
  a->qk.clear();
  if (inflow_edge >= 0) {
    a->tk.assign(t_knots, t_knots + nknots);
    a->qk.assign(q_knots, q_knots + nknots);
    const bool ew = inflow_edge <= 1;
    const int n = ew ? p.ny : p.nx;
    const double h = ew ? p.dy : p.dx;
    int nf = 0;
    for (int k = 0; k < n; ++k) {
      const double s = (k + 0.5) * h;
      if (s >= s0 && s <= s0 + len) ++nf;
    }
    if (nf == 0) return afail(DG2_E_ARG, "no face centre lies in the inflow segment");
    p.in_s0 = s0;
    p.in_s1 = s0 + len;
    p.in_width = nf * h;
  }
  std::vector<long long> gi(ngauge > 0 ? ngauge : 1);
  std::vector<double> gx(ngauge > 0 ? ngauge : 1), ge(ngauge > 0 ? ngauge : 1);
  for (int k = 0; k < ngauge; ++k) {
    int i = (int)std::floor(gauge_xy[2 * k] / p.dx), j = (int)std::floor(gauge_xy[2 * k + 1] / p.dy);
    i = i < 0 ? 0 : (i >= p.nx ? p.nx - 1 : i);
    j = j < 0 ? 0 : (j >= p.ny ? p.ny - 1 : j);
    gi[k] = (long long)j * p.nx + i;
    gx[k] = (gauge_xy[2 * k] - (i + 0.5) * p.dx) / (0.5 * p.dx);
    ge[k] = (gauge_xy[2 * k + 1] - (j + 0.5) * p.dy) / (0.5 * p.dy);
  }
  if (ngauge > 0) {
    ACU(cudaMemcpyAsync(a->ws + L.off_gidx, gi.data(), ngauge * sizeof(long long), cudaMemcpyHostToDevice, a->st));
    if ((r = upload(gx.data(), ngauge, dptr(a, L.off_gxi), a->st))) return r;
    if ((r = upload(ge.data(), ngauge, dptr(a, L.off_geta), a->st))) return r;
  }
  ACU(cudaStreamSynchronize(a->st));
  a->ngauge = ngauge;
  a->have_state = true;
  return DG2_OK;
}

int set_params(Ctx* a, const double* manning, const double* q_knots) {
  if (!a || !a->have_state) return afail(DG2_E_STATE, "dg2_adj_set_problem first");
  if (manning) {
    const int r = upload(manning, (size_t)a->lay.N, dptr(a, a->lay.off_Nm), a->st);
    if (r) return r;
  }
  if (q_knots) a->qk.assign(q_knots, q_knots + a->qk.size());
  ACU(cudaStreamSynchronize(a->st));
  return DG2_OK;
}

int set_schedule(Ctx* a, const double* dts, int nsteps, const int* sample_steps, int nsamples,
                 const double* obs) {
  if (!a || !a->have_state) return afail(DG2_E_STATE, "dg2_adj_set_problem first");
  if (!dts || nsteps < 1 || nsteps > a->max_steps)
    return afail(DG2_E_ARG, "need 1..%d step sizes", a->max_steps);
  for (int k = 0; k < nsteps; ++k)
    if (!(dts[k] > 0.0) || !std::isfinite(dts[k])) return afail(DG2_E_ARG, "step %d: dt must be > 0", k);
  if (nsamples < 0 || (nsamples > 0 && (!sample_steps || !obs)))
    return afail(DG2_E_ARG, "bad samples");
  for (int s = 0; s < nsamples; ++s)
    if (sample_steps[s] < 0 || sample_steps[s] > nsteps)
      return afail(DG2_E_ARG, "sample %d: step must be 0..%d", s, nsteps);
  a->dts.assign(dts, dts + nsteps);
  a->samp_step.assign(sample_steps, sample_steps + nsamples);
  a->obs.assign(obs, obs + (size_t)nsamples * a->ngauge);
  a->have_schedule = true;
  return DG2_OK;
}

int forward(Ctx* a, double* loss, double* gauge_h) {
  int r = check_adj(a);
  if (r) return r;
  double J;
  if ((r = forward_all(a, &J))) return r;
  if (loss) *loss = J;
  if (gauge_h) memcpy(gauge_h, a->gauge_h.data(), a->gauge_h.size() * sizeof(double));
  return DG2_OK;
}

int gradient(Ctx* a, double* loss, double* grad_manning, double* grad_q) {
  int r = check_adj(a);
  if (r) return r;
  const AdjLayout& L = a->lay;
  const int K = (int)a->dts.size();
  double J;
  if ((r = forward_all(a, &J))) return r;
  ACU(cudaMemsetAsync(dptr(a, L.off_lam), 0, (size_t)L.plane9 * sizeof(store), a->st));
  ACU(cudaMemsetAsync(dptr(a, L.off_gn), 0, (size_t)L.N * sizeof(store), a->st));
  ACU(cudaMemsetAsync(a->ws + L.off_gq_step, 0, 2 * (size_t)K * sizeof(double), a->st));
  if ((r = seed_samples(a, K))) return r;
  // snapshot 0 holds U0 again (forward_all advanced it in place)
  ACU(cudaMemcpyAsync(snap(a, 0), dptr(a, L.off_U0), (size_t)L.plane9 * sizeof(store),
                      cudaMemcpyDeviceToDevice, a->st));
  if ((r = reverse_range(a, 0, K, 0, L.nsnap - 1))) return r;
  if (grad_manning && (r = download(dptr(a, L.off_gn), (size_t)L.N, grad_manning, a->st)))
    return r;
  std::vector<double> gqs(2 * (size_t)K);
  ACU(cudaMemcpyAsync(gqs.data(), a->ws + L.off_gq_step, gqs.size() * sizeof(double),
                      cudaMemcpyDeviceToHost, a->st));
  ACU(cudaStreamSynchronize(a->st));
  if (grad_q) {
    std::vector<double> g(a->qk.size(), 0.0);
    double t = a->t0;
    for (int k = 0; k < K; ++k) {
      hydro_grad(a, t, gqs[2 * (size_t)k], g.data());
      hydro_grad(a, t + a->dts[k], gqs[2 * (size_t)k + 1], g.data());
      t += a->dts[k];
    }
    memcpy(grad_q, g.data(), g.size() * sizeof(double));
  }
  if (loss) *loss = J;
  return DG2_OK;
}

int counts(const Ctx* a, int64_t* forward_steps, int64_t* reverse_steps) {
  if (!a) return afail(DG2_E_ARG, "null adjoint context");
  if (forward_steps) *forward_steps = a->fwd_steps;
  if (reverse_steps) *reverse_steps = a->rev_steps;
  return DG2_OK;
}

int destroy(Ctx* a) {
  if (!a) return afail(DG2_E_ARG, "null adjoint context");
  delete a;
  return DG2_OK;
}

}  // namespace DG2_ADJ_NS
}  // namespace dg2
