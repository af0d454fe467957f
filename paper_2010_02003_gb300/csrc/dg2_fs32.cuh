// dg2_fs32.cuh -- FP32 free-surface form of the DG2 step (sm_103a).
//
// The bulk update runs in FP32 on free-surface modes eta0, eta1x, eta1y
// (eta = h + z) and the discharge modes; simulated time, the step size, the
// Courant reduction, the mass ledger and every reduction stay in FP64.
//
// Momentum is written in deviation form.  With h* + z* = eta at every face
// (the revision of Sec. 2.1.2 gives z* = z when h >= 0 and z* = z + h = eta
// when h < 0), the pressure and bed terms of Eq. 4 regroup exactly:
//   Eq. 4a:  dF/dx + 2g h0x z1x / dx  ==  dF_dev/dx + g h0x (eta_E - eta_W) / dx
//   Eq. 4b:  (F_E + F_W) - (F(G+) + F(G-)) + (2g/3) h1x z1x
//        ==  (F_E,dev + F_W,dev) - (F_dev(G+) + F_dev(G-)) + (2g/3) h1x eta1x_bar
// where every *_dev flux is the flux minus the hydrostatic pressure g h^2 / 2
// of the cell's own limit (of the Gauss point for F_dev(G)), and the HLL flux
// is evaluated directly in that deviation form.  Topography is stored as face
// values, so both sides of a face see the same z.  Still water (flat eta,
// q = 0) then gives every term exactly zero in FP32: the lake at rest survives
// rounding, including water held by high ground (clipped limits).
#pragma once
#include "dg2_device.cuh"

namespace dg2 {
namespace f32 {

enum { E0 = 0, E1X, E1Y };  // free-surface modes occupy the h slots
// eta0 is carried as an unevaluated pair hi + lo of FP32 values: plane E0 holds
// hi, plane E0L the remainder lo (|lo| <= half an ulp of hi), updated with
// error-free TwoSum.  One FP32 ulp of the free surface over terrain of a few
// metres is ~1e-6 m, coarser than a rain increment per step or a thin film;
// the pair resolves the depth and conserves mass, all on FP32 units.
enum { E0L = 9 };
constexpr int kPlanes32 = 10;

// s + e == a + b exactly (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

struct __align__(16) D32 {
  int nx, ny, pitch;   // cell planes: ny rows of `pitch` floats
  int zpx;             // x-face topography plane: ny rows of `zpx` floats (nx+1 used)
  long long plane;     // ny * pitch
  float dx, dy, inv_dx, inv_dy, g, tol, ds;
  double dxd, dyd, cfl, dt_max;
  int bc[4];
  int n_in;
  InflowDesc in[kMaxInflow];
  const double* knot_t;
  const double* knot_q;
  double rain, rain_t0, rain_t1, qp;
  long long src_idx;
  float* S;            // 10 planes: eta0 eta1x eta1y qx0 qx1x qx1y qy0 qy1x qy1y, eta0 lo
  float* T;            // 10 planes: stage state
  float* Q;            // 6 planes written by stage 1 for stage 2: DG2-LL the limited slopes
                       // of Un, DG2-NL Un's discharge modes after friction
  const float* ZX;     // z at x-faces: face i of row j at ZX[j * zpx + i], i = 0..nx
  const float* ZY;     // z at y-faces: face j of column i at ZY[j * pitch + i], j = 0..ny
  const float* N;      // Manning n
  double* bpart;
  double* mpart;
  Scalars* sc;
  int ngauge, max_samples;
  const long long* g_idx;
  const double* g_xi;
  const double* g_eta;
  double* samp_t;
  double* samp_h;
  int nblocks;
  Tiles tiles;
  int wd;              // 1: positivity-consistent revision of partially wet cells
};

struct LimF {
  float h, qx, qy, u, v;
};

// Face flux in deviation form: mass, normal momentum minus the LEFT side's
// pressure, tangential momentum, and dP = g (hL^2 - hR^2) / 2 so that the
// right-referenced normal momentum is fn + dP.
struct FaceF {
  float h, n, t, dp;
};

__device__ __forceinline__ LimF revise32(float h, float qx, float qy, float tol) {
  LimF r;
  if (h > tol) {
    r.u = qx / h;
    r.v = qy / h;
  } else {
    r.u = 0.f;
    r.v = 0.f;
  }
  r.h = h > 0.f ? h : 0.f;
  r.qx = r.h * r.u;
  r.qy = r.h * r.v;
  return r;
}

// HLL (same wave speeds as the FP64 path) returned relative to the left pressure.
// A face on a tile edge is evaluated by the edge thread of each tile beside it,
// inside code inlined at different places; every product that could be fused
// with a sum is therefore written as an explicit __fmaf_rn / __fmul_rn /
// __fadd_rn, so the compiler's contraction choices cannot differ between the
// copies and the flux does not depend on where the tile edges fall.
__device__ __forceinline__ FaceF hll_dev(float hL, float qnL, float qtL, float unL, float utL,
                                         float hR, float qnR, float qtR, float unR, float utR,
                                         float g, float tol) {
  FaceF f;
  const float hg = __fmul_rn(0.5f, g);
  f.dp = __fmul_rn(__fmul_rn(hg, __fadd_rn(hL, -hR)), __fadd_rn(hL, hR));
  if (hL <= tol && hR <= tol) {
    f.h = 0.f; f.n = -__fmul_rn(__fmul_rn(hg, hL), hL); f.t = 0.f;
    return f;
  }
  const float cL = sqrtf(__fmul_rn(g, hL)), cR = sqrtf(__fmul_rn(g, hR));
  float sL, sR;
  if (hL <= tol) {
    sL = __fmaf_rn(-2.f, cR, unR);
    sR = __fadd_rn(unR, cR);
  } else if (hR <= tol) {
    sL = __fadd_rn(unL, -cL);
    sR = __fmaf_rn(2.f, cL, unL);
  } else {
    const float us = __fadd_rn(__fmaf_rn(0.5f, __fadd_rn(unL, unR), cL), -cR);
    const float cs = __fmaf_rn(0.25f, __fadd_rn(unL, -unR), __fmul_rn(0.5f, __fadd_rn(cL, cR)));
    sL = fminf(__fadd_rn(unL, -cL), __fadd_rn(us, -cs));
    sR = fmaxf(__fadd_rn(unR, cR), __fadd_rn(us, cs));
  }
  const float mL = __fmul_rn(hL, unL), mR = __fmul_rn(hR, unR);
  const float fLh = mL, fLn = __fmul_rn(mL, unL), fLt = __fmul_rn(mL, utL);
  const float fRh = mR, fRn = __fmaf_rn(mR, unR, -f.dp), fRt = __fmul_rn(mR, utR);
  if (sL >= 0.f) {
    f.h = fLh; f.n = fLn; f.t = fLt;
    return f;
  }
  if (sR <= 0.f) {
    f.h = fRh; f.n = fRn; f.t = fRt;
    return f;
  }
  const float inv = 1.f / __fadd_rn(sR, -sL), sLR = __fmul_rn(sL, sR);
  f.h = __fmul_rn(__fmaf_rn(sR, fLh, __fmaf_rn(-sL, fRh, __fmul_rn(sLR, __fadd_rn(hR, -hL)))), inv);
  f.n = __fmul_rn(__fmaf_rn(sR, fLn, __fmaf_rn(-sL, fRn, __fmul_rn(sLR, __fadd_rn(qnR, -qnL)))), inv);
  f.t = __fmul_rn(__fmaf_rn(sR, fLt, __fmaf_rn(-sL, fRt, __fmul_rn(sLR, __fadd_rn(qtR, -qtL)))), inv);
  return f;
}

__device__ __forceinline__ FaceF flux_x32(const LimF& L, const LimF& R, float g, float tol) {
  return hll_dev(L.h, L.qx, L.qy, L.u, L.v, R.h, R.qx, R.qy, R.u, R.v, g, tol);
}
__device__ __forceinline__ FaceF flux_y32(const LimF& S, const LimF& N, float g, float tol) {
  return hll_dev(S.h, S.qy, S.qx, S.v, S.u, N.h, N.qy, N.qx, N.v, N.u, g, tol);
}

// Pressure-free physical flux of a Gauss point along x (h u, h u^2, h u v) or y.
__device__ __forceinline__ void gauss_dev(float h, float qx, float qy, float tol, bool ydir,
                                          float& fh, float& fx, float& fy) {
  float u = 0.f, v = 0.f;
  if (h > tol) {
    u = qx / h;
    v = qy / h;
  }
  if (!ydir) {
    fh = h * u; fx = h * u * u; fy = h * u * v;
  } else {
    fh = h * v; fx = h * u * v; fy = h * v * v;
  }
}

static __device__ void ghost32(const D32& d, int edge, float s, double t, float& h, float& qx,
                        float& qy) {
  for (int k = 0; k < d.n_in; ++k) {
    const InflowDesc& f = d.in[k];
    if (f.edge != edge || s < f.s0 || s > f.s1) continue;
    const double* tk = d.knot_t + f.koff;
    const double* qk = d.knot_q + f.koff;
    double Q = qk[f.nk - 1];
    if (t <= tk[0]) {
      Q = qk[0];
    } else {
      for (int k2 = 0; k2 + 1 < f.nk; ++k2)
        if (t <= tk[k2 + 1]) {
          Q = qk[k2] + (t - tk[k2]) / (tk[k2 + 1] - tk[k2]) * (qk[k2 + 1] - qk[k2]);
          break;
        }
    }
    const float qin = (float)(Q / f.width);
    const float hin = h > 0.f ? h : 0.f;
    const float hc = cbrtf(qin * qin / d.g);
    const float hg = hin > hc ? hin : hc;
    const float qn = (edge == 0 || edge == 2) ? qin : -qin;
    h = hg;
    if (edge <= 1) { qx = qn; qy = 0.f; } else { qx = 0.f; qy = qn; }
    return;
  }
  if (d.bc[edge] == 1) {
    if (edge == 0 && qx > 0.f) qx = 0.f;
    if (edge == 1 && qx < 0.f) qx = 0.f;
    if (edge == 2 && qy > 0.f) qy = 0.f;
    if (edge == 3 && qy < 0.f) qy = 0.f;
    return;
  }
  if (edge <= 1) qx = -qx; else qy = -qy;
}

__device__ __forceinline__ float minmod3f(float a, float b, float c) {
  if (a > 0.f && b > 0.f && c > 0.f) return fminf(fminf(a, b), c);
  if (a < 0.f && b < 0.f && c < 0.f) return fmaxf(fmaxf(a, b), c);
  return 0.f;
}

__device__ __forceinline__ float limit_comp32(float thresh, float tol, float half, float k0w,
                                              float k1w, float k0, float k1, float k0e,
                                              float k1e) {
  // evaluated for a cell by its own thread and, at a tile edge, by the
  // neighbouring tile's edge thread: explicit roundings (see hll_dev)
  const float r3 = 0.57735026918962576f;  // 1 / sqrt(3)
  const float jE = fabsf((k0e - k1e) - (k0 + k1));
  const float jW = fabsf((k0 - k1) - (k0w + k1w));
  float mag = fmaxf(fabsf(__fmaf_rn(-k1, r3, k0)), fabsf(__fmaf_rn(k1, r3, k0)));
  if (mag < tol) mag = tol;
  if (!(fmaxf(jE, jW) > __fmul_rn(__fmul_rn(thresh, half), mag))) return k1;
  return minmod3f(k1, k0e - k0, k0 - k0w);
}

__device__ __forceinline__ void cell_z(const D32& d, int i, int j, float& z0, float& z1x,
                                       float& z1y, float& zE, float& zW, float& zN, float& zS) {
  zW = d.ZX[(long long)j * d.zpx + i];
  zE = d.ZX[(long long)j * d.zpx + i + 1];
  zS = d.ZY[(long long)j * d.pitch + i];
  zN = d.ZY[(long long)(j + 1) * d.pitch + i];
  z0 = 0.5f * (zE + zW);
  z1x = 0.5f * (zE - zW);
  z1y = 0.5f * (zN - zS);
}

// Wet-dry treatment in free-surface variables (same rule as the FP64 path):
// a zeroed depth slope is eta1 = z1.
__device__ __forceinline__ void wetdry32(float* m, float lo, float z0, float z1x, float z1y,
                                         float zE, float zW, float zN, float zS, float tol) {
  const float h0 = (m[E0] - z0) + lo;
  if (h0 <= tol) {
    m[E1X] = z1x; m[E1Y] = z1y;
#pragma unroll
    for (int k = 3; k < 9; ++k) m[k] = 0.f;
    return;
  }
  const float eta0 = m[E0];
  {
    const bool fe = (((m[E0] - zE) + m[E1X]) + lo <= tol) && !(zE > eta0);
    const bool fw = (((m[E0] - zW) - m[E1X]) + lo <= tol) && !(zW > eta0);
    if (fe || fw) { m[E1X] = z1x; m[QX1X] = 0.f; m[QY1X] = 0.f; }
  }
  {
    const bool fn = (((m[E0] - zN) + m[E1Y]) + lo <= tol) && !(zN > eta0);
    const bool fs = (((m[E0] - zS) - m[E1Y]) + lo <= tol) && !(zS > eta0);
    if (fn || fs) { m[E1Y] = z1y; m[QX1Y] = 0.f; m[QY1Y] = 0.f; }
  }
}

__device__ __forceinline__ float rate32(const D32& d, float h0, float qx0, float qy0) {
  if (!(h0 > d.tol)) return 0.f;
  const float u = qx0 / h0, v = qy0 / h0, c = sqrtf(d.g * h0);
  return fmaxf((fabsf(u) + c) * d.inv_dx, (fabsf(v) + c) * d.inv_dy);
}

static __device__ void schedule32(const D32& d, Scalars* sc, double lam) {
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

// Initial modes from FP64 corner data: face-average topography (rounded to
// FP32 once), free-surface modes by Eq. 3, dry cells with eta modes equal to
// the FP32 topography modes (zero depth exactly).
static __global__ void init32_kernel(D32 d, const double* __restrict__ zc, const double* __restrict__ ec,
                              const double* __restrict__ man, double n_uniform, float* ZXw,
                              float* ZYw, float* Nw) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int W = d.nx + 1;
  // face topography: x-face (i, j) for i <= nx, y-face (i, j) for j <= ny
  if (i <= d.nx && j < d.ny)
    ZXw[(long long)j * d.zpx + i] = (float)(0.5 * (zc[(long long)j * W + i] + zc[(long long)(j + 1) * W + i]));
  if (i < d.nx && j <= d.ny)
    ZYw[(long long)j * d.pitch + i] = (float)(0.5 * (zc[(long long)j * W + i] + zc[(long long)j * W + i + 1]));
  if (i >= d.nx || j >= d.ny) return;
  const long long P = d.plane, c = (long long)j * d.pitch + i;
  const double* r0 = zc + (long long)j * W;
  const double* r1 = zc + (long long)(j + 1) * W;
  // FP32 topography modes exactly as the stage kernels will form them
  const float zW = (float)(0.5 * (r0[i] + r1[i])), zE = (float)(0.5 * (r0[i + 1] + r1[i + 1]));
  const float zS = (float)(0.5 * (r0[i] + r0[i + 1])), zN = (float)(0.5 * (r1[i] + r1[i + 1]));
  const float z0 = 0.5f * (zE + zW), z1x = 0.5f * (zE - zW), z1y = 0.5f * (zN - zS);
  float e0 = z0, e0l = 0.f, e1x = z1x, e1y = z1y;
  if (ec) {
    const double* e0r = ec + (long long)j * W;
    const double* e1r = ec + (long long)(j + 1) * W;
    // depth modes decide wetness exactly as in FP64 (Eq. 3 on eta - z)
    const double a = e0r[i] - r0[i], b = e0r[i + 1] - r0[i + 1];
    const double cc = e1r[i] - r1[i], dd = e1r[i + 1] - r1[i + 1];
    const double h0 = 0.5 * (0.5 * (b + dd) + 0.5 * (a + cc));
    if (h0 > 0.0) {
      const double fE = 0.5 * (e0r[i + 1] + e1r[i + 1]), fW = 0.5 * (e0r[i] + e1r[i]);
      const double fN = 0.5 * (e1r[i] + e1r[i + 1]), fS = 0.5 * (e0r[i] + e0r[i + 1]);
      const double e0d = 0.5 * (fE + fW);
      e0 = (float)e0d;
      e0l = (float)(e0d - (double)e0);
      e1x = (float)(0.5 * (fE - fW));
      e1y = (float)(0.5 * (fN - fS));
    }
  }
  float* S = d.S;
  S[E0 * P + c] = e0;
  S[E0L * P + c] = e0l;
  S[E1X * P + c] = e1x;
  S[E1Y * P + c] = e1y;
#pragma unroll
  for (int k = 3; k < 9; ++k) S[k * P + c] = 0.f;
  Nw[c] = (float)(man ? man[(long long)j * d.nx + i] : n_uniform);
}

// One side of a face: the planar limit's depth h (free-surface form: eta_face
// - z_face) and velocities (tol rule), the depth the face may draw on (hs:
// max(0, h), scaled for a partially wet cell), and whether the side's cell is
// partially wet.  Both sides share the face bed, so the revision below works
// in heights above it.
struct RecF {
  float h, u, v, hs;
  int pw;
};

// A face flux in deviation form plus the lower (west / south) side's revised depth.
struct FaceR32 {
  FaceF f;
  float ha;
};

// Face depths (hi - z_face) +- eta1 + lo of a cell from its free-surface modes:
// hi - z_face is exact for shallow water (Sterbenz), and both sides of a face
// form it from the same terms at rest.
__device__ __forceinline__ void face_depths32(float e0, float e1x, float e1y, float lo, float zE,
                                              float zW, float zN, float zS, float& eh, float& wh,
                                              float& nh, float& sh) {
  eh = ((e0 - zE) + e1x) + lo;
  wh = ((e0 - zW) - e1x) + lo;
  nh = ((e0 - zN) + e1y) + lo;
  sh = ((e0 - zS) - e1y) + lo;
}

// Partially wet test and depth scale of a cell (average depth h0, face depths
// W, E, S, N); wd = 0 keeps the printed revision (never partially wet).
__device__ __forceinline__ bool pw_scale32(float h0, float hW, float hE, float hS, float hN,
                                           float tol, int wd, float& sc) {
  sc = 1.f;
  if (!wd || !(h0 > tol)) return false;
  if (!(hW < 0.f || hE < 0.f || hS < 0.f || hN < 0.f)) return false;
  const float sum = __fadd_rn(__fadd_rn(__fadd_rn(fmaxf(hW, 0.f), fmaxf(hE, 0.f)), fmaxf(hS, 0.f)),
                              fmaxf(hN, 0.f));
  sc = __fdiv_rn(h0, __fmul_rn(0.25f, sum));
  return true;
}

// Velocities by the tol rule; under the default revision (thin), the
// desingularised velocity of the FP64 path at a limit thinner than h0 / 10.
__device__ __forceinline__ RecF make_rec32(float h, float qx, float qy, bool pw, float sc,
                                           float tol, bool thin = false, float h0 = 0.f) {
  RecF r;
  r.h = h;
  r.u = 0.f;
  r.v = 0.f;
  const float eps = __fmul_rn(0.1f, h0);
  if (thin && eps > tol && h < eps) {
    const float hp = h > 0.f ? h : 0.f;
    const float den = __fmaf_rn(h, h, __fmul_rn(eps, eps));
    const float k = __fdiv_rn(__fmul_rn(2.f, hp), den);
    r.u = __fmul_rn(k, qx);
    r.v = __fmul_rn(k, qy);
  } else if (h > tol) {
    r.u = qx / h;
    r.v = qy / h;
  }
  const float hp = h > 0.f ? h : 0.f;
  r.hs = pw ? __fmul_rn(sc, hp) : hp;
  r.pw = pw ? 1 : 0;
  return r;
}

// Revision of the face between lower side a and upper side b (the rule of the
// FP64 path): neither side partially wet, h* = max(0, h); otherwise the
// free-surface revision on the sides' own bed levels, z* = max(za, zb),
// h* = max(0, eta - z*), here in heights above the shared face bed (the free
// surface at h, or hs on a side that is not partially wet; the own bed at
// h - hs, or 0).
// Either way h* + z* is the side's own face free surface, so the deviation
// form of the pressure and bed terms holds.  Written with explicit roundings:
// a face on a tile edge is revised by both tiles beside it.
__device__ __forceinline__ void revise_face32(const RecF& a, const RecF& b, float tol, LimF& ra,
                                              LimF& rb) {
  if (!a.pw && !b.pw) {
    // the flux's velocities follow the tol rule on the revised depth
    ra.h = a.hs; ra.u = a.hs > tol ? a.u : 0.f; ra.v = a.hs > tol ? a.v : 0.f;
    rb.h = b.hs; rb.u = b.hs > tol ? b.u : 0.f; rb.v = b.hs > tol ? b.v : 0.f;
  } else {
    const float ea = a.pw ? a.h : a.hs, eb = b.pw ? b.h : b.hs;
    const float oa = a.pw ? __fadd_rn(a.h, -a.hs) : 0.f;
    const float ob = b.pw ? __fadd_rn(b.h, -b.hs) : 0.f;
    // the side whose bed is z* keeps its offered depth exactly; the other side
    // lies (its free surface - that side's) above it: no thin depth is formed as
    // a difference of two large heights, and equal free surfaces give equal depths
    if (oa >= ob) {
      ra.h = a.hs;
      rb.h = fmaxf(__fadd_rn(a.hs, __fadd_rn(eb, -ea)), 0.f);
    } else {
      rb.h = b.hs;
      ra.h = fmaxf(__fadd_rn(b.hs, __fadd_rn(ea, -eb)), 0.f);
    }
    ra.u = ra.h > tol ? a.u : 0.f; ra.v = ra.h > tol ? a.v : 0.f;
    rb.u = rb.h > tol ? b.u : 0.f; rb.v = rb.h > tol ? b.v : 0.f;
  }
  ra.qx = __fmul_rn(ra.h, a.u); ra.qy = __fmul_rn(ra.h, a.v);
  rb.qx = __fmul_rn(rb.h, b.u); rb.qy = __fmul_rn(rb.h, b.v);
}

// Per-block constants of an RK stage (dt, stage time, rain flag), read once per
// tile; the stage itself is in dg2_fs32_staged.cuh.
struct Blk32 {
  float dt, rainf;
  float gdt;  // friction's g dt (FP32 of the FP64 product)
  double dtd, ts;
  int rain;
  int skip;  // the problem has reached t_end: leave its tiles
};

// Time, ledger, gauges and the next step; opens the next step's tile lists.
// Run by one block of kFinThreads threads per problem.
static __device__ void finalize32_body(const D32& d, int lists_only) {
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
      const double area = d.dxd * d.dyd * (double)d.nx * (double)d.ny;
      if (d.rain != 0.0 && t >= d.rain_t0 && t < d.rain_t1) src1 += d.rain * area;
      if (d.rain != 0.0 && t + dt >= d.rain_t0 && t + dt < d.rain_t1) src2 += d.rain * area;
      if (d.src_idx >= 0) { src1 += d.qp; src2 += d.qp; }
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
            const int gi = (int)(gc % d.pitch), gj = (int)(gc / d.pitch);
            float gz0, gz1x, gz1y, a, b, e, f;
            cell_z(d, gi, gj, gz0, gz1x, gz1y, a, b, e, f);
            const double h = ((double)d.S[gc] - (double)gz0) + (double)d.S[E0L * P + gc] +
                             d.g_xi[k] * (double)(d.S[P + gc] - gz1x) +
                             d.g_eta[k] * (double)(d.S[2 * P + gc] - gz1y);
            d.samp_h[(long long)r * d.ngauge + k] = h > 0.0 ? h : 0.0;
          }
        }
        sc->nsamp = r + 1;
        sc->next_sample += sc->sample_every;
      }
      if (!(dt > 0.0) || !isfinite(tn)) sc->nonfinite = 1;
      sc->steps += 1;
      sc->last_dt = dt;
      schedule32(d, sc, __longlong_as_double((long long)sc->lam_bits));
      if (!sc->fixed_dt && sc->t >= sc->t_end) sc->done = 1;
      sc->tiles_done += sc->n_act;
    }
  }
  if (threadIdx.x == 0) open_lists(sc);
}

static __global__ void __launch_bounds__(256) rate32_kernel(D32 d) {
  __shared__ double red[32];
  __shared__ bool last;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  double lam = 0.0;
  if (i < d.nx && j < d.ny) {
    const long long P = d.plane, c = (long long)j * d.pitch + i;
    float z0, z1x, z1y, zE, zW, zN, zS;
    cell_z(d, i, j, z0, z1x, z1y, zE, zW, zN, zS);
    lam = (double)rate32(d, (d.S[c] - z0) + d.S[E0L * P + c], d.S[QX0 * P + c], d.S[QY0 * P + c]);
  }
  const double bl = block_max<256>(lam, red);
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  Scalars* sc = d.sc;
  if (tid == 0) {
    if (bl > 0.0) atomicMax(&sc->lam_bits, (unsigned long long)__double_as_longlong(bl));
    __threadfence();
    last = atomicAdd(&sc->count, 1u) == gridDim.x * gridDim.y - 1;
  }
  __syncthreads();
  if (last && tid == 0) {
    __threadfence();
    schedule32(d, sc, __longlong_as_double((long long)atomicAdd(&sc->lam_bits, 0ull)));
    sc->count = 0u;
  }
}

// Mass sum(eta0 - z0) dx dy, accumulated in FP64 in a fixed order.
static __global__ void __launch_bounds__(256) mass32_kernel(D32 d) {
  __shared__ double red[32];
  __shared__ bool last;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  double v = 0.0;
  if (i < d.nx && j < d.ny) {
    float z0, z1x, z1y, zE, zW, zN, zS;
    cell_z(d, i, j, z0, z1x, z1y, zE, zW, zN, zS);
    const long long c = (long long)j * d.pitch + i;
    v = ((double)d.S[c] - (double)z0) + (double)d.S[E0L * d.plane + c];
  }
  const double s = block_sum<256>(v, red);
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nb = gridDim.x * gridDim.y;
  Scalars* sc = d.sc;
  if (tid == 0) {
    d.mpart[blockIdx.y * gridDim.x + blockIdx.x] = s;
    __threadfence();
    last = atomicAdd(&sc->count, 1u) == (unsigned int)nb - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double part = 0.0;
  for (int k = tid; k < nb; k += 256) part += __ldcg(&d.mpart[k]);
  const double tot = block_sum<256>(part, red);
  if (tid == 0) {
    sc->mass = tot * d.dxd * d.dyd;
    if (sc->ledger_init) {
      sc->ledger = sc->mass;
      sc->ledger_init = 0;
    }
    sc->count = 0u;
  }
}

}  // namespace f32
}  // namespace dg2
