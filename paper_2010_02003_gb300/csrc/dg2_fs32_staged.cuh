// dg2_fs32_staged.cuh -- the FP32 free-surface RK stage on a tile staged in
// shared memory, with friction fused into the stages (sm_103a).
//
// One block computes one BX x BY tile of cells (one thread per cell) of one
// problem.  Everything the stage reads is first copied into shared memory by
// 16-byte asynchronous copies (cp.async), issued by every thread at once and
// waited for once: the tile's input state planes over the tile and a halo of
// H = 1 (DG2-NL) or 2 (DG2-LL) cells, the face beds around them, and (stage 1)
// the Manning n of those cells; stage 2 also stages the cells' own U^n.
// Columns are staged from i0 - 4 to i0 + BX + 3, so every copy is 16-byte
// aligned (the plane pitch is a multiple of 32 floats).  The arithmetic then
// reads shared memory only, in the phases of dg2_fs32.cuh's stage: face
// records of the tile and of the halo cells beside it, one revision and one
// flux per face, the operator of Eqs. 4-5 and the RK update.
//
// Friction (Sec. 2.1.3, implicit splitting once per step before stage 1) is
// applied here instead of in a pass of its own: stage 1 applies it to every
// staged cell in shared memory before anything else reads them (a cell's
// friction depends on that cell alone, so the halo cells of a tile get exactly
// the values their own tile computes).  Stage 2 needs the post-friction U^n
// for the RK average: in DG2-NL stage 1 stores its own cells' six discharge
// modes after friction in Q (stage 2 reads them in place of U^n's, so it
// evaluates no friction); in DG2-LL, whose Q holds the limited slopes of U^n,
// stage 2 recomputes the averages' friction (the same function with explicit
// roundings inside it, on depths formed alike), so stage 2 averages the U^n
// stage 1 stepped from.
#pragma once
#include "dg2_fs32.cuh"

namespace dg2 {
namespace f32 {

// 16-byte global -> shared copy, asynchronous (cp.async, L2 only).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// waits until at most one committed group of the thread's copies is in flight
__device__ __forceinline__ void cp_async_wait_but_one() {
  asm volatile("cp.async.wait_group 1;\n" ::: "memory");
}

// Row pitch of a 16-wide tile's staging (floats).  48 puts the two rows a warp
// reads at once on disjoint bank halves; 24 (no padding) halves the staging's
// shared memory at the cost of two-way conflicts on half the lanes, and measured
// faster on GB300 (ms per step, 48 -> 24: 2000 x 1000 fully wet DG2-NL 0.331 ->
// 0.323, DG2-LL 0.436 -> 0.413; the floodplain at 1 h DG2-LL 0.090 -> 0.084),
// more resident blocks outweighing the conflicts.
#ifndef DG2_SP16
#define DG2_SP16 24
#endif

// Staged geometry of a BX x BY tile with a halo of H cells.
template <bool LL, int BX, int BY>
struct Geo32 {
  static constexpr int H = LL ? 2 : 1;
  static constexpr int X0 = 4;                   // staged column of the tile's first cell
  static constexpr int SW = BX + 8;              // staged columns: i0 - 4 .. i0 + BX + 3
  static constexpr int Q4 = SW / 4;              // 16-byte copies per staged row
  // row pitch in shared memory (a multiple of 4 floats, for the 16-byte copies)
  static constexpr int SP = BX == 16 ? DG2_SP16 : SW;
  static_assert(SP >= SW && SP % 4 == 0, "staged rows hold the staged columns, 16-byte aligned");
  static constexpr int SR = BY + 2 * H;          // staged rows: j0 - H .. j0 + BY + H - 1
  static constexpr int PL = SR * SP;             // floats per staged plane
};

// Planes of U^n a stage-2 tile stages for its own cells: DG2-NL the four
// depth planes (eta0 hi / lo and its slopes) and the six discharge modes after
// friction stage 1 left in Q; DG2-LL eta0 hi / lo, qx0, qy0, the six limited
// slopes stage 1 left in Q and the Manning n.
constexpr int kOwn32 = 11;

template <bool LL, int STAGE, int BX, int BY>
struct __align__(16) StagedSmem32 {
  using G = Geo32<LL, BX, BY>;
  union {
    struct {
      __align__(16) float u[kPlanes32][G::PL];        // staged input state (eta0 hi 0, lo 9)
      __align__(16) float n[STAGE == 1 ? G::PL : 4];  // Manning n of the staged cells (stage 1)
      __align__(16) float zx[G::SR][G::SP];           // bed of x-face i at column i - (i0 - 4)
      __align__(16) float zy[G::SR + 1][G::SP];       // bed of y-face j at row j - (j0 - H)
    } st;
    struct {
      FaceR32 fx[BY][BX + 1];
      FaceR32 fy[BY + 1][BX];
    } fc;                                      // after the records: one flux per face
  };
  __align__(16) float own[STAGE == 2 ? kOwn32 : 1][BY][BX];  // stage 2: own cells' U^n
  RecF e[BY][BX];
  RecF n[BY][BX];
  RecF hw[BY], he[BY], hs[BX], hn[BX];
  double red[32];
  float redf[32];
};

// Friction of one cell's modes (Sec. 2.1.3): the point-implicit update at the
// centre and at the Gauss points +-1/sqrt(3) of both centrelines, the slopes
// rebuilt by differencing.  Every product that could fuse with a sum is an
// explicit intrinsic, the divisions are __fdividef, and h^(-7/3) is r^7 with
// r = h^(-1/3) from 2^(-log2(h) / 3) on the hardware's base-2 logarithm and
// exponential, refined by one Newton step r <- r (4 - h r^3) / 3 (which squares
// its relative error, ~1e-5 for thin films, to FP32 rounding), so each call
// site gives the same bits.  q = {qx0, qx1x, qx1y, qy0, qy1x, qy1y}; h1x, h1y
// are depth slopes.
__device__ __forceinline__ void friction_point32x(float gn2dt, float tol, float h, float& qx,
                                                  float& qy) {
  if (!(h > tol)) return;
  const float qm = sqrtf(__fmaf_rn(qx, qx, __fmul_rn(qy, qy)));
  float r = exp2f(__fmul_rn(-0.333333343f, __log2f(h)));
  r = __fmul_rn(__fmul_rn(r, __fmaf_rn(-h, __fmul_rn(__fmul_rn(r, r), r), 4.f)), 0.333333343f);
  const float r3 = __fmul_rn(__fmul_rn(r, r), r);
  const float hm73 = __fmul_rn(__fmul_rn(r3, r3), r);
  const float den = __fmaf_rn(__fmul_rn(gn2dt, qm), hm73, 1.f);
  qx = __fdividef(qx, den);
  qy = __fdividef(qy, den);
}

// centre only: the averages' discharges
__device__ __forceinline__ void friction_centre32(float gdt, float n, float tol, float h0,
                                                  float& qx0, float& qy0) {
  if (n == 0.f) return;
  friction_point32x(__fmul_rn(__fmul_rn(gdt, n), n), tol, h0, qx0, qy0);
}

__device__ __forceinline__ void friction_modes32(float gdt, float n, float tol, float h0,
                                                 float h1x, float h1y, float q[6]) {
  if (n == 0.f) return;
  const float r3 = 0.57735026918962576f, hs3 = 0.86602540378443865f;
  if (!(h0 > tol)) {
    // a dry average can still have wet Gauss points only through slopes, which
    // the wet-dry treatment zeroes; nothing to do then
    const bool any = __fmaf_rn(fabsf(h1x), r3, h0) > tol || __fmaf_rn(fabsf(h1y), r3, h0) > tol;
    if (!any) return;
  }
  const float gn2dt = __fmul_rn(__fmul_rn(gdt, n), n);
  const float x0 = q[0], y0 = q[3];
  float cx = x0, cy = y0;
  friction_point32x(gn2dt, tol, h0, cx, cy);
  float nq[2][2];
#pragma unroll
  for (int dd = 0; dd < 2; ++dd) {
    const float h1 = dd == 0 ? h1x : h1y;
    const float x1 = q[1 + dd], y1 = q[4 + dd];
    float xp = __fmaf_rn(x1, r3, x0), yp = __fmaf_rn(y1, r3, y0);
    float xm = __fmaf_rn(-x1, r3, x0), ym = __fmaf_rn(-y1, r3, y0);
    friction_point32x(gn2dt, tol, __fmaf_rn(h1, r3, h0), xp, yp);
    friction_point32x(gn2dt, tol, __fmaf_rn(-h1, r3, h0), xm, ym);
    nq[dd][0] = __fmul_rn(hs3, __fadd_rn(xp, -xm));
    nq[dd][1] = __fmul_rn(hs3, __fadd_rn(yp, -ym));
  }
  q[0] = cx;
  q[3] = cy;
  q[1] = nq[0][0];
  q[4] = nq[0][1];
  q[2] = nq[1][0];
  q[5] = nq[1][1];
}

// Bed of a staged cell (row r, column x of the staging): mean, slopes and the
// four face values.
template <class SM>
__device__ __forceinline__ void staged_z(const SM& sm, int r, int x, float& z0, float& z1x,
                                         float& z1y, float& zE, float& zW, float& zN, float& zS) {
  zW = sm.st.zx[r][x];
  zE = sm.st.zx[r][x + 1];
  zS = sm.st.zy[r][x];
  zN = sm.st.zy[r + 1][x];
  z0 = 0.5f * (zE + zW);
  z1x = 0.5f * (zE - zW);
  z1y = 0.5f * (zN - zS);
}

// Limited slopes (eta, qx, qy) along dir (1 x, 2 y) of the staged cell (r, x),
// which lies inside the grid at (gi, gj): Eqs. 6-7 as limited_slopes32.
template <int SP, class SM>
__device__ __forceinline__ void staged_limited(const D32& d, const SM& sm, int r, int x, int gi,
                                               int gj, int dir, float& se, float& sqx,
                                               float& sqy) {
  const int c = r * SP + x;
  se = sm.st.u[dir][c];
  sqx = sm.st.u[3 + dir][c];
  sqy = sm.st.u[6 + dir][c];
  const bool lo = dir == 1 ? gi > 0 : gj > 0;
  const bool hi = dir == 1 ? gi + 1 < d.nx : gj + 1 < d.ny;
  if (!lo || !hi) return;
  const int cl = dir == 1 ? c - 1 : c - SP, ch = dir == 1 ? c + 1 : c + SP;
  const int rl = dir == 1 ? r : r - 1, xl = dir == 1 ? x - 1 : x;
  const int rh = dir == 1 ? r : r + 1, xh = dir == 1 ? x + 1 : x;
  float z0, z1x, z1y, zE, zW, zN, zS;
  staged_z(sm, rl, xl, z0, z1x, z1y, zE, zW, zN, zS);
  const float hl = (sm.st.u[E0][cl] - z0) + sm.st.u[E0L][cl];
  staged_z(sm, r, x, z0, z1x, z1y, zE, zW, zN, zS);
  const float hc = (sm.st.u[E0][c] - z0) + sm.st.u[E0L][c];
  staged_z(sm, rh, xh, z0, z1x, z1y, zE, zW, zN, zS);
  const float hh = (sm.st.u[E0][ch] - z0) + sm.st.u[E0L][ch];
  if (hl <= d.tol || hc <= d.tol || hh <= d.tol) return;
  const float half = 0.5f * (dir == 1 ? d.dx : d.dy);
  const float* k0 = sm.st.u[E0];
  const float* k1 = sm.st.u[dir];
  se = limit_comp32(d.ds, d.tol, half, k0[cl], k1[cl], k0[c], se, k0[ch], k1[ch]);
  k0 = sm.st.u[QX0];
  k1 = sm.st.u[3 + dir];
  sqx = limit_comp32(d.ds, d.tol, half, k0[cl], k1[cl], k0[c], k1[c], k0[ch], k1[ch]);
  k0 = sm.st.u[QY0];
  k1 = sm.st.u[6 + dir];
  sqy = limit_comp32(d.ds, d.tol, half, k0[cl], k1[cl], k0[c], k1[c], k0[ch], k1[ch]);
}

// Planar limit (face depth, qx, qy) of the staged cell (r, x) at face f (0 E,
// 1 W, 2 N, 3 S), slopes limited when LL: for an edge ghost.
template <bool LL, int SP, class SM>
__device__ __forceinline__ void staged_face_limit(const D32& d, const SM& sm, int r, int x, int gi,
                                                  int gj, int f, float& h, float& qx, float& qy) {
  const int c = r * SP + x;
  const int dir = f <= 1 ? 1 : 2;
  float se = sm.st.u[dir][c], sx = sm.st.u[3 + dir][c], sy = sm.st.u[6 + dir][c];
  if (LL) staged_limited<SP>(d, sm, r, x, gi, gj, dir, se, sx, sy);
  float z0, z1x, z1y, zE, zW, zN, zS;
  staged_z(sm, r, x, z0, z1x, z1y, zE, zW, zN, zS);
  const float e0 = sm.st.u[E0][c], lo = sm.st.u[E0L][c];
  const float x0 = sm.st.u[QX0][c], y0 = sm.st.u[QY0][c];
  if (f == 0) { h = ((e0 - zE) + se) + lo; qx = x0 + sx; qy = y0 + sy; }
  else if (f == 1) { h = ((e0 - zW) - se) + lo; qx = x0 - sx; qy = y0 - sy; }
  else if (f == 2) { h = ((e0 - zN) + se) + lo; qx = x0 + sx; qy = y0 + sy; }
  else { h = ((e0 - zS) - se) + lo; qx = x0 - sx; qy = y0 - sy; }
}

// Record of the staged neighbour (r, x) = grid (gi, gj) at the face it shares
// with a tile cell (side 0: west / south of the face, its east / north limit;
// side 1: east / north, its west / south limit) along dir.
template <bool LL, int SP, class SM>
__device__ __forceinline__ RecF staged_neighbour_rec(const D32& d, const SM& sm, int r, int x,
                                                     int gi, int gj, int dir, int side) {
  const int c = r * SP + x;
  float ex = sm.st.u[E1X][c], xx = sm.st.u[QX1X][c], yx = sm.st.u[QY1X][c];
  float ey = sm.st.u[E1Y][c], xy = sm.st.u[QX1Y][c], yy = sm.st.u[QY1Y][c];
  if (LL) {
    staged_limited<SP>(d, sm, r, x, gi, gj, 1, ex, xx, yx);
    staged_limited<SP>(d, sm, r, x, gi, gj, 2, ey, xy, yy);
  }
  const float e0 = sm.st.u[E0][c], lo = sm.st.u[E0L][c];
  float z0, z1x, z1y, zE, zW, zN, zS;
  staged_z(sm, r, x, z0, z1x, z1y, zE, zW, zN, zS);
  float eh, wh, nh, sh;
  face_depths32(e0, ex, ey, lo, zE, zW, zN, zS, eh, wh, nh, sh);
  float scl;
  const float h0 = (e0 - z0) + lo;
  const bool pw = pw_scale32(h0, wh, eh, sh, nh, d.tol, d.wd, scl);
  const float qx0 = sm.st.u[QX0][c], qy0 = sm.st.u[QY0][c];
  const bool thin = d.wd != 0;
  // the limit at the shared face, selected (one record built whatever dir and side)
  const float hf = dir == 1 ? (side == 0 ? eh : wh) : (side == 0 ? nh : sh);
  const float dqx = dir == 1 ? xx : xy, dqy = dir == 1 ? yx : yy;
  const float qxf = side == 0 ? qx0 + dqx : qx0 - dqx, qyf = side == 0 ? qy0 + dqy : qy0 - dqy;
  return make_rec32(hf, qxf, qyf, pw, scl, d.tol, thin, h0);
}

// One RK stage of the FP32 free-surface form on the tile (bx, by) of problem d.
template <bool LL, int STAGE, int BX, int BY>
__device__ __forceinline__ void stage32_staged(const D32& d, StagedSmem32<LL, STAGE, BX, BY>& sm,
                                               const Blk32& blk, int bx, int by, float& brate,
                                               float& lam, bool& bad, bool& nonq) {
  using G = Geo32<LL, BX, BY>;
  constexpr int H = G::H, SP = G::SP, SR = G::SR, Q4 = G::Q4, X0 = G::X0;
  constexpr int NT = BX * BY;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
  const int i0 = bx * BX, j0 = by * BY;
  const int i = i0 + tx, j = j0 + ty;
  const bool act = i < d.nx && j < d.ny;
  const long long P = d.plane;
  const float* __restrict__ In = STAGE == 1 ? d.S : d.T;
  const float g = d.g, tol = d.tol;
  const float dt = blk.dt, gdt = blk.gdt;
  const double ts = blk.ts;

  // ---- stage the tile, its halo, the face beds (and n / own U^n) ----
  {
    const int xs = i0 - X0;                  // a multiple of 4 floats
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    // one (row, 16-byte column) slot per thread and pass, every plane of it
    for (int k = tid; k < SR * Q4; k += NT) {
      const int r = k / Q4, q = k - r * Q4;
      const int gj = j0 - H + r, gx = xs + 4 * q;
      float* dst = sm.st.u[0] + r * SP + 4 * q;
      float* dn = sm.st.n + (STAGE == 1 ? r * SP + 4 * q : 0);
      if (gj >= 0 && gj < d.ny && gx >= 0 && gx < d.pitch) {
        const float* src = In + (long long)gj * d.pitch + gx;
#pragma unroll
        for (int p = 0; p < kPlanes32; ++p) cp_async16(dst + p * G::PL, src + p * P);
        if (STAGE == 1) cp_async16(dn, d.N + (long long)gj * d.pitch + gx);
      } else {
#pragma unroll
        for (int p = 0; p < kPlanes32; ++p) *reinterpret_cast<float4*>(dst + p * G::PL) = zero4;
        if (STAGE == 1) *reinterpret_cast<float4*>(dn) = zero4;
      }
    }
    for (int k = tid; k < (2 * SR + 1) * Q4; k += NT) {
      const int r2 = k / Q4, q = k - r2 * Q4;
      const int gx = xs + 4 * q;
      if (r2 < SR) {
        const int gj = j0 - H + r2;
        float* dst = &sm.st.zx[r2][4 * q];
        if (gj >= 0 && gj < d.ny && gx >= 0 && gx < d.zpx)
          cp_async16(dst, d.ZX + (long long)gj * d.zpx + gx);
        else
          *reinterpret_cast<float4*>(dst) = zero4;
      } else {
        const int r = r2 - SR, gj = j0 - H + r;   // y-face rows j0 - H .. j0 + BY + H
        float* dst = &sm.st.zy[r][4 * q];
        if (gj >= 0 && gj <= d.ny && gx >= 0 && gx < d.pitch)
          cp_async16(dst, d.ZY + (long long)gj * d.pitch + gx);
        else
          *reinterpret_cast<float4*>(dst) = zero4;
      }
    }
    if (STAGE == 2) {
      // the own cells' U^n is read only by the update: its copies form a group of
      // their own, waited for after the faces
      cp_async_commit();
      constexpr int O4 = BX / 4;
      for (int k = tid; k < BY * O4; k += NT) {
        const int r = k / O4, q = k - r * O4;
        const int gj = j0 + r, gx = i0 + 4 * q;
        float* dst = &sm.own[0][r][4 * q];
        constexpr int OP = BY * BX;            // floats per own plane
        if (gj < d.ny && gx < d.pitch) {
          const long long o = (long long)gj * d.pitch + gx;
          if (!LL) {
            // the depth modes of U^n, its discharge modes after friction (stage 1)
            cp_async16(dst + E0 * OP, d.S + E0 * P + o);
            cp_async16(dst + E1X * OP, d.S + E1X * P + o);
            cp_async16(dst + E1Y * OP, d.S + E1Y * P + o);
            cp_async16(dst + E0L * OP, d.S + E0L * P + o);
#pragma unroll
            for (int p = 0; p < 6; ++p) cp_async16(dst + (QX0 + p) * OP, d.Q + p * P + o);
          } else {
            cp_async16(dst + 0 * OP, d.S + E0 * P + o);
            cp_async16(dst + 1 * OP, d.S + E0L * P + o);
            cp_async16(dst + 2 * OP, d.S + QX0 * P + o);
            cp_async16(dst + 3 * OP, d.S + QY0 * P + o);
#pragma unroll
            for (int p = 0; p < 6; ++p) cp_async16(dst + (4 + p) * OP, d.Q + p * P + o);
          }
          if (LL) cp_async16(dst + (kOwn32 - 1) * OP, d.N + o);
        } else {
#pragma unroll
          for (int p = 0; p < kOwn32; ++p) *reinterpret_cast<float4*>(dst + p * OP) = zero4;
        }
      }
    }
    if (STAGE == 2) {
      cp_async_commit();
      cp_async_wait_but_one();
    } else {
      cp_async_wait_all();
    }
    __syncthreads();
  }

  // ---- stage 1: friction of every staged cell the stage reads, in place ----
  if (STAGE == 1) {
    constexpr int RW = BX + 2 * H;
    for (int k = tid; k < SR * RW; k += NT) {
      const int r = k / RW, cc = k - r * RW;
      const int gi = i0 - H + cc, gj = j0 - H + r;
      if (gi < 0 || gi >= d.nx || gj < 0 || gj >= d.ny) continue;
      const int x = X0 - H + cc, c = r * SP + x;
      float z0, z1x, z1y, zE, zW, zN, zS;
      staged_z(sm, r, x, z0, z1x, z1y, zE, zW, zN, zS);
      const float h0 = (sm.st.u[E0][c] - z0) + sm.st.u[E0L][c];
      float q[6] = {sm.st.u[QX0][c], sm.st.u[QX1X][c], sm.st.u[QX1Y][c],
                    sm.st.u[QY0][c], sm.st.u[QY1X][c], sm.st.u[QY1Y][c]};
      friction_modes32(gdt, sm.st.n[c], tol, h0, sm.st.u[E1X][c] - z1x, sm.st.u[E1Y][c] - z1y, q);
      sm.st.u[QX0][c] = q[0]; sm.st.u[QX1X][c] = q[1]; sm.st.u[QX1Y][c] = q[2];
      sm.st.u[QY0][c] = q[3]; sm.st.u[QY1X][c] = q[4]; sm.st.u[QY1Y][c] = q[5];
    }
    __syncthreads();
  }

  // ---- face records: own cells, then the halo cells beside the tile ----
  const int r0 = ty + H, x0 = tx + X0, c0 = r0 * SP + x0;
  float m[9];
  float z0 = 0.f, z1x = 0.f, z1y = 0.f, zE = 0.f, zW = 0.f, zN = 0.f, zS = 0.f;
  RecF rE, rW, rN, rS;
  float mlo = 0.f;
  if (act) {
#pragma unroll
    for (int k = 0; k < 9; ++k) m[k] = sm.st.u[k][c0];
    mlo = sm.st.u[E0L][c0];
    if (LL) {
      staged_limited<SP>(d, sm, r0, x0, i, j, 1, m[E1X], m[QX1X], m[QY1X]);
      staged_limited<SP>(d, sm, r0, x0, i, j, 2, m[E1Y], m[QX1Y], m[QY1Y]);
    }
    staged_z(sm, r0, x0, z0, z1x, z1y, zE, zW, zN, zS);
    float eh, wh, nh, shh;
    face_depths32(m[E0], m[E1X], m[E1Y], mlo, zE, zW, zN, zS, eh, wh, nh, shh);
    const float eqx = m[QX0] + m[QX1X], eqy = m[QY0] + m[QY1X];
    const float wqx = m[QX0] - m[QX1X], wqy = m[QY0] - m[QY1X];
    const float nqx = m[QX0] + m[QX1Y], nqy = m[QY0] + m[QY1Y];
    const float sqx = m[QX0] - m[QX1Y], sqy = m[QY0] - m[QY1Y];
    float scl;
    const float h0c = (m[E0] - z0) + mlo;
    const bool pw = pw_scale32(h0c, wh, eh, shh, nh, tol, d.wd, scl);
    const bool thin = d.wd != 0;
    rE = make_rec32(eh, eqx, eqy, pw, scl, tol, thin, h0c);
    rW = make_rec32(wh, wqx, wqy, pw, scl, tol, thin, h0c);
    rN = make_rec32(nh, nqx, nqy, pw, scl, tol, thin, h0c);
    rS = make_rec32(shh, sqx, sqy, pw, scl, tol, thin, h0c);
    sm.e[ty][tx] = rE;
    sm.n[ty][tx] = rN;
  }
  {
    // the records beyond the tile, one per thread of the first 2 (BX + BY)
    // threads: west column, east column, south row, north row.  Every thread
    // runs the same code on its side's indices, so a warp holding several
    // sides builds their records together.
    const int t = tid;
    const int ni = d.nx - i0 < BX ? d.nx - i0 : BX, nj = d.ny - j0 < BY ? d.ny - j0 : BY;
    const int kind = t < BY ? 0 : t < 2 * BY ? 1 : t < 2 * BY + BX ? 2 : 3;
    const int q = kind == 0 ? t : kind == 1 ? t - BY : kind == 2 ? t - 2 * BY : t - 2 * BY - BX;
    if (t < 2 * (BX + BY) && q < (kind <= 1 ? nj : ni)) {
      const int dir = kind <= 1 ? 1 : 2, side = kind & 1;
      // the tile cell beside the face (staged row r, column x; grid gi, gj)
      const int r = kind == 0 || kind == 1 ? q + H : kind == 2 ? H : H + nj - 1;
      const int x = kind == 0 ? X0 : kind == 1 ? X0 + ni - 1 : X0 + q;
      const int gi = i0 + x - X0, gj = j0 + r - H;
      // step from it to the neighbour across the face
      const int sx = dir == 1 ? (side == 0 ? -1 : 1) : 0, sy = dir == 2 ? (side == 0 ? -1 : 1) : 0;
      const bool at_edge = dir == 1 ? (side == 0 ? gi == 0 : gi == d.nx - 1)
                                    : (side == 0 ? gj == 0 : gj == d.ny - 1);
      RecF rec;
      if (at_edge) {
        // the ghost of the tile cell's own limit at that face
        const int fo = kind == 0 ? 1 : kind == 1 ? 0 : kind == 2 ? 3 : 2;
        float h, qx, qy;
        staged_face_limit<LL, SP>(d, sm, r, x, gi, gj, fo, h, qx, qy);
        const float s = dir == 1 ? (gj + 0.5f) * d.dy : (gi + 0.5f) * d.dx;
        ghost32(d, kind, s, ts, h, qx, qy);
        rec = make_rec32(h, qx, qy, false, 1.f, tol);
      } else {
        rec = staged_neighbour_rec<LL, SP>(d, sm, r + sy, x + sx, gi + sx, gj + sy, dir, side);
      }
      RecF* dst = kind == 0 ? sm.hw : kind == 1 ? sm.he : kind == 2 ? sm.hs : sm.hn;
      dst[q] = rec;
    }
  }
  __syncthreads();   // the staged planes are dead from here: the face fluxes reuse them

  // ---- one revision and one flux per face ----
  float hWo = 0.f, hSo = 0.f;
  if (act) {
    LimF ra, rb;
    const RecF& Lw = tx > 0 ? sm.e[ty][tx - 1] : sm.hw[ty];
    revise_face32(Lw, rW, tol, ra, rb);
    hWo = rb.h;
    const FaceF fw = flux_x32(ra, rb, g, tol);
    sm.fc.fx[ty][tx] = FaceR32{fw, ra.h};
    if (i == 0) brate += fw.h * d.dy;
    const RecF& Ls = ty > 0 ? sm.n[ty - 1][tx] : sm.hs[tx];
    revise_face32(Ls, rS, tol, ra, rb);
    hSo = rb.h;
    const FaceF fs = flux_y32(ra, rb, g, tol);
    sm.fc.fy[ty][tx] = FaceR32{fs, ra.h};
    if (j == 0) brate += fs.h * d.dx;
  }
  {
    const int t = tid;
    const int ni = d.nx - i0 < BX ? d.nx - i0 : BX;
    const int nj = d.ny - j0 < BY ? d.ny - j0 : BY;
    // the tile's east edge faces (threads 0 .. nj - 1) and north edge faces
    // (threads BY .. BY + ni - 1) on one code path: the north faces' normal is y
    const bool yf = t >= BY;
    const int q = yf ? t - BY : t;
    if (yf ? q < ni : q < nj) {
      LimF ra, rb;
      revise_face32(yf ? sm.n[nj - 1][q] : sm.e[q][ni - 1], yf ? sm.hn[q] : sm.he[q], tol, ra, rb);
      const FaceF f = hll_dev(ra.h, yf ? ra.qy : ra.qx, yf ? ra.qx : ra.qy, yf ? ra.v : ra.u,
                              yf ? ra.u : ra.v, rb.h, yf ? rb.qy : rb.qx, yf ? rb.qx : rb.qy,
                              yf ? rb.v : rb.u, yf ? rb.u : rb.v, g, tol);
      FaceR32* dst = yf ? &sm.fc.fy[nj][q] : &sm.fc.fx[q][ni];
      *dst = FaceR32{f, ra.h};
      if (yf ? j0 + nj == d.ny : i0 + ni == d.nx) brate -= f.h * (yf ? d.dx : d.dy);
    }
  }
  if (STAGE == 2) cp_async_wait_all();   // the own cells' U^n
  __syncthreads();

  // ---- operator (Eqs. 4-5) and the RK update ----
  if (act) {
    const long long c = (long long)j * d.pitch + i;
    const FaceR32 rEf = sm.fc.fx[ty][tx + 1], rWf = sm.fc.fx[ty][tx];
    const FaceR32 rNf = sm.fc.fy[ty + 1][tx], rSf = sm.fc.fy[ty][tx];
    const FaceF fE = rEf.f, fW = rWf.f, gN = rNf.f, gS = rSf.f;
    const float hEo = rEf.ha, hNo = rNf.ha;
    const float FEh = fE.h, FEx = fE.n, FEy = fE.t;
    const float FWh = fW.h, FWx = fW.n + fW.dp, FWy = fW.t;
    const float GNh = gN.h, GNx = gN.t, GNy = gN.n;
    const float GSh = gS.h, GSx = gS.t, GSy = gS.n + gS.dp;
    LimF Es, Ws, Ns, Ss;
    Es.h = hEo; Es.qx = hEo * rE.u; Es.qy = hEo * rE.v;
    Ws.h = hWo; Ws.qx = hWo * rW.u; Ws.qy = hWo * rW.v;
    Ns.h = hNo; Ns.qx = hNo * rN.u; Ns.qy = hNo * rN.v;
    Ss.h = hSo; Ss.qx = hSo * rS.u; Ss.qy = hSo * rS.v;
    const float h0x = 0.5f * (Es.h + Ws.h), x0x = 0.5f * (Es.qx + Ws.qx), y0x = 0.5f * (Es.qy + Ws.qy);
    const float h1x_ = 0.5f * (Es.h - Ws.h), x1x = 0.5f * (Es.qx - Ws.qx), y1x = 0.5f * (Es.qy - Ws.qy);
    const float h0y = 0.5f * (Ns.h + Ss.h), x0y = 0.5f * (Ns.qx + Ss.qx), y0y = 0.5f * (Ns.qy + Ss.qy);
    const float h1y_ = 0.5f * (Ns.h - Ss.h), x1y = 0.5f * (Ns.qx - Ss.qx), y1y = 0.5f * (Ns.qy - Ss.qy);
    const float r3 = 0.57735026918962576f;
    float Fph, Fpx, Fpy, Fmh, Fmx, Fmy, Gph, Gpx, Gpy, Gmh, Gmx, Gmy;
    gauss_dev(h0x + h1x_ * r3, x0x + x1x * r3, y0x + y1x * r3, tol, false, Fph, Fpx, Fpy);
    gauss_dev(h0x - h1x_ * r3, x0x - x1x * r3, y0x - y1x * r3, tol, false, Fmh, Fmx, Fmy);
    gauss_dev(h0y + h1y_ * r3, x0y + x1y * r3, y0y + y1y * r3, tol, true, Gph, Gpx, Gpy);
    gauss_dev(h0y - h1y_ * r3, x0y - x1y * r3, y0y - y1y * r3, tol, true, Gmh, Gmx, Gmy);
    const float idx = d.inv_dx, idy = d.inv_dy;
    const float dEx = 2.f * m[E1X], dEy = 2.f * m[E1Y];  // eta_E - eta_W, eta_N - eta_S
    float L[9];
    L[E0] = -(FEh - FWh) * idx - (GNh - GSh) * idy;
    L[QX0] = -(FEx - FWx) * idx - (GNx - GSx) * idy - g * h0x * dEx * idx;
    L[QY0] = -(FEy - FWy) * idx - (GNy - GSy) * idy - g * h0y * dEy * idy;
    if (blk.rain) L[E0] += blk.rainf;
    if (c == d.src_idx) L[E0] += (float)(d.qp / (d.dxd * d.dyd));
    const float k3x = -3.f * idx, k3y = -3.f * idy, g23 = 2.f * g / 3.f;
    L[E1X] = k3x * ((FEh + FWh) - (Fph + Fmh));
    L[QX1X] = k3x * ((FEx + FWx) - (Fpx + Fmx) + g23 * h1x_ * (0.5f * dEx));
    L[QY1X] = k3x * ((FEy + FWy) - (Fpy + Fmy));
    L[E1Y] = k3y * ((GNh + GSh) - (Gph + Gmh));
    L[QX1Y] = k3y * ((GNx + GSx) - (Gpx + Gmx));
    L[QY1Y] = k3y * ((GNy + GSy) - (Gpy + Gmy) + g23 * h1y_ * (0.5f * dEy));

    float out[9];
    if (STAGE == 1) {
#pragma unroll
      for (int k = 1; k < 9; ++k) out[k] = m[k] + dt * L[k];
      float olo;
      two_sum(m[E0], mlo + dt * L[E0], out[E0], olo);
      wetdry32(out, olo, z0, z1x, z1y, zE, zW, zN, zS, tol);
#pragma unroll
      for (int k = 0; k < 9; ++k) d.T[k * P + c] = out[k];
      d.T[E0L * P + c] = olo;
      if (LL) {
        d.Q[0 * P + c] = m[E1X]; d.Q[1 * P + c] = m[E1Y];
        d.Q[2 * P + c] = m[QX1X]; d.Q[3 * P + c] = m[QX1Y];
        d.Q[4 * P + c] = m[QY1X]; d.Q[5 * P + c] = m[QY1Y];
      } else {
        // U^n's discharge modes after friction, for stage 2's RK average
#pragma unroll
        for (int p = 0; p < 6; ++p) d.Q[p * P + c] = m[QX0 + p];
      }
    } else {
      // U^n after friction (and, in DG2-LL, the limiter of stage 1): the average
      // of the RK2 combination
      float un[9], unlo;
      if (LL) {
        const float nn = sm.own[kOwn32 - 1][ty][tx];
        un[E0] = sm.own[0][ty][tx];
        unlo = sm.own[1][ty][tx];
        un[QX0] = sm.own[2][ty][tx];
        un[QY0] = sm.own[3][ty][tx];
        un[E1X] = sm.own[4][ty][tx]; un[E1Y] = sm.own[5][ty][tx];
        un[QX1X] = sm.own[6][ty][tx]; un[QX1Y] = sm.own[7][ty][tx];
        un[QY1X] = sm.own[8][ty][tx]; un[QY1Y] = sm.own[9][ty][tx];
        friction_centre32(gdt, nn, tol, (un[E0] - z0) + unlo, un[QX0], un[QY0]);
      } else {
        // the discharges arrive with friction applied (stage 1 stored them)
#pragma unroll
        for (int k = 0; k < 9; ++k) un[k] = sm.own[k][ty][tx];
        unlo = sm.own[E0L][ty][tx];
      }
#pragma unroll
      for (int k = 1; k < 9; ++k) out[k] = 0.5f * (un[k] + m[k] + dt * L[k]);
      float olo;
      {
        float s1, e1, r1, e2;
        two_sum(un[E0], m[E0], s1, e1);
        e1 += (unlo + mlo) + dt * L[E0];
        two_sum(s1, e1, r1, e2);
        out[E0] = 0.5f * r1;
        olo = 0.5f * e2;
      }
      wetdry32(out, olo, z0, z1x, z1y, zE, zW, zN, zS, tol);
#pragma unroll
      for (int k = 0; k < 9; ++k) d.S[k * P + c] = out[k];
      d.S[E0L * P + c] = olo;
      const float h0n = (out[E0] - z0) + olo;
      lam = rate32(d, h0n, out[QX0], out[QY0]);
      bad = bad || !(isfinite(out[E0]) && isfinite(olo) && isfinite(out[QX0]) &&
                     isfinite(out[QY0]));
      nonq = !(h0n <= tol) || out[E1X] != z1x || out[E1Y] != z1y;
#pragma unroll
      for (int k = 3; k < 9; ++k) nonq = nonq || out[k] != 0.f;
    }
  }
}

}  // namespace f32
}  // namespace dg2
