// dg2_fv.cuh -- the MUSCL-FV2 and FV1 comparator schemes of Sec. 2.2 (Eqs. 8-10)
// on the FP64 state layout.  The FV schemes hold cell averages only (planes
// h0, qx0, qy0); the slope planes are never read or written.
//
// Per cell and face: MUSCL limits of eta = h + z, h, qx, qy (Eq. 9) with
// Sweby's limiter (beta = 1.25, Eq. 10, r = forward / backward difference, no
// reconstruction across a wet-dry front), the free-surface revision of
// Sec. 2.2.2 (z* = max of the two bed limits, h* = max(0, eta - z*), q* = h* u,
// the own-side lowering of z* behind a wall), the run's Riemann solver and
// Eq. 8's bed term (factor 2 / dx as in Eq. 4a).  Friction is the DG2 friction
// kernel, which on zero slopes acts on the averages alone.
//
// One block per 32 x 8 tile of the step's lists, as the DG2 stage kernels:
// the averages of the tile and a 2-cell halo are staged in shared memory, each
// thread forms its cell's four limits, the tile's edge threads form the limit
// beyond the tile, and every face flux is evaluated once.  Dry-tile skipping
// carries over unchanged: a still, dry cell among still, dry neighbours has zero
// fluxes, and the dry reset removes the discharge its bed term makes.
#pragma once
#include "dg2_device.cuh"

namespace dg2 {
namespace fv {

constexpr int HX = TX + 4, HY = TY + 4;  // staged region: tile + 2-cell halo

struct L4 {
  double eta, h, qx, qy;
};

// A face after the revision: its flux, z* and the revised depths on the lower
// (a: west / south) and upper (b: east / north) side.
struct Face {
  double h, x, y, zs, ha, hb;
};

struct Smem {
  union {
    double A[4][HY][HX];  // eta, h, qx, qy of the staged region
    struct {
      Face fx[TY][TX + 1];  // fx[ty][tx] is the west face of column tx
      Face fy[TY + 1][TX];  // fy[ty][tx] is the south face of row ty
    } f;
  } u;
  L4 e[TY][TX];  // east limit of each cell
  L4 n[TY][TX];  // north limit of each cell
  L4 hw[TY], he[TY], hs[TX], hn[TX];  // limits beyond the tile (neighbour or ghost)
  double red[32];
};

__device__ __forceinline__ double sweby(double r, double beta) {
  const double a = beta * r < 1.0 ? beta * r : 1.0;
  const double b = r < beta ? r : beta;
  const double m = a > b ? a : b;
  return m > 0.0 ? m : 0.0;
}

// Limited slopes (Eq. 10) of the four components of staged cell (a, b) along
// (da, db); zero for FV1, at the domain edge along that direction, and where
// the cell or one of its two neighbours along it is at or below tol_dry.
template <bool ORDER2>
__device__ __forceinline__ void slopes4(const double (*A)[HY][HX], int a, int b, int da, int db,
                                        bool edge, double tol, double s[4]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) s[k] = 0.0;
  if (!ORDER2 || edge) return;
  if (A[1][b - db][a - da] <= tol || A[1][b][a] <= tol || A[1][b + db][a + da] <= tol) return;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double vc = A[k][b][a];
    const double bd = vc - A[k][b - db][a - da], fd = A[k][b + db][a + da] - vc;
    s[k] = bd == 0.0 ? 0.0 : sweby(fd / bd, 1.25) * bd;
  }
}

// Limit of staged cell (a, b) at the face on side sg (+0.5 east / north,
// -0.5 west / south) of the slopes' direction (Eq. 9).
__device__ __forceinline__ L4 lim4(const double (*A)[HY][HX], int a, int b, const double s[4],
                                   double sg) {
  L4 r;
  r.eta = A[0][b][a] + sg * s[0];
  r.h = A[1][b][a] + sg * s[1];
  r.qx = A[2][b][a] + sg * s[2];
  r.qy = A[3][b][a] + sg * s[3];
  return r;
}

// Boundary ghost of the own limit `own` at `edge` (0 W, 1 E, 2 S, 3 N), over
// the same bed.
__device__ __forceinline__ L4 ghost4(const Dev& d, int edge, double s, double t, const L4& own) {
  double h = own.h, qx = own.qx, qy = own.qy;
  ghost(d, edge, s, t, h, qx, qy);
  L4 r;
  r.eta = h + (own.eta - own.h);
  r.h = h;
  r.qx = qx;
  r.qy = qy;
  return r;
}

// Revision of a face (Sec. 2.2.2) from its lower (a) and upper (b) limits and
// the flux across it.
__device__ __forceinline__ Face face(const L4& a, const L4& b, bool ydir, double g, double tol,
                                     int flux) {
  const double za = a.eta - a.h, zb = b.eta - b.h;
  const double zs = za > zb ? za : zb;
  double ha = a.eta - zs, hb = b.eta - zs;
  if (ha < 0.0) ha = 0.0;
  if (hb < 0.0) hb = 0.0;
  // q* = h* u with u of the limit (tol rule on the limit's depth); the flux
  // then takes its velocities from the revised state by the same rule, so a
  // face depth h* at or below tol_dry moves no water by advection
  double ua = 0.0, va = 0.0, ub = 0.0, vb = 0.0;
  if (a.h > tol) { ua = a.qx / a.h; va = a.qy / a.h; }
  if (b.h > tol) { ub = b.qx / b.h; vb = b.qy / b.h; }
  Lim ra, rb;
  ra.h = ha; ra.qx = ha * ua; ra.qy = ha * va;
  rb.h = hb; rb.qx = hb * ub; rb.qy = hb * vb;
  ra.u = ha > tol ? ua : 0.0; ra.v = ha > tol ? va : 0.0;
  rb.u = hb > tol ? ub : 0.0; rb.v = hb > tol ? vb : 0.0;
  const F3 F = ydir ? flux_y(ra, rb, g, tol, flux) : flux_x(ra, rb, g, tol, flux);
  Face r;
  r.h = F.h; r.x = F.x; r.y = F.y;
  r.zs = zs; r.ha = ha; r.hb = hb;
  return r;
}

// One FV stage on the 32 x 8 tile (bx, by).  Stage 1: T = S + dt L(S) (all
// of FV1's update); stage 2 (FV2): S = (S + T + dt L(T)) / 2.  A dry cell
// keeps no discharge.  Accumulates the boundary inflow rate, and in the last
// stage the Courant rate and the non-finite / non-quiescent flags, of the
// thread's cell.
template <bool ORDER2, int STAGE>
__device__ __forceinline__ void fv_tile(const Dev& d, Smem& sm, int bx, int by, double& brate,
                                        double& lam, bool& bad, bool& nonq) {
  const Scalars* sc = d.sc;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i0 = bx * TX, j0 = by * TY, i = i0 + tx, j = j0 + ty;
  const int nx = d.nx, ny = d.ny;
  const bool act = i < nx && j < ny;
  const long long P = d.plane, c = (long long)j * d.pitch + i;
  const double dt = sc->dt;
  const double ts = STAGE == 1 ? sc->t : sc->t + dt;
  const double* __restrict__ In = STAGE == 1 ? d.S : d.T;
  const double g = d.g, tol = d.tol;

  // averages of the tile and its 2-cell halo
  for (int q = ty * TX + tx; q < HX * HY; q += TX * TY) {
    const int a = q % HX, b = q / HX;
    const int gi = i0 - 2 + a, gj = j0 - 2 + b;
    double h = 0.0, z = 0.0, qx = 0.0, qy = 0.0;
    if (gi >= 0 && gi < nx && gj >= 0 && gj < ny) {
      const long long cc = (long long)gj * d.pitch + gi;
      h = In[H0 * P + cc]; z = d.Z[cc]; qx = In[QX0 * P + cc]; qy = In[QY0 * P + cc];
    }
    sm.u.A[0][b][a] = h + z;
    sm.u.A[1][b][a] = h;
    sm.u.A[2][b][a] = qx;
    sm.u.A[3][b][a] = qy;
  }
  __syncthreads();

  const int a = tx + 2, b = ty + 2;
  const bool east_edge = act && (tx == TX - 1 || i == nx - 1);
  const bool north_edge = act && (ty == TY - 1 || j == ny - 1);
  L4 E, W, N, S;
  if (act) {
    const double(*A)[HY][HX] = sm.u.A;
    double s[4];
    slopes4<ORDER2>(A, a, b, 1, 0, i == 0 || i == nx - 1, tol, s);
    E = lim4(A, a, b, s, 0.5);
    W = lim4(A, a, b, s, -0.5);
    slopes4<ORDER2>(A, a, b, 0, 1, j == 0 || j == ny - 1, tol, s);
    N = lim4(A, a, b, s, 0.5);
    S = lim4(A, a, b, s, -0.5);
    sm.e[ty][tx] = E;
    sm.n[ty][tx] = N;
    if (tx == 0) {
      if (i == 0) {
        sm.hw[ty] = ghost4(d, 0, (j + 0.5) * d.dy, ts, W);
      } else {
        slopes4<ORDER2>(A, a - 1, b, 1, 0, i - 1 == 0, tol, s);
        sm.hw[ty] = lim4(A, a - 1, b, s, 0.5);
      }
    }
    if (east_edge) {
      if (i == nx - 1) {
        sm.he[ty] = ghost4(d, 1, (j + 0.5) * d.dy, ts, E);
      } else {
        slopes4<ORDER2>(A, a + 1, b, 1, 0, i + 1 == nx - 1, tol, s);
        sm.he[ty] = lim4(A, a + 1, b, s, -0.5);
      }
    }
    if (ty == 0) {
      if (j == 0) {
        sm.hs[tx] = ghost4(d, 2, (i + 0.5) * d.dx, ts, S);
      } else {
        slopes4<ORDER2>(A, a, b - 1, 0, 1, j - 1 == 0, tol, s);
        sm.hs[tx] = lim4(A, a, b - 1, s, 0.5);
      }
    }
    if (north_edge) {
      if (j == ny - 1) {
        sm.hn[tx] = ghost4(d, 3, (i + 0.5) * d.dx, ts, N);
      } else {
        slopes4<ORDER2>(A, a, b + 1, 0, 1, j + 1 == ny - 1, tol, s);
        sm.hn[tx] = lim4(A, a, b + 1, s, -0.5);
      }
    }
  }
  __syncthreads();  // the staged averages are dead past here (the faces reuse them)

  // one revision and one flux per face
  if (act) {
    const L4& Lw = tx > 0 ? sm.e[ty][tx - 1] : sm.hw[ty];
    const Face fw = face(Lw, W, false, g, tol, d.flux);
    sm.u.f.fx[ty][tx] = fw;
    if (i == 0) brate += fw.h * d.dy;
    if (east_edge) {
      const Face fe = face(E, sm.he[ty], false, g, tol, d.flux);
      sm.u.f.fx[ty][tx + 1] = fe;
      if (i == nx - 1) brate -= fe.h * d.dy;
    }
    const L4& Ls = ty > 0 ? sm.n[ty - 1][tx] : sm.hs[tx];
    const Face fs = face(Ls, S, true, g, tol, d.flux);
    sm.u.f.fy[ty][tx] = fs;
    if (j == 0) brate += fs.h * d.dx;
    if (north_edge) {
      const Face fn = face(N, sm.hn[tx], true, g, tol, d.flux);
      sm.u.f.fy[ty + 1][tx] = fn;
      if (j == ny - 1) brate -= fn.h * d.dx;
    }
  }
  __syncthreads();

  if (act) {
    const Face fw = sm.u.f.fx[ty][tx], fe = sm.u.f.fx[ty][tx + 1];
    const Face fs = sm.u.f.fy[ty][tx], fn = sm.u.f.fy[ty + 1][tx];
    // own-side bed limits, lowered where the own free surface is below z*
    const double dE = E.eta - fe.zs, dW = W.eta - fw.zs, dN = N.eta - fn.zs, dS = S.eta - fs.zs;
    const double zE = fe.zs - (dE < 0.0 ? -dE : 0.0), zW = fw.zs - (dW < 0.0 ? -dW : 0.0);
    const double zN = fn.zs - (dN < 0.0 ? -dN : 0.0), zS = fs.zs - (dS < 0.0 ? -dS : 0.0);
    const double h0x = 0.5 * (fe.ha + fw.hb), z1x = 0.5 * (zE - zW);
    const double h0y = 0.5 * (fn.ha + fs.hb), z1y = 0.5 * (zN - zS);
    const double idx = d.inv_dx, idy = d.inv_dy;
    // Eq. 8
    double Lh = -(fe.h - fw.h) * idx - (fn.h - fs.h) * idy;
    const double Lx = -(fe.x - fw.x) * idx - (fn.x - fs.x) * idy - 2.0 * g * h0x * z1x * idx;
    const double Ly = -(fe.y - fw.y) * idx - (fn.y - fs.y) * idy - 2.0 * g * h0y * z1y * idy;
    if (d.rain != 0.0 && ts >= d.rain_t0 && ts < d.rain_t1) Lh += d.rain;
    if (c == d.src_idx) Lh += d.qp * idx * idy;
    double h, qx, qy;
    if (STAGE == 1) {
      h = d.S[H0 * P + c] + dt * Lh;
      qx = d.S[QX0 * P + c] + dt * Lx;
      qy = d.S[QY0 * P + c] + dt * Ly;
    } else {
      h = 0.5 * (d.S[H0 * P + c] + d.T[H0 * P + c] + dt * Lh);
      qx = 0.5 * (d.S[QX0 * P + c] + d.T[QX0 * P + c] + dt * Lx);
      qy = 0.5 * (d.S[QY0 * P + c] + d.T[QY0 * P + c] + dt * Ly);
    }
    if (h <= tol) { qx = 0.0; qy = 0.0; }
    double* O = STAGE == 1 ? d.T : d.S;
    O[H0 * P + c] = h;
    O[QX0 * P + c] = qx;
    O[QY0 * P + c] = qy;
    if (STAGE == 2 || !ORDER2) {
      lam = cell_rate(d, h, qx, qy);
      bad = bad || !(isfinite(h) && isfinite(qx) && isfinite(qy)) || h < -1.0;
      nonq = !(h <= tol) || qx != 0.0 || qy != 0.0;
    }
  }
}

// The FV stage kernels over the step's tile lists (one block per entry, as
// the DG2 stage kernels).  Stage 1 also copies the frontier tiles' averages
// into T for a computed neighbour's halo.  The last stage (FV2's second, FV1's
// only) writes the tiles' quiescence flags and the Courant rate; FV1's stage
// leaves its result in T for fv1_commit_kernel.
template <bool ORDER2, int STAGE>
static __global__ void __launch_bounds__(TX* TY, 2) fv_stage_kernel(Dev d) {
  __shared__ Smem sm;
  Scalars* sc = d.sc;
  if (sc->done) return;
  constexpr bool last = STAGE == 2 || !ORDER2;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int ntx = d.tiles.ntx;
  const int n_act = sc->n_act;
  const bool all = sc->list_all != 0;
  double lam = 0.0;
  bool bad = false;
  if (STAGE == 2 && (int)blockIdx.x >= n_act) return;
  if ((int)blockIdx.x < n_act) {
    const int tile = all ? (int)blockIdx.x : list_tile(d.tiles, sc, (int)blockIdx.x);
    const int bx = tile % ntx, by = tile / ntx;
    double brate = 0.0;
    bool nonq = false;
    fv_tile<ORDER2, STAGE>(d, sm, bx, by, brate, lam, bad, nonq);
    if (bx == 0 || by == 0 || bx == ntx - 1 || by == d.tiles.nty - 1) {
      const double bsum = block_sum<TX * TY>(brate, sm.red);
      if (tx == 0 && ty == 0) {
        d.bpart[(STAGE - 1) * d.tiles.ntiles + tile] = bsum;
        // FV1's one stage counts for both slots of the step's ledger average
        if (!ORDER2) d.bpart[d.tiles.ntiles + tile] = bsum;
      }
    }
    if (last) {
      const int any_nonq = __syncthreads_or(nonq);
      if (tx == 0 && ty == 0) d.tiles.flag[tile] = any_nonq ? 1 : 0;
    }
    __syncthreads();
  }
  if (STAGE == 1) {
    const int e = (int)blockIdx.x - n_act;
    if (e >= 0 && e < sc->n_front) {
      const int tile = d.tiles.front[e];
      const int i = (tile % ntx) * TX + tx, j = (tile / ntx) * TY + ty;
      if (i < d.nx && j < d.ny) {
        const long long P = d.plane, c = (long long)j * d.pitch + i;
        d.T[H0 * P + c] = d.S[H0 * P + c];
        d.T[QX0 * P + c] = d.S[QX0 * P + c];
        d.T[QY0 * P + c] = d.S[QY0 * P + c];
      }
    }
  }
  if (!last) return;
  if (__syncthreads_or(bad) && tx == 0 && ty == 0) sc->nonfinite = 1;
  const double bl = block_max<TX * TY>(lam, sm.red);
  if (tx == 0 && ty == 0 && bl > 0.0)
    atomicMax(&sc->lam_bits, (unsigned long long)__double_as_longlong(bl));
}

// FV1's end of step: S = T on the computed tiles.
static __global__ void __launch_bounds__(TX* TY) fv1_commit_kernel(Dev d) {
  const Scalars* sc = d.sc;
  if (sc->done) return;
  const int n_act = sc->n_act;
  if ((int)blockIdx.x >= n_act) return;
  const int ntx = d.tiles.ntx;
  const int tile = sc->list_all ? (int)blockIdx.x : list_tile(d.tiles, sc, (int)blockIdx.x);
  const int i = (tile % ntx) * TX + threadIdx.x, j = (tile / ntx) * TY + threadIdx.y;
  if (i >= d.nx || j >= d.ny) return;
  const long long P = d.plane, c = (long long)j * d.pitch + i;
  d.S[H0 * P + c] = d.T[H0 * P + c];
  d.S[QX0 * P + c] = d.T[QX0 * P + c];
  d.S[QY0 * P + c] = d.T[QY0 * P + c];
}

}  // namespace fv
}  // namespace dg2
