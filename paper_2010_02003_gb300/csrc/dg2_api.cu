// dg2_api.cu -- host runtime and C ABI of the GB300 DG2 solver (include/dg2.h).
//
// The context lives on the host; every array lives in the caller's device
// workspace; every kernel and copy goes to the caller's stream.  dg2_run_to
// advances in chunks of steps captured once into a CUDA graph: the stage-2
// kernel's last block advances t on the device and raises a stop flag at
// t_end, so the host only reads the scalars once per chunk.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/dg2.h"
#include "dg2_device.cuh"
#include "dg2_fs32.cuh"
#include "dg2_fv.cuh"
#include "dg2_internal.h"

using dg2::Dev;
using dg2::f32::D32;
using dg2::Scalars;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CU(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(DG2_E_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));          \
  } while (0)

constexpr size_t kAlign = 256;
constexpr int kMaxKnots = 4096;
constexpr int kChunkMin = 16, kChunkMax = 1024;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Layout {
  int pitch, zpx;
  long long plane;
  size_t off_S, off_T, off_Q, off_Z, off_N, off_ZX, off_ZY, off_bpart, off_mpart, off_kt, off_kq;
  size_t off_gidx, off_gxi, off_geta, off_st, off_sh, off_sc, off_tflag, off_tact, off_tforced,
      off_tlist, off_tfront, off_desc, off_es, off_qm, total;
  int nblocks, mblocks, nbx, nby;
};

bool make_layout(int nx, int ny, const dg2_params& p, Layout& L) {
  if (nx < 1 || ny < 1 || p.max_gauges < 0 || p.max_gauges > dg2::kMaxGauges ||
      p.max_samples < 1)
    return false;
  L.pitch = (nx + 31) / 32 * 32;
  L.zpx = (nx + 1 + 31) / 32 * 32;
  L.plane = (long long)L.pitch * ny;
  const bool f32 = p.precision == DG2_FP32;
  const size_t esz = f32 ? sizeof(float) : sizeof(double);
  const size_t pb = (size_t)L.plane * esz;
  // set_dem stages the FP64 corner arrays and Manning field in the stage buffer
  const size_t staging = sizeof(double) * (2 * (size_t)(nx + 1) * (ny + 1) + (size_t)nx * ny);
  const int tw = f32 ? (dg2::ens::f32_small_tiles((long long)nx * ny) ? 16 : 32) : dg2::TX;
  const int th = dg2::TY;
  L.nblocks = ((nx + tw - 1) / tw) * ((ny + th - 1) / th);
  L.mblocks = ((nx + 31) / 32) * ((ny + 7) / 8);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align_up(o + bytes);
    return at;
  };
  const size_t nplanes = f32 ? dg2::f32::kPlanes32 : 9;
  L.off_S = take(nplanes * pb);
  L.off_T = take(nplanes * pb > staging ? nplanes * pb : staging);
  L.off_Q = take(p.variant == DG2_LL || f32 ? 6 * pb : 0);
  L.off_Z = take(f32 ? 0 : 3 * pb);
  L.off_ZX = take(f32 ? (size_t)ny * L.zpx * sizeof(float) : 0);
  L.off_ZY = take(f32 ? (size_t)(ny + 1) * L.pitch * sizeof(float) : 0);
  L.off_N = take(pb);
  L.off_bpart = take(2 * (size_t)L.nblocks * sizeof(double));
  L.off_mpart = take((size_t)L.mblocks * sizeof(double));
  L.off_kt = take((size_t)dg2::kMaxInflow * kMaxKnots * sizeof(double));
  L.off_kq = take((size_t)dg2::kMaxInflow * kMaxKnots * sizeof(double));
  const size_t ng = p.max_gauges > 0 ? p.max_gauges : 1;
  L.off_gidx = take(ng * sizeof(long long));
  L.off_gxi = take(ng * sizeof(double));
  L.off_geta = take(ng * sizeof(double));
  L.off_st = take((size_t)p.max_samples * sizeof(double));
  L.off_sh = take((size_t)p.max_samples * ng * sizeof(double));
  L.off_sc = take(sizeof(Scalars));
  L.off_tflag = take((size_t)L.nblocks);
  L.off_tact = take((size_t)L.nblocks);
  L.off_tforced = take((size_t)L.nblocks);
  L.off_tlist = take((size_t)dg2::kListClasses * L.nblocks * sizeof(int));
  L.off_tfront = take((size_t)L.nblocks * sizeof(int));
  // FP64: the warp-block masks of Un and U1 and stage 1's computed blocks
  L.nbx = (nx + dg2::TX - 1) / dg2::TX * dg2::TBX;
  L.nby = (ny + dg2::TY - 1) / dg2::TY * dg2::TBY;
  L.off_qm = take(f32 ? 0 : 3 * (size_t)L.nbx * L.nby * sizeof(unsigned));
  // FP32: the problem's descriptor and step counters for the shared FP32 kernels
  L.off_desc = take(f32 ? sizeof(D32) : 0);
  L.off_es = take(f32 ? sizeof(dg2::ens::EnsScalars) : 0);
  L.total = o;
  return true;
}

}  // namespace

namespace dg2 {
// Lets the other translation units of the library report through dg2_last_error().
void set_error_text(const std::string& s) { g_err = s; }
}  // namespace dg2

struct dg2_ctx {
  Dev d;          // FP64 launch parameters (also carries the shared scalars/tables)
  D32 f;          // FP32 free-surface launch parameters
  int fp32;
  dg2_params p;
  Layout lay;
  cudaStream_t st;
  char* ws;
  int dem_set;
  // a read of the device scalars found the non-finite flag raised: further steps are
  // refused until dg2_set_dem / dg2_set_state give a valid state again
  int poisoned;
  int64_t launches;
  dim3 sgrid, sblock, pgrid, pblock;
  int g_fric, g_st1, g_st2;   // persistent grid sizes (blocks) of friction / stage 1 / stage 2
  dg2::ens::EnsDev e1;        // FP32: this problem as a set of one for the shared FP32 kernels
  dim3 lgrid, lblock;          // lists_kernel: one thread per tile
  std::vector<double> kt, kq;   // host copies of the knot tables
  // run_to graphs of 16 << k steps, k = 0..6 (dropped when the launch setup changes)
  cudaGraphExec_t graph[7];
  // optional per-kernel event timing of dg2_step
  int timing;
  int timed_steps;
  std::vector<cudaEvent_t> ev;   // 4 per timed step
};

namespace {

// Cells per tile of the context's dry-tile skipping: 32 x 8 for the FP64
// kernels; 16 x 8 or 32 x 8 for a single FP32 problem by its size.
int tile_w(const dg2_ctx* c) {
  return c->fp32 && dg2::ens::f32_small_tiles((long long)c->d.nx * c->d.ny) ? 16 : dg2::TX;
}
int tile_h(const dg2_ctx*) { return dg2::TY; }

int launch_check(dg2_ctx* c, int nkernels) {
  c->launches += nkernels;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(DG2_E_CUDA, "kernel launch failed: %s", cudaGetErrorString(e));
  return DG2_OK;
}

void drop_graph(dg2_ctx* c) {
  for (auto& g : c->graph) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
  }
}

constexpr int kMaxTimedSteps = 8192;

// FP32: uploads the problem's descriptor, which the shared FP32 kernels read
// from device memory (stream-ordered before the next launch).
int sync_desc(dg2_ctx* c) {
  if (!c->fp32) return DG2_OK;
  CU(cudaMemcpyAsync((void*)c->e1.desc, &c->f, sizeof(D32), cudaMemcpyHostToDevice, c->st));
  CU(cudaStreamSynchronize(c->st));
  return DG2_OK;
}

// End of step (time, ledger, gauges, next dt) and the next step's tile lists
// (2 kernels); with lists_only, just the lists (after a new DEM / state /
// forced mask).
void launch_finalize(dg2_ctx* c, int lists_only) {
  if (c->fp32) {
    dg2::ens::launch_end_of_step(c->e1, 1, c->lgrid, lists_only, c->st);
  } else {
    dg2::finalize_kernel<<<1, dg2::kFinThreads, 0, c->st>>>(c->d, lists_only);
    dg2::lists_kernel<<<c->lgrid, c->lblock, 0, c->st>>>(c->d);
  }
}

// Host-side mask of the tiles that must be computed whatever their state: the
// tile holding the point source and the edge tiles whose faces an inflow
// segment covers.  Rain marks every tile (all_forced).
void forced_mask(const Dev& d, int tw, int th, std::vector<unsigned char>& m) {
  const int ntx = (d.nx + tw - 1) / tw, nty = (d.ny + th - 1) / th;
  m.assign((size_t)ntx * nty, 0);
  if (d.src_idx >= 0) {
    const int si = (int)(d.src_idx % d.pitch), sj = (int)(d.src_idx / d.pitch);
    m[(size_t)(sj / th) * ntx + si / tw] = 1;
  }
  for (int k = 0; k < d.n_in; ++k) {
    const dg2::InflowDesc& f = d.in[k];
    const bool ew = f.edge <= 1;
    const int n = ew ? d.ny : d.nx;
    const double h = ew ? d.dy : d.dx;
    for (int q = 0; q < n; ++q) {
      const double sc = (q + 0.5) * h;
      if (sc < f.s0 || sc > f.s1) continue;
      int bx, by;
      if (ew) { by = q / th; bx = f.edge == 0 ? 0 : ntx - 1; }
      else { bx = q / tw; by = f.edge == 2 ? 0 : nty - 1; }
      m[(size_t)by * ntx + bx] = 1;
    }
  }
}

int update_forced_tiles(dg2_ctx* c) {
  Dev& d = c->d;
  std::vector<unsigned char> m;
  forced_mask(d, tile_w(c), tile_h(c), m);
  d.tiles.all_forced = d.rain != 0.0 ? 1 : 0;
  c->f.tiles = d.tiles;
  if (int r0 = sync_desc(c)) return r0;
  CU(cudaMemcpyAsync((void*)d.tiles.forced, m.data(), m.size(), cudaMemcpyHostToDevice, c->st));
  if (c->dem_set) {
    launch_finalize(c, 1);   // the computed set depends on the forced mask
    int r = launch_check(c, 2);
    if (r) return r;
  }
  CU(cudaStreamSynchronize(c->st));
  return DG2_OK;
}

// Copies the tables shared by both precisions (inflows, sources, gauges) from
// the FP64 parameter block into the FP32 one.
void mirror(dg2_ctx* c) {
  D32& f = c->f;
  const Dev& d = c->d;
  f.n_in = d.n_in;
  for (int k = 0; k < dg2::kMaxInflow; ++k) f.in[k] = d.in[k];
  f.rain = d.rain; f.rain_t0 = d.rain_t0; f.rain_t1 = d.rain_t1;
  f.qp = d.qp; f.src_idx = d.src_idx;
  f.ngauge = d.ngauge;
  f.tiles = d.tiles;
}

// Enqueues one RK2 step: friction, stage 1, stage 2, finalize, lists (5 kernels; 4 in
// FP32, whose stages apply friction themselves).  With `timed`, records an event before
// and after each kernel.
void enqueue_step(dg2_ctx* c, bool timed = false) {
  const Dev& d = c->d;
  cudaEvent_t* e = nullptr;
  if (timed && c->timing && c->timed_steps < kMaxTimedSteps) {
    const size_t need = 4 * (size_t)(c->timed_steps + 1);
    while (c->ev.size() < need) {
      cudaEvent_t x;
      if (cudaEventCreate(&x) != cudaSuccess) break;
      c->ev.push_back(x);
    }
    if (c->ev.size() >= need) e = &c->ev[4 * (size_t)c->timed_steps++];
  }
  const bool ll = c->p.variant == DG2_LL;
  if (e) cudaEventRecord(e[0], c->st);
  // FP32: friction is fused into the stage kernels (no launch of its own)
  if (!c->fp32) dg2::friction_kernel<<<c->g_fric, c->sblock, 0, c->st>>>(d);
  if (e) cudaEventRecord(e[1], c->st);
  if (c->p.scheme != DG2_SCHEME_DG2) {
    // the FV comparators: one block per tile of the lists, as the DG2 stages
    if (c->p.scheme == DG2_SCHEME_FV2)
      dg2::fv::fv_stage_kernel<true, 1><<<c->g_st1, c->sblock, 0, c->st>>>(d);
    else
      dg2::fv::fv_stage_kernel<false, 1><<<c->g_st1, c->sblock, 0, c->st>>>(d);
    if (e) cudaEventRecord(e[2], c->st);
    if (c->p.scheme == DG2_SCHEME_FV2)
      dg2::fv::fv_stage_kernel<true, 2><<<c->g_st2, c->sblock, 0, c->st>>>(d);
    else
      dg2::fv::fv1_commit_kernel<<<c->g_st2, c->sblock, 0, c->st>>>(d);
    if (e) cudaEventRecord(e[3], c->st);
    launch_finalize(c, 0);
    return;
  }
  if (c->fp32) {
    dg2::ens::launch_stage32(c->e1, tile_w(c), ll, 1, c->g_st1, c->st);
  } else {
    if (ll) dg2::stage_kernel<true, 1><<<c->g_st1, c->sblock, sizeof(dg2::StageSmem), c->st>>>(d);
    else dg2::stage_kernel<false, 1><<<c->g_st1, c->sblock, sizeof(dg2::StageSmem), c->st>>>(d);
  }
  if (e) cudaEventRecord(e[2], c->st);
  if (c->fp32) {
    dg2::ens::launch_stage32(c->e1, tile_w(c), ll, 2, c->g_st2, c->st);
  } else {
    if (ll) dg2::stage_kernel<true, 2><<<c->g_st2, c->sblock, sizeof(dg2::StageSmem), c->st>>>(d);
    else dg2::stage_kernel<false, 2><<<c->g_st2, c->sblock, sizeof(dg2::StageSmem), c->st>>>(d);
  }
  if (e) cudaEventRecord(e[3], c->st);
  launch_finalize(c, 0);
}

int read_scalars(dg2_ctx* c, Scalars* out) {
  CU(cudaMemcpyAsync(out, c->d.sc, sizeof(Scalars), cudaMemcpyDeviceToHost, c->st));
  CU(cudaStreamSynchronize(c->st));
  if (out->nonfinite) c->poisoned = 1;
  return DG2_OK;
}

// Steps refuse to run on a state already known to be non-finite.
int check_not_poisoned(dg2_ctx* c) {
  if (c->poisoned)
    return fail(DG2_E_NONFINITE,
                "the state became non-finite in an earlier step; dg2_set_state or dg2_set_dem "
                "must provide a valid state before stepping again");
  return DG2_OK;
}

int check_arg_ctx(dg2_ctx* c, bool need_dem) {
  if (!c) return fail(DG2_E_ARG, "null context");
  if (need_dem && !c->dem_set) return fail(DG2_E_STATE, "dg2_set_dem or dg2_set_state first");
  return DG2_OK;
}

int recompute_dt(dg2_ctx* c) {
  if (c->fp32) dg2::f32::rate32_kernel<<<c->pgrid, c->pblock, 0, c->st>>>(c->f);
  else dg2::rate_kernel<<<c->pgrid, c->pblock, 0, c->st>>>(c->d);
  return launch_check(c, 1);
}

void launch_mass(dg2_ctx* c) {
  if (c->fp32) dg2::f32::mass32_kernel<<<c->pgrid, c->pblock, 0, c->st>>>(c->f);
  else dg2::mass_kernel<<<c->pgrid, c->pblock, 0, c->st>>>(c->d);
}

// Marks every tile non-quiescent so the next step computes the whole grid
// (after a new DEM or state; the first stage 2 then sets the true flags).
int reset_tiles(dg2_ctx* c) {
  CU(cudaMemsetAsync(c->d.tiles.flag, 1, (size_t)c->lay.nblocks, c->st));
  // every cell non-quiescent in the cell masks: the first step computes every cell
  if (c->d.qm)
    CU(cudaMemsetAsync(c->d.qm, 0xff, 3 * (size_t)c->d.qplane * sizeof(unsigned), c->st));
  launch_finalize(c, 1);
  return launch_check(c, 2);
}

int reset_ledger(dg2_ctx* c) {
  // mass kernel with the ledger-reset flag set by a one-field copy
  const int one = 1;
  CU(cudaMemcpyAsync(&c->d.sc->ledger_init, &one, sizeof(int), cudaMemcpyHostToDevice, c->st));
  CU(cudaStreamSynchronize(c->st));
  launch_mass(c);
  return launch_check(c, 1);
}

}  // namespace

namespace {

// FP32 contexts: host copies of the face topography and the cell modes of z
// formed exactly as the kernels form them (FP32 sums of face values).
int f32_topo_modes(dg2_ctx* c, std::vector<float>& z0, std::vector<float>& z1x,
                   std::vector<float>& z1y) {
  const int nx = c->f.nx, ny = c->f.ny;
  std::vector<float> zx((size_t)ny * (nx + 1)), zy((size_t)(ny + 1) * nx);
  CU(cudaMemcpy2DAsync(zx.data(), (nx + 1) * sizeof(float), c->f.ZX, c->f.zpx * sizeof(float),
                       (nx + 1) * sizeof(float), ny, cudaMemcpyDeviceToHost, c->st));
  CU(cudaMemcpy2DAsync(zy.data(), nx * sizeof(float), c->f.ZY, c->f.pitch * sizeof(float),
                       nx * sizeof(float), ny + 1, cudaMemcpyDeviceToHost, c->st));
  CU(cudaStreamSynchronize(c->st));
  const size_t n = (size_t)nx * ny;
  z0.resize(n); z1x.resize(n); z1y.resize(n);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const float zW = zx[(size_t)j * (nx + 1) + i], zE = zx[(size_t)j * (nx + 1) + i + 1];
      const float zS = zy[(size_t)j * nx + i], zN = zy[(size_t)(j + 1) * nx + i];
      const size_t k = (size_t)j * nx + i;
      z0[k] = 0.5f * (zE + zW);
      z1x[k] = 0.5f * (zE - zW);
      z1y[k] = 0.5f * (zN - zS);
    }
  return DG2_OK;
}

}  // namespace

extern "C" {

void dg2_default_params(dg2_params* p) {
  if (!p) return;
  p->g = 9.80665;
  p->cfl = 0.3;
  p->tol_dry = 1e-5;
  p->ds_thresh = 10.0;
  p->dt_max = 1.0;
  p->variant = DG2_NL;
  p->precision = DG2_FP64;
  for (int k = 0; k < 4; ++k) p->bc[k] = DG2_WALL;
  p->max_gauges = 64;
  p->max_samples = 4096;
  p->skip_dry_tiles = 1;
  p->flux = DG2_HLL;
  p->scheme = DG2_SCHEME_DG2;
  p->wetdry = DG2_WD_POSITIVE;
}

const char* dg2_last_error(void) { return g_err.c_str(); }

size_t dg2_workspace_bytes(int nx, int ny, const dg2_params* pp) {
  dg2_params p;
  if (pp) p = *pp; else dg2_default_params(&p);
  Layout L;
  if (!make_layout(nx, ny, p, L)) return 0;
  return L.total;
}

int dg2_init_grid(dg2_ctx** out, int nx, int ny, double dx, double dy, const dg2_params* pp,
                  void* dev_workspace, size_t ws_bytes, void* cuda_stream) {
  g_err.clear();
  if (!out) return fail(DG2_E_ARG, "out is null");
  *out = nullptr;
  dg2_params p;
  if (pp) p = *pp; else dg2_default_params(&p);
  if (!(dx > 0.0) || !(dy > 0.0) || !std::isfinite(dx) || !std::isfinite(dy))
    return fail(DG2_E_ARG, "dx, dy must be positive");
  if (!(p.g > 0.0) || !(p.cfl > 0.0) || !(p.tol_dry >= 0.0) || !(p.dt_max > 0.0) ||
      (p.variant != DG2_NL && p.variant != DG2_LL) ||
      (p.precision != DG2_FP64 && p.precision != DG2_FP32))
    return fail(DG2_E_ARG, "invalid parameters (g, cfl, tol_dry, dt_max, variant, precision)");
  if (p.flux != DG2_HLL && p.flux != DG2_ROE) return fail(DG2_E_ARG, "flux must be HLL or ROE");
  if (p.flux == DG2_ROE && p.precision != DG2_FP64)
    return fail(DG2_E_ARG, "the Roe flux is built for DG2_FP64 only");
  if (p.wetdry != DG2_WD_POSITIVE && p.wetdry != DG2_WD_PRINTED)
    return fail(DG2_E_ARG, "wetdry must be DG2_WD_POSITIVE or DG2_WD_PRINTED");
  if (p.scheme != DG2_SCHEME_DG2 && p.scheme != DG2_SCHEME_FV2 && p.scheme != DG2_SCHEME_FV1)
    return fail(DG2_E_ARG, "scheme must be DG2, FV2 or FV1");
  if (p.scheme != DG2_SCHEME_DG2 && (p.precision != DG2_FP64 || p.variant != DG2_NL))
    return fail(DG2_E_ARG, "the FV schemes are built for DG2_FP64 and DG2_NL only");
  for (int k = 0; k < 4; ++k)
    if (p.bc[k] != DG2_WALL && p.bc[k] != DG2_OPEN) return fail(DG2_E_ARG, "bad edge type");
  if ((long long)nx * ny > (1ll << 31)) return fail(DG2_E_ARG, "grid too large");
  Layout L;
  if (!make_layout(nx, ny, p, L))
    return fail(DG2_E_ARG, "invalid grid size or gauge capacities");
  if (!dev_workspace) return fail(DG2_E_ARG, "workspace is null");
  if ((uintptr_t)dev_workspace % kAlign) return fail(DG2_E_ARG, "workspace not 256-byte aligned");
  if (ws_bytes < L.total)
    return fail(DG2_E_NOMEM, "workspace of %zu bytes < %zu needed", ws_bytes, L.total);
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, dev_workspace) != cudaSuccess ||
      attr.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    return fail(DG2_E_ARG, "workspace is not device memory");
  }

  dg2_ctx* c = new dg2_ctx();
  c->p = p;
  c->lay = L;
  c->st = (cudaStream_t)cuda_stream;
  c->ws = (char*)dev_workspace;
  for (auto& g : c->graph) g = nullptr;
  Dev& d = c->d;
  memset(&d, 0, sizeof d);
  d.nx = nx; d.ny = ny; d.pitch = L.pitch; d.plane = L.plane;
  d.dx = dx; d.dy = dy; d.inv_dx = 1.0 / dx; d.inv_dy = 1.0 / dy;
  d.g = p.g; d.cfl = p.cfl; d.ds = p.ds_thresh; d.dt_max = p.dt_max;
  d.tol = p.tol_dry == 0.0 ? 0.0 : p.tol_dry;  // +0: the bit-pattern comparisons want c >= +0
  for (int k = 0; k < 4; ++k) d.bc[k] = p.bc[k];
  c->fp32 = p.precision == DG2_FP32;
  // plane buffers: FP64 depth modes, or FP32 free-surface modes (the FP64
  // pointers then alias the same bytes and are used only for staging)
  d.S = (double*)(c->ws + L.off_S);
  d.T = (double*)(c->ws + L.off_T);
  d.Q = p.variant == DG2_LL ? (double*)(c->ws + L.off_Q) : nullptr;
  d.flux = p.flux;
  d.scheme = p.scheme;
  d.wd = p.wetdry == DG2_WD_POSITIVE ? 1 : 0;
  d.Z = (const double*)(c->ws + L.off_Z);
  d.N = (const double*)(c->ws + L.off_N);
  d.bpart = (double*)(c->ws + L.off_bpart);
  d.mpart = (double*)(c->ws + L.off_mpart);
  d.knot_t = (const double*)(c->ws + L.off_kt);
  d.knot_q = (const double*)(c->ws + L.off_kq);
  d.g_idx = (const long long*)(c->ws + L.off_gidx);
  d.g_xi = (const double*)(c->ws + L.off_gxi);
  d.g_eta = (const double*)(c->ws + L.off_geta);
  d.samp_t = (double*)(c->ws + L.off_st);
  d.samp_h = (double*)(c->ws + L.off_sh);
  d.sc = (Scalars*)(c->ws + L.off_sc);
  d.max_samples = p.max_samples;
  d.src_idx = -1;
  d.nblocks = L.nblocks;
  d.tiles.flag = (unsigned char*)(c->ws + L.off_tflag);
  d.tiles.act = (unsigned char*)(c->ws + L.off_tact);
  d.tiles.forced = (const unsigned char*)(c->ws + L.off_tforced);
  d.tiles.list = (int*)(c->ws + L.off_tlist);
  d.tiles.front = (int*)(c->ws + L.off_tfront);
  d.tiles.ntx = (nx + tile_w(c) - 1) / tile_w(c);
  d.tiles.nty = (ny + tile_h(c) - 1) / tile_h(c);
  d.tiles.ntiles = d.tiles.ntx * d.tiles.nty;
  d.tiles.all_forced = 0;
  d.tiles.skip = p.skip_dry_tiles ? 1 : 0;
  d.qm = c->fp32 ? nullptr : (unsigned*)(c->ws + L.off_qm);
  d.nbx = L.nbx;
  d.nby = L.nby;
  d.qplane = (long long)L.nbx * L.nby;
  {
    D32& f = c->f;
    memset(&f, 0, sizeof f);
    f.nx = nx; f.ny = ny; f.pitch = L.pitch; f.zpx = L.zpx; f.plane = L.plane;
    f.dx = (float)dx; f.dy = (float)dy;
    f.inv_dx = (float)(1.0 / dx); f.inv_dy = (float)(1.0 / dy);
    f.g = (float)p.g; f.tol = (float)p.tol_dry; f.ds = (float)p.ds_thresh;
    f.dxd = dx; f.dyd = dy; f.cfl = p.cfl; f.dt_max = p.dt_max;
    for (int k = 0; k < 4; ++k) f.bc[k] = p.bc[k];
    f.knot_t = d.knot_t; f.knot_q = d.knot_q;
    f.S = (float*)(c->ws + L.off_S);
    f.T = (float*)(c->ws + L.off_T);
    f.Q = (float*)(c->ws + L.off_Q);
    f.ZX = (const float*)(c->ws + L.off_ZX);
    f.ZY = (const float*)(c->ws + L.off_ZY);
    f.N = (const float*)(c->ws + L.off_N);
    f.bpart = d.bpart; f.mpart = d.mpart; f.sc = d.sc;
    f.max_samples = d.max_samples;
    f.g_idx = d.g_idx; f.g_xi = d.g_xi; f.g_eta = d.g_eta;
    f.samp_t = d.samp_t; f.samp_h = d.samp_h;
    f.nblocks = L.nblocks;
    f.src_idx = -1;
    f.tiles = d.tiles;
    f.wd = d.wd;
  }
  c->sblock = dim3(dg2::TX, dg2::TY);
  c->sgrid = dim3((nx + dg2::TX - 1) / dg2::TX, (ny + dg2::TY - 1) / dg2::TY);
  c->pblock = dim3(32, 8);
  c->pgrid = dim3((nx + 31) / 32, (ny + 7) / 8);
  {
    // persistent grids: every resident block of the kernel, capped by the tile count
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const bool ll = p.variant == DG2_LL, f32 = p.precision == DG2_FP32;
    int o1 = 1, o2 = 1;
    // the FP64 stage tile's shared memory is above the 48 KB static limit
    cudaFuncSetAttribute(dg2::stage_kernel<true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(dg2::StageSmem));
    cudaFuncSetAttribute(dg2::stage_kernel<true, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(dg2::StageSmem));
    cudaFuncSetAttribute(dg2::stage_kernel<false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(dg2::StageSmem));
    cudaFuncSetAttribute(dg2::stage_kernel<false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(dg2::StageSmem));
    if (f32) {
      dg2::ens::occupancy32(tile_w(c), ll, &o1, &o2);
    } else {
      if (ll) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, dg2::stage_kernel<true, 1>, dg2::TX * dg2::TY,
                                                      sizeof(dg2::StageSmem));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o2, dg2::stage_kernel<true, 2>, dg2::TX * dg2::TY,
                                                      sizeof(dg2::StageSmem));
      } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, dg2::stage_kernel<false, 1>, dg2::TX * dg2::TY,
                                                      sizeof(dg2::StageSmem));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o2, dg2::stage_kernel<false, 2>, dg2::TX * dg2::TY,
                                                      sizeof(dg2::StageSmem));
      }
    }
    cudaGetLastError();
    const int nt = d.tiles.ntiles;
    auto gsz = [&](int occ) { long long g = (long long)nsm * (occ > 0 ? occ : 1); return (int)(g < nt ? g : nt); };
    c->lblock = dim3(dg2::LTX, dg2::LTY);
    c->lgrid = dim3((d.tiles.ntx + dg2::LTX - 1) / dg2::LTX, (d.tiles.nty + dg2::LTY - 1) / dg2::LTY);
    // friction: one block per tile of the list (the hardware hands blocks to SMs
    // as they free up); measured faster than a persistent grid looping over the
    // list (floodplain 2000 x 1000 from t = 1 h: 0.060 -> 0.051 ms per step)
    c->g_fric = nt;
    const bool loop = f32 ? true : (p.scheme == DG2_SCHEME_DG2 && DG2_TILE_LOOP64);
    c->g_st1 = loop ? gsz(o1) : nt;
    c->g_st2 = loop ? gsz(o2) : nt;
  }

  // zero the state, topography and scalars; t_end / samples at +inf
  cudaError_t e = cudaMemsetAsync(c->ws, 0, L.total, c->st);
  Scalars s0;
  memset(&s0, 0, sizeof s0);
  s0.t_end = INFINITY;
  s0.next_sample = INFINITY;
  s0.dt = p.dt_max;
  s0.dt_cfl = p.dt_max;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d.sc, &s0, sizeof s0, cudaMemcpyHostToDevice, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) {
    delete c;
    return fail(DG2_E_CUDA, "workspace initialisation failed: %s", cudaGetErrorString(e));
  }
  c->e1.desc = c->fp32 ? (const D32*)(c->ws + L.off_desc) : nullptr;
  c->e1.list = d.tiles.list;
  c->e1.front = d.tiles.front;
  c->e1.es = c->fp32 ? (dg2::ens::EnsScalars*)(c->ws + L.off_es) : nullptr;
  c->e1.nmem = 1;
  if (int r = sync_desc(c)) {
    delete c;
    return r;
  }
  *out = c;
  return DG2_OK;
}

int dg2_set_dem(dg2_ctx* c, const double* z_corner, const double* manning, double n_uniform,
                const double* eta_corner) {
  int r = check_arg_ctx(c, false);
  if (r) return r;
  if (!z_corner) return fail(DG2_E_ARG, "z_corner is null");
  if (!manning && !(n_uniform >= 0.0)) return fail(DG2_E_ARG, "n_uniform must be >= 0");
  const int nx = c->d.nx, ny = c->d.ny;
  const size_t nc = (size_t)(nx + 1) * (ny + 1), ncell = (size_t)nx * ny;
  for (size_t k = 0; k < nc; ++k)
    if (!std::isfinite(z_corner[k]) || (eta_corner && !std::isfinite(eta_corner[k])))
      return fail(DG2_E_ARG, "non-finite DEM or free surface at corner %zu", k);
  if (manning)
    for (size_t k = 0; k < ncell; ++k)
      if (!(manning[k] >= 0.0) || !std::isfinite(manning[k]))
        return fail(DG2_E_ARG, "invalid Manning n at cell %zu", k);
  drop_graph(c);
  // stage the corner arrays (and the Manning field) in the stage buffer T
  double* zc = c->d.T;
  double* ec = zc + nc;
  double* mn = ec + nc;
  CU(cudaMemcpyAsync(zc, z_corner, nc * sizeof(double), cudaMemcpyHostToDevice, c->st));
  if (eta_corner)
    CU(cudaMemcpyAsync(ec, eta_corner, nc * sizeof(double), cudaMemcpyHostToDevice, c->st));
  if (manning)
    CU(cudaMemcpyAsync(mn, manning, ncell * sizeof(double), cudaMemcpyHostToDevice, c->st));
  if (c->fp32) {
    const dim3 g1((nx + 1 + 31) / 32, (ny + 1 + 7) / 8);
    dg2::f32::init32_kernel<<<g1, c->pblock, 0, c->st>>>(
        c->f, zc, eta_corner ? ec : nullptr, manning ? mn : nullptr, n_uniform, (float*)c->f.ZX,
        (float*)c->f.ZY, (float*)c->f.N);
  } else {
    dg2::init_kernel<<<c->pgrid, c->pblock, 0, c->st>>>(c->d, zc, eta_corner ? ec : nullptr,
                                                        manning ? mn : nullptr, n_uniform,
                                                        (double*)c->d.Z, (double*)c->d.N);
  }
  if ((r = launch_check(c, 1))) return r;
  CU(cudaMemsetAsync(c->d.T, 0, c->lay.off_Q - c->lay.off_T, c->st));
  // scalars: t = 0, clear run state and samples
  Scalars s0;
  CU(cudaMemcpyAsync(&s0, c->d.sc, sizeof s0, cudaMemcpyDeviceToHost, c->st));
  CU(cudaStreamSynchronize(c->st));
  s0.t = 0.0;
  s0.t_end = INFINITY;
  s0.nsamp = 0;
  s0.done = 0;
  s0.nonfinite = 0;
  c->poisoned = 0;
  s0.steps = 0;
  s0.count = 0;
  s0.lam_bits = 0;
  s0.next_sample = s0.sample_every > 0.0 ? s0.sample_every : INFINITY;
  CU(cudaMemcpyAsync(c->d.sc, &s0, sizeof s0, cudaMemcpyHostToDevice, c->st));
  CU(cudaStreamSynchronize(c->st));
  c->dem_set = 1;
  if ((r = reset_tiles(c))) return r;
  if ((r = reset_ledger(c))) return r;
  if ((r = recompute_dt(c))) return r;
  CU(cudaStreamSynchronize(c->st));
  return DG2_OK;
}

int dg2_set_bc_inflow(dg2_ctx* c, int edge, double s0_m, double len_m, const double* t_knots,
                      const double* q_knots, int nknots) {
  int r = check_arg_ctx(c, false);
  if (r) return r;
  if (edge < 0 || edge > 3) return fail(DG2_E_ARG, "edge must be 0..3");
  if (c->d.n_in >= dg2::kMaxInflow) return fail(DG2_E_ARG, "at most %d inflows", dg2::kMaxInflow);
  if (!t_knots || !q_knots || nknots < 1 || nknots > kMaxKnots)
    return fail(DG2_E_ARG, "need 1..%d knots", kMaxKnots);
  if (!(len_m >= 0.0) || !std::isfinite(s0_m)) return fail(DG2_E_ARG, "bad segment");
  for (int k = 0; k < nknots; ++k) {
    if (!std::isfinite(t_knots[k]) || !std::isfinite(q_knots[k]))
      return fail(DG2_E_ARG, "non-finite knot %d", k);
    if (k && !(t_knots[k] > t_knots[k - 1])) return fail(DG2_E_ARG, "t_knots must increase");
  }
  const bool ew = edge <= 1;
  const int n = ew ? c->d.ny : c->d.nx;
  const double h = ew ? c->d.dy : c->d.dx;
  int nf = 0;
  for (int k = 0; k < n; ++k) {
    const double s = (k + 0.5) * h;
    if (s >= s0_m && s <= s0_m + len_m) ++nf;
  }
  if (nf == 0) return fail(DG2_E_ARG, "no face centre lies in the inflow segment");
  drop_graph(c);
  dg2::InflowDesc& f = c->d.in[c->d.n_in];
  f.edge = edge;
  f.nk = nknots;
  f.koff = c->d.n_in * kMaxKnots;
  f.nfaces = nf;
  f.s0 = s0_m;
  f.s1 = s0_m + len_m;
  f.width = nf * h;
  CU(cudaMemcpyAsync((double*)c->d.knot_t + f.koff, t_knots, nknots * sizeof(double),
                     cudaMemcpyHostToDevice, c->st));
  CU(cudaMemcpyAsync((double*)c->d.knot_q + f.koff, q_knots, nknots * sizeof(double),
                     cudaMemcpyHostToDevice, c->st));
  CU(cudaStreamSynchronize(c->st));
  c->d.n_in += 1;
  if ((r = update_forced_tiles(c))) return r;
  mirror(c);
  return sync_desc(c);
}

int dg2_set_sources(dg2_ctx* c, double rain, double t0, double t1, double px, double py,
                    double qp) {
  int r = check_arg_ctx(c, false);
  if (r) return r;
  if (!std::isfinite(rain) || !std::isfinite(t0) || !std::isfinite(t1) || !std::isfinite(px) ||
      !std::isfinite(py) || !std::isfinite(qp))
    return fail(DG2_E_ARG, "non-finite source parameter");
  drop_graph(c);
  c->d.rain = rain;
  c->d.rain_t0 = t0;
  c->d.rain_t1 = t1;
  c->d.qp = qp;
  c->d.src_idx = -1;
  if (qp != 0.0) {
    int i = (int)std::floor(px / c->d.dx), j = (int)std::floor(py / c->d.dy);
    i = i < 0 ? 0 : (i >= c->d.nx ? c->d.nx - 1 : i);
    j = j < 0 ? 0 : (j >= c->d.ny ? c->d.ny - 1 : j);
    c->d.src_idx = (long long)j * c->d.pitch + i;
  }
  int r2 = update_forced_tiles(c);
  if (r2) return r2;
  mirror(c);
  return sync_desc(c);
}

int dg2_step(dg2_ctx* c, double dt, double* dt_taken) {
  int r = check_arg_ctx(c, true);
  if (r) return r;
  if (!std::isfinite(dt)) return fail(DG2_E_ARG, "dt must be finite");
  if ((r = check_not_poisoned(c))) return r;
  dg2::begin_step_kernel<<<1, 1, 0, c->st>>>(c->d, dt);
  enqueue_step(c, true);
  if ((r = launch_check(c, c->fp32 ? 5 : 6))) return r;
  if (dt_taken) {
    Scalars s;
    if ((r = read_scalars(c, &s))) return r;
    if (s.nonfinite) return fail(DG2_E_NONFINITE, "non-finite state or step at t=%g", s.t);
    *dt_taken = s.last_dt;
  }
  return DG2_OK;
}

int dg2_run_to(dg2_ctx* c, double t_end, int64_t* steps_taken) {
  int r = check_arg_ctx(c, true);
  if (r) return r;
  if (!std::isfinite(t_end)) return fail(DG2_E_ARG, "t_end must be finite");
  if ((r = check_not_poisoned(c))) return r;
  Scalars s;
  if ((r = read_scalars(c, &s))) return r;
  if ((r = check_not_poisoned(c))) return r;
  const long long steps0 = s.steps;
  if (s.t >= t_end) {
    if (steps_taken) *steps_taken = 0;
    return DG2_OK;
  }
  dg2::begin_run_kernel<<<1, 1, 0, c->st>>>(c->d, t_end);
  if ((r = launch_check(c, 1))) return r;
  int level = 0;  // chunk = kChunkMin << level steps
  double t_prev = s.t;
  // The legacy NULL stream cannot be captured: launch the chunk directly there.
  const bool use_graph = c->st != nullptr;
  for (;;) {
    const int chunk = kChunkMin << level;
    if (use_graph) {
      if (!c->graph[level]) {
        cudaGraph_t gr;
        CU(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
        for (int k = 0; k < chunk; ++k) enqueue_step(c);
        cudaError_t e = cudaStreamEndCapture(c->st, &gr);
        if (e != cudaSuccess)
          return fail(DG2_E_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&c->graph[level], gr, 0);
        cudaGraphDestroy(gr);
        if (e != cudaSuccess)
          return fail(DG2_E_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
      }
      CU(cudaGraphLaunch(c->graph[level], c->st));
    } else {
      for (int k = 0; k < chunk; ++k) enqueue_step(c);
      if ((r = launch_check(c, 0))) return r;
    }
    c->launches += (c->fp32 ? 4 : 5) * (int64_t)chunk;
    if ((r = read_scalars(c, &s))) return r;
    if (s.nonfinite) return fail(DG2_E_NONFINITE, "non-finite state or step near t=%g", s.t);
    if (s.done) break;
    if (!(s.t > t_prev)) return fail(DG2_E_NONFINITE, "time stopped advancing at t=%g", s.t);
    t_prev = s.t;
    if ((kChunkMin << level) < kChunkMax) ++level;
  }
  if (steps_taken) *steps_taken = s.steps - steps0;
  return DG2_OK;
}

int dg2_set_gauges(dg2_ctx* c, const double* xy, int ngauge, double every) {
  int r = check_arg_ctx(c, false);
  if (r) return r;
  if (ngauge < 0 || ngauge > c->p.max_gauges)
    return fail(DG2_E_ARG, "ngauge must be 0..%d", c->p.max_gauges);
  if (ngauge > 0 && !xy) return fail(DG2_E_ARG, "xy is null");
  if (!(every >= 0.0) || !std::isfinite(every)) return fail(DG2_E_ARG, "bad sample interval");
  std::vector<long long> idx(ngauge > 0 ? ngauge : 1);
  std::vector<double> xi(ngauge > 0 ? ngauge : 1), et(ngauge > 0 ? ngauge : 1);
  for (int k = 0; k < ngauge; ++k) {
    const double x = xy[2 * k], y = xy[2 * k + 1];
    if (!std::isfinite(x) || !std::isfinite(y)) return fail(DG2_E_ARG, "non-finite gauge %d", k);
    int i = (int)std::floor(x / c->d.dx), j = (int)std::floor(y / c->d.dy);
    i = i < 0 ? 0 : (i >= c->d.nx ? c->d.nx - 1 : i);
    j = j < 0 ? 0 : (j >= c->d.ny ? c->d.ny - 1 : j);
    idx[k] = (long long)j * c->d.pitch + i;
    xi[k] = (x - (i + 0.5) * c->d.dx) / (0.5 * c->d.dx);
    et[k] = (y - (j + 0.5) * c->d.dy) / (0.5 * c->d.dy);
  }
  drop_graph(c);
  if (ngauge > 0) {
    CU(cudaMemcpyAsync((void*)c->d.g_idx, idx.data(), ngauge * sizeof(long long),
                       cudaMemcpyHostToDevice, c->st));
    CU(cudaMemcpyAsync((void*)c->d.g_xi, xi.data(), ngauge * sizeof(double),
                       cudaMemcpyHostToDevice, c->st));
    CU(cudaMemcpyAsync((void*)c->d.g_eta, et.data(), ngauge * sizeof(double),
                       cudaMemcpyHostToDevice, c->st));
  }
  Scalars s;
  if ((r = read_scalars(c, &s))) return r;
  s.sample_every = ngauge > 0 ? every : 0.0;
  s.next_sample = (ngauge > 0 && every > 0.0)
                      ? (std::floor(s.t / every + 1e-9) + 1.0) * every
                      : INFINITY;
  s.nsamp = 0;
  CU(cudaMemcpyAsync(c->d.sc, &s, sizeof s, cudaMemcpyHostToDevice, c->st));
  CU(cudaStreamSynchronize(c->st));
  c->d.ngauge = ngauge;
  mirror(c);
  return sync_desc(c);
}

int dg2_read_gauges(dg2_ctx* c, double* t_out, double* h_out, int cap, int* nsamp) {
  int r = check_arg_ctx(c, false);
  if (r) return r;
  if (cap < 0 || (cap > 0 && (!t_out || (c->d.ngauge > 0 && !h_out))))
    return fail(DG2_E_ARG, "bad output buffers");
  Scalars s;
  if ((r = read_scalars(c, &s))) return r;
  const int kept = s.nsamp < c->d.max_samples ? s.nsamp : c->d.max_samples;
  const int n = kept < cap ? kept : cap;
  if (n > 0) {
    CU(cudaMemcpyAsync(t_out, c->d.samp_t, n * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    if (c->d.ngauge > 0)
      CU(cudaMemcpyAsync(h_out, c->d.samp_h, (size_t)n * c->d.ngauge * sizeof(double),
                         cudaMemcpyDeviceToHost, c->st));
  }
  const int zero = 0;
  CU(cudaMemcpyAsync(&c->d.sc->nsamp, &zero, sizeof(int), cudaMemcpyHostToDevice, c->st));
  CU(cudaStreamSynchronize(c->st));
  if (nsamp) *nsamp = n;
  if (s.nsamp > c->d.max_samples || kept > cap)
    return fail(DG2_E_OVERFLOW, "%d samples recorded, %d returned", s.nsamp, n);
  return DG2_OK;
}

int dg2_mass(dg2_ctx* c, double* mass, double* ledger) {
  int r = check_arg_ctx(c, true);
  if (r) return r;
  launch_mass(c);
  if ((r = launch_check(c, 1))) return r;
  Scalars s;
  if ((r = read_scalars(c, &s))) return r;
  if (mass) *mass = s.mass;
  if (ledger) *ledger = s.ledger;
  return DG2_OK;
}

int dg2_get_state(dg2_ctx* c, double* planes, double* t) {
  int r = check_arg_ctx(c, false);
  if (r) return r;
  if (!planes) return fail(DG2_E_ARG, "planes is null");
  if (c->fp32) {
    // FP32 free-surface modes -> FP64 depth modes h = eta - z
    const int nx = c->f.nx, ny = c->f.ny;
    const size_t n = (size_t)nx * ny;
    std::vector<float> buf(10 * n);
    for (int k = 0; k < 10; ++k)
      CU(cudaMemcpy2DAsync(buf.data() + k * n, nx * sizeof(float), c->f.S + k * c->f.plane,
                           c->f.pitch * sizeof(float), nx * sizeof(float), ny,
                           cudaMemcpyDeviceToHost, c->st));
    std::vector<float> z0, z1x, z1y;
    if ((r = f32_topo_modes(c, z0, z1x, z1y))) return r;
    for (size_t k = 0; k < n; ++k) {
      planes[k] = ((double)buf[k] - (double)z0[k]) + (double)buf[9 * n + k];
      planes[n + k] = (double)buf[n + k] - (double)z1x[k];
      planes[2 * n + k] = (double)buf[2 * n + k] - (double)z1y[k];
    }
    for (size_t k = 3 * n; k < 9 * n; ++k) planes[k] = buf[k];
    Scalars s;
    if ((r = read_scalars(c, &s))) return r;
    if (t) *t = s.t;
    return DG2_OK;
  }
  const size_t w = (size_t)c->d.nx * sizeof(double), pb = (size_t)c->d.pitch * sizeof(double);
  for (int k = 0; k < 9; ++k)
    CU(cudaMemcpy2DAsync(planes + (size_t)k * c->d.nx * c->d.ny, w, c->d.S + k * c->d.plane, pb,
                         w, c->d.ny, cudaMemcpyDeviceToHost, c->st));
  Scalars s;
  if ((r = read_scalars(c, &s))) return r;
  if (t) *t = s.t;
  return DG2_OK;
}

int dg2_set_state(dg2_ctx* c, const double* planes, double t) {
  int r = check_arg_ctx(c, false);
  if (r) return r;
  if (!planes || !std::isfinite(t)) return fail(DG2_E_ARG, "bad planes or t");
  const size_t n = (size_t)9 * c->d.nx * c->d.ny;
  for (size_t k = 0; k < n; ++k)
    if (!std::isfinite(planes[k])) return fail(DG2_E_ARG, "non-finite state value %zu", k);
  if (c->fp32) {
    // FP64 depth modes -> FP32 free-surface modes eta = h + z
    const int nx = c->f.nx, ny = c->f.ny;
    std::vector<float> z0, z1x, z1y;
    if ((r = f32_topo_modes(c, z0, z1x, z1y))) return r;
    std::vector<float> buf(10 * (size_t)nx * ny);
    const size_t m = (size_t)nx * ny;
    for (size_t k = 0; k < m; ++k) {
      const double e0 = planes[k] + (double)z0[k];
      buf[k] = (float)e0;
      buf[9 * m + k] = (float)(e0 - (double)buf[k]);
      buf[m + k] = (float)(planes[m + k] + (double)z1x[k]);
      buf[2 * m + k] = (float)(planes[2 * m + k] + (double)z1y[k]);
    }
    for (size_t k = 3 * m; k < 9 * m; ++k) buf[k] = (float)planes[k];
    for (int k = 0; k < 10; ++k)
      CU(cudaMemcpy2DAsync(c->f.S + k * c->f.plane, c->f.pitch * sizeof(float), buf.data() + k * m,
                           nx * sizeof(float), nx * sizeof(float), ny, cudaMemcpyHostToDevice,
                           c->st));
    CU(cudaStreamSynchronize(c->st));
  } else {
    const size_t w = (size_t)c->d.nx * sizeof(double), pb = (size_t)c->d.pitch * sizeof(double);
    for (int k = 0; k < 9; ++k)
      CU(cudaMemcpy2DAsync(c->d.S + k * c->d.plane, pb, planes + (size_t)k * c->d.nx * c->d.ny,
                           w, w, c->d.ny, cudaMemcpyHostToDevice, c->st));
  }
  Scalars s;
  if ((r = read_scalars(c, &s))) return r;
  s.t = t;
  s.done = 0;
  s.nonfinite = 0;
  c->poisoned = 0;
  s.t_end = INFINITY;
  s.next_sample = s.sample_every > 0.0 ? (std::floor(t / s.sample_every + 1e-9) + 1.0) * s.sample_every
                                       : INFINITY;
  CU(cudaMemcpyAsync(c->d.sc, &s, sizeof s, cudaMemcpyHostToDevice, c->st));
  c->dem_set = 1;
  if ((r = reset_tiles(c))) return r;
  if ((r = reset_ledger(c))) return r;
  if ((r = recompute_dt(c))) return r;
  CU(cudaStreamSynchronize(c->st));
  return DG2_OK;
}

int dg2_get_topo(dg2_ctx* c, double* planes3) {
  int r = check_arg_ctx(c, false);
  if (r) return r;
  if (!planes3) return fail(DG2_E_ARG, "planes3 is null");
  if (c->fp32) {
    std::vector<float> z0, z1x, z1y;
    if ((r = f32_topo_modes(c, z0, z1x, z1y))) return r;
    const size_t n = z0.size();
    for (size_t k = 0; k < n; ++k) {
      planes3[k] = z0[k];
      planes3[n + k] = z1x[k];
      planes3[2 * n + k] = z1y[k];
    }
    return DG2_OK;
  }
  const size_t w = (size_t)c->d.nx * sizeof(double), pb = (size_t)c->d.pitch * sizeof(double);
  for (int k = 0; k < 3; ++k)
    CU(cudaMemcpy2DAsync(planes3 + (size_t)k * c->d.nx * c->d.ny, w, c->d.Z + k * c->d.plane, pb,
                         w, c->d.ny, cudaMemcpyDeviceToHost, c->st));
  CU(cudaStreamSynchronize(c->st));
  return DG2_OK;
}

int dg2_get_time(dg2_ctx* c, double* t, double* dt_next) {
  int r = check_arg_ctx(c, false);
  if (r) return r;
  Scalars s;
  if ((r = read_scalars(c, &s))) return r;
  if (t) *t = s.t;
  if (dt_next) *dt_next = s.dt_cfl;
  return DG2_OK;
}

int dg2_enable_kernel_timing(dg2_ctx* c, int enable) {
  int r = check_arg_ctx(c, false);
  if (r) return r;
  c->timing = enable ? 1 : 0;
  c->timed_steps = 0;
  return DG2_OK;
}

int dg2_kernel_times(dg2_ctx* c, double* ms3, int64_t* nsteps) {
  int r = check_arg_ctx(c, false);
  if (r) return r;
  if (!ms3) return fail(DG2_E_ARG, "ms3 is null");
  CU(cudaStreamSynchronize(c->st));
  double acc[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < c->timed_steps; ++k)
    for (int q = 0; q < 3; ++q) {
      float ms = 0.f;
      CU(cudaEventElapsedTime(&ms, c->ev[4 * k + q], c->ev[4 * k + q + 1]));
      acc[q] += ms;
    }
  for (int q = 0; q < 3; ++q) ms3[q] = acc[q];
  if (nsteps) *nsteps = c->timed_steps;
  c->timed_steps = 0;
  return DG2_OK;
}

int64_t dg2_launch_count(const dg2_ctx* c) { return c ? c->launches : -1; }

int dg2_get_steps(dg2_ctx* c, int64_t* steps) {
  int r = check_arg_ctx(c, false);
  if (r) return r;
  if (!steps) return fail(DG2_E_ARG, "steps is null");
  Scalars s;
  if ((r = read_scalars(c, &s))) return r;
  *steps = s.steps;
  return DG2_OK;
}

int dg2_tile_stats(dg2_ctx* c, int* ntiles, int* n_active, int* n_frontier,
                   int64_t* tiles_computed) {
  int r = check_arg_ctx(c, false);
  if (r) return r;
  Scalars s;
  if ((r = read_scalars(c, &s))) return r;
  if (ntiles) *ntiles = c->d.tiles.ntiles;
  if (n_active) *n_active = s.n_act;
  if (n_frontier) *n_frontier = s.n_front;
  if (tiles_computed) *tiles_computed = s.tiles_done;
  return DG2_OK;
}

int dg2_tile_shape(dg2_ctx* c, int* w, int* h) {
  if (!c) return fail(DG2_E_ARG, "null context");
  if (w) *w = tile_w(c);
  if (h) *h = tile_h(c);
  return DG2_OK;
}

int dg2_destroy(dg2_ctx* c) {
  if (!c) return fail(DG2_E_ARG, "null context");
  drop_graph(c);
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  delete c;
  return DG2_OK;
}

}  // extern "C"

namespace dg2 {
bool ctx_fp32(const dg2_ctx* c) { return c->fp32 != 0; }
int ctx_variant(const dg2_ctx* c) { return c->p.variant; }
bool ctx_ready(const dg2_ctx* c) { return c->dem_set != 0; }
cudaStream_t ctx_stream(const dg2_ctx* c) { return c->st; }
const f32::D32& ctx_d32(const dg2_ctx* c) { return c->f; }
void ctx_forced_mask(const dg2_ctx* c, int tw, int th, std::vector<unsigned char>& m) {
  forced_mask(c->d, tw, th, m);
}
bool ctx_rains(const dg2_ctx* c) { return c->d.rain != 0.0; }
int ctx_reset_tiles(dg2_ctx* c) {
  drop_graph(c);
  return reset_tiles(c);
}
void ctx_count_launches(dg2_ctx* c, int64_t n) { c->launches += n; }
}  // namespace dg2
