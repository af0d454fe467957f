// dg2_ens.cu -- ensembles of FP32 problems advanced together (C ABI in
// include/dg2.h, dg2_ens_*).
//
// Every member is an ordinary FP32 context (its own grid, DEM, Manning field,
// inflows, gauges, time and Courant step).  One step of the ensemble is four
// launches for all members at once: stage 1 (with friction fused) and stage 2
// over one list of (member, tile) entries, a one-block-per-member end of step
// (time, ledger, gauges, the member's next dt), and a lists kernel that
// classifies every tile of every unfinished member and appends the computed
// ones to the next step's list.  A member whose run has reached t_end drops out of the lists;
// the others keep stepping with their own dt.  Chunks of steps are replayed
// from CUDA graphs.  The tile shape (cells per tile, one thread per cell) is a
// template parameter picked among kShapes by dg2_ens_autotune, which times
// real steps of the run under each shape: every shape computes the same cell
// updates bit for bit, only the speed differs.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/dg2.h"
#include "dg2_device.cuh"
#include "dg2_fs32.cuh"
#include "dg2_fs32_staged.cuh"
#include "dg2_internal.h"

using dg2::Scalars;
using dg2::Tiles;
using dg2::f32::D32;

namespace dg2 {
namespace ens {

// Tile shapes the autotuner chooses from (width x height cells).  Every side
// is at least 4 cells: the dependence radius of one DG2-LL step (2 cells per
// stage), so a tile's 3 x 3 tile neighbourhood covers it.
struct Shape {
  int w, h;
};
constexpr Shape kShapes[] = {{32, 8}, {32, 4}, {16, 8}, {64, 4}, {16, 16}};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);
constexpr int kMaxMembers = 1 << (31 - kTileBits);  // list entry = member << kTileBits | tile

__device__ __forceinline__ void unpack(int ent, int& m, int& tile) {
  m = ent >> kTileBits;
  tile = ent & ((1 << kTileBits) - 1);
}

// A member that reached t_end in the previous step keeps its list entries for
// that one step (its lists were built before it was known); its tiles are
// skipped in the stage kernels.

// resident 256-thread blocks per SM asked of the register allocator for the FP32
// stage kernels (twice that for 128-thread tiles)
#ifndef DG2_MINB32
#define DG2_MINB32 3
#endif

// Shared memory of a stage block (dynamic: above the 48 KB static limit for some
// shapes; the limit is raised once per process by prepare_stage32).
template <bool LL, int STAGE, int BX, int BY>
constexpr int stage32_smem() {
  return (int)sizeof(f32::StagedSmem32<LL, STAGE, BX, BY>);
}

template <bool LL, int STAGE, int BX, int BY>
__global__ void __launch_bounds__(BX* BY, BX * BY <= 128 ? 2 * DG2_MINB32 : DG2_MINB32)
    ens_stage_kernel(EnsDev E) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& sm = *reinterpret_cast<f32::StagedSmem32<LL, STAGE, BX, BY>*>(smem_raw);
  __shared__ f32::Blk32 blk;
  // the member's descriptor, copied once per change of member: the stage reads its
  // fields from shared memory instead of global memory
  __shared__ __align__(16) D32 dsm;
  int m_cached = -1;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const bool t0 = tx == 0 && ty == 0;
  const int n_act = E.es->n_act;
  for (int e = blockIdx.x; e < n_act; e += gridDim.x) {
    int m, tile;
    unpack(E.list[e], m, tile);
    if (m != m_cached) {
      static_assert(sizeof(D32) % 16 == 0, "descriptor copied as 16-byte words");
      const int4* src = reinterpret_cast<const int4*>(E.desc + m);
      int4* dst = reinterpret_cast<int4*>(&dsm);
      for (int k = ty * BX + tx; k < (int)(sizeof(D32) / 16); k += BX * BY) dst[k] = src[k];
      m_cached = m;
      __syncthreads();
    }
    const D32& d = dsm;
    if (t0) {
      // the member's step constants, FP64 once per tile
      const Scalars* sc = d.sc;
      const double dtd = sc->dt;
      const double ts = STAGE == 1 ? sc->t : sc->t + dtd;
      blk.dtd = dtd;
      blk.ts = ts;
      blk.dt = (float)dtd;
      blk.gdt = (float)(dtd * (double)d.g);
      blk.rain = d.rain != 0.0 && ts >= d.rain_t0 && ts < d.rain_t1;
      blk.rainf = (float)d.rain;
      blk.skip = sc->done;
    }
    __syncthreads();
    if (blk.skip) {
      __syncthreads();
      continue;
    }
    const int ntx = d.tiles.ntx, nty = d.tiles.nty;
    const int bx = tile % ntx, by = tile / ntx;
    float brate = 0.f, lam = 0.f;
    bool bad = false, nonq = false;
    f32::stage32_staged<LL, STAGE, BX, BY>(d, sm, blk, bx, by, brate, lam, bad, nonq);
    if (bx == 0 || by == 0 || bx == ntx - 1 || by == nty - 1) {
      const double bsum = block_sum<BX * BY>((double)brate, sm.red);
      if (t0) d.bpart[(STAGE - 1) * d.tiles.ntiles + tile] = bsum;
    }
    if (STAGE == 2) {
      const int any_nonq = __syncthreads_or(nonq);
      if (t0) d.tiles.flag[tile] = any_nonq ? 1 : 0;
      if (__syncthreads_or(bad) && t0) d.sc->nonfinite = 1;
      const double bl = (double)block_max_f<BX * BY>(lam, sm.redf);
      if (t0 && bl > 0.0)
        atomicMax(&d.sc->lam_bits, (unsigned long long)__double_as_longlong(bl));
    }
    __syncthreads();
  }
  if (STAGE == 1) {
    // frontier tiles: a computed neighbour reads their stage state as halo
    const int n_front = E.es->n_front;
    for (int e = blockIdx.x; e < n_front; e += gridDim.x) {
      int m, tile;
      unpack(E.front[e], m, tile);
      const D32& d = E.desc[m];
      const int ntx = d.tiles.ntx;
      const int i = (tile % ntx) * BX + tx, j = (tile / ntx) * BY + ty;
      if (i < d.nx && j < d.ny && !d.sc->done) {
        const long long P = d.plane, c = (long long)j * d.pitch + i;
#pragma unroll
        for (int k = 0; k < f32::kPlanes32; ++k) d.T[k * P + c] = d.S[k * P + c];
      }
    }
  }
}

// End of step of every member (one block each): time, ledger, gauges, the
// member's next dt; counts members that reach t_end; opens the next lists.
__global__ void __launch_bounds__(kFinThreads) ens_finalize_kernel(EnsDev E, int lists_only) {
  const D32& d = E.desc[blockIdx.x];
  __shared__ int was_done;
  if (threadIdx.x == 0) was_done = d.sc->done;
  __syncthreads();
  f32::finalize32_body(d, lists_only);
  __syncthreads();
  if (threadIdx.x == 0 && !lists_only && !was_done && d.sc->done) atomicAdd(&E.es->n_done, 1);
  if (threadIdx.x == 0 && d.sc->nonfinite) E.es->bad = 1;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    E.es->n_act = 0;
    E.es->n_front = 0;
  }
}

// Tile lists of the next step for every member that took this step, by the rule of
// lists_kernel (3 x 3 computed, 5 x 5 frontier), appended to the ensemble's
// lists.  blockIdx.z = member; LTX x LTY tiles per block.
__global__ void __launch_bounds__(LTX* LTY) ens_lists_kernel(EnsDev E) {
  const D32& d = E.desc[blockIdx.z];
  const Tiles& T = d.tiles;
  const int ntx = T.ntx, nty = T.nty;
  if ((int)blockIdx.x * LTX >= ntx || (int)blockIdx.y * LTY >= nty) return;
  Scalars* sc = d.sc;
  // A problem that did not take this step (its run is done) keeps its tiles in
  // the lists when it is alone (its flags are unchanged, and a later dg2_step
  // continues from them; the kernels skip a done problem's tiles); an
  // ensemble drops it (dg2_ens_run_to rebuilds every list when it starts).
  const bool live = E.nmem == 1 || !sc->skip_lists;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * LTX + tx;
  const int bx = blockIdx.x * LTX + tx, by = blockIdx.y * LTY + ty;
  const bool in = bx < ntx && by < nty;
  const int t = by * ntx + bx;
  const bool every = !T.skip || T.all_forced;
  __shared__ unsigned char busy[LTY + 4][LTX + 4];
  __shared__ int wa[LTY], wf[LTY], base[2];
  if (!every) {
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
  }
  __syncthreads();
  bool a = false, f = false;
  if (in && live) {
    if (every) {
      a = true;
    } else {
#pragma unroll
      for (int oy = -2; oy <= 2; ++oy)
#pragma unroll
        for (int ox = -2; ox <= 2; ++ox) {
          if (!busy[ty + 2 + oy][tx + 2 + ox]) continue;
          if (ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1) a = true;
          else f = true;
        }
      if (a) f = false;
    }
  }
  if (in) T.act[t] = a ? 1 : 0;
  const unsigned ba = __ballot_sync(0xffffffffu, a), bf = __ballot_sync(0xffffffffu, f);
  const int lane = tid & 31;
  if (lane == 0) { wa[ty] = __popc(ba); wf[ty] = __popc(bf); }
  __syncthreads();
  if (tid == 0) {
    int sa = 0, sf = 0;
    for (int w = 0; w < LTY; ++w) {
      const int xa = wa[w], xf = wf[w];
      wa[w] = sa; sa += xa;
      wf[w] = sf; sf += xf;
    }
    base[0] = sa ? atomicAdd(&E.es->n_act, sa) : 0;
    base[1] = sf ? atomicAdd(&E.es->n_front, sf) : 0;
    if (sa) atomicAdd(&sc->n_act, sa);  // the member's own counts (tiles_done)
    if (sf) atomicAdd(&sc->n_front, sf);
  }
  __syncthreads();
  const unsigned below = (1u << lane) - 1u;
  const int ent = ((int)blockIdx.z << kTileBits) | t;
  if (a) E.list[base[0] + wa[ty] + __popc(ba & below)] = ent;
  if (f) E.front[base[1] + wf[ty] + __popc(bf & below)] = ent;
}

// Starts a run of every member to t_end (the single-problem run_to start);
// counts the members already there.
__global__ void ens_begin_run_kernel(EnsDev E, double t_end) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= E.nmem) return;
  Scalars* sc = E.desc[m].sc;
  begin_run_body(sc, t_end);
  if (sc->done) atomicAdd(&E.es->n_done, 1);
}

template <int BX, int BY>
void launch_shape32(const EnsDev& E, bool ll, int stage, int grid, cudaStream_t st) {
  const dim3 b(BX, BY);
  if (ll) {
    if (stage == 1)
      ens_stage_kernel<true, 1, BX, BY><<<grid, b, stage32_smem<true, 1, BX, BY>(), st>>>(E);
    else
      ens_stage_kernel<true, 2, BX, BY><<<grid, b, stage32_smem<true, 2, BX, BY>(), st>>>(E);
  } else {
    if (stage == 1)
      ens_stage_kernel<false, 1, BX, BY><<<grid, b, stage32_smem<false, 1, BX, BY>(), st>>>(E);
    else
      ens_stage_kernel<false, 2, BX, BY><<<grid, b, stage32_smem<false, 2, BX, BY>(), st>>>(E);
  }
}

template <int BX, int BY>
void prepare_shape32() {
  cudaFuncSetAttribute(ens_stage_kernel<true, 1, BX, BY>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, stage32_smem<true, 1, BX, BY>());
  cudaFuncSetAttribute(ens_stage_kernel<true, 2, BX, BY>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, stage32_smem<true, 2, BX, BY>());
  cudaFuncSetAttribute(ens_stage_kernel<false, 1, BX, BY>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, stage32_smem<false, 1, BX, BY>());
  cudaFuncSetAttribute(ens_stage_kernel<false, 2, BX, BY>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, stage32_smem<false, 2, BX, BY>());
}

void launch_stage32(const EnsDev& E, int tw, bool ll, int stage, int grid, cudaStream_t st) {
  if (tw == 16) launch_shape32<16, 8>(E, ll, stage, grid, st);
  else launch_shape32<32, 8>(E, ll, stage, grid, st);
}

void launch_end_of_step(const EnsDev& E, int nmem, dim3 lgrid, int lists_only, cudaStream_t st) {
  ens_finalize_kernel<<<nmem, kFinThreads, 0, st>>>(E, lists_only);
  ens_lists_kernel<<<lgrid, dim3(LTX, LTY), 0, st>>>(E);
}

template <int BX, int BY>
void occupancy_shape32(bool ll, int* s1, int* s2) {
  const int nt = BX * BY;
  prepare_shape32<BX, BY>();
  if (ll) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(s1, ens_stage_kernel<true, 1, BX, BY>, nt,
                                                  stage32_smem<true, 1, BX, BY>());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(s2, ens_stage_kernel<true, 2, BX, BY>, nt,
                                                  stage32_smem<true, 2, BX, BY>());
  } else {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(s1, ens_stage_kernel<false, 1, BX, BY>, nt,
                                                  stage32_smem<false, 1, BX, BY>());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(s2, ens_stage_kernel<false, 2, BX, BY>, nt,
                                                  stage32_smem<false, 2, BX, BY>());
  }
}

void occupancy32(int tw, bool ll, int* s1, int* s2) {
  if (tw == 16) occupancy_shape32<16, 8>(ll, s1, s2);
  else occupancy_shape32<32, 8>(ll, s1, s2);
}

}  // namespace ens
}  // namespace dg2

using namespace dg2::ens;

namespace {

int efail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  dg2::set_error_text(buf);
  return code;
}

#define ECU(call)                                                                       \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return efail(DG2_E_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));         \
  } while (0)

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }
constexpr int kChunkMin = 16, kChunkMax = 1024, kLevels = 7;

int max_tiles(int nx, int ny) {
  int best = 0;
  for (const Shape& s : kShapes) {
    const int n = ((nx + s.w - 1) / s.w) * ((ny + s.h - 1) / s.h);
    best = n > best ? n : best;
  }
  return best;
}

struct EnsLayout {
  size_t off_desc, off_es, off_list, off_front, total;
  std::vector<size_t> off_flag, off_act, off_forced, off_bpart;
  long long list_cap;
};

bool ens_layout(dg2_ctx* const* mem, int n, EnsLayout& L) {
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align_up(o + bytes);
    return at;
  };
  L.off_desc = take(sizeof(D32) * (size_t)n);
  L.off_es = take(sizeof(EnsScalars));
  L.list_cap = 0;
  L.off_flag.resize(n);
  L.off_act.resize(n);
  L.off_forced.resize(n);
  L.off_bpart.resize(n);
  for (int k = 0; k < n; ++k) {
    const D32& f = dg2::ctx_d32(mem[k]);
    const int mt = max_tiles(f.nx, f.ny);
    if (mt >= (1 << kTileBits)) return false;
    L.list_cap += mt;
    L.off_flag[k] = take((size_t)mt);
    L.off_act[k] = take((size_t)mt);
    L.off_forced[k] = take((size_t)mt);
    L.off_bpart[k] = take(2 * (size_t)mt * sizeof(double));
  }
  L.off_list = take((size_t)L.list_cap * sizeof(int));
  L.off_front = take((size_t)L.list_cap * sizeof(int));
  L.total = o;
  return true;
}

}  // namespace

struct dg2_ens {
  std::vector<dg2_ctx*> mem;
  std::vector<D32> desc;  // host copies of the member descriptors
  EnsLayout lay;
  char* ws;
  cudaStream_t st;
  EnsDev E;
  int variant;
  int shape;              // index into kShapes
  int grid_st1, grid_st2;
  dim3 lgrid;
  int max_ntx, max_nty;
  cudaGraphExec_t graph[kLevels];
  int64_t launches;
  int64_t steps;          // ensemble steps taken (the longest member's count)
  double tune_ms[kNumShapes];
};

namespace {

void drop_graphs(dg2_ens* e) {
  for (auto& g : e->graph) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
  }
}

template <int BX, int BY>
void occupancy(dg2_ens* e, int& s1, int& s2) {
  occupancy_shape32<BX, BY>(e->variant == DG2_LL, &s1, &s2);
}

// Lays the members' tiling out for shape `si` from their current parameters:
// tile grids, forced masks, every tile flagged (the members' states may have
// changed since the ensemble last ran), descriptors uploaded, launch grids
// sized.  Graphs are dropped when the shape or a descriptor changed.
int set_shape(dg2_ens* e, int si) {
  const Shape sh = kShapes[si];
  bool changed = si != e->shape;
  e->shape = si;
  const int n = (int)e->mem.size();
  long long total_tiles = 0;
  e->max_ntx = e->max_nty = 1;
  std::vector<unsigned char> m;
  for (int k = 0; k < n; ++k) {
    D32 f = dg2::ctx_d32(e->mem[k]);
    Tiles& T = f.tiles;
    T.ntx = (f.nx + sh.w - 1) / sh.w;
    T.nty = (f.ny + sh.h - 1) / sh.h;
    T.ntiles = T.ntx * T.nty;
    T.flag = (unsigned char*)(e->ws + e->lay.off_flag[k]);
    T.act = (unsigned char*)(e->ws + e->lay.off_act[k]);
    T.forced = (const unsigned char*)(e->ws + e->lay.off_forced[k]);
    T.list = nullptr;
    T.front = nullptr;
    T.all_forced = dg2::ctx_rains(e->mem[k]) ? 1 : 0;
    f.bpart = (double*)(e->ws + e->lay.off_bpart[k]);
    dg2::ctx_forced_mask(e->mem[k], sh.w, sh.h, m);
    ECU(cudaMemcpyAsync((void*)T.forced, m.data(), m.size(), cudaMemcpyHostToDevice, e->st));
    ECU(cudaMemsetAsync(T.flag, 1, (size_t)T.ntiles, e->st));
    ECU(cudaMemsetAsync(T.act, 0, (size_t)T.ntiles, e->st));
    ECU(cudaMemsetAsync(f.bpart, 0, 2 * (size_t)T.ntiles * sizeof(double), e->st));
    if (memcmp(&e->desc[k], &f, sizeof f) != 0) changed = true;
    e->desc[k] = f;
    total_tiles += T.ntiles;
    e->max_ntx = T.ntx > e->max_ntx ? T.ntx : e->max_ntx;
    e->max_nty = T.nty > e->max_nty ? T.nty : e->max_nty;
  }
  ECU(cudaMemcpyAsync(e->ws + e->lay.off_desc, e->desc.data(), sizeof(D32) * (size_t)n,
                      cudaMemcpyHostToDevice, e->st));
  ECU(cudaStreamSynchronize(e->st));
  if (!changed) return DG2_OK;
  drop_graphs(e);
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int o1 = 1, o2 = 1;
  switch (si) {
    case 0: occupancy<32, 8>(e, o1, o2); break;
    case 1: occupancy<32, 4>(e, o1, o2); break;
    case 2: occupancy<16, 8>(e, o1, o2); break;
    case 3: occupancy<64, 4>(e, o1, o2); break;
    default: occupancy<16, 16>(e, o1, o2); break;
  }
  cudaGetLastError();
  auto gsz = [&](int occ) {
    long long g = (long long)nsm * (occ > 0 ? occ : 1);
    return (int)(g < total_tiles ? g : total_tiles);
  };
  e->grid_st1 = gsz(o1);
  e->grid_st2 = gsz(o2);
  e->lgrid = dim3((e->max_ntx + dg2::LTX - 1) / dg2::LTX, (e->max_nty + dg2::LTY - 1) / dg2::LTY, n);
  return DG2_OK;
}

template <int BX, int BY>
void enqueue_step_shape(dg2_ens* e) {
  const bool ll = e->variant == DG2_LL;
  launch_shape32<BX, BY>(e->E, ll, 1, e->grid_st1, e->st);
  launch_shape32<BX, BY>(e->E, ll, 2, e->grid_st2, e->st);
}

void enqueue_lists(dg2_ens* e, int lists_only) {
  const int n = (int)e->mem.size();
  ens_finalize_kernel<<<n, dg2::kFinThreads, 0, e->st>>>(e->E, lists_only);
  ens_lists_kernel<<<e->lgrid, dim3(dg2::LTX, dg2::LTY), 0, e->st>>>(e->E);
}

// One step of every unfinished member: 4 launches.
void enqueue_step(dg2_ens* e) {
  switch (e->shape) {
    case 0: enqueue_step_shape<32, 8>(e); break;
    case 1: enqueue_step_shape<32, 4>(e); break;
    case 2: enqueue_step_shape<16, 8>(e); break;
    case 3: enqueue_step_shape<64, 4>(e); break;
    default: enqueue_step_shape<16, 16>(e); break;
  }
  enqueue_lists(e, 0);
}

int check_launch(dg2_ens* e, int64_t n) {
  e->launches += n;
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return efail(DG2_E_CUDA, "kernel launch failed: %s", cudaGetErrorString(err));
  return DG2_OK;
}

int read_es(dg2_ens* e, EnsScalars* out) {
  ECU(cudaMemcpyAsync(out, e->E.es, sizeof(EnsScalars), cudaMemcpyDeviceToHost, e->st));
  ECU(cudaStreamSynchronize(e->st));
  return DG2_OK;
}

// Starts a run to t_end: member starts, done count, first lists.
int begin_run(dg2_ens* e, double t_end) {
  const int n = (int)e->mem.size();
  ECU(cudaMemsetAsync(e->E.es, 0, sizeof(EnsScalars), e->st));
  ens_begin_run_kernel<<<(n + 127) / 128, 128, 0, e->st>>>(e->E, t_end);
  enqueue_lists(e, 1);
  return check_launch(e, 3);
}

// Replays `chunk` steps (graph of level `lv` when capturable).
int run_chunk(dg2_ens* e, int lv) {
  const int chunk = kChunkMin << lv;
  if (e->st) {
    if (!e->graph[lv]) {
      cudaGraph_t gr;
      ECU(cudaStreamBeginCapture(e->st, cudaStreamCaptureModeThreadLocal));
      for (int k = 0; k < chunk; ++k) enqueue_step(e);
      cudaError_t err = cudaStreamEndCapture(e->st, &gr);
      if (err != cudaSuccess) return efail(DG2_E_CUDA, "graph capture failed: %s", cudaGetErrorString(err));
      err = cudaGraphInstantiate(&e->graph[lv], gr, 0);
      cudaGraphDestroy(gr);
      if (err != cudaSuccess) return efail(DG2_E_CUDA, "graph instantiate failed: %s", cudaGetErrorString(err));
    }
    ECU(cudaGraphLaunch(e->graph[lv], e->st));
    return check_launch(e, 4 * (int64_t)chunk);
  }
  for (int k = 0; k < chunk; ++k) enqueue_step(e);
  return check_launch(e, 4 * (int64_t)chunk);
}

// After the ensemble moved the members' states, their own tilings must
// recompute every tile once.
int release_members(dg2_ens* e) {
  ECU(cudaStreamSynchronize(e->st));
  for (dg2_ctx* c : e->mem) {
    int r = dg2::ctx_reset_tiles(c);
    if (r) return r;
    ECU(cudaStreamSynchronize(dg2::ctx_stream(c)));
  }
  return DG2_OK;
}

int check_ens(dg2_ens* e) {
  if (!e) return efail(DG2_E_ARG, "null ensemble");
  return DG2_OK;
}

int sync_members(dg2_ens* e) {
  for (dg2_ctx* c : e->mem) ECU(cudaStreamSynchronize(dg2::ctx_stream(c)));
  return DG2_OK;
}

}  // namespace

extern "C" {

size_t dg2_ens_workspace_bytes(dg2_ctx* const* members, int nmembers) {
  if (!members || nmembers < 1 || nmembers > kMaxMembers) return 0;
  for (int k = 0; k < nmembers; ++k)
    if (!members[k] || !dg2::ctx_fp32(members[k])) return 0;
  EnsLayout L;
  if (!ens_layout(members, nmembers, L)) return 0;
  return L.total;
}

int dg2_ens_create(dg2_ens** out, dg2_ctx* const* members, int nmembers, void* dev_workspace,
                   size_t ws_bytes, void* cuda_stream) {
  if (!out) return efail(DG2_E_ARG, "out is null");
  *out = nullptr;
  if (!members || nmembers < 1 || nmembers > kMaxMembers)
    return efail(DG2_E_ARG, "nmembers must be 1..%d", kMaxMembers);
  int variant = -1;
  for (int k = 0; k < nmembers; ++k) {
    dg2_ctx* c = members[k];
    if (!c) return efail(DG2_E_ARG, "member %d is null", k);
    if (!dg2::ctx_fp32(c)) return efail(DG2_E_ARG, "member %d is not an FP32 context", k);
    if (!dg2::ctx_ready(c)) return efail(DG2_E_STATE, "member %d has no DEM or state", k);
    if (variant < 0) variant = dg2::ctx_variant(c);
    if (dg2::ctx_variant(c) != variant) return efail(DG2_E_ARG, "members mix DG2-NL and DG2-LL");
    for (int q = 0; q < k; ++q)
      if (members[q] == c) return efail(DG2_E_ARG, "member %d appears twice", k);
  }
  if (!dev_workspace || ((uintptr_t)dev_workspace % kAlign))
    return efail(DG2_E_ARG, "workspace must be non-null and 256-byte aligned");
  dg2_ens* e = new dg2_ens();
  e->mem.assign(members, members + nmembers);
  if (!ens_layout(members, nmembers, e->lay)) {
    delete e;
    return efail(DG2_E_ARG, "a member has too many tiles");
  }
  if (ws_bytes < e->lay.total) {
    const size_t need = e->lay.total;
    delete e;
    return efail(DG2_E_NOMEM, "workspace too small: %zu < %zu bytes", ws_bytes, need);
  }
  e->ws = (char*)dev_workspace;
  e->st = (cudaStream_t)cuda_stream;
  e->variant = variant;
  e->desc.resize(nmembers);
  for (auto& g : e->graph) g = nullptr;
  e->launches = 0;
  e->steps = 0;
  for (double& t : e->tune_ms) t = -1.0;
  e->E.desc = (const D32*)(e->ws + e->lay.off_desc);
  e->E.list = (int*)(e->ws + e->lay.off_list);
  e->E.front = (int*)(e->ws + e->lay.off_front);
  e->E.es = (EnsScalars*)(e->ws + e->lay.off_es);
  e->E.nmem = nmembers;
  e->shape = -1;
  int r = sync_members(e);
  if (!r) r = set_shape(e, 0);
  if (r) {
    delete e;
    return r;
  }
  *out = e;
  return DG2_OK;
}

int dg2_ens_set_tile_shape(dg2_ens* e, int tile_w, int tile_h) {
  int r = check_ens(e);
  if (r) return r;
  for (int k = 0; k < kNumShapes; ++k)
    if (kShapes[k].w == tile_w && kShapes[k].h == tile_h) return set_shape(e, k);
  return efail(DG2_E_ARG, "unsupported tile shape %dx%d", tile_w, tile_h);
}

int dg2_ens_tile_shape(const dg2_ens* e, int* tile_w, int* tile_h) {
  if (!e) return efail(DG2_E_ARG, "null ensemble");
  if (tile_w) *tile_w = kShapes[e->shape].w;
  if (tile_h) *tile_h = kShapes[e->shape].h;
  return DG2_OK;
}

int dg2_ens_run_to(dg2_ens* e, double t_end, int64_t* steps_taken) {
  int r = check_ens(e);
  if (r) return r;
  if (!std::isfinite(t_end)) return efail(DG2_E_ARG, "t_end must be finite");
  if ((r = sync_members(e))) return r;
  if ((r = set_shape(e, e->shape))) return r;
  if ((r = begin_run(e, t_end))) return r;
  EnsScalars s;
  if ((r = read_es(e, &s))) return r;
  // the start of a run gathers the members' non-finite flags: a member whose state
  // became non-finite is refused until dg2_set_state / dg2_set_dem restore it
  if (s.bad)
    return efail(DG2_E_NONFINITE, "a member's state is non-finite; restore it with "
                                  "dg2_set_state or dg2_set_dem before running");
  const int n = (int)e->mem.size();
  int64_t taken = 0;
  int lv = 0;
  // Every live member advances its own t by a positive dt each step (a zero or
  // non-finite dt raises its non-finite flag), and lands on t_end exactly.
  while (s.n_done < n) {
    if ((r = run_chunk(e, lv))) return r;
    taken += kChunkMin << lv;
    if ((r = read_es(e, &s))) return r;
    if (s.bad) return efail(DG2_E_NONFINITE, "a member's state or step became non-finite");
    if ((kChunkMin << lv) < kChunkMax) ++lv;
  }
  e->steps += taken;
  if (steps_taken) *steps_taken = taken;
  return release_members(e);
}

int dg2_ens_autotune(dg2_ens* e, double t_end, int steps_per_trial, int* tile_w, int* tile_h) {
  int r = check_ens(e);
  if (r) return r;
  if (!std::isfinite(t_end)) return efail(DG2_E_ARG, "t_end must be finite");
  if (steps_per_trial < 4) return efail(DG2_E_ARG, "steps_per_trial must be >= 4");
  if ((r = sync_members(e))) return r;
  if ((r = begin_run(e, t_end))) return r;
  {
    EnsScalars s0;
    if ((r = read_es(e, &s0))) return r;
    if (s0.bad)
      return efail(DG2_E_NONFINITE, "a member's state is non-finite; restore it with "
                                    "dg2_set_state or dg2_set_dem before tuning");
  }
  cudaEvent_t a, b;
  ECU(cudaEventCreate(&a));
  ECU(cudaEventCreate(&b));
  double best = INFINITY;
  int best_k = 0;
  // two passes over the shapes, each trial timed after one untimed step that
  // absorbs the all-tiles step a new tiling starts with; the better pass counts
  for (double& t : e->tune_ms) t = INFINITY;
  for (int pass = 0; pass < 2 && !r; ++pass) {
    for (int k = 0; k < kNumShapes && !r; ++k) {
      if ((r = set_shape(e, k))) break;
      enqueue_lists(e, 1);  // lists for the new tiling (every tile once)
      enqueue_step(e);
      if ((r = check_launch(e, 6))) break;
      cudaEventRecord(a, e->st);
      for (int q = 0; q < steps_per_trial; ++q) enqueue_step(e);
      cudaEventRecord(b, e->st);
      if ((r = check_launch(e, 4 * (int64_t)steps_per_trial))) break;
      cudaError_t err = cudaEventSynchronize(b);
      if (err != cudaSuccess) { r = efail(DG2_E_CUDA, "autotune: %s", cudaGetErrorString(err)); break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      e->steps += steps_per_trial + 1;
      const double per = ms / steps_per_trial;
      if (per < e->tune_ms[k]) e->tune_ms[k] = per;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (r) return r;
  for (int k = 0; k < kNumShapes; ++k)
    if (e->tune_ms[k] < best) { best = e->tune_ms[k]; best_k = k; }
  if ((r = set_shape(e, best_k))) return r;
  EnsScalars s;
  if ((r = read_es(e, &s))) return r;
  if (s.bad) return efail(DG2_E_NONFINITE, "a member's state or step became non-finite");
  if (tile_w) *tile_w = kShapes[best_k].w;
  if (tile_h) *tile_h = kShapes[best_k].h;
  return release_members(e);
}

int dg2_ens_tune_times(const dg2_ens* e, double* ms, int cap) {
  if (!e) return efail(DG2_E_ARG, "null ensemble");
  if (!ms || cap < 1) return efail(DG2_E_ARG, "ms must hold at least one entry");
  for (int k = 0; k < kNumShapes && k < cap; ++k) ms[k] = e->tune_ms[k];
  return kNumShapes;
}

int64_t dg2_ens_launch_count(const dg2_ens* e) { return e ? e->launches : -1; }

int dg2_ens_destroy(dg2_ens* e) {
  if (!e) return efail(DG2_E_ARG, "null ensemble");
  drop_graphs(e);
  delete e;
  return DG2_OK;
}

}  // extern "C"
