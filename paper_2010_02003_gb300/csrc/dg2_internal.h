// dg2_internal.h -- what the library's translation units share about a
// single-problem context (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dg2.h"
#include "dg2_fs32.cuh"

namespace dg2 {
namespace ens {
// Step counters of a set of FP32 problems advanced by the shared FP32 kernels.
struct EnsScalars {
  int n_act;    // entries of the step's list of computed tiles
  int n_front;  // entries of the frontier list (stage-1 copies)
  int n_done;   // problems that reached t_end in the current run
  int bad;      // a problem raised its non-finite flag
};
// Launch parameters of the shared FP32 kernels: problem descriptors and work
// lists of (problem << kTileBits | tile) entries.
struct EnsDev {
  const f32::D32* desc;  // [nmem] in device memory
  int* list;
  int* front;
  EnsScalars* es;
  int nmem;
};
constexpr int kTileBits = 22;

// Tile of a single FP32 problem (cells, one thread each), fixed when the
// context is made: 16 x 8 on grids of up to kF32SmallCells cells, 32 x 8 on
// larger ones.  Measured on GB300 (ms per step, 32 x 8 -> 16 x 8): the
// 2000 x 1000 floodplain from t = 1 h, DG2-LL 0.122 -> 0.104 and DG2-NL
// 0.094 -> 0.079 (tiles of 128 cells leave fewer dry lanes around a narrow
// wet region), the same grid fully wet 0.387 -> 0.377, but the 8192 x 8192
// urban grid under rain 11.66 -> 12.95.
constexpr long long kF32SmallCells = 1ll << 23;
inline bool f32_small_tiles(long long cells) { return cells <= kF32SmallCells; }
// The FP32 kernels of one step on tiles of tw x th cells (16 x 8 or 32 x 8; a
// single problem is a set of one): one RK stage (stage 1 with friction fused),
// and the end of step (finalize + lists; with lists_only just the lists).
// `grid` = persistent blocks; `lgrid` = tile blocks of the lists kernel (z =
// problems).  occupancy32 also raises the stage kernels' dynamic shared memory
// limit for the shape, which must precede their first launch.
void launch_stage32(const EnsDev& E, int tw, bool ll, int stage, int grid, cudaStream_t st);
void launch_end_of_step(const EnsDev& E, int nmem, dim3 lgrid, int lists_only, cudaStream_t st);
void occupancy32(int tw, bool ll, int* st1, int* st2);
}  // namespace ens

// Reports through dg2_last_error().
void set_error_text(const std::string& s);

// Accessors of a context made by dg2_init_grid.
bool ctx_fp32(const dg2_ctx* c);
int ctx_variant(const dg2_ctx* c);
bool ctx_ready(const dg2_ctx* c);                 // a DEM or state has been set
cudaStream_t ctx_stream(const dg2_ctx* c);
const f32::D32& ctx_d32(const dg2_ctx* c);        // FP32 launch parameters
// Tiles of tw x th cells that must be computed whatever their state (inflow
// segments, the point source), row-major over the ntx x nty tile grid.
void ctx_forced_mask(const dg2_ctx* c, int tw, int th, std::vector<unsigned char>& m);
bool ctx_rains(const dg2_ctx* c);
// Marks every tile of the context's own tiling non-quiescent and rebuilds its
// lists (after another launcher changed the state behind its back).
int ctx_reset_tiles(dg2_ctx* c);
void ctx_count_launches(dg2_ctx* c, int64_t n);
}  // namespace dg2
