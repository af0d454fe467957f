// dg2_noalloc.cu -- a mass reduction that allocates nothing (dg2_mass_noalloc).
//
// Some callers cannot allocate device memory at all: code running inside a
// memory pool they do not own, a host application whose allocator is locked
// down, or a plugin handed only raw device pointers.  The regular dg2_mass
// keeps its block partials in the caller's workspace; this entry point keeps
// them in a fixed file-scope __device__ array instead, so the caller passes
// only the input plane and one output double.
//
// The scratch below exists once per GPU that loads this library and lives
// until the process exits.  Every call shares it: two calls that overlap on
// the GPU (different streams, no ordering between them) race on it.
#include <cuda_runtime.h>

#include <cstdio>
#include <string>

#include "../../include/dg2.h"

namespace dg2 {
void set_error_text(const std::string& s);  // dg2_api.cu
}

namespace {

constexpr int kRowsPerBlock = 8;   // one warp per grid row

// Per-row sums of the last call (row j of the grid in slot j) and the count of
// blocks that have finished; the count is cleared before every call and by the
// last block, the row slots are fully rewritten by every call.
__device__ __align__(256) double g_row_sum[DG2_NOALLOC_MAX_ROWS];
__device__ __align__(256) unsigned int g_blocks_done;

struct DevScratch {
  double* rows = nullptr;
  unsigned int* done = nullptr;
};

int noalloc_fail(int code, const std::string& msg) {
  dg2::set_error_text(msg);  // reported by dg2_last_error()
  return code;
}

// Looks up the device addresses of the scratch in the current context.  The
// lookup is repeated on every call rather than cached: a context that is torn
// down and recreated (cudaDeviceReset, a host that rebuilds its context) loads
// the module again, possibly at another address, and a cached pointer would
// then point at memory that is no longer this array.
int scratch_for_current_context(DevScratch* out) {
  void* rows = nullptr;
  void* done = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&rows, g_row_sum);
  if (e == cudaSuccess) e = cudaGetSymbolAddress(&done, g_blocks_done);
  if (e != cudaSuccess)
    return noalloc_fail(DG2_E_CUDA, std::string("cudaGetSymbolAddress failed: ") +
                                        cudaGetErrorString(e));
  out->rows = (double*)rows;
  out->done = (unsigned int*)done;
  return DG2_OK;
}

__global__ void __launch_bounds__(32 * kRowsPerBlock)
    mass_rows_kernel(const double* __restrict__ h0, int nx, int ny, long long pitch, double cell,
                     double* rows, unsigned int* done, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = blockIdx.x * kRowsPerBlock + warp;
  if (j < ny) {
    double s = 0.0;
    const double* r = h0 + (long long)j * pitch;
    for (int i = lane; i < nx; i += 32) s += r[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) rows[j] = s;
  }
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // the last block adds the row sums in a fixed order: deterministic
  __shared__ double part[32 * kRowsPerBlock];
  double s = 0.0;
  for (int k = threadIdx.x; k < ny; k += blockDim.x) s += __ldcg(&rows[k]);
  part[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *out = part[0] * cell;
    *done = 0u;
  }
}

}  // namespace

extern "C" int dg2_mass_noalloc(const double* h0_dev, int nx, int ny, int pitch, double dx,
                                double dy, double* mass_dev, void* cuda_stream) {
  if (!h0_dev || !mass_dev) return noalloc_fail(DG2_E_ARG, "h0_dev and mass_dev are required");
  if (nx < 1 || ny < 1 || pitch < nx)
    return noalloc_fail(DG2_E_ARG, "need nx >= 1, ny >= 1 and pitch >= nx");
  if (ny > DG2_NOALLOC_MAX_ROWS)
    return noalloc_fail(DG2_E_ARG,
                        "ny exceeds DG2_NOALLOC_MAX_ROWS (65536): the fixed scratch holds one "
                        "partial sum per grid row");
  if (!(dx > 0.0) || !(dy > 0.0)) return noalloc_fail(DG2_E_ARG, "dx, dy must be positive");
  DevScratch sc;
  int r = scratch_for_current_context(&sc);
  if (r) return r;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // the block counter must start at zero (an earlier failed launch may have left it set)
  cudaError_t e = cudaMemsetAsync(sc.done, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess)
    return noalloc_fail(DG2_E_CUDA, std::string("clearing the scratch counter failed: ") +
                                        cudaGetErrorString(e));
  const int blocks = (ny + kRowsPerBlock - 1) / kRowsPerBlock;
  mass_rows_kernel<<<blocks, 32 * kRowsPerBlock, 0, st>>>(h0_dev, nx, ny, pitch, dx * dy,
                                                          sc.rows, sc.done, mass_dev);
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return noalloc_fail(DG2_E_CUDA, std::string("launch failed: ") + cudaGetErrorString(e));
  return DG2_OK;
}
