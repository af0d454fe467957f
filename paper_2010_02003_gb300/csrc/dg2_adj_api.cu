// dg2_adj_api.cu -- C ABI of the discrete adjoint (dg2_adj_* in include/dg2.h):
// dispatches each call to the FP64 (dg2::adj, dg2_adj.cu) or the FP32
// (dg2::adj32, dg2_adj32.cu) build of the same adjoint by dg2_params.precision.
#include <cstddef>
#include <cstdint>
#include <string>

#include "../../include/dg2.h"

namespace dg2 {
void set_error_text(const std::string& s);  // dg2_api.cu

#define DG2_ADJ_DECLARE(NS)                                                                    \
  namespace NS {                                                                               \
  struct Ctx;                                                                                  \
  size_t workspace_bytes(int nx, int ny, int nsnap, int max_gauges, int max_steps);            \
  int create(Ctx** out, int nx, int ny, double dx, double dy, const dg2_params* prm, int nsnap, \
             int max_gauges, int max_steps, void* dev_workspace, size_t ws_bytes,              \
             void* cuda_stream);                                                               \
  int set_problem(Ctx* a, const double* z3, const double* state9, double t0,                   \
                  const double* manning, int inflow_edge, double s0, double len,               \
                  const double* t_knots, const double* q_knots, int nknots,                    \
                  const double* gauge_xy, int ngauge);                                         \
  int set_params(Ctx* a, const double* manning, const double* q_knots);                        \
  int set_schedule(Ctx* a, const double* dts, int nsteps, const int* sample_steps,             \
                   int nsamples, const double* obs);                                           \
  int forward(Ctx* a, double* loss, double* gauge_h);                                          \
  int gradient(Ctx* a, double* loss, double* grad_manning, double* grad_q);                    \
  int counts(const Ctx* a, int64_t* forward_steps, int64_t* reverse_steps);                    \
  int destroy(Ctx* a);                                                                         \
  }
DG2_ADJ_DECLARE(adj)
DG2_ADJ_DECLARE(adj32)
#undef DG2_ADJ_DECLARE
}  // namespace dg2

// The handle: one adjoint problem of either precision.
struct dg2_adj {
  int fp32;
  dg2::adj::Ctx* f64;
  dg2::adj32::Ctx* f32;
};

namespace {
int null_handle() {
  dg2::set_error_text("null adjoint context");
  return DG2_E_ARG;
}
}  // namespace

#define DG2_ADJ_CALL(a, fn, ...) \
  ((a)->fp32 ? dg2::adj32::fn((a)->f32, __VA_ARGS__) : dg2::adj::fn((a)->f64, __VA_ARGS__))

extern "C" {

size_t dg2_adj_workspace_bytes(int nx, int ny, int nsnap, int max_gauges, int max_steps) {
  // the FP64 layout, the larger of the two, serves both precisions
  return dg2::adj::workspace_bytes(nx, ny, nsnap, max_gauges, max_steps);
}

int dg2_adj_create(dg2_adj** out, int nx, int ny, double dx, double dy, const dg2_params* prm,
                   int nsnap, int max_gauges, int max_steps, void* dev_workspace, size_t ws_bytes,
                   void* cuda_stream) {
  if (!out) {
    dg2::set_error_text("out is null");
    return DG2_E_ARG;
  }
  *out = nullptr;
  if (!prm) {
    dg2::set_error_text("params is null");
    return DG2_E_ARG;
  }
  if (prm->precision != DG2_FP64 && prm->precision != DG2_FP32) {
    dg2::set_error_text("precision must be DG2_FP64 or DG2_FP32");
    return DG2_E_ARG;
  }
  dg2_adj h{prm->precision == DG2_FP32 ? 1 : 0, nullptr, nullptr};
  const int r = h.fp32 ? dg2::adj32::create(&h.f32, nx, ny, dx, dy, prm, nsnap, max_gauges,
                                            max_steps, dev_workspace, ws_bytes, cuda_stream)
                       : dg2::adj::create(&h.f64, nx, ny, dx, dy, prm, nsnap, max_gauges,
                                          max_steps, dev_workspace, ws_bytes, cuda_stream);
  if (r) return r;
  *out = new dg2_adj(h);
  return DG2_OK;
}

int dg2_adj_set_problem(dg2_adj* a, const double* z3, const double* state9, double t0,
                        const double* manning, int inflow_edge, double s0, double len,
                        const double* t_knots, const double* q_knots, int nknots,
                        const double* gauge_xy, int ngauge) {
  if (!a) return null_handle();
  return DG2_ADJ_CALL(a, set_problem, z3, state9, t0, manning, inflow_edge, s0, len, t_knots,
                      q_knots, nknots, gauge_xy, ngauge);
}

int dg2_adj_set_params(dg2_adj* a, const double* manning, const double* q_knots) {
  if (!a) return null_handle();
  return DG2_ADJ_CALL(a, set_params, manning, q_knots);
}

int dg2_adj_set_schedule(dg2_adj* a, const double* dts, int nsteps, const int* sample_steps,
                         int nsamples, const double* obs) {
  if (!a) return null_handle();
  return DG2_ADJ_CALL(a, set_schedule, dts, nsteps, sample_steps, nsamples, obs);
}

int dg2_adj_forward(dg2_adj* a, double* loss, double* gauge_h) {
  if (!a) return null_handle();
  return DG2_ADJ_CALL(a, forward, loss, gauge_h);
}

int dg2_adj_gradient(dg2_adj* a, double* loss, double* grad_manning, double* grad_q) {
  if (!a) return null_handle();
  return DG2_ADJ_CALL(a, gradient, loss, grad_manning, grad_q);
}

int dg2_adj_counts(const dg2_adj* a, int64_t* forward_steps, int64_t* reverse_steps) {
  if (!a) return null_handle();
  return a->fp32 ? dg2::adj32::counts(a->f32, forward_steps, reverse_steps)
                 : dg2::adj::counts(a->f64, forward_steps, reverse_steps);
}

int dg2_adj_destroy(dg2_adj* a) {
  if (!a) return null_handle();
  const int r = a->fp32 ? dg2::adj32::destroy(a->f32) : dg2::adj::destroy(a->f64);
  delete a;
  return r;
}

}  // extern "C"
