"""Python binding of the C ABI in include/dg2.h (argument marshalling only).

Every function named ``dg2_*`` here calls the library function of the same
name; every step of the solver runs in the library's CUDA kernels.  PyTorch is
used only to own the device workspace and to supply the CUDA stream.  There is
no CPU fallback: if ``libdg2.so`` has not been built, or no CUDA device is
visible, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdg2.so")

DG2_OK, DG2_E_ARG, DG2_E_STATE, DG2_E_CUDA, DG2_E_NONFINITE, DG2_E_NOMEM = 0, -1, -2, -3, -4, -5
DG2_E_OVERFLOW = -7
DG2_NL, DG2_LL = 0, 1
DG2_FP64, DG2_FP32 = 0, 1
DG2_WALL, DG2_OPEN = 0, 1
DG2_HLL, DG2_ROE = 0, 1
DG2_SCHEME_DG2, DG2_SCHEME_FV2, DG2_SCHEME_FV1 = 0, 1, 2
DG2_WD_POSITIVE, DG2_WD_PRINTED = 0, 1
DG2_WEST, DG2_EAST, DG2_SOUTH, DG2_NORTH = 0, 1, 2, 3

# Every symbol declared in include/dg2.h.
EXPORTS = (
    "dg2_default_params", "dg2_last_error", "dg2_workspace_bytes", "dg2_init_grid", "dg2_set_dem",
    "dg2_set_bc_inflow", "dg2_set_sources", "dg2_step", "dg2_run_to", "dg2_set_gauges",
    "dg2_read_gauges", "dg2_mass", "dg2_get_state", "dg2_set_state", "dg2_get_topo",
    "dg2_get_time", "dg2_enable_kernel_timing", "dg2_kernel_times", "dg2_launch_count",
    "dg2_tile_stats", "dg2_tile_shape", "dg2_get_steps", "dg2_mass_noalloc", "dg2_fp64_fma_peak",
    "dg2_destroy",
    "dg2_ens_workspace_bytes", "dg2_ens_create", "dg2_ens_run_to", "dg2_ens_autotune",
    "dg2_ens_set_tile_shape", "dg2_ens_tile_shape", "dg2_ens_tune_times",
    "dg2_ens_launch_count", "dg2_ens_destroy",
    "dg2_adj_workspace_bytes", "dg2_adj_create", "dg2_adj_set_problem", "dg2_adj_set_params",
    "dg2_adj_set_schedule", "dg2_adj_forward", "dg2_adj_gradient", "dg2_adj_counts",
    "dg2_adj_destroy",
)
DG2_NOALLOC_MAX_ROWS = 65536


class Dg2Params(ctypes.Structure):
    _fields_ = [("g", ctypes.c_double), ("cfl", ctypes.c_double), ("tol_dry", ctypes.c_double),
                ("ds_thresh", ctypes.c_double), ("dt_max", ctypes.c_double),
                ("variant", ctypes.c_int), ("precision", ctypes.c_int), ("bc", ctypes.c_int * 4),
                ("max_gauges", ctypes.c_int), ("max_samples", ctypes.c_int),
                ("skip_dry_tiles", ctypes.c_int), ("flux", ctypes.c_int),
                ("scheme", ctypes.c_int), ("wetdry", ctypes.c_int)]


class Dg2Error(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"dg2 error {code}: {msg}")
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Loads libdg2.so and declares its signatures.  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2010_02003_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P, D, I = ctypes.c_void_p, ctypes.c_double, ctypes.c_int
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    i64p = ctypes.POINTER(ctypes.c_int64)
    pp = ctypes.POINTER(Dg2Params)
    sig = {
        "dg2_default_params": (None, [pp]),
        "dg2_last_error": (ctypes.c_char_p, []),
        "dg2_workspace_bytes": (ctypes.c_size_t, [I, I, pp]),
        "dg2_init_grid": (I, [ctypes.POINTER(P), I, I, D, D, pp, P, ctypes.c_size_t, P]),
        "dg2_set_dem": (I, [P, dp, dp, D, dp]),
        "dg2_set_bc_inflow": (I, [P, I, D, D, dp, dp, I]),
        "dg2_set_sources": (I, [P, D, D, D, D, D, D]),
        "dg2_step": (I, [P, D, dp]),
        "dg2_run_to": (I, [P, D, i64p]),
        "dg2_set_gauges": (I, [P, dp, I, D]),
        "dg2_read_gauges": (I, [P, dp, dp, I, ip]),
        "dg2_mass": (I, [P, dp, dp]),
        "dg2_get_state": (I, [P, dp, dp]),
        "dg2_set_state": (I, [P, dp, D]),
        "dg2_get_topo": (I, [P, dp]),
        "dg2_get_time": (I, [P, dp, dp]),
        "dg2_enable_kernel_timing": (I, [P, I]),
        "dg2_kernel_times": (I, [P, dp, i64p]),
        "dg2_launch_count": (ctypes.c_int64, [P]),
        "dg2_get_steps": (I, [P, i64p]),
        "dg2_tile_shape": (I, [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
        "dg2_tile_stats": (I, [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                               ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64)]),
        "dg2_mass_noalloc": (I, [P, I, I, I, D, D, P, P]),
        "dg2_fp64_fma_peak": (I, [I, I, P, dp, dp]),
        "dg2_destroy": (I, [P]),
        "dg2_ens_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(P), I]),
        "dg2_ens_create": (I, [ctypes.POINTER(P), ctypes.POINTER(P), I, P, ctypes.c_size_t, P]),
        "dg2_ens_run_to": (I, [P, D, i64p]),
        "dg2_ens_autotune": (I, [P, D, I, ip, ip]),
        "dg2_ens_set_tile_shape": (I, [P, I, I]),
        "dg2_ens_tile_shape": (I, [P, ip, ip]),
        "dg2_ens_tune_times": (I, [P, dp, I]),
        "dg2_ens_launch_count": (ctypes.c_int64, [P]),
        "dg2_ens_destroy": (I, [P]),
        "dg2_adj_workspace_bytes": (ctypes.c_size_t, [I, I, I, I, I]),
        "dg2_adj_create": (I, [ctypes.POINTER(P), I, I, D, D, pp, I, I, I, P, ctypes.c_size_t, P]),
        "dg2_adj_set_problem": (I, [P, dp, dp, D, dp, I, D, D, dp, dp, I, dp, I]),
        "dg2_adj_set_params": (I, [P, dp, dp]),
        "dg2_adj_set_schedule": (I, [P, dp, I, ip, I, dp]),
        "dg2_adj_forward": (I, [P, dp, dp]),
        "dg2_adj_gradient": (I, [P, dp, dp, dp]),
        "dg2_adj_counts": (I, [P, i64p, i64p]),
        "dg2_adj_destroy": (I, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(code):
    if code < DG2_OK:
        raise Dg2Error(code, load().dg2_last_error().decode())
    return code


def _dp(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


# ---- same-named wrappers of the C entry points -------------------------------

def dg2_default_params() -> Dg2Params:
    p = Dg2Params()
    load().dg2_default_params(ctypes.byref(p))
    return p


def dg2_workspace_bytes(nx: int, ny: int, params: Dg2Params) -> int:
    return int(load().dg2_workspace_bytes(nx, ny, ctypes.byref(params)))


def dg2_init_grid(nx, ny, dx, dy, params, dev_ptr: int, ws_bytes: int, stream_ptr: int):
    h = ctypes.c_void_p()
    _check(load().dg2_init_grid(ctypes.byref(h), nx, ny, dx, dy, ctypes.byref(params),
                                ctypes.c_void_p(dev_ptr), ws_bytes, ctypes.c_void_p(stream_ptr)))
    return h


def dg2_set_dem(ctx, z_corner, manning=None, n_uniform=0.0, eta_corner=None):
    z, m, e = _f64(z_corner), _f64(manning), _f64(eta_corner)
    _check(load().dg2_set_dem(ctx, _dp(z), _dp(m), float(n_uniform), _dp(e)))


def dg2_set_bc_inflow(ctx, edge, s0, length, t_knots, q_knots):
    tk, qk = _f64(t_knots), _f64(q_knots)
    _check(load().dg2_set_bc_inflow(ctx, int(edge), float(s0), float(length), _dp(tk), _dp(qk),
                                    len(tk)))


def dg2_set_sources(ctx, rain=0.0, t0=0.0, t1=0.0, px=0.0, py=0.0, qp=0.0):
    _check(load().dg2_set_sources(ctx, rain, t0, t1, px, py, qp))


def dg2_step(ctx, dt: float = -1.0, want_dt: bool = False):
    out = ctypes.c_double(0.0)
    _check(load().dg2_step(ctx, float(dt), ctypes.byref(out) if want_dt else None))
    return out.value if want_dt else None


def dg2_run_to(ctx, t_end: float) -> int:
    n = ctypes.c_int64(0)
    _check(load().dg2_run_to(ctx, float(t_end), ctypes.byref(n)))
    return n.value


def dg2_set_gauges(ctx, xy, every):
    a = _f64(np.asarray(xy, dtype=np.float64).reshape(-1, 2))
    _check(load().dg2_set_gauges(ctx, _dp(a), a.shape[0], float(every)))


def dg2_read_gauges(ctx, ngauge: int, cap: int = 100000):
    t = np.zeros(cap)
    h = np.zeros((cap, max(ngauge, 1)))
    n = ctypes.c_int(0)
    code = load().dg2_read_gauges(ctx, _dp(t), _dp(h), cap, ctypes.byref(n))
    if code not in (DG2_OK, DG2_E_OVERFLOW):
        _check(code)
    return t[:n.value].copy(), h[:n.value, :ngauge].copy(), code == DG2_E_OVERFLOW


def dg2_mass(ctx):
    m, l = ctypes.c_double(), ctypes.c_double()
    _check(load().dg2_mass(ctx, ctypes.byref(m), ctypes.byref(l)))
    return m.value, l.value


def dg2_get_state(ctx, nx, ny, out=None):
    out = np.zeros((9, ny, nx)) if out is None else out
    t = ctypes.c_double()
    _check(load().dg2_get_state(ctx, _dp(out), ctypes.byref(t)))
    return out, t.value


def dg2_set_state(ctx, planes, t=0.0):
    p = _f64(planes)
    _check(load().dg2_set_state(ctx, _dp(p), float(t)))


def dg2_get_topo(ctx, nx, ny):
    out = np.zeros((3, ny, nx))
    _check(load().dg2_get_topo(ctx, _dp(out)))
    return out


def dg2_get_time(ctx):
    t, dt = ctypes.c_double(), ctypes.c_double()
    _check(load().dg2_get_time(ctx, ctypes.byref(t), ctypes.byref(dt)))
    return t.value, dt.value


def dg2_enable_kernel_timing(ctx, enable: bool):
    _check(load().dg2_enable_kernel_timing(ctx, int(bool(enable))))


def dg2_kernel_times(ctx):
    ms = np.zeros(3)
    n = ctypes.c_int64(0)
    _check(load().dg2_kernel_times(ctx, _dp(ms), ctypes.byref(n)))
    return ms, n.value


def dg2_launch_count(ctx) -> int:
    return int(load().dg2_launch_count(ctx))


def dg2_get_steps(ctx) -> int:
    n = ctypes.c_int64(0)
    _check(load().dg2_get_steps(ctx, ctypes.byref(n)))
    return n.value


def dg2_tile_stats(ctx):
    """(ntiles, n_active, n_frontier, tiles_computed) of the dry-tile skipping."""
    nt, na, nf = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    tc = ctypes.c_int64()
    _check(load().dg2_tile_stats(ctx, ctypes.byref(nt), ctypes.byref(na), ctypes.byref(nf),
                                 ctypes.byref(tc)))
    return nt.value, na.value, nf.value, tc.value


def dg2_tile_shape(ctx):
    """(width, height) in cells of the tiles that dg2_tile_stats counts."""
    w, h = ctypes.c_int(), ctypes.c_int()
    _check(load().dg2_tile_shape(ctx, ctypes.byref(w), ctypes.byref(h)))
    return w.value, h.value


def dg2_mass_noalloc(h0_ptr: int, nx: int, ny: int, pitch: int, dx: float, dy: float,
                     mass_ptr: int, stream_ptr: int = 0):
    """Mass of a device depth plane into a device double, with no device allocation
    (the library's fixed scratch); see include/dg2.h."""
    _check(load().dg2_mass_noalloc(ctypes.c_void_p(h0_ptr), nx, ny, pitch, float(dx), float(dy),
                                   ctypes.c_void_p(mass_ptr), ctypes.c_void_p(stream_ptr)))


def dg2_fp64_fma_peak(blocks_per_sm: int = 4, iters: int = 4096, stream_ptr: int = 0):
    """Measured FP64 FMA throughput of the current GPU: (GFLOP/s, kernel ms)."""
    g, ms = ctypes.c_double(), ctypes.c_double()
    _check(load().dg2_fp64_fma_peak(int(blocks_per_sm), int(iters), stream_ptr, ctypes.byref(g),
                                    ctypes.byref(ms)))
    return g.value, ms.value


def dg2_destroy(ctx):
    _check(load().dg2_destroy(ctx))


def _ctx_array(ctxs):
    return (ctypes.c_void_p * len(ctxs))(*[c.value if isinstance(c, ctypes.c_void_p) else c
                                           for c in ctxs])


def dg2_ens_workspace_bytes(ctxs) -> int:
    return int(load().dg2_ens_workspace_bytes(_ctx_array(ctxs), len(ctxs)))


def dg2_ens_create(ctxs, dev_ptr: int, ws_bytes: int, stream_ptr: int):
    h = ctypes.c_void_p()
    _check(load().dg2_ens_create(ctypes.byref(h), _ctx_array(ctxs), len(ctxs),
                                 ctypes.c_void_p(dev_ptr), ws_bytes, ctypes.c_void_p(stream_ptr)))
    return h


def dg2_ens_run_to(ens, t_end: float) -> int:
    n = ctypes.c_int64(0)
    _check(load().dg2_ens_run_to(ens, float(t_end), ctypes.byref(n)))
    return n.value


def dg2_ens_autotune(ens, t_end: float, steps_per_trial: int = 16):
    w, h = ctypes.c_int(), ctypes.c_int()
    _check(load().dg2_ens_autotune(ens, float(t_end), int(steps_per_trial), ctypes.byref(w),
                                   ctypes.byref(h)))
    return w.value, h.value


def dg2_ens_set_tile_shape(ens, w: int, h: int):
    _check(load().dg2_ens_set_tile_shape(ens, int(w), int(h)))


def dg2_ens_tile_shape(ens):
    w, h = ctypes.c_int(), ctypes.c_int()
    _check(load().dg2_ens_tile_shape(ens, ctypes.byref(w), ctypes.byref(h)))
    return w.value, h.value


def dg2_ens_tune_times(ens):
    ms = np.zeros(16)
    n = _check(load().dg2_ens_tune_times(ens, _dp(ms), len(ms)))
    return ms[:n].copy()


def dg2_ens_launch_count(ens) -> int:
    return int(load().dg2_ens_launch_count(ens))


def dg2_ens_destroy(ens):
    _check(load().dg2_ens_destroy(ens))


def dg2_adj_workspace_bytes(nx, ny, nsnap, max_gauges, max_steps) -> int:
    return int(load().dg2_adj_workspace_bytes(nx, ny, nsnap, max_gauges, max_steps))


def dg2_adj_create(nx, ny, dx, dy, params, nsnap, max_gauges, max_steps, dev_ptr, ws_bytes,
                   stream_ptr):
    h = ctypes.c_void_p()
    _check(load().dg2_adj_create(ctypes.byref(h), nx, ny, float(dx), float(dy), ctypes.byref(params),
                                 nsnap, max_gauges, max_steps, ctypes.c_void_p(dev_ptr), ws_bytes,
                                 ctypes.c_void_p(stream_ptr)))
    return h


def dg2_adj_set_problem(adj, z3, state9, t0, manning, inflow_edge=-1, s0=0.0, length=0.0,
                        t_knots=None, q_knots=None, gauge_xy=None):
    z, u, m = _f64(z3), _f64(state9), _f64(manning)
    tk, qk = _f64(t_knots), _f64(q_knots)
    g = None if gauge_xy is None else _f64(np.asarray(gauge_xy, dtype=np.float64).reshape(-1, 2))
    _check(load().dg2_adj_set_problem(adj, _dp(z), _dp(u), float(t0), _dp(m), int(inflow_edge),
                                      float(s0), float(length), _dp(tk), _dp(qk),
                                      0 if tk is None else len(tk), _dp(g),
                                      0 if g is None else g.shape[0]))


def dg2_adj_set_params(adj, manning=None, q_knots=None):
    m, q = _f64(manning), _f64(q_knots)
    _check(load().dg2_adj_set_params(adj, _dp(m), _dp(q)))


def dg2_adj_set_schedule(adj, dts, sample_steps, obs):
    d = _f64(dts)
    ss = np.ascontiguousarray(sample_steps, dtype=np.int32)
    ob = _f64(obs)
    _check(load().dg2_adj_set_schedule(adj, _dp(d), len(d),
                                       ss.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), len(ss),
                                       _dp(ob)))


def dg2_adj_forward(adj, nsamples, ngauge):
    J = ctypes.c_double()
    h = np.zeros((nsamples, max(ngauge, 1)))
    _check(load().dg2_adj_forward(adj, ctypes.byref(J), _dp(h)))
    return J.value, h[:, :ngauge].copy()


def dg2_adj_gradient(adj, nx, ny, nknots):
    J = ctypes.c_double()
    gn = np.zeros((ny, nx))
    gq = np.zeros(max(nknots, 1))
    _check(load().dg2_adj_gradient(adj, ctypes.byref(J), _dp(gn), _dp(gq)))
    return J.value, gn, gq[:nknots].copy()


def dg2_adj_counts(adj):
    f, r = ctypes.c_int64(), ctypes.c_int64()
    _check(load().dg2_adj_counts(adj, ctypes.byref(f), ctypes.byref(r)))
    return f.value, r.value


def dg2_adj_destroy(adj):
    _check(load().dg2_adj_destroy(adj))


# ---- convenience object owning a torch workspace ----------------------------

class Solver:
    """One DG2 problem on the current CUDA device.  The device workspace is a torch
    uint8 tensor; kernels run on ``stream`` (default: a new torch stream)."""

    def __init__(self, nx, ny, dx, dy=None, *, variant=DG2_NL, precision=DG2_FP64, cfl=0.3,
                 tol_dry=1e-5, ds_thresh=10.0, dt_max=1.0, g=9.80665,
                 bc: Sequence[int] = (DG2_WALL,) * 4, max_gauges=64, max_samples=4096,
                 skip_dry_tiles=True, flux=DG2_HLL, scheme=DG2_SCHEME_DG2,
                 wetdry=DG2_WD_POSITIVE, stream=None, device=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the DG2 solver needs a CUDA device")
        load()
        self.nx, self.ny, self.dx = int(nx), int(ny), float(dx)
        self.dy = float(dx if dy is None else dy)
        p = dg2_default_params()
        p.g, p.cfl, p.tol_dry, p.ds_thresh, p.dt_max = g, cfl, tol_dry, ds_thresh, dt_max
        p.variant, p.precision = int(variant), int(precision)
        for k in range(4):
            p.bc[k] = int(bc[k])
        p.max_gauges, p.max_samples = int(max_gauges), int(max_samples)
        p.skip_dry_tiles = int(bool(skip_dry_tiles))
        p.flux = int(flux)
        p.scheme = int(scheme)
        p.wetdry = int(wetdry)
        self.params = p
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        nbytes = dg2_workspace_bytes(self.nx, self.ny, p)
        if nbytes == 0:
            raise Dg2Error(DG2_E_ARG, "invalid grid size")
        with torch.cuda.device(self.device):
            # a stream of its own by default: dg2_run_to captures CUDA graphs on it, which
            # the legacy default stream does not allow
            self.stream = torch.cuda.Stream(self.device) if stream is None else stream
            # the workspace comes from torch's allocator on the current stream
            self.stream.wait_stream(torch.cuda.current_stream(self.device))
            # over-allocate by the alignment so the base can be rounded up to 256 bytes
            self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
            base = self.workspace.data_ptr()
            self._base = (base + 255) // 256 * 256
            self.ctx = dg2_init_grid(self.nx, self.ny, self.dx, self.dy, p, self._base, nbytes,
                                     self.stream.cuda_stream)
        self.ngauge = 0

    def close(self):
        if getattr(self, "ctx", None):
            dg2_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # set-up
    def set_dem(self, z_corner, manning=None, n_uniform=0.0, eta_corner=None):
        dg2_set_dem(self.ctx, z_corner, manning, n_uniform, eta_corner)

    def add_inflow(self, edge, s0, length, t_knots, q_knots):
        dg2_set_bc_inflow(self.ctx, edge, s0, length, t_knots, q_knots)

    def set_sources(self, rain=0.0, t0=0.0, t1=0.0, px=0.0, py=0.0, qp=0.0):
        dg2_set_sources(self.ctx, rain, t0, t1, px, py, qp)

    def set_gauges(self, xy, every):
        xy = np.asarray(xy, dtype=np.float64).reshape(-1, 2)
        dg2_set_gauges(self.ctx, xy, every)
        self.ngauge = xy.shape[0]

    # stepping
    def step(self, dt: float = -1.0, want_dt: bool = False):
        return dg2_step(self.ctx, dt, want_dt)

    def run_to(self, t_end: float) -> int:
        return dg2_run_to(self.ctx, t_end)

    # outputs
    def state(self):
        return dg2_get_state(self.ctx, self.nx, self.ny)[0]

    def set_state(self, planes, t=0.0):
        dg2_set_state(self.ctx, planes, t)

    def topo(self):
        return dg2_get_topo(self.ctx, self.nx, self.ny)

    def time(self):
        return dg2_get_time(self.ctx)

    def mass(self):
        return dg2_mass(self.ctx)

    def read_gauges(self, cap=100000):
        return dg2_read_gauges(self.ctx, self.ngauge, cap)

    def launches(self) -> int:
        return dg2_launch_count(self.ctx)

    def tile_stats(self):
        return dg2_tile_stats(self.ctx)

    def tile_shape(self):
        return dg2_tile_shape(self.ctx)

    def steps(self) -> int:
        return dg2_get_steps(self.ctx)


def solver_from_case(case, variant=DG2_NL, precision=DG2_FP64, **kw) -> Solver:
    """Builds a Solver from an inputs.Case (DEM, water, roughness, inflows, sources, gauges)."""
    kw.setdefault("dt_max", case.dt_max)
    kw.setdefault("cfl", case.cfl)
    s = Solver(case.nx, case.ny, case.dx, case.dy, variant=variant, precision=precision,
               bc=case.bc, **kw)
    s.set_dem(case.z_corner, case.manning, case.n_uniform, case.eta_corner)
    for f in case.inflows:
        s.add_inflow(f.edge, f.s0, f.length, f.t_knots, f.q_knots)
    r, r0, r1 = case.rain
    px, py, qp = case.point
    if r != 0.0 or qp != 0.0:
        s.set_sources(r, r0, r1, px, py, qp)
    if case.gauges is not None and case.sample_every > 0:
        s.set_gauges(case.gauges, case.sample_every)
    return s


class Ensemble:
    """FP32 Solvers advanced together (one set of launches per step for all of them,
    each member with its own time step).  Read results through the member Solvers."""

    def __init__(self, members: Sequence[Solver], stream=None):
        import torch
        self.members = list(members)
        ctxs = [m.ctx for m in self.members]
        nbytes = dg2_ens_workspace_bytes(ctxs)
        if nbytes == 0:
            raise Dg2Error(DG2_E_ARG, "members must be FP32 solvers (1..512)")
        dev = self.members[0].device
        with torch.cuda.device(dev):
            self.stream = torch.cuda.Stream(dev) if stream is None else stream
            self.stream.wait_stream(torch.cuda.current_stream(dev))
            self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
            base = (self.workspace.data_ptr() + 255) // 256 * 256
            self.ens = dg2_ens_create(ctxs, base, nbytes, self.stream.cuda_stream)

    def run_to(self, t_end: float) -> int:
        return dg2_ens_run_to(self.ens, t_end)

    def autotune(self, t_end: float, steps_per_trial: int = 16):
        return dg2_ens_autotune(self.ens, t_end, steps_per_trial)

    def set_tile_shape(self, w: int, h: int):
        dg2_ens_set_tile_shape(self.ens, w, h)

    def tile_shape(self):
        return dg2_ens_tile_shape(self.ens)

    def tune_times(self):
        return dg2_ens_tune_times(self.ens)

    def launches(self) -> int:
        return dg2_ens_launch_count(self.ens)

    def close(self):
        if getattr(self, "ens", None):
            dg2_ens_destroy(self.ens)
            self.ens = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Adjoint:
    """Discrete adjoint of the DG2-NL step for one problem built from an inputs.Case
    (DEM, initial water, edges, its first inflow, gauges): the misfit of sampled gauge
    depths against observations and its gradients with respect to the Manning n of
    every cell and the inflow knot discharges, for the step with the default face
    revision or (wetdry=DG2_WD_PRINTED) Sec. 2.1.2 as printed, in FP64 or
    (precision=DG2_FP32) FP32 state and arithmetic."""

    def __init__(self, case, *, nsnap=64, max_steps=100000, wetdry=DG2_WD_POSITIVE,
                 precision=DG2_FP64, stream=None, device=None):
        import torch
        self.case = case
        self.nx, self.ny = case.nx, case.ny
        ref = solver_from_case(case, variant=DG2_NL, precision=DG2_FP64, wetdry=wetdry)
        z3, st = ref.topo(), ref.state()
        t0 = ref.time()[0]
        ref.close()
        p = dg2_default_params()
        p.cfl, p.dt_max = case.cfl, case.dt_max
        p.wetdry = int(wetdry)
        p.precision = int(precision)
        for k in range(4):
            p.bc[k] = int(case.bc[k])
        g = np.zeros((0, 2)) if case.gauges is None else np.asarray(case.gauges, dtype=np.float64)
        self.ngauge = g.shape[0]
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        nbytes = dg2_adj_workspace_bytes(self.nx, self.ny, nsnap, max(self.ngauge, 1), max_steps)
        if nbytes == 0:
            raise Dg2Error(DG2_E_ARG, "invalid adjoint sizes")
        with torch.cuda.device(dev):
            self.stream = torch.cuda.Stream(dev) if stream is None else stream
            self.stream.wait_stream(torch.cuda.current_stream(dev))
            self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
            base = (self.workspace.data_ptr() + 255) // 256 * 256
            self.adj = dg2_adj_create(self.nx, self.ny, case.dx, case.dy, p, nsnap,
                                      max(self.ngauge, 1), max_steps, base, nbytes,
                                      self.stream.cuda_stream)
        man = case.manning if case.manning is not None else np.full((self.ny, self.nx), case.n_uniform)
        if case.inflows:
            f = case.inflows[0]
            self.nknots = len(f.t_knots)
            dg2_adj_set_problem(self.adj, z3, st, t0, man, f.edge, f.s0, f.length, f.t_knots,
                                f.q_knots, g)
        else:
            self.nknots = 0
            dg2_adj_set_problem(self.adj, z3, st, t0, man, -1, gauge_xy=g)
        self.nsamples = 0

    def set_schedule(self, dts, sample_steps, obs):
        obs = np.asarray(obs, dtype=np.float64).reshape(len(sample_steps), self.ngauge)
        dg2_adj_set_schedule(self.adj, dts, sample_steps, obs)
        self.nsamples = len(sample_steps)

    def set_params(self, manning=None, q_knots=None):
        dg2_adj_set_params(self.adj, manning, q_knots)

    def forward(self):
        return dg2_adj_forward(self.adj, self.nsamples, self.ngauge)

    def gradient(self):
        return dg2_adj_gradient(self.adj, self.nx, self.ny, self.nknots)

    def counts(self):
        return dg2_adj_counts(self.adj)

    def close(self):
        if getattr(self, "adj", None):
            dg2_adj_destroy(self.adj)
            self.adj = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gauge_misfit(adjoint: Adjoint, manning, q_knots):
    """torch.autograd entry point: J(manning, q_knots) as a 0-d float64 tensor whose
    backward runs the discrete adjoint (dg2_adj_gradient)."""
    import torch

    class _GaugeMisfit(torch.autograd.Function):
        @staticmethod
        def forward(ctx, n_field, q):
            adjoint.set_params(n_field.detach().cpu().numpy(), q.detach().cpu().numpy())
            J, _ = adjoint.forward()
            ctx.save_for_backward(n_field, q)
            return torch.tensor(J, dtype=torch.float64, device=n_field.device)

        @staticmethod
        def backward(ctx, gout):
            n_field, q = ctx.saved_tensors
            adjoint.set_params(n_field.detach().cpu().numpy(), q.detach().cpu().numpy())
            _, gn, gq = adjoint.gradient()
            gn_t = torch.as_tensor(gn, dtype=torch.float64, device=n_field.device)
            gq_t = torch.as_tensor(gq, dtype=torch.float64, device=q.device)
            return gout * gn_t, gout * gq_t

    return _GaugeMisfit.apply(manning, q_knots)
