"""FP64 CPU oracle of the slope-decoupled DG2 scheme (Sec. 2.1, Eqs. 1-7, 11).

TEST INFRASTRUCTURE ONLY: the plain, slow statement of the method that the
CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference legs may import this package; the
product library never does, and this package imports nothing from it.

The arithmetic lives in ``dg2_oracle.c`` (plain C, built with
``-ffp-contract=off``); this module only builds it with gcc and marshals numpy
arrays through ctypes.

Parity status per function (pins live in ``tests/test_oracle_*.py``):
  - spatial operator, HLL flux, RK2 step, mass: pinned (lake at rest, wall
    balance, closed-wall mass, Ritter/Stoker closed forms, order of accuracy,
    transposition / mirror symmetry).
  - face revision of partially wet cells (``wetdry="positive"``, the default;
    ``"paper"`` is Sec. 2.1.2 as printed): pinned by the lake at rest in a basin
    whose bed rises 2 m across a cell, by bit-identity with the printed revision
    on fully wet flow, and by near-positivity and wave speeds on the floodplain's
    dry start (tests/test_oracle_wetdry.py).
  - friction: pinned by the exact solution of the friction ODE at the centre
    and at every Gauss point.
  - limiter: pinned by brute-force detector / minmod cases.
  - inflow ghost, rain: pinned by Manning's normal flow down a plane slope fed
    by the inflow boundary (normal depth; the step's mean face discharge equals
    the inflow) and by rain on a flat closed basin (depth rising at exactly the
    rain rate) (tests/test_oracle_sources.py).
  - point source: pinned by a closed single cell filling at exactly Q / (dx dy)
    and by a symmetric first step about the source cell of a closed basin.
  - taped derivatives (``tape.cpp``, :func:`taped_gradient`): the same C
    source compiled with a recording scalar type; pinned against central
    finite differences of the oracle itself.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dg2_oracle.c")
_LIB = os.path.join(_HERE, "libdg2_oracle.so")
_OMP_LIB = os.path.join(_HERE, "libdg2_oracle_omp.so")
_TAPE_SRC = os.path.join(_HERE, "tape.cpp")
_TAPE_LIB = os.path.join(_HERE, "liboracle_tape.so")

WALL, OPEN = 0, 1
WEST, EAST, SOUTH, NORTH = 0, 1, 2, 3

_lib = None
_omp_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction) into oracle/libdg2_oracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def build_omp(force: bool = False) -> str:
    """The same source with its rows-parallel loops enabled (gcc -fopenmp), for timing the
    oracle on every host core: each cell writes only its own outputs and the edge-flux
    sum is taken afterwards in cell order, so results equal the serial build's bit for
    bit (tests/test_oracle_threads.py)."""
    if force or not os.path.exists(_OMP_LIB) or os.path.getmtime(_OMP_LIB) < os.path.getmtime(_SRC):
        tmp = _OMP_LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
                               "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OMP_LIB)
    return _OMP_LIB


def build_tape(force: bool = False) -> str:
    """Compile the taped oracle (tape.cpp including dg2_oracle.c) with g++."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_TAPE_SRC))
    if force or not os.path.exists(_TAPE_LIB) or os.path.getmtime(_TAPE_LIB) < newest:
        tmp = _TAPE_LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _TAPE_SRC])
        os.replace(tmp, _TAPE_LIB)
    return _TAPE_LIB


_tape = None


def taped_gradient(case, manning, q_knots, dts, sample_steps, obs, limiter=False,
                   wetdry="positive"):
    """Misfit J = sum over samples and gauges of (h_gauge - obs)^2 of the oracle run
    of len(dts) steps from ``case`` (DEM, water, edges, its one inflow with the knot
    discharges ``q_knots``, Manning field ``manning`` (ny, nx)), sampled after the
    step counts ``sample_steps`` at ``case.gauges``; returns (J, dJ/dn (ny, nx),
    dJ/dq (nk,)) from the oracle's own taped derivatives."""
    global _tape
    if _tape is None:
        _tape = ctypes.CDLL(build_tape())
        f = _tape.orc_tape_gradient
        f.restype = ctypes.c_double
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))  # noqa: E731
    nx, ny = case.nx, case.ny
    bc = (ctypes.c_int * 4)(*[int(b) for b in case.bc])
    z = np.ascontiguousarray(case.z_corner, dtype=np.float64)
    eta = None if case.eta_corner is None else np.ascontiguousarray(case.eta_corner, dtype=np.float64)
    man = np.ascontiguousarray(manning, dtype=np.float64).reshape(ny, nx)
    if case.inflows:
        fl = case.inflows[0]
        edge, s0, ln = int(fl.edge), float(fl.s0), float(fl.length)
        tk = np.ascontiguousarray(fl.t_knots, dtype=np.float64)
        qk = np.ascontiguousarray(q_knots, dtype=np.float64)
    else:
        edge, s0, ln = -1, 0.0, 0.0
        tk = np.zeros(1)
        qk = np.zeros(1)
    d = np.ascontiguousarray(dts, dtype=np.float64)
    ss = np.ascontiguousarray(sample_steps, dtype=np.int32)
    g = np.ascontiguousarray(np.asarray(case.gauges, dtype=np.float64).reshape(-1, 2))
    ob = np.ascontiguousarray(obs, dtype=np.float64).reshape(len(ss), g.shape[0])
    gn = np.zeros((ny, nx))
    gq = np.zeros(len(qk))
    J = _tape.orc_tape_gradient(
        ctypes.c_int(nx), ctypes.c_int(ny), ctypes.c_double(case.dx), ctypes.c_double(case.dy),
        ctypes.c_double(9.80665), ctypes.c_double(case.cfl), ctypes.c_double(1e-5),
        ctypes.c_double(10.0), ctypes.c_double(case.dt_max), ctypes.c_int(int(bool(limiter))),
        ctypes.c_int(1 if wetdry == "positive" else 0), bc,
        dp(z), None if eta is None else dp(eta), dp(man), ctypes.c_int(edge), ctypes.c_double(s0),
        ctypes.c_double(ln), dp(tk), dp(qk), ctypes.c_int(len(qk) if edge >= 0 else 0),
        ctypes.c_int(len(d)), dp(d), ctypes.c_int(len(ss)),
        ss.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), ctypes.c_int(g.shape[0]), dp(g), dp(ob),
        dp(gn), dp(gq))
    return J, gn, gq


def _load(omp: bool = False):
    global _lib, _omp_lib
    if omp and _omp_lib is not None:
        return _omp_lib
    if not omp and _lib is not None:
        return _lib
    lib = ctypes.CDLL(build_omp() if omp else build())
    P = ctypes.c_void_p
    D = ctypes.c_double
    I = ctypes.c_int
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    sig = {
        "orc_create": (P, [I, I, D, D, D, D, D, D, D, I, ip]),
        "orc_destroy": (None, [P]),
        "orc_set_dem": (None, [P, dp, dp, D, dp]),
        "orc_add_inflow": (I, [P, I, D, D, dp, dp, I]),
        "orc_set_sources": (None, [P, D, D, D, D, D, D]),
        "orc_cfl_dt": (D, [P]),
        "orc_step": (None, [P, D]),
        "orc_get_state": (None, [P, dp, dp]),
        "orc_set_state": (None, [P, dp, D]),
        "orc_get_topo": (None, [P, dp]),
        "orc_time": (D, [P]),
        "orc_ledger": (D, [P]),
        "orc_mass": (D, [P]),
        "orc_operator": (D, [P, dp, D, dp]),
        "orc_friction": (None, [P, dp, D]),
        "orc_limit": (None, [P, dp, dp]),
        "orc_hll": (None, [P, I, dp, dp, dp]),
        "orc_minmod": (D, [D, D, D]),
        "orc_set_flux": (None, [P, I]),
        "orc_set_scheme": (None, [P, I]),
        "orc_set_wetdry": (None, [P, I]),
        "orc_gauge_h": (D, [P, D, D]),
        "orc_run_to": (ctypes.c_long, [P, D, D, I, dp, dp, dp, I, ip]),
        "orc_set_threads": (I, [I]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if omp:
        _omp_lib = lib
    else:
        _lib = lib
    return lib


def set_threads(n: int) -> int:
    """Thread count of the OpenMP build (the serial build always uses one); returns the
    count in use."""
    return _load(omp=True).orc_set_threads(int(n))


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def minmod(a: float, b: float, c: float) -> float:
    return _load().orc_minmod(a, b, c)


class Oracle:
    """One DG2 problem on an nx x ny grid (x index fastest), FP64 on the CPU.

    State arrays are (9, ny, nx): planes h0, h1x, h1y, qx0, qx1x, qx1y, qy0,
    qy1x, qy1y (Eq. 2).  Corner arrays are (ny+1, nx+1).
    """

    def __init__(self, nx, ny, dx, dy, *, g=9.80665, cfl=0.33, tol_dry=1e-5, ds_thresh=10.0,
                 dt_max=1.0, limiter=False, bc=(WALL, WALL, WALL, WALL), flux="hll",
                 scheme="dg2", wetdry="positive", threads=False):
        # threads=True: the OpenMP build (same results, rows in parallel; set_threads)
        self.lib = _load(omp=bool(threads))
        self.nx, self.ny, self.dx, self.dy = int(nx), int(ny), float(dx), float(dy)
        self.g, self.cfl, self.tol_dry = g, cfl, tol_dry
        bca = (ctypes.c_int * 4)(*[int(b) for b in bc])
        self.h = self.lib.orc_create(self.nx, self.ny, self.dx, self.dy, g, cfl, tol_dry, ds_thresh,
                                     dt_max, int(bool(limiter)), bca)
        if not self.h:
            raise ValueError("bad grid size")
        if flux not in ("hll", "roe"):
            raise ValueError("flux must be 'hll' or 'roe'")
        self.lib.orc_set_flux(self.h, 1 if flux == "roe" else 0)
        if scheme not in ("dg2", "fv2", "fv1"):
            raise ValueError("scheme must be 'dg2', 'fv2' or 'fv1'")
        self.lib.orc_set_scheme(self.h, ("dg2", "fv2", "fv1").index(scheme))
        if wetdry not in ("paper", "positive"):
            raise ValueError("wetdry must be 'paper' or 'positive'")
        self.lib.orc_set_wetdry(self.h, 1 if wetdry == "positive" else 0)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.orc_destroy(h)
            self.h = None

    # -- set-up ---------------------------------------------------------
    def set_dem(self, z_corner, manning=None, n_uniform=0.0, eta_corner=None):
        z = _f64(z_corner)
        assert z.shape == (self.ny + 1, self.nx + 1)
        m = None if manning is None else _f64(manning)
        e = None if eta_corner is None else _f64(eta_corner)
        self.lib.orc_set_dem(self.h, _dp(z), _dp(m), float(n_uniform), _dp(e))

    def add_inflow(self, edge, s0, length, t_knots, q_knots):
        tk, qk = _f64(t_knots), _f64(q_knots)
        if self.lib.orc_add_inflow(self.h, int(edge), float(s0), float(length), _dp(tk), _dp(qk),
                                   len(tk)) != 0:
            raise ValueError("inflow rejected")

    def set_sources(self, rain=0.0, rain_t0=0.0, rain_t1=0.0, px=0.0, py=0.0, qp=0.0):
        self.lib.orc_set_sources(self.h, rain, rain_t0, rain_t1, px, py, qp)

    # -- stepping -------------------------------------------------------
    def cfl_dt(self) -> float:
        return self.lib.orc_cfl_dt(self.h)

    def step(self, dt=None) -> float:
        if dt is None or dt <= 0:
            dt = self.cfl_dt()
        self.lib.orc_step(self.h, float(dt))
        return dt

    def run_to(self, t_end, sample_every=0.0, gauges_xy=None, cap=100000):
        g = np.zeros((0, 2)) if gauges_xy is None else _f64(gauges_xy).reshape(-1, 2)
        ng = g.shape[0]
        t_out = np.zeros(cap)
        h_out = np.zeros((cap, max(ng, 1)))
        ns = ctypes.c_int(0)
        steps = self.lib.orc_run_to(self.h, float(t_end), float(sample_every), ng, _dp(_f64(g)),
                                    _dp(t_out), _dp(h_out), cap, ctypes.byref(ns))
        n = min(ns.value, cap)
        return steps, t_out[:n].copy(), h_out[:n, :ng].copy()

    # -- state ----------------------------------------------------------
    @property
    def t(self) -> float:
        return self.lib.orc_time(self.h)

    def state(self):
        out = np.zeros((9, self.ny, self.nx))
        self.lib.orc_get_state(self.h, _dp(out), None)
        return out

    def set_state(self, planes, t=0.0):
        p = _f64(planes)
        assert p.shape == (9, self.ny, self.nx)
        self.lib.orc_set_state(self.h, _dp(p), float(t))

    def topo(self):
        out = np.zeros((3, self.ny, self.nx))
        self.lib.orc_get_topo(self.h, _dp(out))
        return out

    def mass(self) -> float:
        return self.lib.orc_mass(self.h)

    def ledger(self) -> float:
        return self.lib.orc_ledger(self.h)

    def gauge_h(self, x, y) -> float:
        return self.lib.orc_gauge_h(self.h, float(x), float(y))

    # -- pieces for pin tests -------------------------------------------
    def operator(self, planes, t=0.0):
        p = _f64(planes)
        out = np.zeros_like(p)
        b = self.lib.orc_operator(self.h, _dp(p), float(t), _dp(out))
        return out, b

    def friction(self, planes, dt):
        p = _f64(planes).copy()
        self.lib.orc_friction(self.h, _dp(p), float(dt))
        return p

    def limit(self, planes):
        p = _f64(planes)
        out = np.zeros_like(p)
        self.lib.orc_limit(self.h, _dp(p), _dp(out))
        return out

    def hll(self, direction, left, right):
        l, r = _f64(left), _f64(right)
        f = np.zeros(3)
        self.lib.orc_hll(self.h, int(direction), _dp(l), _dp(r), _dp(f))
        return f
