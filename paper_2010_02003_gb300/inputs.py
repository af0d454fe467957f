"""Seeded synthetic inputs for the DG2 flood solver.

This module is the only code shared by the CUDA path's tests / benchmark and
the CPU oracle.  It holds none of the scheme's arithmetic: it only draws
terrain, initial free surface, Manning fields, hydrographs and gauge points
on the (ny+1) x (nx+1) corner grid that the solver's ``set_dem`` consumes.

The paper's own test data (UK Environment Agency benchmark DEMs and
hydrographs, Sec. 3) are not available; the generators below stand in for
them with the shapes the paper describes: gently sloping or undulating
floodplains, incised channels, a breach / west-edge inflow hydrograph, and
a Gaussian hump for the closed-basin checks.

Every array is float64, row-major, y (north) index first.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

WALL, OPEN = 0, 1
WEST, EAST, SOUTH, NORTH = 0, 1, 2, 3


@dataclass
class Inflow:
    edge: int
    s0: float            # start of the segment along the edge (m)
    length: float        # segment length (m)
    t_knots: np.ndarray  # s
    q_knots: np.ndarray  # m^3/s


@dataclass
class Case:
    """A complete problem description (inputs only)."""
    name: str
    nx: int
    ny: int
    dx: float
    dy: float
    z_corner: np.ndarray                  # (ny+1, nx+1)
    eta_corner: Optional[np.ndarray]      # (ny+1, nx+1) or None (dry)
    manning: Optional[np.ndarray]         # (ny, nx) or None
    n_uniform: float = 0.0
    bc: Tuple[int, int, int, int] = (WALL, WALL, WALL, WALL)
    cfl: float = 0.33
    t_end: float = 10.0
    inflows: List[Inflow] = field(default_factory=list)
    gauges: Optional[np.ndarray] = None   # (ng, 2) x, y in metres
    sample_every: float = 0.0
    rain: Tuple[float, float, float] = (0.0, 0.0, 0.0)        # rate m/s, t0, t1
    point: Tuple[float, float, float] = (0.0, 0.0, 0.0)       # x, y, Q m^3/s
    dt_max: float = 1.0                   # step when nothing is wet, and upper cap


def corner_xy(nx, ny, dx, dy):
    x = np.arange(nx + 1, dtype=np.float64) * dx
    y = np.arange(ny + 1, dtype=np.float64) * dy
    return np.meshgrid(x, y)


# ----------------------------------------------------------------------------
# Closed basin: Gaussian hump, still water, optional circular dam break
# ----------------------------------------------------------------------------

def hump(nx=128, ny=128, dx=1.0, eta=0.5, dam_eta=None, dam_radius=20.0, n_uniform=0.03,
         t_end=10.0, amp=0.8, width2=200.0):
    """Gaussian hump z = amp*exp(-r^2/width2) about the domain centre, still water at `eta`,
    optionally raised to `dam_eta` inside `dam_radius` (a circular dam break).  Closed walls.

    With the defaults this is the 128 x 128, 1 m closed-basin problem: hump of 0.8 m,
    still water at 0.5 m (hump top dry), Manning 0.03, Courant 0.33, 10 s."""
    X, Y = corner_xy(nx, ny, dx, dx)
    xc, yc = 0.5 * nx * dx, 0.5 * ny * dx
    r2 = (X - xc) ** 2 + (Y - yc) ** 2
    z = amp * np.exp(-r2 / width2)
    e = np.full_like(z, eta)
    if dam_eta is not None:
        e[r2 <= dam_radius ** 2] = dam_eta
    return Case(name=f"hump{nx}x{ny}", nx=nx, ny=ny, dx=dx, dy=dx, z_corner=z, eta_corner=e,
                manning=None, n_uniform=n_uniform, t_end=t_end)


def wall_blocks(nx=48, ny=40, dx=1.0, eta=1.3, height=1.5):
    """Flat bed with raised rectangular blocks that stick out of still water."""
    X, Y = corner_xy(nx, ny, dx, dx)
    z = np.zeros_like(X)
    z[:, : 4] = height                                      # west bank
    z[:, nx - 5:] = height                                  # east bank
    z[(X >= 0.3 * nx * dx) & (X <= 0.45 * nx * dx) & (Y >= 0.3 * ny * dx) & (Y <= 0.6 * ny * dx)] = height
    z[: 3, :] = height                                      # south bank
    e = np.full_like(z, eta)
    return Case(name="blocks", nx=nx, ny=ny, dx=dx, dy=dx, z_corner=z, eta_corner=e, manning=None,
                n_uniform=0.0)


# ----------------------------------------------------------------------------
# Synthetic floodplain: fractal terrain + incised sinuous channel + inflow
# ----------------------------------------------------------------------------

def fbm(ny1, nx1, hurst, relief, seed):
    """Fractional-Brownian-motion surface on an ny1 x nx1 grid by spectral synthesis:
    amplitudes |k|^-(H+1), random phases, DC removed, min-max scaled to `relief`."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ky = np.fft.fftfreq(ny1)[:, None]
    kx = np.fft.rfftfreq(nx1)[None, :]
    k = np.sqrt(kx ** 2 + ky ** 2)
    k[0, 0] = 1.0
    amp = k ** (-(hurst + 1.0))
    amp[0, 0] = 0.0
    spec = amp * rng.standard_normal(amp.shape) * np.exp(2j * np.pi * rng.uniform(size=amp.shape))
    f = np.fft.irfft2(spec, s=(ny1, nx1))
    f = (f - f.min()) / max(f.max() - f.min(), 1e-300) * relief
    return f


def floodplain(nx=2000, ny=1000, dx=2.0, seed=2010, hurst=0.8, relief=3.0, channel_width=20.0,
               channel_depth=2.0, q_peak=20.0, t_peak=3600.0, t_end=18000.0, n_channel=0.035,
               n_plain=0.05, inflow_len=40.0, ngauge=8, sample_every=60.0, initial="dry",
               channel_fill=1.0):
    """Synthetic floodplain: fBm terrain (Hurst `hurst`, `relief` m) plus a sinuous incised
    channel; a triangular inflow hydrograph (0 -> q_peak at t_peak -> 0 at 2 t_peak) on a
    west-edge segment centred on the channel (the rest of the west edge is a wall, as for a
    breach in an embankment); the east, south and north edges are transmissive.

    initial="dry": no water; initial="channel": the channel holds `channel_fill` m of water
    above its bed (water surface following the bed, so it drains downhill)."""
    Lx, Ly = nx * dx, ny * dx
    X, Y = corner_xy(nx, ny, dx, dx)
    z = fbm(ny + 1, nx + 1, hurst, relief, seed)

    def yc(x):
        return 0.5 * Ly + 0.1 * Ly * np.sin(2.0 * np.pi * x / (Lx / 3.0))

    in_ch = np.abs(Y - yc(X)) <= 0.5 * channel_width
    z = z - channel_depth * in_ch
    xc = (np.arange(nx) + 0.5) * dx
    ycell = (np.arange(ny) + 0.5) * dx
    XC, YC = np.meshgrid(xc, ycell)
    man = np.where(np.abs(YC - yc(XC)) <= 0.5 * channel_width, n_channel, n_plain).astype(np.float64)
    eta = None
    if initial == "channel":
        eta = np.where(in_ch, z + channel_fill, z)
    tk, qk = [0.0, t_peak, 2.0 * t_peak], [0.0, q_peak, 0.0]
    if t_end > 2.0 * t_peak:
        tk.append(t_end)
        qk.append(0.0)
    inflow = Inflow(edge=WEST, s0=yc(0.0) - 0.5 * inflow_len, length=inflow_len,
                    t_knots=np.array(tk), q_knots=np.array(qk))
    gx = (np.arange(ngauge) + 0.5) * Lx / ngauge
    gauges = np.stack([gx, yc(gx)], axis=1)
    return Case(name=f"floodplain{nx}x{ny}", nx=nx, ny=ny, dx=dx, dy=dx, z_corner=z,
                eta_corner=eta, manning=man, bc=(WALL, OPEN, OPEN, OPEN), t_end=t_end,
                inflows=[inflow], gauges=gauges, sample_every=sample_every)


# ----------------------------------------------------------------------------
# One-dimensional Riemann problems (y-uniform) and smooth waves
# ----------------------------------------------------------------------------

def dam_break_1d(nx=200, ny=4, length=100.0, h_left=1.0, h_right=0.0, x0=None, t_end=3.0):
    """Flat frictionless channel, depth h_left for x < x0 and h_right beyond; walls."""
    dx = length / nx
    x0 = 0.5 * length if x0 is None else x0
    X, _ = corner_xy(nx, ny, dx, dx)
    z = np.zeros_like(X)
    e = np.where(X < x0, h_left, h_right).astype(np.float64)
    # a corner exactly on x0 takes the mean so the cell faces straddle cleanly
    e[np.isclose(X, x0)] = 0.5 * (h_left + h_right)
    return Case(name="dambreak1d", nx=nx, ny=ny, dx=dx, dy=dx, z_corner=z, eta_corner=e,
                manning=None, n_uniform=0.0, t_end=t_end)


def smooth_wave_1d(nx=100, ny=2, length=1.0, h0=1.0, amp=0.1, bed_amp=0.05, t_end=0.05):
    """Smooth water hump over a smooth bed in a walled channel, for convergence studies."""
    dx = length / nx
    X, _ = corner_xy(nx, ny, dx, dx)
    z = bed_amp * np.sin(2.0 * np.pi * X / length) ** 2
    e = h0 + amp * np.exp(-((X - 0.5 * length) / (0.1 * length)) ** 2)
    return Case(name="smooth1d", nx=nx, ny=ny, dx=dx, dy=dx, z_corner=z, eta_corner=e,
                manning=None, n_uniform=0.0, t_end=t_end)


def diamond_basin(n=40, dx=2.0, level=6.5, n_uniform=0.03):
    """Basin z = |x - x0| + |y - y0| (x0 = y0 = n m, bed rising 2 m across a 2 m cell),
    planar inside every cell, under a flat free surface at `level`: with an even
    height + 0.5 the surface crosses cells above their centres, so those cells are
    partially wet (0.5 m average, 1.5 m at the low faces, -0.5 m at the high faces)
    and every cell above them lies wholly above the surface.  Walls all round."""
    x = np.arange(n + 1) * dx
    X, Y = np.meshgrid(x, x)
    z = np.abs(X - n * dx / 2.0) + np.abs(Y - n * dx / 2.0)
    return Case("diamond_basin", n, n, dx, dx, z, np.full_like(z, level), None, n_uniform,
                (WALL, WALL, WALL, WALL), cfl=0.33, t_end=60.0)


def random_terrain(nx, ny, dx=1.0, seed=7, relief=1.0, eta=0.6, dam=True):
    """Small fBm terrain with a still lake (and optionally a raised circular dam) for
    parity runs on ragged sizes: wet/dry fronts everywhere."""
    X, Y = corner_xy(nx, ny, dx, dx)
    z = fbm(ny + 1, nx + 1, 0.8, relief, seed)
    e = np.full_like(z, eta)
    if dam:
        r2 = (X - 0.3 * nx * dx) ** 2 + (Y - 0.6 * ny * dx) ** 2
        e[r2 <= (0.2 * min(nx, ny) * dx) ** 2] = eta + 0.8
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    man = rng.uniform(0.02, 0.06, size=(ny, nx))
    return Case(name=f"terrain{nx}x{ny}", nx=nx, ny=ny, dx=dx, dy=dx, z_corner=z, eta_corner=e,
                manning=man, t_end=5.0)


def flooded_plain(nx=2000, ny=1000, dx=2.0, seed=2010, freeboard=0.5, tilt=1e-4):
    """The floodplain terrain fully under water: free surface `freeboard` m above the
    highest ground at the west edge, falling eastwards with slope `tilt`, so every cell
    is wet and the water starts to move; same inflow and edges as the floodplain."""
    case = floodplain(nx=nx, ny=ny, dx=dx, seed=seed)
    X, _ = corner_xy(nx, ny, dx, dx)
    case.eta_corner = case.z_corner.max() + freeboard - tilt * X
    case.name = f"flooded{nx}x{ny}"
    return case


def urban(nx=8192, ny=8192, dx=0.5, seed=2012, slope=1.0 / 500.0, noise=0.05, nblocks=2000,
          block_min=10.0, block_max=40.0, block_height=5.0, road_every=200.0, road_width=12.0,
          rain_mm_h=50.0, rain_minutes=30.0, q_point=2.0, dt_max=0.05):
    """Urban-style grid: a plane falling eastwards (slope 1:500) with fBm roughness of
    `noise` m, `nblocks` rectangular buildings (sides U[10, 40] m, random positions,
    overlaps allowed) raised `block_height` m, Manning 0.02 on a road grid (12 m
    corridors every 200 m in x and y) and 0.05 elsewhere, rain of 50 mm/h for the first
    30 min and a 2 m^3/s point inflow at the centre; transmissive edges, dry start.
    With the defaults: 8192 x 8192 cells of 0.5 m (a 4096 m square)."""
    Lx, Ly = nx * dx, ny * dx
    X, Y = corner_xy(nx, ny, dx, dx)
    z = slope * (Lx - X) + fbm(ny + 1, nx + 1, 0.8, noise, seed)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    for _ in range(nblocks):
        w, h = rng.uniform(block_min, block_max, size=2)
        x0, y0 = rng.uniform(0.0, Lx), rng.uniform(0.0, Ly)
        i0, i1 = int(x0 / dx), min(int((x0 + w) / dx), nx)
        j0, j1 = int(y0 / dx), min(int((y0 + h) / dx), ny)
        z[j0:j1 + 1, i0:i1 + 1] += block_height
    xc = (np.arange(nx) + 0.5) * dx
    yc = (np.arange(ny) + 0.5) * dx
    road_x = (np.mod(xc, road_every) < road_width)[None, :]
    road_y = (np.mod(yc, road_every) < road_width)[:, None]
    man = np.where(road_x | road_y, 0.02, 0.05).astype(np.float64)
    return Case(name=f"urban{nx}x{ny}", nx=nx, ny=ny, dx=dx, dy=dx, z_corner=z, eta_corner=None,
                manning=man, bc=(OPEN, OPEN, OPEN, OPEN), cfl=0.33, t_end=1800.0,
                rain=(rain_mm_h / 1000.0 / 3600.0, 0.0, rain_minutes * 60.0),
                point=(0.5 * Lx, 0.5 * Ly, q_point), dt_max=dt_max)


# ----------------------------------------------------------------------------
# Ensembles
# ----------------------------------------------------------------------------

def ensemble(n=256, seed=3000, nx_range=(64, 1024), ny_range=(64, 512), dx=2.0,
             n_range=(0.02, 0.08), q_range=(5.0, 40.0), t_peak=1800.0, t_end=3600.0, ngauge=4,
             sample_every=60.0):
    """`n` floodplain scenarios of the recipe above, scenario s drawn with seed + s:
    nx and ny log-uniform in their ranges, one uniform Manning n in `n_range`, an
    inflow peak uniform in `q_range` (triangle peaking at `t_peak`), the terrain of
    the floodplain generator at that size (seed + s), starting dry."""
    cases = []
    for s in range(n):
        rng = np.random.Generator(np.random.PCG64(seed + s))
        nx = int(round(np.exp(rng.uniform(np.log(nx_range[0]), np.log(nx_range[1])))))
        ny = int(round(np.exp(rng.uniform(np.log(ny_range[0]), np.log(ny_range[1])))))
        man = float(rng.uniform(*n_range))
        q = float(rng.uniform(*q_range))
        c = floodplain(nx=nx, ny=ny, dx=dx, seed=seed + s, q_peak=q, t_peak=t_peak, t_end=t_end,
                       n_channel=man, n_plain=man, ngauge=ngauge, sample_every=sample_every)
        c.name = f"member{s}_{nx}x{ny}"
        cases.append(c)
    return cases
