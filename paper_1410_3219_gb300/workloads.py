"""Seeded synthetic inputs shaped like the paper's test problems.

This module only draws generating points and evaluates the initial primitive
fields (rho, vx, vy, p) that each problem statement prescribes at those points.
It holds none of the scheme's arithmetic (no tessellation, no fluxes), so both
the CUDA library and the CPU oracle can be driven from the same inputs.

Every generator returns a dict with
  cfg  : scheme parameters (gamma, cfl, boundary, box, mesh motion, Lloyd and
         limiter constants) as plain numbers;
  x, y : float64 generating-point coordinates;
  rho, vx, vy, p : float64 initial primitive fields at the points;
  name, seed : provenance.

Defaults follow Section 2 of the paper: theta = 0.5, delta_v = 0.2,
delta_p = 0.7 (Section 2.2), Courant number 0.3 (Section 2.3), Lloyd-type
rounding chi = 0.15, eta = 0.02 (Section 6).
"""
from __future__ import annotations

import math

import numpy as np

BC_REFLECTIVE = 0
BC_PERIODIC = 1
MESH_LAGRANGIAN = 0
MESH_EULERIAN = 1
LIM_SWITCHED = 0
LIM_AREPO = 1
LIM_TESS = 2
FP64 = 0
FP32_SPLIT = 1
SCHEME_EXTRAPOLATED = 0
SCHEME_TIME_CENTRED = 1


def default_cfg(**over):
    cfg = dict(gamma=5.0 / 3.0, cfl=0.3, boundary=BC_PERIODIC,
               x0=0.0, x1=1.0, y0=0.0, y1=1.0,
               motion=MESH_LAGRANGIAN, chi=0.15, eta=0.02,
               theta=0.5, delta_v=0.2, delta_p=0.7, limiter=LIM_SWITCHED,
               scheme=SCHEME_EXTRAPOLATED)
    cfg.update(over)
    return cfg


def jittered_lattice(nx, ny, x0, x1, y0, y1, jitter, rng):
    """Points at cell centres (i+1/2)h of an nx-by-ny lattice, each coordinate
    moved by U(-jitter, jitter) lattice spacings.  Row-major order (y slowest)."""
    hx = (x1 - x0) / nx
    hy = (y1 - y0) / ny
    ii, jj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    x = x0 + (ii.ravel() + 0.5) * hx
    y = y0 + (jj.ravel() + 0.5) * hy
    if jitter > 0.0:
        x = x + rng.uniform(-jitter, jitter, x.size) * hx
        y = y + rng.uniform(-jitter, jitter, y.size) * hy
    return x.astype(np.float64), y.astype(np.float64)


def _pack(name, seed, cfg, x, y, rho, vx, vy, p):
    n = x.size
    f = lambda a: np.ascontiguousarray(np.broadcast_to(np.asarray(a, np.float64), (n,)))
    return dict(name=name, seed=seed, cfg=cfg, x=f(x), y=f(y), rho=f(rho),
                vx=f(vx), vy=f(vy), p=f(p))


def sod(n_side=64, seed=1, jitter=0.1, motion=MESH_LAGRANGIAN):
    """2D shock tube split at x = 0.5 on the unit square with reflecting walls:
    rho = 1, p = 1 on the left, rho = 0.125, p = 0.1 on the right, v = 0,
    gamma = 1.4 (the classic Sod states, run as the paper's 1D/2D shock tube
    tests of Sections 3.3 and 4.6)."""
    rng = np.random.default_rng(seed)
    cfg = default_cfg(gamma=1.4, boundary=BC_REFLECTIVE, motion=motion)
    x, y = jittered_lattice(n_side, n_side, 0.0, 1.0, 0.0, 1.0, jitter, rng)
    left = x < 0.5
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    return _pack("sod", seed, cfg, x, y, rho, 0.0, 0.0, p)


def sedov(n=262144, seed=2, e_blast=1.0, n_blast=16, motion=MESH_LAGRANGIAN):
    """Point explosion: n i.i.d. uniform points in [-0.5, 0.5]^2, gamma = 5/3,
    rho = 1, p = 1e-5, reflecting walls, and energy e_blast shared by the
    n_blast points nearest the origin (ties by index).  The deposit pressure
    uses the nominal cell area (box area / n), so the deposited energy equals
    e_blast up to the area spread of those cells."""
    rng = np.random.default_rng(seed)
    cfg = default_cfg(gamma=5.0 / 3.0, boundary=BC_REFLECTIVE, motion=motion,
                      x0=-0.5, x1=0.5, y0=-0.5, y1=0.5)
    x = rng.uniform(-0.5, 0.5, n)
    y = rng.uniform(-0.5, 0.5, n)
    r2 = x * x + y * y
    hot = np.lexsort((np.arange(n), r2))[:n_blast]
    p = np.full(n, 1e-5)
    a_nom = 1.0 / n
    p[hot] = (cfg["gamma"] - 1.0) * e_blast / (n_blast * a_nom)
    return _pack("sedov", seed, cfg, x, y, 1.0, 0.0, 0.0, p)


def kelvin_helmholtz(n_side=1024, seed=3, jitter=0.1, amp=0.01, motion=MESH_LAGRANGIAN):
    """Shear layer in the periodic unit box: p = 2.5, gamma = 5/3,
    rho = 2, vx = +0.5 for |y - 0.5| < 0.25, else rho = 1, vx = -0.5, and
    vy = amp * sin(4 pi x) (Section 4.4 uses a Gaussian-windowed 0.1 seed)."""
    rng = np.random.default_rng(seed)
    cfg = default_cfg(gamma=5.0 / 3.0, boundary=BC_PERIODIC, motion=motion)
    x, y = jittered_lattice(n_side, n_side, 0.0, 1.0, 0.0, 1.0, jitter, rng)
    inner = np.abs(y - 0.5) < 0.25
    rho = np.where(inner, 2.0, 1.0)
    vx = np.where(inner, 0.5, -0.5)
    vy = amp * np.sin(4.0 * math.pi * x)
    return _pack("kelvin_helmholtz", seed, cfg, x, y, rho, vx, vy, 2.5)


def gresho_fields(x, y):
    """Gresho vortex profile of Section 4.3 (centre at the origin): rho = 1,
    azimuthal velocity 5r / 2-5r / 0 and the balancing pressure."""
    r = np.hypot(x, y)
    p = np.where(r < 0.2, 5.0 + 12.5 * r * r,
                 np.where(r < 0.4, 9.0 + 12.5 * r * r - 20.0 * r + 4.0 * np.log(np.maximum(5.0 * r, 1e-300)),
                          3.0 + 4.0 * math.log(2.0)))
    vphi = np.where(r < 0.2, 5.0 * r, np.where(r < 0.4, 2.0 - 5.0 * r, 0.0))
    with np.errstate(invalid="ignore", divide="ignore"):
        ux = np.where(r > 0, -y / np.where(r > 0, r, 1.0), 0.0)
        uy = np.where(r > 0, x / np.where(r > 0, r, 1.0), 0.0)
    return np.ones_like(x), vphi * ux, vphi * uy, p


def gresho(n_side=64, seed=4, jitter=0.1, motion=MESH_LAGRANGIAN, chi=0.15, eta=0.02):
    """Gresho vortex in the periodic box [-0.5, 0.5]^2, gamma = 5/3, peak
    azimuthal velocity 1 at r = 0.2 (Section 4.3)."""
    rng = np.random.default_rng(seed)
    cfg = default_cfg(gamma=5.0 / 3.0, boundary=BC_PERIODIC, motion=motion,
                      x0=-0.5, x1=0.5, y0=-0.5, y1=0.5, chi=chi, eta=eta)
    x, y = jittered_lattice(n_side, n_side, -0.5, 0.5, -0.5, 0.5, jitter, rng)
    rho, vx, vy, p = gresho_fields(x, y)
    return _pack("gresho", seed, cfg, x, y, rho, vx, vy, p)


def advection(n_side=32, seed=0, jitter=0.0, motion=MESH_LAGRANGIAN):
    """Pure advection of Section 4.1: periodic [-0.5, 0.5]^2, p = 1,
    v = (1, 1), rho = 100 inside r < 0.2 and 1 outside."""
    rng = np.random.default_rng(seed)
    cfg = default_cfg(gamma=5.0 / 3.0, boundary=BC_PERIODIC, motion=motion,
                      x0=-0.5, x1=0.5, y0=-0.5, y1=0.5)
    x, y = jittered_lattice(n_side, n_side, -0.5, 0.5, -0.5, 0.5, jitter, rng)
    rho = np.where(np.hypot(x, y) < 0.2, 100.0, 1.0)
    return _pack("advection", seed, cfg, x, y, rho, 1.0, 1.0, 1.0)


def sound_wave(n_side=32, seed=9, jitter=0.1, amp=1e-3, motion=MESH_LAGRANGIAN, scheme=SCHEME_EXTRAPOLATED):
    """Right-moving linear sound wave along x in the periodic unit box:
    gamma = 5/3, rho = 1 + a sin(2 pi x), p = 1 + gamma a sin(2 pi x),
    vx = c a sin(2 pi x) with c = sqrt(gamma); a smooth solution for
    convergence checks."""
    rng = np.random.default_rng(seed)
    g = 5.0 / 3.0
    cfg = default_cfg(gamma=g, boundary=BC_PERIODIC, motion=motion, scheme=scheme)
    x, y = jittered_lattice(n_side, n_side, 0.0, 1.0, 0.0, 1.0, jitter, rng)
    s = np.sin(2.0 * math.pi * x)
    return _pack("sound_wave", seed, cfg, x, y, 1.0 + amp * s, math.sqrt(g) * amp * s, 0.0,
                 1.0 + g * amp * s)


def uniform(n_side=16, seed=5, jitter=0.25, boundary=BC_PERIODIC, rho=1.3, vx=0.4,
            vy=-0.7, p=0.9, motion=MESH_LAGRANGIAN, gamma=1.4):
    """Uniform state on a jittered lattice (free-stream preservation)."""
    rng = np.random.default_rng(seed)
    cfg = default_cfg(gamma=gamma, boundary=boundary, motion=motion)
    x, y = jittered_lattice(n_side, n_side, 0.0, 1.0, 0.0, 1.0, jitter, rng)
    return _pack("uniform", seed, cfg, x, y, rho, vx, vy, p)


def random_smooth(n=300, seed=6, boundary=BC_PERIODIC, motion=MESH_LAGRANGIAN, gamma=1.4,
                  limiter=LIM_SWITCHED):
    """Random points in the unit box with smooth, non-trivial fields in all
    four primitives (exercises every term of the sweep)."""
    rng = np.random.default_rng(seed)
    cfg = default_cfg(gamma=gamma, boundary=boundary, motion=motion, limiter=limiter)
    x = rng.uniform(0.0, 1.0, n)
    y = rng.uniform(0.0, 1.0, n)
    tp = 2.0 * math.pi
    rho = 1.0 + 0.3 * np.sin(tp * x) * np.cos(tp * y)
    vx = 0.4 * np.sin(tp * y)
    vy = -0.3 * np.cos(tp * x)
    p = 1.0 + 0.2 * np.cos(tp * (x + y))
    return _pack("random_smooth", seed, cfg, x, y, rho, vx, vy, p)


def random_mixed(n=500, seed=7, boundary=BC_REFLECTIVE, motion=MESH_LAGRANGIAN, gamma=5.0 / 3.0):
    """Random points with a pressure/density jump plus noise, so that both
    limiter branches and the shock switch fire."""
    rng = np.random.default_rng(seed)
    cfg = default_cfg(gamma=gamma, boundary=boundary, motion=motion)
    x = rng.uniform(0.0, 1.0, n)
    y = rng.uniform(0.0, 1.0, n)
    hot = (x - 0.5) ** 2 + (y - 0.5) ** 2 < 0.04
    rho = np.where(hot, 2.0, 1.0) * (1.0 + 0.05 * rng.uniform(-1, 1, n))
    p = np.where(hot, 5.0, 1.0) * (1.0 + 0.05 * rng.uniform(-1, 1, n))
    vx = 0.3 * rng.uniform(-1, 1, n)
    vy = 0.3 * rng.uniform(-1, 1, n)
    return _pack("random_mixed", seed, cfg, x, y, rho, vx, vy, p)


def batch_mix(n_inst=256, seed=4, n_min=1000, n_max=64000):
    """Independent instances whose sizes are log-uniform in [n_min, n_max],
    problem types cycling Sod / Sedov / Gresho."""
    rng = np.random.default_rng(seed)
    sizes = np.round(np.exp(rng.uniform(math.log(n_min), math.log(n_max), n_inst))).astype(int)
    out = []
    for k, nk in enumerate(sizes):
        kind = k % 3
        side = max(4, int(round(math.sqrt(nk))))
        if kind == 0:
            out.append(sod(n_side=side, seed=1000 + k))
        elif kind == 1:
            out.append(sedov(n=int(nk), seed=1000 + k))
        else:
            out.append(gresho(n_side=side, seed=1000 + k))
    return out
