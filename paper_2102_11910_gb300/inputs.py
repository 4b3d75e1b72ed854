"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle tests.

This module only draws and lays out inputs (grids, point vortices, surface
points of plates, circles and ellipses); it holds none of the method's
arithmetic.  Every generator takes an explicit seed (numpy PCG64).

Workloads (shapes of the paper's synthetic experiments):

* ``plate_vortices_128``: 128 x 128 nodes, dx = 0.02, grid centred on the
  origin; flat plate of chord 1 at 20 deg in uniform flow (1, 0) with 64
  surface points; 256 vortices uniform in [-1, 1]^2, none within 3 dx of the
  plate, strengths normal with variance 0.01.  Seed 1000.
* ``vic_1024``: 1024 x 1024 nodes on [-1, 1]^2 (dx = 2/1023); 1e6 vortices
  uniform in the central 80 % of the domain, strengths normal with variance
  1e-4; no body.  Seed 1001.
* ``pitching_plate_512x768``: 768 (x) by 512 (y) nodes, dx = 0.01, plate of
  chord 1, 256 points, mid-chord 1.5 chords from the upstream edge.  Seed 1002.
"""
import math
from dataclasses import dataclass

import numpy as np


@dataclass
class GridSpec:
    nx: int
    ny: int
    dx: float
    x0: float
    y0: float


@dataclass
class SurfaceSpec:
    x: np.ndarray
    y: np.ndarray
    ds: np.ndarray
    edges: tuple          # surface-point indices of sharp edges (empty for smooth bodies)


def centred_grid(nx, ny, dx):
    """Grid whose node block is centred on the origin."""
    return GridSpec(nx, ny, dx, -0.5 * (nx - 1) * dx, -0.5 * (ny - 1) * dx)


def plate(ns, chord=1.0, alpha=0.0, xc=0.0, yc=0.0):
    """Flat plate: points at the midpoints of ns equal segments.

    xi_p = -1 + (2p - 1)/ns (p = 1..ns) runs from the leading edge (xi = -1) to
    the trailing edge (xi = 1); the chord points along (cos a, -sin a), so the
    leading edge is raised for a > 0.  Edges: first and last point.
    """
    xi = -1.0 + (2.0 * np.arange(1, ns + 1) - 1.0) / ns
    x = xc + 0.5 * chord * xi * math.cos(alpha)
    y = yc - 0.5 * chord * xi * math.sin(alpha)
    return SurfaceSpec(x, y, np.full(ns, chord / ns), (0, ns - 1))


def plate_xi(ns):
    return -1.0 + (2.0 * np.arange(1, ns + 1) - 1.0) / ns


def circle(ns, radius=1.0, xc=0.0, yc=0.0):
    """Circle: theta_p = 2 pi (p - 1)/ns, counter-clockwise from +x."""
    th = 2.0 * np.pi * np.arange(ns) / ns
    return SurfaceSpec(xc + radius * np.cos(th), yc + radius * np.sin(th),
                       np.full(ns, 2.0 * np.pi * radius / ns), ())


def ellipse(ns, a, b, xc=0.0, yc=0.0, rot=0.0):
    """Ellipse with semi-axes a, b: points at equal arc length (numerical inversion)."""
    t = np.linspace(0.0, 2.0 * np.pi, 20001)
    sp = np.sqrt((a * np.sin(t)) ** 2 + (b * np.cos(t)) ** 2)
    s = np.concatenate([[0.0], np.cumsum(0.5 * (sp[1:] + sp[:-1]) * np.diff(t))])
    per = s[-1]
    tp = np.interp(per * np.arange(ns) / ns, s, t)
    x, y = a * np.cos(tp), b * np.sin(tp)
    c, sn = math.cos(rot), math.sin(rot)
    return SurfaceSpec(xc + c * x - sn * y, yc + sn * x + c * y, np.full(ns, per / ns), ())


def uniform_vortices(rng, n, lo, hi, variance, ylo=None, yhi=None):
    """n vortices uniform in [lo, hi] x [ylo, yhi], strengths N(0, variance)."""
    ylo = lo if ylo is None else ylo
    yhi = hi if yhi is None else yhi
    X = rng.uniform(lo, hi, n)
    Y = rng.uniform(ylo, yhi, n)
    G = rng.normal(0.0, math.sqrt(variance), n)
    return X, Y, G


def _dist_to_segment(X, Y, ax, ay, bx, by):
    vx, vy = bx - ax, by - ay
    t = np.clip(((X - ax) * vx + (Y - ay) * vy) / (vx * vx + vy * vy), 0.0, 1.0)
    return np.hypot(X - (ax + t * vx), Y - (ay + t * vy))


def plate_vortices_128(seed=1000, nv=256, ns=64):
    """The single-step plate workload (128^2 nodes, 64 surface points, 256 vortices)."""
    rng = np.random.default_rng(seed)
    grid = centred_grid(128, 128, 0.02)
    alpha = math.radians(20.0)
    body = plate(ns, 1.0, alpha)
    ax, ay = -0.5 * math.cos(alpha), 0.5 * math.sin(alpha)
    X, Y, G = [], [], []
    while len(X) < nv:
        x, y, g = uniform_vortices(rng, nv, -1.0, 1.0, 0.01)
        keep = _dist_to_segment(x, y, ax, ay, -ax, -ay) > 3 * grid.dx
        X += list(x[keep]); Y += list(y[keep]); G += list(g[keep])
    return dict(grid=grid, body=body, X=np.array(X[:nv]), Y=np.array(Y[:nv]), G=np.array(G[:nv]),
                Uinf=1.0, Vinf=0.0, dt=0.01, alpha=alpha)


def _away(X, Y, bodies, d):
    """Mask of points farther than d from every surface point of the bodies."""
    keep = np.ones(len(X), dtype=bool)
    for b in bodies:
        dist = np.min(np.hypot(X[:, None] - b.x[None, :], Y[:, None] - b.y[None, :]), axis=1)
        keep &= dist > d
    return keep


def three_bodies_128(seed=1006, nv=200):
    """Several bodies in one grid (128^2 nodes, dx 0.02, centred): plate A
    (24 points, chord 0.6, 20 deg, both edges), plate B (24 points, chord 0.6,
    -15 deg, trailing edge only) and an ellipse C (40 points, semi-axes 0.25 and
    0.1, no edge), dS/dx 1.25-1.4; nv vortices N(0, 0.01) away from the bodies;
    one new-vortex position near each edge; per-body circulations Gamma_w of
    earlier released vorticity (minus the prescribed circulation for C)."""
    rng = np.random.default_rng(seed)
    grid = centred_grid(128, 128, 0.02)
    A = plate(24, 0.6, math.radians(20.0), -0.5, 0.45)
    B = plate(24, 0.6, math.radians(-15.0), -0.45, -0.5)
    C = ellipse(40, 0.25, 0.1, 0.5, 0.05, 0.3)
    bodies = [A, B, C]
    X, Y, G = [], [], []
    while len(X) < nv:
        x, y, g = uniform_vortices(rng, nv, -1.1, 1.1, 0.01)
        keep = _away(x, y, bodies, 4 * grid.dx)
        X += list(x[keep]); Y += list(y[keep]); G += list(g[keep])
    x = np.concatenate([b.x for b in bodies])
    y = np.concatenate([b.y for b in bodies])
    ds = np.concatenate([b.ds for b in bodies])
    starts = np.array([0, 24, 48, 88])
    edges = [(0, 23), (47,), ()]
    # new vortices: 3 dx off each edge, away from its body's centre
    cen = [(-0.5, 0.45), (-0.45, -0.5), (0.5, 0.05)]
    VX, VY = [], []
    for b, eb in enumerate(edges):
        for k in eb:
            vx, vy = x[k] - cen[b][0], y[k] - cen[b][1]
            r = math.hypot(vx, vy)
            VX.append(x[k] + 3 * grid.dx * vx / r)
            VY.append(y[k] + 3 * grid.dx * vy / r)
    return dict(grid=grid, x=x, y=y, ds=ds, starts=starts, edges=edges, X=np.array(X[:nv]), Y=np.array(Y[:nv]),
                G=np.array(G[:nv]), VX=np.array(VX), VY=np.array(VY), Gamma_w=np.array([0.08, -0.05, 0.03]),
                Uinf=1.0, Vinf=0.0)


def mirrored_plates_128(seed=1007, nv=100):
    """Two plates mirrored in the x axis (24 points each, chord 0.6, +-20 deg,
    centres (-0.3, +-0.35)), 128^2 nodes centred on the origin, and a vortex
    set closed under the mirror (x, y, G) -> (x, -y, -G); uniform flow along x.
    Mirror images: point p of plate B is point p of plate A reflected."""
    rng = np.random.default_rng(seed)
    grid = centred_grid(128, 128, 0.02)
    A = plate(24, 0.6, math.radians(20.0), -0.3, 0.35)
    B = plate(24, 0.6, math.radians(-20.0), -0.3, -0.35)
    X, Y, G = [], [], []
    while len(X) < nv:
        x, y, g = uniform_vortices(rng, nv, -1.1, 1.1, 0.01, 0.05, 1.1)
        keep = _away(x, y, [A, B], 4 * grid.dx)
        X += list(x[keep]); Y += list(y[keep]); G += list(g[keep])
    X, Y, G = np.array(X[:nv]), np.array(Y[:nv]), np.array(G[:nv])
    VX = np.array([A.x[0] - 0.06, A.x[-1] + 0.06])
    VY = np.array([A.y[0] + 0.03, A.y[-1] - 0.03])
    return dict(grid=grid, x=np.concatenate([A.x, B.x]), y=np.concatenate([A.y, B.y]),
                ds=np.concatenate([A.ds, B.ds]), starts=np.array([0, 24, 48]), edges=[(0, 23), (24, 47)],
                X=np.concatenate([X, X]), Y=np.concatenate([Y, -Y]), G=np.concatenate([G, -G]),
                VX=np.concatenate([VX, VX]), VY=np.concatenate([VY, -VY]), Gamma_w=np.array([0.04, -0.04]),
                Uinf=1.0, Vinf=0.0)


def vic_1024(seed=1001, nv=1_000_000, n=1024):
    """The body-free VIC workload: n^2 nodes on [-1,1]^2, nv vortices in the central 80 %."""
    rng = np.random.default_rng(seed)
    dx = 2.0 / (n - 1)
    grid = GridSpec(n, n, dx, -1.0, -1.0)
    X, Y, G = uniform_vortices(rng, nv, -0.8, 0.8, 1e-4)
    return dict(grid=grid, X=X, Y=Y, G=G)


def vic_small(seed, n, nv, variance=1e-4, nyf=1.0):
    """A smaller body-free case of the same recipe (n x round(n*nyf) nodes on [-1,1] in x)."""
    rng = np.random.default_rng(seed)
    ny = int(round(n * nyf))
    dx = 2.0 / (n - 1)
    grid = GridSpec(n, ny, dx, -1.0, -0.5 * (ny - 1) * dx)
    half_y = 0.5 * (ny - 1) * dx
    X, Y, G = uniform_vortices(rng, nv, -0.8, 0.8, variance, -0.8 * half_y, 0.8 * half_y)
    return dict(grid=grid, X=X, Y=Y, G=G)


def pitching_plate_512x768(ns=256):
    """Grid and body-frame plate of the pitching-plate workload."""
    dx = 0.01
    grid = GridSpec(768, 512, dx, -1.5, -0.5 * 511 * dx)
    return dict(grid=grid, ns=ns, chord=1.0, alpha0=math.radians(30.0), amp=math.radians(10.0),
                k=0.5, Uinf=1.0, dt=0.0025)


GRID_SHAPES = ((128, 128), (256, 256), (512, 384), (512, 512))   # (nx, ny)


def batched_instance(rng, shape=None, big=False):
    """One instance of the uneven batch recipe.

    Grid drawn from 128^2, 256^2, 384x512, 512^2 (or 1024^2 with 1e5 vortices
    when `big`), dx = 2/(max(nx, ny) - 1), centred on the origin; one body of
    size 1 at the origin: a flat plate at 5-30 deg releasing at both edges, or
    an ellipse of aspect 2-10 (Kelvin-constrained); surface points 32-256 with
    dS/dx in [1, 4] (below 1 the sheet system is so ill-conditioned that the
    released strengths diverge within a few steps, in FP64 too); 100-20000
    vortices (log-uniform) outside radius 0.55, in x from -0.8 to 0.4 of the
    half-width and at least 0.35 from the top and bottom, strengths normal
    with variance 1e-3.  Those strengths induce speeds that grow like
    sqrt(count) (median ~0.023 sqrt(count) U_inf, peaks about three times
    that), so each instance carries its own time step: at most 0.002, and at
    most half a cell per step at three times that median speed plus U_inf.
    """
    if big:
        nx = ny = 1024
    else:
        nx, ny = GRID_SHAPES[rng.integers(len(GRID_SHAPES))] if shape is None else shape
    dx = 2.0 / (max(nx, ny) - 1)
    grid = centred_grid(nx, ny, dx)
    plate_body = rng.random() < 0.5
    perim = 1.0 if plate_body else None
    if not plate_body:
        ar = rng.uniform(2.0, 10.0)
        a, b = 0.5, 0.5 / ar
        t = np.linspace(0.0, 2 * np.pi, 2001)
        perim = float(np.sum(np.hypot(np.diff(a * np.cos(t)), np.diff(b * np.sin(t)))))
    lo = max(32, int(math.ceil(perim / (4.0 * dx))))
    hi = min(256, int(perim / dx))
    ns = int(rng.integers(lo, max(lo, hi) + 1))
    if plate_body:
        xi = -1.0 + (2.0 * np.arange(1, ns + 1) - 1.0) / ns
        body = dict(xb=0.5 * xi, yb=np.zeros(ns), ds=np.full(ns, 1.0 / ns), edges=(0, ns - 1),
                    alpha0=math.radians(rng.uniform(5.0, 30.0)))
    else:
        e = ellipse(ns, a, b)
        body = dict(xb=e.x, yb=e.y, ds=e.ds, edges=(), alpha0=rng.uniform(0.0, math.pi))
    nv = 100000 if big else int(round(math.exp(rng.uniform(math.log(100), math.log(20000)))))
    hx, hy = 0.5 * (nx - 1) * dx, 0.5 * (ny - 1) * dx - 0.35
    X, Y = np.empty(0), np.empty(0)
    while len(X) < nv:
        # upstream-biased box so that 50 steps of advection stay on the grid
        x = rng.uniform(-0.8 * hx, 0.4 * hx, 2 * nv)
        y = rng.uniform(-hy, hy, 2 * nv)
        keep = np.hypot(x, y) > 0.55
        X, Y = np.concatenate([X, x[keep]]), np.concatenate([Y, y[keep]])
    G = rng.normal(0.0, math.sqrt(1e-3), nv)
    speed = 1.0 + 3.0 * 0.023 * math.sqrt(nv)
    dt = min(0.002, 0.5 * dx / speed)
    return dict(grid=grid, body=body, X=X[:nv], Y=Y[:nv], G=G, Uinf=1.0, dt=dt)


def plate_vortices_1024(seed=1005, nv=100000, ns=256):
    """The large served instance with a plate: 1024^2 nodes, dx = 2/1023,
    centred; a plate of chord 1 at 20 deg with ns = 256 points (dS/dx = 2)
    releasing at both edges; nv vortices placed and drawn as in
    batched_instance (outside radius 0.55, upstream-biased box, strengths
    N(0, 1e-3)) with its CFL step."""
    rng = np.random.default_rng(seed)
    nx = ny = 1024
    dx = 2.0 / (nx - 1)
    grid = centred_grid(nx, ny, dx)
    xi = -1.0 + (2.0 * np.arange(1, ns + 1) - 1.0) / ns
    body = dict(xb=0.5 * xi, yb=np.zeros(ns), ds=np.full(ns, 1.0 / ns), edges=(0, ns - 1), alpha0=math.radians(20.0))
    hx, hy = 0.5 * (nx - 1) * dx, 0.5 * (ny - 1) * dx - 0.35
    X, Y = np.empty(0), np.empty(0)
    while len(X) < nv:
        x = rng.uniform(-0.8 * hx, 0.4 * hx, 2 * nv)
        y = rng.uniform(-hy, hy, 2 * nv)
        keep = np.hypot(x, y) > 0.55
        X, Y = np.concatenate([X, x[keep]]), np.concatenate([Y, y[keep]])
    G = rng.normal(0.0, math.sqrt(1e-3), nv)
    dt = min(0.002, 0.5 * dx / (1.0 + 3.0 * 0.023 * math.sqrt(nv)))
    return dict(grid=grid, body=body, X=X[:nv], Y=Y[:nv], G=G, Uinf=1.0, dt=dt)


def batched_instances(seed=1003, n=256):
    """The uneven batch: n independent instances (seed 1003)."""
    rng = np.random.default_rng(seed)
    return [batched_instance(rng) for _ in range(n)]


def serving_requests(seed=1004, n=4096, big_fraction=0.1):
    """Requests of the serving workload: instances as in the batch, 10 % at
    1024^2 with 1e5 vortices, each for 1-50 steps (uniform)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        r = batched_instance(rng, big=rng.random() < big_fraction)
        r["nsteps"] = int(rng.integers(1, 51))
        out.append(r)
    return out
