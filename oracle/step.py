"""Vortex shedding and time stepping (Sec. 2.4.2-2.4.3, the paper's stepping rules).

Test infrastructure only (see the package docstring).

Rules taken from the paper (Sec. 2.4.2): the first vortex released from an
edge sits 10 dt U_inf from the edge; every later one sits one third of the way
from the edge to the last vortex released from that edge; vortices advect with
the local velocity (forward Euler in the paper).  Readings where the paper is
terse: the "edge" is the Kutta point pushed half a surface segment outward
along the surface; the first offset is along the surface normal at the edge
whose dot product with the free stream is positive; RK2 is Heun's method whose
second stage keeps the new strengths and enforces the Kelvin condition through
the circulation-constrained system (Eq. circsystem) with no further shedding.
"""
import math

import numpy as np

from . import body as B
from .vic import regularize, circulation, streamfunction, node_velocity, interpolate


class Kinematics:
    """Rigid body pitching about the origin: alpha(t) = alpha0 + amp sin(omega t).

    The body is given in its own frame (default: a flat plate of `ns` segment
    midpoints along x, edges at both ends) and turned by -alpha, so a plate's
    chord points along (cos alpha, -sin alpha) and Omega = -amp omega cos(omega t).
    A body with no edges is Kelvin-constrained and releases nothing.
    """

    def __init__(self, ns, chord, alpha0, amp=0.0, omega=0.0, Uinf=1.0, Vinf=0.0, body=None, edge_bounds=None):
        self.ns, self.chord, self.alpha0, self.amp, self.omega = ns, chord, alpha0, amp, omega
        self.Uinf, self.Vinf = Uinf, Vinf
        self.edge_bounds = edge_bounds      # None: Kutta at both edges; else generalized (Sec. 2.5)
        if body is None:
            xi = -1.0 + (2.0 * np.arange(1, ns + 1) - 1.0) / ns
            body = (0.5 * chord * xi, np.zeros(ns), np.full(ns, chord / ns), (0, ns - 1))
        self.xb, self.yb, self.ds, self.edges = body

    def alpha(self, t):
        return self.alpha0 + self.amp * math.sin(self.omega * t)

    def surface(self, t):
        a = self.alpha(t)
        ca, sa = math.cos(a), math.sin(a)
        x = ca * self.xb + sa * self.yb
        y = -sa * self.xb + ca * self.yb
        return x, y, self.ds, tuple(self.edges)

    def Omega(self, t):
        return -self.amp * self.omega * math.cos(self.omega * t)


def _neighbour(k, n):
    """The surface point next to edge point k, away from the edge."""
    return 1 if k == 0 else (n - 2 if k == n - 1 else k + 1)


def edge_point(xs, ys, k):
    """Geometric edge next to Kutta point k: half a segment beyond it."""
    nb = _neighbour(k, len(xs))
    return xs[k] + 0.5 * (xs[k] - xs[nb]), ys[k] + 0.5 * (ys[k] - ys[nb])


def new_vortex_position(xs, ys, k, last, dt, Uinf, Vinf):
    """Placement rule of Sec. 2.4.2 for the vortex released at edge k."""
    ex, ey = edge_point(xs, ys, k)
    if last is None:
        nb = _neighbour(k, len(xs))
        tx, ty = xs[k] - xs[nb], ys[k] - ys[nb]
        nx_, ny_ = -ty, tx
        nrm = math.hypot(nx_, ny_)
        nx_, ny_ = nx_ / nrm, ny_ / nrm
        if nx_ * Uinf + ny_ * Vinf < 0.0:
            nx_, ny_ = -nx_, -ny_
        d = 10.0 * dt * math.hypot(Uinf, Vinf)
        return ex + d * nx_, ey + d * ny_
    return ex + (last[0] - ex) / 3.0, ey + (last[1] - ey) / 3.0


class BodyState:
    def __init__(self):
        self.X = np.zeros(0)
        self.Y = np.zeros(0)
        self.G = np.zeros(0)
        self.last = [None, None]     # index of the last vortex released at each edge
        self.t = 0.0


def _solve_and_velocity(grid, table, kin, t, X, Y, G, shed, dt, last_pos):
    """One stage: sheet solve (two-edge Kutta shedding or Kelvin circulation) and
    velocities at all vortices.  Returns (u, v, newX, newY, newG, info)."""
    xs, ys, ds, edges = kin.surface(t)
    st = B.SurfaceStencil(grid, xs, ys)
    sch = B.Schur(B.schur_matrix(grid, st, ds, table), ds)
    sbp = B.sb_prime(xs, ys, 0.0, 0.0, kin.Omega(t), kin.Uinf, kin.Vinf)
    w = regularize(grid, X, Y, G)
    Gw = circulation(grid, w)
    EinvLw = -B.interp_surface(st, streamfunction(grid, w, table))
    if shed:
        k1, k2 = edges
        p1 = new_vortex_position(xs, ys, k1, last_pos[0], dt, kin.Uinf, kin.Vinf)
        p2 = new_vortex_position(xs, ys, k2, last_pos[1], dt, kin.Uinf, kin.Vinf)
        nX, nY = np.array([p1[0], p2[0]]), np.array([p1[1], p2[1]])
        E = B.EinvL_unit_vortex(grid, st, nX, nY, table)
        if kin.edge_bounds is None:
            f, ft, s0, G1, G2 = B.sheet_kutta_shed2(sch, sbp, EinvLw, k1, k2, E[:, 0], E[:, 1], Gw)
            nG = np.array([G1, G2])
        else:      # an edge inside its bounds releases a vortex of zero strength
            f, ft, s0, nG = B.sheet_edge_shed(sch, sbp, EinvLw, (k1, k2), (E[:, 0], E[:, 1]), Gw, kin.edge_bounds)
    else:
        f, s0 = B.sheet_circulation(sch, sbp, EinvLw, -Gw)
        nX, nY, nG = np.zeros(0), np.zeros(0), np.zeros(0)
    AX, AY, AG = np.concatenate([X, nX]), np.concatenate([Y, nY]), np.concatenate([G, nG])
    wt = regularize(grid, AX, AY, AG) + B.regularize_surface(grid, st, f, ds)
    psi1 = streamfunction(grid, wt, table, pad=1)
    u, v = node_velocity(grid, psi1, kin.Uinf, kin.Vinf)
    info = dict(f=f, s0=s0, Gw=Gw, circ_f=sch.circ(f), psi=psi1[1:-1, 1:-1], st=st, sch=sch, sbp=sbp)
    return interpolate(grid, u, AX, AY), interpolate(grid, v, AX, AY), nX, nY, nG, info


def body_step(grid, table, kin, state, dt, scheme="euler"):
    """Advance the vortex set one step: two-edge Kutta shedding (Sec. 2.4.3) for
    a body with two edges, the Kelvin-constrained sheet otherwise."""
    t = state.t
    release = len(kin.edges) == 2
    last_pos = [None if i is None else (state.X[i], state.Y[i]) for i in state.last]
    u1, v1, nX, nY, nG, info = _solve_and_velocity(grid, table, kin, t, state.X, state.Y, state.G,
                                                   release, dt, last_pos)
    X = np.concatenate([state.X, nX])
    Y = np.concatenate([state.Y, nY])
    G = np.concatenate([state.G, nG])
    if scheme == "euler":
        X, Y = X + dt * u1, Y + dt * v1
    elif scheme == "rk2":
        Xs, Ys = X + dt * u1, Y + dt * v1
        u2, v2, _, _, _, _ = _solve_and_velocity(grid, table, kin, t + dt, Xs, Ys, G, False, dt, None)
        X, Y = X + 0.5 * dt * (u1 + u2), Y + 0.5 * dt * (v1 + v2)
    else:
        raise ValueError(scheme)
    n_old = len(state.X)
    state.X, state.Y, state.G = X, Y, G
    if release:
        state.last = [n_old, n_old + 1]
    state.t = t + dt
    return info


# ----------------------------------------------------------------- several bodies
class MultiBodyState:
    """Vortices, the index of the last vortex released at every edge (edges in
    body order) and the circulation released so far by each body."""

    def __init__(self, n_bodies, n_edges):
        self.X = np.zeros(0)
        self.Y = np.zeros(0)
        self.G = np.zeros(0)
        self.last = [None] * n_edges
        self.released = np.zeros(n_bodies)
        self.t = 0.0


def _multi_surface(kins, t):
    """Concatenated surface of the bodies at time t: points, segment lengths,
    body offsets, edges (global indices, per body) and s'_b of each body's
    rotation in the free stream of the first body."""
    xs, ys, ds, starts, edges, sbp = [], [], [], [0], [], []
    for kin in kins:
        x, y, d, e = kin.surface(t)
        off = starts[-1]
        xs.append(x); ys.append(y); ds.append(d)
        edges.append(tuple(off + k for k in e))
        sbp.append(B.sb_prime(x, y, 0.0, 0.0, kin.Omega(t), kins[0].Uinf, kins[0].Vinf))
        starts.append(off + len(x))
    return (np.concatenate(xs), np.concatenate(ys), np.concatenate(ds), np.array(starts), edges,
            np.concatenate(sbp))


def _multi_stage(grid, table, kins, t, X, Y, G, shed, dt, last_pos, released):
    """One stage with several bodies: the sheet of Eq. kuttasystem4 (Kutta at
    every edge when shedding, otherwise every body circulation-constrained)
    and the velocities at all vortices.  Gamma_w of body b >= 1 is the
    circulation it released; body 0 takes the rest of the flow's circulation
    (so one body is the single-body step)."""
    xs, ys, ds, starts, edges, sbp = _multi_surface(kins, t)
    st = B.SurfaceStencil(grid, xs, ys)
    sch = B.Schur(B.schur_matrix(grid, st, ds, table), ds)
    w = regularize(grid, X, Y, G)
    Gtot = circulation(grid, w)
    Gws = np.concatenate([[Gtot - np.sum(released[1:])], released[1:]])
    EinvLw = -B.interp_surface(st, streamfunction(grid, w, table))
    U, V = kins[0].Uinf, kins[0].Vinf
    if shed:
        pos = []
        e = 0
        for b, eb in enumerate(edges):
            lo, hi = starts[b], starts[b + 1]      # the edge's neighbour is on its own body
            for k in eb:
                pos.append(new_vortex_position(xs[lo:hi], ys[lo:hi], k - lo, last_pos[e], dt, U, V))
                e += 1
        nX, nY = np.array([p[0] for p in pos]), np.array([p[1] for p in pos])
        E = B.EinvL_unit_vortex(grid, st, nX, nY, table)
        f, ft, s0, nG = B.sheet_multibody_shed(sch, sbp, EinvLw, starts, edges, E, Gws)
    else:
        f, ft, s0, _ = B.sheet_multibody_shed(sch, sbp, EinvLw, starts, [()] * len(kins),
                                              np.zeros((len(xs), 0)), Gws)
        nX, nY, nG = np.zeros(0), np.zeros(0), np.zeros(0)
    AX, AY, AG = np.concatenate([X, nX]), np.concatenate([Y, nY]), np.concatenate([G, nG])
    wt = regularize(grid, AX, AY, AG) + B.regularize_surface(grid, st, f, ds)
    psi1 = streamfunction(grid, wt, table, pad=1)
    u, v = node_velocity(grid, psi1, U, V)
    info = dict(f=f, s0=s0, Gws=Gws, starts=starts, edges=edges, ds=ds,
                circ_b=[float(np.dot(ds[a:b], f[a:b])) for a, b in zip(starts[:-1], starts[1:])])
    return interpolate(grid, u, AX, AY), interpolate(grid, v, AX, AY), nX, nY, nG, info


def multibody_step(grid, table, kins, state, dt, scheme="euler"):
    """Advance the vortex set one step with several bodies (Sec. 2.7): one new
    vortex per edge (Kutta), Kelvin per body; the rules of body_step otherwise."""
    t = state.t
    edges_per = [len(k.edges) for k in kins]
    release = sum(edges_per) > 0
    last_pos = [None if i is None else (state.X[i], state.Y[i]) for i in state.last]
    u1, v1, nX, nY, nG, info = _multi_stage(grid, table, kins, t, state.X, state.Y, state.G, release, dt, last_pos,
                                            state.released)
    e = 0
    for b, n in enumerate(edges_per):
        state.released[b] += float(np.sum(nG[e:e + n]))
        e += n
    X = np.concatenate([state.X, nX])
    Y = np.concatenate([state.Y, nY])
    G = np.concatenate([state.G, nG])
    if scheme == "euler":
        X, Y = X + dt * u1, Y + dt * v1
    elif scheme == "rk2":
        Xs, Ys = X + dt * u1, Y + dt * v1
        u2, v2, _, _, _, _ = _multi_stage(grid, table, kins, t + dt, Xs, Ys, G, False, dt, None, state.released)
        X, Y = X + 0.5 * dt * (u1 + u2), Y + 0.5 * dt * (v1 + v2)
    else:
        raise ValueError(scheme)
    n_old = len(state.X)
    state.X, state.Y, state.G = X, Y, G
    if release:
        state.last = [n_old + i for i in range(len(nG))]
    state.t = t + dt
    return info
