"""Pins of the oracle's Heun (RK2) and Euler updates in the time steps
(Sec. 2.4.2: vortices advect with the local velocity; RK2 is Heun's method,
the predictor X + dt u(X), the corrector X + dt/2 (u(X) + u(X_pred))).

Two checks that the oracle cannot pass by agreeing with itself:

* exact translation: a plate along the free stream (zero incidence) with no
  free vorticity carries no sheet and sheds vortices of zero strength, so the
  flow is the uniform stream everywhere and every vortex (a passive tracer of
  zero strength included) must move by exactly U dt per step under both
  schemes.  A corrector without its factor 1/2 moves it twice as far.
* order of accuracy: a co-rotating vortex pair beside a Kelvin-constrained
  cylinder, integrated over a fixed time with dt, dt/2, dt/4.  The
  differences between successive refinements fall by ~4 for Heun (second
  order) and ~2 for Euler (first order).  A corrector that uses u(X_pred)
  alone, or u(X) alone, or a midpoint predictor, is first order and fails.

Both run through `body_step` and `multibody_step`.
"""
import math

import numpy as np
import pytest

from oracle import step as OS
from oracle import vic
from oracle.lgf import lgf_table
from paper_2102_11910_gb300 import inputs


def _grid(n, dx):
    g = inputs.centred_grid(n, n, dx)
    return vic.Grid(g.nx, g.ny, g.dx, g.x0, g.y0), lgf_table(n + 1, n + 1)


def _advance(fn, grid, tab, kin, state, dt, nsteps, scheme):
    for _ in range(nsteps):
        if fn == "single":
            OS.body_step(grid, tab, kin, state, dt, scheme)
        else:
            OS.multibody_step(grid, tab, [kin], state, dt, scheme)
    return state


def _new_state(fn, X, Y, G, n_edges):
    st = OS.BodyState() if fn == "single" else OS.MultiBodyState(1, n_edges)
    st.X, st.Y, st.G = np.array(X, float), np.array(Y, float), np.array(G, float)
    return st


@pytest.mark.parametrize("fn", ["single", "multi"])
@pytest.mark.parametrize("scheme", ["euler", "rk2"])
def test_uniform_stream_translates_vortices_exactly(fn, scheme):
    grid, tab = _grid(64, 0.03)
    U, V, dt, n = 0.8, 0.3, 0.02, 3
    # plate along the free stream: alpha = -atan2(V, U) turns the chord onto (U, V)
    kin = OS.Kinematics(20, 0.6, -math.atan2(V, U), Uinf=U, Vinf=V)
    X0, Y0 = [-0.5, 0.2, 0.1], [0.4, -0.45, 0.35]
    st = _new_state(fn, X0, Y0, [0.0, 0.0, 0.0], 2)
    _advance(fn, grid, tab, kin, st, dt, n, scheme)
    # three tracers and two releases per step, all of zero strength
    assert len(st.X) == 3 + 2 * n
    assert np.abs(st.G).max() < 1e-12
    T = n * dt
    assert np.abs(st.X[:3] - (np.array(X0) + U * T)).max() < 1e-12
    assert np.abs(st.Y[:3] - (np.array(Y0) + V * T)).max() < 1e-12
    assert np.all(np.isfinite(st.X)) and np.all(np.isfinite(st.Y))


def _pair_run(fn, scheme, nsteps, T=0.16):
    grid, tab = _grid(56, 0.04)
    cyl = inputs.circle(24, 0.14, 0.62, -0.05)
    kin = OS.Kinematics(len(cyl.x), 1.0, 0.0, Uinf=0.3, Vinf=0.0, body=(cyl.x, cyl.y, cyl.ds, ()))
    st = _new_state(fn, [-0.2, 0.1], [0.05, -0.1], [1.0, 0.7], 0)
    _advance(fn, grid, tab, kin, st, T / nsteps, nsteps, scheme)
    return np.concatenate([st.X, st.Y])


@pytest.mark.parametrize("fn", ["single", "multi"])
def test_heun_is_second_order_and_euler_first_order(fn):
    r = {}
    for scheme in ("rk2", "euler"):
        a, b, c = (_pair_run(fn, scheme, n) for n in (4, 8, 16))
        e1, e2 = np.abs(a - b).max(), np.abs(b - c).max()
        r[scheme] = e1 / e2
        assert e2 > 1e-9          # the trajectories do depend on dt
    assert 3.3 < r["rk2"] < 4.8, r
    assert 1.7 < r["euler"] < 2.4, r
