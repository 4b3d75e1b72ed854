"""Pins of the oracle's shedding and stepping (Sec. 2.4.2-2.4.3)."""
import math

import numpy as np

from oracle import step as T
from oracle import vic
from oracle.lgf import lgf_table
from paper_2102_11910_gb300 import inputs


def _setup(n=72, dx=0.025, ns=24, amp=0.0):
    g = inputs.centred_grid(n, n, dx)
    grid = vic.Grid(g.nx, g.ny, g.dx, g.x0, g.y0)
    kin = T.Kinematics(ns, 1.0, math.radians(30.0), amp=amp, omega=1.0, Uinf=1.0)
    return grid, lgf_table(n + 1, n + 1), kin


def test_placement_rule():
    """First vortex 10 dt U from the edge along the normal facing the free
    stream; later vortices 1/3 of the way from the edge to the last one."""
    xs, ys, ds, (k1, k2) = T.Kinematics(20, 1.0, math.radians(30.0)).surface(0.0)
    ex, ey = T.edge_point(xs, ys, k2)
    assert abs(math.hypot(ex, ey) - 0.5) < 1e-14           # edge is the plate tip
    p = T.new_vortex_position(xs, ys, k2, None, 0.01, 1.0, 0.0)
    assert abs(math.hypot(p[0] - ex, p[1] - ey) - 0.1) < 1e-14
    tx, ty = xs[k2] - xs[k2 - 1], ys[k2] - ys[k2 - 1]
    assert abs((p[0] - ex) * tx + (p[1] - ey) * ty) < 1e-14   # along the normal
    assert p[0] - ex > 0.0                                  # towards the free stream
    q = T.new_vortex_position(xs, ys, k2, (1.3, -0.7), 0.01, 1.0, 0.0)
    assert abs(q[0] - (ex + (1.3 - ex) / 3)) < 1e-14 and abs(q[1] - (ey + (-0.7 - ey) / 3)) < 1e-14


def test_euler_steps_conserve_circulation_and_satisfy_kutta():
    grid, tab, kin = _setup()
    st = T.BodyState()
    for _ in range(3):
        info = T.body_step(grid, tab, kin, st, 0.02, "euler")
        # Kelvin: bound + all free vortices (including the two new ones) = 0
        assert abs(info["circ_f"] + st.G.sum()) < 1e-12
        ft = info["f"] / info["sch"].f0
        assert abs(ft[0]) < 1e-10 and abs(ft[-1]) < 1e-10
    assert len(st.X) == 6
    # the starting vortices have the expected sense for a plate at positive incidence:
    # trailing-edge vortex counter-clockwise (positive), leading-edge clockwise (negative)
    assert st.G[1] > 0 and st.G[0] < 0


def test_rk2_second_stage_enforces_kelvin():
    grid, tab, kin = _setup(amp=math.radians(10.0))
    st = T.BodyState()
    T.body_step(grid, tab, kin, st, 0.02, "rk2")
    T.body_step(grid, tab, kin, st, 0.02, "rk2")
    assert len(st.X) == 4 and np.all(np.isfinite(st.X))
    assert abs(st.t - 0.04) < 1e-15
