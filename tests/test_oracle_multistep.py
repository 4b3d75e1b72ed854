"""Pins of the oracle's several-body time step (Sec. 2.7 with the stepping
rules of Sec. 2.4.2-2.4.3): one body reproduces the single-body step, Kelvin
holds per body at every stage, and two mirrored plates shed a mirrored wake."""
import math

import numpy as np
import pytest

from oracle import step as OS
from oracle import vic
from oracle.lgf import lgf_table
from paper_2102_11910_gb300 import inputs


@pytest.fixture(scope="module")
def grid72():
    g = inputs.centred_grid(72, 72, 0.025)
    return vic.Grid(g.nx, g.ny, g.dx, g.x0, g.y0), lgf_table(73, 73)


@pytest.mark.parametrize("scheme,amp", [("euler", 0.0), ("rk2", 10.0)])
def test_one_body_is_the_single_body_step(grid72, scheme, amp):
    og, tab = grid72
    kin = OS.Kinematics(24, 1.0, math.radians(30.0), amp=math.radians(amp), omega=1.0, Uinf=1.0)
    a, m = OS.BodyState(), OS.MultiBodyState(1, 2)
    for _ in range(3):
        OS.body_step(og, tab, kin, a, 0.02, scheme)
        OS.multibody_step(og, tab, [kin], m, 0.02, scheme)
    assert len(m.X) == 6
    assert np.abs(m.X - a.X).max() < 1e-12 and np.abs(m.Y - a.Y).max() < 1e-12
    assert np.abs(m.G - a.G).max() < 1e-10 * np.abs(a.G).max()


def _static(x, y, ds, edges, Uinf=1.0):
    """A body at rest whose frame is the world frame (alpha = 0)."""
    return OS.Kinematics(len(x), 1.0, 0.0, Uinf=Uinf, body=(x, y, ds, edges))


def test_mirrored_plates_shed_a_mirrored_wake(grid72):
    og, tab = grid72
    a = inputs.plate(16, 0.5, math.radians(20.0), -0.3, 0.3)
    b = inputs.plate(16, 0.5, math.radians(-20.0), -0.3, -0.3)
    kins = [_static(a.x, a.y, a.ds, a.edges), _static(b.x, b.y, b.ds, b.edges)]
    m = OS.MultiBodyState(2, 4)
    for _ in range(3):
        info = OS.multibody_step(og, tab, kins, m, 0.02, "euler")
        assert abs(info["s0"][0] + info["s0"][1]) < 1e-9 * abs(info["s0"][0])
    X, Y, G = m.X.reshape(3, 4), m.Y.reshape(3, 4), m.G.reshape(3, 4)   # per step: A LE, A TE, B LE, B TE
    assert np.abs(X[:, 2:] - X[:, :2]).max() < 1e-10
    assert np.abs(Y[:, 2:] + Y[:, :2]).max() < 1e-10
    assert np.abs(G[:, 2:] + G[:, :2]).max() < 1e-9 * np.abs(G).max()
    assert np.abs(G).min() > 1e-4


def test_kelvin_per_body_at_every_stage(grid72):
    og, tab = grid72
    a = inputs.plate(16, 0.5, math.radians(25.0), -0.35, 0.25)
    e = inputs.ellipse(30, 0.2, 0.08, 0.35, -0.2)
    kins = [_static(a.x, a.y, a.ds, a.edges), _static(e.x, e.y, e.ds, ())]
    rng = np.random.default_rng(11)
    m = OS.MultiBodyState(2, 2)
    m.X, m.Y, m.G = rng.uniform(-0.8, -0.6, 20), rng.uniform(-0.8, 0.8, 20), rng.normal(0, 0.02, 20)
    total0 = float(np.sum(m.G))
    for _ in range(3):
        n0 = len(m.G)
        info = OS.multibody_step(og, tab, kins, m, 0.02, "euler")
        new = m.G[n0:]
        # the ellipse sheds nothing and keeps zero bound circulation (it has released nothing)
        assert abs(info["circ_b"][1]) < 1e-11
        # the plate balances the free vortices and everything it released, new ones included
        assert abs(info["circ_b"][0] + info["Gws"][0] + np.sum(new)) < 1e-11
        assert abs(info["Gws"][0] - (total0 + np.sum(m.G[20:n0]))) < 1e-12
