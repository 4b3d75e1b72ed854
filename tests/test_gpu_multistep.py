"""GPU time stepping around several bodies (Sec. 2.7 with the rules of
Sec. 2.4.2-2.4.3) against the oracle, from identical initial states for a
few steps, as the single-body stepping tests."""
import math

import numpy as np
import pytest

import paper_2102_11910_gb300 as pf
from oracle import step as OS
from oracle import vic as OV
from oracle.lgf import lgf_table
from paper_2102_11910_gb300 import inputs

pytestmark = pytest.mark.gpu


def _setup(prec, n=72, dx=0.025):
    g = inputs.centred_grid(n, n, dx)
    return pf.Plan(g.nx, g.ny, g.dx, g.x0, g.y0, prec), OV.Grid(g.nx, g.ny, g.dx, g.x0, g.y0), lgf_table(n + 1, n + 1)


def _bodies(kind, amp):
    """(oracle kinematics, GPU kinematics) of the bodies, in their own frames."""
    xi = inputs.plate_xi(16)
    if kind == "plate+ellipse":
        e = inputs.ellipse(30, 0.2, 0.08, 0.3, -0.25)
        specs = [(0.25 * xi - 0.3, np.full(16, 0.3), np.full(16, 0.5 / 16), (0, 15), 0.35, amp, 2.0),
                 (e.x, e.y, e.ds, (), 0.0, 0.0, 0.0)]
    else:        # two plates releasing at one edge each
        specs = [(0.25 * xi - 0.3, np.full(16, 0.3), np.full(16, 0.5 / 16), (15,), 0.3, amp, 2.0),
                 (0.25 * xi - 0.3, np.full(16, -0.3), np.full(16, 0.5 / 16), (15,), -0.3, 0.0, 0.0)]
    ok = [OS.Kinematics(len(x), 1.0, a0, amp=am, omega=om, Uinf=1.0, body=(x, y, d, ed))
          for x, y, d, ed, a0, am, om in specs]
    gk = [pf.BodyKinematics(x, y, d, ed, a0, am, om, 1.0) for x, y, d, ed, a0, am, om in specs]
    return ok, gk


@pytest.mark.parametrize("kind", ["plate+ellipse", "two one-edge plates"])
@pytest.mark.parametrize("prec,scheme,amp", [(pf.PF_FP64, "euler", 0.0), (pf.PF_FP64, "rk2", 0.1),
                                             (pf.PF_MIXED, "euler", 0.0), (pf.PF_MIXED, "rk2", 0.1)])
def test_several_bodies_step_matches_oracle(kind, prec, scheme, amp):
    plan, og, tab = _setup(prec)
    ok, gk = _bodies(kind, amp)
    n_edges = sum(len(k.edges) for k in ok)
    rng = np.random.default_rng(21)
    X0, Y0, G0 = rng.uniform(-0.85, -0.65, 20), rng.uniform(-0.8, 0.8, 20), rng.normal(0, 0.02, 20)
    ost = OS.MultiBodyState(2, n_edges)
    ost.X, ost.Y, ost.G = X0.copy(), Y0.copy(), G0.copy()
    state = pf.State(plan, 64)
    pf.pf_state_set(state, X0, Y0, G0, 0.0)
    nsteps, dt = 3, 0.02
    for _ in range(nsteps):
        OS.multibody_step(og, tab, ok, ost, dt, scheme)
        pf.pf_step_multi(plan, state, dt, gk, scheme=0 if scheme == "euler" else 1)
    pf.pf_sync(plan)
    X, Y, G, t = pf.pf_state_get(state)
    assert len(X) == 20 + n_edges * nsteps and abs(t - nsteps * dt) < 1e-14
    tg = 1e-9 if prec == pf.PF_FP64 else 1e-4
    tx = 1e-11 if prec == pf.PF_FP64 else 1e-6
    assert np.abs(G - ost.G).max() < tg * np.abs(ost.G[20:]).max()
    assert np.abs(X - ost.X).max() < tx and np.abs(Y - ost.Y).max() < tx


def test_one_body_matches_the_single_body_step():
    plan, og, tab = _setup(pf.PF_FP64)
    k = pf.plate_kinematics(24, 1.0, math.radians(30.0), 0.1, 1.0, 1.0)
    a, b = pf.State(plan, 64), pf.State(plan, 64)
    for st in (a, b):
        pf.pf_state_set(st, np.zeros(0), np.zeros(0), np.zeros(0), 0.0)
    for _ in range(3):
        pf.pf_step(plan, a, 0.02, k, scheme=1)
        pf.pf_step_multi(plan, b, 0.02, [k], scheme=1)
    Xa, Ya, Ga, _ = pf.pf_state_get(a)
    Xb, Yb, Gb, _ = pf.pf_state_get(b)
    assert np.abs(Ga - Gb).max() < 1e-9 * np.abs(Ga).max()
    assert np.abs(Xa - Xb).max() < 1e-11 and np.abs(Ya - Yb).max() < 1e-11


def test_invalid_bodies_are_rejected():
    plan, _, _ = _setup(pf.PF_FP64)
    st = pf.State(plan, 8)
    pf.pf_state_set(st, np.zeros(0), np.zeros(0), np.zeros(0), 0.0)
    ok = pf.plate_kinematics(16, 0.5, 0.3, Uinf=1.0)
    bounded = pf.BodyKinematics(ok.xb, ok.yb + 0.3, ok.ds, (0, 15), 0.3, Uinf=1.0, edge_bounds=((-1, 1), (-1, 1)))
    with pytest.raises(pf.GridPfError) as e:
        pf.pf_step_multi(plan, st, 0.02, [ok, bounded])
    assert e.value.name == "PF_ERR_ARG"
    with pytest.raises(pf.GridPfError) as e:        # 2 bodies x 2 edges x 3 steps > 8
        for _ in range(3):
            pf.pf_step_multi(plan, st, 0.02, [ok, pf.BodyKinematics(ok.xb, ok.yb - 0.3, ok.ds, (0, 15), -0.3, Uinf=1.0)])
    assert e.value.name == "PF_ERR_CAPACITY"
