"""GPU time stepping (shedding and advection, Sec. 2.4.2-2.4.3) against the oracle.

Multi-step parity is checked from identical initial states for a few steps;
vortex dynamics amplify differences exponentially, so longer runs are checked
through invariants elsewhere.
"""
import math

import numpy as np
import pytest
import torch

import paper_2102_11910_gb300 as pf
from oracle import step as OS
from oracle import vic as OV
from oracle.lgf import lgf_table
from paper_2102_11910_gb300 import inputs

pytestmark = pytest.mark.gpu


def _setup(prec, n=72, dx=0.025):
    g = inputs.centred_grid(n, n, dx)
    return g, pf.Plan(g.nx, g.ny, g.dx, g.x0, g.y0, prec), OV.Grid(g.nx, g.ny, g.dx, g.x0, g.y0), lgf_table(n + 1, n + 1)


@pytest.mark.parametrize("prec,scheme,amp", [(pf.PF_FP64, "euler", 0.0), (pf.PF_FP64, "rk2", 10.0),
                                             (pf.PF_MIXED, "euler", 0.0), (pf.PF_MIXED, "rk2", 10.0)])
def test_plate_shedding_steps_match_oracle(prec, scheme, amp):
    g, plan, og, tab = _setup(prec)
    ns, dt, nsteps = 24, 0.02, 3
    kin = OS.Kinematics(ns, 1.0, math.radians(30.0), amp=math.radians(amp), omega=1.0, Uinf=1.0)
    ost = OS.BodyState()
    state = pf.State(plan, 64)
    pf.pf_state_set(state, np.zeros(0), np.zeros(0), np.zeros(0), 0.0)
    for _ in range(nsteps):
        OS.body_step(og, tab, kin, ost, dt, scheme)
        pf.pf_step(plan, state, dt, pf.plate_kinematics(ns, 1.0, math.radians(30.0), math.radians(amp), 1.0, 1.0),
                   scheme=0 if scheme == "euler" else 1)
    pf.pf_sync(plan)
    X, Y, G, t = pf.pf_state_get(state)
    assert len(X) == 2 * nsteps and abs(t - nsteps * dt) < 1e-14
    tg = 1e-9 if prec == pf.PF_FP64 else 1e-4
    tx = 1e-11 if prec == pf.PF_FP64 else 1e-6
    assert np.abs(G - ost.G).max() < tg * np.abs(ost.G).max()
    assert np.abs(X - ost.X).max() < tx and np.abs(Y - ost.Y).max() < tx
    # Kelvin: the released vortices carry the opposite of the bound circulation; the
    # trailing-edge vortex of a plate at positive incidence turns counter-clockwise
    assert G[1] > 0 and G[0] < 0


@pytest.mark.parametrize("prec,scheme", [(pf.PF_FP64, 0), (pf.PF_FP64, 1), (pf.PF_MIXED, 1)])
def test_pitching_ellipse_with_vortices_matches_oracle(prec, scheme):
    """Kelvin-constrained body (no edges): ellipse of aspect 3 pitching in a stream,
    with free vortices around it."""
    g, plan, og, tab = _setup(prec)
    e = inputs.ellipse(60, 0.45, 0.15)
    rng = np.random.default_rng(4)
    ang = rng.uniform(0, 2 * np.pi, 40)
    rad = rng.uniform(0.55, 0.8, 40)
    X, Y, G = rad * np.cos(ang), rad * np.sin(ang), rng.normal(0, 0.03, 40)
    kin = OS.Kinematics(60, 1.0, 0.3, amp=0.1, omega=2.0, Uinf=1.0, body=(e.x, e.y, e.ds, ()))
    ost = OS.BodyState()
    ost.X, ost.Y, ost.G = X.copy(), Y.copy(), G.copy()
    state = pf.State(plan, 64)
    pf.pf_state_set(state, X, Y, G, 0.0)
    bk = pf.BodyKinematics(e.x, e.y, e.ds, (), 0.3, 0.1, 2.0, 1.0)
    for _ in range(2):
        OS.body_step(og, tab, kin, ost, 0.02, "euler" if scheme == 0 else "rk2")
        pf.pf_step(plan, state, 0.02, bk, scheme=scheme)
    pf.pf_sync(plan)
    Xg, Yg, Gg, t = pf.pf_state_get(state)
    assert len(Xg) == 40 and np.array_equal(Gg, G)
    tx = 1e-11 if prec == pf.PF_FP64 else 1e-6
    assert np.abs(Xg - ost.X).max() < tx and np.abs(Yg - ost.Y).max() < tx


@pytest.mark.parametrize("prec,scheme", [(pf.PF_FP64, 0), (pf.PF_MIXED, 1)])
def test_body_free_step_matches_oracle(prec, scheme):
    g, plan, og, tab = _setup(prec, n=64, dx=2.0 / 63)
    rng = np.random.default_rng(9)
    X, Y, G = inputs.uniform_vortices(rng, 200, -0.6, 0.6, 1e-3)
    dt = 0.05
    state = pf.State(plan, 256)
    pf.pf_state_set(state, X, Y, G, 0.0)
    pf.pf_step(plan, state, dt, pf.no_body(0.2), scheme=scheme)
    pf.pf_sync(plan)
    Xg, Yg, Gg, t = pf.pf_state_get(state)
    _, _, u1, v1 = OV.vortex_velocity(og, X, Y, G, 0.2, 0.0, tab)
    if scheme == 0:
        Xr, Yr = X + dt * u1, Y + dt * v1
    else:
        _, _, u2, v2 = OV.vortex_velocity(og, X + dt * u1, Y + dt * v1, G, 0.2, 0.0, tab)
        Xr, Yr = X + 0.5 * dt * (u1 + u2), Y + 0.5 * dt * (v1 + v2)
    tol = 1e-13 if prec == pf.PF_FP64 else 1e-7
    assert np.abs(Xg - Xr).max() < tol and np.abs(Yg - Yr).max() < tol
    assert np.array_equal(Gg, G)


def test_step_capacity_is_enforced():
    g, plan, og, tab = _setup(pf.PF_MIXED, n=64)
    state = pf.State(plan, 3)
    pf.pf_state_set(state, np.zeros(2), np.zeros(2), np.zeros(2), 0.0)
    with pytest.raises(pf.GridPfError) as e:
        pf.pf_step(plan, state, 0.01, pf.plate_kinematics(16, 1.0, 0.3, Uinf=1.0))
    assert e.value.name == "PF_ERR_CAPACITY"


def test_step_batch_from_host_threads_matches_single_steps(monkeypatch):
    """pf_step_batch on 20 independent 128^2 instances (enqueued from several
    host threads: the library reads CUDA_DEVICE_MAX_CONNECTIONS at each call)
    gives, instance by instance and bitwise, the states of pf_step called on
    each one alone; a batch naming one plan twice is stepped in order and
    matches too."""
    monkeypatch.setenv("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    rng = np.random.default_rng(1003)
    inst = [inputs.batched_instance(rng, shape=(128, 128)) for _ in range(20)]
    g = inst[0]["grid"]
    base = pf.Plan(g.nx, g.ny, g.dx, g.x0, g.y0, pf.PF_MIXED)

    def make():
        plans, states, bodies = [], [], []
        for r in inst:
            p = pf.pf_plan_clone(base, pf.PF_MIXED, torch.cuda.Stream())
            st = pf.State(p, len(r["X"]) + 16)
            pf.pf_state_set(st, r["X"], r["Y"], r["G"])
            b = r["body"]
            plans.append(p)
            states.append(st)
            bodies.append(pf.BodyKinematics(b["xb"], b["yb"], b["ds"], b["edges"], b["alpha0"], Uinf=r["Uinf"]))
        return plans, states, bodies

    pa, sa, ba = make()
    pb, sb, bb = make()
    for _ in range(2):
        pf.pf_step_batch(pa, sa, ba, 0.002)
        for p, st, b in zip(pb, sb, bb):
            pf.pf_step(p, st, 0.002, b)
    for p in pa + pb:
        pf.pf_sync(p)
    for s1, s2 in zip(sa, sb):
        a, b = pf.pf_state_get(s1), pf.pf_state_get(s2)
        assert len(a[0]) == len(b[0]) > 0
        for u, v in zip(a[:3], b[:3]):
            assert np.array_equal(u, v)
    # one plan named twice: two states stepped in order on it
    shared = pf.pf_plan_clone(base, pf.PF_MIXED, torch.cuda.Stream())
    sc = [pf.State(shared, len(inst[k]["X"]) + 16) for k in (0, 1)]
    for st, k in zip(sc, (0, 1)):
        pf.pf_state_set(st, inst[k]["X"], inst[k]["Y"], inst[k]["G"])
    pd, sd, bd = make()
    plans = [shared, shared] + pd[2:]
    states = sc + sd[2:]
    pf.pf_step_batch(plans, states, bd, 0.002)
    pf.pf_step_batch(plans, states, bd, 0.002)
    pf.pf_sync(shared)
    for k in (0, 1):
        a, b = pf.pf_state_get(sc[k]), pf.pf_state_get(sb[k])
        for u, v in zip(a[:3], b[:3]):
            assert np.array_equal(u, v)
