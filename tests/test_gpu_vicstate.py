"""The tile-ordered vortex state (body-free vortex-in-cell, forward Euler;
Sec. 2.1 operators and the Sec. 2.4.2 advection rule) against the oracle.

A step of the state is R_v, the node velocity and E_v at the vortices, then
X += dt u.  Parity is per step from the state's own positions (teacher
forced): the oracle evaluates the velocity at the positions the state holds
and the state's next positions must be those plus dt u.
"""
import numpy as np
import pytest
import torch

import paper_2102_11910_gb300 as pf
from oracle import vic as OV
from oracle.lgf import lgf_table
from paper_2102_11910_gb300 import inputs

pytestmark = pytest.mark.gpu

# mixed: velocity 1e-5 relative (the path's tolerance); positions hold a
# 24-bit fraction of a cell, so a move is exact to ~2^-24 dx
TOL_U = {pf.PF_FP64: 1e-12, pf.PF_MIXED: 1e-5}


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _case(prec, nx=100, ny=77, nv=3000, seed=5, dx=0.02, variance=1e-3):
    g = inputs.GridSpec(nx, ny, dx, -0.5 * (nx - 1) * dx, -0.4 * (ny - 1) * dx)
    rng = np.random.default_rng(seed)
    X, Y, G = inputs.uniform_vortices(rng, nv, g.x0 + 6 * dx, g.x0 + (nx - 8) * dx, variance,
                                      g.y0 + 6 * dx, g.y0 + (ny - 8) * dx)
    plan = pf.Plan(g.nx, g.ny, g.dx, g.x0, g.y0, prec)
    return g, plan, X, Y, G


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.mark.parametrize("prec", [pf.PF_FP64, pf.PF_MIXED])
def test_set_and_get_round_trip(prec):
    g, plan, X, Y, G = _case(prec)
    st = pf.VicState(plan, 4000)
    pf.pf_vic_state_set(st, _dev(X), _dev(Y), _dev(G))
    Xg, Yg, Gg, nv, t = pf.pf_vic_state_get(st)
    pf.pf_sync(plan)
    assert nv == len(X) and t == 0.0
    tol = 1e-12 * g.dx if prec == pf.PF_FP64 else 2.0 ** -23 * g.dx
    assert np.abs(Xg.cpu().numpy() - X).max() <= tol and np.abs(Yg.cpu().numpy() - Y).max() <= tol
    gt = 0.0 if prec == pf.PF_FP64 else 1e-7
    assert np.abs(Gg.cpu().numpy() - G).max() <= gt * np.abs(G).max()


@pytest.mark.parametrize("prec", [pf.PF_FP64, pf.PF_MIXED])
def test_steps_match_oracle_teacher_forced(prec):
    g, plan, X, Y, G = _case(prec)
    og = OV.Grid(g.nx, g.ny, g.dx, g.x0, g.y0)
    tab = lgf_table(g.nx + 1, g.ny + 1)
    st = pf.VicState(plan, 4000)
    pf.pf_vic_state_set(st, _dev(X), _dev(Y), _dev(G))
    dt, U, V = 0.01, 0.3, -0.1
    dtype = torch.float64 if prec == pf.PF_FP64 else torch.float32
    uq = torch.empty(len(X), dtype=dtype, device="cuda")
    vq = torch.empty_like(uq)
    for k in range(3):
        Xs, Ys, Gs, _, _ = pf.pf_vic_state_get(st)
        Xs, Ys, Gs = (a.cpu().numpy() for a in (Xs, Ys, Gs))
        _, _, ur, vr = OV.vortex_velocity(og, Xs, Ys, Gs, U, V, tab)
        pf.pf_vic_step(st, dt, U, V, uq, vq)
        Xn, Yn, _, nv, t = pf.pf_vic_state_get(st)
        pf.pf_sync(plan)
        assert nv == len(X) and abs(t - (k + 1) * dt) < 1e-15
        assert _rel(np.concatenate([uq.double().cpu().numpy(), vq.double().cpu().numpy()]),
                    np.concatenate([ur, vr])) < TOL_U[prec]
        # the move: exact in FP64; mixed positions are cell + 24-bit fraction,
        # moved in fixed point and rounded to nearest
        tx = 1e-13 if prec == pf.PF_FP64 else 2.0 ** -23 * g.dx + dt * 1e-5 * np.abs(ur).max()
        assert np.abs(Xn.cpu().numpy() - (Xs + dt * uq.double().cpu().numpy())).max() <= tx
        assert np.abs(Yn.cpu().numpy() - (Ys + dt * vq.double().cpu().numpy())).max() <= tx


@pytest.mark.parametrize("prec", [pf.PF_FP64, pf.PF_MIXED])
def test_step_velocity_equals_the_stateless_step(prec):
    """The state's velocity output and pf_vic_velocity on the state's positions
    evaluate the same operators (1100 x 700 nodes: ragged tiles at two edges,
    2e5 vortices)."""
    g = inputs.centred_grid(1100, 700, 2.0 / 1099)
    rng = np.random.default_rng(8)
    X, Y, G = inputs.uniform_vortices(rng, 200000, -0.9, 0.9, 1e-4, -0.55, 0.55)
    plan = pf.Plan(g.nx, g.ny, g.dx, g.x0, g.y0, prec)
    st = pf.VicState(plan, 200000)
    pf.pf_vic_state_set(st, _dev(X), _dev(Y), _dev(G))
    dtype = torch.float64 if prec == pf.PF_FP64 else torch.float32
    for _ in range(2):
        Xs, Ys, Gs, _, _ = pf.pf_vic_state_get(st)
        u0, v0 = pf.pf_vic_velocity(plan, Xs, Ys, Gs, 0.2, 0.0)
        u0, v0 = u0.clone(), v0.clone()
        uq = torch.empty(len(X), dtype=dtype, device="cuda")
        vq = torch.empty_like(uq)
        pf.pf_vic_step(st, 2e-3, 0.2, 0.0, uq, vq)
        pf.pf_sync(plan)
        tol = 1e-12 if prec == pf.PF_FP64 else 1e-6
        assert _rel(torch.cat([uq, vq]).double().cpu().numpy(), torch.cat([u0, v0]).double().cpu().numpy()) < tol
    _, _, Gs, nv, _ = pf.pf_vic_state_get(st)
    pf.pf_sync(plan)
    assert nv == len(X)
    held = G if prec == pf.PF_FP64 else G.astype(np.float32).astype(np.float64)
    assert abs(float(Gs.sum()) - float(held.sum())) < 1e-9     # strengths ride along unchanged


def test_state_is_bitwise_reproducible():
    g, plan, X, Y, G = _case(pf.PF_MIXED, nv=20000, variance=1e-6)
    out = []
    for _ in range(2):
        st = pf.VicState(plan, 20000)
        pf.pf_vic_state_set(st, _dev(X), _dev(Y), _dev(G))
        for _ in range(5):
            pf.pf_vic_step(st, 0.01, 0.4, 0.1)
        Xg, Yg, _, _, _ = pf.pf_vic_state_get(st)
        pf.pf_sync(plan)
        out.append((Xg.clone(), Yg.clone()))
        st.close()
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])


def test_vortex_leaving_the_grid_is_dropped_and_reported():
    g, plan, X, Y, G = _case(pf.PF_MIXED, nv=50)
    X = X.copy()
    X[7] = g.x0 + (g.nx - 4.2) * g.dx        # one cell from the right edge's limit
    st = pf.VicState(plan, 64)
    pf.pf_vic_state_set(st, _dev(X), _dev(Y), _dev(G))
    pf.pf_sync(plan)
    pf.pf_vic_step(st, 0.02, 3.0, 0.0)            # 3 cells per step to the right
    with pytest.raises(pf.GridPfError) as e:
        pf.pf_sync(plan)
    assert e.value.name == "PF_ERR_OUT_OF_DOMAIN"
    Xg, _, _, nv, _ = pf.pf_vic_state_get(st)
    pf.pf_sync(plan)
    assert nv == 49 and np.isnan(Xg[7].item())


def test_too_fast_a_move_is_dropped_and_reported():
    g, plan, X, Y, G = _case(pf.PF_MIXED, nx=256, ny=64, nv=20)
    X = np.full(20, g.x0 + 20.5 * g.dx)
    st = pf.VicState(plan, 64)
    pf.pf_vic_state_set(st, _dev(X), _dev(Y), _dev(G))
    pf.pf_sync(plan)
    pf.pf_vic_step(st, 1.0, 70 * g.dx, 0.0)          # 70 cells: two tiles in one step
    with pytest.raises(pf.GridPfError) as e:
        pf.pf_sync(plan)
    assert e.value.name == "PF_ERR_CAPACITY"
