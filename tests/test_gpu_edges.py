"""GPU generalized edge condition (Sec. 2.5, Eq. twovortex-gen) against the oracle.

The plate of the single-step workload (128^2, 64 points, 256 vortices); the
same vorticity field on both sides (the plan's w, rounded to its precision,
copied back).  Bounds are placed relative to the oracle's intermediate edge
values with wide margins, so both sides classify the edges alike.
"""
import math

import numpy as np
import pytest
import torch

import paper_2102_11910_gb300 as pf
from oracle import body as OB
from oracle import step as OS
from oracle import vic as OV
from oracle.lgf import lgf_table
from paper_2102_11910_gb300 import inputs

pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def case():
    wl = inputs.plate_vortices_128()
    gs = wl["grid"]
    g = OV.Grid(gs.nx, gs.ny, gs.dx, gs.x0, gs.y0)
    b = wl["body"]
    tab = lgf_table(g.nx + 1, g.ny + 1)
    st = OB.SurfaceStencil(g, b.x, b.y)
    S = OB.schur_matrix(g, st, b.ds, tab)
    sch = OB.Schur(S, b.ds)
    X1 = np.array([b.x[0] - 0.06, b.x[-1] + 0.06])
    Y1 = np.array([b.y[0] + 0.03, b.y[-1] - 0.03])
    return dict(wl=wl, gs=gs, g=g, b=b, tab=tab, st=st, S=S, sch=sch, X1=X1, Y1=Y1,
                E=OB.EinvL_unit_vortex(g, st, X1, Y1, tab), cond=np.linalg.cond(S))


def _bounds(kind, v1, v2):
    if kind == "kutta":
        return ((0.0, 0.0), (0.0, 0.0))
    if kind == "inactive":
        return ((v1 - 1.0, v1 + 1.0), (v2 - 1.0, v2 + 1.0))
    if kind == "one":          # edge 0 above its range, edge 1 inside
        return (tuple(sorted((v1 - 2.0 * abs(v1), v1 - 0.5 * abs(v1)))), (v2 - 1.0, v2 + 1.0))
    return (tuple(sorted((0.0, 0.4 * v1))), tuple(sorted((0.0, 0.25 * v2))))      # both active, nonzero targets


@pytest.mark.parametrize("kind", ["kutta", "inactive", "one", "both"])
@pytest.mark.parametrize("prec", [pf.PF_FP64, pf.PF_MIXED])
def test_edge_bounded_sheet_matches_oracle(case, prec, kind):
    c = case
    gs, b = c["gs"], c["b"]
    plan = pf.Plan(gs.nx, gs.ny, gs.dx, gs.x0, gs.y0, prec)
    schur = pf.pf_schur_factor(plan, b.x, b.y, b.ds)
    wl = c["wl"]
    w_dev = pf.pf_regularize(plan, *(torch.from_numpy(a).cuda() for a in (wl["X"], wl["Y"], wl["G"])))
    pf.pf_sync(plan)
    w = w_dev.double().cpu().numpy()
    Gw = OV.circulation(c["g"], w)
    motion = (0.0, 0.0, 0.0, wl["Uinf"], 0.0)
    sbp = OB.sb_prime(b.x, b.y, *motion)
    EinvLw = -OB.interp_surface(c["st"], OV.streamfunction(c["g"], w, c["tab"]))
    fts = OB.intermediate_sheet(c["sch"], sbp, EinvLw)
    k1, k2 = b.edges
    bd = _bounds(kind, fts[k1], fts[k2])
    f_ref, ft_ref, s0_ref, G_ref = OB.sheet_edge_shed(c["sch"], sbp, EinvLw, (k1, k2), (c["E"][:, 0], c["E"][:, 1]),
                                                      Gw, bd)
    f, G, s0 = pf.pf_sheet_solve_edges(plan, schur, w_dev, motion, Gw, [k1, k2], bd, c["X1"], c["Y1"])
    tol = c["cond"] * 1e-15
    assert rel(f.cpu().numpy(), f_ref) < tol
    assert abs(s0 - s0_ref) < tol * max(1.0, abs(s0_ref))
    for a, r in zip(G, G_ref):
        assert (a == 0.0) == (r == 0.0)                  # the same edges shed
        if r != 0.0:
            assert abs(a - r) < tol * abs(r)
    if kind == "kutta":                                  # zero bounds: bitwise the Kutta solve
        fk, Gk, s0k = pf.pf_sheet_solve(plan, schur, w_dev, motion, pf.PF_SHEET_KUTTA_SHED, Gw, [k1, k2],
                                        c["X1"], c["Y1"])
        assert torch.equal(f, fk) and G == Gk and s0 == s0k


@pytest.mark.parametrize("prec", [pf.PF_FP64, pf.PF_MIXED])
def test_leading_edge_bounded_shedding_steps_match_oracle(prec):
    """Plate at 30 deg in a stream; trailing edge under Kutta, leading edge under a
    suction bound wide enough that it sheds nothing: the oracle's teacher-free
    steps (three) and the GPU's agree, and the leading-edge vortices are zero."""
    n, dx = 72, 0.025
    g = inputs.centred_grid(n, n, dx)
    plan = pf.Plan(g.nx, g.ny, g.dx, g.x0, g.y0, prec)
    og = OV.Grid(g.nx, g.ny, g.dx, g.x0, g.y0)
    tab = lgf_table(n + 1, n + 1)
    ns, dt, nsteps = 24, 0.02, 3
    bounds = ((-50.0, 50.0), (0.0, 0.0))
    kin = OS.Kinematics(ns, 1.0, math.radians(30.0), Uinf=1.0, edge_bounds=bounds)
    ost = OS.BodyState()
    state = pf.State(plan, 64)
    pf.pf_state_set(state, np.zeros(0), np.zeros(0), np.zeros(0), 0.0)
    xi = -1.0 + (2.0 * np.arange(1, ns + 1) - 1.0) / ns
    body = pf.BodyKinematics(0.5 * xi, np.zeros(ns), np.full(ns, 1.0 / ns), (0, ns - 1), math.radians(30.0),
                             Uinf=1.0, edge_bounds=bounds)
    for _ in range(nsteps):
        OS.body_step(og, tab, kin, ost, dt, "euler")
        pf.pf_step(plan, state, dt, body)
    pf.pf_sync(plan)
    X, Y, G, t = pf.pf_state_get(state)
    assert len(X) == 2 * nsteps
    assert np.all(G[0::2] == 0.0) and np.all(ost.G[0::2] == 0.0)     # leading edge (point 0) sheds nothing
    tg = 1e-9 if prec == pf.PF_FP64 else 1e-4
    tx = 1e-11 if prec == pf.PF_FP64 else 1e-6
    assert np.abs(G - ost.G).max() < tg * np.abs(ost.G).max()
    assert np.abs(X - ost.X).max() < tx and np.abs(Y - ost.Y).max() < tx
