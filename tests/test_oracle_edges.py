"""Pins of the generalized edge condition (Sec. 2.5, Eq. twovortex-gen) in the oracle.

fmin = fmax = 0 must reproduce the Kutta solves of Sec. 2.4; bounds wide
enough to contain both intermediate edge values must shed nothing and leave
the Kelvin-constrained sheet of Eq. circsystem (bound circulation -Gamma_w);
an active edge must end exactly at its bound, Kelvin must hold in every case,
and the split form must agree with a dense solve of the full system.
"""
import numpy as np
import pytest

from oracle import body as B
from oracle import vic
from oracle.lgf import lgf_table
from paper_2102_11910_gb300 import inputs


@pytest.fixture(scope="module")
def case():
    wl = inputs.plate_vortices_128()
    s = wl["grid"]
    g = vic.Grid(s.nx, s.ny, s.dx, s.x0, s.y0)
    b = wl["body"]
    tab = lgf_table(g.nx + 1, g.ny + 1)
    st = B.SurfaceStencil(g, b.x, b.y)
    S = B.schur_matrix(g, st, b.ds, tab)
    sch = B.Schur(S, b.ds)
    w = vic.regularize(g, wl["X"], wl["Y"], wl["G"])
    EinvLw = -B.interp_surface(st, vic.streamfunction(g, w, tab))
    sbp = B.sb_prime(b.x, b.y, 0.0, 0.0, 0.0, wl["Uinf"], 0.0)
    X1 = np.array([b.x[0] - 0.06, b.x[-1] + 0.06])
    Y1 = np.array([b.y[0] + 0.03, b.y[-1] - 0.03])
    E = B.EinvL_unit_vortex(g, st, X1, Y1, tab)
    fts = B.intermediate_sheet(sch, sbp, EinvLw)
    return dict(b=b, S=S, sch=sch, EinvLw=EinvLw, sbp=sbp, E=E, Gw=vic.circulation(g, w), fts=fts,
                tol=1e-15 * np.linalg.cond(S) * 100)


def _kelvin(c, f, G):
    return c["sch"].circ(f) + np.sum(G) + c["Gw"]


def test_zero_bounds_are_the_kutta_condition(case):
    c = case
    k1, k2 = c["b"].edges
    f, ft, s0, G = B.sheet_edge_shed(c["sch"], c["sbp"], c["EinvLw"], (k1, k2), (c["E"][:, 0], c["E"][:, 1]),
                                     c["Gw"], ((0.0, 0.0), (0.0, 0.0)))
    fk, ftk, s0k, G1, G2 = B.sheet_kutta_shed2(c["sch"], c["sbp"], c["EinvLw"], k1, k2, c["E"][:, 0], c["E"][:, 1],
                                               c["Gw"])
    assert np.abs(f - fk).max() < c["tol"] * np.abs(fk).max()
    assert abs(G[0] - G1) < c["tol"] * abs(G1) and abs(G[1] - G2) < c["tol"] * abs(G2)
    # one edge with zero bounds is the one-vortex Kutta system of Eq. kuttasystem2
    f1, ft1, s01, Gs = B.sheet_edge_shed(c["sch"], c["sbp"], c["EinvLw"], (k2,), (c["E"][:, 1],), c["Gw"],
                                         ((0.0, 0.0),))
    ref = B.sheet_kutta_shed1(c["sch"], c["sbp"], c["EinvLw"], k2, c["E"][:, 1], c["Gw"])
    assert np.abs(f1 - ref[0]).max() < c["tol"] * np.abs(ref[0]).max() and abs(Gs[0] - ref[3]) < c["tol"] * abs(ref[3])


def test_inactive_edges_shed_nothing_and_leave_the_kelvin_sheet(case):
    c = case
    k1, k2 = c["b"].edges
    wide = ((c["fts"][k1] - 1.0, c["fts"][k1] + 1.0), (c["fts"][k2] - 1.0, c["fts"][k2] + 1.0))
    f, ft, s0, G = B.sheet_edge_shed(c["sch"], c["sbp"], c["EinvLw"], (k1, k2), (c["E"][:, 0], c["E"][:, 1]),
                                     c["Gw"], wide)
    assert G[0] == 0.0 and G[1] == 0.0
    ref, _ = B.sheet_circulation(c["sch"], c["sbp"], c["EinvLw"], -c["Gw"])
    assert np.abs(f - ref).max() < c["tol"] * np.abs(ref).max()
    assert abs(_kelvin(c, f, G)) < c["tol"] * abs(c["Gw"])


def test_active_edge_ends_at_its_bound(case):
    c = case
    k1, k2 = c["b"].edges
    v1, v2 = c["fts"][k1], c["fts"][k2]
    # edge 1 above its range (ends at fmax), edge 2 inside
    bounds = ((v1 - 2.0 * abs(v1), v1 - 0.5 * abs(v1)), (v2 - 1.0, v2 + 1.0))
    f, ft, s0, G = B.sheet_edge_shed(c["sch"], c["sbp"], c["EinvLw"], (k1, k2), (c["E"][:, 0], c["E"][:, 1]),
                                     c["Gw"], bounds)
    assert G[1] == 0.0 and G[0] != 0.0
    assert abs(ft[k1] - bounds[0][1]) < c["tol"] * abs(bounds[0][1])
    assert abs(_kelvin(c, f, G)) < c["tol"] * np.abs(G).max()


def test_two_active_edges_match_the_dense_system(case):
    c = case
    k1, k2 = c["b"].edges
    v1, v2 = c["fts"][k1], c["fts"][k2]
    t1, t2 = 0.4 * v1, 0.25 * v2                     # both edges outside [0, 0.4 v] / [0, 0.25 v]
    bounds = tuple(sorted((0.0, t)) for t in (t1, t2))
    f, ft, s0, G = B.sheet_edge_shed(c["sch"], c["sbp"], c["EinvLw"], (k1, k2), (c["E"][:, 0], c["E"][:, 1]),
                                     c["Gw"], bounds)
    sch = c["sch"]
    fm, ftm, s0m, G1m, G2m = B.sheet_edge_shed2_monolithic(c["S"], sch.f0, sch.f0hat, sch.P_Gamma(c["sbp"]),
                                                           c["EinvLw"], k1, k2, c["E"][:, 0], c["E"][:, 1],
                                                           c["Gw"], t1, t2)
    assert np.abs(f - fm).max() < c["tol"] * np.abs(fm).max()
    assert abs(G[0] - G1m) < c["tol"] * abs(G1m) and abs(G[1] - G2m) < c["tol"] * abs(G2m)
    assert abs(ft[k1] - t1) < c["tol"] * abs(t1) and abs(ft[k2] - t2) < c["tol"] * abs(t2)
