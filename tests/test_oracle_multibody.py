"""Pins of the oracle's several-body sheet solve (Sec. 2.7, Eq. kuttasystem4).

The split form is checked against an independent dense solve of the reduced
saddle-point system, against the one-body solves it must reduce to, against
the constraint rows of Eq. kuttasystem4 on the final field, and against the
mirror symmetry of two reflected plates.
"""
import numpy as np
import pytest

from oracle import body as B
from oracle import vic
from oracle.lgf import lgf_table
from paper_2102_11910_gb300 import inputs


def _setup(wl, tab=None):
    gs = wl["grid"]
    g = vic.Grid(gs.nx, gs.ny, gs.dx, gs.x0, gs.y0)
    tab = lgf_table(g.nx + 1, g.ny + 1) if tab is None else tab
    st = B.SurfaceStencil(g, wl["x"], wl["y"])
    S = B.schur_matrix(g, st, wl["ds"], tab)
    sch = B.Schur(S, wl["ds"])
    w = vic.regularize(g, wl["X"], wl["Y"], wl["G"])
    EinvLw = -B.interp_surface(st, vic.streamfunction(g, w, tab))
    sbp = B.sb_prime(wl["x"], wl["y"], 0.0, 0.0, 0.0, wl["Uinf"], wl["Vinf"])
    E = B.EinvL_unit_vortex(g, st, wl["VX"], wl["VY"], tab)
    return dict(wl=wl, g=g, tab=tab, st=st, S=S, sch=sch, w=w, EinvLw=EinvLw, sbp=sbp, E=E,
                cond=np.linalg.cond(S))


@pytest.fixture(scope="module")
def three():
    return _setup(inputs.three_bodies_128())


def _solve(c):
    wl = c["wl"]
    return B.sheet_multibody_shed(c["sch"], c["sbp"], c["EinvLw"], wl["starts"], wl["edges"], c["E"], wl["Gamma_w"])


def test_split_and_monolithic_agree(three):
    c = three
    wl, sch = c["wl"], c["sch"]
    f, ft, s0, G = _solve(c)
    fm, ftm, s0m, Gm = B.sheet_multibody_monolithic(c["S"], sch.f0, sch.f0hat, sch.P_Gamma(c["sbp"]), c["EinvLw"],
                                                   wl["starts"], wl["edges"], c["E"], wl["Gamma_w"])
    tol = c["cond"] * 1e-13
    assert np.abs(f - fm).max() < tol * np.abs(f).max()
    assert np.abs(s0 - s0m).max() < tol * np.abs(s0).max()
    assert np.abs(G - Gm).max() < tol * np.abs(G).max()
    assert len(s0) == 3 and len(G) == 3


def test_kutta_and_per_body_kelvin(three):
    c = three
    wl = c["wl"]
    f, ft, s0, G = _solve(c)
    kk = [k for eb in wl["edges"] for k in eb]
    for k in kk:
        assert abs(ft[k]) < 1e-9 * np.abs(ft).max()
    i = 0
    for b, eb in enumerate(wl["edges"]):
        lo, hi = wl["starts"][b], wl["starts"][b + 1]
        released = sum(G[i:i + len(eb)])
        i += len(eb)
        assert abs(np.dot(wl["ds"][lo:hi], f[lo:hi]) + released + wl["Gamma_w"][b]) < 1e-11


def test_no_penetration_on_final_field(three):
    """E psi + sum_b s0_b 1_b = P^Gamma s'_b for psi = -L^{-1}(w + sum_i Gamma_i d_i + R_s f)
    (Eq. kuttasystem4, second block row)."""
    c = three
    wl, g, st = c["wl"], c["g"], c["st"]
    f, ft, s0, G = _solve(c)
    wt = c["w"] + vic.regularize(g, wl["VX"], wl["VY"], G) + B.regularize_surface(g, st, f, wl["ds"])
    psi = vic.streamfunction(g, wt, c["tab"])
    lhs = B.interp_surface(st, psi) + B.body_indicators(wl["starts"], len(f)) @ s0
    rhs = c["sch"].P_Gamma(c["sbp"])
    assert np.abs(lhs - rhs).max() < 1e-15 * c["cond"] * 100 * np.abs(rhs).max()


@pytest.fixture(scope="module")
def one():
    wl = inputs.plate_vortices_128()
    b = wl["body"]
    d = dict(grid=wl["grid"], x=b.x, y=b.y, ds=b.ds, X=wl["X"], Y=wl["Y"], G=wl["G"],
             VX=np.array([b.x[0] - 0.06, b.x[-1] + 0.06]), VY=np.array([b.y[0] + 0.03, b.y[-1] - 0.03]),
             Uinf=wl["Uinf"], Vinf=0.0)
    return _setup(d), b


def test_one_body_reduces_to_the_single_body_solves(one):
    c, b = one
    sch, sbp, EinvLw, E = c["sch"], c["sbp"], c["EinvLw"], c["E"]
    k1, k2 = b.edges
    starts = [0, len(b.x)]
    tol = c["cond"] * 1e-13
    Gw = 0.07
    f, _, s0, G = B.sheet_multibody_shed(sch, sbp, EinvLw, starts, [(k1, k2)], E, [Gw])
    fr, _, s0r, G1, G2 = B.sheet_kutta_shed2(sch, sbp, EinvLw, k1, k2, E[:, 0], E[:, 1], Gw)
    assert np.abs(f - fr).max() < tol * np.abs(fr).max()
    assert abs(s0[0] - s0r) < tol * abs(s0r) and np.abs(G - [G1, G2]).max() < tol * abs(G1)
    f, _, s0, G = B.sheet_multibody_shed(sch, sbp, EinvLw, starts, [(k2,)], E[:, 1:], [Gw])
    fr, _, s0r, G1 = B.sheet_kutta_shed1(sch, sbp, EinvLw, k2, E[:, 1], Gw)
    assert np.abs(f - fr).max() < tol * np.abs(fr).max() and abs(G[0] - G1) < tol * abs(G1)
    f, _, s0, G = B.sheet_multibody_shed(sch, sbp, EinvLw, starts, [()], E[:, :0], [-0.3])
    fr, s0r = B.sheet_circulation(sch, sbp, EinvLw, 0.3)
    assert np.abs(f - fr).max() < tol * np.abs(fr).max() and len(G) == 0


def test_mirrored_plates_are_antisymmetric():
    """Reflecting the bodies, the vortices (with their strengths negated) and
    the new-vortex positions in the x axis reflects the flow: the sheet, the
    uniform values and the new strengths change sign."""
    c = _setup(inputs.mirrored_plates_128())
    wl = c["wl"]
    f, ft, s0, G = _solve(c)
    n = 24
    tol = c["cond"] * 1e-13
    assert np.abs(f[n:] + f[:n]).max() < tol * np.abs(f).max()
    assert abs(s0[0] + s0[1]) < tol * abs(s0[0])
    assert np.abs(G[2:] + G[:2]).max() < tol * np.abs(G).max()
    assert np.abs(f).max() > 0.1 and abs(s0[0]) > 1e-3
