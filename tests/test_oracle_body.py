"""Pins of the oracle's surface / Schur / constraint algebra (Sec. 2.2-2.4).

Identities the paper states are checked to rounding; closed-form potential
flows (Figs. 3, 4, 5, 7) are checked at the accuracy of the first-order
immersed-boundary discretisation, with convergence where the paper reports it.
"""
import math

import numpy as np
import pytest

from oracle import body as B
from oracle import vic
from oracle.lgf import lgf_table
from paper_2102_11910_gb300 import inputs


def _g(spec):
    return vic.Grid(spec.nx, spec.ny, spec.dx, spec.x0, spec.y0)


@pytest.fixture(scope="module")
def plate_case():
    wl = inputs.plate_vortices_128()
    g = _g(wl["grid"])
    b = wl["body"]
    tab = lgf_table(g.nx + 1, g.ny + 1)
    st = B.SurfaceStencil(g, b.x, b.y)
    S = B.schur_matrix(g, st, b.ds, tab)
    sch = B.Schur(S, b.ds)
    w = vic.regularize(g, wl["X"], wl["Y"], wl["G"])
    psi = vic.streamfunction(g, w, tab)
    EinvLw = -B.interp_surface(st, psi)
    sbp = B.sb_prime(b.x, b.y, 0.0, 0.0, 0.0, wl["Uinf"], 0.0)
    X1 = np.array([b.x[0] - 0.06, b.x[-1] + 0.06])
    Y1 = np.array([b.y[0] + 0.03, b.y[-1] - 0.03])
    E = B.EinvL_unit_vortex(g, st, X1, Y1, tab)
    return dict(g=g, b=b, tab=tab, st=st, S=S, sch=sch, w=w, EinvLw=EinvLw, sbp=sbp,
                X1=X1, Y1=Y1, E=E, Gw=vic.circulation(g, w), wl=wl)


def test_schur_symmetric_and_matches_operator_definition(plate_case):
    """S = -E L^{-1} R_s: symmetric for uniform dS (Sec. 2.2.2); column q equals
    -E_s applied to the direct-sum L^{-1} of R_s e_q."""
    c = plate_case
    S = c["S"]
    assert np.abs(S - S.T).max() < 1e-14 * np.abs(S).max()
    q = 17
    e = np.zeros(len(c["b"].x)); e[q] = 1.0
    col = -B.interp_surface(c["st"], vic.inv_laplacian(c["g"], B.regularize_surface(c["g"], c["st"], e, c["b"].ds), c["tab"]))
    assert np.abs(col - S[:, q]).max() < 1e-13 * np.abs(S[:, q]).max()


def test_f0_identities(plate_case):
    """Stilde 1 = 1 (Eq. Son1); f0hat^T P^Gamma s = 0 (Eq. circrem); Gamma0 = <1, f0>."""
    sch = plate_case["sch"]
    Stilde = sch.S * sch.f0[None, :]
    assert np.abs(Stilde @ sch.ones - 1.0).max() < 1e-9
    s = np.random.default_rng(0).normal(size=len(sch.f0))
    assert abs(np.dot(sch.f0hat, sch.P_Gamma(s))) < 1e-12 * np.abs(s).sum() * np.abs(sch.f0hat).max()
    assert abs(sch.Gamma0 - sch.circ(sch.f0)) < 1e-14 * abs(sch.Gamma0)


def test_two_edge_kutta_constraints(plate_case):
    """Kutta at both edges, Kelvin, and equal edge values g_k1 = g_k2 = s0 (Eqs. kuttasystem3, kuttadiff)."""
    c = plate_case
    sch, (k1, k2), E = c["sch"], c["b"].edges, c["E"]
    f, ft, s0, G1, G2 = B.sheet_kutta_shed2(sch, c["sbp"], c["EinvLw"], k1, k2, E[:, 0], E[:, 1], c["Gw"])
    assert abs(ft[k1]) < 1e-12 and abs(ft[k2]) < 1e-12
    assert abs(sch.circ(f) + G1 + G2 + c["Gw"]) < 1e-12
    fts = B.intermediate_sheet(sch, c["sbp"], c["EinvLw"])
    g = fts + G1 * sch.solve_tilde(E[:, 0]) + G2 * sch.solve_tilde(E[:, 1])
    assert abs(g[k1] - s0) < 1e-10 * max(1, abs(s0)) and abs(g[k2] - s0) < 1e-10 * max(1, abs(s0))


def test_split_unsplit_and_monolithic_agree(plate_case):
    """Eq. twovortex (split), Eq. schurkutta2 (3x3) and the dense (Ns+3) system agree."""
    c = plate_case
    sch, (k1, k2), E = c["sch"], c["b"].edges, c["E"]
    a = B.sheet_kutta_shed2(sch, c["sbp"], c["EinvLw"], k1, k2, E[:, 0], E[:, 1], c["Gw"])
    b3 = B.sheet_kutta_shed2_schur3(sch, c["sbp"], c["EinvLw"], k1, k2, E[:, 0], E[:, 1], c["Gw"])
    m = B.sheet_kutta_shed2_monolithic(sch.S, sch.f0, sch.f0hat, sch.P_Gamma(c["sbp"]), c["EinvLw"],
                                       k1, k2, E[:, 0], E[:, 1], c["Gw"])
    cond = np.linalg.cond(sch.S)
    for other in (b3, m):
        for x, y in zip(a, other):
            x, y = np.atleast_1d(x), np.atleast_1d(y)
            assert np.abs(x - y).max() <= 1e-15 * cond * np.abs(x).max() * 50


def test_no_penetration_on_final_field(plate_case):
    """E psi + s0 1 = P^Gamma s'_b for psi = -L^{-1}(w + G1 d1 + G2 d2 + R_s f) (Eq. kuttasystem3, row 2)."""
    c = plate_case
    g, sch, st, (k1, k2), E = c["g"], c["sch"], c["st"], c["b"].edges, c["E"]
    f, ft, s0, G1, G2 = B.sheet_kutta_shed2(sch, c["sbp"], c["EinvLw"], k1, k2, E[:, 0], E[:, 1], c["Gw"])
    wt = c["w"] + vic.regularize(g, c["X1"], c["Y1"], np.array([G1, G2])) + B.regularize_surface(g, st, f, c["b"].ds)
    psi = vic.streamfunction(g, wt, c["tab"])
    lhs = B.interp_surface(st, psi) + s0
    rhs = sch.P_Gamma(c["sbp"])
    assert np.abs(lhs - rhs).max() < 1e-15 * np.linalg.cond(sch.S) * 100 * np.abs(rhs).max()


def test_given_s0_sheet_satisfies_no_penetration(plate_case):
    """Basic system with s0 prescribed (Eqs. basicblock, vsheet): the sheet f of
    sheet_given_s0 makes the total field obey the no-penetration row
    E psi + s0 1 = s'_b, psi = -L^{-1}(w + R_s f) by direct summation, for
    several s0 (a wrong sign on E L^{-1} w or on s0 fails here)."""
    c = plate_case
    g, sch, st = c["g"], c["sch"], c["st"]
    for s0 in (0.0, 0.37, -1.2):
        f = B.sheet_given_s0(sch, c["sbp"], c["EinvLw"], s0)
        psi = vic.streamfunction(g, c["w"] + B.regularize_surface(g, st, f, c["b"].ds), c["tab"])
        lhs = B.interp_surface(st, psi) + s0
        scale = np.abs(c["sbp"]).max() + abs(s0) + np.abs(c["EinvLw"]).max()
        assert np.abs(lhs - c["sbp"]).max() < 1e-15 * np.linalg.cond(sch.S) * 100 * scale


def test_given_s0_reproduces_the_circulation_solve(plate_case):
    """With s0 set to the multiplier the circulation-constrained solve returns
    (Eq. circsystem), the basic system gives that solve's sheet."""
    c = plate_case
    sch = c["sch"]
    f_c, s0 = B.sheet_circulation(sch, c["sbp"], c["EinvLw"], 0.25)
    f = B.sheet_given_s0(sch, c["sbp"], c["EinvLw"], s0)
    assert abs(sch.circ(f) - 0.25) < 1e-9
    assert np.abs(f - f_c).max() < 1e-15 * np.linalg.cond(sch.S) * 100 * np.abs(f_c).max()


def test_lgf_constant_does_not_change_constrained_solutions(plate_case):
    """Adding a constant to G (the homogeneous part the paper leaves free) leaves
    f, Gamma1, Gamma2 of the Kutta solve unchanged and shifts only s0."""
    c = plate_case
    g, st, b = c["g"], c["st"], c["b"]
    tab2 = c["tab"] + 0.37
    S2 = B.schur_matrix(g, st, b.ds, tab2)
    sch2 = B.Schur(S2, b.ds)
    # E L^{-1} w under the shifted kernel: L^{-1} w gains dx^2 * 0.37 * sum(w)
    EinvLw2 = c["EinvLw"] + g.dx ** 2 * 0.37 * np.sum(c["w"])
    E2 = B.EinvL_unit_vortex(g, st, c["X1"], c["Y1"], tab2)
    k1, k2 = b.edges
    a = B.sheet_kutta_shed2(c["sch"], c["sbp"], c["EinvLw"], k1, k2, c["E"][:, 0], c["E"][:, 1], c["Gw"])
    z = B.sheet_kutta_shed2(sch2, c["sbp"], EinvLw2, k1, k2, E2[:, 0], E2[:, 1], c["Gw"])
    tol = 1e-15 * np.linalg.cond(c["S"]) * 100
    assert np.abs(a[0] - z[0]).max() < tol * np.abs(a[0]).max()
    assert abs(a[3] - z[3]) < tol * abs(a[3]) and abs(a[4] - z[4]) < tol * abs(a[4])


# ------------------------------------------------------- closed-form flows
def _cylinder(R, dx, ratio=2.0, extent=3.4):
    ns = int(round(2 * math.pi * R / (ratio * dx)))
    n = int(extent * R / dx) + 8
    g = _g(inputs.centred_grid(n, n, dx))
    b = inputs.circle(ns, R)
    tab = lgf_table(n + 1, n + 1)
    st = B.SurfaceStencil(g, b.x, b.y)
    sch = B.Schur(B.schur_matrix(g, st, b.ds, tab), b.ds)
    th = 2 * math.pi * np.arange(ns) / ns
    return g, b, tab, st, sch, th


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_translating_cylinder():
    """Fig. 4: cylinder translating at U: gamma = 2 U sin(theta)  (dx/R = 0.03, dS/dx = 2)."""
    g, b, tab, st, sch, th = _cylinder(1.0, 0.03)
    f, _ = B.sheet_circulation(sch, B.sb_prime(b.x, b.y, 1.0, 0, 0, 0, 0), np.zeros(len(th)), 0.0)
    assert _rel(f, 2 * np.sin(th)) < 0.03


def test_cylinder_uniform_flow_with_circulation():
    """gamma = -2 U sin(theta) + Gamma/(2 pi R) (Sec. 2.3, classical)."""
    g, b, tab, st, sch, th = _cylinder(1.0, 0.03)
    f, _ = B.sheet_circulation(sch, B.sb_prime(b.x, b.y, 0, 0, 0, 1.0, 0), np.zeros(len(th)), 1.0)
    assert _rel(f, -2 * np.sin(th) + 1.0 / (2 * math.pi)) < 0.03
    assert abs(sch.circ(f) - 1.0) < 1e-12


def test_vortex_near_cylinder():
    """Fig. 3: vortex Gamma_v at (3R/2, 0), bound circulation -Gamma_v."""
    g, b, tab, st, sch, th = _cylinder(1.0, 0.03)
    w = vic.regularize(g, np.array([1.5]), np.array([0.0]), np.array([1.0]))
    EinvLw = -B.interp_surface(st, vic.streamfunction(g, w, tab))
    f, _ = B.sheet_circulation(sch, np.zeros(len(th)), EinvLw, -1.0)
    ex = -(1.0 / (2 * math.pi)) * (1.5 ** 2 - 1) / (1.5 ** 2 + 1 - 3.0 * np.cos(th))
    assert _rel(f, ex) < 0.05


def test_circle_f0_uniform():
    """Fig. 5: for a circle the sheet of a uniform unit streamfunction is uniform."""
    g, b, tab, st, sch, th = _cylinder(1.0, 0.05, ratio=3.0)
    assert np.std(sch.f0) < 1e-2 * abs(np.mean(sch.f0))


def test_steady_kutta_plate_first_order():
    """Fig. 7: Gamma0 ftilde -> -pi c U sin(alpha)(1 - xi), error ~ dx; Gamma_b -> -pi c U sin(alpha)."""
    errs = []
    al = math.radians(30.0)
    for dx in (0.04, 0.02, 0.01):
        ns = int(round(1.0 / (2 * dx)))
        n = int(1.3 / dx) + 8
        g = _g(inputs.centred_grid(n, n, dx))
        b = inputs.plate(ns, 1.0, al)
        tab = lgf_table(n + 1, n + 1)
        st = B.SurfaceStencil(g, b.x, b.y)
        sch = B.Schur(B.schur_matrix(g, st, b.ds, tab), b.ds)
        f, ft, s0 = B.sheet_kutta_steady(sch, B.sb_prime(b.x, b.y, 0, 0, 0, 1.0, 0), np.zeros(ns), b.edges[1])
        ex = -math.pi * math.sin(al) * (1 - inputs.plate_xi(ns))
        errs.append(_rel(sch.Gamma0 * ft, ex))
        assert abs(ft[b.edges[1]]) < 1e-13
        assert abs(sch.circ(f) + math.pi * math.sin(al)) < 0.03
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(0.8 < r < 1.4 for r in rates), (errs, rates)
