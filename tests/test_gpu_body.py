"""GPU parity of the immersed-body path (Sec. 2.2-2.4) against the FP64 oracle.

Workload: 128^2 nodes, dx = 0.02, flat plate of chord 1 at 20 deg, 64 surface
points, 256 vortices (the single-step plate case).  cond(S) is ~6e5 here
(dS/dx = 0.78 is below the 1-4 range Sec. 2.2.2 recommends), so tolerances on
the sheet scale with it: FP64 results agree to ~cond * 1e-16; the mixed path,
whose vorticity field is FP32, must stay within 1e-4 in sheet strength.
"""
import math

import numpy as np
import pytest
import torch

import paper_2102_11910_gb300 as pf
from oracle import body as OB
from oracle import vic as OV
from oracle.lgf import lgf_table
from paper_2102_11910_gb300 import inputs

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
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
    w = OV.regularize(g, wl["X"], wl["Y"], wl["G"])
    X1 = np.array([b.x[0] - 0.06, b.x[-1] + 0.06])
    Y1 = np.array([b.y[0] + 0.03, b.y[-1] - 0.03])
    return dict(wl=wl, gs=gs, g=g, b=b, tab=tab, st=st, S=S, sch=sch, w=w, X1=X1, Y1=Y1,
                E=OB.EinvL_unit_vortex(g, st, X1, Y1, tab), cond=np.linalg.cond(S))


def _oracle_sheet(c, w, mode, motion):
    """Oracle sheet for vorticity field w (FP64 numpy)."""
    g, st, b, sch = c["g"], c["st"], c["b"], c["sch"]
    EinvLw = -OB.interp_surface(st, OV.streamfunction(g, w, c["tab"]))
    U, V, Om, Ui, Vi = motion
    sbp = OB.sb_prime(b.x, b.y, U, V, Om, Ui, Vi)
    Gw = OV.circulation(g, w)
    k1, k2 = b.edges
    E = c["E"]
    if mode == "given":
        return OB.sheet_given_s0(sch, sbp, EinvLw, 0.3), 0.3, []
    if mode == "circ":
        f, s0 = OB.sheet_circulation(sch, sbp, EinvLw, -0.5)
        return f, s0, []
    if mode == "steady":
        f, ft, s0 = OB.sheet_kutta_steady(sch, sbp, EinvLw, k2)
        return f, s0, []
    if mode == "shed1":
        f, ft, s0, G1 = OB.sheet_kutta_shed1(sch, sbp, EinvLw, k2, E[:, 1], Gw)
        return f, s0, [G1]
    f, ft, s0, G1, G2 = OB.sheet_kutta_shed2(sch, sbp, EinvLw, k1, k2, E[:, 0], E[:, 1], Gw)
    return f, s0, [G1, G2]


def _gpu_sheet(c, plan, schur, w_dev, mode, motion, Gw):
    b = c["b"]
    k1, k2 = b.edges
    if mode == "given":
        return pf.pf_sheet_solve(plan, schur, w_dev, motion, pf.PF_SHEET_GIVEN_S0, 0.3)
    if mode == "circ":
        return pf.pf_sheet_solve(plan, schur, w_dev, motion, pf.PF_SHEET_CIRCULATION, -0.5)
    if mode == "steady":
        return pf.pf_sheet_solve(plan, schur, w_dev, motion, pf.PF_SHEET_KUTTA_STEADY, 0.0, [k2])
    if mode == "shed1":
        return pf.pf_sheet_solve(plan, schur, w_dev, motion, pf.PF_SHEET_KUTTA_SHED, Gw, [k2],
                                 c["X1"][1:], c["Y1"][1:])
    return pf.pf_sheet_solve(plan, schur, w_dev, motion, pf.PF_SHEET_KUTTA_SHED, Gw, [k1, k2], c["X1"], c["Y1"])


def _plan(c, prec):
    gs = c["gs"]
    return pf.Plan(gs.nx, gs.ny, gs.dx, gs.x0, gs.y0, prec)


def test_schur_factor_matches_oracle(case):
    c = case
    plan = _plan(c, pf.PF_FP64)
    schur = pf.pf_schur_factor(plan, c["b"].x, c["b"].y, c["b"].ds)
    gamma0, f0, S = pf.pf_schur_info(schur)
    assert np.abs(S - c["S"]).max() < 1e-13 * np.abs(c["S"]).max()
    tol = c["cond"] * 1e-15
    assert rel(f0, c["sch"].f0) < tol
    assert abs(gamma0 - c["sch"].Gamma0) < tol * abs(c["sch"].Gamma0)


@pytest.mark.parametrize("mode", ["given", "circ", "steady", "shed1", "shed2"])
@pytest.mark.parametrize("prec", [pf.PF_FP64, pf.PF_MIXED])
def test_sheet_solve_matches_oracle(case, prec, mode):
    """Same vorticity field on both sides (rounded to the plan's precision)."""
    c = case
    plan = _plan(c, prec)
    schur = pf.pf_schur_factor(plan, c["b"].x, c["b"].y, c["b"].ds)
    w_dev = torch.from_numpy(c["w"]).to(device="cuda", dtype=plan.dtype).contiguous()
    w_used = w_dev.double().cpu().numpy()
    motion = (0.1, -0.2, 0.3, c["wl"]["Uinf"], 0.0)
    f_ref, s0_ref, g_ref = _oracle_sheet(c, w_used, mode, motion)
    f, g, s0 = _gpu_sheet(c, plan, schur, w_dev, mode, motion, OV.circulation(c["g"], w_used))
    tol = c["cond"] * 1e-15
    assert rel(f.cpu().numpy(), f_ref) < tol
    assert abs(s0 - s0_ref) < tol * max(1.0, abs(s0_ref))
    for a, r in zip(g, g_ref):
        assert abs(a - r) < tol * abs(r)


@pytest.mark.parametrize("prec", [pf.PF_FP64, pf.PF_MIXED])
def test_two_edge_shedding_from_gpu_vorticity(case, prec):
    """End to end on the GPU (regularize + sheet) against the oracle from FP64 positions:
    sheet strength within 1e-4 (mixed) and the Kutta / Kelvin identities hold."""
    c = case
    wl = c["wl"]
    plan = _plan(c, prec)
    schur = pf.pf_schur_factor(plan, c["b"].x, c["b"].y, c["b"].ds)
    dev = [torch.from_numpy(a).cuda() for a in (wl["X"], wl["Y"], wl["G"])]
    w_dev = pf.pf_regularize(plan, *dev)
    pf.pf_sync(plan)
    Gw = float(wl["G"].sum())
    motion = (0.0, 0.0, 0.0, wl["Uinf"], 0.0)
    f, g, s0 = _gpu_sheet(c, plan, schur, w_dev, "shed2", motion, Gw)
    f_ref, s0_ref, g_ref = _oracle_sheet(c, c["w"], "shed2", motion)
    tol = 1e-4 if prec == pf.PF_MIXED else c["cond"] * 1e-15
    assert rel(f.cpu().numpy(), f_ref) < tol
    assert rel(g, g_ref) < tol
    fn = f.cpu().numpy()
    # Kelvin: bound + new + free circulation = 0 (Eq. kuttasystem3, last row)
    assert abs(np.dot(c["b"].ds, fn) + sum(g) + Gw) < 1e-9
    # Kutta: ftilde = f / f0 vanishes at both edges
    _, f0, _ = pf.pf_schur_info(schur)
    k1, k2 = c["b"].edges
    assert abs(fn[k1] / f0[k1]) < 1e-9 * np.abs(fn / f0).max() and abs(fn[k2] / f0[k2]) < 1e-9 * np.abs(fn / f0).max()


def test_out_of_grid_body_is_rejected():
    gs = inputs.centred_grid(64, 64, 0.02)
    plan = pf.Plan(gs.nx, gs.ny, gs.dx, gs.x0, gs.y0, pf.PF_FP64)
    b = inputs.plate(32, 2.0, 0.0)       # chord longer than the grid
    with pytest.raises(pf.GridPfError) as e:
        pf.pf_schur_factor(plan, b.x, b.y, b.ds)
    assert e.value.name == "PF_ERR_OUT_OF_DOMAIN"


@pytest.mark.parametrize("route", [pf.PF_RHS_FFT, pf.PF_RHS_SPARSE])
@pytest.mark.parametrize("prec", [pf.PF_FP64, pf.PF_MIXED])
def test_fft_and_sparse_routes_of_the_surface_rhs_match_the_direct_sum(prec, route):
    """E_s L^-1 w from an FFT solve (the route large grids take: FP64 passes on
    FP64 plans, double-float passes on mixed ones) or from the list of nonzero
    nodes (the route time stepping takes with few vortices) against the direct
    FP64 LGF sum over all nodes (the route pinned to the oracle above): same
    vorticity, same factor; they differ by FP64-class rounding amplified by
    cond(S)."""
    n, dx = 256, 2.0 / 255
    g = inputs.centred_grid(n, n, dx)
    b = inputs.plate(96, 1.0, 0.35)                   # dS/dx = 1.33
    rng = np.random.default_rng(5)
    X, Y, G = inputs.uniform_vortices(rng, 3000, -0.9, 0.9, 1e-3)
    keep = np.hypot(X, Y) > 0.6
    X, Y, G = X[keep], Y[keep], G[keep]
    out = {}
    for r in (pf.PF_RHS_DIRECT, route):
        plan = pf.Plan(g.nx, g.ny, g.dx, g.x0, g.y0, prec)
        pf.pf_plan_set_rhs_route(plan, r)
        schur = pf.pf_schur_factor(plan, b.x, b.y, b.ds)
        w = pf.pf_regularize(plan, *(torch.from_numpy(a).cuda() for a in (X, Y, G)))
        Gw = float(G.sum())
        f, gn, s0 = pf.pf_sheet_solve(plan, schur, w, (0.0, 0.0, 0.0, 1.0, 0.0), pf.PF_SHEET_KUTTA_SHED, Gw,
                                      list(b.edges), np.array([b.x[0] - 0.02, b.x[-1] + 0.02]),
                                      np.array([b.y[0] + 0.01, b.y[-1] - 0.01]))
        _, _, S = pf.pf_schur_info(schur)
        out[r] = (f.cpu().numpy(), np.array(gn), np.linalg.cond(S))
    fd, gd, cond = out[pf.PF_RHS_DIRECT]
    ff, gf, _ = out[route]
    tol = cond * 1e-14
    assert rel(ff, fd) < tol and rel(gf, gd) < tol


@pytest.mark.parametrize("prec", [pf.PF_FP64, pf.PF_MIXED])
def test_pitching_plate_size_sheet_matches_oracle(prec):
    """The pitching-plate configuration at full size: 768 x 512 nodes, dx 0.01,
    plate of 256 points at 30 deg (dS/dx = 0.39, cond(S) ~ 2e9), 2000 vortices
    in its wake, body rotating in the stream.  Factor (f0, Gamma0) and a
    two-edge shedding sheet against the oracle, whose E L^-1 w comes from
    direct sums at the surface stencil nodes; tolerances scale with cond(S)."""
    pw = inputs.pitching_plate_512x768()
    gs = pw["grid"]
    g = OV.Grid(gs.nx, gs.ny, gs.dx, gs.x0, gs.y0)
    b = inputs.plate(pw["ns"], pw["chord"], pw["alpha0"])
    tab = lgf_table(gs.nx + 1, gs.ny + 1)
    st = OB.SurfaceStencil(g, b.x, b.y)
    S = OB.schur_matrix(g, st, b.ds, tab)
    sch = OB.Schur(S, b.ds)
    tol = np.linalg.cond(S) * 1e-15
    rng = np.random.default_rng(31)
    X, Y, G = inputs.uniform_vortices(rng, 2000, 0.7, 3.0, 1e-3, -1.2, 1.2)
    w = OV.regularize(g, X, Y, G)
    k1, k2 = b.edges
    X1 = np.array([b.x[k1] - 3 * gs.dx, b.x[k2] + 3 * gs.dx])
    Y1 = np.array([b.y[k1] + 2 * gs.dx, b.y[k2] - 2 * gs.dx])
    E = OB.EinvL_unit_vortex(g, st, X1, Y1, tab)
    motion = (0.05, -0.1, 0.4, 1.0, 0.0)
    sbp = OB.sb_prime(b.x, b.y, *motion)
    plan = pf.Plan(gs.nx, gs.ny, gs.dx, gs.x0, gs.y0, prec)
    schur = pf.pf_schur_factor(plan, b.x, b.y, b.ds)
    gamma0, f0, _ = pf.pf_schur_info(schur)
    assert rel(f0, sch.f0) < tol
    assert abs(gamma0 - sch.Gamma0) < tol * abs(sch.Gamma0)
    w_dev = torch.from_numpy(w).to(device="cuda", dtype=plan.dtype).contiguous()
    w_used = w_dev.double().cpu().numpy()
    # E L^-1 w = -E psi, psi = -L^-1 w summed directly at the stencil nodes
    nodes, inv = np.unique(np.stack([st.NI.ravel(), st.NJ.ravel()], 1), axis=0, return_inverse=True)
    psi_nodes = -OV.inv_laplacian_at(g, w_used, nodes[:, 0], nodes[:, 1], tab)
    EinvLw = -np.sum(st.W * psi_nodes[inv.reshape(st.W.shape)], axis=1)
    Gw = OV.circulation(g, w_used)
    f_ref, _, s0_ref, G1, G2 = OB.sheet_kutta_shed2(sch, sbp, EinvLw, k1, k2, E[:, 0], E[:, 1], Gw)
    f, gam, s0 = pf.pf_sheet_solve(plan, schur, w_dev, motion, pf.PF_SHEET_KUTTA_SHED, Gw, [k1, k2], X1, Y1)
    pf.pf_sync(plan)
    assert rel(f.cpu().numpy(), f_ref) < tol
    assert abs(s0 - s0_ref) < tol * max(1.0, abs(s0_ref))
    for a, r in zip(gam, (G1, G2)):
        assert abs(a - r) < tol * abs(r)


@pytest.mark.parametrize("seed,prec", [(5, pf.PF_FP64), (8, pf.PF_MIXED)])
def test_largest_served_instance_sheet_matches_oracle(seed, prec):
    """A body at the served path's largest size: 1024^2 nodes, 1e5 vortices,
    Ns ~ 160-270 (seed 5: an ellipse under Kelvin's condition; seed 8: a plate
    shedding at both edges).  The GPU forms E L^-1 w by its FP64 FFT route at
    this size, whose rounding (~1e-15 relative) cond(S) amplifies: the
    tolerance is cond(S) 1e-14, at least 1e-11."""
    r = inputs.batched_instance(np.random.default_rng(seed), big=True)
    gs, b = r["grid"], r["body"]
    g = OV.Grid(gs.nx, gs.ny, gs.dx, gs.x0, gs.y0)
    xb, yb, ds = b["xb"], b["yb"], b["ds"]
    tab = lgf_table(gs.nx + 1, gs.ny + 1)
    st = OB.SurfaceStencil(g, xb, yb)
    S = OB.schur_matrix(g, st, ds, tab)
    sch = OB.Schur(S, ds)
    tol = max(np.linalg.cond(S) * 1e-14, 1e-11)
    w = OV.regularize(g, r["X"], r["Y"], r["G"])
    plan = pf.Plan(gs.nx, gs.ny, gs.dx, gs.x0, gs.y0, prec)
    schur = pf.pf_schur_factor(plan, xb, yb, ds)
    w_dev = torch.from_numpy(w).to(device="cuda", dtype=plan.dtype).contiguous()
    w_used = w_dev.double().cpu().numpy()
    nodes, inv = np.unique(np.stack([st.NI.ravel(), st.NJ.ravel()], 1), axis=0, return_inverse=True)
    psi_nodes = -OV.inv_laplacian_at(g, w_used, nodes[:, 0], nodes[:, 1], tab)
    EinvLw = -np.sum(st.W * psi_nodes[inv.reshape(st.W.shape)], axis=1)
    Gw = OV.circulation(g, w_used)
    motion = (0.0, 0.0, 0.2, r["Uinf"], 0.0)
    sbp = OB.sb_prime(xb, yb, *motion)
    if b["edges"]:
        k1, k2 = b["edges"]
        X1 = np.array([xb[k1] - 3 * gs.dx, xb[k2] + 3 * gs.dx])
        Y1 = np.array([yb[k1], yb[k2]])
        E = OB.EinvL_unit_vortex(g, st, X1, Y1, tab)
        f_ref, _, s0_ref, G1, G2 = OB.sheet_kutta_shed2(sch, sbp, EinvLw, k1, k2, E[:, 0], E[:, 1], Gw)
        g_ref = (G1, G2)
        f, gam, s0 = pf.pf_sheet_solve(plan, schur, w_dev, motion, pf.PF_SHEET_KUTTA_SHED, Gw, [k1, k2], X1, Y1)
    else:
        f_ref, s0_ref = OB.sheet_circulation(sch, sbp, EinvLw, -Gw)
        g_ref = ()
        f, gam, s0 = pf.pf_sheet_solve(plan, schur, w_dev, motion, pf.PF_SHEET_CIRCULATION, -Gw)
    pf.pf_sync(plan)
    assert rel(f.cpu().numpy(), f_ref) < tol
    assert abs(s0 - s0_ref) < tol * max(1.0, abs(s0_ref))
    for a, ref in zip(gam, g_ref):
        assert abs(a - ref) < tol * abs(ref)


def test_coincident_surface_points_give_a_singular_factor():
    """Two surface points at the same place give S two identical rows (Eq.
    vsheet): the factor reports PF_ERR_SINGULAR instead of returning garbage,
    and the plan stays usable."""
    g = inputs.centred_grid(96, 96, 0.02)
    plan = pf.Plan(g.nx, g.ny, g.dx, g.x0, g.y0, pf.PF_FP64)
    b = inputs.plate(32, 1.0, math.radians(20.0))
    x, y, ds = np.insert(b.x, 6, b.x[5]), np.insert(b.y, 6, b.y[5]), np.insert(b.ds, 6, b.ds[5])
    with pytest.raises(pf.GridPfError) as e:
        pf.pf_schur_factor(plan, x, y, ds)
    assert e.value.name == "PF_ERR_SINGULAR"
    schur = pf.pf_schur_factor(plan, b.x, b.y, b.ds)      # the same points without the copy factor fine
    gamma0, _, _ = pf.pf_schur_info(schur)
    assert np.isfinite(gamma0)


def test_mixed_sheet_from_positions_at_pitching_plate_size(capsys):
    """The mixed path end to end at the pitching-plate size (768 x 512, dx 0.01,
    256 points at 30 deg, dS/dx = 0.39, cond(S) ~ 2e9), from FP64 vortex
    positions, against the oracle run from the same positions: through the
    plan's FP32 field (pf_regularize, then pf_sheet_solve, as the mixed time
    step does) and through pf_sheet_solve_vortices (an FP64 right-hand side
    from the vortices).  Both meet the mixed path's 1e-4 sheet tolerance; the
    field's rounding (~1e-7 relative) is white and smoothed by L^-1, so it
    barely excites the directions S amplifies (measured: 1.3e-8 either way)."""
    pw = inputs.pitching_plate_512x768()
    gs = pw["grid"]
    g = OV.Grid(gs.nx, gs.ny, gs.dx, gs.x0, gs.y0)
    b = inputs.plate(pw["ns"], pw["chord"], pw["alpha0"])
    tab = lgf_table(gs.nx + 1, gs.ny + 1)
    st = OB.SurfaceStencil(g, b.x, b.y)
    S = OB.schur_matrix(g, st, b.ds, tab)
    sch = OB.Schur(S, b.ds)
    cond = np.linalg.cond(S)
    rng = np.random.default_rng(31)
    X, Y, G = inputs.uniform_vortices(rng, 2000, 0.7, 3.0, 1e-3, -1.2, 1.2)
    w = OV.regularize(g, X, Y, G)
    k1, k2 = b.edges
    X1 = np.array([b.x[k1] - 3 * gs.dx, b.x[k2] + 3 * gs.dx])
    Y1 = np.array([b.y[k1] + 2 * gs.dx, b.y[k2] - 2 * gs.dx])
    E = OB.EinvL_unit_vortex(g, st, X1, Y1, tab)
    motion = (0.05, -0.1, 0.4, 1.0, 0.0)
    sbp = OB.sb_prime(b.x, b.y, *motion)
    nodes, inv = np.unique(np.stack([st.NI.ravel(), st.NJ.ravel()], 1), axis=0, return_inverse=True)
    EinvLw = OV.inv_laplacian_at(g, w, nodes[:, 0], nodes[:, 1], tab)
    EinvLw = np.sum(st.W * EinvLw[inv.reshape(st.W.shape)], axis=1)
    Gw = OV.circulation(g, w)
    f_ref, _, s0_ref, G1, G2 = OB.sheet_kutta_shed2(sch, sbp, EinvLw, k1, k2, E[:, 0], E[:, 1], Gw)
    plan = pf.Plan(gs.nx, gs.ny, gs.dx, gs.x0, gs.y0, pf.PF_MIXED)
    schur = pf.pf_schur_factor(plan, b.x, b.y, b.ds)
    d = [torch.from_numpy(a).cuda() for a in (X, Y, G)]
    w32 = pf.pf_regularize(plan, *d)
    f_a, gam_a, _ = pf.pf_sheet_solve(plan, schur, w32, motion, pf.PF_SHEET_KUTTA_SHED, Gw, [k1, k2], X1, Y1)
    f_b, gam_b, s0_b = pf.pf_sheet_solve_vortices(plan, schur, *d, motion, pf.PF_SHEET_KUTTA_SHED, Gw, [k1, k2],
                                                  X1, Y1)
    pf.pf_sync(plan)
    err_a = rel(f_a.cpu().numpy(), f_ref)
    err_b = rel(f_b.cpu().numpy(), f_ref)
    eg_b = max(abs(a - r) / abs(r) for a, r in zip(gam_b, (G1, G2)))
    with capsys.disabled():
        print("\n  cond(S) %.2e; sheet error from the FP32 field %.2e, from the vortices %.2e (Gamma_new %.2e)"
              % (cond, err_a, err_b, eg_b))
    eg_a = max(abs(a - r) / abs(r) for a, r in zip(gam_a, (G1, G2)))
    assert err_a < 1e-4 and eg_a < 1e-4
    assert err_b < 1e-4 and eg_b < 1e-4
    assert abs(s0_b - s0_ref) < 1e-4 * max(1.0, abs(s0_ref))
    # and the same solve in an FP64 plan agrees with the FP64 field's route
    p64 = pf.Plan(gs.nx, gs.ny, gs.dx, gs.x0, gs.y0, pf.PF_FP64)
    s64 = pf.pf_schur_factor(p64, b.x, b.y, b.ds)
    f_c, _, _ = pf.pf_sheet_solve_vortices(p64, s64, *d, motion, pf.PF_SHEET_KUTTA_SHED, Gw, [k1, k2], X1, Y1)
    pf.pf_sync(p64)
    assert rel(f_c.cpu().numpy(), f_ref) < cond * 1e-14
