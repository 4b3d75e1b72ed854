"""GPU parity of the surface pressure (Sec. 2.6.1) against the FP64 oracle: the
potential jump of a sheet, the pressure jump from the immersed-boundary
Bernoulli equation, and R_s f, for a cylinder and a plate at dS/dx = 1, in
both precisions (the pressure path is FP64 given the plan's psi)."""
import math

import numpy as np
import pytest
import torch

import paper_2102_11910_gb300 as pf
from oracle import body as OB
from oracle import pressure as OP
from oracle import vic as OV
from oracle.lgf import lgf_table
from paper_2102_11910_gb300 import inputs

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def _case(kind):
    if kind == "cylinder":
        dx, R = 0.05, 1.0
        ns = int(round(2 * math.pi * R / dx))
        n = int(3.4 * R / dx) + 8
        b = inputs.circle(ns, R)
        th = 2 * math.pi * np.arange(ns) / ns
        nxs, nys = np.cos(th), np.sin(th)
        sbp_args = (0, 0, 0, 1.0, 0)
    else:
        dx, n, al = 0.02, 96, math.radians(25.0)
        b = inputs.plate(50, 1.0, al)
        nxs, nys = np.full(50, math.sin(al)), np.full(50, math.cos(al))
        sbp_args = (0, 0, 0.4, 1.0, 0)
    gs = inputs.centred_grid(n, n, dx)
    g = OV.Grid(gs.nx, gs.ny, gs.dx, gs.x0, gs.y0)
    tab = lgf_table(n + 1, n + 1)
    st = OB.SurfaceStencil(g, b.x, b.y)
    sch = OB.Schur(OB.schur_matrix(g, st, b.ds, tab), b.ds)
    f, _ = OB.sheet_circulation(sch, OB.sb_prime(b.x, b.y, *sbp_args), np.zeros(len(b.x)), 0.3)
    return dict(gs=gs, g=g, b=b, tab=tab, st=st, f=f, nxs=nxs, nys=nys,
                cw=OP.curl_weights(g, b.x, b.y, nxs, nys))


@pytest.fixture(scope="module", params=["cylinder", "plate"])
def case(request):
    return _case(request.param)


@pytest.mark.parametrize("prec", [pf.PF_FP64, pf.PF_MIXED])
def test_potential_and_pressure_jump_match_oracle(case, prec):
    c = case
    gs, b = c["gs"], c["b"]
    plan = pf.Plan(gs.nx, gs.ny, gs.dx, gs.x0, gs.y0, prec)
    schur = pf.pf_schur_factor(plan, b.x, b.y, b.ds)
    f_dev = torch.from_numpy(c["f"]).cuda()
    with pytest.raises(pf.GridPfError) as e:
        pf.pf_potential_jump(plan, schur, f_dev)
    assert e.value.name == "PF_ERR_NOT_FACTORED"
    pf.pf_pressure_setup(plan, schur, c["nxs"], c["nys"])
    dphi = pf.pf_potential_jump(plan, schur, f_dev).cpu().numpy()
    ref = OP.potential_jump(c["g"], c["st"], c["cw"], b.ds, c["f"], c["tab"])
    assert rel(dphi, ref) < 1e-10
    assert abs(np.dot(b.ds, dphi)) < 1e-10 * np.abs(dphi).max()
    # pressure jump from the streamfunction of the sheet, the plan's precision on both sides
    g = c["g"]
    psi = OV.streamfunction(g, OB.regularize_surface(g, c["st"], c["f"], b.ds), c["tab"])
    psi_dev = torch.from_numpy(psi.ravel()).to(device="cuda", dtype=plan.dtype).contiguous()
    psi_used = psi_dev.double().cpu().numpy().reshape(psi.shape)
    rng = np.random.default_rng(3)
    dphidt = rng.normal(0.0, 0.1, len(b.x))
    m = (0.2, -0.1, 0.3, 1.0, 0.0)
    dp = pf.pf_pressure_jump(plan, schur, psi_dev, m, f_dev, torch.from_numpy(dphidt).cuda(), 1.3).cpu().numpy()
    us, vs = OP.face_velocity_at_surface(g, b.x, b.y, np.pad(psi_used, 1), m[3], m[4])
    ref = OP.pressure_jump(us, vs, b.x, b.y, c["nxs"], c["nys"], c["f"], m[0], m[1], m[2], dphidt, rho=1.3)
    assert rel(dp, ref) < 1e-12


@pytest.mark.parametrize("prec", [pf.PF_FP64, pf.PF_MIXED])
def test_sheet_regularize_matches_oracle(case, prec):
    c = case
    gs, b = c["gs"], c["b"]
    plan = pf.Plan(gs.nx, gs.ny, gs.dx, gs.x0, gs.y0, prec)
    schur = pf.pf_schur_factor(plan, b.x, b.y, b.ds)
    w = torch.zeros(gs.nx * gs.ny, dtype=plan.dtype, device="cuda")
    pf.pf_sheet_regularize(plan, schur, torch.from_numpy(c["f"]).cuda(), w)
    ref = OB.regularize_surface(c["g"], c["st"], c["f"], b.ds).ravel()
    assert rel(w.double().cpu().numpy(), ref) < (1e-13 if prec == pf.PF_FP64 else 1e-6)


@pytest.mark.parametrize("prec", [pf.PF_FP64, pf.PF_MIXED])
def test_pressure_field_matches_oracle(case, prec):
    """Eq. pgrid at the cell centres, with the surface terms of a body in motion
    (a given sheet, a given dDelta phi/dt) and free vorticity around it."""
    c = case
    gs, b, g = c["gs"], c["b"], c["g"]
    plan = pf.Plan(gs.nx, gs.ny, gs.dx, gs.x0, gs.y0, prec)
    schur = pf.pf_schur_factor(plan, b.x, b.y, b.ds)
    pf.pf_pressure_setup(plan, schur, c["nxs"], c["nys"])
    rng = np.random.default_rng(9)
    X, Y, G = rng.uniform(g.x0 + 0.25 * (g.nx - 1) * g.dx, g.x0 + 0.4 * (g.nx - 1) * g.dx, 30), \
        rng.uniform(g.y0 + 0.3 * (g.ny - 1) * g.dx, g.y0 + 0.7 * (g.ny - 1) * g.dx, 30), rng.normal(0, 0.05, 30)
    w = OV.regularize(g, X, Y, G)
    psi = OV.streamfunction(g, w + OB.regularize_surface(g, c["st"], c["f"], b.ds), c["tab"])
    to_dev = lambda a: torch.from_numpy(a.ravel()).to(device="cuda", dtype=plan.dtype).contiguous()
    psi_d, w_d = to_dev(psi), to_dev(w)
    psi_u, w_u = psi_d.double().cpu().numpy().reshape(psi.shape), w_d.double().cpu().numpy().reshape(w.shape)
    dphidt = rng.normal(0.0, 0.2, len(b.x))
    m = (0.2, -0.1, 0.3, 1.0, 0.0)
    p = pf.pf_pressure_field(plan, psi_d, w_d, m, schur, torch.from_numpy(c["f"]).cuda(),
                             torch.from_numpy(dphidt).cuda(), 1.2).cpu().numpy()
    u, v = OP.face_velocities(g, psi_u, m[3], m[4])
    qx, qy = OP.surface_faces(g, b.x, b.y, c["nxs"], c["nys"], b.ds, dphidt, c["f"], m[0], m[1], m[2])
    ref = OP.pressure_field(g, c["tab"], u, v, w_u, qx, qy, rho=1.2)
    tol = 1e-11 if prec == pf.PF_FP64 else 1e-5
    assert np.abs(p - ref).max() < tol * np.abs(ref).max()
    # without a body: the free-vortex terms alone
    p0 = pf.pf_pressure_field(plan, psi_d, w_d, m).cpu().numpy()
    ref0 = OP.pressure_field(g, c["tab"], u, v, w_u, np.zeros_like(u), np.zeros_like(v), rho=1.0)
    assert np.abs(p0 - ref0).max() < tol * np.abs(ref0).max()
