"""GPU impulse diagnostics (Sec. 2.6.2, Eqs. linimpxd, linimpyd, angimpd) against the oracle.

The GPU reduction is checked on the same inputs as the oracle: the node
vorticity the GPU regularized (copied back) and the sheet strength the GPU
solved; separately, the body-free result is checked against the point-vortex
impulse it must equal, and the ellipse's translation impulse against its
added mass.
"""
import math

import numpy as np
import pytest
import torch

import paper_2102_11910_gb300 as pf
from oracle import vic as OV
from oracle.diagnostics import impulse
from paper_2102_11910_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol", [(pf.PF_FP64, 1e-12), (pf.PF_MIXED, 1e-6)])
def test_body_free_impulse(prec, tol):
    g = inputs.GridSpec(300, 200, 0.01, -1.7, -0.9)
    plan = pf.Plan(g.nx, g.ny, g.dx, g.x0, g.y0, prec)
    rng = np.random.default_rng(17)
    X, Y, G = inputs.uniform_vortices(rng, 20000, -1.6, 1.2, 1e-3, -0.85, 0.95)
    w = pf.pf_regularize(plan, *(torch.from_numpy(a).cuda() for a in (X, Y, G)))
    P = pf.pf_impulse(plan, w)
    og = OV.Grid(g.nx, g.ny, g.dx, g.x0, g.y0)
    ref = impulse(og, w.double().cpu().numpy())            # oracle on the GPU's own w
    # rows are summed in the grid's precision: FP32 rounding for the mixed path
    assert np.abs(P - ref).max() < (1e-13 if prec == pf.PF_FP64 else 1e-6) * np.abs(ref).max()
    exact = np.array([np.sum(G * Y), -np.sum(G * X), -0.5 * np.sum(G * (X * X + Y * Y))])
    assert np.abs(P - exact).max() < tol * np.abs(exact).max()
    assert np.array_equal(P, pf.pf_impulse(plan, w))       # fixed summation order


def test_translating_ellipse_impulse_is_its_added_mass():
    a, b, dx = 1.0, 0.5, 0.02
    per = math.pi * (3 * (a + b) - math.sqrt((3 * a + b) * (a + 3 * b)))
    ns = int(round(per / (2 * dx)))
    n = int(2.6 * a / dx) + 8
    g = inputs.centred_grid(n, n, dx)
    plan = pf.Plan(g.nx, g.ny, g.dx, g.x0, g.y0, pf.PF_FP64)
    e = inputs.ellipse(ns, a, b)
    nx, ny = e.x / a ** 2, e.y / b ** 2
    nn = np.hypot(nx, ny)
    nx, ny = nx / nn, ny / nn
    sch = pf.pf_schur_factor(plan, e.x, e.y, e.ds)
    w = torch.zeros((g.ny, g.nx), dtype=torch.float64, device="cuda")
    og = OV.Grid(g.nx, g.ny, g.dx, g.x0, g.y0)
    for U, V, k, exact in ((1.0, 0.0, 0, math.pi * b * b), (0.0, 1.0, 1, math.pi * a * a)):
        f, _, _ = pf.pf_sheet_solve(plan, sch, w, (U, V, 0.0, 0.0, 0.0), pf.PF_SHEET_CIRCULATION, 0.0)
        P = pf.pf_impulse(plan, w, e.x, e.y, e.ds, f, nx, ny, motion=(U, V, 0.0))
        ref = impulse(og, np.zeros((g.ny, g.nx)), e.x, e.y, e.ds, f.cpu().numpy(), nx, ny, U, V, 0.0)
        assert np.abs(P - ref).max() < 1e-12 * np.abs(ref).max()
        assert abs(P[k] - exact) < 0.08 * exact          # first-order error at dx = 0.02 (~0.07 / 0.02)


def test_impulse_rejects_bad_arguments():
    plan = pf.Plan(64, 64, 0.05, -1.6, -1.6, pf.PF_MIXED)
    w = torch.zeros((64, 64), dtype=torch.float32, device="cuda")
    x = np.zeros(8)
    with pytest.raises(pf.GridPfError):
        pf.pf_impulse(plan, w, x, x, x + 0.1, None)       # surface without a sheet strength
