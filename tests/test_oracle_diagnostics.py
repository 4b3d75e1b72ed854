"""Pins of the impulse oracle (Sec. 2.6.2, Eqs. linimpxd, linimpyd, angimpd).

Body-free: M4' reproduces polynomials up to degree two (zero first and second
moments), so the node terms equal the point-vortex impulses exactly:
P = (sum Gamma Y, -sum Gamma X), Pi_O = -1/2 sum Gamma (X^2 + Y^2).
With a body: the impulse of unit translation is the added mass (Sec. 2.6.3),
which for an ellipse of semi-axes a (along x) and b is pi b^2 for motion
along x and pi a^2 along y (classical); the discrete values converge to it at
first order in dx.
"""
import math

import numpy as np
import pytest

from oracle import body as B
from oracle import vic
from oracle.diagnostics import impulse
from oracle.kernels import m4prime
from oracle.lgf import lgf_table
from paper_2102_11910_gb300 import inputs


def test_m4prime_reproduces_quadratics():
    k = np.arange(-3, 5)
    for x in np.linspace(0.0, 0.999, 37):
        wt = m4prime(k - x)
        for p in range(3):
            assert abs(np.sum(wt * (k - x) ** p) - (1.0 if p == 0 else 0.0)) < 1e-14


def test_body_free_impulse_is_the_point_vortex_impulse():
    g = vic.Grid(70, 53, 0.05, -1.7, -1.2)
    rng = np.random.default_rng(11)
    X, Y, G = rng.uniform(-1.5, 1.6, 200), rng.uniform(-1.0, 1.3, 200), rng.normal(0, 1, 200)
    w = vic.regularize(g, X, Y, G)
    P = impulse(g, w)
    ref = np.array([np.sum(G * Y), -np.sum(G * X), -0.5 * np.sum(G * (X * X + Y * Y))])
    assert np.abs(P - ref).max() < 1e-12 * np.abs(ref).max()


def _ellipse(a, b, dx, ratio=2.0):
    per = math.pi * (3 * (a + b) - math.sqrt((3 * a + b) * (a + 3 * b)))
    ns = int(round(per / (ratio * dx)))
    n = int(2.6 * max(a, b) / dx) + 8
    g = vic.Grid(n, n, dx, -0.5 * (n - 1) * dx, -0.5 * (n - 1) * dx)
    e = inputs.ellipse(ns, a, b)
    tab = lgf_table(n + 1, n + 1)
    st = B.SurfaceStencil(g, e.x, e.y)
    sch = B.Schur(B.schur_matrix(g, st, e.ds, tab), e.ds)
    nx, ny = e.x / a ** 2, e.y / b ** 2          # outward normals of the ellipse
    nn = np.hypot(nx, ny)
    return g, e, sch, nx / nn, ny / nn


def _translation_impulse(g, e, sch, nx, ny, U, V):
    sbp = B.sb_prime(e.x, e.y, U, V, 0.0, 0.0, 0.0)
    f, _ = B.sheet_circulation(sch, sbp, np.zeros(len(e.x)), 0.0)
    return impulse(g, np.zeros((g.ny, g.nx)), e.x, e.y, e.ds, f, nx, ny, U, V, 0.0)


@pytest.mark.parametrize("a,b", [(1.0, 1.0), (1.0, 0.5)])
def test_added_mass_of_translation_converges_first_order(a, b):
    errs = {"x": [], "y": []}
    for dx in (0.08, 0.04):
        g, e, sch, nx, ny = _ellipse(a, b, dx)
        Px = _translation_impulse(g, e, sch, nx, ny, 1.0, 0.0)
        Py = _translation_impulse(g, e, sch, nx, ny, 0.0, 1.0)
        errs["x"].append(abs(Px[0] - math.pi * b * b) / (math.pi * b * b))
        errs["y"].append(abs(Py[1] - math.pi * a * a) / (math.pi * a * a))
        # symmetry of the ellipse about both axes: no cross impulse, no angular
        # impulse (to the accuracy of the numerically placed equal-arc points)
        for P, main in ((Px, Px[0]), (Py, Py[1])):
            assert sorted(np.abs(P))[:2][-1] < 1e-5 * abs(main)
    for k in ("x", "y"):
        assert errs[k][1] < 0.15
        assert 1.7 < errs[k][0] / errs[k][1] < 2.4, errs
