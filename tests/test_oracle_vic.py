"""Pins of the oracle's body-free operators (Sec. 2.1): R_v, L^{-1}, curl, E_v."""
import math

import numpy as np
import pytest

from oracle import vic
from oracle.lgf import lgf_table
from paper_2102_11910_gb300 import inputs


def _grid(n=40, ny=None, dx=0.05):
    ny = n if ny is None else ny
    g = inputs.centred_grid(n, ny, dx)
    return vic.Grid(g.nx, g.ny, g.dx, g.x0, g.y0)


def test_circulation_preserved():
    """<1, w>_N = sum Gamma_q (Sec. 2.1, after Eq. vortexregularization)."""
    g = _grid()
    rng = np.random.default_rng(1)
    X, Y, G = inputs.uniform_vortices(rng, 300, -0.8, 0.8, 0.01)
    w = vic.regularize(g, X, Y, G)
    assert abs(vic.circulation(g, w) - G.sum()) < 1e-13


def test_interpolation_is_transpose_of_regularization():
    """E_v = R_v^T in the node / point inner products (Sec. 2.1)."""
    g = _grid(32, 28)
    rng = np.random.default_rng(2)
    X, Y, G = inputs.uniform_vortices(rng, 50, -0.6, 0.6, 1.0)
    h = rng.normal(size=(g.ny, g.nx))
    lhs = np.dot(vic.interpolate(g, h, X, Y), G)
    rhs = g.dx ** 2 * np.sum(h * vic.regularize(g, X, Y, G))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_interpolation_reproduces_linear_fields():
    g = _grid()
    rng = np.random.default_rng(3)
    X, Y, _ = inputs.uniform_vortices(rng, 100, -0.8, 0.8, 1.0)
    xx, yy = np.meshgrid(g.node_x(), g.node_y())
    field = 0.3 + 1.7 * xx - 2.2 * yy
    assert np.abs(vic.interpolate(g, field, X, Y) - (0.3 + 1.7 * X - 2.2 * Y)).max() < 1e-13


def test_out_of_domain_raises():
    g = _grid(16)
    with pytest.raises(ValueError):
        vic.regularize(g, np.array([g.x0 + 0.5 * g.dx]), np.array([0.0]), np.array([1.0]))


def test_poisson_residual_and_unit_impulse():
    """L0 psi = -dx^2 w at every node, and L applied to L^{-1} of a unit node
    impulse reproduces the impulse."""
    g = _grid(36, 30)
    rng = np.random.default_rng(4)
    X, Y, G = inputs.uniform_vortices(rng, 60, -0.6, 0.6, 0.01)
    w = vic.regularize(g, X, Y, G)
    tab = lgf_table(g.nx + 1, g.ny + 1)
    psi1 = vic.streamfunction(g, w, tab, pad=1)
    res = vic.laplacian_unit(psi1) + g.dx ** 2 * w
    assert np.abs(res).max() < 1e-14 * max(1.0, np.abs(psi1).max())
    imp = np.zeros((g.ny, g.nx)); imp[7, 11] = 1.0
    s = vic.inv_laplacian(g, imp, tab, pad=1)
    back = vic.laplacian_unit(s) / g.dx ** 2
    assert np.abs(back - imp).max() < 1e-12


def test_sampled_direct_sum_matches_field():
    g = _grid(24, 20)
    rng = np.random.default_rng(5)
    w = rng.normal(size=(g.ny, g.nx))
    tab = lgf_table(g.nx + 1, g.ny + 1)
    full = vic.inv_laplacian(g, w, tab)
    ti, tj = np.array([0, 23, 7]), np.array([0, 19, 11])
    assert np.allclose(vic.inv_laplacian_at(g, w, ti, tj, tab), full[tj, ti], rtol=1e-14, atol=0)


def test_sampled_node_velocity_matches_differenced_field():
    g = _grid(30, 26)
    rng = np.random.default_rng(8)
    X, Y, G = inputs.uniform_vortices(rng, 40, -0.5, 0.5, 0.01)
    w = vic.regularize(g, X, Y, G)
    tab = lgf_table(g.nx + 1, g.ny + 1)
    u, v = vic.node_velocity(g, vic.streamfunction(g, w, tab, pad=1), 0.2, -0.1)
    ti, tj = np.array([0, 29, 5, 17]), np.array([0, 25, 13, 2])
    us, vs = vic.node_velocity_at(g, w, ti, tj, tab, 0.2, -0.1)
    assert np.abs(us - u[tj, ti]).max() < 1e-12 and np.abs(vs - v[tj, ti]).max() < 1e-12


def _psi_error(n):
    """Fig. 2 experiment: random vortices in the lower-left quadrant of
    [-1,1]^2; relative L2 error of psi over the upper-right quadrant."""
    rng = np.random.default_rng(7)
    X, Y, G = inputs.uniform_vortices(rng, 10, -0.8, -0.2, 1.0)
    dx = 2.0 / (n - 1)
    g = vic.Grid(n, n, dx, -1.0, -1.0)
    w = vic.regularize(g, X, Y, G)
    psi = vic.streamfunction(g, w, lgf_table(n + 1, n + 1))
    xx, yy = np.meshgrid(g.node_x(), g.node_y())
    sel = (xx >= 0) & (yy >= 0)
    # continuous field -sum Gamma/(2 pi) ln r plus the constant the unit-spacing
    # LGF fixes: G(r/dx) ~ (ln(r/dx) + gamma_E + 1.5 ln 2)/(2 pi)
    c = (math.log(dx) - np.euler_gamma - 1.5 * math.log(2.0)) / (2 * math.pi)
    exact = np.zeros_like(xx)
    for x, y, gq in zip(X, Y, G):
        exact += -gq / (2 * math.pi) * np.log(np.hypot(xx - x, yy - y)) + gq * c
    return np.linalg.norm(psi[sel] - exact[sel]) / np.linalg.norm(exact[sel])


def test_streamfunction_second_order():
    """The discrete streamfunction converges at second order in dx (Fig. 2)."""
    e = [_psi_error(n) for n in (33, 65, 129)]
    rates = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    assert all(1.7 < r < 2.4 for r in rates), (e, rates)


def test_single_vortex_velocity():
    """Node velocity of one vortex far from it approaches Gamma/(2 pi r) (2nd order)."""
    errs = []
    for n in (33, 65):
        dx = 2.0 / (n - 1)
        g = vic.Grid(n, n, dx, -1.0, -1.0)
        w = vic.regularize(g, np.array([-0.5]), np.array([-0.4]), np.array([1.0]))
        psi1 = vic.streamfunction(g, w, lgf_table(n + 1, n + 1), pad=1)
        u, v = vic.node_velocity(g, psi1, 0.3, -0.2)
        xx, yy = np.meshgrid(g.node_x(), g.node_y())
        r2 = (xx + 0.5) ** 2 + (yy + 0.4) ** 2
        sel = r2 > 0.5 ** 2
        ue = -(yy + 0.4) / (2 * math.pi * r2) + 0.3
        ve = (xx + 0.5) / (2 * math.pi * r2) - 0.2
        errs.append(np.sqrt(np.sum((u - ue)[sel] ** 2 + (v - ve)[sel] ** 2) / np.sum(ue[sel] ** 2 + ve[sel] ** 2)))
    assert errs[1] < errs[0] / 3.0 and errs[1] < 1e-3, errs
