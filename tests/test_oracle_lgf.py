"""Pins of the oracle's lattice Green's function (Sec. 2.1: L^{-1} by the LGF).

The table is checked against quantities fixed by the mathematics, not by
re-running its own quadrature: exact lattice values (tests/golden), the
diagonal closed form for large n, the defining equation L0 G = delta at every
table point, and the far-field expansion.
"""
import math
import os

import numpy as np
import pytest

from oracle.lgf import lgf_table, quadrature_nodes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "lgf_exact_values.txt")


@pytest.fixture(scope="module")
def table():
    return lgf_table(400)


def _golden():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        m, n, expr, val = line.split()
        rows.append((int(m), int(n), eval(expr, {"pi": math.pi}), float(val)))
    return rows


def test_exact_values(table):
    for m, n, exact, printed in _golden():
        assert abs(exact - printed) < 1e-15
        assert abs(table[m, n] - exact) < 2e-16 * max(1, exact) * 4
        assert table[m, n] == table[n, m]


def test_origin_is_zero(table):
    assert table[0, 0] == 0.0


@pytest.mark.parametrize("n", [5, 50, 200, 400])
def test_diagonal_closed_form(table, n):
    exact = sum(1.0 / (2 * k - 1) for k in range(1, n + 1)) / math.pi
    assert abs(table[n, n] - exact) < 2e-15


def test_defining_equation_everywhere(table):
    """L0 G = delta_0 at every table point (G even in both indices)."""
    K = 120
    T = table[: K + 2, : K + 2]
    full = np.zeros((2 * K + 3, 2 * K + 3))
    idx = np.abs(np.arange(-(K + 1), K + 2))
    full[:, :] = T[idx[:, None], idx[None, :]]
    lap = full[2:, 1:-1] + full[:-2, 1:-1] + full[1:-1, 2:] + full[1:-1, :-2] - 4 * full[1:-1, 1:-1]
    delta = np.zeros_like(lap)
    delta[K, K] = 1.0
    assert np.abs(lap - delta).max() < 5e-15


def test_far_field(table):
    """G -> (1/2pi)(ln r + gamma_E + 3/2 ln 2) - cos(4 th)/(24 pi r^2) + O(r^-4)."""
    for m, n in [(300, 0), (250, 200), (400, 100), (350, 350)]:
        r = math.hypot(m, n)
        th = math.atan2(n, m)
        asym = (math.log(r) + np.euler_gamma + 1.5 * math.log(2)) / (2 * math.pi) - math.cos(4 * th) / (24 * math.pi * r * r)
        assert abs(table[m, n] - asym) < 5.0 / r ** 4 + 1e-14


def test_independent_of_quadrature_grading():
    """A much finer composite rule gives the same table (quadrature converged)."""
    th, wt = quadrature_nodes(theta_min=1e-12, ratio=1.15, order=32)
    m, n = 137, 59
    u = np.arcsinh(np.sin(0.5 * th))
    f = (1 - np.exp(-2 * m * u) * np.cos(n * th)) / np.sinh(2 * u)
    ref = np.dot(wt, f) / (2 * math.pi)
    assert abs(lgf_table(140)[m, n] - ref) < 1e-14
