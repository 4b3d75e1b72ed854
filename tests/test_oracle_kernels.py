"""Pins of the discrete deltas (Sec. 2.1 M4', Sec. 2.2.1 smoothed three-point).

Neither formula is printed in the paper; both are pinned by the properties the
paper relies on: total circulation is preserved (partition of unity), E = R^T
reproduces constants and linear fields (zero first moment), compact radius-2
support and continuity.
"""
import numpy as np
import pytest

from oracle.kernels import m4prime, yang3


R = np.linspace(0.0, 1.0, 1001)[:, None]
K = np.arange(-3, 4)[None, :]


@pytest.mark.parametrize("kern", [m4prime, yang3])
def test_partition_of_unity_and_first_moment(kern):
    d = kern(R - K)
    assert np.abs(d.sum(axis=1) - 1.0).max() < 1e-14
    assert np.abs(((R - K) * d).sum(axis=1)).max() < 1e-14


@pytest.mark.parametrize("kern", [m4prime, yang3])
def test_support_and_continuity(kern):
    assert kern(np.array([2.0, 2.5, -2.0, -7.0])).tolist() == [0.0, 0.0, 0.0, 0.0]
    for edge in (1.0, 2.0):
        lo, hi = kern(np.array([edge - 1e-9, edge + 1e-9]))
        assert abs(lo - hi) < 1e-7
    x = np.linspace(-2.5, 2.5, 101)
    assert np.allclose(kern(x), kern(-x), atol=0, rtol=0)


def test_m4prime_interpolating_and_second_moment():
    assert m4prime(np.array([0.0, 1.0, -1.0, 2.0])).tolist() == [1.0, 0.0, 0.0, 0.0]
    d = m4prime(R - K)
    assert np.abs(((R - K) ** 2 * d).sum(axis=1)).max() < 1e-14   # reproduces quadratics


def test_yang3_values():
    v = yang3(np.array([0.0, 1.0]))
    assert abs(v[0] - 0.6182) < 1e-4 and abs(v[1] - 0.1909) < 1e-4
    assert np.all(yang3(np.linspace(-1.99, 1.99, 399)) > 0)
