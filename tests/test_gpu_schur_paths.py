"""The Schur inverse on every path it takes: blocked Gauss-Jordan with a ragged
last panel (33 points), several full panels (256), the largest blocked size
(1024) and the unblocked fallback above it (1100).  The refined f0 = S^-1 1 and
a given-s0 sheet solve with w = 0 (right-hand side s'_b - s0 1, known in
closed form) are compared with numpy's LU solve of the GPU's own S."""
import math

import numpy as np
import pytest
import torch

import paper_2102_11910_gb300 as pf
from paper_2102_11910_gb300 import inputs

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


@pytest.mark.parametrize("ns", [33, 256, 1024, 1100])
def test_inverse_paths_match_a_dense_solve(ns):
    a, b = 0.45, 0.3
    e = inputs.ellipse(ns, a, b, 0.0, 0.0, 0.4)
    dx = e.ds[0] / 2.0                                   # dS/dx = 2
    n = int(math.ceil(2.3 * a / dx)) + 16
    g = inputs.centred_grid(n, n, dx)
    plan = pf.Plan(g.nx, g.ny, g.dx, g.x0, g.y0, pf.PF_FP64)
    schur = pf.pf_schur_factor(plan, e.x, e.y, e.ds)
    gamma0, f0, S = pf.pf_schur_info(schur)
    cond = np.linalg.cond(S)
    ref = np.linalg.solve(S, np.ones(ns))
    assert rel(f0, ref) < cond * 1e-14
    assert abs(gamma0 - np.dot(e.ds, ref)) < cond * 1e-14 * abs(gamma0)
    U, V, Om, s0 = 0.3, -0.2, 0.5, 0.1
    w = torch.zeros(g.nx * g.ny, dtype=torch.float64, device="cuda")
    f, _, s0o = pf.pf_sheet_solve(plan, schur, w, (U, V, Om, 0.0, 0.0), pf.PF_SHEET_GIVEN_S0, s0)
    sb = U * e.y - V * e.x - 0.5 * Om * (e.x ** 2 + e.y ** 2)
    assert rel(f.cpu().numpy(), np.linalg.solve(S, sb - s0)) < cond * 1e-14
