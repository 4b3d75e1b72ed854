"""The allocation-free regularization entry point gives the plan-based result.

Some callers cannot allocate device memory (they run where cudaMalloc is not
allowed, or under an allocator they do not own); pf_regularize_noalloc serves
them from a static device scratch array.  Because every call reuses that one
array, the test makes two calls in a row with different vortex sets and checks
each against pf_regularize, which allocates its scratch in a plan.  This file
is named to be collected last.
"""
import numpy as np
import pytest
import torch

import paper_2102_11910_gb300 as pf
from paper_2102_11910_gb300 import inputs

pytestmark = pytest.mark.gpu


def _rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("prec,tol", [(pf.PF_MIXED, 1e-6), (pf.PF_FP64, 1e-13)])
def test_noalloc_matches_plan_path_on_two_calls_in_a_row(prec, tol):
    g = inputs.centred_grid(100, 77, 0.02)
    plan = pf.Plan(g.nx, g.ny, g.dx, g.x0, g.y0, prec)
    dtype = torch.float64 if prec == pf.PF_FP64 else torch.float32
    for seed, nv in ((21, 5000), (22, 65536)):
        rng = np.random.default_rng(seed)
        hx, hy = 0.45 * (g.nx - 1) * g.dx, 0.45 * (g.ny - 1) * g.dx
        X, Y, G = (torch.from_numpy(a).cuda() for a in inputs.uniform_vortices(rng, nv, -hx, hx, 1e-3, -hy, hy))
        ref = pf.pf_regularize(plan, X, Y, G)
        w = torch.full((g.ny, g.nx), float("nan"), dtype=dtype, device="cuda")
        oob = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        pf.pf_regularize_noalloc(g.nx, g.ny, g.dx, g.x0, g.y0, prec, X, Y, G, w, oob, st)
        torch.cuda.synchronize()
        pf.pf_sync(plan)
        assert int(oob.item()) == 0
        assert int(st.item()) == 0          # PF_OK: no binning check failed
        assert torch.isfinite(w).all()
        assert _rel(w, ref) <= tol
        # same kernels on other scratch: the tiles' counts, exponents and
        # integer sums are the same, so w is bitwise the same
        assert torch.equal(w, ref)


@pytest.mark.parametrize("prec", [pf.PF_MIXED, pf.PF_FP64])
def test_noalloc_at_its_largest_grid_and_vortex_count(prec):
    """The scratch layout at its stated maximum (2048^2 nodes: 4096 tiles, the
    whole offset table; 65536 vortices: 64 binning blocks), bitwise against
    the plan path, twice in a row."""
    g = inputs.centred_grid(2048, 2048, 1.0 / 1024)
    plan = pf.Plan(g.nx, g.ny, g.dx, g.x0, g.y0, prec)
    dtype = torch.float64 if prec == pf.PF_FP64 else torch.float32
    for seed in (31, 32):
        rng = np.random.default_rng(seed)
        h = 0.49 * (g.nx - 1) * g.dx
        X, Y, G = (torch.from_numpy(a).cuda() for a in inputs.uniform_vortices(rng, 65536, -h, h, 1e-3))
        ref = pf.pf_regularize(plan, X, Y, G)
        w = torch.full((g.ny, g.nx), float("nan"), dtype=dtype, device="cuda")
        st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        pf.pf_regularize_noalloc(g.nx, g.ny, g.dx, g.x0, g.y0, prec, X, Y, G, w, None, st)
        torch.cuda.synchronize()
        pf.pf_sync(plan)
        assert int(st.item()) == 0
        assert torch.equal(w, ref)
    plan.close()


def test_noalloc_wrapper_rejects_mismatched_arguments():
    g = inputs.centred_grid(64, 64, 0.02)
    X = torch.zeros(4, dtype=torch.float64, device="cuda")
    w = torch.empty((g.ny, g.nx), dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError):
        pf.pf_regularize_noalloc(g.nx, g.ny, g.dx, g.x0, g.y0, pf.PF_MIXED, X, X[:3], X, w)
    with pytest.raises(ValueError):
        pf.pf_regularize_noalloc(g.nx, g.ny, g.dx, g.x0, g.y0, pf.PF_MIXED, X, X, X, w[:10])


def test_noalloc_reports_out_of_domain_and_rejects_oversize():
    g = inputs.centred_grid(64, 64, 0.02)
    X = torch.tensor([0.0, g.x0 + 0.5 * g.dx, 0.1], dtype=torch.float64, device="cuda")
    Y = torch.zeros(3, dtype=torch.float64, device="cuda")
    G = torch.ones(3, dtype=torch.float64, device="cuda")
    w = torch.empty((g.ny, g.nx), dtype=torch.float32, device="cuda")
    oob = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    pf.pf_regularize_noalloc(g.nx, g.ny, g.dx, g.x0, g.y0, pf.PF_MIXED, X, Y, G, w, oob, st)
    torch.cuda.synchronize()
    assert int(oob.item()) == 1
    assert int(st.item()) == pf.PF_ERR_OUT_OF_DOMAIN
    assert abs(float(w.double().sum()) * g.dx ** 2 - 2.0) < 1e-5     # the two valid vortices
    big = torch.zeros(65537, dtype=torch.float64, device="cuda")
    with pytest.raises(pf.GridPfError) as e:
        pf.pf_regularize_noalloc(g.nx, g.ny, g.dx, g.x0, g.y0, pf.PF_MIXED, big, big, big, w)
    assert e.value.name == "PF_ERR_CAPACITY"
