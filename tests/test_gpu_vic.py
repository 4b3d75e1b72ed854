"""GPU parity of the body-free VIC path (Sec. 2.1) against the FP64 oracle.

Tolerances: the all-FP64 path must match the oracle to 1e-12 relative (L2)
and the mixed FP32 path to 1e-5 relative in streamfunction and velocity.
"""
import math

import numpy as np
import pytest
import torch

import paper_2102_11910_gb300 as pf
from oracle import vic as OV
from oracle.lgf import lgf_table
from paper_2102_11910_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {pf.PF_FP64: 1e-12, pf.PF_MIXED: 1e-5}


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _case(nx, ny, nv, seed, variance=1e-2):
    g = inputs.centred_grid(nx, ny, 2.0 / (nx - 1))
    rng = np.random.default_rng(seed)
    hx, hy = 0.5 * (nx - 1) * g.dx, 0.5 * (ny - 1) * g.dx
    X, Y, G = inputs.uniform_vortices(rng, nv, -0.8 * hx, 0.8 * hx, variance, -0.8 * hy, 0.8 * hy)
    return g, X, Y, G


def _plan(g, prec):
    return pf.Plan(g.nx, g.ny, g.dx, g.x0, g.y0, prec)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _og(g):
    return OV.Grid(g.nx, g.ny, g.dx, g.x0, g.y0)


@pytest.mark.parametrize("nx,ny", [(1024, 1024), (100, 77), (768, 512)])
def test_lgf_table_matches_oracle(nx, ny):
    g = inputs.centred_grid(nx, ny, 0.01)
    plan = _plan(g, pf.PF_FP64)
    T = pf.pf_lgf_table(plan)              # [n, m]
    ref = lgf_table(nx, ny).T              # oracle [m, n] -> [n, m]
    assert np.abs(T - ref).max() < 2e-14


@pytest.mark.parametrize("prec", [pf.PF_FP64, pf.PF_MIXED])
@pytest.mark.parametrize("nx,ny,nv", [(64, 64, 300), (100, 77, 500), (37, 45, 40)])
def test_regularize(prec, nx, ny, nv):
    g, X, Y, G = _case(nx, ny, nv, 11)
    plan = _plan(g, prec)
    w = pf.pf_regularize(plan, _dev(X), _dev(Y), _dev(G))
    pf.pf_sync(plan)
    ref = OV.regularize(_og(g), X, Y, G)
    assert rel(w.cpu().numpy(), ref) < (1e-13 if prec == pf.PF_FP64 else 1e-6)
    # integer accumulation: bitwise reproducible run to run
    w2 = pf.pf_regularize(plan, _dev(X), _dev(Y), _dev(G))
    assert torch.equal(w, w2)


@pytest.mark.parametrize("prec", [pf.PF_FP64, pf.PF_MIXED])
def test_regularize_is_unaffected_by_the_previous_call(prec):
    """Every binning pass reads only what the current call wrote: on a 2048^2
    grid (4096 tiles, sixteen per thread in the tile scan), regularizing new
    vortices straight after other ones gives bitwise what a repeat of the same
    call gives, and the velocity step likewise.  (Dependent kernels launched
    while the previous kernel still ran once read stale cache lines of the
    in-place offset table here.)"""
    g = inputs.centred_grid(2048, 2048, 1.0 / 1024)
    plan = _plan(g, prec)
    h = 0.49 * (g.nx - 1) * g.dx
    sets = [inputs.uniform_vortices(np.random.default_rng(s), 200000, -h, h, 1e-3) for s in (41, 42, 43)]
    for X, Y, G in sets:
        d = [_dev(a) for a in (X, Y, G)]
        w1 = pf.pf_regularize(plan, *d)
        w2 = pf.pf_regularize(plan, *d)
        u1, v1 = pf.pf_vic_velocity(plan, *d, 0.3, 0.0)
        u1, v1 = u1.clone(), v1.clone()
        u2, v2 = pf.pf_vic_velocity(plan, *d, 0.3, 0.0)
        pf.pf_sync(plan)
        assert torch.equal(w1, w2)
        assert torch.equal(u1, u2) and torch.equal(v1, v2)
    ref = OV.regularize(_og(g), *sets[-1])          # the last set against the oracle
    assert rel(w1.cpu().numpy(), ref) < TOL[prec] / (1.0 if prec == pf.PF_FP64 else 10.0)
    plan.close()


@pytest.mark.parametrize("prec", [pf.PF_FP64, pf.PF_MIXED])
@pytest.mark.parametrize("nblob,nspread", [(6000, 2000), (70000, 500)])
def test_regularize_dense_and_sparse_tiles(prec, nblob, nspread):
    """One grid holding tiles of a few records and one tile of thousands or of
    more than 65536 (where the FP32 deposit leaves its split 32-bit sums for
    64-bit ones): a Gaussian blob of vortices on a uniform spread."""
    g = inputs.centred_grid(96, 96, 2.0 / 95)
    rng = np.random.default_rng(17)
    cx, cy = g.x0 + 48.3 * g.dx, g.y0 + 47.6 * g.dx          # inside node tile (1, 1)
    Xb = cx + 4.0 * g.dx * rng.standard_normal(nblob)
    Yb = cy + 4.0 * g.dx * rng.standard_normal(nblob)
    Gb = rng.normal(0.0, 0.1, nblob)
    Xs, Ys, Gs = inputs.uniform_vortices(rng, nspread, g.x0 + 2 * g.dx, g.x0 + 92 * g.dx, 1e-2,
                                         g.y0 + 2 * g.dx, g.y0 + 92 * g.dx)
    X, Y, G = (np.concatenate(p) for p in ((Xb, Xs), (Yb, Ys), (Gb, Gs)))
    keep = (X > g.x0 + 1.5 * g.dx) & (X < g.x0 + 92.5 * g.dx) & (Y > g.y0 + 1.5 * g.dx) & (Y < g.y0 + 92.5 * g.dx)
    X, Y, G = X[keep], Y[keep], G[keep]
    plan = _plan(g, prec)
    w = pf.pf_regularize(plan, _dev(X), _dev(Y), _dev(G))
    pf.pf_sync(plan)
    ref = OV.regularize(_og(g), X, Y, G)
    # the fixed-point step of a tile grows with its record count x max|Gamma|
    # (each term is rounded to 2^-sh with 2^(61-sh) > count max|Gamma|): a
    # 70000-record tile leaves ~2e-13 in FP64, within the FP64 path's 1e-12
    assert rel(w.cpu().numpy(), ref) < TOL[prec] / (1.0 if prec == pf.PF_FP64 else 10.0)
    w2 = pf.pf_regularize(plan, _dev(X), _dev(Y), _dev(G))
    assert torch.equal(w, w2)


@pytest.mark.parametrize("prec", [pf.PF_FP64, pf.PF_MIXED])
@pytest.mark.parametrize("nx,ny", [(64, 64), (100, 77), (37, 45), (128, 48), (300, 200), (600, 100)])
def test_poisson_solve(prec, nx, ny):
    g, X, Y, G = _case(nx, ny, 200, 12)
    og = _og(g)
    w = OV.regularize(og, X, Y, G)
    plan = _plan(g, prec)
    wt = torch.from_numpy(w).to(device="cuda", dtype=plan.dtype)
    psi = pf.pf_poisson_solve(plan, wt)
    pf.pf_sync(plan)
    ref = OV.streamfunction(og, w, lgf_table(nx + 1, ny + 1))
    assert rel(psi.cpu().numpy(), ref) < TOL[prec]


@pytest.mark.parametrize("prec", [pf.PF_FP64, pf.PF_MIXED])
@pytest.mark.parametrize("nx,ny", [(64, 64), (100, 77), (37, 45), (300, 200), (600, 100)])
def test_velocity_solve(prec, nx, ny):
    g, X, Y, G = _case(nx, ny, 200, 13)
    og = _og(g)
    w = OV.regularize(og, X, Y, G)
    plan = _plan(g, prec)
    wt = torch.from_numpy(w).to(device="cuda", dtype=plan.dtype)
    uv = pf.pf_velocity_solve(plan, wt, 0.7, -0.3).cpu().numpy()
    pf.pf_sync(plan)
    psi1 = OV.streamfunction(og, w, lgf_table(nx + 1, ny + 1), pad=1)
    u, v = OV.node_velocity(og, psi1, 0.7, -0.3)
    assert rel(uv[..., 0], u) < TOL[prec]
    assert rel(uv[..., 1], v) < TOL[prec]


@pytest.mark.parametrize("prec", [pf.PF_FP64, pf.PF_MIXED])
def test_interpolate(prec):
    g, X, Y, G = _case(80, 70, 1000, 14)
    rng = np.random.default_rng(3)
    f = rng.normal(size=(g.ny, g.nx, 2))
    plan = _plan(g, prec)
    uq, vq = pf.pf_interpolate(plan, torch.from_numpy(f).to(device="cuda", dtype=plan.dtype).contiguous(), _dev(X), _dev(Y))
    pf.pf_sync(plan)
    og = _og(g)
    assert rel(uq.cpu().numpy(), OV.interpolate(og, f[..., 0], X, Y)) < (1e-13 if prec == pf.PF_FP64 else 1e-6)
    assert rel(vq.cpu().numpy(), OV.interpolate(og, f[..., 1], X, Y)) < (1e-13 if prec == pf.PF_FP64 else 1e-6)


@pytest.mark.parametrize("prec", [pf.PF_FP64, pf.PF_MIXED])
@pytest.mark.parametrize("n,nv", [(64, 400), (128, 3000), (96, 0)])
def test_vic_velocity_end_to_end(prec, n, nv):
    g, X, Y, G = _case(n, n, nv, 15, variance=1e-4)
    plan = _plan(g, prec)
    uq, vq = pf.pf_vic_velocity(plan, _dev(X), _dev(Y), _dev(G), 0.25, 0.0)
    pf.pf_sync(plan)
    if nv == 0:
        assert uq.numel() == 0
        return
    _, _, ru, rv = OV.vortex_velocity(_og(g), X, Y, G, 0.25, 0.0)
    assert rel(uq.cpu().numpy(), ru) < TOL[prec]
    assert rel(vq.cpu().numpy(), rv) < TOL[prec]
    # host-buffer entry point gives the same numbers, from pageable inputs (staged
    # through a copy) and from page-locked ones (read in place by the first kernel)
    hu, hv = pf.pf_vic_velocity_host(plan, torch.from_numpy(X), torch.from_numpy(Y), torch.from_numpy(G), 0.25, 0.0)
    assert torch.equal(hu, uq.cpu()) and torch.equal(hv, vq.cpu())
    pX, pY, pG = (torch.from_numpy(a).pin_memory() for a in (X, Y, G))
    hu, hv = pf.pf_vic_velocity_host(plan, pX, pY, pG, 0.25, 0.0)
    assert torch.equal(hu, uq.cpu()) and torch.equal(hv, vq.cpu())


def test_async_host_steps_on_two_plans_in_turn_match_the_device_step():
    """pf_vic_velocity_host_async on two plans in turn (each synchronised
    before its next step, the other's step in flight meanwhile) gives, step
    after step, bitwise the velocities of the device-buffer step."""
    g, X, Y, G = _case(128, 128, 3000, 18, variance=1e-4)
    plans = [_plan(g, pf.PF_MIXED) for _ in range(2)]
    ru, rv = pf.pf_vic_velocity(plans[0], _dev(X), _dev(Y), _dev(G), 0.25, -0.1)
    pf.pf_sync(plans[0])
    ru, rv = ru.cpu(), rv.cpu()
    hX, hY, hG = (torch.from_numpy(a).pin_memory() for a in (X, Y, G))
    outs = [(torch.full((len(X),), float("nan")).pin_memory(), torch.full((len(X),), float("nan")).pin_memory())
            for _ in range(2)]
    for k in range(6):
        pl, (hu, hv) = plans[k % 2], outs[k % 2]
        if k >= 2:
            pf.pf_sync(pl)
            assert torch.equal(hu, ru) and torch.equal(hv, rv)
            hu.fill_(float("nan"))
            hv.fill_(float("nan"))
        pf.pf_vic_velocity_host_async(pl, hX, hY, hG, 0.25, -0.1, hu, hv)
    for pl, (hu, hv) in zip(plans, outs):
        pf.pf_sync(pl)
        assert torch.equal(hu, ru) and torch.equal(hv, rv)
    # pageable host buffers take the same path (their copies do not overlap)
    pu, pv = torch.empty(len(X)), torch.empty(len(X))
    pf.pf_vic_velocity_host_async(plans[1], torch.from_numpy(X), torch.from_numpy(Y), torch.from_numpy(G),
                                  0.25, -0.1, pu, pv)
    pf.pf_sync(plans[1])
    assert torch.equal(pu, ru) and torch.equal(pv, rv)
    with pytest.raises(ValueError):
        pf.pf_vic_velocity_host_async(plans[1], hX, hY, hG, 0.25, -0.1, pu, pv[:-1])


def test_out_of_domain_is_reported_not_dropped_silently():
    g, X, Y, G = _case(64, 64, 100, 16)
    X = X.copy()
    X[5] = g.x0 + 0.5 * g.dx          # stencil would leave the grid
    X[7] = g.x0 + 62.9 * g.dx
    plan = _plan(g, pf.PF_MIXED)
    pf.pf_regularize(plan, _dev(X), _dev(Y), _dev(G))
    with pytest.raises(pf.GridPfError) as e:
        pf.pf_sync(plan)
    assert e.value.name == "PF_ERR_OUT_OF_DOMAIN" and "2 points" in str(e.value)
    assert pf.pf_sync(plan) == 0       # the status is cleared once reported


@pytest.mark.parametrize("prec", [pf.PF_FP64, pf.PF_MIXED])
def test_odd_count_across_blocks_and_out_of_domain(prec):
    """5001 vortices over several binning blocks, the last one odd-sized, 7
    of them off the grid (first and last vortices among them): w matches the
    oracle on the others, and the 7 are reported."""
    g, X, Y, G = _case(96, 80, 5001, 19)
    X, Y = X.copy(), Y.copy()
    off = [0, 1, 777, 2048, 4095, 4999, 5000]
    X[off[:4]] = g.x0 - 3.0 * g.dx
    Y[off[4:]] = g.y0 + (g.ny + 2) * g.dx
    keep = np.ones(len(X), bool)
    keep[off] = False
    plan = _plan(g, prec)
    w = pf.pf_regularize(plan, _dev(X), _dev(Y), _dev(G))
    with pytest.raises(pf.GridPfError) as e:
        pf.pf_sync(plan)
    assert e.value.name == "PF_ERR_OUT_OF_DOMAIN" and "7 points" in str(e.value)
    ref = OV.regularize(_og(g), X[keep], Y[keep], G[keep])
    assert rel(w.cpu().numpy(), ref) < (1e-13 if prec == pf.PF_FP64 else 1e-6)


@pytest.mark.parametrize("prec", [pf.PF_FP64, pf.PF_MIXED])
@pytest.mark.parametrize("tile", [32, 16])
def test_vortices_off_the_grid_get_zero_velocity(prec, tile):
    """The 7 vortices off the grid of the test above are left out of R_v and
    get u = v = 0 (their outputs start as NaN); the others match the oracle
    run without them.  Both tile edges."""
    g, X, Y, G = _case(96, 80, 5001, 19, variance=1e-4)
    X, Y = X.copy(), Y.copy()
    off = [0, 1, 777, 2048, 4095, 4999, 5000]
    X[off[:4]] = g.x0 - 3.0 * g.dx
    Y[off[4:]] = g.y0 + (g.ny + 2) * g.dx
    keep = np.ones(len(X), bool)
    keep[off] = False
    plan = _plan(g, prec)
    pf.pf_launch_config_set(plan, tile=tile)
    dtype = torch.float64 if prec == pf.PF_FP64 else torch.float32
    uq = torch.full((len(X),), float("nan"), dtype=dtype, device="cuda")
    vq = torch.full_like(uq, float("nan"))
    pf.pf_vic_velocity(plan, _dev(X), _dev(Y), _dev(G), 0.25, 0.0, uq, vq)
    with pytest.raises(pf.GridPfError) as e:
        pf.pf_sync(plan)
    assert e.value.name == "PF_ERR_OUT_OF_DOMAIN" and "7 points" in str(e.value)
    u, v = uq.cpu().numpy(), vq.cpu().numpy()
    assert np.all(u[off] == 0.0) and np.all(v[off] == 0.0)
    _, _, ru, rv = OV.vortex_velocity(_og(g), X[keep], Y[keep], G[keep], 0.25, 0.0)
    assert rel(u[keep], ru) < TOL[prec] and rel(v[keep], rv) < TOL[prec]


def test_full_size_vic_sampled_against_oracle():
    """1024^2 nodes, 1e6 vortices: w on every node, and psi / velocity at sampled
    nodes and vortices computed one by one by the oracle's direct sums."""
    wl = inputs.vic_1024()
    g = wl["grid"]
    og = _og(g)
    X, Y, G = wl["X"], wl["Y"], wl["G"]
    w_ref = OV.regularize(og, X, Y, G)
    tab = lgf_table(g.nx + 1, g.ny + 1)
    rng = np.random.default_rng(5)
    for prec in (pf.PF_FP64, pf.PF_MIXED):
        plan = _plan(g, prec)
        dX, dY, dG = _dev(X), _dev(Y), _dev(G)
        w = pf.pf_regularize(plan, dX, dY, dG)
        psi = pf.pf_poisson_solve(plan, w).cpu().numpy()
        uq, vq = pf.pf_vic_velocity(plan, dX, dY, dG)
        pf.pf_sync(plan)
        assert rel(w.cpu().numpy(), w_ref) < (1e-13 if prec == pf.PF_FP64 else 1e-6)
        # psi at sampled nodes (including the corners)
        ti = np.concatenate([[0, g.nx - 1, 0, g.nx - 1], rng.integers(0, g.nx, 12)])
        tj = np.concatenate([[0, 0, g.ny - 1, g.ny - 1], rng.integers(0, g.ny, 12)])
        ref = -OV.inv_laplacian_at(og, w_ref, ti, tj, tab)
        assert rel(psi[tj, ti], ref) < TOL[prec]
        # velocity at sampled vortices: node velocities of the 4x4 stencil, one by one
        qs = rng.integers(0, len(X), 6)
        u_s, v_s = [], []
        for q in qs:
            ci = int(math.floor((X[q] - g.x0) / g.dx)); cj = int(math.floor((Y[q] - g.y0) / g.dx))
            bi, bj = np.meshgrid(np.arange(ci - 1, ci + 3), np.arange(cj - 1, cj + 3))
            un, vn = OV.node_velocity_at(og, w_ref, bi.ravel(), bj.ravel(), tab)
            big = OV.Grid(8, 8, g.dx, g.x0 + (ci - 3) * g.dx, g.y0 + (cj - 3) * g.dx)
            U = np.zeros((8, 8)); V = np.zeros((8, 8))
            U[2:6, 2:6] = un.reshape(4, 4); V[2:6, 2:6] = vn.reshape(4, 4)
            u_s.append(OV.interpolate(big, U, X[q:q + 1], Y[q:q + 1])[0])
            v_s.append(OV.interpolate(big, V, X[q:q + 1], Y[q:q + 1])[0])
        got = np.concatenate([uq.cpu().numpy()[qs], vq.cpu().numpy()[qs]])
        assert rel(got, np.concatenate([u_s, v_s])) < TOL[prec]


def test_largest_grid_sampled_against_oracle():
    """The largest grid a plan takes along x, 2048 x 1800 nodes (4096-point
    padded transforms on both axes; 1800 rows leave a ragged last row of
    tiles), 2e5 vortices: w on every node, psi and vortex velocities at
    sampled points by the oracle's direct sums."""
    nx, ny, nv = 2048, 1800, 200_000
    g = inputs.centred_grid(nx, ny, 2.0 / (nx - 1))
    rng = np.random.default_rng(23)
    hx, hy = 0.5 * (nx - 1) * g.dx, 0.5 * (ny - 1) * g.dx
    X, Y, G = inputs.uniform_vortices(rng, nv, -0.8 * hx, 0.8 * hx, 1e-4, -0.8 * hy, 0.8 * hy)
    og = _og(g)
    w_ref = OV.regularize(og, X, Y, G)
    tab = lgf_table(nx + 1, ny + 1)
    ti = np.concatenate([[0, nx - 1, 0, nx - 1], rng.integers(0, nx, 8)])
    tj = np.concatenate([[0, 0, ny - 1, ny - 1], rng.integers(0, ny, 8)])
    psi_ref = -OV.inv_laplacian_at(og, w_ref, ti, tj, tab)
    qs = rng.integers(0, nv, 4)
    u_s, v_s = [], []
    for q in qs:
        ci = int(math.floor((X[q] - g.x0) / g.dx)); cj = int(math.floor((Y[q] - g.y0) / g.dx))
        bi, bj = np.meshgrid(np.arange(ci - 1, ci + 3), np.arange(cj - 1, cj + 3))
        un, vn = OV.node_velocity_at(og, w_ref, bi.ravel(), bj.ravel(), tab)
        box = OV.Grid(8, 8, g.dx, g.x0 + (ci - 3) * g.dx, g.y0 + (cj - 3) * g.dx)
        U = np.zeros((8, 8)); V = np.zeros((8, 8))
        U[2:6, 2:6] = un.reshape(4, 4); V[2:6, 2:6] = vn.reshape(4, 4)
        u_s.append(OV.interpolate(box, U, X[q:q + 1], Y[q:q + 1])[0])
        v_s.append(OV.interpolate(box, V, X[q:q + 1], Y[q:q + 1])[0])
    for prec in (pf.PF_FP64, pf.PF_MIXED):
        plan = _plan(g, prec)
        assert plan.P == 4096 and plan.Q == 4096
        dX, dY, dG = _dev(X), _dev(Y), _dev(G)
        w = pf.pf_regularize(plan, dX, dY, dG)
        psi = pf.pf_poisson_solve(plan, w).cpu().numpy()
        uq, vq = pf.pf_vic_velocity(plan, dX, dY, dG)
        pf.pf_sync(plan)
        assert rel(w.cpu().numpy(), w_ref) < (1e-13 if prec == pf.PF_FP64 else 1e-6)
        assert rel(psi[tj, ti], psi_ref) < TOL[prec]
        got = np.concatenate([uq.cpu().numpy()[qs], vq.cpu().numpy()[qs]])
        assert rel(got, np.concatenate([u_s, v_s])) < TOL[prec]
        del plan
