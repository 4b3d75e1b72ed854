"""Launch configurations of the transfer and Poisson passes, and the autotuner.

Every configuration computes the same operators (R_v, L^-1 with the curl,
E_v; Sec. 2.1 and 2.3): each must match the FP64 oracle within the plan
precision's tolerance, and the block partition of the binning and the threads
per tile block must not change a single bit.
"""
import itertools

import numpy as np
import pytest
import torch

import paper_2102_11910_gb300 as pf
from oracle import vic as OV
from paper_2102_11910_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_W = {pf.PF_FP64: 1e-13, pf.PF_MIXED: 1e-6}
TOL_U = {pf.PF_FP64: 1e-12, pf.PF_MIXED: 1e-5}
CONFIGS = [dict(tile=t, min_span=s, tile_threads=n, fft=f)
           for t, s, n, f in itertools.product((32, 16), (256, 4096), (128, 256), (0, 1))]


def _rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _case(nx, ny, nv, seed):
    g = inputs.centred_grid(nx, ny, 2.0 / (nx - 1))
    rng = np.random.default_rng(seed)
    hx, hy = 0.5 * (nx - 1) * g.dx, 0.5 * (ny - 1) * g.dx
    X, Y, G = inputs.uniform_vortices(rng, nv, -0.85 * hx, 0.85 * hx, 1e-4, -0.85 * hy, 0.85 * hy)
    return g, X, Y, G


@pytest.mark.parametrize("prec", [pf.PF_FP64, pf.PF_MIXED])
def test_every_launch_configuration_matches_the_oracle(prec):
    """100 x 77 nodes: ragged last tiles at both edges for 16 and 32; the padded
    torus (256 x 256) admits both FFT families."""
    g, X, Y, G = _case(100, 77, 3000, 31)
    og = OV.Grid(g.nx, g.ny, g.dx, g.x0, g.y0)
    w_ref = OV.regularize(og, X, Y, G)
    _, _, ur, vr = OV.vortex_velocity(og, X, Y, G, 0.25, -0.1)
    plan = pf.Plan(g.nx, g.ny, g.dx, g.x0, g.y0, prec)
    dX, dY, dG = _dev(X), _dev(Y), _dev(G)
    for cfg in CONFIGS:
        pf.pf_launch_config_set(plan, **cfg)
        assert pf.pf_launch_config_get(plan) == cfg
        w = pf.pf_regularize(plan, dX, dY, dG)
        uq, vq = pf.pf_vic_velocity(plan, dX, dY, dG, 0.25, -0.1)
        pf.pf_sync(plan)
        assert _rel(w.cpu().numpy(), w_ref) < TOL_W[prec], cfg
        assert _rel(np.concatenate([uq.cpu().numpy(), vq.cpu().numpy()]), np.concatenate([ur, vr])) < TOL_U[prec], cfg


@pytest.mark.parametrize("prec", [pf.PF_FP64, pf.PF_MIXED])
@pytest.mark.parametrize("tile,fft", [(32, 0), (16, 1)])
def test_block_partition_and_threads_leave_results_bitwise_unchanged(prec, tile, fft):
    """5e4 vortices on 300 x 200 nodes: 196 binning blocks at min_span 256 down
    to 13 at 4096; integer deposit sums and per-vortex E_v make w and (u, v)
    independent of the partition and of the threads per tile."""
    g, X, Y, G = _case(300, 200, 50000, 32)
    plan = pf.Plan(g.nx, g.ny, g.dx, g.x0, g.y0, prec)
    dX, dY, dG = _dev(X), _dev(Y), _dev(G)
    out = []
    for span in (256, 512, 1024, 2048, 4096):
        for threads in (128, 256):
            pf.pf_launch_config_set(plan, tile=tile, min_span=span, tile_threads=threads, fft=fft)
            w = pf.pf_regularize(plan, dX, dY, dG).clone()
            uq, vq = pf.pf_vic_velocity(plan, dX, dY, dG, 0.3, 0.0)
            pf.pf_sync(plan)
            out.append((w, uq.clone(), vq.clone()))
    for w, uq, vq in out[1:]:
        assert torch.equal(w, out[0][0]) and torch.equal(uq, out[0][1]) and torch.equal(vq, out[0][2])


def test_small_tile_is_offered_up_to_4096_tiles():
    g, X, Y, G = _case(1024, 1024, 200000, 33)                      # 64 x 64 tiles of 16
    plan2 = pf.Plan(g.nx, g.ny, g.dx, g.x0, g.y0, pf.PF_MIXED)
    w32 = pf.pf_regularize(plan2, _dev(X), _dev(Y), _dev(G)).clone()
    pf.pf_launch_config_set(plan2, tile=16)
    w16 = pf.pf_regularize(plan2, _dev(X), _dev(Y), _dev(G))
    pf.pf_sync(plan2)
    assert _rel(w16.cpu().numpy(), w32.cpu().numpy()) < 1e-6
    big = pf.Plan(1040, 1024, 1e-3, 0.0, 0.0, pf.PF_MIXED)           # 65 x 64 tiles of 16
    with pytest.raises(pf.GridPfError) as e:
        pf.pf_launch_config_set(big, tile=16)
    assert e.value.name == "PF_ERR_ARG"
    assert pf.pf_launch_config_get(big)["tile"] == 32


@pytest.mark.parametrize("bad", [dict(tile=8), dict(tile=64), dict(min_span=300), dict(min_span=8192),
                                 dict(tile_threads=64), dict(tile_threads=512), dict(fft=2)])
def test_invalid_configurations_are_rejected_and_leave_the_plan_unchanged(bad):
    plan = pf.Plan(128, 128, 0.02, -1.27, -1.27, pf.PF_MIXED)
    before = pf.pf_launch_config_get(plan)
    with pytest.raises(pf.GridPfError) as e:
        pf.pf_launch_config_set(plan, **bad)
    assert e.value.name == "PF_ERR_ARG"
    assert pf.pf_launch_config_get(plan) == before


def test_new_plans_start_from_the_default_and_clones_copy_the_source():
    plan = pf.Plan(256, 256, 0.01, -1.0, -1.0, pf.PF_MIXED)
    assert pf.pf_launch_config_get(plan) == dict(tile=32, min_span=1024, tile_threads=256, fft=0)
    pf.pf_launch_config_set(plan, tile=16, min_span=512, tile_threads=128, fft=1)
    clone = pf.pf_plan_clone(plan, pf.PF_FP64, torch.cuda.Stream())
    assert pf.pf_launch_config_get(clone) == dict(tile=16, min_span=512, tile_threads=128, fft=1)


@pytest.mark.parametrize("prec", [pf.PF_FP64, pf.PF_MIXED])
def test_autotune_sets_the_fastest_valid_configuration_and_caches_it(prec, tmp_path):
    cache = tmp_path / "launch.cache"
    g, X, Y, G = _case(256, 192, 20000, 34)
    plan = pf.Plan(g.nx, g.ny, g.dx, g.x0, g.y0, prec)
    cfg, us = pf.pf_autotune(plan, 20000, str(cache), reps=3)
    assert us > 0 and pf.pf_launch_config_get(plan) == cfg
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and lines[0].startswith("gridpf-launch-config 1 ")
    assert ("fp64" if prec == pf.PF_FP64 else "mixed") in lines[0].split()
    # a second plan of the same grid takes the cached line without timing (the
    # time returned is the one written, to the file's three decimals)
    plan2 = pf.Plan(g.nx, g.ny, g.dx, g.x0, g.y0, prec)
    cfg2, us2 = pf.pf_autotune(plan2, 30000, str(cache), reps=3)        # same power of two
    assert cfg2 == cfg and abs(us2 - us) < 1e-3 + 1e-9 * us
    assert len(cache.read_text().splitlines()) == 1
    # another power of two is a new key
    pf.pf_autotune(plan2, 70000, str(cache), reps=1)
    assert len(cache.read_text().splitlines()) == 2
    # the tuned plan still computes the operators
    og = OV.Grid(g.nx, g.ny, g.dx, g.x0, g.y0)
    _, _, ur, vr = OV.vortex_velocity(og, X, Y, G, 0.25, 0.0)
    uq, vq = pf.pf_vic_velocity(plan, _dev(X), _dev(Y), _dev(G), 0.25, 0.0)
    pf.pf_sync(plan)
    assert _rel(np.concatenate([uq.cpu().numpy(), vq.cpu().numpy()]), np.concatenate([ur, vr])) < TOL_U[prec]


def test_autotune_rejects_bad_arguments():
    plan = pf.Plan(128, 128, 0.02, -1.27, -1.27, pf.PF_MIXED)
    for nv, reps in ((0, 3), (1000, 0)):
        with pytest.raises(pf.GridPfError) as e:
            pf.pf_autotune(plan, nv, None, reps)
        assert e.value.name == "PF_ERR_ARG"
