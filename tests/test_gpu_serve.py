"""Request server: continuous batching on one GPU.

A request's result must not depend on what else is running: the same request
alone, in a mix with other grids and bodies, and through pf_step directly
gives bitwise identical vortices (deterministic kernels, no shared mutable
state between instances).
"""
import math
import time

import numpy as np
import pytest

import paper_2102_11910_gb300 as pf
from paper_2102_11910_gb300 import inputs

pytestmark = pytest.mark.gpu


def _grid(n):
    g = inputs.centred_grid(n, n, 3.0 / (n - 1))
    return (g.nx, g.ny, g.dx, g.x0, g.y0)


def _drain(server, tickets, timeout=120.0):
    pending = set(tickets)
    done = []
    t0 = time.time()
    while pending:
        fin = pf.pf_server_progress(server)
        for t in fin:
            pending.discard(t)
            done.append(t)
        if time.time() - t0 > timeout:
            raise TimeoutError("server did not finish: %d pending" % len(pending))
        time.sleep(0.001)
    return done


def _request_a():
    rng = np.random.default_rng(31)
    X, Y, G = inputs.uniform_vortices(rng, 60, -1.2, 1.2, 1e-3, -1.2, -0.5)
    body = pf.plate_kinematics(32, 1.0, math.radians(25.0), Uinf=1.0)
    return dict(grid=_grid(128), X=X, Y=Y, G=G, nsteps=5, dt=0.02, body=body, scheme=1)


def _others():
    out = []
    for k, n in enumerate((256, 128, 192, 256)):
        rng = np.random.default_rng(100 + k)
        X, Y, G = inputs.uniform_vortices(rng, 200 + 100 * k, -1.0, 1.0, 1e-3, -1.3, -0.7)
        if k % 2:
            e = inputs.ellipse(48, 0.5, 0.12)
            body = pf.BodyKinematics(e.x, e.y, e.ds, (), 0.2, 0.05, 1.0, 1.0)
        else:
            body = pf.plate_kinematics(40, 1.0, math.radians(15.0 + 5 * k), Uinf=1.0)
        out.append(dict(grid=_grid(n), X=X, Y=Y, G=G, nsteps=3 + k, dt=0.02, body=body, scheme=k % 2))
    return out


def _submit(server, r):
    return pf.pf_server_submit(server, r["grid"], r["X"], r["Y"], r["G"], r["nsteps"], r["dt"], r["body"],
                               scheme=r["scheme"])


def _cap(r):
    return len(r["X"]) + 2 * r["nsteps"]


@pytest.mark.parametrize("prec", [pf.PF_MIXED, pf.PF_FP64])
def test_result_is_the_same_alone_and_in_the_mix(prec):
    a = _request_a()
    server = pf.Server(max_slots=8, hbm_budget_bytes=4 << 30, precision=prec)
    ta = _submit(server, a)
    _drain(server, [ta])
    alone = pf.pf_server_result(server, ta, _cap(a))
    # the mix: others first, A in the middle, more after
    others = _others()
    ts = [_submit(server, r) for r in others[:2]]
    tb = _submit(server, a)
    ts += [_submit(server, r) for r in others[2:]]
    q, active, used = pf.pf_server_stats(server)
    assert active >= 2                      # requests run concurrently
    _drain(server, ts + [tb])
    mixed = pf.pf_server_result(server, tb, _cap(a))
    for x, y in zip(alone[:3], mixed[:3]):
        assert np.array_equal(x, y)
    for t, r in zip(ts, others):
        X, Y, G, lat = pf.pf_server_result(server, t, _cap(r))
        assert np.all(np.isfinite(X)) and lat > 0
    # and through pf_step directly, on a state of the server's instance size (a
    # power of two, at least 1024: the sheet's route is chosen for it)
    g = a["grid"]
    plan = pf.Plan(g[0], g[1], g[2], g[3], g[4], prec)
    state = pf.State(plan, 1024)
    pf.pf_state_set(state, a["X"], a["Y"], a["G"], 0.0)
    for _ in range(a["nsteps"]):
        pf.pf_step(plan, state, a["dt"], a["body"], scheme=a["scheme"])
    pf.pf_sync(plan)
    X, Y, G, t = pf.pf_state_get(state)
    assert np.array_equal(X, alone[0]) and np.array_equal(Y, alone[1]) and np.array_equal(G, alone[2])
    server.close()


def test_admission_respects_the_memory_budget():
    """Same-shape requests under a budget that holds the shape's tables and two
    instances: never more than two resident, the budget never exceeded."""
    reqs = [dict(r, grid=_grid(256)) for r in _others()] * 2
    probe = pf.Server(max_slots=1, hbm_budget_bytes=1 << 30)
    t = _submit(probe, reqs[0])
    one = pf.pf_server_stats(probe)[2]            # tables + one instance
    _drain(probe, [t])
    probe.close()
    budget = int(one * 1.9)                         # instances are about the same size here
    server = pf.Server(max_slots=8, hbm_budget_bytes=budget, precision=pf.PF_MIXED)
    tickets, max_active = [], 0
    for r in reqs:
        tickets.append(_submit(server, r))
        max_active = max(max_active, pf.pf_server_stats(server)[1])
    pending = set(tickets)
    t0 = time.time()
    while pending:
        for t in pf.pf_server_progress(server):
            pending.discard(t)
        q, active, used = pf.pf_server_stats(server)
        max_active = max(max_active, active)
        assert used <= budget
        assert time.time() - t0 < 120
    assert 1 <= max_active <= 2
    for t, r in zip(tickets, reqs):
        pf.pf_server_result(server, t, _cap(r))
    server.close()


def test_submit_checks_capacity():
    a = _request_a()
    server = pf.Server(max_slots=2, hbm_budget_bytes=1 << 30)
    with pytest.raises(pf.GridPfError) as e:
        pf.pf_server_submit(server, a["grid"], a["X"], a["Y"], a["G"], a["nsteps"], a["dt"], a["body"],
                            capacity=len(a["X"]))
    assert e.value.name == "PF_ERR_CAPACITY"
    server.close()


def test_a_request_that_can_never_fit_fails_instead_of_waiting():
    """With nothing else resident, a request whose grid tables and instance
    exceed the budget can never be admitted: it finishes with PF_ERR_OOM (and
    the requests behind it still run once it is out of the way)."""
    a = _request_a()
    big = dict(a, grid=_grid(512))
    probe = pf.Server(max_slots=1, hbm_budget_bytes=1 << 30)
    t = _submit(probe, a)
    one = pf.pf_server_stats(probe)[2]            # 128^2 tables + one instance
    _drain(probe, [t])
    probe.close()
    server = pf.Server(max_slots=4, hbm_budget_bytes=int(one * 1.5), precision=pf.PF_MIXED)
    tb = _submit(server, big)                      # 512^2 needs ~16x the 128^2 footprint
    ta = _submit(server, a)
    done = _drain(server, [tb, ta], timeout=60.0)
    assert set(done) == {tb, ta}
    with pytest.raises(pf.GridPfError) as e:
        pf.pf_server_result(server, tb, _cap(big))
    assert e.value.name == "PF_ERR_OOM"
    X, Y, G, _ = pf.pf_server_result(server, ta, _cap(a))
    assert len(X) == len(a["X"]) + 2 * a["nsteps"] and np.all(np.isfinite(X))
    server.close()
