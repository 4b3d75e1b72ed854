"""Batched steps captured as one CUDA graph (pf_batch_*).

A graph batch runs pf_step's kernels (Sec. 2.4 stepping with the Kutta and
Kelvin sheet solve of Sec. 2.2-2.3) with the vortex counts read on the device
and launches sized by each state's capacity.  With the surface right-hand
side's route pinned, that changes no arithmetic: the states after graph
steps are bitwise those of pf_step.  With the automatic route, an instance
gives bitwise the same result alone and in the batch.
"""
import numpy as np
import pytest
import torch

import paper_2102_11910_gb300 as pf
from paper_2102_11910_gb300 import inputs

pytestmark = pytest.mark.gpu

SHAPES = ((128, 128), (256, 256), (512, 384))


def _instances(n, seed=1003, shapes=SHAPES):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        r = inputs.batched_instance(rng, shape=shapes[i % len(shapes)])
        # keep the instances small enough for a quick test
        m = min(len(r["X"]), 3000)
        r["X"], r["Y"], r["G"] = r["X"][:m], r["Y"][:m], r["G"][:m]
        out.append(r)
    return out


def _build(inst, prec=pf.PF_MIXED, route=None, extra=16, body_free=()):
    plans, states, bodies = [], [], []
    for i, r in enumerate(inst):
        g = r["grid"]
        p = pf.Plan(g.nx, g.ny, g.dx, g.x0, g.y0, prec, stream=torch.cuda.Stream())
        if route is not None:
            pf.pf_plan_set_rhs_route(p, route)
        st = pf.State(p, len(r["X"]) + extra)
        pf.pf_state_set(st, r["X"], r["Y"], r["G"])
        b = r["body"]
        if i in body_free:
            k = pf.no_body(Uinf=r["Uinf"])
        else:
            k = pf.BodyKinematics(b["xb"], b["yb"], b["ds"], b["edges"], b["alpha0"], Uinf=r["Uinf"])
        plans.append(p)
        states.append(st)
        bodies.append(k)
    return plans, states, bodies


def _assert_same_states(sa, sb):
    for s1, s2 in zip(sa, sb):
        a, b = pf.pf_state_get(s1), pf.pf_state_get(s2)
        assert len(a[0]) == len(b[0]) > 0
        for u, v in zip(a[:3], b[:3]):
            assert np.array_equal(u, v)
        assert a[3] == pytest.approx(b[3], abs=1e-15)


@pytest.mark.parametrize("prec", [pf.PF_MIXED, pf.PF_FP64])
@pytest.mark.parametrize("scheme", [0, 1])
def test_graph_steps_are_bitwise_pf_step_with_the_route_pinned(prec, scheme):
    """Plates and ellipses on three grid shapes, one body-free instance; three
    graph steps against three pf_step calls per instance."""
    inst = _instances(6)
    dts = [r["dt"] for r in inst]
    pa, sa, ba = _build(inst, prec, route=pf.PF_RHS_SPARSE, body_free=(5,))
    pb, sb, bb = _build(inst, prec, route=pf.PF_RHS_SPARSE, body_free=(5,))
    batch = pf.Batch(pa, sa, ba, dts, scheme)
    batch.step(2)
    batch.step(1)
    for p, st, b, dt in zip(pb, sb, bb, dts):
        for _ in range(3):
            pf.pf_step(p, st, dt, b, scheme=scheme)
    for p in pa + pb:
        pf.pf_sync(p)
    _assert_same_states(sa, sb)
    # stepping on with pf_step after the graph keeps both in lock step
    for p, st, b, dt in zip(pa, sa, ba, dts):
        pf.pf_step(p, st, dt, b, scheme=scheme)
    for p, st, b, dt in zip(pb, sb, bb, dts):
        pf.pf_step(p, st, dt, b, scheme=scheme)
    for p in pa + pb:
        pf.pf_sync(p)
    _assert_same_states(sa, sb)
    batch.close()


def test_each_instance_is_bitwise_the_same_alone_and_in_the_batch():
    """Automatic route (chosen for each state's capacity): eight instances in
    one graph against each in a graph of its own."""
    inst = _instances(8, seed=1007)
    dts = [r["dt"] for r in inst]
    pa, sa, ba = _build(inst)
    batch = pf.Batch(pa, sa, ba, dts)
    batch.step(3)
    alone = []
    for r, dt in zip(inst, dts):
        p, s, b = _build([r])
        one = pf.Batch(p, s, b, [dt])
        one.step(3)
        alone.append((p[0], s[0], one))
    for p in pa:
        pf.pf_sync(p)
    for p, _, _ in alone:
        pf.pf_sync(p)
    _assert_same_states(sa, [s for _, s, _ in alone])


def test_batch_reports_capacity_before_launching():
    inst = _instances(2)
    pa, sa, ba = _build(inst, extra=4)          # room for two steps of two releases
    batch = pf.Batch(pa, sa, ba, [r["dt"] for r in inst])
    before = [pf.pf_state_get(s) for s in sa]
    with pytest.raises(pf.GridPfError) as e:
        batch.step(3)
    assert e.value.name == "PF_ERR_CAPACITY"
    for s, b in zip(sa, before):
        a = pf.pf_state_get(s)
        assert np.array_equal(a[0], b[0]) and a[3] == b[3]
    batch.step(2)
    for p in pa:
        pf.pf_sync(p)
    assert [len(pf.pf_state_get(s)[0]) for s in sa] == [len(b[0]) + (4 if len(r["body"]["edges"]) else 0)
                                                       for b, r in zip(before, inst)]


def test_batch_rejects_what_a_fixed_graph_cannot_run():
    inst = _instances(2)
    pa, sa, ba = _build(inst)
    dts = [r["dt"] for r in inst]
    pitching = pf.plate_kinematics(32, 1.0, 0.5, 0.1, 1.0, Uinf=1.0)
    cases = [
        ([pa[0], pa[0]], [sa[0], sa[1]], ba, dts),          # one plan twice
        ([pa[0], pa[1]], [sa[0], sa[0]], ba, dts),          # one state twice
        ([pa[1], pa[0]], sa, ba, dts),                      # state of another plan
        (pa, sa, [ba[0], pitching], dts),                   # pose changes in time
        (pa, sa, ba, [dts[0], 0.0]),                        # no step length
    ]
    for plans, states, bodies, dt in cases:
        with pytest.raises(pf.GridPfError) as e:
            pf.Batch(plans, states, bodies, dt)
        assert e.value.name == "PF_ERR_ARG"
    pf.pf_timing_enable(pa[0], True)
    with pytest.raises(pf.GridPfError) as e:
        pf.Batch(pa, sa, ba, dts)
    assert e.value.name == "PF_ERR_ARG"
    pf.pf_timing_enable(pa[0], False)
    legacy = pf.Plan(128, 128, 0.02, -1.27, -1.27, pf.PF_MIXED, stream=torch.cuda.default_stream())
    st = pf.State(legacy, 10)
    with pytest.raises(pf.GridPfError) as e:
        pf.Batch([legacy], [st], [pf.no_body(Uinf=1.0)], [0.01])
    assert e.value.name == "PF_ERR_ARG"
