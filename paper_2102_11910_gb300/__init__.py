"""GB300 implementation of the grid potential-flow vortex method of
Beckers & Eldredge, "Planar potential flow on Cartesian grids" (arXiv 2102.11910).

The computation lives in the CUDA library ``libgridpf.so`` (C ABI declared in
``include/gridpf.h``).  This module only marshals torch tensors to that ABI:
each function has the C entry point's name and forwards device pointers and
sizes.  PyTorch provides device memory and the current CUDA stream.
"""
import ctypes
import os

import torch

from . import _native
from ._native import GridPfError

PF_FP64 = 0
PF_MIXED = 1
# status codes (include/gridpf.h)
(PF_OK, PF_ERR_ARG, PF_ERR_OOM, PF_ERR_CUDA, PF_ERR_OUT_OF_DOMAIN, PF_ERR_SINGULAR, PF_ERR_TIMEOUT,
 PF_ERR_NOT_FACTORED, PF_ERR_CAPACITY, PF_ERR_INTERNAL) = range(10)


def _ptr(t, dtype=None, name="tensor"):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """Handle of a pf_plan (one grid, one precision, one CUDA stream)."""

    def __init__(self, nx, ny, dx, x0, y0, precision=PF_MIXED, stream=None):
        L = _native.lib()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.nx, self.ny, self.dx, self.x0, self.y0 = int(nx), int(ny), float(dx), float(x0), float(y0)
        self.precision = int(precision)
        self.dtype = torch.float64 if self.precision == PF_FP64 else torch.float32
        desc = _native.PfGridDesc(self.nx, self.ny, self.dx, self.x0, self.y0, self.precision)
        h = ctypes.c_void_p()
        _native.check(L.pf_plan_create(ctypes.byref(desc), ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h)),
                      "pf_plan_create")
        self.handle = h
        P, Q = ctypes.c_int32(), ctypes.c_int32()
        _native.check(L.pf_plan_fft_size(h, ctypes.byref(P), ctypes.byref(Q)), "pf_plan_fft_size", h)
        self.P, self.Q = P.value, Q.value

    def close(self):
        if getattr(self, "handle", None):
            _native.lib().pf_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def field(self, comps=1):
        shape = (self.ny, self.nx) if comps == 1 else (self.ny, self.nx, comps)
        return torch.empty(shape, dtype=self.dtype, device="cuda")


def pf_plan_clone(src, precision=None, stream=None):
    """A plan on `stream` sharing src's LGF tables and spectra (own workspaces)."""
    precision = src.precision if precision is None else int(precision)
    stream = torch.cuda.current_stream() if stream is None else stream
    p = Plan.__new__(Plan)
    p.stream = stream
    p.nx, p.ny, p.dx, p.x0, p.y0, p.P, p.Q = src.nx, src.ny, src.dx, src.x0, src.y0, src.P, src.Q
    p.precision = precision
    p.dtype = torch.float64 if precision == PF_FP64 else torch.float32
    h = ctypes.c_void_p()
    _native.check(_native.lib().pf_plan_clone(src.handle, precision, ctypes.c_void_p(stream.cuda_stream),
                                              ctypes.byref(h)), "pf_plan_clone", src.handle)
    p.handle = h
    return p


def pf_plan_create(nx, ny, dx, x0, y0, precision=PF_MIXED, stream=None):
    return Plan(nx, ny, dx, x0, y0, precision, stream)


def pf_plan_destroy(plan):
    plan.close()


def pf_sync(plan):
    """Wait for the plan's stream; raise GridPfError on a sticky error.  Returns
    the number of out-of-domain points (0 when there were none)."""
    n = ctypes.c_int64()
    st = _native.lib().pf_sync(plan.handle, ctypes.byref(n))
    if st != 0 and st != 4:
        _native.check(st, "pf_sync", plan.handle)
    if st == 4:
        raise GridPfError(st, "pf_sync", "%d points out of domain" % n.value)
    return n.value


def pf_lgf_table(plan):
    import numpy as np
    out = np.empty((plan.ny + 1, plan.nx + 1), dtype=np.float64)
    _native.check(_native.lib().pf_lgf_table(plan.handle, out.ctypes.data_as(ctypes.c_void_p)), "pf_lgf_table",
                  plan.handle)
    return out


def pf_regularize(plan, X, Y, G, w=None):
    w = plan.field() if w is None else w
    nv = X.numel()
    _native.check(_native.lib().pf_regularize(plan.handle, _ptr(X, torch.float64, "X"), _ptr(Y, torch.float64, "Y"),
                                              _ptr(G, torch.float64, "G"), nv, _ptr(w, plan.dtype, "w")),
                  "pf_regularize", plan.handle)
    return w


def pf_poisson_solve(plan, w, psi=None):
    psi = plan.field() if psi is None else psi
    _native.check(_native.lib().pf_poisson_solve(plan.handle, _ptr(w, plan.dtype, "w"), _ptr(psi, plan.dtype, "psi")),
                  "pf_poisson_solve", plan.handle)
    return psi


def pf_velocity_solve(plan, w, Uinf=0.0, Vinf=0.0, uv=None):
    uv = plan.field(2) if uv is None else uv
    _native.check(_native.lib().pf_velocity_solve(plan.handle, _ptr(w, plan.dtype, "w"), float(Uinf), float(Vinf),
                                                  _ptr(uv, plan.dtype, "uv")), "pf_velocity_solve", plan.handle)
    return uv


def pf_interpolate(plan, uv, Xq, Yq, uq=None, vq=None):
    n = Xq.numel()
    uq = torch.empty(n, dtype=plan.dtype, device="cuda") if uq is None else uq
    vq = torch.empty(n, dtype=plan.dtype, device="cuda") if vq is None else vq
    _native.check(_native.lib().pf_interpolate(plan.handle, _ptr(uv, plan.dtype, "uv"), _ptr(Xq, torch.float64, "Xq"),
                                               _ptr(Yq, torch.float64, "Yq"), n, _ptr(uq, plan.dtype, "uq"),
                                               _ptr(vq, plan.dtype, "vq")), "pf_interpolate", plan.handle)
    return uq, vq


def pf_vic_velocity(plan, X, Y, G, Uinf=0.0, Vinf=0.0, uq=None, vq=None):
    n = X.numel()
    uq = torch.empty(n, dtype=plan.dtype, device="cuda") if uq is None else uq
    vq = torch.empty(n, dtype=plan.dtype, device="cuda") if vq is None else vq
    _native.check(_native.lib().pf_vic_velocity(plan.handle, _ptr(X, torch.float64, "X"), _ptr(Y, torch.float64, "Y"),
                                                _ptr(G, torch.float64, "G"), n, float(Uinf), float(Vinf),
                                                _ptr(uq, plan.dtype, "uq"), _ptr(vq, plan.dtype, "vq")),
                  "pf_vic_velocity", plan.handle)
    return uq, vq


def pf_vic_velocity_host(plan, X, Y, G, Uinf=0.0, Vinf=0.0, uq=None, vq=None):
    """Host-buffer variant: X, Y, G, uq, vq are CPU tensors (pinned recommended)."""
    n = X.numel()
    for t, nm in ((X, "X"), (Y, "Y"), (G, "G")):
        if t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
            raise ValueError("%s must be a contiguous CPU float64 tensor" % nm)
    uq = torch.empty(n, dtype=plan.dtype) if uq is None else uq
    vq = torch.empty(n, dtype=plan.dtype) if vq is None else vq
    c = ctypes.c_void_p
    _native.check(_native.lib().pf_vic_velocity_host(plan.handle, c(X.data_ptr()), c(Y.data_ptr()), c(G.data_ptr()), n,
                                                     float(Uinf), float(Vinf), c(uq.data_ptr()), c(vq.data_ptr())),
                  "pf_vic_velocity_host", plan.handle)
    return uq, vq


def pf_vic_velocity_host_async(plan, X, Y, G, Uinf, Vinf, uq, vq):
    """Asynchronous host-buffer step: queues the copies in, the step and the
    copies out on the plan's stream and returns.  X, Y, G, uq, vq are CPU
    tensors (page-locked for the copies to overlap other work); they are in use
    until pf_sync(plan) returns."""
    n = X.numel()
    for t, nm in ((X, "X"), (Y, "Y"), (G, "G")):
        if t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous() or t.numel() != n:
            raise ValueError("%s must be a contiguous CPU float64 tensor of %d elements" % (nm, n))
    for t, nm in ((uq, "uq"), (vq, "vq")):
        if t.is_cuda or t.dtype != plan.dtype or not t.is_contiguous() or t.numel() != n:
            raise ValueError("%s must be a contiguous CPU %s tensor of %d elements" % (nm, plan.dtype, n))
    c = ctypes.c_void_p
    _native.check(_native.lib().pf_vic_velocity_host_async(plan.handle, c(X.data_ptr()), c(Y.data_ptr()),
                                                           c(G.data_ptr()), n, float(Uinf), float(Vinf),
                                                           c(uq.data_ptr()), c(vq.data_ptr())),
                  "pf_vic_velocity_host_async", plan.handle)


def pf_timing_enable(plan, on=True):
    _native.check(_native.lib().pf_timing_enable(plan.handle, 1 if on else 0), "pf_timing_enable", plan.handle)


def _config_dict(c):
    return {"tile": c.tile, "min_span": c.min_span, "tile_threads": c.tile_threads, "fft": c.fft}


def pf_launch_config_get(plan):
    """The plan's launch configuration: {tile, min_span, tile_threads, fft}."""
    c = _native.PfLaunchConfig()
    _native.check(_native.lib().pf_launch_config_get(plan.handle, ctypes.byref(c)), "pf_launch_config_get",
                  plan.handle)
    return _config_dict(c)


def pf_launch_config_set(plan, tile=None, min_span=None, tile_threads=None, fft=None):
    """Set some or all of the plan's launch configuration (the others kept)."""
    cur = pf_launch_config_get(plan)
    for k, v in (("tile", tile), ("min_span", min_span), ("tile_threads", tile_threads), ("fft", fft)):
        if v is not None:
            cur[k] = int(v)
    c = _native.PfLaunchConfig(cur["tile"], cur["min_span"], cur["tile_threads"], cur["fft"])
    _native.check(_native.lib().pf_launch_config_set(plan.handle, ctypes.byref(c)), "pf_launch_config_set",
                  plan.handle)


def pf_autotune(plan, nv, cache_path=None, reps=5):
    """Time every launch configuration on nv synthetic vortices, set the fastest
    (or the one cached under this device, grid, precision and nv's power of two
    in the text file cache_path); returns (config dict, median microseconds)."""
    c = _native.PfLaunchConfig()
    us = ctypes.c_double()
    path = None if cache_path is None else os.fsencode(cache_path)
    _native.check(_native.lib().pf_autotune(plan.handle, int(nv), path, int(reps), ctypes.byref(c), ctypes.byref(us)),
                  "pf_autotune", plan.handle)
    return _config_dict(c), us.value


def pf_timing_report(plan):
    """Per-kernel CUDA-event times since timing was enabled: {name: (launches, total_ms)}."""
    buf = ctypes.create_string_buffer(1 << 16)
    _native.check(_native.lib().pf_timing_report(plan.handle, buf, len(buf)), "pf_timing_report", plan.handle)
    out = {}
    for line in buf.value.decode().splitlines():
        name, n, ms = line.split()
        out[name] = (int(n), float(ms))
    return out


class VicState:
    """Handle of a pf_vic_state: a tile-ordered vortex set stepped on `plan`'s
    stream (body-free vortex-in-cell, forward Euler)."""

    def __init__(self, plan, capacity):
        self.plan = plan
        h = ctypes.c_void_p()
        _native.check(_native.lib().pf_vic_state_create(plan.handle, int(capacity), ctypes.byref(h)),
                      "pf_vic_state_create", plan.handle)
        self.handle = h
        self.nv0 = 0

    def close(self):
        if getattr(self, "handle", None):
            _native.lib().pf_vic_state_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pf_vic_state_set(state, X, Y, G):
    n = X.numel()
    if Y.numel() != n or G.numel() != n:
        raise ValueError("X, Y and G must have the same length")
    _native.check(_native.lib().pf_vic_state_set(state.handle, _ptr(X, torch.float64, "X"), _ptr(Y, torch.float64, "Y"),
                                                 _ptr(G, torch.float64, "G"), n),
                  "pf_vic_state_set", state.plan.handle)
    state.nv0 = n


def pf_vic_state_get(state):
    """(X, Y, G, nv, t): device FP64 tensors indexed like the set call's input."""
    n = state.nv0
    X, Y, G = (torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(3))
    nv = ctypes.c_int64()
    t = ctypes.c_double()
    _native.check(_native.lib().pf_vic_state_get(state.handle, _ptr(X), _ptr(Y), _ptr(G), ctypes.byref(nv),
                                                 ctypes.byref(t)),
                  "pf_vic_state_get", state.plan.handle)
    return X, Y, G, nv.value, t.value


def pf_vic_step(state, dt, Uinf=0.0, Vinf=0.0, uq=None, vq=None):
    """One Euler step; with uq, vq (device tensors of the plan's precision) the
    velocities the vortices moved with are written at their indices."""
    dtype = state.plan.dtype
    if (uq is None) != (vq is None):
        raise ValueError("give both uq and vq or neither")
    if uq is not None and (uq.numel() < state.nv0 or vq.numel() < state.nv0):
        raise ValueError("uq and vq must hold the set call's vortex count")
    _native.check(_native.lib().pf_vic_step(state.handle, float(dt), float(Uinf), float(Vinf),
                                            _ptr(uq, dtype, "uq"), _ptr(vq, dtype, "vq")),
                  "pf_vic_step", state.plan.handle)


def pf_regularize_noalloc(nx, ny, dx, x0, y0, precision, X, Y, G, w, out_of_domain=None, status=None, stream=None):
    """Allocation-free regularization (no plan; static device scratch, nv <= 65536).

    `w` must be a preallocated CUDA tensor of ny*nx elements of the precision's
    dtype; `out_of_domain` an optional CUDA int64 tensor and `status` an
    optional CUDA int32 tensor of at least one element, which receive the
    out-of-domain count and the device-side status code.  Every tensor must be
    on the current CUDA device (the library resolves its scratch there)."""
    desc = _native.PfGridDesc(int(nx), int(ny), float(dx), float(x0), float(y0), int(precision))
    dtype = torch.float64 if int(precision) == PF_FP64 else torch.float32
    nv = X.numel()
    if Y.numel() != nv or G.numel() != nv:
        raise ValueError("X, Y and G must have the same length")
    if w.numel() != int(nx) * int(ny):
        raise ValueError("w must hold nx*ny = %d elements, got %d" % (int(nx) * int(ny), w.numel()))
    if out_of_domain is not None and out_of_domain.numel() < 1:
        raise ValueError("out_of_domain must hold at least one element")
    if status is not None and status.numel() < 1:
        raise ValueError("status must hold at least one element")
    dev = torch.cuda.current_device()
    for name, t in (("X", X), ("Y", Y), ("G", G), ("w", w), ("out_of_domain", out_of_domain), ("status", status)):
        if t is not None and t.is_cuda and t.device.index != dev:
            raise ValueError("%s is on cuda:%d, the current device is cuda:%d" % (name, t.device.index, dev))
    if stream is None:
        stream = torch.cuda.current_stream()
    st = _native.lib().pf_regularize_noalloc(ctypes.byref(desc), _ptr(X, torch.float64, "X"), _ptr(Y, torch.float64, "Y"),
                                             _ptr(G, torch.float64, "G"), nv, _ptr(w, dtype, "w"),
                                             _ptr(out_of_domain, torch.int64, "out_of_domain"),
                                             _ptr(status, torch.int32, "status"), ctypes.c_void_p(stream.cuda_stream))
    _native.check(st, "pf_regularize_noalloc")
    return w


PF_SHEET_GIVEN_S0 = 0
PF_SHEET_CIRCULATION = 1
PF_SHEET_KUTTA_STEADY = 2
PF_SHEET_KUTTA_SHED = 3


class Schur:
    """Handle of a pf_schur (factorised Schur complement of one body on a plan's grid)."""

    def __init__(self, plan, handle, ns):
        self.plan, self.handle, self.ns = plan, handle, ns

    def close(self):
        if getattr(self, "handle", None):
            _native.lib().pf_schur_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _host_f64(a):
    import numpy as np
    return np.ascontiguousarray(a, dtype=np.float64)


def pf_schur_factor(plan, x, y, ds):
    """Factor S = -E L^-1 R_s for surface points (x, y) with segment lengths ds (host arrays)."""
    x, y, ds = _host_f64(x), _host_f64(y), _host_f64(ds)
    c = ctypes.c_void_p
    desc = _native.PfBodyDesc(len(x), c(x.ctypes.data), c(y.ctypes.data), c(ds.ctypes.data))
    h = ctypes.c_void_p()
    _native.check(_native.lib().pf_schur_factor(plan.handle, ctypes.byref(desc), ctypes.byref(h)), "pf_schur_factor",
                  plan.handle)
    return Schur(plan, h, len(x))


def pf_schur_info(schur):
    """(Gamma0, f0, S) as host numpy arrays."""
    import numpy as np
    g = ctypes.c_double()
    f0 = np.empty(schur.ns)
    S = np.empty((schur.ns, schur.ns))
    _native.check(_native.lib().pf_schur_info(schur.handle, ctypes.byref(g), f0.ctypes.data_as(ctypes.c_void_p),
                                              S.ctypes.data_as(ctypes.c_void_p)), "pf_schur_info", schur.plan.handle)
    return g.value, f0, S


def pf_sheet_solve(plan, schur, w, motion, mode, param=0.0, edges=(), Xnew=None, Ynew=None, f=None):
    """Bound sheet for free vorticity w (device field).  motion = (U, V, Omega, Uinf, Vinf).
    Returns (f device float64 tensor, gamma_new host list, s0)."""
    import numpy as np
    f = torch.empty(schur.ns, dtype=torch.float64, device="cuda") if f is None else f
    ed = np.ascontiguousarray(edges, dtype=np.int32)
    ne = len(ed)
    xn = _host_f64(Xnew if Xnew is not None else np.zeros(max(ne, 1)))
    yn = _host_f64(Ynew if Ynew is not None else np.zeros(max(ne, 1)))
    gn = np.zeros(max(ne, 1))
    s0 = ctypes.c_double()
    m = _native.PfMotion(*[float(v) for v in motion])
    c = ctypes.c_void_p
    _native.check(_native.lib().pf_sheet_solve(plan.handle, schur.handle, _ptr(w, plan.dtype, "w"), ctypes.byref(m),
                                               int(mode), float(param), ne, c(ed.ctypes.data) if ne else None,
                                               c(xn.ctypes.data), c(yn.ctypes.data), _ptr(f, torch.float64, "f"),
                                               c(gn.ctypes.data), ctypes.byref(s0)), "pf_sheet_solve", plan.handle)
    return f, list(gn[:ne]), s0.value


def pf_sheet_solve_vortices(plan, schur, X, Y, G, motion, mode, param=0.0, edges=(), Xnew=None, Ynew=None, f=None):
    """Bound sheet for the free vorticity of point vortices (device FP64 X, Y, G),
    E_s L^-1 R_v Gamma summed in FP64 from the vortices themselves.
    Returns (f device float64 tensor, gamma_new host list, s0)."""
    import numpy as np
    n = X.numel()
    if Y.numel() != n or G.numel() != n:
        raise ValueError("X, Y and G must have the same length")
    f = torch.empty(schur.ns, dtype=torch.float64, device="cuda") if f is None else f
    ed = np.ascontiguousarray(edges, dtype=np.int32)
    ne = len(ed)
    xn = _host_f64(Xnew if Xnew is not None else np.zeros(max(ne, 1)))
    yn = _host_f64(Ynew if Ynew is not None else np.zeros(max(ne, 1)))
    gn = np.zeros(max(ne, 1))
    s0 = ctypes.c_double()
    m = _native.PfMotion(*[float(v) for v in motion])
    c = ctypes.c_void_p
    _native.check(_native.lib().pf_sheet_solve_vortices(
        plan.handle, schur.handle, _ptr(X, torch.float64, "X"), _ptr(Y, torch.float64, "Y"),
        _ptr(G, torch.float64, "G"), n, ctypes.byref(m), int(mode), float(param), ne, c(ed.ctypes.data) if ne else None,
        c(xn.ctypes.data), c(yn.ctypes.data), _ptr(f, torch.float64, "f"), c(gn.ctypes.data), ctypes.byref(s0)),
        "pf_sheet_solve_vortices", plan.handle)
    return f, list(gn[:ne]), s0.value


PF_MAX_BODIES = _native.MAX_BODIES


def pf_sheet_solve_multi(plan, schur, w, starts, edges, motions, gamma_w, Xnew=None, Ynew=None, f=None):
    """Several bodies sharing one factor (pf_sheet_solve_multi).  starts: the
    B + 1 point offsets of the bodies in the factor; edges: per body a tuple of
    0-2 surface indices; motions: per body (U, V, Omega, Uinf, Vinf) (the free
    stream is the first body's), or one tuple for all; gamma_w: per body.
    Xnew, Ynew: one new vortex per edge, edges in body order.
    Returns (f device float64 tensor, gamma_new array, s0 array)."""
    import numpy as np
    nb = len(starts) - 1
    if nb < 1 or nb > PF_MAX_BODIES or len(edges) != nb or len(gamma_w) != nb:
        raise ValueError("between 1 and %d bodies, with edges and gamma_w per body" % PF_MAX_BODIES)
    if len(motions) == 5 and not hasattr(motions[0], "__len__"):
        motions = [motions] * nb
    mb = _native.PfMultibody()
    mb.n_bodies = nb
    for b in range(nb + 1):
        mb.start[b] = int(starts[b])
    for b in range(nb):
        if len(edges[b]) > 2:
            raise ValueError("at most two edges per body")
        mb.n_edges[b] = len(edges[b])
        for j, k in enumerate(edges[b]):
            mb.edge[b][j] = int(k)
        mb.motion[b] = _native.PfMotion(*[float(v) for v in motions[b]])
        mb.gamma_w[b] = float(gamma_w[b])
    ne = sum(len(e) for e in edges)
    f = torch.empty(schur.ns, dtype=torch.float64, device="cuda") if f is None else f
    xn = _host_f64(Xnew if Xnew is not None else np.zeros(max(ne, 1)))
    yn = _host_f64(Ynew if Ynew is not None else np.zeros(max(ne, 1)))
    if len(xn) < ne or len(yn) < ne:
        raise ValueError("one new vortex per edge")
    gn = np.zeros(max(ne, 1))
    s0 = np.zeros(nb)
    c = ctypes.c_void_p
    _native.check(_native.lib().pf_sheet_solve_multi(plan.handle, schur.handle, _ptr(w, plan.dtype, "w"),
                                                     ctypes.byref(mb), c(xn.ctypes.data), c(yn.ctypes.data),
                                                     _ptr(f, torch.float64, "f"), c(gn.ctypes.data),
                                                     c(s0.ctypes.data)), "pf_sheet_solve_multi", plan.handle)
    return f, gn[:ne].copy(), s0


def pf_step_multi(plan, state, dt, bodies, scheme=0):
    """One step around several bodies (a list of BodyKinematics, at most
    PF_MAX_BODIES; the free stream is the first one's)."""
    if not 1 <= len(bodies) <= PF_MAX_BODIES:
        raise ValueError("between 1 and %d bodies" % PF_MAX_BODIES)
    arr = (_native.PfBodyKinematics * len(bodies))(*[b.struct for b in bodies])
    _native.check(_native.lib().pf_step_multi(plan.handle, state.handle, len(bodies), arr, float(dt), int(scheme)),
                  "pf_step_multi", plan.handle)


def pf_sheet_regularize(plan, schur, f, w):
    """w += R_s f in place (device tensors: f float64 of ns, w of the plan's precision)."""
    _native.check(_native.lib().pf_sheet_regularize(plan.handle, schur.handle, _ptr(f, torch.float64, "f"),
                                                    _ptr(w, plan.dtype, "w")), "pf_sheet_regularize", plan.handle)
    return w


def pf_pressure_setup(plan, schur, nx, ny):
    """Unit surface normals (host arrays) and the factor of the jump operator (Sec. 2.6.1)."""
    nx, ny = _host_f64(nx), _host_f64(ny)
    c = ctypes.c_void_p
    _native.check(_native.lib().pf_pressure_setup(plan.handle, schur.handle, c(nx.ctypes.data), c(ny.ctypes.data)),
                  "pf_pressure_setup", plan.handle)


def pf_potential_jump(plan, schur, f, dphi=None):
    """Delta phi of the sheet f (device float64 tensors)."""
    dphi = torch.empty(schur.ns, dtype=torch.float64, device="cuda") if dphi is None else dphi
    _native.check(_native.lib().pf_potential_jump(plan.handle, schur.handle, _ptr(f, torch.float64, "f"),
                                                  _ptr(dphi, torch.float64, "dphi")), "pf_potential_jump", plan.handle)
    return dphi


def pf_pressure_jump(plan, schur, psi, motion, f, dphi_dt=None, rho=1.0, dp=None):
    """Delta p across the surface (Eq. surfbernoulli); motion = (U, V, Omega, Uinf, Vinf)."""
    dp = torch.empty(schur.ns, dtype=torch.float64, device="cuda") if dp is None else dp
    m = _native.PfMotion(*[float(v) for v in motion])
    _native.check(_native.lib().pf_pressure_jump(plan.handle, schur.handle, _ptr(psi, plan.dtype, "psi"),
                                                 ctypes.byref(m), _ptr(f, torch.float64, "f"),
                                                 _ptr(dphi_dt, torch.float64, "dphi_dt") if dphi_dt is not None else None,
                                                 float(rho), _ptr(dp, torch.float64, "dp")), "pf_pressure_jump",
                  plan.handle)
    return dp


def pf_pressure_field(plan, psi, w, motion, schur=None, f=None, dphi_dt=None, rho=1.0, p=None):
    """Pressure at the cell centres (Eq. pgrid), a (ny-1, nx-1) float64 device tensor.
    motion = (U, V, Omega, Uinf, Vinf); schur, f, dphi_dt: the surface terms (optional)."""
    p = torch.empty((plan.ny - 1, plan.nx - 1), dtype=torch.float64, device="cuda") if p is None else p
    m = _native.PfMotion(*[float(v) for v in motion])
    _native.check(_native.lib().pf_pressure_field(plan.handle, schur.handle if schur is not None else None,
                                                  _ptr(psi, plan.dtype, "psi"), _ptr(w, plan.dtype, "w"),
                                                  ctypes.byref(m), _ptr(f, torch.float64, "f"),
                                                  _ptr(dphi_dt, torch.float64, "dphi_dt"), float(rho),
                                                  _ptr(p, torch.float64, "p")), "pf_pressure_field", plan.handle)
    return p


PF_RHS_AUTO, PF_RHS_DIRECT, PF_RHS_FFT, PF_RHS_SPARSE = 0, 1, 2, 3


def pf_plan_set_rhs_route(plan, route):
    """Route of E_s L^-1 w in the sheet solves: PF_RHS_AUTO, PF_RHS_DIRECT, PF_RHS_FFT or PF_RHS_SPARSE."""
    _native.check(_native.lib().pf_plan_set_rhs_route(plan.handle, int(route)), "pf_plan_set_rhs_route", plan.handle)


def pf_impulse(plan, w, x=None, y=None, ds=None, f=None, nx=None, ny=None, motion=None):
    """(P_x, P_y, Pi_O) of the fluid about the origin for node vorticity w (device
    field) and, optionally, a surface (host arrays x, y, ds, normals nx, ny) with
    its sheet strength f (device float64).  motion = (U, V, Omega) of the body."""
    import numpy as np
    c = ctypes.c_void_p
    desc = None
    keep = []
    if x is not None:
        x, y, ds = _host_f64(x), _host_f64(y), _host_f64(ds)
        keep += [x, y, ds]
        desc = _native.PfBodyDesc(len(x), c(x.ctypes.data), c(y.ctypes.data), c(ds.ctypes.data))
    pn = [None, None]
    if nx is not None:
        nx, ny = _host_f64(nx), _host_f64(ny)
        keep += [nx, ny]
        pn = [c(nx.ctypes.data), c(ny.ctypes.data)]
    m = _native.PfMotion(*(list(float(v) for v in motion) + [0.0, 0.0])) if motion is not None else None
    out = np.zeros(3)
    _native.check(_native.lib().pf_impulse(plan.handle, _ptr(w, plan.dtype, "w"),
                                           ctypes.byref(desc) if desc is not None else None, pn[0], pn[1],
                                           _ptr(f, torch.float64, "f") if f is not None else None,
                                           ctypes.byref(m) if m is not None else None,
                                           c(out.ctypes.data)), "pf_impulse", plan.handle)
    return out


def pf_sheet_solve_edges(plan, schur, w, motion, gamma_w, edges, bounds, Xnew, Ynew, f=None):
    """Generalized edge condition: bounds = ((lo0, hi0)[, (lo1, hi1)]) on the edge
    values of ftilde.  Returns (f device float64 tensor, gamma_new host list, s0)."""
    import numpy as np
    f = torch.empty(schur.ns, dtype=torch.float64, device="cuda") if f is None else f
    ed = np.ascontiguousarray(edges, dtype=np.int32)
    ne = len(ed)
    bd = _host_f64([v for pair in bounds for v in pair])
    xn, yn = _host_f64(Xnew), _host_f64(Ynew)
    gn = np.zeros(ne)
    s0 = ctypes.c_double()
    m = _native.PfMotion(*[float(v) for v in motion])
    c = ctypes.c_void_p
    _native.check(_native.lib().pf_sheet_solve_edges(plan.handle, schur.handle, _ptr(w, plan.dtype, "w"),
                                                     ctypes.byref(m), float(gamma_w), ne, c(ed.ctypes.data),
                                                     c(bd.ctypes.data), c(xn.ctypes.data), c(yn.ctypes.data),
                                                     _ptr(f, torch.float64, "f"), c(gn.ctypes.data), ctypes.byref(s0)),
                  "pf_sheet_solve_edges", plan.handle)
    return f, list(gn), s0.value


class State:
    """Handle of a pf_state (device-resident vortex set)."""

    def __init__(self, plan, capacity):
        h = ctypes.c_void_p()
        _native.check(_native.lib().pf_state_create(plan.handle, int(capacity), ctypes.byref(h)), "pf_state_create",
                      plan.handle)
        self.plan, self.handle, self.capacity = plan, h, int(capacity)

    def close(self):
        if getattr(self, "handle", None):
            _native.lib().pf_state_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pf_state_create(plan, capacity):
    return State(plan, capacity)


def pf_state_set(state, X, Y, G, t=0.0):
    X, Y, G = _host_f64(X), _host_f64(Y), _host_f64(G)
    c = ctypes.c_void_p
    _native.check(_native.lib().pf_state_set(state.handle, c(X.ctypes.data), c(Y.ctypes.data), c(G.ctypes.data),
                                             len(X), float(t)), "pf_state_set", state.plan.handle)


def pf_state_get(state):
    """(X, Y, G, t) as host numpy arrays."""
    import numpy as np
    X = np.empty(state.capacity)
    Y = np.empty(state.capacity)
    G = np.empty(state.capacity)
    nv = ctypes.c_int64()
    t = ctypes.c_double()
    c = ctypes.c_void_p
    _native.check(_native.lib().pf_state_get(state.handle, c(X.ctypes.data), c(Y.ctypes.data), c(G.ctypes.data),
                                             ctypes.byref(nv), ctypes.byref(t)), "pf_state_get", state.plan.handle)
    n = nv.value
    return X[:n].copy(), Y[:n].copy(), G[:n].copy(), t.value


class BodyKinematics:
    """A rigid body in its own frame (host arrays), pitching about the origin:
    world = body turned by -alpha(t), alpha(t) = alpha0 + amp sin(omega t).
    edges: () for a Kelvin-constrained body, or the two surface-point indices
    at which vortices are released."""

    def __init__(self, xb, yb, ds, edges=(), alpha0=0.0, amp=0.0, omega=0.0, Uinf=0.0, Vinf=0.0, edge_bounds=None):
        """edge_bounds: None (Kutta) or ((lo0, hi0), (lo1, hi1)) for the generalized edge condition."""
        self.xb, self.yb, self.ds = _host_f64(xb), _host_f64(yb), _host_f64(ds)
        e = list(edges)
        c = ctypes.c_void_p
        eb = [float(v) for pair in edge_bounds for v in pair] if edge_bounds is not None else [0.0] * 4
        self.struct = _native.PfBodyKinematics(len(self.xb), c(self.xb.ctypes.data), c(self.yb.ctypes.data),
                                               c(self.ds.ctypes.data), len(e), (ctypes.c_int32 * 2)(*(e + [0, 0])[:2]),
                                               float(alpha0), float(amp), float(omega), float(Uinf), float(Vinf),
                                               1 if edge_bounds is not None else 0, (ctypes.c_double * 4)(*eb))


def plate_kinematics(ns, chord=1.0, alpha0=0.0, amp=0.0, omega=0.0, Uinf=0.0, Vinf=0.0):
    """Flat plate along the body x axis (ns segment midpoints, leading edge first),
    releasing vortices at both ends."""
    import numpy as np
    xi = -1.0 + (2.0 * np.arange(1, ns + 1) - 1.0) / ns
    return BodyKinematics(0.5 * chord * xi, np.zeros(ns), np.full(ns, chord / ns), (0, ns - 1), alpha0, amp, omega,
                          Uinf, Vinf)


def no_body(Uinf=0.0, Vinf=0.0):
    k = BodyKinematics([], [], [], (), 0.0, 0.0, 0.0, Uinf, Vinf)
    return k


def pf_step(plan, state, dt, body=None, scheme=0):
    """Advance the state by dt (scheme 0 Euler, 1 RK2) with an optional BodyKinematics."""
    body = no_body() if body is None else body
    _native.check(_native.lib().pf_step(plan.handle, state.handle, ctypes.byref(body.struct), float(dt), int(scheme)),
                  "pf_step", plan.handle)


def pf_step_batch(plans, states, bodies, dt, scheme=0):
    """One step of many independent instances (each on its own plan's stream;
    a large batch of distinct plans and states is enqueued from several host
    threads).  dt: one step length for all, or one per instance."""
    n = len(plans)
    P = (ctypes.c_void_p * n)(*[p.handle.value for p in plans])
    S = (ctypes.c_void_p * n)(*[s.handle.value for s in states])
    B = (_native.PfBodyKinematics * n)(*[b.struct for b in bodies])
    dts = [float(dt)] * n if not hasattr(dt, "__len__") else [float(d) for d in dt]
    if len(dts) != n:
        raise ValueError("one step length per instance")
    D = (ctypes.c_double * n)(*dts)
    _native.check(_native.lib().pf_step_batch(n, P, S, B, D, int(scheme)), "pf_step_batch")


class Batch:
    """Handle of a pf_batch: independent instances whose steps were captured
    once into a CUDA graph; step(n) launches it n times.  Keeps the plans,
    states and bodies alive while it lives."""

    def __init__(self, plans, states, bodies, dt, scheme=0):
        n = len(plans)
        self.plans, self.states, self.bodies = list(plans), list(states), list(bodies)
        P = (ctypes.c_void_p * n)(*[p.handle.value for p in plans])
        S = (ctypes.c_void_p * n)(*[s.handle.value for s in states])
        B = (_native.PfBodyKinematics * n)(*[b.struct for b in bodies])
        dts = [float(dt)] * n if not hasattr(dt, "__len__") else [float(d) for d in dt]
        if len(dts) != n:
            raise ValueError("one step length per instance")
        D = (ctypes.c_double * n)(*dts)
        h = ctypes.c_void_p()
        _native.check(_native.lib().pf_batch_create(n, P, S, B, D, int(scheme), ctypes.byref(h)), "pf_batch_create",
                      plans[0].handle if n else None)
        self.handle = h

    def step(self, nsteps=1):
        _native.check(_native.lib().pf_batch_step(self.handle, int(nsteps)), "pf_batch_step", self.plans[0].handle)

    def close(self):
        if getattr(self, "handle", None):
            _native.lib().pf_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pf_batch_create(plans, states, bodies, dt, scheme=0):
    return Batch(plans, states, bodies, dt, scheme)


def pf_batch_step(batch, nsteps=1):
    batch.step(nsteps)


class Server:
    """Request server (pf_server): continuous batching of time-stepping requests."""

    def __init__(self, max_slots=16, hbm_budget_bytes=8 << 30, precision=PF_MIXED):
        cfg = _native.PfServerConfig(int(max_slots), int(hbm_budget_bytes), int(precision))
        h = ctypes.c_void_p()
        _native.check(_native.lib().pf_server_create(ctypes.byref(cfg), ctypes.byref(h)), "pf_server_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            _native.lib().pf_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pf_server_submit(server, grid, X, Y, G, nsteps, dt, body=None, capacity=None, scheme=0):
    """grid: (nx, ny, dx, x0, y0).  Returns the ticket."""
    body = no_body() if body is None else body
    X, Y, G = _host_f64(X), _host_f64(Y), _host_f64(G)
    nv = len(X)
    if capacity is None:
        capacity = nv + (2 * nsteps if len(body.xb) and body.struct.n_edges == 2 else 0)
    c = ctypes.c_void_p
    req = _native.PfRequest(_native.PfGridDesc(int(grid[0]), int(grid[1]), float(grid[2]), float(grid[3]),
                                               float(grid[4]), 0), body.struct,
                            c(X.ctypes.data), c(Y.ctypes.data), c(G.ctypes.data), nv, int(capacity), int(nsteps),
                            float(dt), int(scheme))
    t = ctypes.c_int64()
    _native.check(_native.lib().pf_server_submit(server.handle, ctypes.byref(req), ctypes.byref(t)),
                  "pf_server_submit")
    return t.value


def pf_server_progress(server, max_done=1024):
    buf = (ctypes.c_int64 * max_done)()
    n = ctypes.c_int32()
    _native.check(_native.lib().pf_server_progress(server.handle, max_done, buf, ctypes.byref(n)),
                  "pf_server_progress")
    return list(buf[:n.value])


def pf_server_result(server, ticket, capacity):
    """(X, Y, G, latency_s) of a finished request; raises on its error status."""
    import numpy as np
    X = np.empty(max(capacity, 1))
    Y = np.empty(max(capacity, 1))
    G = np.empty(max(capacity, 1))
    nv = ctypes.c_int64()
    lat = ctypes.c_double()
    c = ctypes.c_void_p
    _native.check(_native.lib().pf_server_result(server.handle, int(ticket), c(X.ctypes.data), c(Y.ctypes.data),
                                                 c(G.ctypes.data), ctypes.byref(nv), ctypes.byref(lat)),
                  "pf_server_result")
    n = nv.value
    return X[:n].copy(), Y[:n].copy(), G[:n].copy(), lat.value


def pf_server_stats(server):
    q = ctypes.c_int32()
    a = ctypes.c_int32()
    u = ctypes.c_int64()
    _native.check(_native.lib().pf_server_stats(server.handle, ctypes.byref(q), ctypes.byref(a), ctypes.byref(u)),
                  "pf_server_stats")
    return q.value, a.value, u.value
