"""Pressure (Sec. 2.6.1): the jump in scalar potential carried by the bound
vortex sheet, the pressure jump across the surface from the immersed-boundary
Bernoulli equation, and the pressure field at the cell centres (Eq. pgrid,
second half of this module).

Test infrastructure only (see the package docstring).

The grid is staggered (Sec. 2.1, Fig. 1a): psi on the nodes (x_i, y_j); the
velocity component u = d psi/dy on the x-faces (x_i, y_j + dx/2) as
(psi[i, j+1] - psi[i, j])/dx and v = -d psi/dx on the y-faces
(x_i + dx/2, y_j) as -(psi[i+1, j] - psi[i, j])/dx (the discrete curl C).
E_f interpolates each component to the surface from its own face lattice with
the smoothed three-point function (the surface kernel of Sec. 2.2.1); R_f is
its transpose carrying dS_p / dx^2, as R_s.

* surface curl C_s psi = n . E_f C psi  (nodes -> surface); its transpose
  C_s^T sigma = C^T R_f (n o sigma)     (surface -> nodes);
* jump in scalar potential of a sheet f (Eq. dphi and the relation above it):
  Delta phi = -(C_s L^-1 C_s^T)^-1 C_s L^-1 R_s f, defined up to a uniform
  value (the null space); here fixed by sum_p dS_p Delta phi_p = 0 through a
  Lagrange multiplier;
* pressure jump (Eq. surfbernoulli):
  Delta p = -rho (E_f u - v_s) . (f z x n) - rho d(Delta phi)/dt,
  z x n = (-n_y, n_x), v_s = (U - Omega y, V + Omega x).

Arrays of node data are indexed [j, i] as in vic.py.
"""
import numpy as np

from .kernels import yang3
from .vic import stencil_1d


def curl_weights(grid, xs, ys, nxs, nys):
    """Node stencil of C_s for every surface point: (NI, NJ, W), each (ns, 64),
    with (C_s psi)_p = sum_k W[p, k] psi[NJ[p, k], NI[p, k]].

    x-faces: u at (x_i, y_j + dx/2), interpolated with nodes i on x and the
    half-shifted lattice on y; y-faces: v at (x_i + dx/2, y_j) alike."""
    dx = grid.dx
    ns = len(xs)
    NI = np.zeros((ns, 64), dtype=np.int64)
    NJ = np.zeros((ns, 64), dtype=np.int64)
    W = np.zeros((ns, 64))
    # u-faces: x stencil on nodes, y stencil on the lattice y0 + dx/2 (face row j between nodes j, j+1)
    ixu, wxu = stencil_1d(xs, grid.x0, dx, grid.nx, yang3)
    iyu, wyu = stencil_1d(ys, grid.y0 + 0.5 * dx, dx, grid.ny - 1, yang3)
    # v-faces: x stencil on the lattice x0 + dx/2, y stencil on nodes
    ixv, wxv = stencil_1d(xs, grid.x0 + 0.5 * dx, dx, grid.nx - 1, yang3)
    iyv, wyv = stencil_1d(ys, grid.y0, dx, grid.ny, yang3)
    k = 0
    for b in range(4):
        for a in range(4):
            wu = nxs * wxu[:, a] * wyu[:, b] / dx          # n_x u, u = (psi[j+1] - psi[j]) / dx
            NI[:, k], NJ[:, k], W[:, k] = ixu[:, a], iyu[:, b] + 1, wu
            NI[:, k + 1], NJ[:, k + 1], W[:, k + 1] = ixu[:, a], iyu[:, b], -wu
            wv = nys * wxv[:, a] * wyv[:, b] / dx          # n_y v, v = -(psi[i+1] - psi[i]) / dx
            NI[:, k + 2], NJ[:, k + 2], W[:, k + 2] = ixv[:, a] + 1, iyv[:, b], -wv
            NI[:, k + 3], NJ[:, k + 3], W[:, k + 3] = ixv[:, a], iyv[:, b], wv
            k += 4
    return NI, NJ, W


def apply_curl(cw, psi):
    """C_s psi for a node field psi[j, i]."""
    NI, NJ, W = cw
    return np.sum(W * psi[NJ, NI], axis=1)


def _lgf_pair_sum(NIa, NJa, Wa, NIb, NJb, Wb, table):
    """M[p, q] = sum_k sum_l Wa[p, k] G(node_a(p, k) - node_b(q, l)) Wb[q, l]."""
    out = np.empty((NIa.shape[0], NIb.shape[0]))
    for p in range(NIa.shape[0]):
        di = np.abs(NIa[p][:, None, None] - NIb[None, :, :])
        dj = np.abs(NJa[p][:, None, None] - NJb[None, :, :])
        out[p] = np.einsum("k,kql,ql->q", Wa[p], table[di, dj], Wb)
    return out


def jump_matrix(grid, cw, ds, table):
    """K = C_s L^-1 C_s^T with L^-1 = dx^2 G * and C_s^T = C^T R_f (n o .):
    K[p, q] = dS_q sum a_p(m) G(m - m') a_q(m')."""
    NI, NJ, W = cw
    return _lgf_pair_sum(NI, NJ, W, NI, NJ, W, table) * np.asarray(ds)[None, :]


def potential_jump(grid, st, cw, ds, f, table):
    """Delta phi of the sheet f: K Delta phi = -C_s L^-1 R_s f with
    sum dS Delta phi = 0 (augmented system, multiplier for the uniform null space)."""
    ns = len(ds)
    K = jump_matrix(grid, cw, ds, table)
    # C_s L^-1 R_s f = sum a_p(m) G(m - m') (dS_q f_q d_q(m'))  (the dx^2 of L^-1 and 1/dx^2 of R_s cancel)
    NI, NJ, W = cw
    rhs = -_lgf_pair_sum(NI, NJ, W, st.NI, st.NJ, st.W, table) @ (np.asarray(ds) * f)
    A = np.zeros((ns + 1, ns + 1))
    A[:ns, :ns] = K
    A[:ns, ns] = 1.0
    A[ns, :ns] = ds
    x = np.linalg.solve(A, np.concatenate([rhs, [0.0]]))
    return x[:ns]


def face_velocity_at_surface(grid, xs, ys, psi_pad1, Uinf, Vinf):
    """E_f C psi + uniform flow: (u_s, v_s) at the surface points, each
    component interpolated from its own faces; psi_pad1 is psi on the grid
    extended by one node on every side (index [j + 1, i + 1])."""
    dx = grid.dx
    p = psi_pad1
    ixu, wxu = stencil_1d(xs, grid.x0, dx, grid.nx, yang3)
    iyu, wyu = stencil_1d(ys, grid.y0 + 0.5 * dx, dx, grid.ny - 1, yang3)
    ixv, wxv = stencil_1d(xs, grid.x0 + 0.5 * dx, dx, grid.nx - 1, yang3)
    iyv, wyv = stencil_1d(ys, grid.y0, dx, grid.ny, yang3)
    us = np.zeros(len(xs))
    vs = np.zeros(len(xs))
    for b in range(4):
        for a in range(4):
            i, j = ixu[:, a], iyu[:, b]
            us += wxu[:, a] * wyu[:, b] * (p[j + 2, i + 1] - p[j + 1, i + 1]) / dx
            i, j = ixv[:, a], iyv[:, b]
            vs += wxv[:, a] * wyv[:, b] * -(p[j + 1, i + 2] - p[j + 1, i + 1]) / dx
    return us + Uinf, vs + Vinf


def pressure_jump(us, vs, xs, ys, nxs, nys, f, U, V, Omega, dphi_dt, rho=1.0):
    """Eq. surfbernoulli: Delta p = -rho (E_f u - v_s) . (f z x n) - rho d(Delta phi)/dt."""
    vsx = U - Omega * ys
    vsy = V + Omega * xs
    tx, ty = -nys, nxs                       # z x n
    return -rho * ((us - vsx) * f * tx + (vs - vsy) * f * ty) - rho * dphi_dt


# ----------------------------------------------------------------- pressure field
# Eq. pgrid at the cell centres (x_i + dx/2, y_j + dx/2), i < nx - 1, j < ny - 1,
# read with the surface term inside the divergence (L^-1 acts on centre data):
#   p = -rho/2 |u|^2 - rho L^-1 D [ w x u + R_f(n o d(Delta phi)/dt - v_s x f) ],
# w the free vorticity on the nodes, u the face velocity of the whole flow,
# D the divergence from the faces to the centres, L^-1 = dx^2 G * on the centre
# lattice (the same five-point Laplacian).  Face arrays: u[j, i] on the x-face
# (x_i, y_j + dx/2), shape (ny - 1, nx); v[j, i] on the y-face (x_i + dx/2, y_j),
# shape (ny, nx - 1).

def face_velocities(grid, psi, Uinf, Vinf):
    """u = (psi[j+1, i] - psi[j, i]) / dx + Uinf, v = -(psi[j, i+1] - psi[j, i]) / dx + Vinf."""
    dx = grid.dx
    return (psi[1:, :] - psi[:-1, :]) / dx + Uinf, -(psi[:, 1:] - psi[:, :-1]) / dx + Vinf


def lamb_faces(w, u, v):
    """w x u = (-w v, w u) on the faces: the x-component on the x-faces with w
    averaged over the face's two nodes and v over the four y-faces around it,
    the y-component on the y-faces alike; faces on the grid's edge take the
    missing neighbours as zero."""
    ny, nx = w.shape
    vpad = np.zeros((ny, nx + 1))
    vpad[:, 1:-1] = v                          # y-face (i - 1/2, j) at vpad[j, i]
    v_at_x = 0.25 * (vpad[:-1, :-1] + vpad[:-1, 1:] + vpad[1:, :-1] + vpad[1:, 1:])   # (ny - 1, nx)
    lx = -0.5 * (w[:-1, :] + w[1:, :]) * v_at_x
    upad = np.zeros((ny + 1, nx))
    upad[1:-1, :] = u                          # x-face (i, j - 1/2) at upad[j, i]
    u_at_y = 0.25 * (upad[:-1, :-1] + upad[1:, :-1] + upad[:-1, 1:] + upad[1:, 1:])   # (ny, nx - 1)
    ly = 0.5 * (w[:, :-1] + w[:, 1:]) * u_at_y
    return lx, ly


def surface_faces(grid, xs, ys, nxs, nys, ds, dphi_dt, f, U, V, Omega):
    """R_f(n o d(Delta phi)/dt - v_s x f) on the faces: the x-component on the
    u lattice, the y-component on the v lattice, each with dS/dx^2 and the
    smoothed three-point weights; v_s x (f z) = (v_sy f, -v_sx f)."""
    dx = grid.dx
    vsx, vsy = U - Omega * ys, V + Omega * xs
    ax = nxs * dphi_dt - vsy * f
    ay = nys * dphi_dt + vsx * f
    qx = np.zeros((grid.ny - 1, grid.nx))
    qy = np.zeros((grid.ny, grid.nx - 1))
    ixu, wxu = stencil_1d(xs, grid.x0, dx, grid.nx, yang3)
    iyu, wyu = stencil_1d(ys, grid.y0 + 0.5 * dx, dx, grid.ny - 1, yang3)
    ixv, wxv = stencil_1d(xs, grid.x0 + 0.5 * dx, dx, grid.nx - 1, yang3)
    iyv, wyv = stencil_1d(ys, grid.y0, dx, grid.ny, yang3)
    for b in range(4):
        for a in range(4):
            np.add.at(qx, (iyu[:, b], ixu[:, a]), ds * ax * wxu[:, a] * wyu[:, b])
            np.add.at(qy, (iyv[:, b], ixv[:, a]), ds * ay * wxv[:, a] * wyv[:, b])
    return qx / dx ** 2, qy / dx ** 2


def divergence(grid, qx, qy):
    """D q at the centres: (qx[j, i+1] - qx[j, i] + qy[j+1, i] - qy[j, i]) / dx."""
    return (qx[:, 1:] - qx[:, :-1] + qy[1:, :] - qy[:-1, :]) / grid.dx


def pressure_field(grid, table, u, v, w, qx_s, qy_s, rho=1.0):
    """Eq. pgrid at the cell centres (the surface faces qx_s, qy_s may be zero)."""
    from .vic import Grid, inv_laplacian
    lx, ly = lamb_faces(w, u, v)
    src = divergence(grid, lx + qx_s, ly + qy_s)
    gc = Grid(grid.nx - 1, grid.ny - 1, grid.dx, grid.x0 + 0.5 * grid.dx, grid.y0 + 0.5 * grid.dx)
    ke = 0.5 * (u[:, :-1] ** 2 + u[:, 1:] ** 2) + 0.5 * (v[:-1, :] ** 2 + v[1:, :] ** 2)
    return -0.5 * rho * ke - rho * inv_laplacian(gc, src, table)
