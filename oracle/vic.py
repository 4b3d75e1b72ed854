"""Grid-level operators of the basic (body-free) problem, Sec. 2.1.

Test infrastructure only (see the package docstring).

Conventions (shared with the library's documented interface, not with its code):
node (i, j) sits at (x0 + i dx, y0 + j dx); node fields are numpy arrays of
shape (ny, nx) indexed [j, i] (x fastest).  L = L0 / dx^2 is the 5-point
Laplacian, so L^{-1} = dx^2 (G *) with G the unit-spacing LGF (oracle.lgf).
"""
import numpy as np

from .kernels import m4prime
from .lgf import lgf_table


class Grid:
    def __init__(self, nx, ny, dx, x0, y0):
        self.nx, self.ny, self.dx, self.x0, self.y0 = int(nx), int(ny), float(dx), float(x0), float(y0)

    def node_x(self):
        return self.x0 + self.dx * np.arange(self.nx)

    def node_y(self):
        return self.y0 + self.dx * np.arange(self.ny)


def stencil_1d(pos, origin, dx, n, kernel):
    """Indices and weights of the four nodes a radius-2 kernel can touch.

    For a point at grid coordinate g = (pos - origin)/dx the nodes are
    floor(g)-1 .. floor(g)+2; all others have kernel weight exactly zero.
    Raises if any of the four nodes lies outside [0, n).
    """
    g = (np.asarray(pos, dtype=np.float64) - origin) / dx
    c = np.floor(g).astype(np.int64)
    idx = c[:, None] + np.arange(-1, 3)[None, :]
    if idx.size and (idx.min() < 0 or idx.max() >= n):
        raise ValueError("point stencil leaves the grid")
    wts = kernel(idx - g[:, None])          # d((x_i - X)/dx)
    return idx, wts


def regularize(grid, X, Y, Gam):
    """w = (1/dx^2) sum_q Gamma_q d((x-X_q)/dx) d((y-Y_q)/dx)  (Eq. vortexregularization).

    d is M4'.  Accumulation runs over vortices in index order.
    """
    w = np.zeros((grid.ny, grid.nx))
    if len(X) == 0:
        return w
    ix, wx = stencil_1d(X, grid.x0, grid.dx, grid.nx, m4prime)
    iy, wy = stencil_1d(Y, grid.y0, grid.dx, grid.ny, m4prime)
    for a in range(4):
        for b in range(4):
            np.add.at(w, (iy[:, b], ix[:, a]), np.asarray(Gam) * wx[:, a] * wy[:, b])
    return w / grid.dx ** 2


def circulation(grid, w):
    """Gamma_w = <1, w>_N = dx^2 sum w  (Sec. 2.1 node inner product)."""
    return grid.dx ** 2 * float(np.sum(w))


def inv_laplacian(grid, src, table=None, pad=0):
    """L^{-1} src = dx^2 * sum_{i',j'} G(i-i', j-j') src[j', i']  by direct summation.

    Evaluated on the grid extended by `pad` nodes on every side (the LGF gives
    the unbounded solution anywhere).  Returns shape (ny+2 pad, nx+2 pad).
    For each source-row offset the sum over source columns is one matrix
    product with the Toeplitz matrix G(i-i', d).
    """
    ny, nx = src.shape
    P = pad
    if table is None:
        table = lgf_table(nx + P, ny + P)
    ti = np.arange(-P, nx + P)            # target columns
    si = np.arange(nx)                    # source columns
    dcol = np.abs(ti[:, None] - si[None, :])
    out = np.zeros((ny + 2 * P, nx + 2 * P))
    tj = np.arange(-P, ny + P)            # target rows
    # for every signed row offset delta = j - j', all (target, source) row pairs
    # with that offset share the Toeplitz matrix T[t, s] = G(ti - si, |delta|)
    for delta in range(-(ny - 1 + P), ny + P):
        jp = tj - delta
        ok = (jp >= 0) & (jp < ny)
        if not np.any(ok):
            continue
        T = table[dcol, abs(delta)]       # (nx + 2P, nx)
        out[ok] += src[jp[ok]] @ T.T
    return grid.dx ** 2 * out


def inv_laplacian_at(grid, src, ti, tj, table):
    """(L^{-1} src) at individual target nodes (ti[k], tj[k]), one by one."""
    ny, nx = src.shape
    J, I = np.nonzero(src)
    vals = src[J, I]
    out = np.empty(len(ti))
    for k in range(len(ti)):
        out[k] = np.dot(table[np.abs(ti[k] - I), np.abs(tj[k] - J)], vals)
    return grid.dx ** 2 * out


def node_velocity_at(grid, src, ti, tj, table, Uinf=0.0, Vinf=0.0):
    """Node velocity of psi = -L^{-1} src at individual nodes, one by one.

    Same centred differences as node_velocity (Eq. velsf), applied to the
    kernel before the sum (the operators are linear):
    u = -(dx/2) sum src (G(i-i', j+1-j') - G(i-i', j-1-j')),
    v = +(dx/2) sum src (G(i+1-i', j-j') - G(i-1-i', j-j')).
    Differencing the kernel avoids cancelling two large sums.
    """
    J, I = np.nonzero(src)
    vals = src[J, I]
    u = np.empty(len(ti))
    v = np.empty(len(ti))
    for k in range(len(ti)):
        di = np.abs(ti[k] - I)
        dy = table[di, np.abs(tj[k] + 1 - J)] - table[di, np.abs(tj[k] - 1 - J)]
        dj = np.abs(tj[k] - J)
        dxk = table[np.abs(ti[k] + 1 - I), dj] - table[np.abs(ti[k] - 1 - I), dj]
        u[k] = -0.5 * grid.dx * np.dot(dy, vals) + Uinf
        v[k] = 0.5 * grid.dx * np.dot(dxk, vals) + Vinf
    return u, v


def laplacian_unit(field):
    """L0 applied at interior nodes: s(i+1,j)+s(i-1,j)+s(i,j+1)+s(i,j-1)-4 s(i,j)."""
    f = field
    return f[1:-1, 2:] + f[1:-1, :-2] + f[2:, 1:-1] + f[:-2, 1:-1] - 4.0 * f[1:-1, 1:-1]


def streamfunction(grid, w, table=None, pad=0):
    """psi = -L^{-1} w (Sec. 2.1, particular solution; uniform flow added separately)."""
    return -inv_laplacian(grid, w, table, pad)


def node_velocity(grid, psi_pad1, Uinf=0.0, Vinf=0.0):
    """Node velocity from psi given on the grid extended by one node.

    u = d psi/dy, v = -d psi/dx by centred differences (Eq. velsf), followed by
    the simple face-to-node average the paper prescribes before interpolation;
    the two combine to (psi[j+1] - psi[j-1])/(2 dx) and -(psi[i+1] - psi[i-1])/(2 dx).
    The uniform flow (Uinf, Vinf) is the curl of the homogeneous solution
    psi_inf = Uinf y - Vinf x and is added exactly.
    """
    p = psi_pad1
    dx = grid.dx
    u = (p[2:, 1:-1] - p[:-2, 1:-1]) / (2.0 * dx) + Uinf
    v = -(p[1:-1, 2:] - p[1:-1, :-2]) / (2.0 * dx) + Vinf
    return u, v


def interpolate(grid, field, X, Y):
    """E_v field at points: sum d((x_i-X)/dx) d((y_j-Y)/dx) field_ij  (E_v = R_v^T, Sec. 2.1)."""
    if len(X) == 0:
        return np.zeros(0)
    ix, wx = stencil_1d(X, grid.x0, grid.dx, grid.nx, m4prime)
    iy, wy = stencil_1d(Y, grid.y0, grid.dx, grid.ny, m4prime)
    out = np.zeros(len(X))
    for a in range(4):
        for b in range(4):
            out += wx[:, a] * wy[:, b] * field[iy[:, b], ix[:, a]]
    return out


def vortex_velocity(grid, X, Y, Gam, Uinf=0.0, Vinf=0.0, table=None):
    """One body-free VIC evaluation: R_v, psi = -L^{-1} w, curl, E_v.

    Returns (w, psi, u_q, v_q): w and psi on the grid, velocity at the vortices.
    """
    w = regularize(grid, X, Y, Gam)
    if table is None:
        table = lgf_table(grid.nx + 1, grid.ny + 1)
    psi1 = streamfunction(grid, w, table, pad=1)
    u, v = node_velocity(grid, psi1, Uinf, Vinf)
    return w, psi1[1:-1, 1:-1], interpolate(grid, u, X, Y), interpolate(grid, v, X, Y)
