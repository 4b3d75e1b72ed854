"""Linear and angular impulse of the fluid (Sec. 2.6, Eqs. linimpxd, linimpyd, angimpd).

Test infrastructure only (see the package docstring).

The impulse about the origin has a volume part over the grid vorticity w and a
surface part over the bound sheet f plus the body's tangential slip:

    P_x  =  <y, w>_N + <y_s, f + n_x v_y - n_y v_x>_S
    P_y  = -<x, w>_N - <x_s, f + n_x v_y - n_y v_x>_S
    Pi_O = -1/2 <x^2 + y^2, w>_N - 1/2 <x_s^2 + y_s^2, f + n_x v_y - n_y v_x>_S

with <a, b>_N = dx^2 sum_ij a_ij b_ij (nodes) and <a, b>_S = sum_p dS_p a_p b_p
(surface points), n the unit normal into the fluid and v the surface
velocity.  The force and moment on a single body are -rho dP/dt and
-rho dPi_O/dt (Eq. FMimp).
"""
import numpy as np


def rigid_surface_velocity(xs, ys, U, V, Omega):
    """Velocity of a rigid body point: (U - Omega y, V + Omega x)."""
    return U - Omega * np.asarray(ys), V + Omega * np.asarray(xs)


def impulse(grid, w, xs=None, ys=None, ds=None, f=None, nxs=None, nys=None, U=0.0, V=0.0, Omega=0.0):
    """(P_x, P_y, Pi_O) of Eqs. linimpxd, linimpyd, angimpd.

    `w` is the node vorticity, shape (ny, nx).  Without a surface (xs None)
    only the node terms remain.  Without normals the slip term n x v is left
    out of the surface density (a zero-thickness plate, whose two sides
    cancel it).
    """
    x = grid.node_x()[None, :]
    y = grid.node_y()[:, None]
    dA = grid.dx ** 2
    Px = dA * np.sum(y * w)
    Py = -dA * np.sum(x * w)
    Pi = -0.5 * dA * np.sum((x * x + y * y) * w)
    if xs is not None:
        xs, ys, ds, f = (np.asarray(a, dtype=np.float64) for a in (xs, ys, ds, f))
        dens = f.copy()
        if nxs is not None:
            vx, vy = rigid_surface_velocity(xs, ys, U, V, Omega)
            dens = dens + np.asarray(nxs) * vy - np.asarray(nys) * vx
        Px += np.sum(ds * ys * dens)
        Py -= np.sum(ds * xs * dens)
        Pi -= 0.5 * np.sum(ds * (xs * xs + ys * ys) * dens)
    return np.array([Px, Py, Pi])
