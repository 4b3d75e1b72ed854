"""Lattice Green's function (LGF) of the unit-spacing 5-point Laplacian.

Test infrastructure only (see the package docstring).

Definition (Sec. 2.1, the particular solution s = -L^{-1} w with the LGF of the
5-point Laplacian, refs. katsura71 / cserti00 / liska14 of the paper):

    G(m, n) = 1/(4 pi^2) * Int_{[-pi,pi]^2} (1 - cos(m a + n b)) / (4 - 2 cos a - 2 cos b) da db

so that L0 G = delta_0 with L0 s = s(i+1,j)+s(i-1,j)+s(i,j+1)+s(i,j-1)-4 s(i,j)
and the additive constant fixed by G(0,0) = 0 (the paper leaves the homogeneous
part free; this is the reading used throughout).

Integrating over a by residues leaves a single integral.  With
h = sin(theta/2), u = asinh(h):

    G(m, n) = 1/(2 pi) * Int_0^pi [1 - exp(-2|m| u) cos(n theta)] / sinh(2u) dtheta

because with A = 2 - cos(theta) one has sqrt(A^2-1) = sinh(2u) and
A - sqrt(A^2-1) = exp(-2u).  The numerator is split as
(1 - e^{-2mu}) + e^{-2mu} (1 - cos n theta) so both pieces stay finite at
theta = 0, and 1 - cos(n theta) is evaluated as 2 sin^2(n theta / 2).

The integral is done with composite Gauss-Legendre on geometrically graded
panels towards theta = 0 (the only place the integrand varies on the scale
1/|m|).  The larger of |m|, |n| is put in the exponent (G(m,n) = G(n,m)), so the
oscillating factor never has more than a few periods where exp(-2mu) is not
negligible.
"""
import numpy as np

_GL_ORDER = 24


def _panels(theta_min=1e-10, ratio=1.35):
    """Breakpoints 0, theta_min, theta_min*ratio, ..., pi."""
    b = [0.0, theta_min]
    while b[-1] * ratio < np.pi:
        b.append(b[-1] * ratio)
    b.append(np.pi)
    return np.array(b)


def quadrature_nodes(theta_min=1e-10, ratio=1.35, order=_GL_ORDER):
    """Composite Gauss-Legendre nodes and weights on [0, pi]."""
    x, w = np.polynomial.legendre.leggauss(order)
    b = _panels(theta_min, ratio)
    lo, hi = b[:-1], b[1:]
    half = 0.5 * (hi - lo)
    mid = 0.5 * (hi + lo)
    th = (mid[:, None] + half[:, None] * x[None, :]).ravel()
    wt = (half[:, None] * w[None, :]).ravel()
    return th, wt


def lgf_table(K, L=None):
    """Return T with T[m, n] = G(m, n) for 0 <= m <= K, 0 <= n <= L (float64).

    G is even in m and n, so this quadrant determines G(m, n) for |m| <= K,
    |n| <= L.
    """
    if L is None:
        L = K
    N = max(K, L)
    th, wt = quadrature_nodes()
    h = np.sin(0.5 * th)
    u = np.arcsinh(h)
    s = np.sinh(2.0 * u)                      # sqrt((2 - cos th)^2 - 1)
    idx = np.arange(N + 1, dtype=np.float64)
    # first piece: depends on the larger index only
    E = np.exp(-2.0 * idx[:, None] * u[None, :])            # (N+1, nodes): e^{-2 m u}
    one_minus = -np.expm1(-2.0 * idx[:, None] * u[None, :])  # 1 - e^{-2 m u}
    first = one_minus @ (wt / s)                            # (N+1,)
    # second piece: sum_k w_k e^{-2 m u_k}/s_k * 2 sin^2(n th_k / 2)
    A = E * (wt / s)[None, :]
    B = 2.0 * np.sin(0.5 * idx[None, :] * th[:, None]) ** 2  # (nodes, N+1)
    second = A @ B                                          # (m, n) with m in exponent
    full = (first[:, None] + second) / (2.0 * np.pi)        # valid where m >= n
    # symmetric completion: G(m, n) uses the larger index in the exponent
    mm, nn = np.meshgrid(np.arange(N + 1), np.arange(N + 1), indexing="ij")
    big = np.maximum(mm, nn)
    small = np.minimum(mm, nn)
    G = full[big, small]
    G[0, 0] = 0.0
    return G[: K + 1, : L + 1].copy()


def lgf(m, n, table):
    """G(m, n) for integer arrays m, n (any sign) from a quadrant table."""
    return table[np.abs(m), np.abs(n)]
