"""Immersed surface, Schur complement and constrained sheet solves (Sec. 2.2-2.4).

Test infrastructure only (see the package docstring).

Notation follows the paper: S = -E L^{-1} R_s (Eq. vsheet), f0 = S^{-1} 1
(Eq. f0), f0hat = D_dS f0, Gamma0 = <1, f0>_S (Eq. circ0), circulation
removal P^Gamma = I - 1 f0hat^T / Gamma0 (Eq. circrem), decomposition
f = f0 o ftilde with Stilde = S D_f0 (Eqs. decomposition, Son1), Kutta
projection P_k = I - 1 e_k^T.  `EinvLw` always denotes E L^{-1} w = -E psi*
where psi* = -L^{-1} w is the field of the free vorticity alone.
"""
import numpy as np
import scipy.linalg

from .kernels import yang3, m4prime
from .vic import stencil_1d


# ----------------------------------------------------------------- transfer
class SurfaceStencil:
    """Nodes and smoothed-three-point weights of every surface point (Sec. 2.2.1)."""

    def __init__(self, grid, xs, ys):
        self.ix, self.wx = stencil_1d(xs, grid.x0, grid.dx, grid.nx, yang3)
        self.iy, self.wy = stencil_1d(ys, grid.y0, grid.dx, grid.ny, yang3)
        ns = len(xs)
        # flattened 16-node stencils: (ns, 16)
        self.NI = np.repeat(self.ix[:, None, :], 4, axis=1).reshape(ns, 16)   # [p, b*4+a] -> ix[p,a]
        self.NJ = np.repeat(self.iy[:, :, None], 4, axis=2).reshape(ns, 16)   # -> iy[p,b]
        self.W = (self.wy[:, :, None] * self.wx[:, None, :]).reshape(ns, 16)


def interp_surface(st, field):
    """E_s field: sum_ij d((x_i - x_p)/dx) d((y_j - y_p)/dx) field_ij (no dx factor)."""
    return np.sum(st.W * field[st.NJ, st.NI], axis=1)


def regularize_surface(grid, st, f, ds):
    """R_s f = (1/dx^2) sum_p dS_p f_p d d, the transpose of E_s in the node and
    surface inner products (Sec. 2.2.1)."""
    out = np.zeros((grid.ny, grid.nx))
    np.add.at(out, (st.NJ, st.NI), st.W * (ds * f)[:, None])
    return out / grid.dx ** 2


def point_vortex_stencil(grid, X, Y):
    """16-node M4' stencil of point vortices, flattened like SurfaceStencil."""
    ix, wx = stencil_1d(X, grid.x0, grid.dx, grid.nx, m4prime)
    iy, wy = stencil_1d(Y, grid.y0, grid.dx, grid.ny, m4prime)
    n = len(X)
    NI = np.repeat(ix[:, None, :], 4, axis=1).reshape(n, 16)
    NJ = np.repeat(iy[:, :, None], 4, axis=2).reshape(n, 16)
    W = (wy[:, :, None] * wx[:, None, :]).reshape(n, 16)
    return NI, NJ, W


def _local_lgf_sum(NIa, NJa, Wa, NIb, NJb, Wb, table):
    """M[p, q] = sum over the 16 x 16 node pairs of Wa[p] G(node_a - node_b) Wb[q]."""
    out = np.empty((NIa.shape[0], NIb.shape[0]))
    for p in range(NIa.shape[0]):
        dI = np.abs(NIa[p][:, None, None] - NIb[None, :, :])     # (16, nb, 16)
        dJ = np.abs(NJa[p][:, None, None] - NJb[None, :, :])
        Gv = table[dI, dJ]
        out[p] = np.einsum("a,aqb,qb->q", Wa[p], Gv, Wb)
    return out


def schur_matrix(grid, st, ds, table):
    """S = -E L^{-1} R_s  (Eq. vsheet).

    With L^{-1} = dx^2 G* and R_s carrying dS_q/dx^2:
    S[p, q] = -dS_q sum_{ij} sum_{i'j'} d_p(ij) G(i-i', j-j') d_q(i'j').
    """
    M = _local_lgf_sum(st.NI, st.NJ, st.W, st.NI, st.NJ, st.W, table)
    return -M * ds[None, :]


def EinvL_unit_vortex(grid, st, X, Y, table):
    """E_s L^{-1} d_j for unit point vortices at (X[j], Y[j]); returns (ns, nv)."""
    NI, NJ, W = point_vortex_stencil(grid, np.atleast_1d(X), np.atleast_1d(Y))
    # L^{-1} d_j = dx^2 G * (dx^-2 M4'M4') -> the dx factors cancel
    return _local_lgf_sum(st.NI, st.NJ, st.W, NI, NJ, W, table)


# ----------------------------------------------------------------- factor
class Schur:
    """Dense LU of S and the per-geometry quantities f0, f0hat, Gamma0 (Eqs. f0, circ0)."""

    def __init__(self, S, ds):
        self.S = S
        self.ds = np.asarray(ds, dtype=np.float64)
        self.lu = scipy.linalg.lu_factor(S)
        self.ones = np.ones(S.shape[0])
        self.f0 = self.solve(self.ones)
        self.f0hat = self.ds * self.f0
        self.Gamma0 = float(np.sum(self.f0hat))

    def solve(self, r):
        return scipy.linalg.lu_solve(self.lu, r)

    def solve_tilde(self, r):
        """Stilde^{-1} r with Stilde = S D_f0, i.e. D_f0^{-1} S^{-1} r."""
        return self.solve(r) / (self.f0[:, None] if np.ndim(r) == 2 else self.f0)

    def circ(self, f):
        """<1, f>_S = sum dS f  (Eq. circdef)."""
        return float(np.dot(self.ds, f))

    def P_Gamma(self, s):
        """Circulation removal P^Gamma s = s - 1 (f0hat^T s)/Gamma0  (Eq. circrem)."""
        return s - self.ones * (np.dot(self.f0hat, s) / self.Gamma0)

    def f0hat_Pk(self, v, k):
        """f0hat^T P_k v with P_k = I - 1 e_k^T."""
        return float(np.dot(self.f0hat, v) - self.Gamma0 * v[k])


def body_streamfunction(xs, ys, U, V, Omega):
    """psi_b = U y - V x - Omega/2 (x^2 + y^2)  (Eq. sfsurf)."""
    return U * ys - V * xs - 0.5 * Omega * (xs * xs + ys * ys)


def sb_prime(xs, ys, U, V, Omega, Uinf, Vinf):
    """s'_b = psi_b - E psi_inf with psi_inf = Uinf y - Vinf x (Sec. 2.2.2).

    E reproduces linear fields exactly, so E psi_inf = Uinf y_p - Vinf x_p.
    """
    return body_streamfunction(xs, ys, U - Uinf, V - Vinf, Omega)


# ----------------------------------------------------------------- solves
def sheet_given_s0(sch, sbp, EinvLw, s0):
    """Basic system (Eq. basicblock / vsheet): f = S^{-1}(s'_b - s0 1 - E psi*)."""
    return sch.solve(sbp - s0 * sch.ones + EinvLw)


def sheet_circulation(sch, sbp, EinvLw, Gamma_b):
    """Circulation-constrained system (Eq. circsystem): s0 is the multiplier.

    From Eq. circs0: Gamma_b = <1, S^{-1}(s'_b + E L^{-1} w)> - s0 Gamma0.
    Returns (f, s0).
    """
    fs = sch.solve(sbp + EinvLw)
    s0 = (sch.circ(fs) - Gamma_b) / sch.Gamma0
    return fs - s0 * sch.f0, s0


def intermediate_sheet(sch, sbp, EinvLw):
    """ftilde* = Stilde^{-1}(P^Gamma s'_b + E L^{-1} w)  (Eq. intermedsoln)."""
    return sch.solve_tilde(sch.P_Gamma(sbp) + EinvLw)


def sheet_kutta_steady(sch, sbp, EinvLw, k):
    """Steady Kutta at point k (Eqs. kuttasystem, s0): returns (f, ftilde, s0)."""
    fts = intermediate_sheet(sch, sbp, EinvLw)
    s0 = fts[k]
    ft = fts - s0 * sch.ones                     # P_k ftilde*
    return sch.f0 * ft, ft, s0


def sheet_kutta_shed1(sch, sbp, EinvLw, k, EinvLd1, Gamma_w):
    """One new vortex, Kutta at k and Kelvin (Eq. kuttasystem2).

    Gamma1 = (-Gamma_w - f0hat^T P_k ftilde*) / (1 + f0hat^T P_k ftilde_1),
    s0 = e_k^T(ftilde* + Gamma1 ftilde_1), ftilde = P_k(ftilde* + Gamma1 ftilde_1).
    Returns (f, ftilde, s0, Gamma1).
    """
    fts = intermediate_sheet(sch, sbp, EinvLw)
    ft1 = sch.solve_tilde(EinvLd1)
    G1 = (-Gamma_w - sch.f0hat_Pk(fts, k)) / (1.0 + sch.f0hat_Pk(ft1, k))
    g = fts + G1 * ft1
    s0 = g[k]
    ft = g - s0 * sch.ones
    return sch.f0 * ft, ft, s0, G1


def sheet_kutta_shed2(sch, sbp, EinvLw, k1, k2, EinvLd1, EinvLd2, Gamma_w):
    """Two new vortices, Kutta at k1 and k2 and Kelvin: split form (Eq. twovortex).

    Returns (f, ftilde, s0, Gamma1, Gamma2).
    """
    fts = intermediate_sheet(sch, sbp, EinvLw)
    ft1 = sch.solve_tilde(EinvLd1)
    ft2 = sch.solve_tilde(EinvLd2)
    A = np.array([[1.0 + sch.f0hat_Pk(ft1, k1), 1.0 + sch.f0hat_Pk(ft2, k1)],
                  [1.0 + sch.f0hat_Pk(ft1, k2), 1.0 + sch.f0hat_Pk(ft2, k2)]])
    b = -np.array([Gamma_w + sch.f0hat_Pk(fts, k1), Gamma_w + sch.f0hat_Pk(fts, k2)])
    G1, G2 = np.linalg.solve(A, b)
    g = fts + G1 * ft1 + G2 * ft2
    s0 = 0.5 * (g[k1] + g[k2])
    ft = 0.5 * ((g - g[k1]) + (g - g[k2]))       # 1/2 (P_k1 + P_k2) g
    return sch.f0 * ft, ft, s0, G1, G2


def edge_targets(fts, edges, bounds):
    """Generalized edge condition (Sec. 2.5): for each edge k the intermediate
    value e_k^T ftilde* is tested against [fmin_k, fmax_k]; an edge outside its
    range is active and its target is the bound it crossed.
    Returns [(k, active, target)]."""
    out = []
    for k, (lo, hi) in zip(edges, bounds):
        v = fts[k]
        if lo <= v <= hi:
            out.append((k, False, 0.0))
        else:
            out.append((k, True, lo if v < lo else hi))
    return out


def sheet_edge_shed(sch, sbp, EinvLw, edges, EinvLds, Gamma_w, bounds):
    """New vortices at one or two edges under the generalized edge condition
    (Sec. 2.5, Eq. twovortex-gen), Kelvin over the whole flow.

    Active edges solve A Gamma = b with A_ij = 1 + f0hat^T P_ki ftilde_j and
    b_i = -(Gamma_w + f0hat^T P_ki ftilde* + Gamma0 target_i); an edge inside
    its range sheds nothing (Gamma = 0).  Then g = ftilde* + sum Gamma_j ftilde_j
    and s0 = g_k - target_k on the active edges (their mean for two); with no
    active edge Kelvin alone fixes s0 = (f0hat^T ftilde* + Gamma_w)/Gamma0.
    fmin = fmax = 0 is the Kutta condition.  Returns (f, ftilde, s0, Gammas).
    """
    fts = intermediate_sheet(sch, sbp, EinvLw)
    fts_j = [sch.solve_tilde(e) for e in EinvLds]
    tg = edge_targets(fts, edges, bounds)
    act = [i for i, (_, a, _) in enumerate(tg) if a]
    G = np.zeros(len(edges))
    if act:
        A = np.array([[1.0 + sch.f0hat_Pk(fts_j[j], tg[i][0]) for j in act] for i in act])
        b = -np.array([Gamma_w + sch.f0hat_Pk(fts, tg[i][0]) + sch.Gamma0 * tg[i][2] for i in act])
        G[act] = np.linalg.solve(A, b)
    g = fts + sum(G[j] * fts_j[j] for j in range(len(edges)))
    if act:
        s0 = float(np.mean([g[tg[i][0]] - tg[i][2] for i in act]))
    else:
        s0 = (float(np.dot(sch.f0hat, fts)) + Gamma_w) / sch.Gamma0
    ft = g - s0 * sch.ones
    return sch.f0 * ft, ft, s0, G


def sheet_edge_shed2_monolithic(S, f0, f0hat, PGsb, EinvLw, k1, k2, EinvLd1, EinvLd2, Gamma_w, t1, t2):
    """Dense (Ns+3) solve of the two-edge system with edge targets t1, t2
    (both edges active; Sec. 2.5): the rows of Eq. kuttasystem3 with
    e_k1^T ftilde = t1, e_k2^T ftilde = t2."""
    ns = S.shape[0]
    A = np.zeros((ns + 3, ns + 3))
    A[:ns, :ns] = S * f0[None, :]
    A[:ns, ns] = 1.0
    A[:ns, ns + 1] = -EinvLd1
    A[:ns, ns + 2] = -EinvLd2
    A[ns, k1] = 1.0
    A[ns + 1, k2] = 1.0
    A[ns + 2, :ns] = f0hat
    A[ns + 2, ns + 1] = 1.0
    A[ns + 2, ns + 2] = 1.0
    rhs = np.concatenate([PGsb + EinvLw, [t1, t2, -Gamma_w]])
    x = np.linalg.solve(A, rhs)
    ft = x[:ns]
    return f0 * ft, ft, x[ns], x[ns + 1], x[ns + 2]


def sheet_kutta_shed2_schur3(sch, sbp, EinvLw, k1, k2, EinvLd1, EinvLd2, Gamma_w):
    """Same solution from the unsplit 3x3 Schur problem (Eq. schurkutta2)."""
    fts = intermediate_sheet(sch, sbp, EinvLw)
    ft1 = sch.solve_tilde(EinvLd1)
    ft2 = sch.solve_tilde(EinvLd2)
    Sm = np.array([[-1.0, ft1[k1], ft2[k1]],
                   [-1.0, ft1[k2], ft2[k2]],
                   [-sch.Gamma0, 1.0 + np.dot(sch.f0hat, ft1), 1.0 + np.dot(sch.f0hat, ft2)]])
    rhs = np.array([-fts[k1], -fts[k2], -Gamma_w - np.dot(sch.f0hat, fts)])
    s0, G1, G2 = np.linalg.solve(Sm, rhs)
    ft = fts + G1 * ft1 + G2 * ft2 - s0 * sch.ones
    return sch.f0 * ft, ft, s0, G1, G2


def sheet_kutta_shed2_monolithic(S, f0, f0hat, PGsb, EinvLw, k1, k2, EinvLd1, EinvLd2, Gamma_w):
    """Dense solve of the reduced (Ns+3) system of Eq. kuttasystem3.

    Unknowns (ftilde, s0, Gamma1, Gamma2); rows:
      Stilde ftilde + s0 1 - Gamma1 E L^{-1} d1 - Gamma2 E L^{-1} d2 = P^Gamma s'_b + E L^{-1} w
      e_k1^T ftilde = 0,  e_k2^T ftilde = 0,  f0hat^T ftilde + Gamma1 + Gamma2 = -Gamma_w.
    """
    ns = S.shape[0]
    A = np.zeros((ns + 3, ns + 3))
    A[:ns, :ns] = S * f0[None, :]
    A[:ns, ns] = 1.0
    A[:ns, ns + 1] = -EinvLd1
    A[:ns, ns + 2] = -EinvLd2
    A[ns, k1] = 1.0
    A[ns + 1, k2] = 1.0
    A[ns + 2, :ns] = f0hat
    A[ns + 2, ns + 1] = 1.0
    A[ns + 2, ns + 2] = 1.0
    rhs = np.concatenate([PGsb + EinvLw, [0.0, 0.0, -Gamma_w]])
    x = np.linalg.solve(A, rhs)
    ft = x[:ns]
    return f0 * ft, ft, x[ns], x[ns + 1], x[ns + 2]


# ----------------------------------------------------------------- several bodies
def body_indicators(starts, ns):
    """Columns 1_b (Sec. 2.7): one where a surface point belongs to body b.
    Body b holds the points starts[b] .. starts[b+1]-1 of the concatenated set."""
    nb = len(starts) - 1
    ind = np.zeros((ns, nb))
    for b in range(nb):
        ind[starts[b]:starts[b + 1], b] = 1.0
    return ind


def _edge_list(edges):
    """Edges in body order, with the body each belongs to."""
    kk, owner = [], []
    for b, eb in enumerate(edges):
        for k in eb:
            kk.append(int(k))
            owner.append(b)
    return kk, owner


def sheet_multibody_shed(sch, sbp, EinvLw, starts, edges, EinvLds, Gamma_ws):
    """Several bodies sharing one Schur complement (Sec. 2.7, Eq. kuttasystem4).

    The surface points of all bodies are concatenated; body b has its own
    uniform value s0_b (the term sum_b 1_b s0_b), a Kutta condition at each of
    its edges (edges[b]: 0, 1 or 2 surface indices) with one new vortex per
    edge, and Kelvin's condition over itself and the vorticity it released:
    <1_b, f> + (its new strengths) = -Gamma_ws[b].  A body without edges is
    circulation-constrained (its Gamma_ws is minus the prescribed circulation).
    EinvLds[:, i] = E L^{-1} d_i for the new vortex of the i-th edge (edges in
    body order).

    Split form, as Eq. twovortex generalised: ftilde* and ftilde_i as for one
    body, g_b = Stilde^{-1} 1_b, ftilde = ftilde* + sum_i Gamma_i ftilde_i -
    sum_b s0_b g_b; the E Kutta rows e_k^T ftilde = 0 and the B Kelvin rows
    f0hat_b^T ftilde + sum_{i of b} Gamma_i = -Gamma_w,b (f0hat_b = f0hat o 1_b)
    are a dense (E + B) system in (Gamma, s0).  Returns (f, ftilde, s0, Gammas).
    """
    ns = len(sbp)
    ind = body_indicators(starts, ns)
    nb = ind.shape[1]
    kk, owner = _edge_list(edges)
    ne = len(kk)
    fts = intermediate_sheet(sch, sbp, EinvLw)
    ftj = [sch.solve_tilde(EinvLds[:, i]) for i in range(ne)]
    gb = [sch.solve_tilde(ind[:, b]) for b in range(nb)]
    M = np.zeros((ne + nb, ne + nb))
    rhs = np.zeros(ne + nb)
    for r, k in enumerate(kk):                        # Kutta rows
        for i in range(ne):
            M[r, i] = ftj[i][k]
        for b in range(nb):
            M[r, ne + b] = -gb[b][k]
        rhs[r] = -fts[k]
    for c in range(nb):                               # Kelvin rows
        f0h = sch.f0hat * ind[:, c]
        for i in range(ne):
            M[ne + c, i] = float(np.dot(f0h, ftj[i])) + (1.0 if owner[i] == c else 0.0)
        for b in range(nb):
            M[ne + c, ne + b] = -float(np.dot(f0h, gb[b]))
        rhs[ne + c] = -Gamma_ws[c] - float(np.dot(f0h, fts))
    x = np.linalg.solve(M, rhs)
    G, s0 = x[:ne], x[ne:]
    ft = fts + sum(G[i] * ftj[i] for i in range(ne)) - sum(s0[b] * gb[b] for b in range(nb))
    return sch.f0 * ft, ft, s0, G


def sheet_multibody_monolithic(S, f0, f0hat, PGsb, EinvLw, starts, edges, EinvLds, Gamma_ws):
    """Dense solve of Eq. kuttasystem4 with psi eliminated, unknowns
    (ftilde, s0_1..s0_B, Gamma_1..Gamma_E):
      Stilde ftilde + sum_b s0_b 1_b - sum_i Gamma_i E L^{-1} d_i = P^Gamma s'_b + E L^{-1} w
      e_k^T ftilde = 0 at every edge
      f0hat_b^T ftilde + sum_{i of b} Gamma_i = -Gamma_w,b for every body."""
    ns = S.shape[0]
    ind = body_indicators(starts, ns)
    nb = ind.shape[1]
    kk, owner = _edge_list(edges)
    ne = len(kk)
    n = ns + nb + ne
    A = np.zeros((n, n))
    A[:ns, :ns] = S * f0[None, :]
    A[:ns, ns:ns + nb] = ind
    for i in range(ne):
        A[:ns, ns + nb + i] = -EinvLds[:, i]
        A[ns + i, kk[i]] = 1.0
    for b in range(nb):
        A[ns + ne + b, :ns] = f0hat * ind[:, b]
        for i in range(ne):
            if owner[i] == b:
                A[ns + ne + b, ns + nb + i] = 1.0
    rhs = np.concatenate([PGsb + EinvLw, np.zeros(ne), -np.asarray(Gamma_ws, dtype=np.float64)])
    x = np.linalg.solve(A, rhs)
    ft = x[:ns]
    return f0 * ft, ft, x[ns:ns + nb], x[ns + nb:]
