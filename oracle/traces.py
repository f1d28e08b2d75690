"""Corrected interpolation of one-sided boundary data (Sec. 5.5) — oracle.

For a boundary point p the grid values are made smooth across Gamma with the
correction function before a polynomial fit: for the '+' (Omega) side the data
are v(q) + C(q) at nodes q outside Omega and v(q) inside; for the '-' side
v(q) - C(q) at inside nodes and v(q) outside.  The fitted Taylor polynomial of
degree p in (q - p)/h gives the one-sided value (coefficient of 1) and normal
derivative (n . gradient coefficients / h).

Reading of the interpolation stencil (the paper leaves it open and its Taylor
factor is garbled): for the side s, the nodes of side s within R_s h of p plus
the irregular nodes of the other side within R_o h of p (squared distances in
units of h, compared with R^2), fitted by weighted least squares with the weight
exp(-|q - p|^2 / (4 h^2)) on each equation.  C is then
needed only at irregular nodes, one grid step from Gamma, where the local
Cauchy problem is well conditioned (Sec. 5.3: the solution is needed "one step
away from the boundary"); nodes farther across Gamma would see the
exponential growth of rough density modes in the Cauchy extension.  The
Gaussian weight keeps the fit local where a one-sided extension has a short
radius of analyticity (high-curvature tips).
R_s = 4, R_o = 2.5 (p = 4); R_s = 3, R_o = 1.5 (p = 2).

Several interfaces (labels l, C^(l) as in ``correction``): at a point of
Gamma^(k) the '+' side is label t = 1 + k and the '-' side label t = 0; the
datum of a node q of another label is made smooth from side t with
u(q) + C^(t)(q) - C^(l_q)(q).  Reading: where another interface is close (a
node of a third label, neither 0 nor 1 + k, within R_s h of the point) every
node of another label within R_o h is taken, irregular or not.  Between two
close interfaces the side in the gap holds only the one or two grid columns
inside the gap, and the irregular nodes on either side add one more each:
too few distinct columns for a degree-p fit (the least-squares problem is
rank deficient).  C^(t) and C^(l_q) are then needed at nodes up to R_o h
from their own interfaces (further correction entries).  Elsewhere the rule
of one interface holds, node for node.
"""
from __future__ import annotations

import numpy as np

from . import collocation as CO
from . import geometry as G


TRACE_WEIGHT_SCALE = 4.0


def radii(order: int):
    return (4.0, 2.5) if order == 4 else (3.0, 1.5)


def disc_offsets(d: int, rs: float) -> np.ndarray:
    """Integer offsets o with |o| <= ceil(rs) + 1 per axis (candidate window)."""
    r = int(np.ceil(rs)) + 1
    rng = np.arange(-r, r + 1)
    return np.stack(np.meshgrid(*([rng] * d), indexing="ij"), -1).reshape(-1, d)


def trace_stencils(grid: G.Grid, x: np.ndarray, nrm: np.ndarray, labels: np.ndarray,
                   irr: np.ndarray, order: int, iface=None, holds=None):
    """Per DOF: for each side, the stencil nodes and least-squares weight rows
    for the value and the normal derivative.  Returns a list over DOFs of
    dicts {side: (nodes (k, d), w_value (k,), w_dn (k,), t)}, side in (+1, -1),
    t the side's label, and a flag `close` per DOF.  `iface`: interface of
    each DOF (default 0); `holds[k]`: grid mask of the nodes with a correction
    entry for k (needed only with several interfaces)."""
    lab = labels.astype(np.int64)
    if iface is None:
        iface = np.zeros(x.shape[0], dtype=np.int64)
    d = grid.dim
    E = CO.exponents(d, order)
    rs, ro = radii(order)
    offs = disc_offsets(d, rs)
    out = []
    for j in range(x.shape[0]):
        p = x[j]
        n0 = G.round_half_up((p - grid.lo) / grid.h)
        nodes = n0 + offs
        ok = np.all((nodes >= 0) & (nodes <= grid.n), axis=1)
        nodes = nodes[ok]
        xi = (grid.coord(nodes) - p) / grid.h
        r2 = xi[:, 0] * xi[:, 0]
        for k in range(1, d):
            r2 = r2 + xi[:, k] * xi[:, k]
        idx = tuple(nodes.T)
        lq = lab[idx]
        # a third label within R_s h: another interface is close
        close = bool(np.any((lq != 0) & (lq != int(iface[j]) + 1) & (r2 <= rs * rs)))
        ir = np.ones(lq.shape, dtype=bool) if close else irr[idx]
        rec = {"close": close}
        for side in (1, -1):
            t = int(iface[j]) + 1 if side == 1 else 0
            same = lq == t
            avail = (np.ones(lq.shape, dtype=bool) if (t == 0 or holds is None or close)
                     else holds[t - 1][idx])
            keep = (same & (r2 <= rs * rs)) | (~same & ir & avail & (r2 <= ro * ro))
            wt = np.exp(-r2[keep] / TRACE_WEIGHT_SCALE)
            V = CO.phi(E, xi[keep]) * wt[:, None]
            P = np.linalg.pinv(V) * wt[None, :]
            wv = P[0]
            wn = (nrm[j] @ P[1:1 + d]) / grid.h
            rec[side] = (nodes[keep], wv, wn, t)
        out.append(rec)
    return out


def one_sided(stencils, u: np.ndarray, cgrids: np.ndarray, labels: np.ndarray):
    """(value^+, value^-, d_n^+, d_n^-) at every DOF from grid values u and the
    correction functions on the grid (cgrids[l] = C^(l), cgrids[0] = 0)."""
    nb = len(stencils)
    lab = labels.astype(np.int64)
    vp, vm, dp, dm = (np.zeros(nb) for _ in range(4))
    for j, rec in enumerate(stencils):
        for side in (1, -1):
            nodes, wv, wn, t = rec[side]
            idx = tuple(nodes.T)
            lq = lab[idx]
            shift = cgrids[t][idx] - cgrids[(lq,) + idx]
            w = np.where(lq == t, u[idx], u[idx] + shift)
            if side == 1:
                vp[j], dp[j] = wv @ w, wn @ w
            else:
                vm[j], dm[j] = wv @ w, wn @ w
    return vp, vm, dp, dm
