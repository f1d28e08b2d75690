"""Correction function and corrected right-hand side (Sec. 5.2, 5.3) — oracle.

* Partition of unity with the closest-point weight of Sec. 5.3: C_h(x) =
  C_{h,i*}(x) where p_{i*} is the primary point closest to x.  Reading for ties:
  squared distances |x - p_i|^2 are compared, and every i within 1e-12 h^2 of the
  minimum counts as closest; the lowest index among them wins.
* Irregular nodes I_h (Sec. 5.2): interior nodes whose stencil set S_P holds
  nodes of both classes.
* Correction term (eq. (crc-formula)), with c the full stencil coefficients
  (which already carry 1/h^2; reading of the LTE derivation, eq. (LTE)):
      C_P = - sum_{Q in S_P, Q outside} c_{Q-P} C(Q)   for P inside,
      C_P = + sum_{Q in S_P, Q inside}  c_{Q-P} C(Q)   for P outside.
* Several interfaces (the remark on arbitrarily close interfaces, Sec. 5.2):
  nodes carry labels l (0 outside, 1 + k in Omega^(k)), C^(k) = u^(k) - u^(0)
  is the correction function of interface k (C^(0) = 0), and the value that
  makes Q's datum smooth from P's side is u^(l_P)(Q) - u^(l_Q)(Q) =
  C^(l_P)(Q) - C^(l_Q)(Q), so
      C_P = - sum_{Q in S_P, l_Q != l_P} c_{Q-P} (C^(l_P)(Q) - C^(l_Q)(Q)),
  which is the rule above for one interface.  Irregular nodes: interior nodes
  with a node of another label in S_P.  C^(k) is held at every irregular node
  Q for each k >= 1 among the labels of S_Q (Q included): the correction
  entries, ordered by node (C order) then k.  Each entry takes the closest
  primary point of its own interface.
"""
from __future__ import annotations

import numpy as np
import scipy.spatial

from . import boxsolve as BS

TIE_EPS = 1e-12


def stencil_offsets(d: int, order: int):
    """S_P offsets: all of {-1,0,1}^d (compact scheme) or the 5/7-point star."""
    offs = BS.offsets(d)
    if order == 2:
        offs = [o for o in offs if sum(1 for v in o if v != 0) <= 1]
    return offs


def irregular_nodes(labels: np.ndarray, order: int) -> np.ndarray:
    """Boolean mask of I_h over the grid (only interior nodes can be set):
    nodes P with a node of another label (class, for one interface) in S_P."""
    lab = labels.astype(np.int64)
    d = lab.ndim
    n = lab.shape[0] - 1
    inner = tuple(slice(1, n) for _ in range(d))
    other = np.zeros((n - 1,) * d, dtype=bool)
    for o in stencil_offsets(d, order):
        sl = tuple(slice(1 + ok, n + ok) for ok in o)
        other |= lab[sl] != lab[inner]
    mask = np.zeros(lab.shape, dtype=bool)
    mask[inner] = other
    return mask


def correction_entries(labels: np.ndarray, irr: np.ndarray, order: int):
    """(nodes (ne, d), iface (ne,)): the correction entries (node Q, k) in
    node order then k, for k + 1 among the labels >= 1 of S_Q."""
    lab = labels.astype(np.int64)
    d = lab.ndim
    nodes = np.argwhere(irr)                   # interior nodes: S_Q in the grid
    nk = max(int(lab.max()), 1)
    has = np.zeros((nodes.shape[0], nk), dtype=bool)
    for o in stencil_offsets(d, order):
        v = lab[tuple((nodes + np.asarray(o)).T)]
        for k in range(nk):
            has[:, k] |= v == k + 1
    qi, k = np.nonzero(has)                    # node order, then k
    return nodes[qi], k.astype(np.int64)


def closest_primary(points: np.ndarray, x: np.ndarray, h: float) -> np.ndarray:
    """Index of the closest primary point to each x (tie rule above).  A k-d tree
    proposes the 8 nearest candidates; the rule is then applied exactly."""
    k = min(8, points.shape[0])
    tree = scipy.spatial.cKDTree(points)
    _, cand = tree.query(x, k=k)
    cand = np.asarray(cand).reshape(x.shape[0], k)
    diff = x[:, None, :] - points[cand]
    d2 = diff[..., 0] * diff[..., 0]
    for j in range(1, x.shape[1]):
        d2 = d2 + diff[..., j] * diff[..., j]
    dmin = d2.min(axis=1)
    ok = d2 <= dmin[:, None] + TIE_EPS * h * h
    big = np.iinfo(np.int64).max
    return np.where(ok, cand, big).min(axis=1)


def correction_terms(cgrids: np.ndarray, labels: np.ndarray, irr: np.ndarray,
                     d: int, order: int, h: float, kappa: float) -> np.ndarray:
    """C_P of eq. (crc-formula) on the grid (zero off I_h).  cgrids[l] holds
    C^(l)(Q) (cgrids[0] = 0) at every node where it is needed (the entries)."""
    c = BS.stencil_coeffs(d, order, h, kappa)
    lab = labels.astype(np.int64)
    n = lab.shape[0] - 1
    inner = tuple(slice(1, n) for _ in range(d))
    lp = lab[inner]
    acc = np.zeros((n - 1,) * d)
    for o in stencil_offsets(d, order):
        w = BS.coeff_of(c, o)
        sl = tuple(slice(1 + ok, n + ok) for ok in o)
        lq = lab[sl]
        c_p = np.take_along_axis(cgrids[(slice(None),) + sl], lp[None], 0)[0]   # C^(l_P)(Q)
        c_q = np.take_along_axis(cgrids[(slice(None),) + sl], lq[None], 0)[0]   # C^(l_Q)(Q)
        acc += np.where(lq != lp, w * (c_q - c_p), 0.0)
    out = np.zeros(lab.shape)
    out[inner] = np.where(irr[inner], acc, 0.0)
    return out
