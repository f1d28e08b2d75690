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


def irregular_nodes(inside: np.ndarray, order: int) -> np.ndarray:
    """Boolean mask of I_h over the grid (only interior nodes can be set)."""
    d = inside.ndim
    n = inside.shape[0] - 1
    inner = tuple(slice(1, n) for _ in range(d))
    any_in = np.zeros((n - 1,) * d, dtype=bool)
    any_out = np.zeros((n - 1,) * d, dtype=bool)
    for o in stencil_offsets(d, order):
        sl = tuple(slice(1 + ok, n + ok) for ok in o)
        any_in |= inside[sl]
        any_out |= ~inside[sl]
    mask = np.zeros_like(inside)
    mask[inner] = any_in & any_out
    return mask


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


def correction_terms(cgrid: np.ndarray, inside: np.ndarray, irr: np.ndarray,
                     d: int, order: int, h: float, kappa: float) -> np.ndarray:
    """C_P of eq. (crc-formula) on the grid (zero off I_h).  `cgrid` holds C(Q)
    at every node where it is needed (at least all of I_h)."""
    c = BS.stencil_coeffs(d, order, h, kappa)
    n = inside.shape[0] - 1
    inner = tuple(slice(1, n) for _ in range(d))
    ins = inside[inner]
    acc = np.zeros((n - 1,) * d)
    for o in stencil_offsets(d, order):
        w = BS.coeff_of(c, o)
        sl = tuple(slice(1 + ok, n + ok) for ok in o)
        q_in = inside[sl]
        cq = cgrid[sl]
        # P inside: subtract over outside Q; P outside: add over inside Q.
        acc += np.where(ins & ~q_in, -w * cq, 0.0)
        acc += np.where(~ins & q_in, w * cq, 0.0)
    out = np.zeros_like(cgrid)
    out[inner] = np.where(irr[inner], acc, 0.0)
    return out
