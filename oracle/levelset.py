"""Analytic level-set functions H and their gradients (Sec. 5.1).

Omega = {H < 0}; Gamma = {H = 0}; n = grad H / |grad H| (outward from Omega).
Kind codes and parameter layouts are the ones in ``workloads``.
"""
from __future__ import annotations

import numpy as np

import workloads as W


class Sampled:
    """A level-set function known by its values at the grid nodes (the
    grid-sampled kind): samples of shape (N+1,)*d on [lo, lo + N h]^d.
    Between nodes H is the tensor-product cubic Lagrange interpolant on the
    4^d nodes around the point (O(h^4) away from the nodes, exact at them,
    exact for every polynomial of degree <= 3 per axis)."""

    def __init__(self, samples, lo: float, h: float):
        self.samples = np.asarray(samples, dtype=np.float64)
        self.d = self.samples.ndim
        self.n = self.samples.shape[0] - 1
        self.lo = float(lo)
        self.h = float(h)


def params(w):
    """The level-set parameters of a workload as the functions below take them:
    a Sampled object for the grid-sampled kind, the parameter list otherwise."""
    if w.ls_kind == W.LS_GRID:
        return Sampled(w.extra["samples"], w.lo, w.h)
    return w.ls_params


# Cubic Lagrange basis on the nodes t = -1, 0, 1, 2 of the cell [0, 1] and its
# derivative (every product written out in the same order as on the GPU)
def _lagrange(t):
    tm1, tm2, tp1 = t - 1.0, t - 2.0, t + 1.0
    w = [-(t * tm1 * tm2) / 6.0, (tp1 * tm1 * tm2) / 2.0, -(tp1 * t * tm2) / 2.0, (tp1 * t * tm1) / 6.0]
    dw = [-(tm1 * tm2 + t * tm2 + t * tm1) / 6.0, (tm1 * tm2 + tp1 * tm2 + tp1 * tm1) / 2.0,
          -(t * tm2 + tp1 * tm2 + tp1 * t) / 2.0, (t * tm1 + tp1 * tm1 + tp1 * t) / 6.0]
    return w, dw


def _cell(S: Sampled, xk):
    """Per axis: the first of the four interpolation nodes i0 - 1 (i0 clamped
    to [1, N - 2]) and the local coordinate t in the cell [i0, i0 + 1].  A
    coordinate within 1e-10 (in units of h) of a node is taken as that node,
    so H at a node is its sample exactly."""
    u = (xk - S.lo) / S.h
    k = np.rint(u)
    u = np.where(np.abs(u - k) <= 1e-10, k, u)
    i0 = np.clip(np.floor(u), 1, S.n - 2)
    return i0.astype(np.int64) - 1, u - i0


def _sampled(S: Sampled, X: np.ndarray, grad: bool):
    X = np.asarray(X, dtype=np.float64)
    shp = X.shape[:-1]
    Xf = X.reshape(-1, S.d)
    base, wts, dwts = [], [], []
    for k in range(S.d):
        b, t = _cell(S, Xf[:, k])
        w, dw = _lagrange(t)
        base.append(b)
        wts.append(w)
        dwts.append(dw)
    val = np.zeros(Xf.shape[0])
    g = np.zeros(Xf.shape)
    if S.d == 2:
        for a in range(4):
            row = np.zeros(Xf.shape[0])
            drow = np.zeros(Xf.shape[0])
            for b in range(4):
                v = S.samples[base[0] + a, base[1] + b]
                row = row + wts[1][b] * v
                drow = drow + dwts[1][b] * v
            val = val + wts[0][a] * row
            g[:, 0] = g[:, 0] + dwts[0][a] * row
            g[:, 1] = g[:, 1] + wts[0][a] * drow
    else:
        for a in range(4):
            for b in range(4):
                row = np.zeros(Xf.shape[0])
                drow = np.zeros(Xf.shape[0])
                for c in range(4):
                    v = S.samples[base[0] + a, base[1] + b, base[2] + c]
                    row = row + wts[2][c] * v
                    drow = drow + dwts[2][c] * v
                wab = wts[0][a] * wts[1][b]
                val = val + wab * row
                g[:, 0] = g[:, 0] + (dwts[0][a] * wts[1][b]) * row
                g[:, 1] = g[:, 1] + (wts[0][a] * dwts[1][b]) * row
                g[:, 2] = g[:, 2] + wab * drow
    g = g / S.h
    return (g.reshape(shp + (S.d,)) if grad else val.reshape(shp))


def H(kind: int, p, X: np.ndarray) -> np.ndarray:
    """Level-set value at points X (..., d)."""
    if kind == W.LS_GRID:
        return _sampled(p, X, False)
    if kind == W.LS_ELLIPSE:
        cx, cy, a, b, th = p[:5]
        x = X[..., 0] - cx
        y = X[..., 1] - cy
        c, s = np.cos(th), np.sin(th)
        u = (x * c + y * s) / a
        v = (y * c - x * s) / b
        return u * u + v * v - 1.0
    if kind == W.LS_STAR:
        cx, cy, r0, amp, k = p[:5]
        x = X[..., 0] - cx
        y = X[..., 1] - cy
        r = np.sqrt(x * x + y * y)
        th = np.arctan2(y, x)
        return r - r0 - amp * np.sin(k * th)
    if kind == W.LS_ELLIPSOID:
        cx, cy, cz, a, b, c = p[:6]
        u = (X[..., 0] - cx) / a
        v = (X[..., 1] - cy) / b
        w = (X[..., 2] - cz) / c
        return u * u + v * v + w * w - 1.0
    if kind == W.LS_TORUS:
        big, small = p[:2]
        x, y, z = X[..., 0], X[..., 1], X[..., 2]
        rho = np.sqrt(x * x + y * y)
        t = rho - big
        return t * t + z * z - small * small
    if kind in (W.LS_DISCS, W.LS_SPHERES):
        return _nearest_ball(p, 2 if kind == W.LS_DISCS else 3, X)[1]
    if kind == W.LS_UNION:
        return _union_argmin(p, X)[1]
    if kind == W.LS_MOLECULE:
        r, level, na = p[0], p[1], int(p[2])
        acc = np.zeros(X.shape[:-1])
        for k in range(na):
            cx, cy, cz = p[3 + 3 * k: 6 + 3 * k]
            dx = X[..., 0] - cx
            dy = X[..., 1] - cy
            dz = X[..., 2] - cz
            acc = acc + np.exp(-(dx * dx + dy * dy + dz * dz) / (r * r))
        return level - acc
    raise ValueError(f"unknown level-set kind {kind}")


def _nearest_ball(p, d: int, X: np.ndarray):
    """Union of n equal discs/balls (Sec. 5.1 with several interfaces): per
    point the first centre with the smallest |X - c_k|^2 - r^2, and that value
    (sums in the order x, y, z, then minus r^2)."""
    r, n = p[0], int(p[1])
    best = np.zeros(X.shape[:-1], dtype=np.int64)
    bv = None
    for k in range(n):
        c = p[2 + d * k: 2 + d * (k + 1)]
        v = (X[..., 0] - c[0]) * (X[..., 0] - c[0]) + (X[..., 1] - c[1]) * (X[..., 1] - c[1])
        if d == 3:
            v = v + (X[..., 2] - c[2]) * (X[..., 2] - c[2])
        v = v - r * r
        if bv is None:
            bv = v
        else:
            take = v < bv
            bv = np.where(take, v, bv)
            best = np.where(take, k, best)
    return best, bv


def n_interfaces(kind: int, p) -> int:
    """Interfaces Gamma^(k) (components Omega^(k) of Omega) the level set
    describes: the balls of a ball union, the components of a union, else one."""
    if kind in (W.LS_DISCS, W.LS_SPHERES):
        return int(p[1])
    if kind == W.LS_UNION:
        return int(p[0])
    return 1


def _union_argmin(p, X: np.ndarray):
    """Per point the first component with the smallest H_k, and that value."""
    best = np.zeros(X.shape[:-1], dtype=np.int64)
    bv = None
    for k, (kind, q) in enumerate(W.union_components(p)):
        v = H(kind, q, X)
        if bv is None:
            bv = v
        else:
            take = v < bv
            bv = np.where(take, v, bv)
            best = np.where(take, k, best)
    return best, bv


def labels(kind: int, p, X: np.ndarray) -> np.ndarray:
    """Side label of points X (the remark on arbitrarily close interfaces in
    Sec. 5.2 with Omega^(0) outside): 0 outside Omega, 1 + k in Omega^(k).
    Several interfaces: k is the first interface with the smallest H_k (for a
    point inside two overlapping components, the one it lies deeper in)."""
    if kind in (W.LS_DISCS, W.LS_SPHERES):
        k, v = _nearest_ball(p, 2 if kind == W.LS_DISCS else 3, X)
        return np.where(v < 0.0, k + 1, 0).astype(np.uint8)
    if kind == W.LS_UNION:
        k, v = _union_argmin(p, X)
        return np.where(v < 0.0, k + 1, 0).astype(np.uint8)
    return np.where(H(kind, p, X) < 0.0, 1, 0).astype(np.uint8)


def H_iface(kind: int, p, k: int, X: np.ndarray) -> np.ndarray:
    """Level-set function H_k of interface k alone: |X - c_k|^2 - r^2 for ball
    k of a ball union (the arithmetic of _nearest_ball), the component's own
    function for a union, H itself for one interface."""
    if kind == W.LS_UNION:
        ck, q = W.union_components(p)[k]
        return H(ck, q, X)
    if kind in (W.LS_DISCS, W.LS_SPHERES):
        d = 2 if kind == W.LS_DISCS else 3
        r = p[0]
        c = p[2 + d * k: 2 + d * (k + 1)]
        v = (X[..., 0] - c[0]) * (X[..., 0] - c[0]) + (X[..., 1] - c[1]) * (X[..., 1] - c[1])
        if d == 3:
            v = v + (X[..., 2] - c[2]) * (X[..., 2] - c[2])
        return v - r * r
    return H(kind, p, X)


def grad_H_iface(kind: int, p, k: int, X: np.ndarray) -> np.ndarray:
    """Gradient of H_k."""
    if kind == W.LS_UNION:
        ck, q = W.union_components(p)[k]
        return grad_H(ck, q, X)
    if kind in (W.LS_DISCS, W.LS_SPHERES):
        d = 2 if kind == W.LS_DISCS else 3
        c = np.asarray(p[2 + d * k: 2 + d * (k + 1)], dtype=np.float64)
        return 2.0 * (X[..., :d] - c)
    return grad_H(kind, p, X)


def grad_H(kind: int, p, X: np.ndarray) -> np.ndarray:
    """Analytic gradient of H at points X (..., d) (of the interpolant for
    the grid-sampled kind)."""
    if kind == W.LS_GRID:
        return _sampled(p, X, True)
    if kind == W.LS_ELLIPSE:
        cx, cy, a, b, th = p[:5]
        x = X[..., 0] - cx
        y = X[..., 1] - cy
        c, s = np.cos(th), np.sin(th)
        u = (x * c + y * s) / a
        v = (y * c - x * s) / b
        gx = 2.0 * u * (c / a) + 2.0 * v * (-s / b)
        gy = 2.0 * u * (s / a) + 2.0 * v * (c / b)
        return np.stack([gx, gy], -1)
    if kind == W.LS_STAR:
        cx, cy, r0, amp, k = p[:5]
        x = X[..., 0] - cx
        y = X[..., 1] - cy
        r2 = x * x + y * y
        r = np.sqrt(r2)
        th = np.arctan2(y, x)
        dth = amp * k * np.cos(k * th)
        gx = x / r + dth * y / r2
        gy = y / r - dth * x / r2
        return np.stack([gx, gy], -1)
    if kind == W.LS_ELLIPSOID:
        cx, cy, cz, a, b, c = p[:6]
        return np.stack([2.0 * (X[..., 0] - cx) / (a * a),
                         2.0 * (X[..., 1] - cy) / (b * b),
                         2.0 * (X[..., 2] - cz) / (c * c)], -1)
    if kind == W.LS_TORUS:
        big, small = p[:2]
        x, y, z = X[..., 0], X[..., 1], X[..., 2]
        rho = np.sqrt(x * x + y * y)
        f = 2.0 * (rho - big) / rho
        return np.stack([f * x, f * y, 2.0 * z], -1)
    if kind in (W.LS_DISCS, W.LS_SPHERES):
        d = 2 if kind == W.LS_DISCS else 3
        k, _ = _nearest_ball(p, d, X)
        C = np.asarray(p[2: 2 + d * int(p[1])], dtype=np.float64).reshape(-1, d)[k]
        return 2.0 * (X[..., :d] - C)
    if kind == W.LS_UNION:
        k, _ = _union_argmin(p, X)
        g = np.zeros(X.shape)
        for j, (ck, q) in enumerate(W.union_components(p)):
            g = np.where((k == j)[..., None], grad_H(ck, q, X), g)
        return g
    if kind == W.LS_MOLECULE:
        r, level, na = p[0], p[1], int(p[2])
        g = np.zeros(X.shape)
        for k in range(na):
            cx, cy, cz = p[3 + 3 * k: 6 + 3 * k]
            d = X - np.array([cx, cy, cz])
            e = np.exp(-np.sum(d * d, -1) / (r * r))
            g = g + (2.0 / (r * r)) * e[..., None] * d
        return g
    raise ValueError(f"unknown level-set kind {kind}")
