"""Geometry of the KFBI discretisation (Sec. 5.1, 5.2, 5.4) — oracle.

Grid: box [lo, hi]^d, N intervals, h = (hi - lo)/N, nodes x_i = lo + i h,
arrays of shape (N+1,)*d with axis d-1 fastest (C order).

Steps, in the paper's order:
  * classification of nodes (Sec. 5.2): inside Omega iff H(node) < 0; with
    several interfaces Gamma^(k) every node also carries the label of its
    side (0 outside, 1 + k inside Gamma^(k)), the subdomains Omega^(i) of the
    remark on arbitrarily close interfaces (Sec. 5.2);
  * intersections of Gamma with grid lines by a bracketed Newton/bisection
    iteration (Sec. 5.1), unit normal n = grad H/|grad H|.  A grid edge whose
    end nodes carry labels a != b crosses Gamma^(a-1) (if a > 0) and
    Gamma^(b-1) (if b > 0): one root of H_k per crossed interface k, so an
    edge between two close interfaces holds two points;
  * overlapping surface decomposition Gamma_r = {|n . e_r| > cos(alpha)}, Gamma_r^h
    = its intersections with e_r-lines, Gamma^h = union = the DOF set (Sec. 5.1);
  * reference plane Pi_m with m = argmax_k |n_k| (Sec. 5.1);
  * collocation-point selection (Sec. 5.4): interpolation sets of degree p-2
    (PDE, d-dim), p (Dirichlet, (d-1)-dim), p-1 (Neumann, (d-1)-dim).

Readings where the paper is silent (the same written rules bind the CUDA path):
  * cos(alpha) = 0.707 in 2D (reproduces the point counts N_b of Table 1),
    0.4 in 3D (alpha in (acos(1/sqrt d), pi/2));
  * DOF order: family r ascending, then the grid line (other axes
    lexicographic, lower axis slowest), then the edge position along the line,
    then, on an edge with two points, the interface of the edge's first node
    first;
  * an interface k is crossed on an edge only where H_k changes sign along
    it (a node inside two overlapping components takes the label of the one
    it lies deeper in, and the edge to the other component crosses one
    interface);
  * root iteration: start at the linear interpolant, Newton step, bisection
    whenever Newton leaves the bracket, stop when |ds| <= 1e-15 N h, 1e-15 of
    the box width, about the FP64 spacing of a coordinate there (<= 64
    steps);
  * stencil rules: see ``collocation_stencil``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

import workloads as W

from . import levelset as LS

ROOT_MAX_IT = 64
ROOT_TOL = 1e-15


@dataclass
class Grid:
    dim: int
    n: int
    lo: float
    h: float

    def coord(self, idx):
        """Node coordinate lo + i*h (two roundings, no fused multiply-add)."""
        return self.lo + np.asarray(idx, dtype=np.float64) * self.h

    def coords(self) -> np.ndarray:
        i = np.arange(self.n + 1)
        x = self.coord(i)
        return np.stack(np.meshgrid(*([x] * self.dim), indexing="ij"), -1)


def classify(grid: Grid, kind: int, p) -> np.ndarray:
    """Node classes (Sec. 5.2): True = inside Omega (H < 0), the '+' side."""
    return LS.H(kind, p, grid.coords()) < 0.0


def label_nodes(grid: Grid, kind: int, p) -> np.ndarray:
    """Node labels: 0 outside Omega, 1 + k in Omega^(k) (uint8)."""
    return LS.labels(kind, p, grid.coords())


def find_roots(grid: Grid, kind: int, p, x0: np.ndarray, r: int, iface: int = 0,
               steps: list | None = None) -> np.ndarray:
    """Offsets s in [0, h] with H_k(x0 + s e_r) = 0 (k = iface) on edges where
    H_k changes sign (Sec. 5.1), by Newton's method safeguarded with bisection.
    With a list `steps`, the number of steps each root took is appended."""
    h = grid.h
    m = x0.shape[0]
    Hk = lambda X: LS.H_iface(kind, p, iface, X)
    xb = x0.copy()
    xb[:, r] = grid.lo + (np.round((x0[:, r] - grid.lo) / h) + 1.0) * h
    ha = Hk(x0)
    hb = Hk(xb)
    neg_a = ha < 0.0
    s = h * ha / (ha - hb)
    lo_s = np.zeros(m)
    hi_s = np.full(m, h)
    active = np.ones(m, dtype=bool)
    taken = np.zeros(m, dtype=np.int64)
    for _ in range(ROOT_MAX_IT):
        if not active.any():
            break
        idx = np.nonzero(active)[0]
        taken[idx] += 1
        X = x0[idx].copy()
        X[:, r] = x0[idx, r] + s[idx]
        f = Hk(X)
        df = LS.grad_H_iface(kind, p, iface, X)[:, r]
        done_zero = f == 0.0
        same = (f < 0.0) == neg_a[idx]
        lo_s[idx] = np.where(same, s[idx], lo_s[idx])
        hi_s[idx] = np.where(same, hi_s[idx], s[idx])
        with np.errstate(divide="ignore", invalid="ignore"):
            s_new = s[idx] - f / df
        bad = ~((s_new > lo_s[idx]) & (s_new < hi_s[idx])) | (df == 0.0)
        s_new = np.where(bad, 0.5 * (lo_s[idx] + hi_s[idx]), s_new)
        s_new = np.where(done_zero, s[idx], s_new)
        conv = done_zero | (np.abs(s_new - s[idx]) <= ROOT_TOL * (grid.n * h))
        s[idx] = s_new
        active[idx[conv]] = False
    if steps is not None:
        steps.extend(taken.tolist())
    return s


@dataclass
class Surface:
    """The DOF set Gamma^h with its per-family line index (CSR)."""

    x: np.ndarray        # (Nb, d) point coordinates
    n: np.ndarray        # (Nb, d) unit outward normals
    family: np.ndarray   # (Nb,) r: the point lies on an e_r grid line
    line: np.ndarray     # (Nb,) linear index of that line over the other axes
    edge: np.ndarray     # (Nb,) index of the edge's first node along e_r
    axis: np.ndarray     # (Nb,) reference axis m = argmax |n_k|
    line_start: list     # per family: CSR offsets of length (N+1)^(d-1) + 1
    iface: np.ndarray    # (Nb,) the interface Gamma^(k) the point lies on

    @property
    def nb(self) -> int:
        return self.x.shape[0]


def other_axes(d: int, r: int):
    return [k for k in range(d) if k != r]


def surface_points(grid: Grid, kind: int, p, cos_alpha: float,
                   labels: np.ndarray) -> Surface:
    """Gamma^h = union over r of the e_r-line intersections with |n_r| > cos(alpha).
    `labels`: node labels (``label_nodes``); a boolean inside mask is accepted
    for level sets with one interface."""
    d, n = grid.dim, grid.n
    if labels.dtype == bool:
        assert LS.n_interfaces(kind, p) == 1
    lab = labels.astype(np.int64)
    xs, ns, fam, line, edge, ifc = [], [], [], [], [], []
    starts = []
    nl = (n + 1) ** (d - 1)
    for r in range(d):
        a = np.moveaxis(np.take(lab, np.arange(0, n), axis=r), r, -1)
        b = np.moveaxis(np.take(lab, np.arange(1, n + 1), axis=r), r, -1)
        idx = np.argwhere(a != b)                    # C order = DOF order
        la = a[tuple(idx.T)]
        lb = b[tuple(idx.T)]
        oth = other_axes(d, r)
        x0 = np.zeros((idx.shape[0], d))
        for j, ax in enumerate(oth):
            x0[:, ax] = grid.coord(idx[:, j])
        x0[:, r] = grid.coord(idx[:, -1])
        xb = x0.copy()
        xb[:, r] = grid.coord(idx[:, -1] + 1)
        # candidate points: slot 0 on the first node's interface, slot 1 on
        # the second node's, each only where that H_k changes sign
        cand = []
        for slot, lk in ((0, la), (1, lb)):
            for k in np.unique(lk[lk > 0] - 1):
                sel = np.nonzero((lk == k + 1))[0]
                ha = LS.H_iface(kind, p, int(k), x0[sel]) < 0.0
                hb = LS.H_iface(kind, p, int(k), xb[sel]) < 0.0
                sel = sel[ha != hb]
                if sel.size:
                    cand.append((sel, slot, int(k)))
        E, S, K, X, NRM = [], [], [], [], []
        for sel, slot, k in cand:
            s = find_roots(grid, kind, p, x0[sel], r, k)
            Xk = x0[sel].copy()
            Xk[:, r] = x0[sel, r] + s
            g = LS.grad_H_iface(kind, p, k, Xk)
            E.append(sel)
            S.append(np.full(sel.size, slot))
            K.append(np.full(sel.size, k))
            X.append(Xk)
            NRM.append(g / np.sqrt(np.sum(g * g, -1))[:, None])
        if E:
            E, S, K = np.concatenate(E), np.concatenate(S), np.concatenate(K)
            X, NRM = np.concatenate(X), np.concatenate(NRM)
        else:
            E = S = K = np.zeros(0, dtype=np.int64)
            X = NRM = np.zeros((0, d))
        order = np.lexsort((S, E))
        E, K, X, NRM = E[order], K[order], X[order], NRM[order]
        keep = np.abs(NRM[:, r]) > cos_alpha
        li = np.zeros(E.shape[0], dtype=np.int64)
        for j in range(d - 1):
            li = li * (n + 1) + idx[E, j]
        xs.append(X[keep])
        ns.append(NRM[keep])
        fam.append(np.full(int(keep.sum()), r))
        line.append(li[keep])
        edge.append(idx[E[keep], -1])
        ifc.append(K[keep])
        counts = np.bincount(li[keep], minlength=nl)
        starts.append(np.concatenate([[0], np.cumsum(counts)]))
    x = np.concatenate(xs)
    nn = np.concatenate(ns)
    off = np.cumsum([0] + [len(f) for f in fam])
    line_start = [st + off[r] for r, st in enumerate(starts)]
    axis = np.argmax(np.abs(nn), axis=1)
    return Surface(x, nn, np.concatenate(fam), np.concatenate(line),
                   np.concatenate(edge), axis, line_start,
                   np.concatenate(ifc).astype(np.int64))


# ---------------------------------------------------------------------------
# Collocation-point selection (Sec. 5.4)
# ---------------------------------------------------------------------------

def pde_offsets(d: int, order: int):
    """Grid-node offsets of the degree-(p-2) PDE interpolation set (unisolvent)."""
    if order == 2:
        return [(0,) * d]
    if d == 2:
        return [(0, 0), (1, 0), (-1, 0), (0, 1), (0, -1), (1, 1)]
    return [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1),
            (0, 0, -1), (1, 1, 0), (1, 0, 1), (0, 1, 1)]


def lattice_sets(order: int, shifted: bool = True):
    """3D reference-plane lattices for the Dirichlet (degree p) and Neumann
    (degree p-1) conditions, in a fixed order: the principal lattices
    {a, b >= 0, a + b <= deg}, shifted by (-1, -1) for p = 4 when `shifted`."""
    low = -1 if (order == 4 and shifted) else 0
    top_d = order + 2 * low
    top_n = order - 1 + 2 * low
    dset = [(a, b) for a in range(low, order + 1) for b in range(low, order + 1)
            if a + b <= top_d]
    nset = [(a, b) for (a, b) in dset if a + b <= top_n]
    return dset, nset


def n_boundary_points(d: int, order: int):
    if d == 2:
        return order + 1, order
    dset, nset = lattice_sets(order)
    return len(dset), len(nset)


def round_half_up(v):
    return np.floor(v + 0.5).astype(np.int64)


def axis_order(nrm: np.ndarray, m: int, cos_alpha: float):
    """Reference axes to try: m first, then the others by decreasing |n_k|
    (ties to the lower k) among those with |n_k| > cos(alpha)."""
    d = nrm.shape[0]
    rest = [k for k in range(d) if k != m and abs(nrm[k]) > cos_alpha]
    rest.sort(key=lambda k: (-abs(nrm[k]), k))
    return [m] + rest


class LineIndex:
    """Look-up of the DOFs of one family on one grid line."""

    def __init__(self, grid: Grid, surf: Surface):
        self.g = grid
        self.s = surf

    def nearest(self, fam: int, other_idx, s_pred: float, iface: int = 0) -> int:
        """DOF of family `fam` on interface `iface` on the e_fam line through the
        other-axis node indices `other_idx`, nearest to coordinate s_pred along
        e_fam, within 2h; ties to the lower DOF index; -1 if none."""
        n = self.g.n
        for j in other_idx:
            if j < 0 or j > n:
                return -1
        li = 0
        for j in other_idx:
            li = li * (n + 1) + j
        st = self.s.line_start[fam]
        best, bestd = -1, math.inf
        for q in range(st[li], st[li + 1]):
            if self.s.iface[q] != iface:
                continue
            dist = abs(self.s.x[q, fam] - s_pred)
            if dist <= 2.0 * self.g.h and dist < bestd:
                best, bestd = q, dist
        return best


class GeometryError(RuntimeError):
    pass


def collocation_stencil(grid: Grid, surf: Surface, lines: LineIndex, i: int,
                        order: int, cos_alpha: float):
    """Collocation points of primary point p_i (Sec. 5.4).

    Returns (pde_nodes (k, d) int, dir_dofs list, neu_dofs list, axis used).

    2D: reference line = e_m grid lines; candidates are the lines whose
    tangential index k is within 4 of round(kappa), kappa = (p_t - lo)/h, ordered
    by (|k - kappa|, k).  On each, the family-m DOF nearest to the tangent-line
    prediction s_pred = p_m - n_t (x_t - p_t)/n_m within 2h is taken; lines
    without one are skipped.  The first p+1 such points are the Dirichlet points,
    the first p the Neumann points.
    3D: the reference-plane node (j0, k0) nearest to the projection of p_i
    (round half up), sign s_k = +1 if the projection is >= the node, else -1, and
    the lattices (j0 + o1 a, k0 + o2 b) of ``lattice_sets``; every lattice line
    must carry a family-m DOF near the tangent-plane prediction.  Tried in turn:
    the shifted lattice with orientations (s1,s2), (-s1,s2), (s1,-s2), (-s1,-s2),
    then the unshifted lattice (one quadrant) with the same orientations.
    Both: if no point set is complete, the next reference axis (``axis_order``)
    is tried; otherwise GeometryError.
    PDE points: nodes round(p_i) + ``pde_offsets``.
    Several interfaces: only points of p_i's own interface are taken (the
    local Cauchy problem of Sec. 5.3 is posed on one interface).
    """
    d = grid.dim
    p = surf.x[i]
    nv = surf.n[i]
    n0 = round_half_up((p - grid.lo) / grid.h)
    pde = np.array([n0 + np.array(o) for o in pde_offsets(d, order)], dtype=np.int64)
    nd, nn = n_boundary_points(d, order)
    for m in axis_order(nv, int(surf.axis[i]), cos_alpha):
        if d == 2:
            t = 1 - m
            kap = (p[t] - grid.lo) / grid.h
            j0 = int(math.floor(kap + 0.5))
            cands = [k for k in range(j0 - 4, j0 + 5)]
            cands.sort(key=lambda k: (abs(k - kap), k))
            found = []
            for k in cands:
                xt = grid.lo + k * grid.h
                s_pred = p[m] - nv[t] * (xt - p[t]) / nv[m]
                q = lines.nearest(m, [k], s_pred, int(surf.iface[i]))
                if q >= 0:
                    found.append(q)
                    if len(found) == nd:
                        break
            if len(found) == nd:
                return pde, found, found[:nn], m
        else:
            t1, t2 = other_axes(3, m)
            k1 = (p[t1] - grid.lo) / grid.h
            k2 = (p[t2] - grid.lo) / grid.h
            j0 = int(math.floor(k1 + 0.5))
            l0 = int(math.floor(k2 + 0.5))
            s1 = 1 if k1 >= j0 else -1
            s2 = 1 if k2 >= l0 else -1
            tries = []
            for shifted in ((True, False) if order == 4 else (True,)):
                dset, nset = lattice_sets(order, shifted)
                for o in ((s1, s2), (-s1, s2), (s1, -s2), (-s1, -s2)):
                    tries.append((dset, nset, o))
            for dset, nset, (o1, o2) in tries:
                found = {}
                ok = True
                for (a, b) in dset:
                    j = j0 + o1 * a
                    k = l0 + o2 * b
                    x1 = grid.lo + j * grid.h
                    x2 = grid.lo + k * grid.h
                    s_pred = p[m] - (nv[t1] * (x1 - p[t1]) + nv[t2] * (x2 - p[t2])) / nv[m]
                    q = lines.nearest(m, [j, k], s_pred, int(surf.iface[i]))
                    if q < 0:
                        ok = False
                        break
                    found[(a, b)] = q
                if ok:
                    return (pde, [found[ab] for ab in dset],
                            [found[ab] for ab in nset], m)
    raise GeometryError(f"no complete collocation stencil at DOF {i}")
