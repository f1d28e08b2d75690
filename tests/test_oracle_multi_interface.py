"""Pins of several disjoint interfaces (the union-of-discs level set; the
separated case of Sec. 7.1.2's multiple interfaces, without multiply crossed
grid edges).

PM1 the geometry of the union is the union of the geometries: node classes
    are the OR of the single-disc classes, and the DOFs (family, grid line,
    position, normal) are those of the discs set up one at a time with the
    ellipse level set (a = b = r), a different formula for the same circle.
PM2 the interface problem on four discs converges at 4th order (> 12x from
    N = 128 to 256) on both sides.
"""
import numpy as np

import workloads as W
from oracle import geometry as G
from oracle import kfbi as K


def _dofs(w):
    grid = G.Grid(w.dim, w.n, w.lo, w.h)
    inside = G.classify(grid, w.ls_kind, w.ls_params)
    s = G.surface_points(grid, w.ls_kind, w.ls_params, w.cosa(), inside)
    return inside, s


def test_union_geometry_is_the_union():
    w = W.discs_interface_2d(128)
    inside, s = _dofs(w)
    r, n = w.ls_params[0], int(w.ls_params[1])
    ins_or = np.zeros_like(inside)
    pts, nrm = [], []
    for k in range(n):
        cx, cy = w.ls_params[2 + 2 * k: 4 + 2 * k]
        wk = W.Workload("disc", 2, w.n, w.lo, w.hi, W.LS_ELLIPSE, [cx, cy, r, r, 0.0],
                        W.KIND_INTERFACE_MU)
        ik, sk = _dofs(wk)
        ins_or |= ik
        pts.append(sk.x)
        nrm.append(sk.n)
    assert np.array_equal(inside, ins_or)
    P, Nn = np.concatenate(pts), np.concatenate(nrm)
    assert P.shape == s.x.shape
    key = lambda X: np.lexsort(np.round(X, 9).T[::-1])
    a, b = key(s.x), key(P)
    assert np.abs(s.x[a] - P[b]).max() < 1e-12
    assert np.abs(s.n[a] - Nn[b]).max() < 1e-12


def test_four_discs_converge():
    errs = []
    for n in (128, 256):
        w = W.discs_interface_2d(n)
        P = K.Problem(w)
        d = W.grid_data(w)
        g1, g2 = W.boundary_data(w, P.surf.x, P.surf.n)
        u, x, it, rel = P.solve(g1, g2, d)
        e = np.abs(u - W.exact_grid(w, P.inside))
        m = np.zeros_like(P.inside)
        m[1:-1, 1:-1] = True
        errs.append((e[m & P.inside].max(), e[m & ~P.inside].max()))
        assert it <= 30
    for side in (0, 1):
        assert errs[0][side] / errs[1][side] > 12.0 and errs[1][side] < 1e-8, errs
