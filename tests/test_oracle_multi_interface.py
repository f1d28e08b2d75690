"""Pins of several disjoint interfaces (the union-of-discs level set; the
separated case of Sec. 7.1.2's multiple interfaces, without multiply crossed
grid edges).

PM1 the geometry of the union is the union of the geometries: node classes
    are the OR of the single-disc classes, and the DOFs (family, grid line,
    position, normal) are those of the discs set up one at a time with the
    ellipse level set (a = b = r), a different formula for the same circle.
PM2 the interface problem on four discs converges at 4th order (> 12x from
    N = 128 to 256) on both sides.
Close and touching interfaces: test_oracle_close_interfaces.py.
"""
import numpy as np
import workloads as W
from oracle import geometry as G
from oracle import kfbi as K


def _dofs(w):
    grid = G.Grid(w.dim, w.n, w.lo, w.h)
    lab = G.label_nodes(grid, w.ls_kind, w.ls_params)
    s = G.surface_points(grid, w.ls_kind, w.ls_params, w.cosa(), lab)
    return lab > 0, s


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


def _union_vs_singles(w, single):
    inside, s = _dofs(w)
    d = w.dim
    r, n = w.ls_params[0], int(w.ls_params[1])
    ins_or = np.zeros_like(inside)
    pts, nrm = [], []
    for k in range(n):
        c = list(w.ls_params[2 + d * k: 2 + d * (k + 1)])
        wk = W.Workload("ball", d, w.n, w.lo, w.hi, single, single_params(c, r),
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


def single_params(c, r):
    return [c[0], c[1], r, r, 0.0] if len(c) == 2 else [c[0], c[1], c[2], r, r, r]


def test_random_separated_discs_and_spheres():
    """PM1 on seeded random layouts: 2D (3 or 4 discs) and 3D (2 spheres),
    every pair at least 6 h apart."""
    rng = np.random.default_rng(5968)
    for d, n, trials in ((2, 128, 3), (3, 32, 1)):
        h = 2.0 / n
        for _ in range(trials):
            r = rng.uniform(0.15, 0.25) if d == 2 else rng.uniform(0.2, 0.25)
            m = int(rng.integers(3, 5)) if d == 2 else 2
            cs = []
            for _attempt in range(10000):
                c = rng.uniform(-0.95 + r + 4 * h, 0.95 - r - 4 * h, size=d)
                if all(np.linalg.norm(c - q) > 2 * r + 6 * h for q in cs):
                    cs.append(c)
                if len(cs) == m:
                    break
            assert len(cs) == m
            kind = W.LS_DISCS if d == 2 else W.LS_SPHERES
            params = [r, float(m)] + [float(v) for c in cs for v in c]
            w = W.Workload("balls", d, n, -1.0, 1.0, kind, params, W.KIND_INTERFACE_MU)
            _union_vs_singles(w, W.LS_ELLIPSE if d == 2 else W.LS_ELLIPSOID)
