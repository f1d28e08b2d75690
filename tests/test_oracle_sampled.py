"""Pins of the oracle's grid-sampled level set (interfaces known only by the
values of a level-set function at the grid nodes; cubic Lagrange
interpolation between nodes)."""
import numpy as np

import workloads as W
from oracle import geometry as G
from oracle import kfbi as K
from oracle import levelset as LS


def test_interpolant_is_exact_for_cubics_per_axis():
    """Values and gradients of any polynomial of degree <= 3 in each
    variable are reproduced to rounding, at nodes (exactly) and between them,
    near the box faces as well."""
    rng = np.random.default_rng(1)
    for d, n in ((2, 24), (3, 12)):
        lo, h = -1.0, 2.0 / n
        C = rng.standard_normal((4,) * d)

        def poly(X):
            v = np.zeros(X.shape[:-1])
            gr = np.zeros(X.shape)
            for idx in np.ndindex(*C.shape):
                term = C[idx] * np.prod([X[..., k] ** idx[k] for k in range(d)], axis=0)
                v = v + term
                for k in range(d):
                    if idx[k]:
                        dk = C[idx] * idx[k] * np.prod(
                            [X[..., m] ** (idx[m] - (m == k)) for m in range(d)], axis=0)
                        gr[..., k] = gr[..., k] + dk
            return v, gr
        g = G.Grid(d, n, lo, h)
        S = LS.Sampled(poly(g.coords())[0], lo, h)
        X = rng.uniform(-1.0, 1.0, size=(300, d))
        v, gr = poly(X)
        assert np.abs(LS.H(W.LS_GRID, S, X) - v).max() < 1e-11
        assert np.abs(LS.grad_H(W.LS_GRID, S, X) - gr).max() < 1e-9
        nodes = g.coords().reshape(-1, d)
        assert np.array_equal(LS.H(W.LS_GRID, S, nodes), S.samples.reshape(-1))


def test_sampled_quadrics_give_the_analytic_geometry():
    """Samples of the ellipse / ellipsoid level sets (quadratic, so the
    interpolant is exact): the node classes, DOF families, points and normals
    of the analytic kinds, 2D and 3D."""
    for w in (W.ellipse_dirichlet_2d(128),
              W.Workload("e3", 3, 32, -1.0, 1.0, W.LS_ELLIPSOID, [0.05, -0.03, 0.02, 0.8, 0.7, 0.6],
                         W.KIND_DIRICHLET, kappa=1.0, exact="exp3")):
        g = G.Grid(w.dim, w.n, w.lo, w.h)
        S = LS.Sampled(LS.H(w.ls_kind, w.ls_params, g.coords()), w.lo, w.h)
        ia = G.classify(g, w.ls_kind, w.ls_params)
        isamp = G.classify(g, W.LS_GRID, S)
        assert np.array_equal(ia, isamp)
        sa = G.surface_points(g, w.ls_kind, w.ls_params, w.cosa(), ia)
        ss = G.surface_points(g, W.LS_GRID, S, w.cosa(), isamp)
        assert sa.nb == ss.nb and np.array_equal(sa.family, ss.family)
        assert np.array_equal(sa.line, ss.line) and np.array_equal(sa.edge, ss.edge)
        assert np.abs(sa.x - ss.x).max() < 1e-13
        assert np.abs(sa.n - ss.n).max() < 1e-12


def test_sampled_interface_problem_converges_at_fourth_order():
    """The 2D interface problem on a shape known only by its samples: the
    error against the exact solution falls at order >= 3.5 from N = 64 to 256
    (the interpolated interface is O(h^4) from the sampled function's zero set)."""
    errs = []
    for n in (64, 128, 256):
        w = W.sampled_interface_2d(n)
        P = K.Problem(w)
        data = W.grid_data(w)
        g1, g2 = W.boundary_data(w, P.surf.x, P.surf.n)
        u, _, _, _ = P.solve(g1, g2, data, rtol=1e-12)
        # the interface of the sampled problem is the interpolant's zero set,
        # the exact solution's sides are decided by the same node classes
        ex = W.exact_grid(w, P.inside)
        errs.append(np.abs(u - ex)[1:-1, 1:-1].max())
    orders = [np.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert min(orders) >= 3.5, (errs, orders)
