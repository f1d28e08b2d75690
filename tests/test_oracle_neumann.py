"""Pins of the oracle's interior Neumann BVP, eq. (bie-N) with the mean-zero
projection of Sec. 7.2.1.

PN1 convergence of the 2D Neumann problem (Poisson, projected; modified
    Helmholtz, not projected) on the rotated ellipse of Sec. 7.1.1: from N = 64
    to N = 512 the maximum error (after removing its mean over Omega, the
    solution being fixed up to a constant for kappa = 0) falls by more than
    500x, i.e. faster than third order on average.  A wrong sign of psi/2, a
    doubled average or a wrong sign of the right-hand side leaves an O(1)
    error.
PN2 the second-order scheme converges (>= 4x over two refinements).
PN3 the projection: for kappa = 0 the right-hand side and every operator
    application have zero mean (the paper's definition); for kappa > 0 they
    are not projected.
PN4 3D solves on a resolved ellipsoid (Poisson, projected; modified
    Helmholtz, not projected) reach the error of a 4th-order method at N = 32.
"""
import numpy as np

import workloads as W
from oracle import kfbi as K


def _solve(w, rtol=1e-10):
    P = K.Problem(w)
    d = W.grid_data(w)
    g1, g2 = W.boundary_data(w, P.surf.x, P.surf.n)
    u, x, it, rel = P.solve(g1, g2, d, rtol=rtol)
    e = (u - W.exact_grid(w, P.inside))[P.inside]
    return P, float(np.abs(e - e.mean()).max()), it


def test_neumann_convergence_2d():
    for kappa, bound in ((0.0, 1e-6), (1.0, 2e-6)):
        _, e64, it64 = _solve(W.neumann_ellipse_2d(64, kappa))
        _, e512, it512 = _solve(W.neumann_ellipse_2d(512, kappa))
        assert e512 < bound, (kappa, e512)
        assert e64 / e512 > 500.0, (kappa, e64, e512)
        assert it64 <= 20 and it512 <= 20


def test_neumann_second_order():
    w = W.neumann_ellipse_2d(64)
    w.order = 2
    _, e64, _ = _solve(w)
    w = W.neumann_ellipse_2d(256)
    w.order = 2
    _, e256, _ = _solve(w)
    assert e256 < 1e-3 and e64 / e256 > 4.0, (e64, e256)


def test_neumann_projection():
    rng = np.random.default_rng(7)
    for kappa in (0.0, 1.0):
        w = W.neumann_ellipse_2d(64, kappa)
        P = K.Problem(w)
        d = W.grid_data(w)
        g1, g2 = W.boundary_data(w, P.surf.x, P.surf.n)
        b = P.bie_rhs(g1, g2, d)
        ys = [P.apply(rng.standard_normal(P.nb)) for _ in range(3)]
        for y in [b] + ys:
            m = abs(float(np.mean(y))) / float(np.abs(y).max())
            if kappa == 0.0:
                assert m < 1e-14, m
        if kappa > 0.0:
            assert max(abs(float(np.mean(y))) / float(np.abs(y).max()) for y in ys) > 1e-6


def test_neumann_3d_small():
    for kappa in (0.0, 1.0):
        w = W.Workload("ell3n", 3, 32, -1.0, 1.0, W.LS_ELLIPSOID,
                       [0.05, -0.03, 0.02, 0.8, 0.7, 0.6], W.KIND_NEUMANN, kappa=kappa,
                       exact="exp3")
        P, e, it = _solve(w)
        assert e < 1e-3 and it <= 30, (kappa, e, it)
