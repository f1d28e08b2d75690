"""Pins of the oracle's BIE operators, GMRES and end-to-end solves
(Sec. 3, 4, 6, 7; Algorithm 1).

P3 Gauss's lemma: for the interior Dirichlet operator with kappa = 0, A 1 = 1.
P4 linearity, and mu = 0 gives A = I/2 exactly.  (Exact mirror symmetry is
   not expected: the tie rules favour lower indices.)
P5 brute force: dense assembly + numpy.linalg.solve agrees with GMRES.
P6 convergence of configs 1 and 2 under refinement (>= 3.5).
P7 the paper's printed Table 1 (Sec. 7.1.1): N_b, iterations and errors.
"""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import kfbi as K

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_table1.json")


def _solve(w, rtol=1e-10):
    P = K.Problem(w)
    d = W.grid_data(w)
    g1, g2 = W.boundary_data(w, P.surf.x, P.surf.n)
    u, x, it, rel = P.solve(g1, g2, d, rtol=rtol)
    return P, u, x, it


def _errs(w, P, u):
    ex = W.exact_grid(w, P.inside)
    if w.kind == W.KIND_DIRICHLET:
        return K.errors(u, ex, P.inside)[0]
    mask = np.zeros_like(P.inside)
    mask[tuple(slice(1, w.n) for _ in range(w.dim))] = True
    return K.errors(u, ex, mask)[0]


def test_gauss_lemma_operator():
    for w in (W.ellipse_dirichlet_2d(64), W.paper_table1_2d(64)):
        P = K.Problem(w)
        assert np.abs(P.apply(np.ones(P.nb)) - 1.0).max() < 1e-12


def test_linearity_and_mu_zero():
    P = K.Problem(W.flower_interface_2d(256))
    rng = np.random.default_rng(0)
    x, y = rng.standard_normal(P.nb), rng.standard_normal(P.nb)
    lhs = P.apply(2.0 * x - 3.0 * y)
    rhs = 2.0 * P.apply(x) - 3.0 * P.apply(y)
    assert np.abs(lhs - rhs).max() < 1e-10 * np.abs(rhs).max()
    w = W.flower_interface_2d(256, contrast=1.0)
    P1 = K.Problem(w)
    assert np.abs(P1.apply(x) - 0.5 * x).max() == 0.0


def test_gmres_matches_dense_solve():
    w = W.ellipse_dirichlet_2d(48)
    P = K.Problem(w)
    A = np.array([P.apply(e) for e in np.eye(P.nb)]).T
    d = W.grid_data(w)
    g1, g2 = W.boundary_data(w, P.surf.x, P.surf.n)
    b = P.bie_rhs(g1, g2, d)
    x_dense = np.linalg.solve(A, b)
    x_g, it, rel = K.gmres(P.apply, b, rtol=1e-14)
    assert np.abs(x_g - x_dense).max() < 1e-11 * np.abs(x_dense).max()
    # restarted GMRES reaches the same solution
    x_r, it_r, _ = K.gmres(P.apply, b, rtol=1e-13, restart=5, max_iter=400)
    assert np.abs(x_r - x_dense).max() < 1e-10 * np.abs(x_dense).max()
    # the spectrum of the second-kind operator is bounded away from 0
    ev = np.linalg.eigvals(A)
    assert np.abs(ev).min() > 0.1 and np.abs(ev).max() < 1.5


def test_convergence_config1():
    errs = []
    its = []
    for n in (64, 128, 256):
        w = W.ellipse_dirichlet_2d(n)
        P, u, x, it = _solve(w, rtol=1e-12)
        errs.append(_errs(w, P, u))
        its.append(it)
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders.min() > 3.5, (errs, orders)
    assert max(its) <= 14


def test_convergence_config2_low_contrast():
    errs = []
    for n in (128, 256, 512):
        w = W.flower_interface_2d(n, contrast=10.0)
        P, u, x, it = _solve(w, rtol=1e-12)
        errs.append(_errs(w, P, u))
        assert it <= 30
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders.min() > 3.2 and orders.mean() > 3.8, (errs, orders)


def test_config2_high_contrast_accuracy():
    w = W.flower_interface_2d(256)
    P, u, x, it = _solve(w)
    assert _errs(w, P, u) < 2e-8
    assert P.nb == 442 and it <= 30


def test_paper_table1_loose_pin():
    """P7: Sec. 7.1.1 Table 1 — N_b within 3 points, iterations within 2 and
    the maximum error within 3x of the printed values."""
    rows = json.load(open(GOLDEN))["rows"]
    for row in rows[:3]:
        w = W.paper_table1_2d(row["N"])
        P, u, x, it = _solve(w)
        assert abs(P.nb - row["Nb"]) <= 3
        assert abs(it - row["iterations"]) <= 2
        e = _errs(w, P, u)
        assert e < 3.0 * row["einf"], (row, e)


def test_3d_dirichlet_small():
    """3D path: Gauss's lemma (kappa = 0) and a modified-Helmholtz solve on a
    resolved ellipsoid with the error of a 4th-order method at this size."""
    w = W.Workload("ell3", 3, 32, -1.0, 1.0, W.LS_ELLIPSOID, [0.05, -0.03, 0.02, 0.8, 0.7, 0.6],
                   W.KIND_DIRICHLET, kappa=0.0, exact="exp3")
    P = K.Problem(w)
    assert np.abs(P.apply(np.ones(P.nb)) - 1.0).max() < 1e-12
    w.kappa = 1.0
    P, u, x, it = _solve(w)
    assert it <= 20
    assert _errs(w, P, u) < 1e-4
