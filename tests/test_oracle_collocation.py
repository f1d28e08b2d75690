"""Pins of the collocation step (Sec. 5.3.1, 5.4).

P2: when a, b and f~ come from a polynomial of degree <= p, the collocation
solution reproduces that polynomial exactly (to roundoff), for every primary
point, in 2D and 3D, p = 2 and 4, kappa = 0 and kappa > 0.  The monomial
derivatives are pinned against symbolic differentiation, and the square-system
counts against the formula of Sec. 5.4.
"""
import numpy as np
import pytest
import sympy

import workloads as W
from oracle import collocation as CO
from oracle import geometry as G
from oracle import kfbi as K


def test_counts_square_system():
    # Sec. 5.4: PDE sum_{i<=p-2} (i+1)(i+2)/2, Dirichlet (p+1)(p+2)/2, Neumann p(p+1)/2 in 3D
    for p in (2, 4):
        n_pde = sum((i + 1) * (i + 2) // 2 for i in range(p - 1))
        nd, nn = G.n_boundary_points(3, p)
        assert (len(G.pde_offsets(3, p)), nd, nn) == (n_pde, (p + 1) * (p + 2) // 2, p * (p + 1) // 2)
        assert n_pde + nd + nn == CO.exponents(3, p).shape[0]
        nd2, nn2 = G.n_boundary_points(2, p)
        assert len(G.pde_offsets(2, p)) + nd2 + nn2 == CO.exponents(2, p).shape[0]
    assert CO.exponents(2, 4).shape[0] == 15 and CO.exponents(3, 4).shape[0] == 35


@pytest.mark.parametrize("d", [2, 3])
def test_monomial_derivatives_match_sympy(d):
    E = CO.exponents(d, 4)
    syms = sympy.symbols("x0:%d" % d)
    rng = np.random.default_rng(0)
    pt = rng.uniform(-2, 2, size=d)
    sub = {s: v for s, v in zip(syms, pt)}
    ph = CO.phi(E, pt[None])[0]
    gr = CO.grad_phi(E, pt[None])[0]
    lp = CO.lap_phi(E, pt[None])[0]
    for j, e in enumerate(E):
        m = sympy.Integer(1)
        for s, k in zip(syms, e):
            m = m * s ** int(k)
        assert abs(float(m.subs(sub)) - ph[j]) < 1e-12
        for k in range(d):
            assert abs(float(sympy.diff(m, syms[k]).subs(sub)) - gr[k, j]) < 1e-11
        lap = sum(sympy.diff(m, s, 2) for s in syms)
        assert abs(float(sympy.sympify(lap).subs(sub)) - lp[j]) < 1e-10


def _poly_problem(w, seed):
    P = K.Problem(w)
    rng = np.random.default_rng(seed)
    E = CO.exponents(w.dim, w.order)
    c = rng.standard_normal(E.shape[0])

    def val(X):
        return CO.phi(E, X) @ c

    def grad(X):
        return np.einsum("...ke,e->...k", CO.grad_phi(E, X), c)

    def lap(X):
        return CO.lap_phi(E, X) @ c
    return P, val, grad, lap


@pytest.mark.parametrize("mk,order,kappa", [
    (lambda: W.ellipse_dirichlet_2d(48), 4, 0.0),
    (lambda: W.ellipse_dirichlet_2d(48), 4, 2.5),
    (lambda: W.ellipse_dirichlet_2d(48), 2, 0.0),
    (lambda: W.flower_interface_2d(160), 4, 0.0),
])
def test_polynomial_exactness_2d(mk, order, kappa):
    w = mk()
    w.order = order
    w.kind = W.KIND_DIRICHLET
    w.kappa = kappa
    P, val, grad, lap = _poly_problem(w, 11)
    x, n = P.surf.x, P.surf.n
    a = val(x)
    b = np.sum(grad(x) * n, -1)
    X = P.grid.coords()
    ft = lap(X) - kappa * val(X)
    coef = P.collocation(a, b, ft)
    cv = P.c_values(coef)
    xc = P.grid.coord(P.cnode_idx)
    assert np.abs(cv - val(xc)).max() < 1e-10 * max(1.0, np.abs(val(xc)).max())


def test_polynomial_exactness_3d():
    w = W.Workload("ell3", 3, 32, -1.0, 1.0, W.LS_ELLIPSOID, [0.05, -0.03, 0.02, 0.8, 0.7, 0.6],
                   W.KIND_DIRICHLET, kappa=1.5, exact="exp3")
    P, val, grad, lap = _poly_problem(w, 5)
    x, n = P.surf.x, P.surf.n
    X = P.grid.coords()
    coef = P.collocation(val(x), np.sum(grad(x) * n, -1), lap(X) - 1.5 * val(X))
    cv = P.c_values(coef)
    xc = P.grid.coord(P.cnode_idx)
    assert np.abs(cv - val(xc)).max() < 1e-9 * max(1.0, np.abs(val(xc)).max())
    cond = np.linalg.cond(P.M)
    assert np.median(cond) < 1e4


def test_condition_numbers_in_paper_range():
    """Sec. 5.4 remark: cond(M) is O(10^2 - 10^3) independent of h."""
    meds = []
    for n in (64, 128, 256):
        P = K.Problem(W.ellipse_dirichlet_2d(n))
        c = np.linalg.cond(P.M)
        meds.append(np.median(c))
        assert c.max() < 1e4
    assert 30 < min(meds) and max(meds) < 3e3
    assert max(meds) / min(meds) < 3.0
