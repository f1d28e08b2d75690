"""Pins of the oracle's compact schemes and box solve (Sec. 5.2, Algorithm 1 Step 3.3).

P1: (a) A_h applied stencil-by-stencil to a discrete sine mode equals the
closed-form eigenvalue times the mode; (b) the DST-I solve equals a sparse
direct solve; (c) the schemes converge at their stated order for a smooth
manufactured solution; (d) row sums vanish for kappa = 0 (constants in the
kernel of the interior stencil).
"""
import itertools

import numpy as np
import pytest

from oracle import boxsolve as BS


@pytest.mark.parametrize("d,order,kappa", [(2, 4, 0.0), (2, 4, 3.0), (2, 2, 1.0),
                                           (3, 4, 0.0), (3, 4, 2.0), (3, 2, 0.5)])
def test_sine_modes_are_eigenvectors(d, order, kappa):
    n = 12 if d == 2 else 8
    h = 2.0 / n
    lam = BS.eigenvalues(d, order, n, h, kappa)
    rng = np.random.default_rng(1)
    for _ in range(3):
        p = rng.integers(1, n, size=d)
        i = np.arange(n + 1)
        mode = np.ones((n + 1,) * d)
        for ax in range(d):
            shape = [1] * d
            shape[ax] = n + 1
            mode = mode * np.sin(p[ax] * np.pi * i / n).reshape(shape)
        Au = BS.apply_operator(mode, d, order, h, kappa)
        inner = tuple(slice(1, n) for _ in range(d))
        expect = lam[tuple(p - 1)] * mode[inner]
        assert np.abs(Au[inner] - expect).max() < 1e-10 * np.abs(lam).max()


@pytest.mark.parametrize("d,order,kappa,n", [(2, 4, 0.0, 16), (2, 4, 5.0, 32), (2, 2, 0.0, 20),
                                             (3, 4, 1.0, 12), (3, 2, 0.0, 10)])
def test_dst_equals_sparse_direct(d, order, kappa, n):
    rng = np.random.default_rng(7)
    r = np.zeros((n + 1,) * d)
    r[tuple(slice(1, n) for _ in range(d))] = rng.standard_normal((n - 1,) * d)
    h = 2.0 / n
    u1 = BS.dst_solve(r, d, order, h, kappa)
    u2 = BS.direct_solve(r, d, order, h, kappa)
    assert np.abs(u1 - u2).max() < 1e-12 * np.abs(u2).max()


def _manufactured(d, n, kappa):
    """u = prod sin(pi (x_k + 1)/2) on [-1, 1]^d: zero on the box boundary."""
    h = 2.0 / n
    x = -1.0 + np.arange(n + 1) * h
    X = np.meshgrid(*([x] * d), indexing="ij")
    s = [np.sin(np.pi * (xk + 1) / 2) for xk in X]
    u = np.prod(s, axis=0)
    lam = -(np.pi / 2) ** 2 * d
    f = (lam - kappa) * u              # Lap u - kappa u
    lapf = lam * f
    return u, f, lapf, h


@pytest.mark.parametrize("d,order,kappa,ns,rate", [(2, 4, 0.0, (16, 32, 64), 3.8),
                                                   (2, 4, 4.0, (16, 32, 64), 3.8),
                                                   (2, 2, 1.0, (16, 32, 64), 1.9),
                                                   (3, 4, 1.0, (8, 16, 32), 3.7)])
def test_convergence_order(d, order, kappa, ns, rate):
    errs = []
    for n in ns:
        u, f, lapf, h = _manufactured(d, n, kappa)
        rhs = f + (h * h / 12.0) * lapf if order == 4 else f
        inner = tuple(slice(1, n) for _ in range(d))
        r = np.zeros_like(u)
        r[inner] = rhs[inner]
        uh = BS.dst_solve(r, d, order, h, kappa)
        errs.append(np.abs(uh - u).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders.min() > rate, (errs, orders)


@pytest.mark.parametrize("d", [2, 3])
def test_row_sums_vanish(d):
    for order in (2, 4):
        c = BS.stencil_coeffs(d, order, 0.1, 0.0)
        tot = sum(BS.coeff_of(c, o) for o in itertools.product((-1, 0, 1), repeat=d))
        assert abs(tot) < 1e-9
        # the kappa part of the compact scheme sums to kappa
        ck = BS.stencil_coeffs(d, order, 1e30, 1.0)
        totk = sum(BS.coeff_of(ck, o) for o in itertools.product((-1, 0, 1), repeat=d))
        assert abs(totk + 1.0) < 1e-12


def test_boundary_lift_moves_dirichlet_data():
    """Solving with outer data g_B equals solving the homogeneous problem for u - E g_B."""
    d, order, n, kappa = 2, 4, 16, 0.7
    h = 2.0 / n
    x = -1.0 + np.arange(n + 1) * h
    X, Y = np.meshgrid(x, x, indexing="ij")
    gb = np.cos(X) * np.exp(Y)          # data on the boundary layer
    inner = (slice(1, n), slice(1, n))
    A = BS.sparse_matrix(d, order, n, h, kappa)
    rng = np.random.default_rng(3)
    f = np.zeros((n + 1, n + 1))
    f[inner] = rng.standard_normal((n - 1, n - 1))
    r = f - BS.boundary_lift(gb, d, order, h, kappa)
    u = BS.dst_solve(r, d, order, h, kappa)
    u[0, :], u[-1, :], u[:, 0], u[:, -1] = gb[0, :], gb[-1, :], gb[:, 0], gb[:, -1]
    # full operator (including boundary neighbours) reproduces f at interior nodes
    Au = BS.apply_operator(u, d, order, h, kappa)
    assert np.abs(Au[inner] - f[inner]).max() < 1e-9
    assert A.shape[0] == (n - 1) ** 2
