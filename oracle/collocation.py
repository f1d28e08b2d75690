"""Mesh-free collocation for the local Cauchy problem (Sec. 5.3, 5.3.1) — oracle.

On each partition Omega_{Gamma,i} centred at the primary point p_i, the local
correction function is a Taylor polynomial of degree <= p in the scaled local
coordinates xi = (x - p_i)/h:

    C_{h,i}(x) = sum_{|e| <= p} d_e phi_e(xi),   phi_e(xi) = prod_k xi_k^{e_k}.

The collocation equations (eq. (cau-appro)) are multiplied through so that all
rows are O(1) in xi (the scaling remark at the end of Sec. 5.4):
    PDE row       (Lap_xi - kappa h^2) phi_e(xi_j)      = h^2 f~(x_j)
    Dirichlet row  phi_e(xi_j)                           = a(x_j)
    Neumann row    n(x_j) . grad_xi phi_e(xi_j)          = h b(x_j)
which scales rows only, so the square system M U = Q (eq. (cau-ls)) has the
same solution.  It is solved by Householder QR (Sec. 5.4).
Basis order: graded lexicographic — total degree ascending, then the exponent
of x descending, then of y descending (so phi_0 = 1, phi_1..phi_d = xi_1..xi_d).
"""
from __future__ import annotations

import numpy as np


def exponents(d: int, p: int):
    out = []
    for t in range(p + 1):
        if d == 2:
            for l in range(t, -1, -1):
                out.append((l, t - l))
        else:
            for l in range(t, -1, -1):
                for m in range(t - l, -1, -1):
                    out.append((l, m, t - l - m))
    return np.array(out, dtype=np.int64)


def _pow(x, e):
    return np.where(e == 0, 1.0, x ** np.maximum(e, 0))


def phi(E: np.ndarray, xi: np.ndarray) -> np.ndarray:
    """Monomials phi_e(xi): xi (..., d) -> (..., n_dof)."""
    out = np.ones(xi.shape[:-1] + (E.shape[0],))
    for k in range(E.shape[1]):
        out = out * _pow(xi[..., k:k + 1], E[:, k])
    return out


def grad_phi(E: np.ndarray, xi: np.ndarray) -> np.ndarray:
    """d phi_e / d xi_k: (..., d, n_dof)."""
    d = E.shape[1]
    gs = []
    for k in range(d):
        g = np.ones(xi.shape[:-1] + (E.shape[0],))
        for j in range(d):
            if j == k:
                g = g * E[:, j] * _pow(xi[..., j:j + 1], E[:, j] - 1)
            else:
                g = g * _pow(xi[..., j:j + 1], E[:, j])
        gs.append(g)
    return np.stack(gs, -2)


def lap_phi(E: np.ndarray, xi: np.ndarray) -> np.ndarray:
    """Lap_xi phi_e: (..., n_dof)."""
    d = E.shape[1]
    tot = np.zeros(xi.shape[:-1] + (E.shape[0],))
    for k in range(d):
        g = np.ones(xi.shape[:-1] + (E.shape[0],))
        for j in range(d):
            if j == k:
                g = g * E[:, j] * (E[:, j] - 1) * _pow(xi[..., j:j + 1], E[:, j] - 2)
            else:
                g = g * _pow(xi[..., j:j + 1], E[:, j])
        tot = tot + g
    return tot


def collocation_matrix(E, p_i, h, kappa, pde_x, dir_x, neu_x, neu_n):
    """M of eq. (cau-ls) for one primary point: rows PDE, Dirichlet, Neumann."""
    xi_p = (pde_x - p_i) / h
    xi_d = (dir_x - p_i) / h
    xi_n = (neu_x - p_i) / h
    rows_p = lap_phi(E, xi_p) - kappa * h * h * phi(E, xi_p)
    rows_d = phi(E, xi_d)
    g = grad_phi(E, xi_n)                    # (k, d, n_dof)
    rows_n = np.einsum("kd,kde->ke", neu_n, g)
    return np.concatenate([rows_p, rows_d, rows_n], 0)


def collocation_rhs(h, ftilde_pde, a_dir, b_neu):
    """Q of eq. (cau-ls): [h^2 f~ ; a ; h b]."""
    return np.concatenate([h * h * np.asarray(ftilde_pde), np.asarray(a_dir),
                           h * np.asarray(b_neu)], -1)


def qr_factor(M: np.ndarray):
    """Householder QR of a stack of square collocation matrices."""
    return np.linalg.qr(M)


def qr_solve(Qf: np.ndarray, Rf: np.ndarray, rhs: np.ndarray) -> np.ndarray:
    """Solve R d = Q^T rhs by back substitution (stacked)."""
    y = np.einsum("...ji,...j->...i", Qf, rhs)
    n = Rf.shape[-1]
    d = np.zeros_like(y)
    for i in range(n - 1, -1, -1):
        acc = y[..., i] - np.einsum("...j,...j->...", Rf[..., i, i + 1:], d[..., i + 1:])
        d[..., i] = acc / Rf[..., i, i]
    return d


def eval_poly(E, coef, p_i, h, x):
    """C_{h,i}(x) = sum_e d_e phi_e((x - p_i)/h)."""
    return np.sum(coef * phi(E, (x - p_i) / h), -1)
