"""Compact finite-difference schemes on the box and their fast solve — oracle.

The 9-point (2D) and 27-point (3D) fourth-order compact schemes of eqs.
(9p-cds)/(27p-cds) for Lap u - kappa u = f, and the standard 5/7-point
second-order scheme, written in the general form of eq. (FDS-gene):
    sum_{offsets o in {-1,0,1}^d} c_o u_{P+o} = F_P.
Coefficients depend only on the number of nonzero components of o.

The box solve (Algorithm 1, Step 3.3) is the exact solution of the scheme with
homogeneous Dirichlet data by the sine transform: sin(p pi i / N) products are
eigenvectors of every operator above, with eigenvalue
    lambda = sum_o c_o prod_k cos(p_k pi o_k / N)      (closed form below).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.fft
import scipy.sparse
import scipy.sparse.linalg


def stencil_coeffs(d: int, order: int, h: float, kappa: float):
    """c indexed by the number of nonzero offset components (0..d)."""
    ih2 = 1.0 / (h * h)
    if order == 2:
        c = [-2.0 * d * ih2 - kappa, ih2] + [0.0] * (d - 1)
        return np.array(c)
    if d == 2:   # eq. (9p-cds)
        return np.array([-10.0 / 3.0 * ih2 - 2.0 / 3.0 * kappa,
                         2.0 / 3.0 * ih2 - kappa / 12.0,
                         1.0 / 6.0 * ih2])
    # eq. (27p-cds)
    return np.array([-25.0 / 6.0 * ih2 - 0.5 * kappa,
                     5.0 / 12.0 * ih2 - kappa / 12.0,
                     1.0 / 8.0 * ih2,
                     1.0 / 48.0 * ih2])


def offsets(d: int):
    return [o for o in itertools.product((-1, 0, 1), repeat=d)]


def coeff_of(c, o):
    return c[sum(1 for v in o if v != 0)]


def apply_operator(u: np.ndarray, d: int, order: int, h: float, kappa: float) -> np.ndarray:
    """A_h u at interior nodes (boundary layer of the result is 0)."""
    c = stencil_coeffs(d, order, h, kappa)
    n = u.shape[0] - 1
    out = np.zeros_like(u)
    inner = tuple(slice(1, n) for _ in range(d))
    for o in offsets(d):
        w = coeff_of(c, o)
        if w == 0.0:
            continue
        sl = tuple(slice(1 + ok, n + ok) for ok in o)
        out[inner] += w * u[sl]
    return out


def eigenvalues(d: int, order: int, n: int, h: float, kappa: float) -> np.ndarray:
    """Closed-form eigenvalues on the (N-1)^d sine modes, written with
    s_k = sin^2(k pi / 2N) (cos(k pi/N) = 1 - 2 s_k) so that the low modes carry
    no cancellation:
      9-point:  h^-2 [-4 (s_p + s_q) + 8/3 s_p s_q] - kappa [1 - (s_p + s_q)/3]
      27-point: h^-2 [-4 S1 + 8/3 S2 - 4/3 S3]      - kappa [1 - S1/3]
      5/7-point: h^-2 (-4 S1) - kappa
    (S1, S2, S3 the elementary symmetric sums of the s_k).  Expanding c = 1 - 2s
    in h^-2[-10/3 + 4/3 (c_p + c_q) + 2/3 c_p c_q] - kappa[2/3 + (c_p + c_q)/6]
    (and the 27-point analogue from eq. (27p-cds)) gives these forms."""
    sk = np.sin(np.arange(1, n) * np.pi / (2 * n)) ** 2
    S = np.meshgrid(*([sk] * d), indexing="ij")
    ih2 = 1.0 / (h * h)
    s1 = sum(S)
    if order == 2:
        return ih2 * (-4.0 * s1) - kappa
    if d == 2:
        sp, sq = S
        return ih2 * (-4.0 * s1 + 8.0 / 3.0 * sp * sq) - kappa * (1.0 - s1 / 3.0)
    sx, sy, sz = S
    s2 = sx * sy + sy * sz + sz * sx
    s3 = sx * sy * sz
    return ih2 * (-4.0 * s1 + 8.0 / 3.0 * s2 - 4.0 / 3.0 * s3) - kappa * (1.0 - s1 / 3.0)


def dst_solve(rhs: np.ndarray, d: int, order: int, h: float, kappa: float) -> np.ndarray:
    """u = A_h^{-1} rhs on the interior (zero boundary layer), by DST-I."""
    n = rhs.shape[0] - 1
    inner = tuple(slice(1, n) for _ in range(d))
    lam = eigenvalues(d, order, n, h, kappa)
    coef = scipy.fft.dstn(rhs[inner], type=1) / lam
    u = np.zeros_like(rhs)
    u[inner] = scipy.fft.idstn(coef, type=1)
    return u


def sparse_matrix(d: int, order: int, n: int, h: float, kappa: float):
    """A_h on the (N-1)^d interior unknowns as a sparse matrix (for pins)."""
    c = stencil_coeffs(d, order, h, kappa)
    m = n - 1
    shape = (m,) * d
    idx = np.arange(m ** d).reshape(shape)
    rows, cols, vals = [], [], []
    for o in offsets(d):
        w = coeff_of(c, o)
        if w == 0.0:
            continue
        src = tuple(slice(max(0, -ok), m - max(0, ok)) for ok in o)
        dst = tuple(slice(max(0, ok), m - max(0, -ok)) for ok in o)
        rows.append(idx[src].ravel())
        cols.append(idx[dst].ravel())
        vals.append(np.full(idx[src].size, w))
    A = scipy.sparse.csr_matrix((np.concatenate(vals), (np.concatenate(rows),
                                                         np.concatenate(cols))),
                                shape=(m ** d, m ** d))
    return A


def direct_solve(rhs: np.ndarray, d: int, order: int, h: float, kappa: float) -> np.ndarray:
    """Same solve by a sparse direct factorisation (pin for ``dst_solve``)."""
    n = rhs.shape[0] - 1
    inner = tuple(slice(1, n) for _ in range(d))
    A = sparse_matrix(d, order, n, h, kappa)
    u = np.zeros_like(rhs)
    u[inner] = scipy.sparse.linalg.spsolve(A.tocsc(), rhs[inner].ravel()).reshape((n - 1,) * d)
    return u


def boundary_lift(gb: np.ndarray, d: int, order: int, h: float, kappa: float) -> np.ndarray:
    """sum over box-boundary neighbours Q of c_{Q-P} g_B(Q), at interior P:
    moving nonhomogeneous outer Dirichlet data to the right-hand side."""
    gb_only = gb.copy()
    n = gb.shape[0] - 1
    inner = tuple(slice(1, n) for _ in range(d))
    gb_only[inner] = 0.0
    return apply_operator(gb_only, d, order, h, kappa)
