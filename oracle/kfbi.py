"""KFBI operators, GMRES and final evaluation (Sec. 3, 4, 6; Algorithm 1) — oracle.

Every layer-potential evaluation solves the equivalent simple interface problem
eq. (con-ifp) in unit-sigma form (reading: the box operator is Lap - kappa~ with
kappa~ = kappa/sigma, the form of eq. (bie-ifp-2)):
    Lap u - kappa~ u = F  in B \\ Gamma,  [u] = a,  [d_n u] = b,  u = g_B on dB,
in the four steps of Algorithm 1, Step 3:
  3.1 collocation fit of the local correction functions (``collocation``);
  3.2 corrected right-hand side (``correction``);
  3.3 box solve (``boxsolve.dst_solve``);
  3.4 corrected interpolation of the traces (``traces``).

Problem kinds:
  * interior Dirichlet BVP, eq. (bie-D): unknown phi at the DOFs,
        A phi = phi/2 + K phi,   K phi = avg of D phi (direct value on Gamma),
        b     = g_D - G f,       G f   = avg of N f (continuous across Gamma),
    solution u = D phi + N f (one more potential solve with both data).
    Reading: the boundary integrals are the direct values on Gamma, i.e. the
    averages avg = (trace^+ + trace^-)/2 of the one-sided limits, and the 1/2
    of eq. (bie-D) is applied exactly.  (Using trace^+ alone makes every DOF
    that no collocation stencil uses a near-null mode of the discrete operator.)
  * interface problem, mu-form (kappa_1/sigma_1 = kappa_2/sigma_2): unknown
    psi = [d_n u], mu = (sigma_out - sigma_in)/(sigma_out + sigma_in),
        A psi = psi/2 - mu * avg d_n(v[psi]),   v[psi] = potential with b = psi,
        b     = g2/(sigma_in + sigma_out) + mu * avg d_n(w),
    where w has a = g1, the piecewise f/sigma and the outer data g_B, and
    avg = (d_n^+ + d_n^-)/2.  (K' psi is read as -avg d_n of -S psi.)
  * interior Neumann BVP, eq. (bie-N): unknown psi at the DOFs (unit-sigma
    form, psi = [d_n u] of u = -S psi + N f),
        A psi = psi/2 - K' psi = psi/2 + avg d_n(v[psi]),
        b     = g_N/sigma - d_n G f,   d_n G f = avg d_n of N f,
    solution u = -S psi + N f.  For kappa~ = 0 the operator is singular (its
    adjoint kills constants) and the solution is fixed up to a constant: as in
    Sec. 7.2.1, b and every operator application have their mean subtracted.
    Reading: the mean is the plain arithmetic mean over the N_b DOFs, and the
    projection is applied only when kappa~ = 0.
GMRES (Algorithm 1, Step 4): unrestarted up to `restart` steps, modified
Gram-Schmidt Arnoldi, Givens rotations, stop at ||b - A x|| <= rtol ||b||.
"""
from __future__ import annotations

import numpy as np

import workloads as W

from . import boxsolve as BS
from . import collocation as CO
from . import correction as CR
from . import geometry as G
from . import levelset as LS
from . import traces as TR


class Problem:
    """Set-up of one geometry (all integer decisions) plus the operators."""

    def __init__(self, w: W.Workload, kt: float | None = None):
        self.w = w
        d, n = w.dim, w.n
        self.d, self.n, self.order = d, n, w.order
        self.grid = G.Grid(d, n, w.lo, w.h)
        self.h = w.h
        if kt is not None:
            self.kt = kt
        elif w.kind in (W.KIND_DIRICHLET, W.KIND_NEUMANN):
            self.kt = w.kappa / w.sigma_in
        else:
            self.kt = w.kappa
        self.cos_alpha = w.cosa()
        lsp = LS.params(w)
        self.n_iface = LS.n_interfaces(w.ls_kind, lsp)
        self.labels = G.label_nodes(self.grid, w.ls_kind, lsp)
        self.inside = self.labels > 0
        self.surf = G.surface_points(self.grid, w.ls_kind, lsp,
                                     self.cos_alpha, self.labels)
        s = self.surf
        self.nb = s.nb
        lines = G.LineIndex(self.grid, s)
        self.E = CO.exponents(d, self.order)
        self.ndof = self.E.shape[0]
        pde, dirs, neus, used_axis = [], [], [], []
        for i in range(self.nb):
            pn, di, ne, m = G.collocation_stencil(self.grid, s, lines, i,
                                                  self.order, self.cos_alpha)
            pde.append(pn)
            dirs.append(di)
            neus.append(ne)
            used_axis.append(m)
        self.pde_nodes = np.array(pde)               # (Nb, n_pde, d)
        self.dir_idx = np.array(dirs, dtype=np.int64)
        self.neu_idx = np.array(neus, dtype=np.int64)
        self.stencil_axis = np.array(used_axis, dtype=np.int64)
        Ms = []
        for i in range(self.nb):
            Ms.append(CO.collocation_matrix(
                self.E, s.x[i], self.h, self.kt, self.grid.coord(self.pde_nodes[i]),
                s.x[self.dir_idx[i]], s.x[self.neu_idx[i]], s.n[self.neu_idx[i]]))
        self.M = np.array(Ms)
        self.Qf, self.Rf = CO.qr_factor(self.M)
        self.irr = CR.irregular_nodes(self.labels, self.order)
        # C^(k) is needed by the correction terms (one entry per irregular
        # node and interface k of its stencil) and by the traces.
        self.cnode_idx, self.cnode_iface = CR.correction_entries(self.labels, self.irr,
                                                                 self.order)
        holds = np.zeros((max(self.n_iface, 1),) + self.labels.shape, dtype=bool)
        holds[(self.cnode_iface,) + tuple(self.cnode_idx.T)] = True
        self.trace_st = TR.trace_stencils(self.grid, s.x, s.n, self.labels, self.irr,
                                          self.order, s.iface, holds)
        if any(rec["close"] for rec in self.trace_st):
            self._add_trace_entries()
        self.cnode_owner = np.zeros(self.cnode_idx.shape[0], dtype=np.int64)
        for k in range(self.n_iface):
            on_k = np.nonzero(s.iface == k)[0]
            ent = self.cnode_iface == k
            if ent.any():
                own = CR.closest_primary(s.x[on_k], self.grid.coord(self.cnode_idx[ent]), self.h)
                self.cnode_owner[ent] = on_k[own]

    def _add_trace_entries(self):
        """Close interfaces: the entries (q, k) the trace stencils of points
        near another interface need (C^(t) and C^(l_q) at every node q of
        another label than the side's t), merged with the correction-term
        entries, in node order then k."""
        n1 = self.n + 1
        keys = set()
        lin = lambda q: int(np.ravel_multi_index(tuple(q), (n1,) * self.d))
        for q, k in zip(self.cnode_idx, self.cnode_iface):
            keys.add((lin(q), int(k)))
        for rec in self.trace_st:
            if not rec["close"]:
                continue
            for side in (1, -1):
                nodes, _, _, t = rec[side]
                lq = self.labels[tuple(nodes.T)].astype(np.int64)
                for q, l in zip(nodes, lq):
                    if l == t:
                        continue
                    if t > 0:
                        keys.add((lin(q), t - 1))
                    if l > 0:
                        keys.add((lin(q), int(l) - 1))
        keys = sorted(keys)
        li = np.array([k[0] for k in keys], dtype=np.int64)
        self.cnode_idx = np.stack(np.unravel_index(li, (n1,) * self.d), -1).astype(np.int64)
        self.cnode_iface = np.array([k[1] for k in keys], dtype=np.int64)

    # -- Step 3.1 ----------------------------------------------------------
    def collocation(self, a: np.ndarray, b: np.ndarray, ftilde_grid=None) -> np.ndarray:
        """Coefficients d_i of every local correction function (eq. (cau-ls))."""
        if ftilde_grid is None:
            ft = np.zeros(self.pde_nodes.shape[:2])
        elif ftilde_grid.ndim == self.d + 1:
            # one f~ grid per interface: each DOF takes its own interface's
            nodes = tuple(np.moveaxis(self.pde_nodes, -1, 0))
            ft = ftilde_grid[(self.surf.iface[:, None],) + nodes]
        else:
            ft = ftilde_grid[tuple(np.moveaxis(self.pde_nodes, -1, 0))]
        Q = CO.collocation_rhs(self.h, ft, a[self.dir_idx], b[self.neu_idx])
        return CO.qr_solve(self.Qf, self.Rf, Q)

    def c_values(self, coef: np.ndarray) -> np.ndarray:
        """C_h^(k) at the correction entries (irregular node, interface k)."""
        own = self.cnode_owner
        x = self.grid.coord(self.cnode_idx)
        return CO.eval_poly(self.E, coef[own], self.surf.x[own], self.h, x)

    def c_grid(self, cvals: np.ndarray) -> np.ndarray:
        """cgrids[l] = C^(l) on the grid at its entries, cgrids[0] = 0."""
        g = np.zeros((self.n_iface + 1,) + self.inside.shape)
        g[(self.cnode_iface + 1,) + tuple(self.cnode_idx.T)] = cvals
        return g

    # -- Step 3.2 ----------------------------------------------------------
    def rhs(self, cvals, F_in=None, F_out=None, L_in=None, L_out=None, g_b=None):
        """Right-hand side of eq. (corrected-FDS): F + h^2/12 Lap F (p = 4) from
        the node's own side, plus C_P, minus the outer-boundary lift."""
        shape = self.inside.shape
        R = np.zeros(shape)
        if F_in is not None:
            F = self._own_side(F_in, F_out)
            R = R + F
            if self.order == 4:
                L = self._own_side(L_in, L_out)
                R = R + self.h * self.h / 12.0 * L
        R = R + CR.correction_terms(self.c_grid(cvals), self.labels, self.irr,
                                    self.d, self.order, self.h, self.kt)
        if g_b is not None:
            R = R - BS.boundary_lift(g_b, self.d, self.order, self.h, self.kt)
        inner = tuple(slice(1, self.n) for _ in range(self.d))
        out = np.zeros(shape)
        out[inner] = R[inner]
        return out

    def _own_side(self, G_in, G_out):
        """Each node's own side's grid: G_in (or G_in[k] for label 1 + k, one
        grid per interface) inside, G_out outside."""
        if G_in.ndim == self.d + 1:
            out = G_out.copy()
            for k in range(G_in.shape[0]):
                out = np.where(self.labels == k + 1, G_in[k], out)
            return out
        return np.where(self.inside, G_in, G_out)

    # -- Step 3.3 ----------------------------------------------------------
    def box_solve(self, R, g_b=None):
        u = BS.dst_solve(R, self.d, self.order, self.h, self.kt)
        if g_b is not None:
            bmask = np.ones(u.shape, dtype=bool)
            bmask[tuple(slice(1, self.n) for _ in range(self.d))] = False
            u[bmask] = g_b[bmask]
        return u

    # -- Step 3.4 ----------------------------------------------------------
    def traces(self, u, cvals):
        """(value^+, value^-, d_n^+, d_n^-) at every DOF."""
        return TR.one_sided(self.trace_st, u, self.c_grid(cvals), self.labels)

    # -- one potential: Steps 3.1-3.4 ----------------------------------------
    def potential(self, a, b, F_in=None, F_out=None, L_in=None, L_out=None, g_b=None):
        ft = None
        if F_in is not None:
            ft = F_in - F_out                        # per interface if F_in is
        coef = self.collocation(a, b, ft)
        cv = self.c_values(coef)
        R = self.rhs(cv, F_in, F_out, L_in, L_out, g_b)
        u = self.box_solve(R, g_b)
        return u, cv, coef, R

    # -- BIE operators ---------------------------------------------------------
    def _mu(self):
        w = self.w
        return (w.sigma_out - w.sigma_in) / (w.sigma_out + w.sigma_in)

    def apply(self, x: np.ndarray) -> np.ndarray:
        z = np.zeros(self.nb)
        if self.w.kind == W.KIND_DIRICHLET:
            u, cv, _, _ = self.potential(x, z)
            vp, vm, _, _ = self.traces(u, cv)
            return 0.5 * x + 0.5 * (vp + vm)
        u, cv, _, _ = self.potential(z, x)
        _, _, dp, dm = self.traces(u, cv)
        if self.w.kind == W.KIND_NEUMANN:
            return self.project(0.5 * x + 0.5 * (dp + dm))
        return 0.5 * x - self._mu() * 0.5 * (dp + dm)

    def project(self, y: np.ndarray) -> np.ndarray:
        """Neumann BVP with kappa~ = 0: remove the mean (Sec. 7.2.1)."""
        if self.w.kind == W.KIND_NEUMANN and self.kt == 0.0:
            return y - np.mean(y)
        return y

    def unit_sigma_data(self, data):
        """Physical f on each side divided by sigma (eq. (bie-ifp-2))."""
        w = self.w
        so = w.sigma_in if w.kind in (W.KIND_DIRICHLET, W.KIND_NEUMANN) else w.sigma_out
        return (data["f_in"] / w.sigma_in, data["f_out"] / so,
                data["lapf_in"] / w.sigma_in, data["lapf_out"] / so)

    def bie_rhs(self, g1, g2, data) -> np.ndarray:
        """Right-hand side of the BIE (Algorithm 1, Step 1)."""
        Fi, Fo, Li, Lo = self.unit_sigma_data(data)
        z = np.zeros(self.nb)
        if self.w.kind == W.KIND_DIRICHLET:
            Fo = np.zeros_like(Fo)
            Lo = np.zeros_like(Lo)
            u, cv, _, _ = self.potential(z, z, Fi, Fo, Li, Lo)
            vp, vm, _, _ = self.traces(u, cv)
            return g1 - 0.5 * (vp + vm)
        w = self.w
        if w.kind == W.KIND_NEUMANN:
            u, cv, _, _ = self.potential(z, z, Fi, np.zeros_like(Fo), Li, np.zeros_like(Lo))
            _, _, dp, dm = self.traces(u, cv)
            return self.project(g2 / w.sigma_in - 0.5 * (dp + dm))
        u, cv, _, _ = self.potential(g1, z, Fi, Fo, Li, Lo, data["g_b"])
        _, _, dp, dm = self.traces(u, cv)
        return g2 / (w.sigma_in + w.sigma_out) + self._mu() * 0.5 * (dp + dm)

    def evaluate(self, density, g1, data) -> np.ndarray:
        """Grid solution from the converged density (superposition)."""
        Fi, Fo, Li, Lo = self.unit_sigma_data(data)
        if self.w.kind == W.KIND_DIRICHLET:
            Fo = np.zeros_like(Fo)
            Lo = np.zeros_like(Lo)
            u, _, _, _ = self.potential(density, np.zeros(self.nb), Fi, Fo, Li, Lo)
            return u
        if self.w.kind == W.KIND_NEUMANN:
            z = np.zeros_like(Fo)
            u, _, _, _ = self.potential(np.zeros(self.nb), density, Fi, z, Li, z)
            return u
        u, _, _, _ = self.potential(g1, density, Fi, Fo, Li, Lo, data["g_b"])
        return u

    def solve(self, g1, g2, data, rtol=1e-10, restart=100, max_iter=200, x0=None):
        b = self.bie_rhs(g1, g2, data)
        x, it, rel = gmres(self.apply, b, x0=x0, rtol=rtol, restart=restart,
                           max_iter=max_iter)
        u = self.evaluate(x, g1, data)
        return u, x, it, rel


class InterfaceSystem:
    """General interface problem, eqs. (IFP) and (bie-ifp-1): any sigma_i,
    kappa_i, unknowns phi = u_1 and psi = sigma_2 d_n u_2 at the DOFs
    (x = [phi; psi], 2 N_b entries), Omega_1 the inside of Gamma.

    With G_i the Green's function of sigma_i Lap - kappa_i and the unit-sigma
    potentials of kappa~_i = kappa_i/sigma_i (S_i = S~_i/sigma_i, K_i = K~_i,
    K'_i = K~'_i, D_i = sigma_i D~_i), the potential w_i of box operator
    Lap - kappa~_i with jumps [u] = phi, [d_n u] = psi/sigma_i equals
    D~_i phi - S_i psi, so (avg = mean of the two one-sided limits)
        avg value   w_i = K_i phi - S_i psi,
        sigma_i avg d_n w_i = D_i phi - K'_i psi,
    and the left-hand side of eq. (bie-ifp-1) is
        A [phi; psi] = [phi - (avg w_1 - avg w_2);
                        psi - (sigma_1 avg d_n w_1 - sigma_2 avg d_n w_2)].
    Right-hand side: with P_1 the kappa~_1 potential of [d_n u] = g2/sigma_1
    and F = f_1/sigma_1 in Omega_1 (G_1 f_1 - S_1 g2), and P_2 the kappa~_2
    potential of [u] = g1, F = f_2/sigma_2 in Omega_2 and the outer data g_B
    (G_2 f_2 + K_2 g1),
        b = [g1/2 + avg P_1 + avg P_2;
             -g2/2 + sigma_1 avg d_n P_1 + sigma_2 avg d_n P_2].
    Solution: u_1 (extended by 0) is the kappa~_1 potential of [u] = phi,
    [d_n u] = (psi + g2)/sigma_1, F = f_1/sigma_1 in Omega_1; u_2 (0 in
    Omega_1) the kappa~_2 potential of [u] = -(phi - g1), [d_n u] =
    -psi/sigma_2, F = f_2/sigma_2 in Omega_2, outer data g_B.
    Reading: the outer boundary data of the paper's homogeneous condition
    may be non-zero and enter through P_2 and u_2 only."""

    def __init__(self, w: W.Workload):
        self.w = w
        self.s1, self.s2 = w.sigma_in, w.sigma_out
        self.P1 = Problem(w, kt=w.kappa / w.sigma_in)
        self.P2 = Problem(w, kt=w.kappa_out / w.sigma_out)
        self.nb = self.P1.nb
        self.inside = self.P1.inside
        self.surf = self.P1.surf

    def _avg(self, P, a, b, *data):
        u, cv, _, _ = P.potential(a, b, *data)
        vp, vm, dp, dm = P.traces(u, cv)
        return 0.5 * (vp + vm), 0.5 * (dp + dm)

    def apply(self, x: np.ndarray) -> np.ndarray:
        nb = self.nb
        phi, psi = x[:nb], x[nb:]
        v1, d1 = self._avg(self.P1, phi, psi / self.s1)
        v2, d2 = self._avg(self.P2, phi, psi / self.s2)
        return np.concatenate([phi - (v1 - v2), psi - (self.s1 * d1 - self.s2 * d2)])

    def _sides(self, data):
        zi = np.zeros_like(data["f_in"])
        zo = np.zeros_like(data["f_out"])
        side1 = (data["f_in"] / self.s1, zo, data["lapf_in"] / self.s1, zo)
        side2 = (zi, data["f_out"] / self.s2, zi, data["lapf_out"] / self.s2)
        return side1, side2

    def bie_rhs(self, g1, g2, data) -> np.ndarray:
        side1, side2 = self._sides(data)
        z = np.zeros(self.nb)
        v1, d1 = self._avg(self.P1, z, g2 / self.s1, *side1)
        v2, d2 = self._avg(self.P2, g1, z, *side2, data["g_b"])
        return np.concatenate([0.5 * g1 + v1 + v2, -0.5 * g2 + self.s1 * d1 + self.s2 * d2])

    def evaluate(self, x, g1, g2, data) -> np.ndarray:
        nb = self.nb
        phi, psi = x[:nb], x[nb:]
        side1, side2 = self._sides(data)
        u1 = self.P1.potential(phi, (psi + g2) / self.s1, *side1)[0]
        u2 = self.P2.potential(-(phi - g1), -psi / self.s2, *side2, data["g_b"])[0]
        return np.where(self.inside, u1, u2)

    def solve(self, g1, g2, data, rtol=1e-10, restart=100, max_iter=200):
        b = self.bie_rhs(g1, g2, data)
        x, it, rel = gmres(self.apply, b, rtol=rtol, restart=restart, max_iter=max_iter)
        return self.evaluate(x, g1, g2, data), x, it, rel


def gmres(apply, b, x0=None, rtol=1e-10, restart=100, max_iter=200, strict=True):
    """GMRES with modified Gram-Schmidt Arnoldi and Givens rotations.
    Returns (x, iterations = operator applications in Arnoldi, relative
    residual estimate).  When max_iter is reached: raises RuntimeError if
    `strict`, else returns the iterate (used to compare at a fixed count)."""
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros(n), 0, 0.0
    total = 0
    while True:
        r = b - apply(x) if np.any(x != 0.0) else b.copy()
        beta = np.linalg.norm(r)
        if beta <= rtol * bnorm:
            return x, total, beta / bnorm
        m = restart
        V = np.zeros((m + 1, n))
        Hm = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j_end = 0
        res = beta
        for j in range(m):
            wv = apply(V[j])
            total += 1
            for i in range(j + 1):
                Hm[i, j] = np.dot(wv, V[i])
                wv = wv - Hm[i, j] * V[i]
            Hm[j + 1, j] = np.linalg.norm(wv)
            if Hm[j + 1, j] != 0.0:
                V[j + 1] = wv / Hm[j + 1, j]
            for i in range(j):
                t = cs[i] * Hm[i, j] + sn[i] * Hm[i + 1, j]
                Hm[i + 1, j] = -sn[i] * Hm[i, j] + cs[i] * Hm[i + 1, j]
                Hm[i, j] = t
            rr = np.hypot(Hm[j, j], Hm[j + 1, j])
            cs[j] = Hm[j, j] / rr
            sn[j] = Hm[j + 1, j] / rr
            Hm[j, j] = rr
            Hm[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            res = abs(g[j + 1])
            j_end = j + 1
            if res <= rtol * bnorm or total >= max_iter:
                break
        y = np.zeros(j_end)
        for i in range(j_end - 1, -1, -1):
            y[i] = (g[i] - np.dot(Hm[i, i + 1:j_end], y[i + 1:j_end])) / Hm[i, i]
        x = x + V[:j_end].T @ y
        if res <= rtol * bnorm:
            return x, total, res / bnorm
        if total >= max_iter:
            if not strict:
                return x, total, res / bnorm
            raise RuntimeError(f"GMRES not converged in {max_iter} iterations "
                               f"(rel. residual {res / bnorm:.3e})")


def errors(u, exact, mask):
    """||e||_inf and RMS ||e||_2 over the nodes in mask (Sec. 7)."""
    e = np.abs(u - exact)[mask]
    return float(e.max()), float(np.sqrt(np.mean(e * e)))
