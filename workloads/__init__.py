"""Seeded synthetic workloads for the correction-function KFBI solver.

This module holds only problem *inputs*: level-set specifications (kind code +
parameter vector), manufactured exact solutions, the data those solutions induce
at given interface points (Dirichlet data g_D, jumps g1 = [u] and
g2 = [sigma d_n u]) and on grid nodes (right-hand sides f and their Laplacians),
and the seeded instance draws of the batched and learned workloads.  It contains
none of the method's arithmetic (no classification, no collocation, no finite
differences, no box solve), so both the CPU oracle and the CUDA path may import
it without sharing any of the method.

Sign conventions follow Sec. 2 and Sec. 5 of the paper: the level set H is
negative inside Omega (the "+" side), the unit normal n = grad H / |grad H|
points out of Omega, and jumps are [v] = v(inside) - v(outside).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Level-set kind codes (values shared with the C header's kfbi_levelset_kind).
LS_ELLIPSE = 1      # 2D: p = [cx, cy, a, b, theta]
LS_STAR = 2         # 2D: p = [cx, cy, R0, A, k]; r = R0 + A sin(k theta)
LS_ELLIPSOID = 3    # 3D: p = [cx, cy, cz, a, b, c]
LS_TORUS = 4        # 3D: p = [R, r] (axis z, centred at the origin)
LS_MOLECULE = 5     # 3D: p = [r, level, n_atoms, x1, y1, z1, x2, ...]
LS_DISCS = 6        # 2D: p = [r, n, x1, y1, ...], union of n separated discs
LS_SPHERES = 7      # 3D: p = [r, n, x1, y1, z1, ...], union of n separated balls
LS_GRID = 8         # H sampled at the grid nodes: p = [], samples in extra["samples"]
LS_UNION = 9        # p = [m, kind_1, params_1..., kind_m, params_m...]: m interfaces,
                    # each of an analytic kind (ellipse, star, ellipsoid, torus)

# Parameters per component of a union (the layouts above).
UNION_PARAMS = {LS_ELLIPSE: 5, LS_STAR: 5, LS_ELLIPSOID: 6, LS_TORUS: 2}


def union_components(p):
    """[(kind, params), ...] of a union's parameter vector."""
    m = int(p[0])
    out, at = [], 1
    for _ in range(m):
        kind = int(p[at])
        cnt = UNION_PARAMS[kind]
        out.append((kind, list(p[at + 1: at + 1 + cnt])))
        at += 1 + cnt
    return out


def union_params(components):
    """Parameter vector of a union from [(kind, params), ...]."""
    p = [float(len(components))]
    for kind, q in components:
        assert len(q) == UNION_PARAMS[kind]
        p += [float(kind)] + [float(v) for v in q]
    return p


def n_interfaces(ls_kind: int, p) -> int:
    """Number of interfaces (components of Omega, each with its own side
    label 1 + k): the balls of a ball union, the components of a union, else 1."""
    if ls_kind in (LS_DISCS, LS_SPHERES):
        return int(p[1])
    if ls_kind == LS_UNION:
        return int(p[0])
    return 1

# Problem kinds (shared with kfbi_problem_kind).
KIND_DIRICHLET = 0  # interior Dirichlet BVP, eq. (bie-D)
KIND_INTERFACE_MU = 1  # two-medium interface problem, kappa = 0, mu-form BIE
KIND_NEUMANN = 2    # interior Neumann BVP, eq. (bie-N)
KIND_INTERFACE_GENERAL = 3  # interface problem, any kappa_i/sigma_i, eq. (bie-ifp-1)

BOX_DST = 0
BOX_MG = 1
PREC_FP64 = 0
PREC_MIXED = 1


@dataclass
class Workload:
    """One synthetic problem: geometry, coefficients and manufactured solution."""

    name: str
    dim: int
    n: int
    lo: float
    hi: float
    ls_kind: int
    ls_params: list
    kind: int
    sigma_in: float = 1.0
    sigma_out: float = 1.0
    kappa: float = 0.0
    order: int = 4
    cos_alpha: float | None = None
    kappa_out: float = 0.0   # kappa of Omega_2 (general interface problem only)
    exact: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def h(self) -> float:
        return (self.hi - self.lo) / self.n

    def cosa(self) -> float:
        """cos(alpha) of the overlapping surface decomposition.  2D: 0.707, just
        inside the admissible range alpha > 45 deg, which reproduces the paper's
        Table 1 point counts N_b; 3D: 0.4."""
        if self.cos_alpha is not None:
            return self.cos_alpha
        return 0.707 if self.dim == 2 else 0.4


# ---------------------------------------------------------------------------
# Manufactured solutions.  Each returns callables u(X), grad u(X), lap u(X) for
# points X of shape (..., d).  They are the data of the synthetic problems.
# ---------------------------------------------------------------------------

def _sol_exp_sin():
    # u = e^x sin y (harmonic)
    u = lambda X: np.exp(X[..., 0]) * np.sin(X[..., 1])
    g = lambda X: np.stack([np.exp(X[..., 0]) * np.sin(X[..., 1]),
                            np.exp(X[..., 0]) * np.cos(X[..., 1])], -1)
    lap = lambda X: np.zeros(X.shape[:-1])
    return u, g, lap


def _sol_paper_table1():
    # u = exp(x) sin(cos(pi/3) x + sin(pi/3) y); lap u = 2 cos(pi/3) e^x cos(.)
    ca, sa = math.cos(math.pi / 3), math.sin(math.pi / 3)
    arg = lambda X: ca * X[..., 0] + sa * X[..., 1]
    u = lambda X: np.exp(X[..., 0]) * np.sin(arg(X))
    g = lambda X: np.stack([np.exp(X[..., 0]) * (np.sin(arg(X)) + ca * np.cos(arg(X))),
                            np.exp(X[..., 0]) * sa * np.cos(arg(X))], -1)
    lap = lambda X: 2.0 * ca * np.exp(X[..., 0]) * np.cos(arg(X))
    return u, g, lap


def _sol_sin_cos():
    # u = sin x cos y; lap u = -2 u
    u = lambda X: np.sin(X[..., 0]) * np.cos(X[..., 1])
    g = lambda X: np.stack([np.cos(X[..., 0]) * np.cos(X[..., 1]),
                            -np.sin(X[..., 0]) * np.sin(X[..., 1])], -1)
    lap = lambda X: -2.0 * np.sin(X[..., 0]) * np.cos(X[..., 1])
    return u, g, lap


def _sol_r2():
    # u = |x|^2 ; lap u = 2 d
    u = lambda X: np.sum(X * X, axis=-1)
    g = lambda X: 2.0 * X
    lap = lambda X: np.full(X.shape[:-1], 2.0 * X.shape[-1])
    return u, g, lap


def _sol_exp3():
    # u = e^{x+y+z}/10 ; lap u = 3 u
    u = lambda X: np.exp(X[..., 0] + X[..., 1] + X[..., 2]) / 10.0
    g = lambda X: np.repeat(u(X)[..., None], 3, axis=-1)
    lap = lambda X: 3.0 * u(X)
    return u, g, lap


def _sol_exp_cos3():
    # u = e^z (cos 2x + cos 3y), the Neumann torus example of Sec. 7;
    # lap u = e^z (-3 cos 2x - 8 cos 3y)
    u = lambda X: np.exp(X[..., 2]) * (np.cos(2 * X[..., 0]) + np.cos(3 * X[..., 1]))
    g = lambda X: np.stack([-2 * np.exp(X[..., 2]) * np.sin(2 * X[..., 0]),
                            -3 * np.exp(X[..., 2]) * np.sin(3 * X[..., 1]),
                            np.exp(X[..., 2]) * (np.cos(2 * X[..., 0]) + np.cos(3 * X[..., 1]))], -1)
    lap = lambda X: np.exp(X[..., 2]) * (-3 * np.cos(2 * X[..., 0]) - 8 * np.cos(3 * X[..., 1]))
    return u, g, lap


def _sol_zero(d):
    u = lambda X: np.zeros(X.shape[:-1])
    g = lambda X: np.zeros(X.shape)
    lap = lambda X: np.zeros(X.shape[:-1])
    return u, g, lap


def _sol_harmonic3(amps):
    # u = sum_k a_k h_k with h in {1, x, y, z, xy, yz, zx, x^2 - y^2}
    a = np.asarray(amps, dtype=np.float64)

    def u(X):
        x, y, z = X[..., 0], X[..., 1], X[..., 2]
        return (a[0] + a[1] * x + a[2] * y + a[3] * z + a[4] * x * y + a[5] * y * z
                + a[6] * z * x + a[7] * (x * x - y * y))

    def g(X):
        x, y, z = X[..., 0], X[..., 1], X[..., 2]
        gx = a[1] + a[4] * y + a[6] * z + 2 * a[7] * x
        gy = a[2] + a[4] * x + a[5] * z - 2 * a[7] * y
        gz = a[3] + a[5] * y + a[6] * x
        return np.stack([gx, gy, gz], -1)

    lap = lambda X: np.zeros(X.shape[:-1])
    return u, g, lap


# Solutions with a closed-form bi-Laplacian: (u, grad u, lap u, lap lap u), so
# that lap f = sigma lap lap u - kappa lap u needs no per-solution case.

def _sol4_exp_68():
    # u = exp(0.6 x + 0.8 y): lap u = u (0.36 + 0.64 = 1)
    u = lambda X: np.exp(0.6 * X[..., 0] + 0.8 * X[..., 1])
    g = lambda X: np.stack([0.6 * u(X), 0.8 * u(X)], -1)
    return u, g, u, u


def _sol4_sinsin_pi():
    # u = sin(pi (x + 1)/2) sin(pi (y + 1)/2): lap u = -(pi^2/2) u
    k = 0.5 * math.pi
    sx = lambda X: np.sin(k * (X[..., 0] + 1.0))
    sy = lambda X: np.sin(k * (X[..., 1] + 1.0))
    u = lambda X: sx(X) * sy(X)
    g = lambda X: np.stack([k * np.cos(k * (X[..., 0] + 1.0)) * sy(X),
                            k * sx(X) * np.cos(k * (X[..., 1] + 1.0))], -1)
    lam = -2.0 * k * k
    return u, g, (lambda X: lam * u(X)), (lambda X: lam * lam * u(X))


def _sol4_torus_in():
    # u = sin^2(2x) cos^2(2y) cos z = (1 - cos 4x)(1 + cos 4y) cos z / 4; every
    # product of cosines is an eigenfunction of lap (eigenvalues -1, -17, -17, -33)
    def parts(X):
        c4x, c4y, cz = np.cos(4 * X[..., 0]), np.cos(4 * X[..., 1]), np.cos(X[..., 2])
        return c4x, c4y, cz
    u = lambda X: np.sin(2 * X[..., 0]) ** 2 * np.cos(2 * X[..., 1]) ** 2 * np.cos(X[..., 2])

    def g(X):
        s2x, c2y, cz = np.sin(2 * X[..., 0]), np.cos(2 * X[..., 1]), np.cos(X[..., 2])
        return np.stack([2.0 * np.sin(4 * X[..., 0]) * c2y * c2y * cz,
                         -2.0 * s2x * s2x * np.sin(4 * X[..., 1]) * cz,
                         -s2x * s2x * c2y * c2y * np.sin(X[..., 2])], -1)

    def lap(X):
        c4x, c4y, cz = parts(X)
        return (-1.0 - 17.0 * c4y + 17.0 * c4x + 33.0 * c4x * c4y) * cz / 4.0

    def lap2(X):
        c4x, c4y, cz = parts(X)
        return (1.0 + 289.0 * c4y - 289.0 * c4x - 1089.0 * c4x * c4y) * cz / 4.0
    return u, g, lap, lap2


def _sol4_exp_cos3():
    u, g, lap = _sol_exp_cos3()
    # lap(e^z cos kx) = (1 - k^2) e^z cos kx: eigenvalues -3 and -8
    lap2 = lambda X: np.exp(X[..., 2]) * (9 * np.cos(2 * X[..., 0]) + 64 * np.cos(3 * X[..., 1]))
    return u, g, lap, lap2


def _sol4_cos3():
    # u = cos x cos y cos z: lap u = -3 u
    u = lambda X: np.cos(X[..., 0]) * np.cos(X[..., 1]) * np.cos(X[..., 2])
    g = lambda X: np.stack([-np.sin(X[..., 0]) * np.cos(X[..., 1]) * np.cos(X[..., 2]),
                            -np.cos(X[..., 0]) * np.sin(X[..., 1]) * np.cos(X[..., 2]),
                            -np.cos(X[..., 0]) * np.cos(X[..., 1]) * np.sin(X[..., 2])], -1)
    return u, g, (lambda X: -3.0 * u(X)), (lambda X: 9.0 * u(X))


def _sol4_exp3():
    u, g, lap = _sol_exp3()
    return u, g, lap, (lambda X: 9.0 * u(X))


def _sol4_harmonic3(amps):
    u, g, lap = _sol_harmonic3(amps)
    return u, g, lap, lap


def _sol4_cos_cosh():
    # u = cos x cosh y (harmonic)
    u = lambda X: np.cos(X[..., 0]) * np.cosh(X[..., 1])
    g = lambda X: np.stack([-np.sin(X[..., 0]) * np.cosh(X[..., 1]),
                            np.cos(X[..., 0]) * np.sinh(X[..., 1])], -1)
    z = lambda X: np.zeros(X.shape[:-1])
    return u, g, z, z


_SOL4 = {"exp_68": _sol4_exp_68, "cos_cosh": _sol4_cos_cosh, "sinsin_pi": _sol4_sinsin_pi, "torus_in": _sol4_torus_in,
         "exp_cos3": _sol4_exp_cos3, "cos3": _sol4_cos3, "exp3": _sol4_exp3}


def _sol4(w: Workload, name: str):
    if name == "harmonic3":
        return _sol4_harmonic3(w.extra["amps"])
    return _SOL4[name]()


def is_multi(w: Workload) -> bool:
    """A workload whose interfaces have different interior solutions (one
    smooth solution u^(k) per component Omega^(k), u^(0) outside)."""
    return w.exact == "multi"


def multi_solutions(w: Workload):
    """([(u, grad, lap, lap2) of each interface k], (u, grad, lap, lap2)
    outside) of a workload with per-interface solutions
    (extra["sol_in"] = names per interface, extra["sol_out"] = the name outside)."""
    return ([_sol4(w, nm) for nm in w.extra["sol_in"]], _sol4(w, w.extra["sol_out"]))


def solutions(w: Workload):
    """(u_in, grad_in, lap_in), (u_out, grad_out, lap_out) of a workload
    (of its first interface for a per-interface workload)."""
    e = w.exact
    if e == "multi":
        ins, out = multi_solutions(w)
        return ins[0][:3], out[:3]
    if e == "exp_sin":
        s = _sol_exp_sin()
        return s, _sol_zero(2)
    if e == "paper_table1":
        return _sol_paper_table1(), _sol_zero(2)
    if e == "sincos_r2":
        return _sol_sin_cos(), _sol_r2()
    if e == "exp3":
        return _sol_exp3(), _sol_zero(3)
    if e == "harmonic3":
        return _sol_harmonic3(w.extra["amps"]), _sol_zero(3)
    if e == "exp_cos3":
        return _sol_exp_cos3(), _sol_zero(3)
    if e == "sincos_expsin":
        return _sol_sin_cos(), _sol_exp_sin()
    if e == "exp3_harmonic3":
        return _sol_exp3(), _sol_harmonic3(w.extra["amps"])
    if e == "waves_io":
        return _sol_waves(w.extra["seed_in"]), _sol_waves(w.extra["seed_out"])
    raise ValueError(f"unknown exact solution {e!r}")


def grid_coords(w: Workload) -> np.ndarray:
    """Node coordinates x_i = lo + i h, shape (N+1,)*d + (d,), axis d-1 fastest."""
    n = w.n
    i = np.arange(n + 1)
    x = w.lo + i * w.h
    mesh = np.meshgrid(*([x] * w.dim), indexing="ij")
    return np.stack(mesh, -1)


def _grid_data_multi(w: Workload):
    """grid_data of a per-interface workload: f_in, lapf_in and u_in have a
    leading axis of length K (grid k is interface k's f, smoothly extended)."""
    assert w.kind in (KIND_INTERFACE_MU, KIND_INTERFACE_GENERAL, KIND_DIRICHLET)
    X = grid_coords(w)
    ins, (uo, _, lo_, l2o) = multi_solutions(w)
    if w.kind == KIND_DIRICHLET:
        # interior BVP: f = sigma lap u - kappa u inside, no outer data
        f_in = np.stack([w.sigma_in * li(X) - w.kappa * ui(X) for ui, _, li, _ in ins])
        lapf_in = np.stack([w.sigma_in * l2(X) - w.kappa * li(X) for _, _, li, l2 in ins])
        z = np.zeros(X.shape[:-1])
        return dict(f_in=f_in, f_out=z, lapf_in=lapf_in, lapf_out=z.copy(),
                    u_in=np.stack([ui(X) for ui, _, _, _ in ins]), u_out=z.copy(), g_b=z.copy())
    # the mu-form workloads are Poisson problems (as in grid_data)
    k_in, k_out = (w.kappa, w.kappa_out) if w.kind == KIND_INTERFACE_GENERAL else (0.0, 0.0)
    f_in = np.stack([w.sigma_in * li(X) - k_in * ui(X) for ui, _, li, _ in ins])
    lapf_in = np.stack([w.sigma_in * l2(X) - k_in * li(X) for _, _, li, l2 in ins])
    f_out = w.sigma_out * lo_(X) - k_out * uo(X)
    lapf_out = w.sigma_out * l2o(X) - k_out * lo_(X)
    u_out = uo(X)
    gb = np.zeros_like(f_out)
    bmask = np.ones(f_out.shape, dtype=bool)
    bmask[tuple(slice(1, -1) for _ in range(w.dim))] = False
    gb[bmask] = u_out[bmask]
    return dict(f_in=f_in, f_out=f_out, lapf_in=lapf_in, lapf_out=lapf_out,
                u_in=np.stack([ui(X) for ui, _, _, _ in ins]), u_out=u_out, g_b=gb)


def grid_data(w: Workload):
    """Right-hand-side grids of the physical PDE on each side.

    Returns dict with f_in, f_out (= sigma_side * lap u_side - kappa u_side, the f of
    eqs. (BVP)/(IFP), smoothly extended to the whole box), their Laplacians
    lapf_in, lapf_out (for the h^2/12 Lap f term of eqs. (9p-cds)/(27p-cds)),
    the exact solution on both sides, and the outer boundary values g_B.
    Laplacians of f are formed from the closed forms of the solutions.
    Per-interface workloads: see _grid_data_multi.
    """
    if is_multi(w):
        return _grid_data_multi(w)
    X = grid_coords(w)
    (ui, gi, li), (uo, go, lo_) = solutions(w)
    d = w.dim
    if w.kind in (KIND_DIRICHLET, KIND_NEUMANN):
        s, k = w.sigma_in, w.kappa
        f_in = s * li(X) - k * ui(X)
        f_out = np.zeros_like(f_in)
        lapf_in = _lap_of_f(w, X, inside=True)
        lapf_out = np.zeros_like(f_in)
        u_out_grid = np.zeros_like(f_in)
    elif w.kind == KIND_INTERFACE_GENERAL:
        f_in = w.sigma_in * li(X) - w.kappa * ui(X)
        f_out = w.sigma_out * lo_(X) - w.kappa_out * uo(X)
        lapf_in = _lap_of_f(w, X, inside=True)
        lapf_out = _lap_of_f(w, X, inside=False)
        u_out_grid = uo(X)
    else:
        f_in = w.sigma_in * li(X)
        f_out = w.sigma_out * lo_(X)
        lapf_in = _lap_of_f(w, X, inside=True)
        lapf_out = _lap_of_f(w, X, inside=False)
        u_out_grid = uo(X)
    gb = np.zeros_like(f_in)
    bmask = np.zeros(f_in.shape, dtype=bool)
    for ax in range(d):
        sl0 = [slice(None)] * d
        sl0[ax] = 0
        sl1 = [slice(None)] * d
        sl1[ax] = -1
        bmask[tuple(sl0)] = True
        bmask[tuple(sl1)] = True
    if w.kind in (KIND_INTERFACE_MU, KIND_INTERFACE_GENERAL):
        gb[bmask] = u_out_grid[bmask]
    return dict(f_in=f_in, f_out=f_out, lapf_in=lapf_in, lapf_out=lapf_out,
                u_in=ui(X), u_out=u_out_grid, g_b=gb)


def _lap_of_f(w: Workload, X, inside: bool):
    """Closed-form Laplacian of the physical f on one side."""
    e = w.exact
    if e in ("exp_sin", "harmonic3", "waves_io"):
        return np.zeros(X.shape[:-1])
    if e == "paper_table1":
        # f = lap u = 2 ca e^x cos(arg); lap(e^x cos(arg)) = 2 e^x * (-ca sin(arg)) + 0
        ca, sa = math.cos(math.pi / 3), math.sin(math.pi / 3)
        arg = ca * X[..., 0] + sa * X[..., 1]
        return w.sigma_in * 2.0 * ca * (-2.0 * ca * np.exp(X[..., 0]) * np.sin(arg))
    if e == "sincos_r2":
        if inside:  # f = sigma_in * (-2 sin x cos y); lap = sigma_in * 4 sin x cos y
            return w.sigma_in * 4.0 * np.sin(X[..., 0]) * np.cos(X[..., 1])
        return np.zeros(X.shape[:-1])
    if e == "sincos_expsin":
        # inside f = (-2 sigma - kappa) sin x cos y, lap f = -2 f; outside
        # u = e^x sin y is harmonic, so f = -kappa u has lap f = 0
        if inside:
            return -2.0 * (-2.0 * w.sigma_in - w.kappa) * np.sin(X[..., 0]) * np.cos(X[..., 1])
        return np.zeros(X.shape[:-1])
    if e == "exp_cos3":  # f = sigma lap u - kappa u with lap(e^z cos kx) = (1 - k^2) e^z cos kx
        ez = np.exp(X[..., 2])
        c2, c3 = np.cos(2 * X[..., 0]), np.cos(3 * X[..., 1])
        s, k = w.sigma_in, w.kappa
        return s * ez * (9 * c2 + 64 * c3) - k * ez * (-3 * c2 - 8 * c3)
    if e in ("exp3", "exp3_harmonic3"):  # f = (3 - kappa) u sigma-scaled; lap f = 3 f
        if not inside:  # zero, or harmonic outside: f = -kappa u has lap f = 0
            return np.zeros(X.shape[:-1])
        u = np.exp(X[..., 0] + X[..., 1] + X[..., 2]) / 10.0
        return 3.0 * (w.sigma_in * 3.0 - w.kappa) * u
    raise ValueError(e)


def boundary_data(w: Workload, pts: np.ndarray, normals: np.ndarray, iface=None):
    """Interface data at points with unit normals (outward from Omega).

    Dirichlet BVP: returns (g_D, None).  Neumann BVP: returns
    (None, g_N) with g_N = sigma d_n u.  Interface problem: returns
    (g1, g2) with g1 = u_in - u_out and g2 = sigma_in d_n u_in - sigma_out d_n u_out,
    the jump conditions of eq. (IFP-bc).  Per-interface workloads take the
    interface index of every point (`iface`) and use that interface's u_in.
    """
    if is_multi(w):
        ins, (uo, go, _, _) = multi_solutions(w)
        iface = np.asarray(iface)
        ui_v = np.zeros(pts.shape[0])
        gi_v = np.zeros(pts.shape)
        for k, (ui, gi, _, _) in enumerate(ins):
            m = iface == k
            ui_v[m] = ui(pts[m])
            gi_v[m] = gi(pts[m])
        dn_in = np.sum(gi_v * normals, -1)
        if w.kind == KIND_DIRICHLET:
            return ui_v, None
        if w.kind == KIND_NEUMANN:
            return None, w.sigma_in * dn_in
        return (ui_v - uo(pts),
                w.sigma_in * dn_in - w.sigma_out * np.sum(go(pts) * normals, -1))
    (ui, gi, _), (uo, go, _) = solutions(w)
    if w.kind == KIND_DIRICHLET:
        return ui(pts), None
    if w.kind == KIND_NEUMANN:
        return None, w.sigma_in * np.sum(gi(pts) * normals, -1)
    g1 = ui(pts) - uo(pts)
    g2 = (w.sigma_in * np.sum(gi(pts) * normals, -1)
          - w.sigma_out * np.sum(go(pts) * normals, -1))
    return g1, g2


def exact_grid(w: Workload, inside_mask: np.ndarray) -> np.ndarray:
    """Exact solution on the grid, side chosen by the given inside mask (a
    node label array, 0 outside and 1 + k in interface k, for per-interface
    workloads)."""
    X = grid_coords(w)
    if is_multi(w):
        ins, out = multi_solutions(w)
        lab = np.asarray(inside_mask).astype(np.int64)
        u = out[0](X)
        for k, s in enumerate(ins):
            u = np.where(lab == k + 1, s[0](X), u)
        return u
    (ui, _, _), (uo, _, _) = solutions(w)
    return np.where(inside_mask, ui(X), uo(X))


# ---------------------------------------------------------------------------
# The configured workloads.
# ---------------------------------------------------------------------------

def ellipse_dirichlet_2d(n: int = 64) -> Workload:
    """2D interior Dirichlet Poisson BVP: x^2/0.36 + y^2/0.16 < 1, u = e^x sin y."""
    return Workload("ellipse_dirichlet_2d", 2, n, -1.0, 1.0, LS_ELLIPSE,
                    [0.0, 0.0, 0.6, 0.4, 0.0], KIND_DIRICHLET, exact="exp_sin")


def paper_table1_2d(n: int = 64) -> Workload:
    """The paper's first 2D example (Sec. 7.1.1): rotated ellipse a=1, b=0.5,
    theta=-pi/6 in [-1.2, 1.2]^2 with u = exp(x) sin(cos(pi/3)x + sin(pi/3)y)."""
    return Workload("paper_table1_2d", 2, n, -1.2, 1.2, LS_ELLIPSE,
                    [0.0, 0.0, 1.0, 0.5, -math.pi / 6], KIND_DIRICHLET,
                    exact="paper_table1")


def flower_interface_2d(n: int = 256, contrast: float = 1000.0) -> Workload:
    """2D Poisson interface problem, flower r = 0.5 + 0.1 sin(5 theta),
    sigma_in/sigma_out = contrast, u_in = sin x cos y, u_out = x^2 + y^2."""
    return Workload("flower_interface_2d", 2, n, -1.0, 1.0, LS_STAR,
                    [0.0, 0.0, 0.5, 0.1, 5.0], KIND_INTERFACE_MU,
                    sigma_in=contrast, sigma_out=1.0, exact="sincos_r2")


def torus_helmholtz_3d(n: int = 128) -> Workload:
    """3D Dirichlet modified-Helmholtz BVP (kappa = 1) inside the torus
    (sqrt(x^2+y^2) - 0.5)^2 + z^2 < 0.2^2, u = e^{x+y+z}/10."""
    return Workload("torus_helmholtz_3d", 3, n, -1.0, 1.0, LS_TORUS, [0.5, 0.2],
                    KIND_DIRICHLET, kappa=1.0, exact="exp3")


def neumann_torus_3d(n: int = 64, kappa: float = 0.0) -> Workload:
    """The paper's 3D Neumann example (Sec. 7.2.1): torus (1 - sqrt(x^2+y^2))^2
    + z^2 < 0.4^2 in [-1.5, 1.5]^3, u = e^z (cos 2x + cos 3y), Poisson
    (kappa = 0, solution fixed up to a constant) or modified Helmholtz.
    cos(alpha) = 0.55, inside the admissible range (0, 1/sqrt(3)) of 3D: fewer
    overlapping DOFs than 0.4 and a GMRES count at tolerance 1e-10 close to
    the paper's.  At N = 64 the box wall lies 2.1 h from the torus, too close
    for a one-sided outside trace fit (the library refuses that grid)."""
    return Workload("neumann_torus_3d", 3, n, -1.5, 1.5, LS_TORUS, [1.0, 0.4],
                    KIND_NEUMANN, kappa=kappa, cos_alpha=0.55, exact="exp_cos3")


def neumann_ellipse_2d(n: int = 64, kappa: float = 0.0) -> Workload:
    """2D interior Neumann BVP on the rotated ellipse of the paper's first
    example; Poisson with that example's solution, or modified Helmholtz
    (kappa > 0) with u = e^x sin y (harmonic, f = -kappa u)."""
    return Workload("neumann_ellipse_2d", 2, n, -1.2, 1.2, LS_ELLIPSE,
                    [0.0, 0.0, 1.0, 0.5, -math.pi / 6], KIND_NEUMANN, kappa=kappa,
                    exact="paper_table1" if kappa == 0.0 else "exp_sin")


def hetero_interface_2d(n: int = 128, sigma_in: float = 1.0, kappa_in: float = 0.0,
                        sigma_out: float = 4.0, kappa_out: float = 10.0) -> Workload:
    """2D interface problem with different operators on the two sides (the
    coefficients of the paper's heterogeneous example, Sec. 7.2.5: Poisson
    inside, modified Helmholtz outside) on the flower r = 0.5 + 0.1 sin 5 theta,
    u_in = sin x cos y, u_out = e^x sin y, outer Dirichlet data from u_out."""
    return Workload("hetero_interface_2d", 2, n, -1.0, 1.0, LS_STAR,
                    [0.0, 0.0, 0.5, 0.1, 5.0], KIND_INTERFACE_GENERAL,
                    sigma_in=sigma_in, sigma_out=sigma_out, kappa=kappa_in,
                    kappa_out=kappa_out, exact="sincos_expsin")


def hetero_sphere_3d(n: int = 256) -> Workload:
    """3D heterogeneous interface problem with Sec. 7.2.5's coefficients
    (sigma_1 = 1, kappa_1 = 0 inside; sigma_2 = 4, kappa_2 = 10 outside) on one
    sphere of radius 0.7 in [-1.5, 1.5]^3; u_1 = e^(x+y+z)/10, u_2 a fixed
    harmonic quadratic, outer Dirichlet data from u_2."""
    return Workload("hetero_sphere_3d", 3, n, -1.5, 1.5, LS_ELLIPSOID,
                    [0.0, 0.0, 0.0, 0.7, 0.7, 0.7], KIND_INTERFACE_GENERAL,
                    sigma_in=1.0, sigma_out=4.0, kappa=0.0, kappa_out=10.0,
                    exact="exp3_harmonic3",
                    extra={"amps": [0.3, 0.2, -0.1, 0.25, 0.15, -0.2, 0.1, 0.05]})


def discs_interface_2d(n: int = 128, contrast: float = 10.0) -> Workload:
    """2D Poisson interface problem with four disjoint interfaces: discs of
    radius 0.25 centred at (+-0.45, +-0.45) (0.4 apart), sigma_in/sigma_out =
    contrast, u_in = sin x cos y, u_out = x^2 + y^2."""
    return Workload("discs_interface_2d", 2, n, -1.0, 1.0, LS_DISCS,
                    [0.25, 4.0, -0.45, -0.45, 0.45, -0.45, -0.45, 0.45, 0.45, 0.45],
                    KIND_INTERFACE_MU, sigma_in=contrast, sigma_out=1.0, exact="sincos_r2")


def hetero_spheres_3d(n: int = 256, radius: float = 0.6) -> Workload:
    """Sec. 7.2.5's heterogeneous problem (sigma_1 = 1, kappa_1 = 0 inside;
    sigma_2 = 4, kappa_2 = 10 outside) with its three sphere centres
    (0.5, 0.5, 0.5), (-0.5, -0.5, 0.5), (0.5, -0.5, -0.5); the paper's radius
    is 0.7 (the spheres 0.0142 apart), radius 0.6 leaves them 0.21 apart; box
    [-1.5, 1.5]^3, u_1 = e^(x+y+z)/10, u_2 a fixed harmonic quadratic."""
    return Workload("hetero_spheres_3d", 3, n, -1.5, 1.5, LS_SPHERES,
                    [radius, 3.0, 0.5, 0.5, 0.5, -0.5, -0.5, 0.5, 0.5, -0.5, -0.5],
                    KIND_INTERFACE_GENERAL, sigma_in=1.0, sigma_out=4.0, kappa=0.0,
                    kappa_out=10.0, exact="exp3_harmonic3",
                    extra={"amps": [0.3, 0.2, -0.1, 0.25, 0.15, -0.2, 0.1, 0.05]})


def touching_interfaces_2d(n: int = 256) -> Workload:
    """Sec. 7.1.2's multiple interfaces (Table 2): eight circles of radius
    0.383 centred at (cos(m pi/4), sin(m pi/4)), m = 1..8, and the five-fold
    star r = 0.514 (1 + 0.2 sin 5 theta) at the origin, in [-1.7, 1.7]^2.
    Neighbouring circles overlap by 6.3e-4 (2 * 0.383 > 2 sin(pi/8)) and the
    star's tip at theta = pi/2 is 2e-4 from the circle above it.  Poisson
    interface problem, sigma_i = 1, sigma_e = 3, u = exp(0.6 x + 0.8 y) in
    every interior component, sin(pi (x+1)/2) sin(pi (y+1)/2) outside."""
    comps = [(LS_ELLIPSE, [math.cos(m * math.pi / 4), math.sin(m * math.pi / 4), 0.383, 0.383, 0.0])
             for m in range(1, 9)]
    comps.append((LS_STAR, [0.0, 0.0, 0.514, 0.514 * 0.2, 5.0]))
    return Workload("touching_interfaces_2d", 2, n, -1.7, 1.7, LS_UNION, union_params(comps),
                    KIND_INTERFACE_MU, sigma_in=1.0, sigma_out=3.0, exact="multi",
                    extra={"sol_in": ["exp_68"] * 9, "sol_out": "sinsin_pi"})


def torus_ellipsoid_3d(n: int = 128) -> Workload:
    """Sec. 7.2.4's arbitrarily close interfaces (Table 6): the torus
    (1 - sqrt(x^2 + y^2))^2 + z^2 < 0.4^2 and the ellipsoid x^2/0.36 +
    y^2/0.36 + z^2 < 1, which touch along the circle x^2 + y^2 = 0.36, z = 0;
    box [-1.5, 1.5]^3, Poisson interface problem, sigma_i = 1, sigma_e = 3,
    u = sin^2(2x) cos^2(2y) cos z in the torus, e^z (cos 2x + cos 3y) in the
    ellipsoid, cos x cos y cos z outside."""
    comps = [(LS_TORUS, [1.0, 0.4]), (LS_ELLIPSOID, [0.0, 0.0, 0.0, 0.6, 0.6, 1.0])]
    return Workload("torus_ellipsoid_3d", 3, n, -1.5, 1.5, LS_UNION, union_params(comps),
                    KIND_INTERFACE_MU, sigma_in=1.0, sigma_out=3.0, exact="multi",
                    extra={"sol_in": ["torus_in", "exp_cos3"], "sol_out": "cos3"})


def close_discs_2d(n: int = 128, gap: float = 0.004) -> Workload:
    """Two circles of radius 0.4 a distance `gap` apart across x = 0.0039
    (centres (0.0039 -+ (0.4 + gap/2), 0.013)) in [-1, 1]^2, so that for N
    up to 256 the gap holds no grid node and x-edges across it cross both
    circles; different interior solutions: exp(0.6 x + 0.8 y) in the left
    disc, cos x cosh y in the right one, sin(pi (x+1)/2) sin(pi (y+1)/2)
    outside; Poisson interface problem, sigma_i = 1, sigma_e = 3."""
    c = 0.4 + 0.5 * gap
    comps = [(LS_ELLIPSE, [0.0039 - c, 0.013, 0.4, 0.4, 0.0]),
             (LS_ELLIPSE, [0.0039 + c, 0.013, 0.4, 0.4, 0.0])]
    return Workload("close_discs_2d", 2, n, -1.0, 1.0, LS_UNION, union_params(comps),
                    KIND_INTERFACE_MU, sigma_in=1.0, sigma_out=3.0, exact="multi",
                    extra={"sol_in": ["exp_68", "cos_cosh"], "sol_out": "sinsin_pi"})


def molecule_dirichlet_3d(n: int = 64) -> Workload:
    """3D Dirichlet modified-Helmholtz BVP (kappa = 1) inside a three-atom
    Gaussian-sum surface 0.5 - sum_k exp(-|x - x_k|^2 / 0.4^2) < 0 (atoms at
    (+-0.3, 0, 0) and (0, 0.3, 0.1)), u = e^{x+y+z}/10."""
    return Workload("molecule_dirichlet_3d", 3, n, -1.0, 1.0, LS_MOLECULE,
                    [0.4, 0.5, 3.0, -0.3, 0.0, 0.0, 0.3, 0.0, 0.0, 0.0, 0.3, 0.1],
                    KIND_DIRICHLET, kappa=1.0, exact="exp3")


def wobbly_samples(dim: int, n: int, lo: float, hi: float) -> np.ndarray:
    """Node values of a smooth level-set function that no analytic kind
    describes: 2D (x/0.62)^2 + (y/0.45)^2 + 0.25 sin(3x) sin(4y) - 1, 3D
    (x/0.6)^2 + (y/0.5)^2 + (z/0.45)^2 + 0.2 sin(3x) sin(3y) cos(2z) - 1;
    shape (N+1,)*d, axis d-1 fastest."""
    h = (hi - lo) / n
    x = lo + np.arange(n + 1) * h
    X = np.stack(np.meshgrid(*([x] * dim), indexing="ij"), -1)
    if dim == 2:
        return ((X[..., 0] / 0.62) ** 2 + (X[..., 1] / 0.45) ** 2
                + 0.25 * np.sin(3 * X[..., 0]) * np.sin(4 * X[..., 1]) - 1.0)
    return ((X[..., 0] / 0.6) ** 2 + (X[..., 1] / 0.5) ** 2 + (X[..., 2] / 0.45) ** 2
            + 0.2 * np.sin(3 * X[..., 0]) * np.sin(3 * X[..., 1]) * np.cos(2 * X[..., 2]) - 1.0)


def moving_samples(dim: int, n: int, lo: float, hi: float, t: float) -> np.ndarray:
    """Node values at time t of a moving interface: the wobbly shape of
    wobbly_samples rotated by 0.6 t about the z axis and translated by
    0.08 (sin 2t, cos 3t[, 0]) - (0, 0.08[, 0]), so t = 0 is wobbly_samples
    itself."""
    h = (hi - lo) / n
    x = lo + np.arange(n + 1) * h
    X = np.stack(np.meshgrid(*([x] * dim), indexing="ij"), -1)
    c = np.array([0.08 * math.sin(2 * t), 0.08 * math.cos(3 * t) - 0.08] + [0.0] * (dim - 2))
    th = 0.6 * t
    Y = X - c
    xr = math.cos(th) * Y[..., 0] + math.sin(th) * Y[..., 1]
    yr = -math.sin(th) * Y[..., 0] + math.cos(th) * Y[..., 1]
    if dim == 2:
        return (xr / 0.62) ** 2 + (yr / 0.45) ** 2 + 0.25 * np.sin(3 * xr) * np.sin(4 * yr) - 1.0
    z = Y[..., 2]
    return ((xr / 0.6) ** 2 + (yr / 0.5) ** 2 + (z / 0.45) ** 2
            + 0.2 * np.sin(3 * xr) * np.sin(3 * yr) * np.cos(2 * z) - 1.0)


def moving_interface_2d(n: int = 1024, t: float = 0.0, contrast: float = 10.0) -> Workload:
    """The interface problem of sampled_interface_2d on the moving shape of
    moving_samples at time t (sigma_in/sigma_out = contrast, u_in = sin x cos
    y, u_out = x^2 + y^2: the exact solution holds for every position)."""
    return Workload(f"moving_interface_2d_t{t:g}", 2, n, -1.0, 1.0, LS_GRID, [], KIND_INTERFACE_MU,
                    sigma_in=contrast, sigma_out=1.0, exact="sincos_r2",
                    extra={"samples": moving_samples(2, n, -1.0, 1.0, t)})


def sampled_interface_2d(n: int = 256, contrast: float = 10.0) -> Workload:
    """2D Poisson interface problem whose interface is known only by grid
    samples of a level-set function (wobbly_samples), sigma_in/sigma_out =
    contrast, u_in = sin x cos y, u_out = x^2 + y^2."""
    return Workload("sampled_interface_2d", 2, n, -1.0, 1.0, LS_GRID, [], KIND_INTERFACE_MU,
                    sigma_in=contrast, sigma_out=1.0, exact="sincos_r2",
                    extra={"samples": wobbly_samples(2, n, -1.0, 1.0)})


def sampled_dirichlet_3d(n: int = 64) -> Workload:
    """3D Dirichlet modified-Helmholtz BVP (kappa = 1) inside a surface known
    only by grid samples (wobbly_samples), u = e^{x+y+z}/10."""
    return Workload("sampled_dirichlet_3d", 3, n, -1.0, 1.0, LS_GRID, [], KIND_DIRICHLET,
                    kappa=1.0, exact="exp3", extra={"samples": wobbly_samples(3, n, -1.0, 1.0)})


def star_batch_2d(count: int = 64, seed: int = 5965, sizes=(128, 256, 512, 1024)):
    """Batched star-interface instances: R0~U[0.4,0.6], A~U[0,0.15], k~U{3..7},
    contrast = 10^U[0,3], N ~ U(sizes), drawn in that order per instance."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        r0 = rng.uniform(0.4, 0.6)
        a = rng.uniform(0.0, 0.15)
        k = int(rng.integers(3, 8))
        contrast = 10.0 ** rng.uniform(0.0, 3.0)
        n = int(rng.choice(np.asarray(sizes)))
        out.append(Workload(f"star_{i}", 2, n, -1.0, 1.0, LS_STAR,
                            [0.0, 0.0, r0, a, float(k)], KIND_INTERFACE_MU,
                            sigma_in=contrast, sigma_out=1.0, exact="sincos_r2"))
    return out


def ellipsoid_harmonic_3d(rng: np.random.Generator, n: int = 256,
                          contrast: float = 10.0) -> Workload:
    """Ellipsoid interface with axes ~U[0.3,0.7]^3, contrast 10, and interior
    solution a random sum of 8 harmonic polynomials (amplitudes N(0,1)),
    exterior solution 0."""
    axes = rng.uniform(0.3, 0.7, size=3)
    amps = rng.standard_normal(8)
    return harmonic_ellipsoid_3d(axes, amps, n, contrast)


def harmonic_ellipsoid_3d(axes, amps, n: int, contrast: float = 10.0) -> Workload:
    """The ellipsoid interface problem above with given axes and amplitudes."""
    return Workload("ellipsoid_harmonic_3d", 3, n, -1.0, 1.0, LS_ELLIPSOID,
                    [0.0, 0.0, 0.0, *[float(a) for a in axes]], KIND_INTERFACE_MU,
                    sigma_in=contrast, sigma_out=1.0, exact="harmonic3",
                    extra={"amps": [float(a) for a in amps]})


def warm_start_training_set(seed: int, geometries: int, draws: int):
    """(axes, amplitudes) pairs of the learned-start training solves: `geometries`
    ellipsoids (axes ~U[0.3,0.7]^3), each with `draws` amplitude vectors
    (N(0,1)^8), all from one seeded generator."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(geometries):
        axes = rng.uniform(0.3, 0.7, size=3)
        out.append((axes, [rng.standard_normal(8) for _ in range(draws)]))
    return out


def wave_field(seed: int, terms: int = 8):
    """A fixed harmonic field sum_k a_k exp(p_k . x) cos(q_k . x + c_k) with
    |p_k| = |q_k| and p_k orthogonal to q_k (so each term is harmonic), drawn
    once from a seeded generator: a_k ~ N(0,1), |p_k| ~ U[0.5, 1.5], directions
    uniform, c_k ~ U[0, 2 pi).  Returns (P, Q, a, c) of shapes (terms, 3),
    (terms, 3), (terms,), (terms,)."""
    rng = np.random.default_rng(seed)
    P, Q, A, C = [], [], [], []
    for _ in range(terms):
        u = rng.standard_normal(3)
        u /= np.linalg.norm(u)
        v = rng.standard_normal(3)
        v -= (v @ u) * u
        v /= np.linalg.norm(v)
        s = rng.uniform(0.5, 1.5)
        P.append(s * u)
        Q.append(s * v)
        A.append(rng.standard_normal())
        C.append(rng.uniform(0.0, 2.0 * np.pi))
    return np.array(P), np.array(Q), np.array(A), np.array(C)


def _sol_waves(seed):
    P, Q, A, C = wave_field(seed)

    def u(X):
        return np.exp(X @ P.T) * np.cos(X @ Q.T + C) @ A

    def g(X):
        e = np.exp(X @ P.T) * A
        cs = np.cos(X @ Q.T + C)
        sn = np.sin(X @ Q.T + C)
        return (e * cs) @ P - (e * sn) @ Q

    lap = lambda X: np.zeros(X.shape[:-1])
    return u, g, lap


def wave_ellipsoid_3d(axes, n: int, contrast: float = 10.0) -> Workload:
    """3D interface problem of the learned start: an ellipsoid with the given
    axes in [-1, 1]^3, sigma_in/sigma_out = contrast, u_in and u_out two fixed
    harmonic fields (wave_field, seeds 5968 and 5969), outer Dirichlet data
    from u_out.  The geometry varies from problem to problem, the fields do
    not; the fields are not polynomials (the method is not exact for them),
    and with u_out != 0 the density [d_n u] is not a multiple of the flux jump
    g2."""
    return Workload("wave_ellipsoid_3d", 3, n, -1.0, 1.0, LS_ELLIPSOID,
                    [0.0, 0.0, 0.0, *[float(a) for a in axes]], KIND_INTERFACE_MU,
                    sigma_in=contrast, sigma_out=1.0, exact="waves_io",
                    extra={"seed_in": 5968, "seed_out": 5969})


def ellipsoid_axes(seed: int, count: int):
    """`count` ellipsoid axis triples ~U[0.3, 0.7]^3 from one seeded generator."""
    rng = np.random.default_rng(seed)
    return [rng.uniform(0.3, 0.7, size=3) for _ in range(count)]


def sine_grid_rhs(dim: int, n: int, seed: int) -> np.ndarray:
    """Seeded random interior right-hand side for box-solve tests, shape (N+1,)*d
    with zero boundary layer."""
    rng = np.random.default_rng(seed)
    r = np.zeros((n + 1,) * dim)
    inner = tuple(slice(1, n) for _ in range(dim))
    r[inner] = rng.standard_normal((n - 1,) * dim)
    return r
