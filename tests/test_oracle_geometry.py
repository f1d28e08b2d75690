"""Pins of the oracle's geometry (Sec. 5.1, 5.2): intersections, normals,
surface decomposition, irregular nodes, closest primary points."""
import math

import numpy as np
import scipy.optimize

import workloads as W
from oracle import correction as CR
from oracle import geometry as G
from oracle import kfbi as K
from oracle import levelset as LS


def test_circle_intersections_closed_form():
    """For a circle x^2+y^2 = R^2 the e_x-line intersections are +-sqrt(R^2 - y^2)
    and the normal is x/R (closed form)."""
    R = 0.553
    w = W.Workload("circ", 2, 40, -1.0, 1.0, W.LS_STAR, [0.0, 0.0, R, 0.0, 3.0],
                   W.KIND_DIRICHLET, exact="exp_sin", cos_alpha=0.5)
    g = G.Grid(2, w.n, w.lo, w.h)
    ins = G.classify(g, w.ls_kind, w.ls_params)
    s = G.surface_points(g, w.ls_kind, w.ls_params, 0.5, ins)
    f0 = s.family == 0
    y = s.x[f0, 1]
    xr = np.sqrt(R * R - y * y)
    assert np.abs(np.abs(s.x[f0, 0]) - xr).max() < 1e-14
    assert np.abs(s.n[f0] - s.x[f0] / R).max() < 1e-13
    # count: lines y = lo + j h with |y| < R and |n_x| = sqrt(1 - y^2/R^2) > 0.5 carry two points
    ys = g.coord(np.arange(w.n + 1))
    expect = 2 * int(np.sum((np.abs(ys) < R) & (np.sqrt(np.maximum(0, 1 - ys ** 2 / R ** 2)) > 0.5)))
    assert int(f0.sum()) == expect


def test_roots_match_brentq_and_lie_between_nodes():
    w = W.flower_interface_2d(128)
    g = G.Grid(2, w.n, w.lo, w.h)
    ins = G.classify(g, w.ls_kind, w.ls_params)
    s = G.surface_points(g, w.ls_kind, w.ls_params, w.cosa(), ins)
    rng = np.random.default_rng(2)
    for i in rng.choice(s.nb, 40, replace=False):
        r = s.family[i]
        x0 = s.x[i].copy()
        x0[r] = g.coord(s.edge[i])

        def f(t):
            X = x0.copy()
            X[r] = x0[r] + t
            return LS.H(w.ls_kind, w.ls_params, X[None])[0]
        t = scipy.optimize.brentq(f, 0.0, g.h, xtol=1e-18, rtol=1e-15)
        assert abs((s.x[i, r] - x0[r]) - t) < 1e-14
        assert abs(LS.H(w.ls_kind, w.ls_params, s.x[i][None])[0]) < 1e-13
    assert np.all(np.abs(np.linalg.norm(s.n, axis=1) - 1) < 1e-14)
    assert np.all(np.abs(s.n[np.arange(s.nb), s.family]) > w.cosa())


def test_irregular_nodes_brute_force():
    w = W.ellipse_dirichlet_2d(32)
    g = G.Grid(2, w.n, w.lo, w.h)
    ins = G.classify(g, w.ls_kind, w.ls_params)
    for order in (2, 4):
        irr = CR.irregular_nodes(ins, order)
        for i in range(1, w.n):
            for j in range(1, w.n):
                cls = set()
                for a in (-1, 0, 1):
                    for b in (-1, 0, 1):
                        if order == 2 and a != 0 and b != 0:
                            continue
                        cls.add(bool(ins[i + a, j + b]))
                assert irr[i, j] == (len(cls) == 2)
        assert not irr[0].any() and not irr[:, 0].any()


def test_closest_primary_brute_force():
    P = K.Problem(W.ellipse_dirichlet_2d(64))
    x = P.grid.coord(P.cnode_idx)
    pts = P.surf.x
    for q, own in zip(x, P.cnode_owner):
        d2 = np.sum((pts - q) ** 2, 1)
        best = np.nonzero(d2 <= d2.min() + CR.TIE_EPS * P.h ** 2)[0].min()
        assert own == best


def test_collocation_stencil_rules():
    """Dirichlet/Neumann points are DOFs of the reference family on distinct grid
    lines near p; PDE points are round(p) + offsets."""
    P = K.Problem(W.flower_interface_2d(256))
    s = P.surf
    for i in range(P.nb):
        m = P.stencil_axis[i]
        dd = P.dir_idx[i]
        assert np.all(s.family[dd] == m)
        t = 1 - m
        lines = np.round((s.x[dd, t] - P.grid.lo) / P.h).astype(int)
        assert len(set(lines.tolist())) == len(dd)
        assert np.abs(s.x[dd, t] - s.x[i, t]).max() <= 4.5 * P.h
        assert set(P.neu_idx[i].tolist()) <= set(dd.tolist())
        n0 = np.floor((s.x[i] - P.grid.lo) / P.h + 0.5).astype(int)
        assert np.all(P.pde_nodes[i][0] == n0)


def test_gauss_lemma_constant_correction():
    """P3: with a = 1, b = 0, kappa = 0 the collocation gives C = 1 exactly and the
    corrected scheme's solution is the indicator of Omega_h."""
    P = K.Problem(W.ellipse_dirichlet_2d(64))
    coef = P.collocation(np.ones(P.nb), np.zeros(P.nb))
    cv = P.c_values(coef)
    assert np.abs(cv - 1).max() < 1e-12
    u, _, _, _ = P.potential(np.ones(P.nb), np.zeros(P.nb))
    inner = tuple(slice(1, P.n) for _ in range(2))
    assert np.abs(u[inner] - P.inside[inner]).max() < 1e-11


def test_molecule_single_atom_is_a_sphere():
    """A one-atom Gaussian-sum surface level - exp(-|x - c|^2 / r^2) = 0 is the
    sphere |x - c| = r sqrt(-ln level): the same node classes, DOFs (points,
    families) and normals as the sphere written as an ellipsoid with equal
    axes, up to the root tolerance."""
    r, level, c = 0.45, 0.4, (0.03, -0.02, 0.05)
    R = r * math.sqrt(-math.log(level))
    g = G.Grid(3, 24, -1.0, 2.0 / 24)
    mol = [r, level, 1.0, *c]
    sph = [*c, R, R, R]
    ins_m = G.classify(g, W.LS_MOLECULE, mol)
    ins_s = G.classify(g, W.LS_ELLIPSOID, sph)
    assert np.array_equal(ins_m, ins_s)
    sm = G.surface_points(g, W.LS_MOLECULE, mol, 0.4, ins_m)
    ss = G.surface_points(g, W.LS_ELLIPSOID, sph, 0.4, ins_s)
    assert sm.nb == ss.nb and sm.nb > 100
    assert np.array_equal(sm.family, ss.family)
    assert np.abs(sm.x - ss.x).max() < 1e-13
    assert np.abs(sm.n - ss.n).max() < 1e-12
    # points on the sphere, normals radial
    d = sm.x - np.asarray(c)
    assert np.abs(np.linalg.norm(d, axis=1) - R).max() < 1e-13
    assert np.abs(sm.n - d / R).max() < 1e-12


def test_molecule_gradient_central_differences():
    """The analytic gradient of a three-atom surface against central finite
    differences of H (step 1e-5: error O(1e-10) for these Gaussians)."""
    w = W.molecule_dirichlet_3d(64)
    rng = np.random.default_rng(7)
    X = rng.uniform(-0.8, 0.8, size=(200, 3))
    g = LS.grad_H(w.ls_kind, w.ls_params, X)
    e = 1e-5
    fd = np.zeros_like(X)
    for k in range(3):
        dx = np.zeros(3)
        dx[k] = e
        fd[:, k] = (LS.H(w.ls_kind, w.ls_params, X + dx) - LS.H(w.ls_kind, w.ls_params, X - dx)) / (2 * e)
    assert np.abs(g - fd).max() < 1e-8
    # far from every atom H -> level (the sum of Gaussians vanishes)
    far = LS.H(w.ls_kind, w.ls_params, np.array([[40.0, 0.0, 0.0]]))[0]
    assert far == w.ls_params[1]


def test_root_iteration_stops_by_its_tolerance():
    """The root iteration's stopping rule (|ds| <= 1e-15 N h, about the FP64
    spacing of a coordinate in the box) is met, not the step limit: on every
    sign-changing edge of the flower and of a grid-sampled shape at 512^2
    the roots take at most 4 steps on average and stop before the limit, and
    sampled roots agree with brentq on the interpolant to 1e-14.  (A
    tolerance of 1e-15 h lies below the rounding noise of the Newton steps:
    roots then took 8-11 steps on average and some ran to the limit.)"""
    rng = np.random.default_rng(5)
    for w in (W.flower_interface_2d(512), W.moving_interface_2d(512, 0.15)):
        g = G.Grid(2, w.n, w.lo, w.h)
        p = LS.params(w)
        xs = g.coord(np.arange(w.n + 1))
        X, Y = np.meshgrid(xs, xs, indexing="ij")
        P = np.stack([X.ravel(), Y.ravel()], -1)
        Hn = LS.H_iface(w.ls_kind, p, 0, P).reshape(w.n + 1, w.n + 1)
        i, j = np.nonzero((Hn[:, :-1] < 0) != (Hn[:, 1:] < 0))
        x0 = np.stack([xs[i], xs[j]], -1)
        steps = []
        s = G.find_roots(g, w.ls_kind, p, x0, 1, steps=steps)
        steps = np.asarray(steps)
        assert len(steps) == len(x0) > 500
        assert steps.mean() <= 4.0 and steps.max() < G.ROOT_MAX_IT, (steps.mean(), steps.max())
        assert np.all((s >= 0.0) & (s <= g.h))
        for k in rng.choice(len(x0), 20, replace=False):
            def f(t):
                Xk = x0[k].copy()
                Xk[1] = x0[k, 1] + t
                return LS.H_iface(w.ls_kind, p, 0, Xk[None])[0]
            t = scipy.optimize.brentq(f, 0.0, g.h, xtol=1e-18, rtol=1e-15)
            assert abs(s[k] - t) < 1e-14, (k, s[k], t)
