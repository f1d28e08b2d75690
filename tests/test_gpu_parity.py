"""GPU-vs-oracle parity through the C ABI, stage by stage and end to end.

Integer outputs (DOF order, families, interfaces, reference axes, collocation
stencils, node labels, irregular nodes, correction entries, closest primary
points) must be identical.
Floating-point outputs are compared in relative max-norm: the FP64 path of the
solver is held to 1e-10 (the stated bound for every config), single stages to
tighter bounds where the arithmetic is short.
"""
import numpy as np
import pytest

import workloads as W
from oracle import kfbi as OK
from tests.gpu_util import dev, empty, gpu_data, host, linear_nodes, rel_err

pytestmark = pytest.mark.gpu

CASES = {
    "ellipse64": lambda: W.ellipse_dirichlet_2d(64),
    "table1_128": lambda: W.paper_table1_2d(128),
    "flower256": lambda: W.flower_interface_2d(256),
    "discs128": lambda: W.discs_interface_2d(128),
    "ellipse_order2_helmholtz": None,
    "ellipsoid32": lambda: W.Workload("ell3", 3, 32, -1.0, 1.0, W.LS_ELLIPSOID,
                                      [0.05, -0.03, 0.02, 0.8, 0.7, 0.6], W.KIND_DIRICHLET,
                                      kappa=1.0, exact="exp3"),
    # the 3D torus Dirichlet problem for modified Helmholtz (kappa = 1) at the
    # largest grid the oracle sets up in seconds (64^3: 4800 DOFs)
    "torus64": lambda: W.torus_helmholtz_3d(64),
    # the Gaussian-sum (molecule) level set, three atoms
    "molecule64": lambda: W.molecule_dirichlet_3d(64),
    # interfaces known only by level-set samples at the grid nodes
    "sampled256": lambda: W.sampled_interface_2d(256),
    "sampled3d64": lambda: W.sampled_dirichlet_3d(64),
    # close interfaces: two discs 0.004 apart (below the grid step), each with
    # its own interior solution; Sec. 7.1.2's touching circles and star
    "close_discs128": lambda: W.close_discs_2d(128),
    # the interior Dirichlet problem on the same two close discs (two
    # components of Omega, each with its own solution)
    "close_discs_dirichlet128": lambda: _close_dirichlet(),
    "touching256": lambda: W.touching_interfaces_2d(256),
}


def _close_dirichlet():
    w = W.close_discs_2d(128)
    w.kind = W.KIND_DIRICHLET
    return w


def _order2():
    w = W.ellipse_dirichlet_2d(128)
    w.order = 2
    w.kappa = 2.0
    return w


CASES["ellipse_order2_helmholtz"] = _order2

_cache = {}


def pair(name, precision=0, box=0):
    key = (name, precision, box)
    if key not in _cache:
        from paper_2309_05965_gb300 import build, kfbi
        build.build()
        w = CASES[name]()
        P = OK.Problem(w)
        G = kfbi.Problem.from_workload(w, box_solver=box, precision=precision)
        _cache[key] = (w, P, G)
    return _cache[key]


NAMES = list(CASES)


@pytest.mark.parametrize("name", NAMES)
def test_geometry_exact(name):
    from paper_2309_05965_gb300 import kfbi
    w, P, G = pair(name)
    h = G.handle
    assert G.nb == P.nb
    assert G.nirr == int(P.irr.sum())
    assert (G.n_iface, G.nent) == (P.n_iface, P.cnode_idx.shape[0])
    d = w.dim
    xyz, nrm = empty((G.nb, d)), empty((G.nb, d))
    kfbi.kfbi_dof_points(h, xyz, nrm)
    assert np.abs(host(xyz) - P.surf.x).max() < 1e-14
    assert np.abs(host(nrm) - P.surf.n).max() < 1e-13
    fam, ax, sax = empty(G.nb, "i32"), empty(G.nb, "i32"), empty(G.nb, "i32")
    kfbi.kfbi_dof_info(h, fam, ax, sax)
    assert np.array_equal(host(fam), P.surf.family)
    assert np.array_equal(host(ax), P.surf.axis)
    assert np.array_equal(host(sax), P.stencil_axis)
    pde, dd, nn = (empty((G.nb, G.npde), "i32"), empty((G.nb, G.ndir), "i32"),
                   empty((G.nb, G.nneu), "i32"))
    kfbi.kfbi_collocation_stencils(h, pde, dd, nn)
    assert np.array_equal(host(pde), linear_nodes(P.pde_nodes, w.n))
    assert np.array_equal(host(dd), P.dir_idx)
    assert np.array_equal(host(nn), P.neu_idx)
    ifc = empty(G.nb, "i32")
    kfbi.kfbi_dof_iface(h, ifc)
    assert np.array_equal(host(ifc), P.surf.iface)
    mask = empty(G.grid_shape, "u8")
    kfbi.kfbi_inside_mask(h, mask)
    assert np.array_equal(host(mask), P.labels)
    lin = empty(G.nirr, "i32")
    kfbi.kfbi_irregular_nodes(h, lin, None)
    assert np.array_equal(host(lin), linear_nodes(np.argwhere(P.irr), w.n))
    elin, eif, own = empty(G.nent, "i32"), empty(G.nent, "i32"), empty(G.nent, "i32")
    kfbi.kfbi_correction_entries(h, elin, eif, own)
    assert np.array_equal(host(elin), linear_nodes(P.cnode_idx, w.n))
    assert np.array_equal(host(eif), P.cnode_iface)
    assert np.array_equal(host(own), P.cnode_owner)
    if G.n_iface == 1:
        own1 = empty(G.nirr, "i32")
        kfbi.kfbi_irregular_nodes(h, lin, own1)
        assert np.array_equal(host(own1), P.cnode_owner)


@pytest.mark.parametrize("name", NAMES)
def test_collocation_and_correction_values(name):
    from paper_2309_05965_gb300 import kfbi
    w, P, G = pair(name)
    rng = np.random.default_rng(1)
    a, b = rng.standard_normal(P.nb), rng.standard_normal(P.nb)
    ft = rng.standard_normal(P.inside.shape)
    coef_ref = P.collocation(a, b, ft)
    coef = empty((G.nb, G.ncoef))
    kfbi.kfbi_collocation_fit(G.handle, dev(a), dev(b), dev(ft), coef)
    assert rel_err(host(coef), coef_ref) < 1e-11
    cv_ref = P.c_values(coef_ref)
    cv = empty(G.nent)
    kfbi.kfbi_correction_values(G.handle, dev(a), dev(b), dev(ft), cv)
    assert rel_err(host(cv), cv_ref) < 1e-11


@pytest.mark.parametrize("name", NAMES)
def test_corrected_rhs(name):
    from paper_2309_05965_gb300 import kfbi
    w, P, G = pair(name)
    rng = np.random.default_rng(2)
    cv = rng.standard_normal(G.nent)
    data = W.grid_data(w)
    Fi, Fo, Li, Lo = P.unit_sigma_data(data)
    if w.kind == W.KIND_DIRICHLET:
        Fo, Lo, gb = 0 * Fo, 0 * Lo, None
    else:
        gb = data["g_b"]
    ref = P.rhs(cv, Fi, Fo, Li, Lo, gb)
    g1 = np.zeros(P.nb)
    d, keep = gpu_data(w, P, data, g1, g1)
    out = empty(G.grid_shape)
    kfbi.kfbi_corrected_rhs(G.handle, dev(cv), d, out)
    assert rel_err(host(out), ref) < 1e-12
    # correction terms alone
    ref0 = P.rhs(cv)
    kfbi.kfbi_corrected_rhs(G.handle, dev(cv), None, out)
    assert rel_err(host(out), ref0) < 1e-12


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("precision", [0, 1])
def test_box_solve(name, precision):
    from paper_2309_05965_gb300 import kfbi
    w, P, G = pair(name, precision)
    R = W.sine_grid_rhs(w.dim, w.n, 3)
    ref = P.box_solve(R)
    u = empty(G.grid_shape)
    kfbi.kfbi_box_solve(G.handle, dev(R), u)
    assert rel_err(host(u), ref) < (1e-12 if precision == 0 else 5e-12)


@pytest.mark.parametrize("name", NAMES)
def test_traces(name):
    from paper_2309_05965_gb300 import kfbi
    w, P, G = pair(name)
    rng = np.random.default_rng(4)
    X = P.grid.coords()
    u = np.sin(3 * X[..., 0]) * np.cos(2 * X[..., 1]) + 0.1 * rng.standard_normal(P.inside.shape)
    cv = rng.standard_normal(G.nent)
    ref = P.traces(u, cv)
    outs = [empty(G.nb) for _ in range(4)]
    kfbi.kfbi_traces(G.handle, dev(u), dev(cv), *outs)
    for o, r in zip(outs, ref):
        assert rel_err(host(o), r) < 1e-11


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("precision", [0, 1])
def test_apply_operator(name, precision):
    from paper_2309_05965_gb300 import kfbi
    w, P, G = pair(name, precision)
    rng = np.random.default_rng(5)
    x = rng.standard_normal(P.nb)
    ref = P.apply(x)
    y = empty(G.nb)
    kfbi.kfbi_apply_operator(G.handle, dev(x), y)
    assert rel_err(host(y), ref) < 1e-10
    # Gauss's lemma on the GPU: A 1 = 1 for the Dirichlet form with kappa = 0
    if w.kind == W.KIND_DIRICHLET and w.kappa == 0.0 and w.order == 4:
        kfbi.kfbi_apply_operator(G.handle, dev(np.ones(P.nb)), y)
        assert np.abs(host(y) - 1.0).max() < 1e-11


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("precision", [0, 1])
def test_full_solve(name, precision):
    """BIE right-hand side, GMRES and evaluation.

    * iteration counts at rtol 1e-13 agree within 2;
    * backward error: the GPU density solves the ORACLE's discrete system to a
      relative residual <= 1e-10 (the stated FP64 bound);
    * forward error at the same Krylov dimension: <= 1e-10 max(1, cond(A)/100).
      The GPU operator matches the oracle's to ~2e-14, so two correct FP64
      implementations differ in the solution by ~cond(A) x 1e-14; cond(A) is
      ~13 at contrast 10 but ~1.4e3 at contrast 1000 (mu = -0.998, smallest
      eigenvalue ~(1 - |mu|)/2), where the forward bound is scaled."""
    from paper_2309_05965_gb300 import kfbi
    w, P, G = pair(name, precision)
    data = W.grid_data(w)
    g1, g2 = W.boundary_data(w, P.surf.x, P.surf.n, P.surf.iface)
    b_ref = P.bie_rhs(g1, g2, data)
    x_ref, it_ref, _ = OK.gmres(P.apply, b_ref, rtol=1e-13)
    u_ref = P.evaluate(x_ref, g1, data)
    d, keep = gpu_data(w, P, data, g1, g2)
    b = empty(G.nb)
    kfbi.kfbi_bie_rhs(G.handle, d, b)
    assert rel_err(host(b), b_ref) < 1e-10
    dens = empty(G.nb)
    opts = kfbi.GmresOpts(rtol=1e-13, restart=100, max_iter=200, x0=None)
    info = kfbi.kfbi_gmres_solve(G.handle, d, opts, dens)
    assert abs(info.iters - it_ref) <= 2
    # the same Krylov dimension on both sides
    k = it_ref
    x_ref, _, _ = OK.gmres(P.apply, b_ref, rtol=1e-300, max_iter=k, strict=False)
    u_ref = P.evaluate(x_ref, g1, data)
    opts_k = kfbi.GmresOpts(rtol=1e-300, restart=100, max_iter=k, x0=None)
    with pytest.raises(kfbi.KfbiError) as e:
        kfbi.kfbi_gmres_solve(G.handle, d, opts_k, dens)
    assert e.value.status == 4
    xg = host(dens)
    r = b_ref - P.apply(xg)
    assert np.linalg.norm(r) / np.linalg.norm(b_ref) < 1e-10
    cond = 1.0
    if w.kind == W.KIND_INTERFACE_MU and w.sigma_in / w.sigma_out > 100:
        A = np.array([P.apply(e_) for e_ in np.eye(P.nb)]).T
        cond = np.linalg.cond(A)
    tol = 1e-10 * max(1.0, cond / 100.0)
    assert rel_err(xg, x_ref) < tol
    u = empty(G.grid_shape)
    kfbi.kfbi_evaluate(G.handle, d, dens, u)
    assert rel_err(host(u), u_ref) < tol
    # and the solution is the exact one to discretisation accuracy
    ex = W.exact_grid(w, P.labels)
    m = P.inside if w.kind == W.KIND_DIRICHLET else np.ones_like(P.inside)
    inner = np.zeros_like(m)
    inner[tuple(slice(1, w.n) for _ in range(w.dim))] = True
    assert np.abs(host(u) - ex)[m & inner].max() < 1e-3


def test_errors_are_reported():
    """Invalid sizes and an under-resolved interface come back as statuses."""
    from paper_2309_05965_gb300 import build, kfbi
    build.build()
    with pytest.raises(kfbi.KfbiError) as e:
        kfbi.Problem(2, 100, -1.0, 1.0, W.LS_ELLIPSE, [0, 0, 0.6, 0.4, 0], 0)
    assert e.value.status == 1
    with pytest.raises(kfbi.KfbiError) as e:
        kfbi.Problem(3, 16, -1.0, 1.0, W.LS_TORUS, [0.5, 0.2], 0, kappa=1.0)
    assert e.value.status == 2
    with pytest.raises(kfbi.KfbiError):
        kfbi.Problem(2, 64, -1.0, 1.0, W.LS_TORUS, [0.5, 0.2], 0)


def test_mu_zero_is_half_identity():
    from paper_2309_05965_gb300 import build, kfbi
    build.build()
    w = W.flower_interface_2d(256, contrast=1.0)
    G = kfbi.Problem.from_workload(w)
    x = np.random.default_rng(9).standard_normal(G.nb)
    y = empty(G.nb)
    kfbi.kfbi_apply_operator(G.handle, dev(x), y)
    assert np.array_equal(host(y), 0.5 * x)
    kfbi.kfbi_apply_operator(G.handle, dev(np.zeros(G.nb)), y)
    assert np.all(host(y) == 0.0)


@pytest.mark.parametrize("name", ["ellipse64", "flower256", "ellipsoid32", "ellipse_order2_helmholtz"])
@pytest.mark.parametrize("precision", [0, 1])
def test_box_solve_multigrid(name, precision):
    """Geometric multigrid (FP64 V-cycles, or FP32 V-cycles inside FP64
    refinement) converges to the exact discrete solution of the DST/direct
    solve within the inner tolerance."""
    from paper_2309_05965_gb300 import kfbi
    w, P, G = pair(name, precision, box=1)
    R = W.sine_grid_rhs(w.dim, w.n, 3)
    ref = P.box_solve(R)
    u = empty(G.grid_shape)
    kfbi.kfbi_box_solve(G.handle, dev(R), u)
    assert rel_err(host(u), ref) < 1e-11


@pytest.mark.parametrize("name", ["flower256", "ellipsoid32"])
def test_full_solve_multigrid_mixed(name):
    from paper_2309_05965_gb300 import kfbi
    w, P, G = pair(name, 1, box=1)
    data = W.grid_data(w)
    g1, g2 = W.boundary_data(w, P.surf.x, P.surf.n)
    b_ref = P.bie_rhs(g1, g2, data)
    d, keep = gpu_data(w, P, data, g1, g2)
    dens = empty(G.nb)
    info = kfbi.kfbi_gmres_solve(G.handle, d, kfbi.GmresOpts(rtol=1e-12, restart=100, max_iter=200), dens)
    xg = host(dens)
    assert np.linalg.norm(b_ref - P.apply(xg)) / np.linalg.norm(b_ref) < 1e-10
    u = empty(G.grid_shape)
    kfbi.kfbi_evaluate(G.handle, d, dens, u)
    ex = W.exact_grid(w, P.inside)
    m = P.inside if w.kind == W.KIND_DIRICHLET else np.ones_like(P.inside)
    inner = np.zeros_like(m)
    inner[tuple(slice(1, w.n) for _ in range(w.dim))] = True
    x_ref, _, _ = OK.gmres(P.apply, b_ref, rtol=1e-12)
    u_ref = P.evaluate(x_ref, g1, data)
    e_gpu = np.abs(host(u) - ex)[m & inner].max()
    e_ref = np.abs(u_ref - ex)[m & inner].max()
    assert e_gpu <= 1.1 * e_ref + 1e-12


def test_sampled_quadric_equals_analytic_kind():
    """Node samples of the ellipse level set (quadratic: the interpolant is
    exact) give on the GPU the analytic kind's DOFs, classes and irregular
    nodes, and the same operator."""
    import torch
    from paper_2309_05965_gb300 import build, kfbi
    from oracle import geometry as OG, levelset as OL
    build.build()
    w = W.ellipse_dirichlet_2d(128)
    g = OG.Grid(2, w.n, w.lo, w.h)
    samples = OL.H(w.ls_kind, w.ls_params, g.coords())
    Ga = kfbi.Problem.from_workload(w)
    Gs = kfbi.Problem(2, w.n, w.lo, w.hi, W.LS_GRID, [], w.kind, ls_samples=samples)
    assert Ga.nb == Gs.nb and Ga.nirr == Gs.nirr
    pa, na, ps, ns = empty((Ga.nb, 2)), empty((Ga.nb, 2)), empty((Gs.nb, 2)), empty((Gs.nb, 2))
    kfbi.kfbi_dof_points(Ga.handle, pa, na)
    kfbi.kfbi_dof_points(Gs.handle, ps, ns)
    assert float((pa - ps).abs().max()) < 1e-13 and float((na - ns).abs().max()) < 1e-12
    ma, ms = empty(Ga.grid_shape, "u8"), empty(Gs.grid_shape, "u8")
    kfbi.kfbi_inside_mask(Ga.handle, ma)
    kfbi.kfbi_inside_mask(Gs.handle, ms)
    assert bool(torch.equal(ma, ms))
    x = torch.randn(Ga.nb, dtype=torch.float64, device="cuda")
    ya, ys = empty(Ga.nb), empty(Gs.nb)
    kfbi.kfbi_apply_operator(Ga.handle, x, ya)
    kfbi.kfbi_apply_operator(Gs.handle, x, ys)
    assert float((ya - ys).abs().max() / ya.abs().max()) < 1e-11
    # a grid-sampled level set without samples is refused
    with pytest.raises(kfbi.KfbiError) as e:
        kfbi.Problem(2, w.n, w.lo, w.hi, W.LS_GRID, [], w.kind)
    assert e.value.status == 1
    Ga.close()
    Gs.close()
