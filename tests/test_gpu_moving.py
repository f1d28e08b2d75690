"""Moving interfaces (the level-set method of the paper's closing remarks):
kfbi_update_levelset gives a problem a new interface on the same grid.

* After an update, the problem is the one a fresh kfbi_create_problem builds
  for the new interface: sizes, DOF points and interfaces, side labels,
  stencils and correction entries identical; the operator, the BIE
  right-hand side and a full solve bit-identical.  Covered: a grid-sampled
  shape moving over several time steps (2D 128^2, 3D 64^3), changes of kind
  (analytic ellipse -> samples -> two close discs with their own solutions
  -> back), and the general interface kind (its second side operator is
  updated with it).
* A moving interface problem solved at each of its positions is the exact
  solution to discretisation accuracy.
* At 1024^2, where a set-up needs several arena chunks, updates between two
  shapes of different size equal fresh creates, bit for bit.
* An invalid level set (a kind of the other dimension, a non-finite
  sample) is refused with KFBI_ERR_ARG, and a valid update afterwards works.
"""
import numpy as np
import pytest

import workloads as W
from tests.gpu_util import dev, empty, gpu_data, host

pytestmark = pytest.mark.gpu


def _snapshot(G, w):
    """Every integer query and the operator, right-hand side and solution."""
    from paper_2309_05965_gb300 import kfbi
    h, d = G.handle, w.dim
    out = {"sizes": (G.nb, G.nirr, G.nent, G.n_iface)}
    xyz, nrm = empty((G.nb, d)), empty((G.nb, d))
    kfbi.kfbi_dof_points(h, xyz, nrm)
    ifc = empty(G.nb, "i32")
    kfbi.kfbi_dof_iface(h, ifc)
    lab = empty(G.grid_shape, "u8")
    kfbi.kfbi_inside_mask(h, lab)
    pde, dd, nn = (empty((G.nb, G.npde), "i32"), empty((G.nb, G.ndir), "i32"),
                   empty((G.nb, G.nneu), "i32"))
    kfbi.kfbi_collocation_stencils(h, pde, dd, nn)
    elin, eif, own = empty(G.nent, "i32"), empty(G.nent, "i32"), empty(G.nent, "i32")
    kfbi.kfbi_correction_entries(h, elin, eif, own)
    for k, v in (("x", xyz), ("n", nrm), ("iface", ifc), ("labels", lab), ("pde", pde),
                 ("dir", dd), ("neu", nn), ("elin", elin), ("eif", eif), ("own", own)):
        out[k] = host(v)
    nx = 2 * G.nb if w.kind == W.KIND_INTERFACE_GENERAL else G.nb
    x = np.random.default_rng(3).standard_normal(nx)
    y = empty(nx)
    kfbi.kfbi_apply_operator(h, dev(x), y)
    out["Ax"] = host(y)
    g1, g2 = W.boundary_data(w, out["x"], out["n"], out["iface"])
    d_, keep = gpu_data(w, None, W.grid_data(w), g1, g2)
    b = empty(nx)
    kfbi.kfbi_bie_rhs(h, d_, b)
    out["b"] = host(b)
    dens = empty(nx)
    info = kfbi.kfbi_gmres_solve(h, d_, kfbi.GmresOpts(rtol=1e-10, restart=100, max_iter=200), dens)
    u = empty(G.grid_shape)
    kfbi.kfbi_evaluate(h, d_, dens, u)
    out["iters"] = info.iters
    out["u"] = host(u)
    e = np.abs(out["u"] - W.exact_grid(w, out["labels"]))
    m = np.zeros(e.shape, dtype=bool)
    m[tuple(slice(1, w.n) for _ in range(w.dim))] = True
    if w.kind == W.KIND_DIRICHLET:
        m &= out["labels"] > 0
    out["err"] = float(e[m].max())
    return out


def _same(a, b):
    assert a["sizes"] == b["sizes"]
    for k in a:
        if k in ("sizes", "iters", "err"):
            continue
        assert np.array_equal(a[k], b[k]), k
    assert a["iters"] == b["iters"]


def _ls_of(w):
    return w.ls_kind, w.ls_params, w.extra.get("samples")


def _moving(dim, n, t):
    if dim == 2:
        return W.moving_interface_2d(n, t)
    return W.Workload(f"moving3_{t}", 3, n, -1.0, 1.0, W.LS_GRID, [], W.KIND_DIRICHLET, kappa=1.0,
                      exact="exp3", extra={"samples": W.moving_samples(3, n, -1.0, 1.0, t)})


@pytest.mark.parametrize("dim,n", [(2, 128), (3, 64)])
def test_update_equals_fresh_create_moving(dim, n):
    from paper_2309_05965_gb300 import build, kfbi
    build.build()
    w0 = _moving(dim, n, 0.0)
    G = kfbi.Problem.from_workload(w0, precision=kfbi.MIXED)
    for t in (0.4, 0.8, 1.2):
        w = _moving(dim, n, t)
        G.update_levelset(*_ls_of(w))
        F = kfbi.Problem.from_workload(w, precision=kfbi.MIXED)
        a, b = _snapshot(G, w), _snapshot(F, w)
        _same(a, b)
        F.close()
        assert a["err"] < (1e-6 if dim == 2 else 1e-3), (t, a["err"])
    G.close()


def test_update_across_kinds_and_interfaces():
    """ellipse (one interface) -> samples -> two discs 0.004 apart with their
    own solutions (several interfaces) -> the ellipse again."""
    from paper_2309_05965_gb300 import build, kfbi
    build.build()
    n = 128
    ell = W.Workload("ell", 2, n, -1.0, 1.0, W.LS_ELLIPSE, [0.03, -0.02, 0.62, 0.45, 0.3],
                     W.KIND_INTERFACE_MU, sigma_in=1.0, sigma_out=3.0, exact="multi",
                     extra={"sol_in": ["exp_68"], "sol_out": "sinsin_pi"})
    smp = W.Workload("smp", 2, n, -1.0, 1.0, W.LS_GRID, [], W.KIND_INTERFACE_MU,
                     sigma_in=1.0, sigma_out=3.0, exact="multi",
                     extra={"sol_in": ["exp_68"], "sol_out": "sinsin_pi",
                            "samples": W.moving_samples(2, n, -1.0, 1.0, 0.5)})
    close = W.close_discs_2d(n)
    G = kfbi.Problem.from_workload(ell)
    for w in (smp, close, ell):
        G.update_levelset(*_ls_of(w))
        F = kfbi.Problem.from_workload(w)
        _same(_snapshot(G, w), _snapshot(F, w))
        F.close()
    G.close()


def test_update_general_kind():
    """The general interface system updates its second side operator too."""
    from paper_2309_05965_gb300 import build, kfbi
    build.build()
    w0 = W.hetero_interface_2d(128)
    G = kfbi.Problem.from_workload(w0, precision=kfbi.MIXED)
    w1 = W.hetero_interface_2d(128)
    w1.ls_kind, w1.ls_params = W.LS_ELLIPSE, [0.02, 0.01, 0.6, 0.42, 0.2]
    G.update_levelset(*_ls_of(w1))
    F = kfbi.Problem.from_workload(w1, precision=kfbi.MIXED)
    _same(_snapshot(G, w1), _snapshot(F, w1))
    F.close()
    G.close()


def test_invalid_update_is_refused_and_recoverable():
    from paper_2309_05965_gb300 import build, kfbi
    build.build()
    w = W.moving_interface_2d(128, 0.0)
    G = kfbi.Problem.from_workload(w)
    with pytest.raises(kfbi.KfbiError) as e:
        G.update_levelset(W.LS_ELLIPSOID, [0, 0, 0, 0.5, 0.5, 0.5])   # a 3D kind in 2D
    assert e.value.status == 1
    for v in (np.nan, np.inf):   # a non-finite sample
        smp = W.moving_samples(2, 128, -1.0, 1.0, 0.2).copy()
        smp[40, 77] = v
        with pytest.raises(kfbi.KfbiError) as e:
            G.update_levelset(W.LS_GRID, [], smp)
        assert e.value.status == 1 and "finite" in str(e.value)
    w2 = W.moving_interface_2d(128, 0.3)
    G.update_levelset(*_ls_of(w2))
    F = kfbi.Problem.from_workload(w2)
    _same(_snapshot(G, w2), _snapshot(F, w2))
    F.close()
    G.close()


def test_update_grows_and_merges_the_geometry_arena_1024():
    """At 1024^2 a set-up takes ~30 MB (the closest-point cell lists alone
    12.6 MB), more than the arena's first 16 MB chunk: the create grows the
    arena to several chunks, the first update merges them into one, and the
    updates between a small ellipse and the flower reuse or regrow it.  Every
    state equals the freshly created problem, bit for bit (small -> flower ->
    small -> flower)."""
    from paper_2309_05965_gb300 import build, kfbi
    build.build()
    big = W.flower_interface_2d(1024)
    small = W.flower_interface_2d(1024)
    small.ls_kind, small.ls_params = W.LS_ELLIPSE, [0.05, -0.03, 0.2, 0.15, 0.3]
    G = kfbi.Problem.from_workload(small, precision=kfbi.MIXED)
    for w in (big, small, big):
        G.update_levelset(*_ls_of(w))
        F = kfbi.Problem.from_workload(w, precision=kfbi.MIXED)
        a, b = _snapshot(G, w), _snapshot(F, w)
        _same(a, b)
        F.close()
        assert a["err"] < 1e-7, a["err"]
    G.close()
