"""Close and touching interfaces on the GPU (the remark on arbitrarily close
interfaces in Sec. 5.2), end to end through the C ABI against the exact
solutions, at sizes beyond the oracle's reach.  Element-by-element parity
with the oracle for these geometries is in test_gpu_parity.py (two discs
0.004 apart, Table 2's circles and star at 256^2) and
test_gpu_interface_system.py (Sec. 7.2.5's spheres 0.0142 apart at 64^3).

* Sec. 7.1.2 (Table 2), eight circles and a star: N_b within 1 % of the
  table's, errors within 15x (256^2) and 4x (512^2, 1024^2) of the table's
  (the excess at 256^2 is the star's arm tip, as with the star alone);
* Sec. 7.2.4 (Table 6), torus and ellipsoid touching along a circle, with a
  different solution in each: 4th-order convergence from 128^3 to 256^3 in
  each region, errors within 6x of the table's, and at 128^3 within 2x of
  the torus and the ellipsoid solved alone (each with its own solution):
  the largest errors sit on the torus away from the touching circle, at the
  level the torus alone has here (N_b is 1.43x the table's: the 3D surface
  decomposition here keeps |n_r| > 0.4, more overlap than the paper's);
* mixed precision matches FP64 to 1.1x in error.
"""
import json
import pathlib

import numpy as np
import pytest

import workloads as W
from tests.gpu_util import empty, gpu_data, host

pytestmark = pytest.mark.gpu

GOLDEN = pathlib.Path(__file__).parent / "golden"


def solve(w, precision, rtol=1e-10, relax=0.0):
    """(N_b, GMRES iterations, error grid, labels) of one GPU solve."""
    from paper_2309_05965_gb300 import build, kfbi
    build.build()
    G = kfbi.Problem.from_workload(w, precision=precision, relax=relax)
    xyz, nrm = empty((G.nb, w.dim)), empty((G.nb, w.dim))
    kfbi.kfbi_dof_points(G.handle, xyz, nrm)
    ifc = empty(G.nb, "i32")
    kfbi.kfbi_dof_iface(G.handle, ifc)
    g1, g2 = W.boundary_data(w, host(xyz), host(nrm), host(ifc))
    data = W.grid_data(w)
    d, keep = gpu_data(w, None, data, g1, g2)
    nx = 2 * G.nb if w.kind == W.KIND_INTERFACE_GENERAL else G.nb
    dens = empty(nx)
    info = kfbi.kfbi_gmres_solve(G.handle, d, kfbi.GmresOpts(rtol=rtol, restart=100, max_iter=300),
                                 dens)
    u = empty(G.grid_shape)
    kfbi.kfbi_evaluate(G.handle, d, dens, u)
    lab = empty(G.grid_shape, "u8")
    kfbi.kfbi_inside_mask(G.handle, lab)
    lab = host(lab)
    e = np.abs(host(u) - W.exact_grid(w, lab))
    inner = np.zeros(e.shape, dtype=bool)
    inner[tuple(slice(1, w.n) for _ in range(w.dim))] = True
    e[~inner] = 0.0
    nb = G.nb
    G.close()
    return nb, info.iters, e, lab


@pytest.mark.parametrize("n,factor", [(256, 15.0), (512, 4.0), (1024, 4.0)])
def test_touching_interfaces_table2(n, factor):
    row = json.loads((GOLDEN / "paper_table2.json").read_text())["rows"][str(n)]
    w = W.touching_interfaces_2d(n)
    errs = {}
    for prec in (0, 1):
        nb, it, e, lab = solve(w, prec)
        assert abs(nb - row["n_b"]) <= 0.01 * row["n_b"], (nb, row)
        assert it <= 1.5 * row["iters"], (it, row)
        errs[prec] = (e[lab > 0].max(), e[lab == 0].max())
        assert errs[prec][0] < factor * row["einf_in"], (n, prec, errs[prec], row)
        assert errs[prec][1] < factor * row["einf_out"], (n, prec, errs[prec], row)
    for side in (0, 1):
        assert errs[1][side] <= 1.1 * errs[0][side] + 1e-13, errs


def test_torus_ellipsoid_table6_512():
    """Table 6's finest grid, 512^3 (~0.8 M DOFs), mixed precision: errors in
    every region within 7x of the table's (measured 1.23e-8 / 1.23e-8 /
    1.26e-8 against 2.1e-9: the table converges faster than 4th order from
    256^3, 20.6x, this method at 15.5x) and 4th order from 256^3 (> 12x)."""
    rows = json.loads((GOLDEN / "paper_table6.json").read_text())["rows"]
    errs = {}
    for n in (256, 512):
        _, it, e, lab = solve(W.torus_ellipsoid_3d(n), 1, relax=0.03)
        errs[n] = (e[lab == 1].max(), e[lab == 2].max(), e[lab == 0].max())
        assert it <= 1.5 * rows[str(n)]["iters"], (n, it)
    want = (rows["512"]["einf_torus"], rows["512"]["einf_ellipsoid"], rows["512"]["einf_out"])
    for k in range(3):
        assert errs[512][k] < 7.0 * want[k], (errs, want)
        assert errs[256][k] / errs[512][k] > 12.0, errs


def _alone(kind, params, sol, n):
    w = W.Workload("alone", 3, n, -1.5, 1.5, W.LS_UNION, W.union_params([(kind, params)]),
                   W.KIND_INTERFACE_MU, sigma_in=1.0, sigma_out=3.0, exact="multi",
                   extra={"sol_in": [sol], "sol_out": "cos3"})
    _, _, e, lab = solve(w, 0)
    return e.max()


def test_torus_ellipsoid_table6():
    rows = json.loads((GOLDEN / "paper_table6.json").read_text())["rows"]
    per_n = {}
    for n in (128, 256):
        row = rows[str(n)]
        w = W.torus_ellipsoid_3d(n)
        errs = {}
        for prec in (0, 1):
            nb, it, e, lab = solve(w, prec, relax=0.03 if prec else 0.0)
            assert 1.0 <= nb / row["n_b"] <= 1.6, (nb, row)
            assert it <= 1.5 * row["iters"], (it, row)
            errs[prec] = (e[lab == 1].max(), e[lab == 2].max(), e[lab == 0].max())
            want = (row["einf_torus"], row["einf_ellipsoid"], row["einf_out"])
            for got, ref in zip(errs[prec], want):
                assert got < 6.0 * ref, (n, prec, errs[prec], want)
        for k in range(3):
            assert errs[1][k] <= 1.1 * errs[0][k] + 1e-13, errs
        per_n[n] = errs[0]
    for k in range(3):
        assert per_n[128][k] / per_n[256][k] > 12.0, per_n
    alone = max(_alone(W.LS_TORUS, [1.0, 0.4], "torus_in", 128),
                _alone(W.LS_ELLIPSOID, [0.0, 0.0, 0.0, 0.6, 0.6, 1.0], "exp_cos3", 128))
    assert max(per_n[128]) < 2.0 * alone, (per_n[128], alone)
